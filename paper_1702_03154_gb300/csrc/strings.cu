// strings.cu -- byte-string keys (Sec. 4.4, Table 2).
//
// The method takes 64-bit keys; a byte string becomes one by this library's
// rule: h = mix(seed + (len + 1) G), then for every group of 8 bytes in order
// (the last one padded with zero bytes) h = mix(h ^ w) with w the group read
// as a little-endian integer; the key is h.  One thread per string.  A group
// is assembled from the one or two aligned 8-byte words that hold its bytes,
// and a word is read only if it holds at least one byte of the string, so no
// load leaves the pages the string lives on.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace bbh {

static constexpr int kStrThreads = 256;

// Bytes [a, a + r) (1 <= r <= 8) of memory as a little-endian integer.
__device__ __forceinline__ u64 load_group(uintptr_t a, unsigned r) {
  const uintptr_t a0 = a & ~(uintptr_t)7;
  const unsigned sh = (unsigned)(a & 7) * 8;
  u64 w = *reinterpret_cast<const u64 *>(a0) >> sh;
  if (sh && r > 8 - (sh >> 3)) w |= *reinterpret_cast<const u64 *>(a0 + 8) << (64 - sh);
  if (r < 8) w &= (1ull << (8 * r)) - 1ull;
  return w;
}

__global__ void __launch_bounds__(kStrThreads)
k_string_keys(const unsigned char *__restrict__ bytes, u64 total, const u64 *__restrict__ off,
              u64 n, u64 seed, u64 *__restrict__ out, unsigned *__restrict__ bad) {
  const u64 G = 0x9E3779B97F4A7C15ull;
  const u64 stride = (u64)gridDim.x * kStrThreads;
  for (u64 i = (u64)blockIdx.x * kStrThreads + threadIdx.x; i < n; i += stride) {
    const u64 o0 = off[i], o1 = off[i + 1];
    if (o0 > o1 || o1 > total) {  // a string outside the buffer: report, read nothing
      atomicOr(bad, 1u);
      out[i] = 0;
      continue;
    }
    const u64 len = o1 - o0;
    u64 h = mix64(seed + (len + 1) * G);
    const uintptr_t base = (uintptr_t)(bytes + o0);
    for (u64 k = 0; k < len; k += 8) {
      const unsigned r = len - k < 8 ? (unsigned)(len - k) : 8u;
      h = mix64(h ^ load_group(base + k, r));
    }
    out[i] = h;
  }
}

}  // namespace bbh

using namespace bbh;

extern "C" int mphf_string_keys(const uint8_t *d_bytes, uint64_t total_bytes,
                                const uint64_t *d_offsets, uint64_t n, uint64_t seed,
                                uint64_t *d_out, void *stream) {
  if (n == 0) return MPHF_OK;
  if (!d_offsets || !d_out || ((uintptr_t)d_offsets & 7) || ((uintptr_t)d_out & 7) ||
      (total_bytes && !d_bytes))
    return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf flag;
  int rc = dev_alloc(flag, sizeof(unsigned), s);
  if (rc != MPHF_OK) return rc;
  unsigned h_bad = 0;
  cudaError_t e = cudaMemsetAsync(flag.p, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    const unsigned grid = grid_for(n, kStrThreads, (unsigned)sm_count() * 8);
    {
      LaunchScope ls("string_keys", s);
      k_string_keys<<<grid, kStrThreads, 0, s>>>(d_bytes, total_bytes, (const u64 *)d_offsets, n,
                                                  seed, (u64 *)d_out, (unsigned *)flag.p);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  dev_free(flag, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "mphf_string_keys");
  return h_bad ? MPHF_EINVAL : MPHF_OK;
}
