// ceiling.cu -- measurement kernels for the throughput ceilings that the
// build and lookup kernels are held against: random loads (one 32-byte sector
// or one 8-byte word each) and random 64-bit atomicOr over an array that the
// caller places in L2 (tens of MB) or in HBM (many GB).  The method does
// exactly these accesses: a lookup probe is one random sector load per level
// (Algorithm 3 with the ranks of Sec. 3.1), and ArrayFill's hit / collision
// marks are random atomic ORs (Sec. 3.2: the fill is bound by its random
// accesses).  The caller times a launch with events on its stream.
#include <cuda_runtime.h>

#include "common.cuh"

namespace bbh {

static constexpr int kCeilThreads = 256;
static constexpr int kCeilUnroll = 8;  // independent accesses in flight per thread

// Per-thread slot streams: a 64-bit linear congruential step (Knuth's MMIX
// multiplier and increment); the high 32 bits pick a slot by a 32x32-bit
// multiply-high, so an index costs three or four instructions and the
// ceiling is set by the memory system, not by the index arithmetic.
__device__ __forceinline__ u64 lcg_step(u64 x) {
  return x * 6364136223846793005ull + 1442695040888963407ull;
}

template <int WIDTH>
__global__ void __launch_bounds__(kCeilThreads)
k_ceiling_loads(const unsigned char *__restrict__ buf, unsigned slots, u64 rounds, u64 seed,
                u64 *__restrict__ sink) {
  const u64 tid = (u64)blockIdx.x * kCeilThreads + threadIdx.x;
  u64 x[kCeilUnroll];
#pragma unroll
  for (int u = 0; u < kCeilUnroll; u++) x[u] = mix64(seed + tid * kCeilUnroll + u);
  unsigned acc = 0;
  for (u64 r = 0; r < rounds; r++) {
#pragma unroll
    for (int u = 0; u < kCeilUnroll; u++) {
      x[u] = lcg_step(x[u]);
      const u64 slot = __umulhi((unsigned)(x[u] >> 32), slots);
      if (WIDTH == 32) {
        unsigned v0, v1, v2, v3, v4, v5, v6, v7;
        asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3), "=r"(v4), "=r"(v5), "=r"(v6),
                       "=r"(v7)
                     : "l"(buf + slot * 32));
        acc ^= v0 ^ v1 ^ v2 ^ v3 ^ v4 ^ v5 ^ v6 ^ v7;
      } else {
        const u64 v = __ldg((const u64 *)(buf + slot * 8));
        acc ^= (unsigned)v ^ (unsigned)(v >> 32);
      }
    }
  }
  // a data-dependent store keeps every load live
  if (acc == 0x9E3779B9u) sink[tid & 1023] = acc;
}

template <bool RET>
__global__ void __launch_bounds__(kCeilThreads)
k_ceiling_atomics(u64 *__restrict__ buf, unsigned words, u64 rounds, u64 seed,
                  u64 *__restrict__ sink) {
  const u64 tid = (u64)blockIdx.x * kCeilThreads + threadIdx.x;
  u64 x[kCeilUnroll];
#pragma unroll
  for (int u = 0; u < kCeilUnroll; u++) x[u] = mix64(seed + tid * kCeilUnroll + u);
  u64 acc = 0;
  for (u64 r = 0; r < rounds; r++) {
#pragma unroll
    for (int u = 0; u < kCeilUnroll; u++) {
      x[u] = lcg_step(x[u]);
      const u64 w = __umulhi((unsigned)(x[u] >> 32), words);
      const u64 bit = 1ull << (x[u] & 63);
      if (RET)
        acc ^= atomicOr(buf + w, bit);
      else
        atomicOr(buf + w, bit);  // result unused: a reduction
    }
  }
  if (RET && acc == 0x9E3779B97F4A7C15ull) sink[tid & 1023] = acc;
}

// Streaming copy, 16 bytes a thread per step, four steps in flight: the
// HBM bandwidth that a kernel streaming its keys can reach.
__global__ void __launch_bounds__(kCeilThreads)
k_ceiling_copy(const uint4 *__restrict__ src, uint4 *__restrict__ dst, u64 n16) {
  const u64 stride = (u64)gridDim.x * kCeilThreads;
  u64 i = (u64)blockIdx.x * kCeilThreads + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) v[u] = __ldcs(src + i + u * stride);
#pragma unroll
    for (int u = 0; u < 4; u++) __stcs(dst + i + u * stride, v[u]);
  }
  for (; i < n16; i += stride) __stcs(dst + i, __ldcs(src + i));
}

}  // namespace bbh

using namespace bbh;

extern "C" int mphf_ceiling_copy(const void *d_src, void *d_dst, uint64_t bytes, void *stream) {
  if (!d_src || !d_dst || ((uintptr_t)d_src & 15) || ((uintptr_t)d_dst & 15) || (bytes & 15))
    return MPHF_EINVAL;
  const u64 n16 = bytes / 16;
  if (n16 == 0) return MPHF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  {
    LaunchScope ls("ceiling_copy", s);
    k_ceiling_copy<<<(unsigned)sm_count() * 8, kCeilThreads, 0, s>>>((const uint4 *)d_src,
                                                                      (uint4 *)d_dst, n16);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

// Grid for a ceiling launch: `ops` accesses spread over whole rounds of
// kCeilUnroll per thread, 8 CTAs per SM (enough warps to cover latency).
static int ceiling_grid(uint64_t ops, unsigned *grid, u64 *rounds) {
  const u64 threads = (u64)sm_count() * 8 * kCeilThreads;
  u64 r = ops / (threads * kCeilUnroll);
  if (r < 1) r = 1;
  *grid = (unsigned)(threads / kCeilThreads);
  *rounds = r;
  return MPHF_OK;
}

extern "C" int mphf_ceiling_random_loads(const void *d_buf, uint64_t bytes, uint32_t width,
                                         uint64_t n_loads, uint64_t seed, uint64_t *d_sink,
                                         uint64_t *performed, void *stream) {
  if (!d_buf || !d_sink || (width != 8 && width != 32) || ((uintptr_t)d_buf & 31) ||
      ((uintptr_t)d_sink & 7))
    return MPHF_EINVAL;
  const u64 slots = bytes / width;
  if (slots == 0 || slots > 0xffffffffull) return MPHF_EINVAL;
  unsigned grid;
  u64 rounds;
  ceiling_grid(n_loads, &grid, &rounds);
  cudaStream_t s = (cudaStream_t)stream;
  {
    LaunchScope ls(width == 32 ? "ceiling_loads32" : "ceiling_loads8", s);
    if (width == 32)
      k_ceiling_loads<32><<<grid, kCeilThreads, 0, s>>>((const unsigned char *)d_buf,
                                                         (unsigned)slots, rounds, seed, (u64 *)d_sink);
    else
      k_ceiling_loads<8><<<grid, kCeilThreads, 0, s>>>((const unsigned char *)d_buf,
                                                        (unsigned)slots, rounds, seed, (u64 *)d_sink);
  }
  MPHF_CUDA(cudaGetLastError());
  if (performed) *performed = (u64)grid * kCeilThreads * kCeilUnroll * rounds;
  return MPHF_OK;
}

extern "C" int mphf_ceiling_random_atomics(uint64_t *d_buf, uint64_t words, int with_return,
                                           uint64_t n_ops, uint64_t seed, uint64_t *d_sink,
                                           uint64_t *performed, void *stream) {
  if (!d_buf || !d_sink || ((uintptr_t)d_buf & 7) || ((uintptr_t)d_sink & 7)) return MPHF_EINVAL;
  if (words == 0 || words > 0xffffffffull) return MPHF_EINVAL;
  unsigned grid;
  u64 rounds;
  ceiling_grid(n_ops, &grid, &rounds);
  cudaStream_t s = (cudaStream_t)stream;
  {
    LaunchScope ls(with_return ? "ceiling_atomics_ret" : "ceiling_atomics", s);
    if (with_return)
      k_ceiling_atomics<true><<<grid, kCeilThreads, 0, s>>>((u64 *)d_buf, (unsigned)words, rounds, seed,
                                                             (u64 *)d_sink);
    else
      k_ceiling_atomics<false><<<grid, kCeilThreads, 0, s>>>((u64 *)d_buf, (unsigned)words, rounds,
                                                              seed, (u64 *)d_sink);
  }
  MPHF_CUDA(cudaGetLastError());
  if (performed) *performed = (u64)grid * kCeilThreads * kCeilUnroll * rounds;
  return MPHF_OK;
}
