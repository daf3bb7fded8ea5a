// sort.cu -- the fallback table of Sec. 3.5: the keys left after the last
// level, sorted ascending (looked up by binary search), with a check for equal
// neighbours (duplicate keys always collide, so they all end up here).
//
// Bitonic sorting network: one CTA in shared memory for up to 4096 keys (the
// usual case: a handful of keys at gamma = 1, none at gamma >= 2), else the
// same network in global memory over a power-of-two copy padded with
// UINT64_MAX (padding sorts last, so the first n entries are the n keys).
#include <cuda_runtime.h>

#include "common.cuh"

namespace bbh {

static constexpr int kSmemSortN = 4096;
static constexpr int kSortThreads = 1024;

__device__ __forceinline__ void cmp_swap(u64 &a, u64 &b, bool up) {
  if ((a > b) == up) {
    u64 t = a;
    a = b;
    b = t;
  }
}

__global__ void __launch_bounds__(kSortThreads)
k_sort_small(u64 *__restrict__ keys, unsigned n, unsigned int *__restrict__ dup) {
  __shared__ u64 s[kSmemSortN];
  unsigned P = 1;
  while (P < n) P <<= 1;
  for (unsigned i = threadIdx.x; i < P; i += kSortThreads) s[i] = i < n ? keys[i] : ~0ull;
  __syncthreads();
  for (unsigned k = 2; k <= P; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      for (unsigned i = threadIdx.x; i < P; i += kSortThreads) {
        unsigned l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          u64 a = s[i], b = s[l];
          cmp_swap(a, b, up);
          s[i] = a;
          s[l] = b;
        }
      }
      __syncthreads();
    }
  }
  for (unsigned i = threadIdx.x; i < n; i += kSortThreads) {
    keys[i] = s[i];
    if (i + 1 < n && s[i] == s[i + 1]) atomicOr(dup, 1u);
  }
}

__global__ void k_pad_copy(const u64 *__restrict__ src, u64 n, u64 *__restrict__ dst, u64 P) {
  u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride)
    dst[i] = i < n ? src[i] : ~0ull;
}

__global__ void k_bitonic_step(u64 *__restrict__ a, u64 P, u64 j, u64 k) {
  u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
    u64 l = i ^ j;
    if (l > i) {
      bool up = (i & k) == 0;
      u64 x = a[i], y = a[l];
      if ((x > y) == up) {
        a[i] = y;
        a[l] = x;
      }
    }
  }
}

__global__ void k_copy_back_check(const u64 *__restrict__ src, u64 n, u64 *__restrict__ dst,
                                  unsigned int *__restrict__ dup) {
  u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    u64 v = src[i];
    dst[i] = v;
    if (i + 1 < n && v == src[i + 1]) atomicOr(dup, 1u);
  }
}

int sort_fallback(u64 *keys, u64 n, unsigned int *d_dup_flag, cudaStream_t s) {
  if (n <= 1) return MPHF_OK;
  if (n <= (u64)kSmemSortN) {
    LaunchScope ls("fallback_sort", s);
    k_sort_small<<<1, kSortThreads, 0, s>>>(keys, (unsigned)n, d_dup_flag);
    MPHF_CUDA(cudaGetLastError());
    return MPHF_OK;
  }
  u64 P = 1;
  while (P < n) P <<= 1;
  DevBuf tmp;
  int rc = dev_alloc(tmp, P * sizeof(u64), s);
  if (rc != MPHF_OK) return rc;
  u64 *a = (u64 *)tmp.p;
  unsigned grid = grid_for(P, 256 * 4, (unsigned)sm_count() * 8);
  {
    LaunchScope ls("fallback_sort", s);
    k_pad_copy<<<grid, 256, 0, s>>>(keys, n, a, P);
  }
  for (u64 k = 2; k <= P; k <<= 1) {
    for (u64 j = k >> 1; j > 0; j >>= 1) {
      LaunchScope ls("fallback_sort", s);
      k_bitonic_step<<<grid, 256, 0, s>>>(a, P, j, k);
    }
  }
  {
    LaunchScope ls("fallback_sort", s);
    k_copy_back_check<<<grid, 256, 0, s>>>(a, n, keys, d_dup_flag);
  }
  cudaError_t e = cudaGetLastError();
  dev_free(tmp, s);
  if (e != cudaSuccess) return cuda_fail(e, "fallback sort");
  return MPHF_OK;
}

}  // namespace bbh
