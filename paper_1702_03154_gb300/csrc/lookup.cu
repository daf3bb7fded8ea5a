// lookup.cu -- batched queries (Algorithm 3 with the minimal index of
// Sec. 2.2.3 and the rank checkpoints of Sec. 3.1).
//
// One thread answers two keys (one 16-byte load, one 16-byte store).  Both
// keys probe level 0 together, then the still-unanswered ones probe level 1,
// and so on, so a thread keeps two independent loads in flight.  The index of
// a key placed at global bit g is rank[g / 512] plus the ones of the words of
// its 512-bit block before g.
#include <cuda_runtime.h>

#include "common.cuh"

namespace bbh {

static constexpr int kLookupThreads = 256;

struct LevelTable {
  u64 s[MPHF_MAX_LEVELS];
  u64 m[MPHF_MAX_LEVELS];
  u64 off[MPHF_MAX_LEVELS];
};

struct LookupArgs {
  const u64 *A;
  const u64 *rank;
  const u64 *fb;
  u64 n_fb;
  u64 N;
  uint32_t L_used;
};

// Ones of A strictly before global bit g, given the word w = A[g / 64].
__device__ __forceinline__ u64 rank_before(const LookupArgs &a, u64 g, u64 w) {
  const u64 b = g >> 9;
  u64 r = __ldg(a.rank + b);
  const u64 wi = g >> 6;
  for (u64 j = b << 3; j < wi; j++) r += __popcll(__ldg(a.A + j));
  return r + __popcll(w & ((1ull << (g & 63)) - 1ull));
}

__device__ __forceinline__ u64 fallback_index(const LookupArgs &a, u64 x) {
  u64 lo = 0, hi = a.n_fb;
  while (lo < hi) {
    u64 mid = lo + ((hi - lo) >> 1);
    if (__ldg(a.fb + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  if (lo < a.n_fb && __ldg(a.fb + lo) == x) return a.N - a.n_fb + lo;
  return MPHF_NOT_FOUND;
}

template <int K>
__device__ __forceinline__ void query_keys(const LookupArgs &a, const LevelTable &t, const u64 (&x)[K],
                                           u64 (&res)[K]) {
  bool open[K];
#pragma unroll
  for (int k = 0; k < K; k++) {
    open[k] = true;
    res[k] = MPHF_NOT_FOUND;
  }
  for (uint32_t d = 0; d < a.L_used; d++) {
    bool any = false;
    u64 g[K], w[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (open[k]) {
        g[k] = t.off[d] + level_pos(x[k], t.s[d], t.m[d]);
        w[k] = __ldg(a.A + (g[k] >> 6));
      }
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (open[k]) {
        if ((w[k] >> (g[k] & 63)) & 1ull) {
          res[k] = rank_before(a, g[k], w[k]);
          open[k] = false;
        } else {
          any = true;
        }
      }
    }
    if (!any) break;
  }
  if (a.n_fb) {
#pragma unroll
    for (int k = 0; k < K; k++)
      if (open[k]) res[k] = fallback_index(a, x[k]);
  }
}

__global__ void __launch_bounds__(kLookupThreads)
k_lookup_vec(const uint4 *__restrict__ keys2, u64 npairs, uint4 *__restrict__ out2, LookupArgs a,
             LevelTable t) {
  const u64 stride = (u64)gridDim.x * kLookupThreads;
  for (u64 i = (u64)blockIdx.x * kLookupThreads + threadIdx.x; i < npairs; i += stride) {
    uint4 v = __ldcs(keys2 + i);
    u64 x[2] = {((u64)v.y << 32) | v.x, ((u64)v.w << 32) | v.z};
    u64 r[2];
    query_keys<2>(a, t, x, r);
    __stcs(out2 + i, make_uint4((unsigned)r[0], (unsigned)(r[0] >> 32), (unsigned)r[1],
                                (unsigned)(r[1] >> 32)));
  }
}

__global__ void __launch_bounds__(kLookupThreads)
k_lookup_scalar(const u64 *__restrict__ keys, u64 n, u64 *__restrict__ out, LookupArgs a,
                LevelTable t) {
  const u64 stride = (u64)gridDim.x * kLookupThreads;
  for (u64 i = (u64)blockIdx.x * kLookupThreads + threadIdx.x; i < n; i += stride) {
    u64 x[1] = {keys[i]};
    u64 r[1];
    query_keys<1>(a, t, x, r);
    out[i] = r[0];
  }
}

static void fill_tables(const mphf_t *h, LookupArgs &a, LevelTable &t) {
  a.A = (const u64 *)h->A.p;
  a.rank = (const u64 *)h->rank.p;
  a.fb = (const u64 *)h->fb.p;
  a.n_fb = h->n_fb;
  a.N = h->N;
  a.L_used = h->L_used;
  for (uint32_t d = 0; d < MPHF_MAX_LEVELS; d++) {
    t.s[d] = d < h->L_used ? h->s[d] : 0;
    t.m[d] = d < h->L_used ? h->m[d] : 0;
    t.off[d] = d < h->L_used ? h->off[d] : 0;
  }
}

int lookup_impl(const mphf_t *h, const u64 *keys, u64 n, u64 *out, cudaStream_t s) {
  LookupArgs a;
  LevelTable t;
  fill_tables(h, a, t);
  const unsigned maxb = (unsigned)sm_count() * 16;
  const bool aligned = (((uintptr_t)keys | (uintptr_t)out) & 15) == 0;
  if (aligned) {
    u64 npairs = n >> 1;
    if (npairs) {
      unsigned g = grid_for(npairs, kLookupThreads * 2, maxb);
      LaunchScope ls("lookup", s);
      k_lookup_vec<<<g, kLookupThreads, 0, s>>>(reinterpret_cast<const uint4 *>(keys), npairs,
                                                reinterpret_cast<uint4 *>(out), a, t);
    }
    if (n & 1) {
      LaunchScope ls("lookup", s);
      k_lookup_scalar<<<1, kLookupThreads, 0, s>>>(keys + (n - 1), 1, out + (n - 1), a, t);
    }
  } else {
    unsigned g = grid_for(n, kLookupThreads * 2, maxb);
    LaunchScope ls("lookup", s);
    k_lookup_scalar<<<g, kLookupThreads, 0, s>>>(keys, n, out, a, t);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

}  // namespace bbh

using namespace bbh;

extern "C" int mphf_lookup(const mphf_t *h, const uint64_t *d_keys, uint64_t n, uint64_t *d_out,
                           void *stream) {
  if (!h) return MPHF_EINVAL;
  if (n == 0) return MPHF_OK;
  if (!d_keys || !d_out || (((uintptr_t)d_keys | (uintptr_t)d_out) & 7)) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->L_used == 0 && h->n_fb == 0) {  // empty function: every key is a miss
    MPHF_CUDA(cudaMemsetAsync(d_out, 0xff, n * 8, s));
    return MPHF_OK;
  }
  return lookup_impl(h, (const u64 *)d_keys, n, (u64 *)d_out, s);
}

extern "C" int mphf_lookup_host(const mphf_t *h, const uint64_t *h_keys, uint64_t n,
                                uint64_t *h_out, void *stream) {
  if (!h) return MPHF_EINVAL;
  if (n == 0) return MPHF_OK;
  if (!h_keys || !h_out) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf kb, ob;
  int rc = dev_alloc(kb, n * 8, s);
  if (rc != MPHF_OK) return rc;
  rc = dev_alloc(ob, n * 8, s);
  if (rc != MPHF_OK) {
    dev_free(kb, s);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(kb.p, h_keys, n * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    rc = mphf_lookup(h, (const uint64_t *)kb.p, n, (uint64_t *)ob.p, stream);
    if (rc == MPHF_OK) e = cudaMemcpyAsync(h_out, ob.p, n * 8, cudaMemcpyDeviceToHost, s);
  }
  dev_free(kb, s);
  dev_free(ob, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mphf_lookup_host");
  return rc;
}
