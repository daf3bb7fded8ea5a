// lookup.cu -- batched queries (Algorithm 3 with the minimal index of
// Sec. 2.2.3 and the rank checkpoints of Sec. 3.1).
//
// A key needs e^{1/gamma} level probes on average but up to L; a warp that
// kept 32 keys in lock-step would idle most lanes while its slowest key walks
// down the levels.  Instead each warp copies a chunk of 32 * kPerLane keys
// into shared memory, and every lane works through its own kPerLane keys
// with kSlots independent query slots: each round every active slot probes
// its current level (one 8-byte load of A); a slot whose bit is set computes
// its rank and writes the result over its key in shared memory; a retired
// slot takes the lane's next key.  Lanes only meet again at the end of the
// chunk, which is then written out with coalesced stores.
//
// Rank of global bit g: rank[g / 512] plus the ones of the words of g's
// 512-bit block before g (loaded as 16-byte pairs, only those needed).
#include <cuda_runtime.h>

#include "common.cuh"

namespace bbh {

static constexpr int kLookupWarps = 8;
static constexpr int kLookupThreads = kLookupWarps * 32;
static constexpr int kSlots = 2;
static constexpr int kPerLane = 32;
static constexpr unsigned kChunk = 32 * kPerLane;  // keys per warp chunk

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

// Ones of A strictly before global bit g; w = A[g / 64] (already loaded).
__device__ __forceinline__ u64 rank_before(const u64 *__restrict__ A, const u64 *__restrict__ rank,
                                           u64 g, u64 w) {
  const u64 b = g >> 9;
  const unsigned k = (unsigned)(g >> 6) & 7u;  // word of g inside its block
  const uint4 *blk = reinterpret_cast<const uint4 *>(A + (b << 3));
  u64 r = __ldg(rank + b);
  uint4 v[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    v[j] = make_uint4(0, 0, 0, 0);
    if ((unsigned)(2 * j) < k) v[j] = __ldg(blk + j);
  }
  unsigned c = 0;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    unsigned lo = (unsigned)(2 * j) < k ? 0xffffffffu : 0u;
    unsigned hi = (unsigned)(2 * j + 1) < k ? 0xffffffffu : 0u;
    c += __popc(v[j].x & lo) + __popc(v[j].y & lo) + __popc(v[j].z & hi) + __popc(v[j].w & hi);
  }
  return r + c + __popcll(w & ((1ull << (g & 63)) - 1ull));
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

__global__ void __launch_bounds__(kLookupThreads)
k_lookup(const u64 *__restrict__ keys, u64 n, u64 *__restrict__ out, LookupArgs a, LevelTable t) {
  extern __shared__ __align__(16) u64 lbuf[];  // [kLookupWarps][kChunk]
  __shared__ u64 ts[MPHF_MAX_LEVELS], tm[MPHF_MAX_LEVELS], toff[MPHF_MAX_LEVELS];
  for (unsigned i = threadIdx.x; i < a.L_used; i += kLookupThreads) {
    ts[i] = t.s[i];
    tm[i] = t.m[i];
    toff[i] = t.off[i];
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  u64 *buf = lbuf + (u64)wib * kChunk;
  const u64 nchunks = (n + kChunk - 1) / kChunk;
  const u64 nwarps = ((u64)gridDim.x * kLookupThreads) >> 5;
  for (u64 chunk = ((u64)blockIdx.x * kLookupThreads + threadIdx.x) >> 5; chunk < nchunks;
       chunk += nwarps) {
    const u64 base = chunk * kChunk;
    const unsigned cnt = (unsigned)min((u64)kChunk, n - base);
    for (unsigned i = lane; i < cnt; i += 32) buf[i] = __ldcs(keys + base + i);
    __syncwarp();
    // this lane's keys: j = lane + 32 k, k < kPerLane, j < cnt
    unsigned nxt = lane;
    u64 x[kSlots];
    unsigned jj[kSlots], lvl[kSlots];
    bool act[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      act[s] = nxt < cnt;
      jj[s] = nxt;
      lvl[s] = 0;
      x[s] = act[s] ? buf[nxt] : 0;
      nxt += 32;
    }
    for (;;) {
      bool any = false;
#pragma unroll
      for (int s = 0; s < kSlots; s++) any |= act[s];
      if (!any) break;
      u64 g[kSlots], w[kSlots];
#pragma unroll
      for (int s = 0; s < kSlots; s++) {
        if (act[s]) {
          const unsigned d = lvl[s];
          g[s] = toff[d] + level_pos(x[s], ts[d], tm[d]);
          w[s] = __ldg(a.A + (g[s] >> 6));
        }
      }
#pragma unroll
      for (int s = 0; s < kSlots; s++) {
        if (act[s]) {
          bool done = false;
          u64 r = 0;
          if ((w[s] >> (g[s] & 63)) & 1ull) {
            r = rank_before(a.A, a.rank, g[s], w[s]);
            done = true;
          } else if (++lvl[s] >= a.L_used) {
            r = a.n_fb ? fallback_index(a, x[s]) : MPHF_NOT_FOUND;
            done = true;
          }
          if (done) {
            buf[jj[s]] = r;  // result replaces the key
            act[s] = nxt < cnt;
            jj[s] = nxt;
            lvl[s] = 0;
            if (act[s]) x[s] = buf[nxt];
            nxt += 32;
          }
        }
      }
    }
    __syncwarp();
    for (unsigned i = lane; i < cnt; i += 32) __stcs(out + base + i, buf[i]);
    __syncwarp();
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
  static bool attr = false;
  const size_t smem = (size_t)kLookupWarps * kChunk * 8;
  if (!attr) {
    MPHF_CUDA(cudaFuncSetAttribute(k_lookup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  LookupArgs a;
  LevelTable t;
  fill_tables(h, a, t);
  const u64 chunks = (n + kChunk - 1) / kChunk;
  u64 grid = (chunks + kLookupWarps - 1) / kLookupWarps;
  const u64 maxb = (u64)sm_count() * 3;
  if (grid > maxb) grid = maxb;
  if (grid < 1) grid = 1;
  LaunchScope ls("lookup", s);
  k_lookup<<<(unsigned)grid, kLookupThreads, smem, s>>>(keys, n, out, a, t);
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
