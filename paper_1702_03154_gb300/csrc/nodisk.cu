// nodisk.cu -- construction without storing the level key sets (Sec. 3.4,
// second disk strategy; Sec. 4.5's trillion-key run).
//
// The default build copies F_d and compacts it into F_{d+1} at every level.
// Here level d instead reads every input key again and asks the levels
// already built whether the key was placed there (the query of Algorithm 3
// up to level d-1); the keys that were not are exactly F_d, and they go
// through ArrayFill (Algorithm 2) for level d.  No key is stored, so the
// device holds only the bit arrays: with keys generated on the fly (the
// SplitMix64 stream key(j) of mphf_keygen, as Sec. 4.5 streams its keys)
// N is bounded by the size of the bit arrays instead of 8 bytes per key.
// Once |F_d| falls to keep_fraction * N (Sec. 4.5 uses 2%), F_d is collected
// once and the remaining levels run on the stored list.
//
// ArrayFill uses L2/HBM atomics on an interleaved hit/collision array (bits
// 0-31 of a word: first hits of 32 positions, bits 32-63: collisions).  The
// result is the same set function as every other path: identical A, ranks
// and fallback.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "sector.cuh"

namespace bbh {

static constexpr int kNdThreads = 256;
static constexpr int kNdKeys = 4;  // keys per thread in flight

struct NdLevel {
  const u64 *A;  // A_d (m / 64 words)
  u64 m, s;
};

enum { SRC_GEN = 0, SRC_ARRAY = 1 };

// The keys of a pass: generated (key(j) = mix(key_seed + (key_start + j + 1) G))
// or read from memory.  Levels [check_lo, d) are asked whether each key was
// placed there.
struct NdSrc {
  int kind;
  const u64 *keys;
  u64 n, key_seed, key_start;
  int check_lo;
};

__device__ __forceinline__ u64 nd_key(const NdSrc &src, u64 i) {
  if (src.kind == SRC_GEN) return mix64(src.key_seed + (src.key_start + i + 1) * 0x9E3779B97F4A7C15ull);
  return __ldcs(src.keys + i);
}

__device__ __forceinline__ bool nd_bit(const NdLevel &l, u64 x) {
  const u64 p = level_pos(x, l.s, l.m);
  return (__ldg(l.A + (p >> 6)) >> (p & 63)) & 1ull;
}

__device__ __forceinline__ void nd_fill(u64 *__restrict__ AC, u64 p) {
  const u64 w = p >> 5;
  const u64 hit = 1ull << (p & 31);
  const u64 old = atomicOr(AC + w, hit);
  if ((old & hit) && !(old & (hit << 32))) atomicOr(AC + w, hit << 32);
}

// ArrayFill of level d over the keys of src that no level in [check_lo, d) placed.
__global__ void __launch_bounds__(kNdThreads)
k_nd_fill(NdSrc src, const NdLevel *__restrict__ lvs, int d, u64 *__restrict__ AC) {
  __shared__ NdLevel sl[MPHF_MAX_LEVELS];
  for (int j = threadIdx.x; j <= d; j += kNdThreads) sl[j] = lvs[j];
  __syncthreads();
  const NdLevel cur = sl[d];
  const u64 per = (u64)kNdThreads * kNdKeys;
  for (u64 base = (u64)blockIdx.x * per + threadIdx.x; base < src.n; base += (u64)gridDim.x * per) {
    u64 x[kNdKeys];
    bool live[kNdKeys];
#pragma unroll
    for (int u = 0; u < kNdKeys; u++) {
      const u64 i = base + (u64)u * kNdThreads;
      live[u] = i < src.n;
      x[u] = live[u] ? nd_key(src, i) : 0;
    }
    for (int j = src.check_lo; j < d; j++) {
#pragma unroll
      for (int u = 0; u < kNdKeys; u++)
        if (live[u] && nd_bit(sl[j], x[u])) live[u] = false;
    }
#pragma unroll
    for (int u = 0; u < kNdKeys; u++)
      if (live[u]) nd_fill(AC, level_pos(x[u], cur.s, cur.m));
  }
}

// A_d = hit & ~collision, and the number of its ones.
__global__ void __launch_bounds__(kNdThreads)
k_nd_extract(const u64 *__restrict__ AC, u64 nwords, u64 *__restrict__ A, u64 *__restrict__ weight) {
  __shared__ u64 red[kNdThreads / 32];
  u64 c = 0;
  for (u64 w = (u64)blockIdx.x * kNdThreads + threadIdx.x; w < nwords;
       w += (u64)gridDim.x * kNdThreads) {
    const u64 a0 = AC[2 * w], a1 = AC[2 * w + 1];
    const u64 lo = (a0 & 0xffffffffull) & ~(a0 >> 32);
    const u64 hi = (a1 & 0xffffffffull) & ~(a1 >> 32);
    const u64 a = lo | (hi << 32);
    A[w] = a;
    c += __popcll(a);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int i = 0; i < kNdThreads / 32; i++) t += red[i];
    if (t) atomicAdd(weight, t);
  }
}

// Keys of src that no level in [check_lo, hi] placed, appended to F (at most
// cap; more raises *overflow).
__global__ void __launch_bounds__(kNdThreads)
k_nd_collect(NdSrc src, const NdLevel *__restrict__ lvs, int hi, u64 *__restrict__ F,
             u64 *__restrict__ cnt, u64 cap, unsigned *__restrict__ overflow) {
  __shared__ NdLevel sl[MPHF_MAX_LEVELS];
  for (int j = threadIdx.x; j <= hi; j += kNdThreads) sl[j] = lvs[j];
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  const u64 stride = (u64)gridDim.x * kNdThreads;
  const u64 n_round = (src.n + 31) & ~31ull;  // whole warps stay in the loop together
  for (u64 i = (u64)blockIdx.x * kNdThreads + threadIdx.x; i < n_round; i += stride) {
    bool live = i < src.n;
    const u64 x = live ? nd_key(src, i) : 0;
    for (int j = src.check_lo; j <= hi && live; j++)
      if (nd_bit(sl[j], x)) live = false;
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    if (!bal) continue;
    u64 base = 0;
    if (lane == 0) base = atomicAdd(cnt, (u64)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (live) {
      const u64 k = base + __popc(bal & ((1u << lane) - 1u));
      if (k < cap) F[k] = x;
      else atomicOr(overflow, 1u);
    }
  }
}

static int nd_build(NdSrc src0, u64 N, double gamma, uint32_t L, u64 seed, double keep,
                    cudaStream_t st, mphf_t **out) {
  mphf_t *h = handle_new();
  if (!h) return MPHF_ENOMEM;
  cudaGetDevice(&h->device);
  h->N = N;
  h->gamma = gamma;
  h->L = L;
  h->seed = seed;
  h->path = 5;
  for (uint32_t d = 0; d < L; d++) h->s[d] = level_seed(seed, d);
  if (N == 0) {
    *out = h;
    return MPHF_OK;
  }
  int rc = MPHF_OK;
  std::vector<DevBuf> Ad;        // A_d of every level built
  std::vector<NdLevel> hl(MPHF_MAX_LEVELS);
  DevBuf dl, AC, counters, F, Fnext, Aall;
  u64 *d_weight = nullptr, *d_cnt = nullptr, *d_total = nullptr;
  unsigned *d_over = nullptr, *d_dup = nullptr;
  NdSrc src = src0;
  u64 n_d = N, off = 0;
  uint32_t d = 0;
  u64 n_fb = 0;
  const unsigned grid = (unsigned)sm_count() * 8;

#define NTRY(x)                    \
  do {                             \
    rc = (x);                      \
    if (rc != MPHF_OK) goto fail;  \
  } while (0)
#define NCUDA(x)                                        \
  do {                                                  \
    cudaError_t e_ = (x);                               \
    if (e_ != cudaSuccess) {                            \
      rc = cuda_fail(e_, #x);                           \
      goto fail;                                        \
    }                                                   \
  } while (0)

  NTRY(dev_alloc(dl, sizeof(NdLevel) * MPHF_MAX_LEVELS, st));
  // counters: weight, collected count, rank total, overflow + duplicate flags
  NTRY(dev_alloc(counters, 64, st));
  d_weight = (u64 *)counters.p;
  d_cnt = d_weight + 1;
  d_total = d_weight + 2;
  d_over = (unsigned *)(d_weight + 3);
  d_dup = d_over + 1;
  for (;;) {
    const u64 m = level_bits(n_d, gamma);
    DevBuf a;
    NTRY(dev_alloc(a, m / 8, st));
    Ad.push_back(a);
    hl[d] = NdLevel{(const u64 *)a.p, m, h->s[d]};
    NCUDA(cudaMemcpyAsync((NdLevel *)dl.p + d, &hl[d], sizeof(NdLevel), cudaMemcpyHostToDevice, st));
    NTRY(dev_alloc(AC, m / 4, st));  // 2 bits per position
    NCUDA(cudaMemsetAsync(AC.p, 0, m / 4, st));
    NCUDA(cudaMemsetAsync(counters.p, 0, 64, st));
    {
      LaunchScope ls("nd_fill", st);
      k_nd_fill<<<grid, kNdThreads, 0, st>>>(src, (const NdLevel *)dl.p, (int)d, (u64 *)AC.p);
    }
    {
      LaunchScope ls("nd_extract", st);
      k_nd_extract<<<grid, kNdThreads, 0, st>>>((const u64 *)AC.p, m / 64, (u64 *)a.p, d_weight);
    }
    NCUDA(cudaGetLastError());
    dev_free(AC, st);
    u64 wgt = 0;
    NCUDA(cudaMemcpyAsync(&wgt, d_weight, 8, cudaMemcpyDeviceToHost, st));
    NCUDA(cudaStreamSynchronize(st));
    if (wgt > n_d) {
      rc = MPHF_EINTERNAL;
      goto fail;
    }
    h->n[d] = n_d;
    h->m[d] = m;
    h->off[d] = off;
    off += m;
    const u64 n_next = n_d - wgt;
    if (n_next == 0) {
      h->L_used = d + 1;
      break;
    }
    const bool last = d + 1 == L;
    const bool stored = F.p != nullptr && src.keys == (const u64 *)F.p;  // src is F_d itself
    // Collect F_{d+1} once it is small enough (always for the fallback, and
    // at every level once the keys are a stored list).
    if (last || stored || (double)n_next <= keep * (double)N) {
      NTRY(dev_alloc(Fnext, n_next * 8, st));
      {
        LaunchScope ls("nd_collect", st);
        k_nd_collect<<<grid, kNdThreads, 0, st>>>(src, (const NdLevel *)dl.p, (int)d,
                                                  (u64 *)Fnext.p, d_cnt, n_next, d_over);
      }
      NCUDA(cudaGetLastError());
      u64 got = 0;
      unsigned over = 0;
      NCUDA(cudaMemcpyAsync(&got, d_cnt, 8, cudaMemcpyDeviceToHost, st));
      NCUDA(cudaMemcpyAsync(&over, d_over, 4, cudaMemcpyDeviceToHost, st));
      NCUDA(cudaStreamSynchronize(st));
      if (over || got != n_next) {
        rc = MPHF_EINTERNAL;
        goto fail;
      }
      dev_free(F, st);
      F = Fnext;
      Fnext = DevBuf();
      src.kind = SRC_ARRAY;
      src.keys = (const u64 *)F.p;
      src.n = n_next;
      src.check_lo = (int)d + 1;
    }
    if (last) {
      h->L_used = L;
      n_fb = n_next;
      break;
    }
    n_d = n_next;
    d++;
  }
  h->n[h->L_used] = n_fb;
  h->n_fb = n_fb;
  h->M = off;
  h->n_rank = (h->M + MPHF_RANK_BLOCK - 1) / MPHF_RANK_BLOCK;
  // A = A_0 || A_1 || ..., then the sectors with their ranks
  NTRY(dev_alloc(Aall, h->M / 8, st));
  for (uint32_t j = 0; j < h->L_used; j++)
    NCUDA(cudaMemcpyAsync((u64 *)Aall.p + h->off[j] / 64, Ad[j].p, h->m[j] / 8,
                          cudaMemcpyDeviceToDevice, st));
  for (auto &a : Ad) dev_free(a, st);
  Ad.clear();
  NTRY(make_sectors(h, ASrc{(const u64 *)Aall.p, h->M / 64, nullptr, h->M / 64}, d_total, st));
  dev_free(Aall, st);
  if (n_fb) {  // Sec. 3.5: the leftover keys, sorted; equal neighbours are duplicates
    NTRY(sort_fallback((u64 *)F.p, n_fb, d_dup, st));
    NTRY(dev_alloc(h->fb, n_fb * 8, st));
    NCUDA(cudaMemcpyAsync(h->fb.p, F.p, n_fb * 8, cudaMemcpyDeviceToDevice, st));
  }
  {
    u64 tot = 0;
    unsigned dup = 0;
    NCUDA(cudaMemcpyAsync(&tot, d_total, 8, cudaMemcpyDeviceToHost, st));
    NCUDA(cudaMemcpyAsync(&dup, d_dup, 4, cudaMemcpyDeviceToHost, st));
    NCUDA(cudaStreamSynchronize(st));
    if (dup) {
      rc = MPHF_EDUPLICATE;
      goto fail;
    }
    if (tot != N - n_fb) {
      rc = MPHF_EINTERNAL;
      goto fail;
    }
  }
  dev_free(F, st);
  dev_free(dl, st);
  dev_free(counters, st);
  *out = h;
  return MPHF_OK;

fail:
  cudaGetLastError();
  for (auto &a : Ad) dev_free(a, st);
  dev_free(AC, st);
  dev_free(F, st);
  dev_free(Fnext, st);
  dev_free(Aall, st);
  dev_free(dl, st);
  dev_free(counters, st);
  dev_free(h->S, st);
  dev_free(h->SB, st);
  dev_free(h->fb, st);
  cudaStreamSynchronize(st);
  handle_delete(h);
  return rc;
#undef NTRY
#undef NCUDA
}

static bool nd_args_ok(double gamma, uint32_t levels, double keep) {
  return gamma >= 1.0 && !isinf(gamma) && levels >= 1 && levels <= MPHF_MAX_LEVELS &&
         keep >= 0.0 && keep <= 1.0;
}

}  // namespace bbh

using namespace bbh;

extern "C" int mphf_build_nodisk(const uint64_t *d_keys, uint64_t n, double gamma, uint32_t levels,
                                 uint64_t seed, double keep_fraction, void *stream, mphf_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (!nd_args_ok(gamma, levels, keep_fraction) || (n > 0 && !d_keys) || ((uintptr_t)d_keys & 7))
    return MPHF_EINVAL;
  NdSrc src{SRC_ARRAY, (const u64 *)d_keys, n, 0, 0, 0};
  return nd_build(src, n, gamma, levels, seed, keep_fraction, (cudaStream_t)stream, out);
}

extern "C" int mphf_build_generated(uint64_t n, uint64_t key_seed, uint64_t key_start,
                                    double gamma, uint32_t levels, uint64_t seed,
                                    double keep_fraction, void *stream, mphf_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (!nd_args_ok(gamma, levels, keep_fraction)) return MPHF_EINVAL;
  NdSrc src{SRC_GEN, nullptr, n, key_seed, key_start, 0};
  return nd_build(src, n, gamma, levels, seed, keep_fraction, (cudaStream_t)stream, out);
}
