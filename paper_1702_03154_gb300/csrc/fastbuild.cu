// fastbuild.cu -- bucketed construction: ArrayFill in shared memory.
//
// The keys of a level are kept grouped by position range ("buckets" of P
// consecutive positions of A_d, P a power of two).  One CTA then runs the
// whole of Algorithm 2 for a bucket with its hit / collision bits in shared
// memory (no L2 atomics), writes the bucket's slice of A_d with plain stores
// and counts weight(A_d).  Once every bucket is filled, |F_{d+1}| =
// |F_d| - weight(A_d) and |A_{d+1}| are known, so compaction can place each
// surviving key straight into its level-(d+1) bucket: the survivors of a tile
// are counting-sorted by destination bucket in shared memory, one atomicAdd
// per (tile, bucket) reserves their slots, and they are written out as
// contiguous runs.  The caller's keys are first partitioned the same way for
// level 0.  Levels with at most T keys run in a single CTA (k_tail) that keeps
// keys and bit arrays in shared memory and loops over all remaining levels,
// sorting the fallback (Sec. 3.5) at the end.
//
// Every bound (bucket capacity, bucket count, flat buffer) is checked on the
// device; when one is exceeded the build is redone by the unbucketed path in
// build.cu, so results never depend on these choices.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "fastbuild.cuh"
#include "sector.cuh"

namespace bbh {


// Each thread owns kKPT consecutive keys of a tile, staged by asynchronous
// copies: a thread takes its keys of tile t into registers, then starts
// copying its keys of the next tile into the same slots while tile t is
// split.  Slot layout: pair q (keys 2q, 2q+1) of thread t at 16-byte unit
// q * kTT + t, so a warp's reads of one pair hit consecutive 16-byte units.
template <bool ALIGNED>
__global__ void __launch_bounds__(kTT, 2)
k_partition0(const u64 *__restrict__ keys, u64 n, FastMeta *__restrict__ meta, FastCfg cfg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const FLevel lv = meta->lv[0];
  const unsigned nb = (unsigned)lv.B;
  SplitSmem sm = carve_split(smem, (unsigned)kBmax);
  split_clear(sm, nb);
  __syncthreads();
  u64 *inbuf = reinterpret_cast<u64 *>(smem + split_smem_bytes((unsigned)kBmax));
  auto slot = [&](int k) -> u64 * { return inbuf + 2 * ((k >> 1) * kTT + threadIdx.x) + (k & 1); };
  const u64 s0 = level_seed(cfg.seed, 0);
  const unsigned sh = ilog2_u64(lv.P);
  const unsigned mask = (unsigned)(lv.P - 1);
  const u64 ntiles = ceil_div(n, kTile);
  const unsigned base = threadIdx.x * kKPT;
  auto prefetch = [&](u64 t) {
    if (t < ntiles) {
      const u64 *src = keys + t * kTile;
      const u64 rem = n - t * kTile;
      const unsigned nt = rem < (u64)kTile ? (unsigned)rem : (unsigned)kTile;
      if (ALIGNED && base + kKPT <= nt) {
#pragma unroll
        for (int k = 0; k < kKPT; k += 2) cp_async16(slot(k), src + base + k);
      } else {
#pragma unroll
        for (int k = 0; k < kKPT; k++)
          if (base + k < nt) cp_async8(slot(k), src + base + k);
      }
    }
    cp_async_commit();
  };
  u64 t = blockIdx.x;
  prefetch(t);
  for (; t < ntiles; t += gridDim.x) {
    cp_async_wait0();  // this thread's copies of tile t have landed
    const u64 rem = n - t * kTile;
    const unsigned nt = rem < (u64)kTile ? (unsigned)rem : (unsigned)kTile;
    u64 x[kKPT];
    bool ok[kKPT];
#pragma unroll
    for (int k = 0; k < kKPT; k += 2) {
      const uint4 v = *reinterpret_cast<const uint4 *>(slot(k));
      x[k] = ((u64)v.y << 32) | v.x;
      x[k + 1] = ((u64)v.w << 32) | v.z;
    }
#pragma unroll
    for (int k = 0; k < kKPT; k++) {
      ok[k] = base + k < nt;
      if (!ok[k]) x[k] = 0;
    }
    prefetch(t + gridDim.x);
    unsigned dst[kKPT], lp[kKPT];
#pragma unroll
    for (int k = 0; k < kKPT; k++) {
      const u64 p = ok[k] ? level_pos(x[k], s0, lv.m) : 0;
      dst[k] = (unsigned)(p >> sh);
      lp[k] = (unsigned)p & mask;
    }
    multisplit_write<true>(x, lp, dst, ok, nb, sm, cfg.X, cfg.XP, UniformDest{cfg.cntX, lv.cap},
                           &meta->status);
  }
  cp_async_wait0();
}

// ---------------------------------------------------------------------------
// Fill (Algorithm 2) of level d, one bucket per CTA iteration, bits in shared
// memory; writes A_d and weight(A_d); the last CTA sizes level d+1.
// ---------------------------------------------------------------------------
__device__ void finish_level(FastMeta *meta, int d, const FastCfg &cfg) {
  volatile FLevel *vl = meta->lv;
  const u64 n = vl[d].n, m = vl[d].m, w = vl[d].weight;
  if (w > n) atomicOr(&meta->status, ST_INTERNAL);
  const u64 nn = w > n ? 0 : n - w;
  FLevel nx;
  memset(&nx, 0, sizeof(nx));
  nx.n = nn;
  nx.off = vl[d].off + m;
  if (nn == 0) {
    nx.mode = LM_DONE;
    meta->levels_used = d + 1;
  } else if ((uint32_t)(d + 1) == cfg.L) {
    nx.mode = LM_FLAT;  // fallback
    if (nn > cfg.flat_cap) atomicOr(&meta->status, ST_OVERFLOW);
  } else if (nn <= cfg.T) {
    nx.mode = LM_FLAT;  // tail
    nx.m = level_bits(nn, cfg.gamma);
  } else {
    size_bucketed(nx, nn, cfg.gamma, cfg.Pmin, cfg.Pmax, cfg.Btarget, cfg.cap_scale);
    nx.off = vl[d].off + m;
    nx.mode = LM_BUCKETED;
    // the arenas were allocated before level 0 ran (level 1's from a bound on
    // |F_1|): a level that does not fit sends the build to the unbucketed path
    const u64 acap = ((d + 1) & 1) ? cfg.capY : cfg.capX;
    const bool a_fits = ((nx.off - cfg.m0) >> 6) + (nx.m >> 6) <= cfg.arena_words;
    if (nx.B > cfg.Bmax || nx.B * nx.cap > acap || !a_fits) {
      atomicOr(&meta->status, ST_OVERFLOW);
      nx.mode = LM_NONE;
    }
  }
  meta->lv[d + 1] = nx;
  __threadfence();
}

__global__ void __launch_bounds__(kTT, 2)
k_fill_buckets(FastMeta *__restrict__ meta, int d, FastCfg cfg) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ u64 red[kTT / 32];
  __shared__ unsigned sred[kTT / 32 + 2];
  __shared__ bool last;
  if (meta->lv[d].mode != LM_BUCKETED || meta->status) return;
  const FLevel lv = meta->lv[d];
  const unsigned *parena = (d & 1) ? cfg.YP : cfg.XP;
  const u64 *cnt = (d & 1) ? cfg.cntY : cfg.cntX;
  u64 *Alev = (d == 0) ? cfg.A0 : cfg.arena + ((lv.off - cfg.m0) >> 6);
  const unsigned Pw = (unsigned)(lv.P >> 5);  // 32-bit words per bit array
  unsigned *hit = reinterpret_cast<unsigned *>(smem);
  unsigned *col = hit + Pw;
  u64 wsum = 0, got = 0;
  for (u64 b = blockIdx.x; b < lv.B; b += gridDim.x) {
    for (unsigned i = threadIdx.x; i < 2 * Pw; i += kTT) hit[i] = 0;
    __syncthreads();
    const u64 nk = min(cnt[b], lv.cap);
    got += (threadIdx.x == 0) ? cnt[b] : 0;
    const unsigned *pb = parena + b * lv.cap;
    const uint4 *pb4 = reinterpret_cast<const uint4 *>(pb);  // cap % 4 == 0: 16-byte aligned
    // 4 positions per 16-byte load, U loads in flight per thread
    constexpr int U = 4;
    for (u64 i0 = threadIdx.x; 4 * i0 < nk; i0 += (u64)U * kTT) {
      unsigned q[4 * U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const u64 i = i0 + (u64)u * kTT;
        if (4 * i + 3 < nk) {
          const uint4 v = __ldcs(pb4 + i);
          q[4 * u] = v.x;
          q[4 * u + 1] = v.y;
          q[4 * u + 2] = v.z;
          q[4 * u + 3] = v.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; j++) q[4 * u + j] = (4 * i + j < nk) ? __ldcs(pb + 4 * i + j) : ~0u;
        }
      }
#pragma unroll
      for (int j = 0; j < 4 * U; j++) {
        const unsigned p = q[j];
        if (p != ~0u) {
          const unsigned bit = 1u << (p & 31);
          const unsigned old = atomicOr(hit + (p >> 5), bit);
          if (old & bit) atomicOr(col + (p >> 5), bit);
        }
      }
    }
    __syncthreads();
    // A_d words of this bucket: positions [b P, min((b+1) P, m))
    const u64 w0 = (b * lv.P) >> 6;
    const u64 wend = min((b + 1) * lv.P, lv.m) >> 6;
    for (u64 w = w0 + threadIdx.x; w < wend; w += kTT) {
      const unsigned j = (unsigned)(w - w0) * 2;
      const u64 a = (u64)(hit[j] & ~col[j]) | ((u64)(hit[j + 1] & ~col[j + 1]) << 32);
      Alev[w] = a;
      wsum += __popcll(a);
    }
    __syncthreads();
  }
  const u64 tw = block_sum<kTT>(wsum, red);
  const u64 tg = block_sum<kTT>(got, red);
  if (threadIdx.x == 0) {
    if (tw) atomicAdd(&meta->lv[d].weight, tw);
    if (tg) atomicAdd(&meta->seen[d], tg);
    __threadfence();
    unsigned t = atomicAdd(&meta->lv[d].done, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    // the buckets must hold exactly |F_d| keys
    if (*(volatile u64 *)&meta->seen[d] != meta->lv[d].n) atomicOr(&meta->status, ST_INTERNAL);
    finish_level(meta, d, cfg);
  }
  if (last) {
    __syncthreads();
    // zero the counters of the arena that level d+1 is written into
    const FLevel nx = meta->lv[d + 1];
    if (nx.mode == LM_BUCKETED) {
      u64 *c2 = ((d + 1) & 1) ? cfg.cntY : cfg.cntX;
      for (u64 i = threadIdx.x; i < nx.B; i += kTT) c2[i] = 0;
    }
    // compaction units (kIn entries) before each bucket of level d, so that
    // the compaction can hand every CTA the same number of units
    const unsigned B = (unsigned)lv.B;
    const unsigned per = (B + kTT - 1) / kTT;
    const unsigned lo = threadIdx.x * per;
    const unsigned hi = lo + per < B ? lo + per : B;
    auto units = [&](unsigned b) -> unsigned {
      const u64 nk = min(cnt[b], lv.cap);
      return (unsigned)((nk + kIn - 1) / kIn);
    };
    unsigned su = 0;
    for (unsigned b = lo; b < hi; b++) su += units(b);
    unsigned total;
    unsigned pre = block_scan_u32<kTT>(su, sred, &total);
    for (unsigned b = lo; b < hi; b++) {
      cfg.upre[b] = pre;
      pre += units(b);
    }
    if (threadIdx.x == 0) cfg.upre[B] = total;
  }
}

// ---------------------------------------------------------------------------
// Compaction of level d: keys whose A_d bit is 0 go to their level-(d+1)
// bucket (or, for a small or final level, to the flat buffer).  The survivors
// of a tile are first packed densely in shared memory so that their
// level-(d+1) hashes are computed by full warps.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTT, 2)
k_compact_buckets(FastMeta *__restrict__ meta, int d, FastCfg cfg) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned scnt[3];  // survivors of the last three units (rotating)
  if (meta->lv[d].mode != LM_BUCKETED || meta->status) return;
  const FLevel lv = meta->lv[d];
  const FLevel nx = meta->lv[d + 1];
  if (nx.mode == LM_DONE || nx.mode == LM_NONE) return;
  // this CTA's share of the level's units (kIn-entry slices of the buckets)
  const unsigned *upre = cfg.upre;
  const unsigned U = upre[lv.B];
  const unsigned u0 = (unsigned)(((u64)U * blockIdx.x) / gridDim.x);
  const unsigned u1 = (unsigned)(((u64)U * (blockIdx.x + 1)) / gridDim.x);
  if (u0 >= u1) return;
  const bool flat = nx.mode == LM_FLAT;
  const unsigned nb = flat ? 1u : (unsigned)nx.B;
  if (nb > cfg.nbcap) {  // more destinations than the arrays were sized for
    if (threadIdx.x == 0) atomicOr(&meta->status, ST_OVERFLOW);
    return;
  }
  // the stage holds up to kTile + kIn survivors: a full tile goes to the
  // multisplit, the rest waits for the next one
  SplitSmem sm = carve_split(smem, (unsigned)cfg.nbcap, kTile + kIn);
  u64 *segA = reinterpret_cast<u64 *>(smem + split_smem_bytes((unsigned)cfg.nbcap, kTile + kIn));
  u64 *stage = sm.sorted;
  const u64 *arena = (d & 1) ? cfg.Y : cfg.X;
  const unsigned *parena = (d & 1) ? cfg.YP : cfg.XP;
  const u64 *cnt = (d & 1) ? cfg.cntY : cfg.cntX;
  u64 *out = flat ? cfg.flat : (((d + 1) & 1) ? cfg.Y : cfg.X);
  unsigned *pout = flat ? nullptr : (((d + 1) & 1) ? cfg.YP : cfg.XP);
  u64 *ocnt = flat ? &meta->n_flat : (((d + 1) & 1) ? cfg.cntY : cfg.cntX);
  const u64 ocap = flat ? cfg.flat_cap : nx.cap;
  const u64 *Alev = (d == 0) ? cfg.A0 : cfg.arena + ((lv.off - cfg.m0) >> 6);
  const u64 s_n = level_seed(cfg.seed, d + 1);
  const unsigned shn = flat ? 0u : ilog2_u64(nx.P);
  const unsigned maskn = flat ? 0u : (unsigned)(nx.P - 1);
  const unsigned lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;

  // bucket of unit u0: the last b with upre[b] <= u0 (empty buckets own no unit)
  unsigned b = 0;
  {
    unsigned lo = 0, hi = (unsigned)lv.B;
    while (hi - lo > 1) {
      const unsigned mid = (lo + hi) >> 1;
      if (upre[mid] <= u0) lo = mid;
      else hi = mid;
    }
    b = lo;
  }
  unsigned ubase = upre[b], bnext = upre[b + 1];
  auto load_segA = [&](unsigned bb) {
    const u64 w0 = ((u64)bb * lv.P) >> 6;
    const u64 wend = min((u64)(bb + 1) * lv.P, lv.m) >> 6;
    for (u64 w = w0 + threadIdx.x; w < wend; w += kTT) segA[w - w0] = Alev[w];
  };
  if (threadIdx.x < 3) scnt[threadIdx.x] = 0;
  split_clear(sm, nb);
  load_segA(b);
  __syncthreads();

  // multisplit the ns staged survivors into level d+1's buckets (or the flat list)
  auto flush = [&](unsigned ns) {
    u64 x[kKPT];
    unsigned dst[kKPT], lp[kKPT];
    bool ok[kKPT];
#pragma unroll
    for (int k = 0; k < kKPT; k++) {
      const unsigned i = (unsigned)k * kTT + threadIdx.x;
      ok[k] = i < ns;
      x[k] = ok[k] ? stage[i] : 0;
      dst[k] = 0;
      lp[k] = 0;
      if (ok[k] && !flat) {
        const u64 p = level_pos(x[k], s_n, nx.m);
        dst[k] = (unsigned)(p >> shn);
        lp[k] = (unsigned)p & maskn;
      }
    }
    __syncthreads();  // the staging area is reused by the writer
    if (flat)
      multisplit_write<false>(x, lp, dst, ok, nb, sm, out, pout, UniformDest{ocnt, ocap},
                              &meta->status);
    else
      multisplit_write<true>(x, lp, dst, ok, nb, sm, out, pout, UniformDest{ocnt, ocap},
                             &meta->status);
  };

  unsigned ns = 0;  // staged survivors (the same value in every thread)
  unsigned it = 0;
  for (unsigned u = u0; u < u1; u++, it++) {
    if (u >= bnext) {  // next non-empty bucket: its slice of A_d replaces the old one
      do {
        b++;
        ubase = bnext;
        bnext = upre[b + 1];
      } while (u >= bnext);
      __syncthreads();
      load_segA(b);
      __syncthreads();
    }
    // 1. test kInPT consecutive entries per thread (16-byte loads); a key whose
    // A_d bit is 0 survives to F_{d+1} (Algorithm 1)
    const u64 nk = min(cnt[b], lv.cap);
    const u64 e0 = (u64)(u - ubase) * kIn + (u64)threadIdx.x * kInPT;
    const unsigned *pe = parena + (u64)b * lv.cap + e0;
    const u64 *ke = arena + (u64)b * lv.cap + e0;
    // pull this thread's entries of the next unit of the bucket into L2 now, so
    // that their loads one unit later do not wait for HBM
    if (u + 1 < u1 && u + 1 < bnext && e0 + kIn < nk) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ke + kIn));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(pe + kIn));
    }
    unsigned pk[kInPT];
    u64 xk[kInPT];
    if (e0 + kInPT <= nk) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(pe));
      pk[0] = v.x;
      pk[1] = v.y;
      pk[2] = v.z;
      pk[3] = v.w;
#pragma unroll
      for (int k = 0; k < kInPT; k += 2) {
        const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(ke + k));
        xk[k] = ((u64)w.y << 32) | w.x;
        xk[k + 1] = ((u64)w.w << 32) | w.z;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kInPT; k++) {
        pk[k] = e0 + k < nk ? __ldcs(pe + k) : ~0u;
        xk[k] = e0 + k < nk ? __ldcs(ke + k) : 0;
      }
    }
    unsigned bal[kInPT], tot = 0;
    bool keep[kInPT];
#pragma unroll
    for (int k = 0; k < kInPT; k++) {
      const unsigned p = pk[k];
      keep[k] = p != ~0u && !((segA[p >> 6] >> (p & 63)) & 1ull);
      bal[k] = __ballot_sync(0xffffffffu, keep[k]);
      tot += __popc(bal[k]);
    }
    // one reservation per warp and unit in the rotating counter of this unit
    unsigned wbase = 0;
    if (lane == 0 && tot) wbase = atomicAdd(&scnt[it % 3], tot);
    wbase = ns + __shfl_sync(0xffffffffu, wbase, 0);
#pragma unroll
    for (int k = 0; k < kInPT; k++) {
      if (keep[k]) stage[wbase + __popc(bal[k] & lt)] = xk[k];
      wbase += __popc(bal[k]);
    }
    // the counter of unit it+1 was last read after the barrier of unit it-2,
    // which every thread has passed: reset it for the next unit
    if (threadIdx.x == 0) scnt[(it + 1) % 3] = 0;
    __syncthreads();
    ns += scnt[it % 3];
    // 2.+3. a full tile of survivors: hash and write it; the survivors past it
    // (fewer than kIn, beyond the multisplit's part of the stage) move to the
    // front for the next tile
    if (ns >= (unsigned)kTile) {
      flush(kTile);
      const unsigned left = ns - kTile;
      for (unsigned i = threadIdx.x; i < left; i += kTT) stage[i] = stage[kTile + i];
      __syncthreads();
      ns = left;
    }
  }
  if (ns) flush(ns);
}

// ---------------------------------------------------------------------------
// Single-CTA level loop: levels d0.. of a key set of at most kTailMaxKeys keys,
// keys and bit arrays in shared memory.  Writes A_d words, level metadata and
// the sorted fallback.
// ---------------------------------------------------------------------------
// Tail of the bucketed build: finds the first level (<= dlim) whose keys were
// sent to the flat buffer and runs the remaining levels there.
__global__ void __launch_bounds__(kTailThreads, 1)
k_tail(FastMeta *__restrict__ meta, int dlim, FastCfg cfg, u64 mcap) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int t_level;
  if (meta->status || meta->tail_done) return;
  if (threadIdx.x == 0) {
    int t = -1;
    for (int d = 0; d <= dlim && d <= (int)cfg.L; d++) {
      const unsigned md = meta->lv[d].mode;
      if (md == LM_FLAT || md == LM_DONE) {
        t = d;
        break;
      }
      if (md != LM_BUCKETED) break;
    }
    t_level = t;
  }
  __syncthreads();
  const int t = t_level;
  if (t < 0) return;  // not reached yet: the host enqueues more levels
  FLevel *lvs = meta->lv;
  if (lvs[t].mode == LM_DONE) {
    if (threadIdx.x == 0) meta->tail_done = 1;
    return;
  }
  const u64 n = lvs[t].n;
  if (threadIdx.x == 0 && meta->n_flat != n) atomicOr(&meta->status, ST_INTERNAL);
  if ((uint32_t)t == cfg.L && n > kTailMaxKeys) {
    // large fallback: sorted on the host side of the build (sort.cu)
    if (threadIdx.x == 0) {
      meta->n_fb = n;
      meta->levels_used = cfg.L;
      meta->tail_done = 2;
    }
    return;
  }
  TailSmem sm = carve_tail(smem, mcap);
  for (unsigned i = threadIdx.x; i < n; i += kTailThreads) sm.keys[i] = cfg.flat[i];
  __syncthreads();
  unsigned used = cta_levels<kTailThreads, (int)kTailMaxKeys>(
      sm, n, t, lvs[t].off, lvs, cfg.gamma, cfg.L, cfg.seed, cfg.A0,
                             cfg.arena, cfg.m0, cfg.arena_words, cfg.flat, &meta->n_fb,
                             &meta->status);
  if (threadIdx.x == 0) {
    meta->levels_used = used;
    meta->tail_done = 1;
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static bool g_attr_set = false;
double g_cap_scale = 1.0;
static size_t g_split_bytes, g_compact_bytes;

static int set_attrs() {
  if (g_attr_set) return MPHF_OK;

  g_split_bytes = split_smem_bytes((unsigned)kBmax);
  // compaction: its largest layout (kBmax destinations) + the bucket's slice of A_d
  g_compact_bytes = split_smem_bytes((unsigned)kBmax, kTile + kIn) + kPmax / 8;
  MPHF_CUDA(cudaFuncSetAttribute(k_partition0<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(g_split_bytes + kTile * 8)));
  MPHF_CUDA(cudaFuncSetAttribute(k_partition0<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(g_split_bytes + kTile * 8)));
  MPHF_CUDA(cudaFuncSetAttribute(k_compact_buckets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)g_compact_bytes));
  MPHF_CUDA(cudaFuncSetAttribute(k_fill_buckets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kPmax / 4)));
  MPHF_CUDA(cudaFuncSetAttribute(k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
  g_attr_set = true;
  return MPHF_OK;
}

// Expected |F_{d+1}| from |F_d| (a key is alone with probability (1 - 1/m)^(n-1)).
static double expect_next(double n, double gamma) {
  const double m = (double)level_bits((u64)n, gamma);
  return n * (1.0 - pow(1.0 - 1.0 / m, n - 1.0));
}

struct FastScratch {
  DevBuf meta, X, Y, XP, YP, cntX, cntY, flat, A0, arena, upre;
  void release(cudaStream_t s) {
    dev_free(upre, s);
    dev_free(meta, s); dev_free(X, s); dev_free(Y, s); dev_free(XP, s); dev_free(YP, s);
    dev_free(cntX, s); dev_free(cntY, s); dev_free(flat, s); dev_free(A0, s); dev_free(arena, s);
  }
};

// Level 1's bucket arena, allocated before level 0 runs: slots for any level
// size the device may pick for |F_1| <= n1_hi = E|F_1| + 10 sqrt(N) + 256
// (|F_1| has a standard deviation below sqrt(N)).  With B <= Bb buckets of
// cap = cap_scale (mean + 8 sqrt(mean) + 64) slots, the means summing to at
// most n + P, B cap <= cap_scale (n + P + 8 sqrt(B (n + P)) + 64 B) + 4 B.
static u64 level1_bound(u64 N, double gamma, u64 Btarget, u64 Pmax, double cap_scale,
                        u64 *n1_hi_out, u64 *Bb_out) {
  const double ev1 = expect_next((double)N, gamma);  // E|F_1|
  u64 n1_hi = (u64)ceil(ev1 + 10.0 * sqrt((double)N) + 256.0);
  if (n1_hi > N) n1_hi = N;
  const u64 m1_hi = level_bits(n1_hi, gamma);
  u64 Bb = ceil_div(m1_hi, Pmax);
  if (Bb < Btarget) Bb = Btarget;
  const double tot = (double)(n1_hi + Pmax);
  *n1_hi_out = n1_hi;
  *Bb_out = Bb;
  return (u64)(cap_scale * (tot + 8.0 * sqrt((double)Bb * tot) + 64.0 * (double)Bb)) + 4 * Bb + 64;
}

// Largest level size the tail may take for this gamma (keys + 2 bit arrays in 200 KB).
static u64 tail_limit(double gamma, u64 *mcap_out) {
  u64 T = kTailMaxKeys;
  while (T > 64) {
    u64 mc = level_bits(T, gamma);
    if (tail_smem_bytes(mc) <= 200 * 1024) {
      *mcap_out = mc;
      return T;
    }
    T >>= 1;
  }
  *mcap_out = level_bits(64, gamma);
  return 64;
}

// Returns MPHF_OK with *fallback_needed = false on success; *fallback_needed =
// true (and nothing allocated) when a device-side bound was exceeded.
int fast_build(const u64 *keys, u64 N, double gamma, uint32_t L, u64 seed, cudaStream_t st,
               mphf_t *h, bool *fallback_needed, KeyFeed *feed) {
  *fallback_needed = false;
  int rc = set_attrs();
  if (rc != MPHF_OK) return rc;
  u64 mcap = 0;
  const u64 T = tail_limit(gamma, &mcap);
  if (level_bits(T, gamma) > mcap) mcap = level_bits(T, gamma);
  FastScratch sc;
  FastCfg cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gamma = gamma;
  cfg.L = L;
  cfg.seed = seed;
  cfg.Bmax = kBmax;
  cfg.T = T;
  cfg.Pmin = 4096;
  cfg.Pmax = kPmax;
  cfg.Btarget = (u64)sm_count() * 4;
  cfg.cap_scale = g_cap_scale;
  FastMeta hm;
  memset(&hm, 0, sizeof(hm));
  const u64 m0 = level_bits(N, gamma);
  cfg.m0 = m0;
  FastMeta *meta = nullptr;
  int dlim = 0;
  int D = 1;  // levels (from 0) launched before the first look at the device's progress
  size_t comp_bytes = g_compact_bytes;  // compaction's shared memory for this build

#define FTRY(x)                    \
  do {                             \
    rc = (x);                      \
    if (rc != MPHF_OK) goto fail;  \
  } while (0)
#define FCUDA(x)                                        \
  do {                                                  \
    cudaError_t e_ = (x);                               \
    if (e_ != cudaSuccess) {                            \
      rc = cuda_fail(e_, #x);                           \
      goto fail;                                        \
    }                                                   \
  } while (0)

  FTRY(dev_alloc(sc.meta, sizeof(FastMeta), st));
  meta = (FastMeta *)sc.meta.p;
  FTRY(dev_alloc(sc.A0, m0 / 8, st));
  cfg.A0 = (u64 *)sc.A0.p;
  if (N <= T) {
    // the whole function in one CTA
    hm.lv[0].n = N;
    hm.lv[0].m = m0;
    hm.lv[0].mode = LM_FLAT;
    hm.n_flat = N;
    FTRY(dev_alloc(sc.flat, N * 8, st));
    cfg.flat = (u64 *)sc.flat.p;
    cfg.flat_cap = N;
    u64 arena_words = (u64)(L > 1 ? L - 1 : 1) * (level_bits(N, gamma) / 64);
    FTRY(dev_alloc(sc.arena, arena_words * 8, st));
    cfg.arena = (u64 *)sc.arena.p;
    cfg.arena_words = arena_words;
    if (feed) FTRY(feed->ensure(N, st));
    FCUDA(cudaMemcpyAsync(cfg.flat, keys, N * 8, cudaMemcpyDeviceToDevice, st));
    FCUDA(cudaMemcpyAsync(meta, &hm, sizeof(hm), cudaMemcpyHostToDevice, st));
    {
      LaunchScope ls("tail", st);
      k_tail<<<1, kTailThreads, tail_smem_bytes(mcap), st>>>(meta, 0, cfg, mcap);
    }
    FCUDA(cudaGetLastError());
  } else {
    size_bucketed(hm.lv[0], N, gamma, cfg.Pmin, cfg.Pmax, cfg.Btarget, cfg.cap_scale);
    hm.lv[0].off = 0;
    hm.lv[0].mode = LM_BUCKETED;
    if (hm.lv[0].B > kBmax) {
      *fallback_needed = true;
      sc.release(st);
      return MPHF_OK;
    }
    cfg.capX = hm.lv[0].B * hm.lv[0].cap;
    FTRY(dev_alloc(sc.X, cfg.capX * 8, st));
    FTRY(dev_alloc(sc.XP, cfg.capX * 4, st));
    cfg.XP = (unsigned *)sc.XP.p;
    FTRY(dev_alloc(sc.cntX, kBmax * 8, st));
    FTRY(dev_alloc(sc.cntY, kBmax * 8, st));
    FTRY(dev_alloc(sc.upre, (kBmax + 1) * 4, st));
    cfg.upre = (unsigned *)sc.upre.p;
    cfg.X = (u64 *)sc.X.p;
    cfg.cntX = (u64 *)sc.cntX.p;
    cfg.cntY = (u64 *)sc.cntY.p;
    {
      // Level 1 is sized on the device by the last CTA of level 0's fill; its
      // buffers come from a bound on |F_1| so that no host round trip sits
      // between the levels.  |F_1| (keys not alone in their bin at level 0)
      // has mean N - N (1 - 1/m_0)^(N-1) and a standard deviation below
      // sqrt(N); the bound adds 10 of those.  With n1 <= n1_hi, any level
      // size the device picks (B buckets of cap slots, B <= Bb) fits
      //   capY = n1_hi + Pmax + 8 sqrt(Bb (n1_hi + Pmax)) + 64 Bb (+ rounding),
      // since the bucket means sum to at most n + P and sqrt is concave.  A
      // level that does not fit anyway (duplicate-heavy input) is caught by
      // finish_level and the build is redone by the unbucketed path.
      const double ev1 = expect_next((double)N, gamma);  // E|F_1|
      u64 n1_hi = 0, Bb = 0;
      cfg.capY = level1_bound(N, gamma, cfg.Btarget, cfg.Pmax, cfg.cap_scale, &n1_hi, &Bb);
      const u64 m1_hi = level_bits(n1_hi, gamma);
      FTRY(dev_alloc(sc.Y, cfg.capY * 8, st));
      FTRY(dev_alloc(sc.YP, cfg.capY * 4, st));
      cfg.Y = (u64 *)sc.Y.p;
      cfg.YP = (unsigned *)sc.YP.p;
      cfg.flat_cap = n1_hi < (1ull << 22) ? n1_hi : (1ull << 22);
      if (cfg.flat_cap < T) cfg.flat_cap = T;
      FTRY(dev_alloc(sc.flat, cfg.flat_cap * 8, st));
      cfg.flat = (u64 *)sc.flat.p;
      cfg.arena_words = (u64)(L > 1 ? L - 1 : 1) * (m1_hi / 64);
      FTRY(dev_alloc(sc.arena, cfg.arena_words * 8, st));
      cfg.arena = (u64 *)sc.arena.p;
      // destination buckets of any compaction: level 1 has the most keys of
      // the levels >= 1, and a smaller level never takes more than Btarget
      // buckets (its width shrinks first), so Bb bounds them all; the
      // compaction checks it and falls back if ever exceeded
      cfg.nbcap = Bb < kBmax ? Bb : kBmax;
      comp_bytes = split_smem_bytes((unsigned)cfg.nbcap, kTile + kIn) + kPmax / 8;
      // predicted number of bucketed levels after level 0
      double e = ev1;
      D = 1;
      while (e > (double)T && D < (int)L) {
        e = expect_next(e, gamma);
        D++;
      }
    }
    FCUDA(cudaMemsetAsync(sc.cntX.p, 0, kBmax * 8, st));
    FCUDA(cudaMemcpyAsync(meta, &hm, sizeof(hm), cudaMemcpyHostToDevice, st));
    // Level-0 partition.  Keys still arriving from the host are partitioned
    // one chunk per launch as each chunk lands (the buckets' counters only
    // grow, so the launches compose); chunk starts are multiples of kTile.
    const u64 pstep = feed && feed->chunk ? feed->chunk : N;
    for (u64 c0 = 0; c0 < N; c0 += pstep) {
      const u64 cn = N - c0 < pstep ? N - c0 : pstep;
      if (feed) FTRY(feed->ensure(c0 + cn, st));
      const u64 *kc = keys + c0;
      const unsigned gridP = grid_for(cn, kTile, (unsigned)sm_count() * 2);
      LaunchScope ls("partition", st);
      if (((uintptr_t)kc & 15) == 0)
        k_partition0<true><<<gridP, kTT, g_split_bytes + kTile * 8, st>>>(kc, cn, meta, cfg);
      else
        k_partition0<false><<<gridP, kTT, g_split_bytes + kTile * 8, st>>>(kc, cn, meta, cfg);
    }
    {
      LaunchScope ls("fill_buckets", st);
      k_fill_buckets<<<(unsigned)(hm.lv[0].B < (u64)sm_count() * 2 ? hm.lv[0].B
                                                                    : (u64)sm_count() * 2),
                       kTT,
                       (size_t)(hm.lv[0].P / 4), st>>>(meta, 0, cfg);
    }
    FCUDA(cudaGetLastError());
    {
      for (int round = 0; round < 64; round++) {
        for (; dlim < D && dlim < (int)L; dlim++) {
          {
            LaunchScope ls("compact_buckets", st);
            k_compact_buckets<<<(unsigned)sm_count() * 2, kTT, comp_bytes, st>>>(meta, dlim, cfg);
          }
          if (dlim + 1 < (int)L) {
            LaunchScope ls("fill_buckets", st);
            k_fill_buckets<<<(unsigned)sm_count() * 2, kTT, (size_t)(cfg.Pmax / 4), st>>>(
                meta, dlim + 1, cfg);
          }
        }
        {
          LaunchScope ls("tail", st);
          k_tail<<<1, kTailThreads, tail_smem_bytes(mcap), st>>>(meta, dlim, cfg, mcap);
        }
        FCUDA(cudaGetLastError());
        FCUDA(cudaMemcpyAsync(&hm, meta, sizeof(hm), cudaMemcpyDeviceToHost, st));
        FCUDA(cudaStreamSynchronize(st));
        if (hm.status || hm.tail_done || dlim >= (int)L) break;
        D = dlim + 2;
      }
    }
  }
  if (N <= T) {
    FCUDA(cudaMemcpyAsync(&hm, meta, sizeof(hm), cudaMemcpyDeviceToHost, st));
    FCUDA(cudaStreamSynchronize(st));
  }
  if (hm.status & ST_OVERFLOW) {
    *fallback_needed = true;
    sc.release(st);
    return MPHF_OK;
  }
  if (hm.status & ST_DUPLICATE) {
    rc = MPHF_EDUPLICATE;
    goto fail;
  }
  if (hm.status || !hm.tail_done) {
    rc = MPHF_EINTERNAL;
    goto fail;
  }
  {
    // handle: level metadata, A = A_0 || arena, rank, fallback
    const uint32_t used = hm.levels_used;
    if (used < 1 || used > L) {
      rc = MPHF_EINTERNAL;
      goto fail;
    }
    h->L_used = used;
    for (uint32_t d = 0; d < used; d++) {
      h->n[d] = hm.lv[d].n;
      h->m[d] = hm.lv[d].m;
      h->off[d] = hm.lv[d].off;
    }
    const u64 n_fb = (used == L) ? hm.lv[L].n : 0;
    h->n[used] = n_fb;
    h->n_fb = n_fb;
    h->M = h->off[used - 1] + h->m[used - 1];
    h->n_rank = (h->M + MPHF_RANK_BLOCK - 1) / MPHF_RANK_BLOCK;
    u64 placed = 0;
    for (uint32_t d = 0; d < used; d++) placed += hm.lv[d].weight;
    if (placed + n_fb != N) {
      rc = MPHF_EINTERNAL;
      goto fail;
    }
    // A = A_0 || (A_1 A_2 ... in the arena), stored as sectors with their ranks
    FTRY(make_sectors(h, ASrc{(const u64 *)sc.A0.p, m0 / 64, (const u64 *)sc.arena.p, h->M / 64},
                      &meta->rank_total, st));
    unsigned *dflag = &meta->dup;
    if (n_fb) {
      if (hm.tail_done == 2) FTRY(sort_fallback(cfg.flat, n_fb, dflag, st));
      FTRY(dev_alloc(h->fb, n_fb * 8, st));
      FCUDA(cudaMemcpyAsync(h->fb.p, cfg.flat, n_fb * 8, cudaMemcpyDeviceToDevice, st));
    }
    FCUDA(cudaMemcpyAsync(&hm, meta, sizeof(hm), cudaMemcpyDeviceToHost, st));
    FCUDA(cudaStreamSynchronize(st));
    if (hm.dup) {
      rc = MPHF_EDUPLICATE;
      goto fail;
    }
    if (hm.rank_total != N - n_fb) {
      rc = MPHF_EINTERNAL;
      goto fail;
    }
  }
  sc.release(st);
  return MPHF_OK;

fail:
  cudaGetLastError();
  sc.release(st);
  cudaStreamSynchronize(st);
  return rc;
#undef FTRY
#undef FCUDA
}

}  // namespace bbh

// Test hooks (host arithmetic only, no device work): the bucketed level size
// the device picks for n keys, and the level-1 arena bound of an N-key build.
extern "C" int mphf_debug_size_level(uint64_t n, double gamma, uint64_t btarget, uint64_t *B,
                                     uint64_t *cap, uint64_t *P) {
  if (!B || !cap || !P || !(gamma >= 1.0) || btarget == 0) return MPHF_EINVAL;
  bbh::FLevel lv;
  memset(&lv, 0, sizeof(lv));
  bbh::size_bucketed(lv, n, gamma, 4096, bbh::kPmax, btarget, 1.0);
  *B = lv.B;
  *cap = lv.cap;
  *P = lv.P;
  return MPHF_OK;
}

extern "C" int mphf_debug_level1_bound(uint64_t N, double gamma, uint64_t btarget,
                                       uint64_t *n1_hi, uint64_t *capY, uint64_t *Bb) {
  if (!n1_hi || !capY || !Bb || !(gamma >= 1.0) || btarget == 0) return MPHF_EINVAL;
  bbh::u64 nh = 0, bb = 0;
  *capY = bbh::level1_bound(N, gamma, btarget, bbh::kPmax, 1.0, &nh, &bb);
  *n1_hi = nh;
  *Bb = bb;
  return MPHF_OK;
}
