// batched.cu -- many independent key sets built together.
//
// Every set gets exactly the function mphf_build would give it (same seed,
// same conventions); only the scheduling differs.  All sets advance level by
// level together:
//   * sets with at most T keys never leave shared memory: one CTA per set runs
//     all of its levels (k_btail, the same single-CTA loop as the plain build);
//   * larger sets are kept in position-range buckets (global bucket list:
//     bucket = (set, index)); one launch per phase and level processes the
//     buckets of all sets: ArrayFill in shared memory (k_bfill), sizing of the
//     next level of every set (k_bfin_sets / k_bfin_scan / k_bfin_desc: per set,
//     one CTA's scans over the sets, per set again) and the
//     compaction of the survivors into their next-level buckets (k_bcompact);
//     a set whose level has at most T keys moves to its flat range and joins
//     the single-CTA tail.
// The level loop is recorded once as a CUDA graph and replayed.  Bucket width
// (and so the number of buckets per set) is a tunable chosen by an autotuner.
// A set that exceeds any of its reserved bounds is rebuilt on its own with
// mphf_build, so results never depend on these choices.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "fastbuild.cuh"
#include "sector.cuh"

namespace bbh {

enum : unsigned { LM_FAILED = 4 };

struct BLvl {     // one set's state at one level of the bucketed loop
  u64 n, m, off;  // |F_d|, |A_d| bits, first bit of A_d in the set's A
  u64 P, B;       // bucket width (power of two), buckets
  u64 bbase;      // first global bucket
  u64 cap, aoff;  // slots per bucket, arena index of the set's bucket 0
  u64 weight;     // ones of A_d
  unsigned mode, sh;
};

struct BSet {     // per set
  u64 key_off, n0, m0;
  u64 a0_off;             // word offset of A_{s,0} in the A0 arena
  u64 at_off, at_words;   // levels >= 1: word offset / capacity in the tail arena
  u64 flat_off, flat_cap; // flat range (tail input, then fallback)
  u64 n_flat;             // keys appended to the flat range
  u64 n_fb;               // fallback keys
  u64 rank_total;         // ones of the set's A (rank table check)
  unsigned levels_used, status, small, tail_level;
};

// Tile t of the partition (keys [t kTile, (t + 1) kTile) of the concatenated
// sets): the sets it overlaps, the global buckets their keys can go to, and,
// when the whole tile lies in one bucketed set, that set's level-0 parameters.
struct BTile {
  u64 gb0;        // first global bucket of the tile's bucketed sets
  u64 m, base;    // one-set tile: the set's m_0 and its first bucket - gb0
  unsigned sa;    // first set overlapping the tile
  unsigned nb;    // destination buckets (0: no bucketed key in the tile)
  unsigned sh;    // one-set tile: log2 of the set's bucket width
  unsigned one;   // 1: the tile lies in one bucketed set
};

struct BCfg {
  double gamma;
  uint32_t L;
  u64 seed;
  unsigned S;
  const u64 *keys;
  BSet *sets;
  BLvl *lvl[2];                      // level state by d & 1
  unsigned *bset[2], *bidx[2];       // bucket descriptors by d & 1
  u64 *cnt[2];                       // bucket counters by d & 1
  u64 *btotal;                       // [2] buckets of the level held in slot d & 1
  u64 bcap;                          // descriptor / counter capacity
  u64 *X[2];                         // key arenas by d & 1
  unsigned *XP[2];                   // position arenas
  u64 acap[2];
  u64 *flat;
  u64 *A0, *arena;
  FLevel *hist;                      // [S][L + 1]
  u64 T, Pmin, Pmax;
  u64 Bset_max;
  double cap_scale;
  unsigned *status;                  // global (any overflow of a shared bound)
  unsigned *upre;                    // [bcap + 1] compaction units before each bucket of level d
  BTile *tiles;                      // [ceil(total / kTile)] partition tile headers
  u64 *fin;                          // [3 S] level finish: per-set counts, then their prefixes
  unsigned *fit;                     // [2] level finish: the next level's buckets fit, by d & 1
};

__host__ __device__ inline void size_set_level(BLvl &lv, u64 n, const BCfg &c) {
  lv.n = n;
  lv.m = level_bits(n, c.gamma);
  u64 want = ceil_div(lv.m, c.Bset_max);  // keep B <= Bset_max
  u64 P = c.Pmin;
  while (P < want && P < c.Pmax) P <<= 1;
  // spread a set over several buckets where it is cheap to do so
  while (P > c.Pmin && ceil_div(lv.m, P) < 4 && P > 4096) P >>= 1;
  lv.P = P;
  lv.sh = ilog2_u64(P);
  lv.B = ceil_div(lv.m, P);
  double mean = (double)n * (double)P / (double)lv.m;
  u64 cap = (u64)(c.cap_scale * (mean + 8.0 * sqrt(mean) + 64.0));
  lv.cap = (cap + 3) & ~3ull;
}

__device__ __forceinline__ u64 *set_level_words(const BCfg &c, const BSet &st, int d, u64 off) {
  return d == 0 ? c.A0 + st.a0_off : c.arena + st.at_off + ((off - st.m0) >> 6);
}

__device__ __forceinline__ void fail_set(BSet *st) { atomicOr(&st->status, ST_OVERFLOW); }

// ---------------------------------------------------------------------------
// Level 0: partition the keys of the large sets into their position buckets.
// ---------------------------------------------------------------------------
struct PartDest {
  const unsigned *bset, *bidx;
  const BLvl *lvl;
  u64 *cnt;
  u64 gb0;
  __device__ __forceinline__ DestRun operator()(unsigned i) const {
    const u64 gb = gb0 + i;
    const BLvl &lv = lvl[bset[gb]];
    return DestRun{cnt + gb, lv.aoff + (u64)bidx[gb] * lv.cap, lv.cap};
  }
};

// One thread per tile (the headers the partition reads, so that no thread of
// it searches the set offsets while the others wait).
__global__ void k_btiles(const u64 *__restrict__ key_off, u64 total, BCfg c,
                         BTile *__restrict__ tiles) {
  const u64 ntiles = ceil_div(total, kTile);
  const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const u64 t0 = t * kTile, t1 = min(t0 + kTile, total);
  // sets overlapping [t0, t1): key_off is non-decreasing with S + 1 entries
  unsigned lo = 0, hi = c.S;  // first s with key_off[s + 1] > t0
  while (lo < hi) {
    const unsigned mid = (lo + hi) >> 1;
    if (key_off[mid + 1] > t0) hi = mid;
    else lo = mid + 1;
  }
  unsigned sb = lo;
  while (sb + 1 < c.S && key_off[sb + 1] < t1) sb++;
  // global buckets of the large sets in [sa, sb] are consecutive
  u64 g0 = ~0ull, g1 = 0;
  for (unsigned s = lo; s <= sb; s++) {
    const BLvl &lv = c.lvl[0][s];
    if (lv.mode == LM_BUCKETED) {
      g0 = min(g0, lv.bbase);
      g1 = max(g1, lv.bbase + lv.B);
    }
  }
  BTile h;
  h.sa = lo;
  h.gb0 = g0 == ~0ull ? 0 : g0;
  h.nb = g0 == ~0ull ? 0u : (unsigned)(g1 - g0);
  if (g0 != ~0ull && g1 - g0 > kBmax) {
    for (unsigned s = lo; s <= sb; s++)
      if (c.lvl[0][s].mode == LM_BUCKETED) fail_set(&c.sets[s]);
    h.nb = 0;
  }
  h.one = (lo == sb && c.lvl[0][lo].mode == LM_BUCKETED) ? 1u : 0u;
  h.m = h.one ? c.lvl[0][lo].m : 0;
  h.sh = h.one ? c.lvl[0][lo].sh : 0;
  h.base = h.one ? c.lvl[0][lo].bbase - h.gb0 : 0;
  tiles[t] = h;
}

// Each thread owns kKPT consecutive keys of a tile, staged by asynchronous
// copies while the previous tile is split (the layout of k_partition0).
template <bool ALIGNED>
__global__ void __launch_bounds__(kTT, 2)
k_bpartition0(const u64 *__restrict__ key_off, u64 total, BCfg c) {
  extern __shared__ __align__(16) unsigned char smem[];
  SplitSmem sm = carve_split(smem, (unsigned)kBmax);
  split_clear(sm, (unsigned)kBmax);
  __syncthreads();
  u64 *inbuf = reinterpret_cast<u64 *>(smem + split_smem_bytes((unsigned)kBmax));
  auto slot = [&](int k) -> u64 * { return inbuf + 2 * ((k >> 1) * kTT + threadIdx.x) + (k & 1); };
  const u64 s0 = level_seed(c.seed, 0);
  const u64 ntiles = ceil_div(total, kTile);
  const unsigned tb = threadIdx.x * kKPT;
  auto prefetch = [&](u64 t) {
    if (t < ntiles) {
      const u64 *src = c.keys + t * kTile;
      const u64 rem = total - t * kTile;
      const unsigned nt = rem < (u64)kTile ? (unsigned)rem : (unsigned)kTile;
      if (ALIGNED && tb + kKPT <= nt) {
#pragma unroll
        for (int k = 0; k < kKPT; k += 2) cp_async16(slot(k), src + tb + k);
      } else {
#pragma unroll
        for (int k = 0; k < kKPT; k++)
          if (tb + k < nt) cp_async8(slot(k), src + tb + k);
      }
    }
    cp_async_commit();
  };
  u64 t = blockIdx.x;
  prefetch(t);
  for (; t < ntiles; t += gridDim.x) {
    const BTile hd = c.tiles[t];
    cp_async_wait0();  // this thread's copies of tile t have landed
    const u64 t0 = t * kTile;
    const unsigned nt = (unsigned)min((u64)kTile, total - t0);
    u64 x[kKPT];
#pragma unroll
    for (int k = 0; k < kKPT; k += 2) {
      const uint4 v = *reinterpret_cast<const uint4 *>(slot(k));
      x[k] = ((u64)v.y << 32) | v.x;
      x[k + 1] = ((u64)v.w << 32) | v.z;
    }
    // the slots are read before the next tile's copies into them are issued
    prefetch(t + gridDim.x);
    if (hd.nb == 0) continue;  // the same in every thread
    unsigned dst[kKPT], lp[kKPT];
    bool ok[kKPT];
    if (hd.one) {  // one set: its parameters for every key, no per-key set search
      const unsigned mask = (1u << hd.sh) - 1u;
#pragma unroll
      for (int k = 0; k < kKPT; k++) {
        ok[k] = tb + k < nt;
        const u64 p = level_pos(x[k], s0, hd.m);
        dst[k] = (unsigned)(hd.base + (p >> hd.sh));
        lp[k] = (unsigned)p & mask;
      }
    } else {
      unsigned s = hd.sa;
#pragma unroll
      for (int k = 0; k < kKPT; k++) {
        const u64 i = t0 + tb + k;
        ok[k] = false;
        dst[k] = 0;
        lp[k] = 0;
        if (tb + k < nt) {
          while (key_off[s + 1] <= i) s++;  // monotone in k
          const BLvl &lv = c.lvl[0][s];
          if (lv.mode == LM_BUCKETED) {
            const u64 p = level_pos(x[k], s0, lv.m);
            dst[k] = (unsigned)(lv.bbase + (p >> lv.sh) - hd.gb0);
            lp[k] = (unsigned)(p & (lv.P - 1));
            ok[k] = true;
          }
        }
      }
    }
    multisplit_write<true>(x, lp, dst, ok, hd.nb, sm, c.X[0], c.XP[0],
                           PartDest{c.bset[0], c.bidx[0], c.lvl[0], c.cnt[0], hd.gb0}, c.status);
  }
  cp_async_wait0();
}

// ---------------------------------------------------------------------------
// ArrayFill of one level for the buckets of every set.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTT, 2) k_bfill(int d, BCfg c) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int sl = d & 1;
  const u64 nbk = c.btotal[sl];
  unsigned *hit = reinterpret_cast<unsigned *>(smem);
  __shared__ int skip;
  for (u64 gb = blockIdx.x; gb < nbk; gb += gridDim.x) {
    const unsigned s = c.bset[sl][gb];
    const unsigned j = c.bidx[sl][gb];
    BSet *st = &c.sets[s];
    const BLvl lv = c.lvl[sl][s];
    __syncthreads();
    if (threadIdx.x == 0) skip = (lv.mode != LM_BUCKETED || st->status) ? 1 : 0;
    __syncthreads();
    if (skip) continue;  // one decision for the whole CTA
    const unsigned Pw = (unsigned)(lv.P >> 5);
    unsigned *col = hit + Pw;
    for (unsigned i = threadIdx.x; i < 2 * Pw; i += kTT) hit[i] = 0;
    __syncthreads();
    const u64 c0 = c.cnt[sl][gb];
    if (c0 > lv.cap && threadIdx.x == 0) fail_set(st);
    const u64 nk = min(c0, lv.cap);
    const unsigned *pb = c.XP[sl] + lv.aoff + (u64)j * lv.cap;
    const uint4 *pb4 = reinterpret_cast<const uint4 *>(pb);
    for (u64 i = threadIdx.x; 4 * i < nk; i += kTT) {
      unsigned q[4];
      if (4 * i + 3 < nk) {
        const uint4 v = __ldcs(pb4 + i);
        q[0] = v.x;
        q[1] = v.y;
        q[2] = v.z;
        q[3] = v.w;
      } else {
#pragma unroll
        for (int jj = 0; jj < 4; jj++) q[jj] = (4 * i + jj < nk) ? __ldcs(pb + 4 * i + jj) : ~0u;
      }
#pragma unroll
      for (int jj = 0; jj < 4; jj++) {
        const unsigned p = q[jj];
        if (p != ~0u) {
          const unsigned bit = 1u << (p & 31);
          const unsigned old = atomicOr(hit + (p >> 5), bit);
          if (old & bit) atomicOr(col + (p >> 5), bit);
        }
      }
    }
    __syncthreads();
    const bool fits = d == 0 || ((lv.off - st->m0) >> 6) + (lv.m >> 6) <= st->at_words;
    u64 *Alev = set_level_words(c, *st, d, lv.off);
    const u64 w0 = ((u64)j * lv.P) >> 6;
    const u64 wend = min(((u64)j + 1) * lv.P, lv.m) >> 6;
    u64 wsum = 0;
    for (u64 w = w0 + threadIdx.x; w < wend; w += kTT) {
      const unsigned jj = (unsigned)(w - w0) * 2;
      const u64 a = (u64)(hit[jj] & ~col[jj]) | ((u64)(hit[jj + 1] & ~col[jj + 1]) << 32);
      if (fits) Alev[w] = a;
      wsum += __popcll(a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_down_sync(0xffffffffu, wsum, o);
    if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(&c.lvl[sl][s].weight, wsum);
    if (!fits && threadIdx.x == 0) fail_set(st);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Next-level sizing for every set, in three launches: per set (one thread a
// set) record level d, decide where level d+1 lives and count its buckets,
// arena slots and level d's compaction units; one CTA scans those counts over
// the sets; per set again, lay out level d+1's buckets, zero their counters
// and turn level d's unit counts into the prefix the compaction reads.
// ---------------------------------------------------------------------------
static constexpr int kFinSetThreads = 256;
static constexpr int kFinishThreads = 1024;

// 1. one thread per set
__global__ void __launch_bounds__(kFinSetThreads) k_bfin_sets(int d, BCfg c) {
  const unsigned s = blockIdx.x * kFinSetThreads + threadIdx.x;
  if (s >= c.S) return;
  const int sl = d & 1, nl = (d + 1) & 1;
  BSet *st = &c.sets[s];
  const BLvl cur = c.lvl[sl][s];
  BLvl nx = cur;
  if (cur.mode == LM_BUCKETED && !st->status) {
    FLevel &h = c.hist[(u64)s * (c.L + 1) + d];
    h.n = cur.n;
    h.m = cur.m;
    h.off = cur.off;
    h.weight = cur.weight;
    if (cur.weight > cur.n) atomicOr(&st->status, ST_INTERNAL);
    const u64 nn = cur.weight > cur.n ? 0 : cur.n - cur.weight;
    memset(&nx, 0, sizeof(nx));
    nx.n = nn;
    nx.off = cur.off + cur.m;
    if (nn == 0) {
      nx.mode = LM_DONE;
      st->levels_used = d + 1;
    } else if ((uint32_t)(d + 1) == c.L) {
      nx.mode = LM_FLAT;
      st->tail_level = d + 1;
      if (nn > st->flat_cap) fail_set(st);
    } else if (nn <= c.T) {
      nx.mode = LM_FLAT;
      nx.m = level_bits(nn, c.gamma);
      st->tail_level = d + 1;
    } else {
      size_set_level(nx, nn, c);
      nx.off = cur.off + cur.m;
      nx.mode = LM_BUCKETED;
    }
  } else if (cur.mode == LM_BUCKETED) {
    nx.mode = LM_FAILED;
  }
  u64 nb = 0, ns = 0;
  if (nx.mode == LM_BUCKETED && !st->status) {
    nb = nx.B;
    ns = nx.B * nx.cap;
  } else if (nx.mode == LM_BUCKETED) {
    nx.mode = LM_FAILED;
  }
  nx.weight = 0;
  c.lvl[nl][s] = nx;
  // level d's compaction units (kIn entries) of this set's buckets, parked in
  // upre until the prefix over sets is known
  u64 nu = 0;
  if (cur.mode == LM_BUCKETED) {
    for (u64 j = 0; j < cur.B; j++) {
      const u64 g = cur.bbase + j;
      const u64 nk = c.cnt[sl][g] < cur.cap ? c.cnt[sl][g] : cur.cap;
      const unsigned u = (unsigned)((nk + kIn - 1) / kIn);
      c.upre[g] = u;
      nu += u;
    }
  }
  c.fin[3 * (u64)s] = nb;
  c.fin[3 * (u64)s + 1] = ns;
  c.fin[3 * (u64)s + 2] = nu;
}

// 2. one CTA: exclusive scans of the three counts over the sets (in place),
// the fit check of level d+1's buckets and slots, the totals
__global__ void __launch_bounds__(kFinishThreads, 1) k_bfin_scan(int d, BCfg c) {
  __shared__ u64 red[3][kFinishThreads / 32];
  const int sl = d & 1, nl = (d + 1) & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned per = (c.S + kFinishThreads - 1) / kFinishThreads;
  const unsigned lo = threadIdx.x * per, hi = min(lo + per, c.S);
  u64 v[3] = {0, 0, 0};
  for (unsigned s = lo; s < hi; s++)
    for (int k = 0; k < 3; k++) v[k] += c.fin[3 * (u64)s + k];
  u64 x[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    x[k] = v[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, x[k], o);
      if (lane >= o) x[k] += y;
    }
    if (lane == 31) red[k][warp] = x[k];
  }
  __syncthreads();
  u64 pre[3], tot[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    u64 w = lane < kFinishThreads / 32 ? red[k][lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    const u64 before = __shfl_sync(0xffffffffu, w, (warp + 31) & 31);
    tot[k] = __shfl_sync(0xffffffffu, w, kFinishThreads / 32 - 1);
    pre[k] = (warp ? before : 0) + x[k] - v[k];
  }
  for (unsigned s = lo; s < hi; s++)
    for (int k = 0; k < 3; k++) {
      const u64 t = c.fin[3 * (u64)s + k];
      c.fin[3 * (u64)s + k] = pre[k];
      pre[k] += t;
    }
  if (threadIdx.x == 0) {
    const bool fit = tot[0] <= c.bcap && tot[1] <= c.acap[nl];
    c.btotal[nl] = fit ? tot[0] : 0;
    c.fit[nl] = fit ? 1u : 0u;
    c.upre[c.btotal[sl]] = (unsigned)tot[2];
  }
}

// 3. one thread per set: level d+1's bucket layout, level d's unit prefix
__global__ void __launch_bounds__(kFinSetThreads) k_bfin_desc(int d, BCfg c) {
  const unsigned s = blockIdx.x * kFinSetThreads + threadIdx.x;
  if (s >= c.S) return;
  const int sl = d & 1, nl = (d + 1) & 1;
  const BLvl cur = c.lvl[sl][s];
  if (cur.mode == LM_BUCKETED) {
    unsigned pre = (unsigned)c.fin[3 * (u64)s + 2];
    for (u64 j = 0; j < cur.B; j++) {
      const u64 g = cur.bbase + j;
      const unsigned u = c.upre[g];
      c.upre[g] = pre;
      pre += u;
    }
  }
  BLvl &nx = c.lvl[nl][s];
  if (nx.mode != LM_BUCKETED) return;
  if (!c.fit[nl]) {
    fail_set(&c.sets[s]);
    nx.mode = LM_FAILED;
    return;
  }
  const u64 gb = c.fin[3 * (u64)s], ao = c.fin[3 * (u64)s + 1];
  nx.bbase = gb;
  nx.aoff = ao;
  for (u64 j = 0; j < nx.B; j++) {
    c.bset[nl][gb + j] = s;
    c.bidx[nl][gb + j] = (unsigned)j;
    c.cnt[nl][gb + j] = 0;
  }
}

// The three launches of level d's finish.
static void launch_bfinish(int d, const BCfg &c, cudaStream_t st) {
  const unsigned gs = (c.S + kFinSetThreads - 1) / kFinSetThreads;
  k_bfin_sets<<<gs, kFinSetThreads, 0, st>>>(d, c);
  k_bfin_scan<<<1, kFinishThreads, 0, st>>>(d, c);
  k_bfin_desc<<<gs, kFinSetThreads, 0, st>>>(d, c);
}

// ---------------------------------------------------------------------------
// Compaction of level d for the buckets of every set.
// ---------------------------------------------------------------------------
struct SetBucketDest {
  u64 *cnt;
  u64 bbase, aoff, cap;
  __device__ __forceinline__ DestRun operator()(unsigned i) const {
    return DestRun{cnt + bbase + i, aoff + (u64)i * cap, cap};
  }
};
struct SetFlatDest {
  u64 *counter;
  u64 base, cap;
  __device__ __forceinline__ DestRun operator()(unsigned) const {
    return DestRun{counter, base, cap};
  }
};

__global__ void __launch_bounds__(kTT, 2) k_bcompact(int d, BCfg c) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned scnt[3];  // survivors of the last three units (rotating)
  __shared__ int b_skip;
  __shared__ unsigned b_set;
  __shared__ u64 b_kbase, b_nk, b_w0, b_wend;
  __shared__ const u64 *b_A;
  const int sl = d & 1, nl = (d + 1) & 1;
  const u64 nbk = c.btotal[sl];
  if (nbk == 0) return;
  // this CTA's share of the level's units (kIn-entry slices of the buckets)
  const unsigned *upre = c.upre;
  const unsigned U = upre[nbk];
  const unsigned u0 = (unsigned)(((u64)U * blockIdx.x) / gridDim.x);
  const unsigned u1 = (unsigned)(((u64)U * (blockIdx.x + 1)) / gridDim.x);
  if (u0 >= u1) return;
  // destinations of one flush: the next-level buckets of one set (at most
  // Bset_max); the stage holds kTile + kIn survivors of that set
  SplitSmem sm = carve_split(smem, (unsigned)c.Bset_max, kTile + kIn);
  split_clear(sm, (unsigned)c.Bset_max);  // every flush follows a block barrier
  u64 *segA = reinterpret_cast<u64 *>(smem + split_smem_bytes((unsigned)c.Bset_max, kTile + kIn));
  u64 *stage = sm.sorted;
  const u64 s_n = level_seed(c.seed, d + 1);
  const unsigned lane = threadIdx.x & 31;
  const unsigned ltm = (1u << lane) - 1u;

  // multisplit the ns staged survivors of set s into its level d+1 buckets (or flat range)
  auto flush = [&](unsigned ns, unsigned s) {
    const BLvl nx = c.lvl[nl][s];
    BSet *st = &c.sets[s];
    const bool flat = nx.mode == LM_FLAT;
    if (!flat && nx.B > c.Bset_max) {  // more buckets than the arrays hold: the set is rebuilt alone
      if (threadIdx.x == 0) fail_set(st);
      return;
    }
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
        dst[k] = (unsigned)(p >> nx.sh);
        lp[k] = (unsigned)(p & (nx.P - 1));
      }
    }
    __syncthreads();  // the staging area is reused by the writer
    if (flat)
      multisplit_write<false>(x, lp, dst, ok, 1u, sm, c.flat, nullptr,
                              SetFlatDest{&st->n_flat, st->flat_off, st->flat_cap}, &st->status);
    else
      multisplit_write<true>(x, lp, dst, ok, (unsigned)nx.B, sm, c.X[nl], c.XP[nl],
                             SetBucketDest{c.cnt[nl], nx.bbase, nx.aoff, nx.cap}, &st->status);
  };

  // bucket holding unit u0: the last g with upre[g] <= u0 (empty buckets own no unit)
  u64 gb = 0;
  {
    u64 lo = 0, hi = nbk;
    while (hi - lo > 1) {
      const u64 mid = (lo + hi) >> 1;
      if (upre[mid] <= u0) lo = mid;
      else hi = mid;
    }
    gb = lo;
  }
  unsigned ubase = upre[gb], bnext = upre[gb + 1];
  bool fresh = true;        // the bucket of the current unit is not loaded yet
  unsigned cur_set = ~0u;   // set whose survivors are staged
  bool skip = true;
  unsigned ns = 0, it = 0;
  if (threadIdx.x < 3) scnt[threadIdx.x] = 0;
  for (unsigned u = u0; u < u1; u++) {
    if (u >= bnext) {
      do {
        gb++;
        ubase = bnext;
        bnext = upre[gb + 1];
      } while (u >= bnext);
      fresh = true;
    }
    if (fresh) {
      // one thread reads the bucket's set state (another CTA may be raising
      // that set's status right now); every thread takes the same decision
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned s = c.bset[sl][gb];
        const unsigned j = c.bidx[sl][gb];
        const BSet *st = &c.sets[s];
        const BLvl lv = c.lvl[sl][s];
        const BLvl nx = c.lvl[nl][s];
        b_skip = (lv.mode != LM_BUCKETED || *(volatile const unsigned *)&st->status ||
                  (nx.mode != LM_BUCKETED && nx.mode != LM_FLAT)) ? 1 : 0;
        b_set = s;
        b_kbase = lv.aoff + (u64)j * lv.cap;
        b_nk = c.cnt[sl][gb] < lv.cap ? c.cnt[sl][gb] : lv.cap;
        b_w0 = ((u64)j * lv.P) >> 6;
        b_wend = min(((u64)j + 1) * lv.P, lv.m) >> 6;
        b_A = set_level_words(c, *st, d, lv.off);
      }
      __syncthreads();
      const unsigned s = b_set;
      skip = b_skip != 0;
      if (s != cur_set) {
        if (ns) flush(ns, cur_set);  // survivors of another set leave first
        ns = 0;
        cur_set = s;
      }
      if (!skip) {
        const u64 w0 = b_w0, wend = b_wend;
        const u64 *Alev = b_A;
        for (u64 w = w0 + threadIdx.x; w < wend; w += kTT) segA[w - w0] = Alev[w];
        __syncthreads();
      }
      fresh = false;
    }
    if (skip) continue;
    // 1. test kInPT consecutive entries per thread (16-byte loads); a key whose
    // A_d bit is 0 survives to F_{d+1} (Algorithm 1)
    const u64 nk = b_nk;
    const u64 e0 = (u64)(u - ubase) * kIn + (u64)threadIdx.x * kInPT;
    const unsigned *pe = c.XP[sl] + b_kbase + e0;
    const u64 *ke = c.X[sl] + b_kbase + e0;
    // next unit of the bucket into L2 now (its loads come one unit later)
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
    unsigned wbase = 0;
    if (lane == 0 && tot) wbase = atomicAdd(&scnt[it % 3], tot);
    wbase = ns + __shfl_sync(0xffffffffu, wbase, 0);
#pragma unroll
    for (int k = 0; k < kInPT; k++) {
      if (keep[k]) stage[wbase + __popc(bal[k] & ltm)] = xk[k];
      wbase += __popc(bal[k]);
    }
    // the counter of unit it+1 was last read after the barrier of unit it-2,
    // which every thread has passed: reset it for the next unit
    if (threadIdx.x == 0) scnt[(it + 1) % 3] = 0;
    __syncthreads();
    ns += scnt[it % 3];
    it++;
    // 2.+3. a full tile of this set's survivors: hash and write it; the rest
    // (fewer than kIn) move to the front of the stage for the next tile
    if (ns >= (unsigned)kTile) {
      flush(kTile, cur_set);
      const unsigned left = ns - kTile;
      for (unsigned i = threadIdx.x; i < left; i += kTT) stage[i] = stage[kTile + i];
      __syncthreads();
      ns = left;
    }
  }
  if (ns) flush(ns, cur_set);
}

// ---------------------------------------------------------------------------
// Single-CTA tail of every set (sets that never left shared memory start at
// level 0 from the caller's keys).
// ---------------------------------------------------------------------------
// Batched tails are small: sets join the tail at MAXK keys and run on NT
// threads with ~MAXK * 8 bytes of shared memory, so that several tails share
// an SM (the tail is a chain of short, barrier-bound levels).  Two shapes are
// compiled; the autotuner picks one per size class.
template <int NT, int MAXK>
__global__ void __launch_bounds__(NT) k_btail(BCfg c, u64 mcap, int dlim) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned s = blockIdx.x;
  BSet *st = &c.sets[s];
  if (st->status || st->levels_used) return;
  const unsigned t = st->tail_level;
  if (!st->small && (t == 0 || (int)t > dlim)) return;  // not there yet
  FLevel *hist = c.hist + (u64)s * (c.L + 1);
  u64 n, off;
  if (st->small) {
    n = st->n0;
    off = 0;
  } else {
    const BLvl &lv = c.lvl[t & 1][s];
    n = lv.n;
    off = lv.off;
    if (st->n_flat != n) {
      if (threadIdx.x == 0) atomicOr(&st->status, ST_INTERNAL);
      return;
    }
  }
  if (n > (u64)MAXK) {  // a fallback too large to sort here
    if (threadIdx.x == 0) fail_set(st);
    return;
  }
  TailSmem sm = carve_tail(smem, mcap, MAXK);
  const u64 *src = st->small ? c.keys + st->key_off : c.flat + st->flat_off;
  for (unsigned i = threadIdx.x; i < n; i += blockDim.x) sm.keys[i] = src[i];
  if (threadIdx.x == 0) {
    hist[st->small ? 0 : t].n = n;
    hist[st->small ? 0 : t].off = off;
  }
  __syncthreads();
  const unsigned used = cta_levels<NT, MAXK>(
      sm, n, st->small ? 0 : (int)t, off, hist, c.gamma, c.L, c.seed,
                                   c.A0 + st->a0_off, c.arena + st->at_off, st->m0, st->at_words,
                                   c.flat + st->flat_off, &st->n_fb, &st->status);
  if (threadIdx.x == 0) st->levels_used = used;
}

// ---------------------------------------------------------------------------
// Finalisation: each set's A = A_0 || later levels, stored as sectors with
// their ranks (sector.cuh), and its fallback, packed into one arena shared by
// the handles.
// ---------------------------------------------------------------------------
struct BOut {
  u64 a0_off, at_off, m0, M;       // sources and total bits
  u64 S_dst, nsect, SB_dst;        // 64-bit word offsets in the output arena
  u64 fb_src, n_fb, fb_dst;
};

__global__ void k_bassemble(const BOut *__restrict__ outs, unsigned S, const u64 *__restrict__ flat,
                            u64 *__restrict__ dst) {
  for (unsigned s = blockIdx.x; s < S; s += gridDim.x) {
    const BOut o = outs[s];
    for (u64 i = threadIdx.x; i < o.n_fb; i += blockDim.x) dst[o.fb_dst + i] = flat[o.fb_src + i];
  }
}

static constexpr int kSectT = 256;
static_assert(((1u << kSBShift) % kSectT) == 0, "a chunk must not straddle superblocks");

// One CTA per set: chunks of kSectT sectors in order, a running count of ones
// carried from chunk to chunk (and reset into SB at every superblock).
__global__ void __launch_bounds__(kSectT) k_bsectors(const BOut *__restrict__ outs, unsigned S,
                                                    const u64 *__restrict__ A0,
                                                    const u64 *__restrict__ arena,
                                                    u64 *__restrict__ dst, u64 *__restrict__ totals) {
  __shared__ unsigned warp_sums[kSectT / 32];
  for (unsigned s = blockIdx.x; s < S; s += gridDim.x) {
    const BOut o = outs[s];
    const u64 W0 = o.m0 >> 6, W = o.M >> 6;
    unsigned *Sd = reinterpret_cast<unsigned *>(dst + o.S_dst);
    u64 *SB = dst + o.SB_dst;
    u64 running = 0, sbase = 0;
    for (u64 c0 = 0; c0 < o.nsect; c0 += kSectT) {
      if ((c0 & ((1ull << kSBShift) - 1)) == 0) {
        sbase = running;
        if (threadIdx.x == 0) SB[c0 >> kSBShift] = running;
      }
      const u64 t = c0 + threadIdx.x;
      unsigned w[kSectWords];
      unsigned c = 0;
      if (t < o.nsect) {
        const u64 q0 = t * kSectWords, k0 = q0 >> 1;
        unsigned h[8];
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const u64 k = k0 + i;
          const u64 u = k < W0 ? A0[o.a0_off + k] : (k < W ? arena[o.at_off + (k - W0)] : 0ull);
          h[2 * i] = (unsigned)u;
          h[2 * i + 1] = (unsigned)(u >> 32);
        }
        const bool odd = q0 & 1;
#pragma unroll
        for (int i = 0; i < (int)kSectWords; i++) {
          w[i] = odd ? h[i + 1] : h[i];
          c += __popc(w[i]);
        }
      }
      // block exclusive scan of c
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      unsigned x = c;
#pragma unroll
      for (int of = 1; of < 32; of <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, of);
        if (lane >= of) x += y;
      }
      if (lane == 31) warp_sums[warp] = x;
      __syncthreads();
      unsigned before = 0, tot = 0;
      for (int i = 0; i < kSectT / 32; i++) {
        if (i < warp) before += warp_sums[i];
        tot += warp_sums[i];
      }
      __syncthreads();
      if (t < o.nsect) {
        const unsigned rel = (unsigned)(running - sbase) + before + x - c;
        uint4 *p = reinterpret_cast<uint4 *>(Sd + 8 * t);
        p[0] = make_uint4(rel, w[0], w[1], w[2]);
        p[1] = make_uint4(w[3], w[4], w[5], w[6]);
      }
      running += tot;
    }
    if (threadIdx.x == 0) totals[s] = running;
  }
}

// ---------------------------------------------------------------------------
// Host side: persistent workspace, recorded level loop, autotuned bucket width.
// ---------------------------------------------------------------------------
struct BatchTune {
  u64 Pmax = 128 * 1024;
  u64 Bset_max = 64;
  u64 tail_keys = 8192;  // tail shape: 8192 keys on 512 threads, or 4096 on 256
};

static cudaError_t launch_btail(const BatchTune &t, const BCfg &c, u64 mcap, size_t smem, int dlim,
                                cudaStream_t st) {
  if (t.tail_keys == 4096) k_btail<256, 4096><<<c.S, 256, smem, st>>>(c, mcap, dlim);
  else k_btail<512, 8192><<<c.S, 512, smem, st>>>(c, mcap, dlim);
  return cudaGetLastError();
}

static std::mutex g_bmu;
static std::map<u64, BatchTune> g_tuned;  // key: size class
static double g_bcap_scale = 1.0;

static u64 size_class(unsigned S, u64 total) {
  unsigned a = 0, b = 0;
  while ((1ull << a) < S) a++;
  while ((1ull << b) < total) b++;
  return ((u64)a << 32) | b;
}

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  BCfg cfg;
  int D = -1;
  u64 total = 0, nbk = 0, mcap = 0;
  u64 tail_keys = 0;   // tail shape and its shared memory: a new tuning re-records
  size_t tail_b = 0;
  unsigned kernels = 0;
  cudaStream_t stream = nullptr;
};

struct Workspace {
  DevBuf bufs[24];
  size_t want[24] = {0};
  GraphCache g;
  void *pin = nullptr;  // pinned host staging for the per-set results
  size_t pin_bytes = 0;
};
static Workspace g_ws;

// Pinned host staging of at least `bytes` (kept across calls; the read-back
// of per-set state and level history is a few MB for thousands of sets).
static int pin_get(size_t bytes, void **p) {
  if (g_ws.pin && g_ws.pin_bytes >= bytes) {
    *p = g_ws.pin;
    return MPHF_OK;
  }
  if (g_ws.pin) cudaFreeHost(g_ws.pin);
  g_ws.pin = nullptr;
  g_ws.pin_bytes = 0;
  cudaError_t e = cudaMallocHost(&g_ws.pin, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g_ws.pin = nullptr;
    set_cuda_error(e, "cudaMallocHost(batched staging)");
    return MPHF_ENOMEM;
  }
  g_ws.pin_bytes = bytes;
  *p = g_ws.pin;
  return MPHF_OK;
}

// Grow workspace slot i to at least `bytes` (kept across calls).
static int ws_get(int i, size_t bytes, cudaStream_t st, void **p) {
  DevBuf &b = g_ws.bufs[i];
  if (b.p && b.bytes >= bytes) {
    *p = b.p;
    return MPHF_OK;
  }
  if (b.p) {
    cudaStreamSynchronize(st);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t sz = bytes < 256 ? 256 : bytes;
  cudaError_t e = cudaMalloc(&b.p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    set_cuda_error(e, "cudaMalloc(workspace)");
    return MPHF_ENOMEM;
  }
  b.bytes = sz;
  *p = b.p;
  return MPHF_OK;
}

}  // namespace bbh

// Shared ownership of a batched arena by many handles.
struct mphf_shared {
  bbh::DevBuf arena;
  std::atomic<int> refs{0};
};

namespace bbh {

void release_shared(mphf_shared *sh) {
  if (!sh) return;
  if (sh->refs.fetch_sub(1) == 1) {
    dev_free(sh->arena, 0);  // stream-ordered on the legacy stream, like a handle's own arrays
    delete sh;
  }
}

int build_single(const u64 *keys, u64 N, double gamma, uint32_t L, u64 seed, cudaStream_t st,
                 mphf_t **out);  // build.cu

static int batched_impl(const u64 *d_keys, const u64 *h_off, unsigned S, double gamma, uint32_t L,
                        u64 seed, cudaStream_t st, mphf_t **out, const BatchTune &tune,
                        unsigned *n_rebuilt) {
  int rc = MPHF_OK;
  *n_rebuilt = 0;
  static bool attr = false;
  const size_t split_b = split_smem_bytes((unsigned)kBmax);
  // compaction: per-set destination arrays (Bset_max) + a stage of kTile + kIn
  // + the bucket's slice of A_d; the attribute admits the largest Bset_max
  const size_t comp_b = split_smem_bytes((unsigned)tune.Bset_max, kTile + kIn) + kPmax / 8;
  const size_t comp_max = split_smem_bytes((unsigned)kBmax, kTile + kIn) + kPmax / 8;
  u64 mcap = 0;
  u64 T = tune.tail_keys;  // keep a tail's shared memory small enough for several CTAs per SM
  while (T > 64 && tail_smem_bytes(level_bits(T, gamma), tune.tail_keys) > 96 * 1024) T >>= 1;
  mcap = level_bits(T, gamma);
  const size_t tail_b = tail_smem_bytes(mcap, tune.tail_keys);
  if (!attr) {
    MPHF_CUDA(cudaFuncSetAttribute(k_bpartition0<true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(split_b + kTile * 8)));
    MPHF_CUDA(cudaFuncSetAttribute(k_bpartition0<false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(split_b + kTile * 8)));
    MPHF_CUDA(cudaFuncSetAttribute(k_bcompact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)comp_max));
    MPHF_CUDA(cudaFuncSetAttribute(k_bfill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(kPmax / 4)));
    // tail_b <= 96 KB by the choice of T above
    MPHF_CUDA(cudaFuncSetAttribute(k_btail<512, 8192>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   100 * 1024));
    MPHF_CUDA(cudaFuncSetAttribute(k_btail<256, 4096>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   100 * 1024));
    attr = true;
  }
  for (unsigned s = 0; s < S; s++) out[s] = nullptr;
  const u64 total = h_off[S] - h_off[0];
  BCfg c;
  memset(&c, 0, sizeof(c));
  c.gamma = gamma;
  c.L = L;
  c.seed = seed;
  c.S = S;
  c.T = T;
  c.Pmin = 4096;
  c.Pmax = tune.Pmax;
  c.Bset_max = tune.Bset_max;
  c.cap_scale = g_bcap_scale;
  // ---- host plan: per-set level 0
  std::vector<BSet> hs(S);
  std::vector<BLvl> hl0(S);
  std::vector<u64> koff(S + 1);
  u64 a0_words = 0, nbk = 0, nslots = 0, flat_total = 0, large_keys = 0;
  for (unsigned s = 0; s < S; s++) {
    BSet &b = hs[s];
    memset(&b, 0, sizeof(b));
    koff[s] = h_off[s] - h_off[0];
    b.key_off = koff[s];
    b.n0 = h_off[s + 1] - h_off[s];
    b.m0 = b.n0 ? level_bits(b.n0, gamma) : 0;
    b.a0_off = a0_words;
    a0_words += b.m0 / 64;
    BLvl &l = hl0[s];
    memset(&l, 0, sizeof(l));
    if (b.n0 == 0) {
      l.mode = LM_DONE;
      b.levels_used = 0;
      b.small = 0;
      continue;
    }
    if (b.n0 <= T) {
      b.small = 1;
      l.mode = LM_FLAT;
      b.flat_off = flat_total;
      b.flat_cap = b.n0;
      flat_total += b.n0;
    } else {
      size_set_level(l, b.n0, c);
      l.off = 0;
      l.mode = LM_BUCKETED;
      l.bbase = nbk;
      l.aoff = nslots;
      nbk += l.B;
      nslots += l.B * l.cap;
      large_keys += b.n0;
      b.flat_off = flat_total;
      b.flat_cap = T;
      flat_total += T;
    }
  }
  koff[S] = total;
  // tail arena (levels >= 1): a generous bound per set, checked on the device
  const double grow = 1.5 * exp(1.0 / gamma) + 0.5;
  u64 at_words = 0;
  for (unsigned s = 0; s < S; s++) {
    BSet &b = hs[s];
    if (!b.n0) continue;
    const u64 n1 = b.small ? b.n0 : (u64)ceil((double)b.n0 * (1.0 - exp(-1.0 / gamma)) * 1.05 + 64);
    const u64 w = (u64)(grow * (double)(level_bits(n1 < b.n0 ? n1 : b.n0, gamma) / 64)) + 2 * L;
    b.at_off = at_words;
    b.at_words = w;
    at_words += w;
  }
  // ---- workspace (persistent across calls so the recorded graph can be replayed)
  void *p;
  const u64 bcap = nbk + (u64)S * 2 + 64;
  c.bcap = bcap;
  c.acap[0] = nslots;
  {
    const double q = 1.0 - exp(-1.0 / gamma);  // expected share of keys left after level 0
    c.acap[1] = (u64)((double)nslots * std::min(1.0, q + 0.12)) + (u64)S * 4096;
  }
#define WS(i, bytes, dst)                                   \
  do {                                                      \
    rc = ws_get(i, (size_t)(bytes), st, &p);                \
    if (rc != MPHF_OK) return rc;                           \
    *(void **)(dst) = p;                                    \
  } while (0)
  WS(0, sizeof(BSet) * S, &c.sets);
  WS(1, sizeof(BLvl) * S, &c.lvl[0]);
  WS(2, sizeof(BLvl) * S, &c.lvl[1]);
  WS(3, 4 * bcap, &c.bset[0]);
  WS(4, 4 * bcap, &c.bset[1]);
  WS(5, 4 * bcap, &c.bidx[0]);
  WS(6, 4 * bcap, &c.bidx[1]);
  WS(7, 8 * bcap, &c.cnt[0]);
  WS(8, 8 * bcap, &c.cnt[1]);
  WS(9, 16, &c.btotal);
  WS(10, 8 * (c.acap[0] + 4), &c.X[0]);
  WS(11, 8 * (c.acap[1] + 4), &c.X[1]);
  WS(12, 4 * (c.acap[0] + 4), &c.XP[0]);
  WS(13, 4 * (c.acap[1] + 4), &c.XP[1]);
  WS(14, 8 * (flat_total + 4), &c.flat);
  WS(15, 8 * (a0_words + 4), &c.A0);
  WS(16, 8 * (at_words + 4), &c.arena);
  WS(17, sizeof(FLevel) * (u64)S * (L + 1), &c.hist);
  WS(18, 16, &c.status);
  WS(19, sizeof(u64) * (S + 1), &p);
  u64 *d_koff = (u64 *)p;
  WS(20, 4 * (bcap + 1), &c.upre);
  WS(21, sizeof(BTile) * (ceil_div(total, kTile) + 1), &c.tiles);
  WS(22, 24 * (u64)S, &c.fin);
  WS(23, 16, &c.fit);
#undef WS
  c.keys = d_keys;
  // ---- level-0 bucket descriptors on the host
  std::vector<unsigned> hb_set(nbk), hb_idx(nbk);
  for (unsigned s = 0; s < S; s++) {
    if (hl0[s].mode != LM_BUCKETED) continue;
    for (u64 j = 0; j < hl0[s].B; j++) {
      hb_set[hl0[s].bbase + j] = s;
      hb_idx[hl0[s].bbase + j] = (unsigned)j;
    }
  }
  u64 bt[2] = {nbk, 0};
  MPHF_CUDA(cudaMemcpyAsync(c.sets, hs.data(), sizeof(BSet) * S, cudaMemcpyHostToDevice, st));
  MPHF_CUDA(cudaMemcpyAsync(c.lvl[0], hl0.data(), sizeof(BLvl) * S, cudaMemcpyHostToDevice, st));
  if (nbk) {
    MPHF_CUDA(cudaMemcpyAsync(c.bset[0], hb_set.data(), 4 * nbk, cudaMemcpyHostToDevice, st));
    MPHF_CUDA(cudaMemcpyAsync(c.bidx[0], hb_idx.data(), 4 * nbk, cudaMemcpyHostToDevice, st));
    MPHF_CUDA(cudaMemsetAsync(c.cnt[0], 0, 8 * nbk, st));
  }
  MPHF_CUDA(cudaMemcpyAsync(c.btotal, bt, 16, cudaMemcpyHostToDevice, st));
  MPHF_CUDA(cudaMemcpyAsync(d_koff, koff.data(), 8 * (S + 1), cudaMemcpyHostToDevice, st));
  MPHF_CUDA(cudaMemsetAsync(c.status, 0, 16, st));
  MPHF_CUDA(cudaMemsetAsync(c.hist, 0, sizeof(FLevel) * (u64)S * (L + 1), st));
  // ---- predicted number of bucketed levels (largest set)
  u64 nmax = 0;
  for (unsigned s = 0; s < S; s++)
    if (!hs[s].small) nmax = std::max(nmax, hs[s].n0);
  int D = 0;
  {
    double e = (double)nmax;
    while (e > (double)T && D < (int)L) {
      const double m = (double)level_bits((u64)e, gamma);
      e = e * (1.0 - pow(1.0 - 1.0 / m, e - 1.0));
      D++;
    }
  }
  // ---- the level loop, recorded as a graph: partition, then per level fill,
  // finish, compaction; then the single-CTA tails
  const unsigned grid2 = (unsigned)sm_count() * 2;
  unsigned nk_rec = 0;
  auto record = [&](int Dl) -> int {
    if (nbk) {
      const u64 ntiles = ceil_div(total, kTile);
      k_btiles<<<(unsigned)ceil_div(ntiles, 256), 256, 0, st>>>(d_koff, total, c, c.tiles);
      if (((uintptr_t)c.keys & 15) == 0)
        k_bpartition0<true><<<grid2, kTT, split_b + kTile * 8, st>>>(d_koff, total, c);
      else
        k_bpartition0<false><<<grid2, kTT, split_b + kTile * 8, st>>>(d_koff, total, c);
      nk_rec += 2;
    }
    for (int d = 0; d <= Dl && d < (int)L; d++) {
      if (nbk) {
        k_bfill<<<grid2, kTT, kPmax / 4, st>>>(d, c);
        launch_bfinish(d, c, st);
        k_bcompact<<<grid2, kTT, comp_b, st>>>(d, c);
        nk_rec += 5;
      }
    }
    nk_rec++;
    return launch_btail(tune, c, mcap, tail_b, Dl + 1, st) == cudaSuccess ? MPHF_OK : MPHF_ECUDA;
  };
  // replay the recorded loop when the configuration is unchanged
  GraphCache &gc = g_ws.g;
  bool reuse = gc.exec && gc.D == D && gc.stream == st && gc.total == total && gc.nbk == nbk &&
               gc.mcap == mcap && gc.tail_keys == tune.tail_keys && gc.tail_b == tail_b &&
               memcmp(&gc.cfg, &c, sizeof(c)) == 0;
  if (!reuse) {
    if (gc.exec) {
      cudaGraphExecDestroy(gc.exec);
      gc.exec = nullptr;
    }
    // record on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the caller's
    static cudaStream_t cap = nullptr;
    if (!cap) MPHF_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaStream_t user = st;
    st = cap;
    MPHF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rrc = record(D);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    st = user;
    if (rrc != MPHF_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return cuda_fail(e != cudaSuccess ? e : cudaErrorUnknown, "graph capture");
    }
    e = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      gc.exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    gc.cfg = c;
    gc.D = D;
    gc.total = total;
    gc.nbk = nbk;
    gc.mcap = mcap;
    gc.tail_keys = tune.tail_keys;
    gc.tail_b = tail_b;
    gc.kernels = nk_rec;
    gc.stream = st;
  }
  {
    LaunchScope ls("batched_levels", st);
    MPHF_CUDA(cudaGraphLaunch(gc.exec, st));
  }
  add_launches(gc.kernels > 0 ? gc.kernels - 1 : 0);
  // ---- read back per-set results (pinned staging)
  const size_t rs_bytes = (sizeof(BSet) * S + 255) & ~(size_t)255;
  const u64 n_hist = (u64)S * (L + 1);
  void *pin = nullptr;
  rc = pin_get(rs_bytes + sizeof(FLevel) * n_hist, &pin);
  if (rc != MPHF_OK) return rc;
  BSet *rs = (BSet *)pin;
  FLevel *hist = (FLevel *)((char *)pin + rs_bytes);
  unsigned gstat[4] = {0, 0, 0, 0};
  MPHF_CUDA(cudaMemcpyAsync(rs, c.sets, sizeof(BSet) * S, cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaMemcpyAsync(gstat, c.status, 16, cudaMemcpyDeviceToHost, st));
  // the level histogram too, in the same round trip (read again below if
  // levels had to be added)
  MPHF_CUDA(cudaMemcpyAsync(hist, c.hist, sizeof(FLevel) * n_hist, cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaStreamSynchronize(st));
  bool extended = false;
  // sets whose loop did not finish within D levels (prediction short): run the
  // remaining levels unrecorded
  for (int extra = 0; extra < 64; extra++) {
    bool pending = false;
    for (unsigned s = 0; s < S; s++)
      if (rs[s].n0 && !rs[s].status && !rs[s].levels_used) pending = true;
    if (!pending || D + 1 >= (int)L) break;
    // continue from level D+1: compaction of D was recorded; fill/finish/compact D+1..
    const int d0 = D + 1;
    D = std::min((int)L - 1, D + 2);
    for (int d = d0; d <= D; d++) {
      {
        LaunchScope ls("bfill", st);
        k_bfill<<<grid2, kTT, kPmax / 4, st>>>(d, c);
      }
      {
        LaunchScope ls("bfinish", st);
        launch_bfinish(d, c, st);
      }
      {
        LaunchScope ls("bcompact", st);
        k_bcompact<<<grid2, kTT, comp_b, st>>>(d, c);
      }
    }
    {
      LaunchScope ls("btail", st);
      MPHF_CUDA(launch_btail(tune, c, mcap, tail_b, D + 1, st));
    }
    MPHF_CUDA(cudaGetLastError());
    MPHF_CUDA(cudaMemcpyAsync(rs, c.sets, sizeof(BSet) * S, cudaMemcpyDeviceToHost, st));
    MPHF_CUDA(cudaStreamSynchronize(st));
    gc.D = -1;  // the recorded graph no longer matches this build
    extended = true;
  }
  for (unsigned s = 0; s < S; s++)
    if (rs[s].status & ST_DUPLICATE) return MPHF_EDUPLICATE;
  if (extended) {
    MPHF_CUDA(cudaMemcpyAsync(hist, c.hist, sizeof(FLevel) * n_hist, cudaMemcpyDeviceToHost, st));
    MPHF_CUDA(cudaStreamSynchronize(st));
  }
  // ---- output layout
  std::vector<BOut> bo(S);
  std::vector<char> okset(S, 0);
  u64 out_words = 0;
  for (unsigned s = 0; s < S; s++) {
    const BSet &b = rs[s];
    BOut &o = bo[s];
    memset(&o, 0, sizeof(o));
    if (b.n0 == 0) {
      okset[s] = 1;
      continue;
    }
    const bool good = !b.status && b.levels_used >= 1 && b.levels_used <= L;
    if (!good) continue;
    const FLevel *hl = &hist[(u64)s * (L + 1)];
    const unsigned U = b.levels_used;
    u64 placed = 0;
    for (unsigned d = 0; d < U; d++) placed += hl[d].weight;
    const u64 n_fb = (U == L) ? b.n_fb : 0;
    if (placed + n_fb != b.n0) continue;  // rebuild this one on its own
    o.a0_off = b.a0_off;
    o.at_off = b.at_off;
    o.m0 = b.m0;
    o.M = hl[U - 1].off + hl[U - 1].m;
    o.nsect = n_sectors(o.M, kSectWords);
    o.fb_src = b.flat_off;
    o.n_fb = n_fb;
    o.S_dst = out_words;  // 8-word (64-byte) steps keep every sector 32-byte aligned
    out_words += (o.nsect * 4 + 7) & ~7ull;
    o.SB_dst = out_words;
    out_words += (n_superblocks(o.nsect) + 7) & ~7ull;
    o.fb_dst = out_words;
    out_words += (n_fb + 7) & ~7ull;
    okset[s] = 1;
  }
  mphf_shared *sh = new (std::nothrow) mphf_shared();
  if (!sh) return MPHF_ENOMEM;
  if (out_words) {
    rc = dev_alloc(sh->arena, out_words * 8, st);  // stream-ordered pool: fast to reuse
    if (rc != MPHF_OK) {
      delete sh;
      return rc;
    }
    DevBuf dbo, dtot;
    rc = dev_alloc(dbo, sizeof(BOut) * S, st);
    if (rc == MPHF_OK) rc = dev_alloc(dtot, 8 * S, st);
    if (rc != MPHF_OK) {
      dev_free(dbo, st);
      dev_free(sh->arena, st);
      delete sh;
      return rc;
    }
    std::vector<u64> totals(S, 0);
    cudaMemcpyAsync(dbo.p, bo.data(), sizeof(BOut) * S, cudaMemcpyHostToDevice, st);
    {
      LaunchScope ls("bassemble", st);
      k_bassemble<<<grid2 * 2, 256, 0, st>>>((const BOut *)dbo.p, S, c.flat,
                                           (u64 *)sh->arena.p);
    }
    {
      LaunchScope ls("bsectors", st);
      k_bsectors<<<grid2 * 2, kSectT, 0, st>>>((const BOut *)dbo.p, S, c.A0, c.arena,
                                              (u64 *)sh->arena.p, (u64 *)dtot.p);
    }
    cudaMemcpyAsync(totals.data(), dtot.p, 8 * S, cudaMemcpyDeviceToHost, st);
    dev_free(dbo, st);
    dev_free(dtot, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) {
      dev_free(sh->arena, st);
      delete sh;
      return cuda_fail(e2, "batched finalise");
    }
    for (unsigned s = 0; s < S; s++)
      if (okset[s] && rs[s].n0 && totals[s] != rs[s].n0 - bo[s].n_fb) okset[s] = 0;
  }
  // ---- handles (the device and the level seeds are the same for every set)
  int live = 0;
  int device = 0;
  cudaGetDevice(&device);
  u64 seeds[MPHF_MAX_LEVELS];
  for (uint32_t d = 0; d < L; d++) seeds[d] = level_seed(seed, d);
  std::vector<mphf_t *> recs;
  {
    unsigned n_ok = 0;
    for (unsigned s = 0; s < S; s++) n_ok += okset[s] ? 1 : 0;
    recs.resize(n_ok);
    if (n_ok && !handle_new_n(n_ok, recs.data(), false)) {
      rc = MPHF_ENOMEM;
      recs.clear();
      for (unsigned s = 0; s < S; s++) okset[s] = 0;
    }
  }
  unsigned next_rec = 0;
  for (unsigned s = 0; s < S; s++) {
    if (!okset[s]) continue;
    mphf_t *h = recs[next_rec++];
    h->device = device;
    const BSet &b = rs[s];
    h->N = b.n0;
    h->gamma = gamma;
    h->L = L;
    h->seed = seed;
    memcpy(h->s, seeds, L * sizeof(u64));
    h->path = 3;
    h->n[0] = 0;  // an empty set: no level; the tables are written below otherwise
    if (b.n0) {
      const FLevel *hl = &hist[(u64)s * (L + 1)];
      h->L_used = b.levels_used;
      for (unsigned d = 0; d < b.levels_used; d++) {
        h->n[d] = hl[d].n;
        h->m[d] = hl[d].m;
        h->off[d] = hl[d].off;
      }
      h->n_fb = bo[s].n_fb;
      h->n[b.levels_used] = h->n_fb;
      h->M = bo[s].M;
      h->n_rank = (h->M + MPHF_RANK_BLOCK - 1) / MPHF_RANK_BLOCK;
      h->n_sect = bo[s].nsect;
      u64 *base = (u64 *)sh->arena.p;
      h->S.p = base + bo[s].S_dst;
      h->S.bytes = h->n_sect * sector_bytes(kSectWords);
      h->SB.p = base + bo[s].SB_dst;
      h->SB.bytes = n_sb_entries(h->n_sect, kSectWords) * 8;
      h->fb.p = h->n_fb ? base + bo[s].fb_dst : nullptr;
      h->fb.bytes = h->n_fb * 8;
      h->shared = sh;
      live++;
    }
    out[s] = h;
  }
  if (live) sh->refs.store(live);
  else {
    dev_free(sh->arena, st);
    delete sh;
  }
  if (rc != MPHF_OK) return rc;
  // ---- sets that hit a bound: built on their own
  for (unsigned s = 0; s < S; s++) {
    if (out[s]) continue;
    rc = build_single(d_keys + koff[s], h_off[s + 1] - h_off[s], gamma, L, seed, st, &out[s]);
    if (rc != MPHF_OK) return rc;
    (*n_rebuilt)++;
  }
  return MPHF_OK;
}

}  // namespace bbh

using namespace bbh;

extern "C" int mphf_build_batched_host_offsets(const uint64_t *d_keys, const uint64_t *h_offsets,
                                               uint32_t S, double gamma, uint32_t levels,
                                               uint64_t seed, void *stream, mphf_t **out) {
  if (!out || !h_offsets || S == 0) return MPHF_EINVAL;
  for (uint32_t s = 0; s < S; s++) out[s] = nullptr;
  if (!(gamma >= 1.0) || isinf(gamma) || levels < 1 || levels > MPHF_MAX_LEVELS) return MPHF_EINVAL;
  for (uint32_t s = 0; s < S; s++)
    if (h_offsets[s + 1] < h_offsets[s]) return MPHF_EINVAL;
  if (h_offsets[S] > h_offsets[0] && (!d_keys || ((uintptr_t)d_keys & 7))) return MPHF_EINVAL;
  const u64 total = h_offsets[S] - h_offsets[0];
  BatchTune tune;
  {
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_tuned.find(size_class(S, total));
    if (it != g_tuned.end()) tune = it->second;
  }
  unsigned rebuilt = 0;
  std::lock_guard<std::mutex> lk(g_bmu);
  const u64 *keys = (const u64 *)d_keys + h_offsets[0];
  int rc = batched_impl(keys, (const u64 *)h_offsets, S, gamma, levels, seed,
                        (cudaStream_t)stream, out, tune, &rebuilt);
  if (rc != MPHF_OK) {
    for (uint32_t s = 0; s < S; s++) {
      mphf_free(out[s]);
      out[s] = nullptr;
    }
    cudaStreamSynchronize((cudaStream_t)stream);
  }
  return rc;
}

extern "C" int mphf_autotune_batched(const uint64_t *d_keys, const uint64_t *h_offsets, uint32_t S,
                                     double gamma, uint32_t levels, uint64_t seed, void *stream,
                                     double *best_ms) {
  if (!h_offsets || S == 0) return MPHF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const u64 total = h_offsets[S] - h_offsets[0];
  std::vector<BatchTune> cands;
  for (u64 P : {32768ull, 65536ull, 131072ull, 262144ull})
    for (u64 B : {16ull, 64ull})
      for (u64 tk : {4096ull, 8192ull}) {
        BatchTune t;
        t.Pmax = P;
        t.Bset_max = B;
        t.tail_keys = tk;
        cands.push_back(t);
      }
  std::vector<mphf_t *> outs(S, nullptr);
  double best = 1e30;
  BatchTune bt;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::lock_guard<std::mutex> lk(g_bmu);
  const u64 *keys = (const u64 *)d_keys + h_offsets[0];
  for (const BatchTune &t : cands) {
    double tmin = 1e30;
    for (int rep = 0; rep < 2; rep++) {
      unsigned rebuilt = 0;
      cudaEventRecord(e0, st);
      int rc = batched_impl(keys, (const u64 *)h_offsets, S, gamma, levels, seed, st, outs.data(),
                            t, &rebuilt);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      for (auto &h : outs) {
        mphf_free(h);
        h = nullptr;
      }
      if (rc != MPHF_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rebuilt) ms += 1e6f;  // a configuration that overflows loses
      tmin = std::min(tmin, (double)ms);
    }
    if (tmin < best) {
      best = tmin;
      bt = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_tuned[size_class(S, total)] = bt;
  if (best_ms) *best_ms = best;
  return MPHF_OK;
}

extern "C" int mphf_batched_tuning(uint32_t S, uint64_t total_keys, uint64_t *pmax,
                                   uint64_t *bset_max, uint64_t *tail_keys) {
  std::lock_guard<std::mutex> lk(g_bmu);
  auto it = g_tuned.find(size_class(S, total_keys));
  const BatchTune t = it != g_tuned.end() ? it->second : BatchTune();
  if (pmax) *pmax = t.Pmax;
  if (bset_max) *bset_max = t.Bset_max;
  if (tail_keys) *tail_keys = t.tail_keys;
  return it != g_tuned.end() ? MPHF_OK : MPHF_EINVAL;
}

extern "C" int mphf_batched_set_tuning(uint32_t S, uint64_t total_keys, uint64_t pmax,
                                       uint64_t bset_max, uint64_t tail_keys) {
  if (pmax < 4096 || pmax > kPmax || (pmax & (pmax - 1))) return MPHF_EINVAL;
  if (bset_max < 1 || bset_max > kBmax) return MPHF_EINVAL;
  if (tail_keys != 4096 && tail_keys != 8192) return MPHF_EINVAL;
  BatchTune t;
  t.Pmax = pmax;
  t.Bset_max = bset_max;
  t.tail_keys = tail_keys;
  std::lock_guard<std::mutex> lk(g_bmu);
  g_tuned[size_class(S, total_keys)] = t;
  return MPHF_OK;
}

extern "C" int mphf_batched_debug_config(double cap_scale) {
  if (!(cap_scale > 0.0) || cap_scale > 16.0) return MPHF_EINVAL;
  std::lock_guard<std::mutex> lk(g_bmu);
  g_bcap_scale = cap_scale;
  return MPHF_OK;
}

extern "C" void mphf_workspace_release(void) {
  std::lock_guard<std::mutex> lk(g_bmu);
  if (g_ws.g.exec) cudaGraphExecDestroy(g_ws.g.exec);
  g_ws.g.exec = nullptr;
  g_ws.g.D = -1;
  for (auto &b : g_ws.bufs) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (g_ws.pin) cudaFreeHost(g_ws.pin);
  g_ws.pin = nullptr;
  g_ws.pin_bytes = 0;
}

// The offsets in device memory: read back (S + 1 words, waiting on the
// stream) and the host-offset build runs on them.
extern "C" int mphf_build_batched(const uint64_t *d_keys, const uint64_t *d_offsets, uint32_t S,
                                  double gamma, uint32_t levels, uint64_t seed, void *stream,
                                  mphf_t **out) {
  if (!out || !d_offsets || S == 0 || ((uintptr_t)d_offsets & 7)) return MPHF_EINVAL;
  for (uint32_t s = 0; s < S; s++) out[s] = nullptr;
  std::vector<uint64_t> off((size_t)S + 1);
  cudaStream_t st = (cudaStream_t)stream;
  MPHF_CUDA(cudaMemcpyAsync(off.data(), d_offsets, off.size() * sizeof(uint64_t),
                            cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaStreamSynchronize(st));
  return mphf_build_batched_host_offsets(d_keys, off.data(), S, gamma, levels, seed, stream, out);
}
