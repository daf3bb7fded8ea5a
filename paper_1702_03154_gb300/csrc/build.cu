// build.cu -- level-by-level construction (Algorithm 1 with ArrayFill,
// Algorithm 2) of the cascading-bit-array MPHF on one GPU.
//
// Per level d the GPU form of ArrayFill is: every key of F_d sets its
// position's hit bit with one 64-bit atomicOr; a key that finds the hit bit
// already set marks the collision bit (a second atomicOr).  The hit and
// collision bits of 32 consecutive positions share one 64-bit word ("AC"
// layout: bits 0-31 hit, bits 32-63 collision), so both atomics of a key touch
// the same L2 sector.  Extraction then computes A_d = hit & ~collision into
// the concatenated A, counts weight(A_d), and derives |F_{d+1}| = |F_d| -
// weight(A_d) before any key is moved.  Compaction of level d streams F_d
// again, keeps the keys whose A_d bit is 0 (they form F_{d+1}, Algorithm 1),
// packs them with warp ballots (each warp reserving its own output run), and --
// since |A_{d+1}| is already known -- runs level d+1's ArrayFill on the
// survivors in the same pass, so F_{d+1} is read once less.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "fastbuild.cuh"
#include "sector.cuh"

namespace bbh {

int fast_build(const u64 *keys, u64 N, double gamma, uint32_t L, u64 seed, cudaStream_t st,
               mphf_t *h, bool *fallback_needed, KeyFeed *feed);
extern double g_cap_scale;

static constexpr int kFillThreads = 256;
static constexpr int kFillUnroll = 4;      // uint4 loads (2 keys each) in flight per thread
static constexpr int kExtractThreads = 256;
static constexpr int kCompactThreads = 256;
static constexpr int kCompactKPT = 16;     // keys per thread per tile
static constexpr int kCompactTile = kCompactThreads * kCompactKPT;

// ArrayFill for one key at position p of an AC array (Alg. 2, read as the
// three implications of Sec. 2.2.1: first hit sets A; a later hit sees A set
// and records the collision; the final A is hit & ~collision).
__device__ __forceinline__ void fill_position(u64 *__restrict__ AC, u64 p) {
  u64 w = p >> 5;
  u64 hit = 1ull << (p & 31);
  u64 old = atomicOr(AC + w, hit);
  if ((old & hit) && !(old & (hit << 32))) atomicOr(AC + w, hit << 32);
}

__device__ __forceinline__ uint4 load_stream(const uint4 *p) { return __ldcs(p); }

// ---------------------------------------------------------------------------
// Level-0 ArrayFill over the caller's keys.  2 keys per 16-byte load, several
// loads in flight per thread; keys are read with the streaming (evict-first)
// hint so that the AC array keeps its L2 lines.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFillThreads)
k_fill_vec(const uint4 *__restrict__ keys2, u64 npairs, u64 s, u64 m, u64 *__restrict__ AC) {
  const u64 stride = (u64)gridDim.x * kFillThreads * kFillUnroll;
  for (u64 base = (u64)blockIdx.x * kFillThreads * kFillUnroll + threadIdx.x; base < npairs;
       base += stride) {
    uint4 v[kFillUnroll];
#pragma unroll
    for (int u = 0; u < kFillUnroll; u++) {
      u64 i = base + (u64)u * kFillThreads;
      v[u] = i < npairs ? load_stream(keys2 + i) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < kFillUnroll; u++) {
      u64 i = base + (u64)u * kFillThreads;
      if (i < npairs) {
        u64 x0 = ((u64)v[u].y << 32) | v[u].x;
        u64 x1 = ((u64)v[u].w << 32) | v[u].z;
        fill_position(AC, level_pos(x0, s, m));
        fill_position(AC, level_pos(x1, s, m));
      }
    }
  }
}

__global__ void __launch_bounds__(kFillThreads)
k_fill_scalar(const u64 *__restrict__ keys, u64 n, u64 s, u64 m, u64 *__restrict__ AC) {
  const u64 stride = (u64)gridDim.x * kFillThreads;
  for (u64 i = (u64)blockIdx.x * kFillThreads + threadIdx.x; i < n; i += stride)
    fill_position(AC, level_pos(__ldcs(keys + i), s, m));
}

// |F_{d+1}| = |F_d| - weight(A_d) and the next level's size and offset.
__device__ void size_next_level(BuildMeta *meta, int d, int L, double gamma) {
  volatile BuildMeta *vm = meta;
  const u64 m = vm->m[d];
  u64 wgt = vm->weight[d];
  u64 n = vm->n[d];
  if (wgt > n) {  // cannot happen: every set bit is one distinct key
    atomicExch(&meta->status, (unsigned)MPHF_EINTERNAL);
    wgt = n;
  }
  u64 nn = n - wgt;
  vm->n[d + 1] = nn;
  vm->off[d + 1] = vm->off[d] + m;
  vm->m[d + 1] = (nn > 0 && d + 1 < L) ? level_bits(nn, gamma) : 0;
}

// ---------------------------------------------------------------------------
// Extract A_d = hit & ~collision, count weight(A_d), zero the AC array for
// reuse two levels later, and (last block) size level d+1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kExtractThreads)
k_extract(u64 *__restrict__ AC, u64 *__restrict__ A0, u64 *__restrict__ Aarena,
          BuildMeta *__restrict__ meta, int d, int L, double gamma) {
  const u64 m = meta->m[d];
  if (m == 0) return;  // level not built
  const u64 m0 = meta->m[0];
  u64 *Alev = (d == 0) ? A0 : Aarena + ((meta->off[d] - m0) >> 6);
  const u64 W = m >> 6;
  const u64 stride = (u64)gridDim.x * kExtractThreads;
  u64 local = 0;
  uint4 *AC4 = reinterpret_cast<uint4 *>(AC);
  for (u64 w = (u64)blockIdx.x * kExtractThreads + threadIdx.x; w < W; w += stride) {
    uint4 v = AC4[w];  // AC words 2w, 2w+1 = positions [64w, 64w + 64)
    u64 a = (u64)(v.x & ~v.y) | ((u64)(v.z & ~v.w) << 32);
    Alev[w] = a;
    local += __popcll(a);
    AC4[w] = make_uint4(0, 0, 0, 0);
  }
  // block reduction of the popcounts
  __shared__ u64 red[kExtractThreads / 32];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 sum = 0;
    for (int i = 0; i < kExtractThreads / 32; i++) sum += red[i];
    if (sum) atomicAdd(&meta->weight[d], sum);
    __threadfence();
    unsigned int t = atomicAdd(&meta->done[d], 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    size_next_level(meta, d, L, gamma);
  }
}

// One thread: level d+1's size once weight(A_d) is complete (grouped levels).
__global__ void k_level_done(BuildMeta *__restrict__ meta, int d, int L, double gamma) {
  __threadfence();
  size_next_level(meta, d, L, gamma);
}

// ---------------------------------------------------------------------------
// Compaction of level d (+ ArrayFill of level d+1 on the survivors).
// Warps work independently on warp tiles of 32 * kCompactKPT keys: a warp
// packs its surviving keys into its own shared-memory segment with ballots,
// reserves their output range with one atomicAdd and writes them out as one
// run.  No block barrier: the warps of a block drift apart, so the loads of
// one overlap the arithmetic of another.  The output order of F_{d+1} is
// therefore not the input order; nothing downstream depends on it (ArrayFill
// is a function of the key set).
// ---------------------------------------------------------------------------
template <bool VEC>
__global__ void __launch_bounds__(kCompactThreads, 4)
k_compact(const u64 *__restrict__ F, u64 n_in, u64 *__restrict__ Fout, const u64 *__restrict__ A0,
          const u64 *__restrict__ Aarena, u64 *__restrict__ ACnext, BuildMeta *__restrict__ meta,
          int d, u64 s_d, u64 s_next, int do_fill, u64 cap) {
  // n_in: keys of F, or ~0 for all of level d (|F_d|, from meta)
  const u64 n = n_in == ~0ull ? meta->n[d] : n_in;
  const u64 m = meta->m[d];
  if (m == 0 || n == 0 || meta->n[d + 1] == 0) return;
  const u64 m0 = meta->m[0];
  const u64 *Alev = (d == 0) ? A0 : Aarena + ((meta->off[d] - m0) >> 6);
  const u64 m_next = do_fill ? meta->m[d + 1] : 0;

  __shared__ u64 stage[kCompactTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  u64 *seg = stage + warp * (32 * kCompactKPT);
  constexpr u64 kWT = 32 * kCompactKPT;  // keys per warp tile

  const u64 nwt = (n + kWT - 1) / kWT;
  const u64 wstride = (u64)gridDim.x * (kCompactThreads / 32);
  for (u64 wt = (u64)blockIdx.x * (kCompactThreads / 32) + warp; wt < nwt; wt += wstride) {
    const u64 t0 = wt * kWT;
    u64 x[kCompactKPT];
    bool valid[kCompactKPT];
    if (VEC) {
      // lane l reads pairs (t0/2 + k*32 + l), k < KPT/2
      const uint4 *F2 = reinterpret_cast<const uint4 *>(F);
#pragma unroll
      for (int k = 0; k < kCompactKPT / 2; k++) {
        u64 i = t0 + (u64)k * 64 + 2 * lane;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (i + 1 < n) {
          v = load_stream(F2 + (i >> 1));
        } else if (i < n) {  // odd tail: never read past the last key
          u64 t = __ldcs(F + i);
          v.x = (unsigned)t;
          v.y = (unsigned)(t >> 32);
        }
        x[2 * k] = ((u64)v.y << 32) | v.x;
        x[2 * k + 1] = ((u64)v.w << 32) | v.z;
        valid[2 * k] = i < n;
        valid[2 * k + 1] = i + 1 < n;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kCompactKPT; k++) {
        u64 i = t0 + (u64)k * 32 + lane;
        valid[k] = i < n;
        x[k] = valid[k] ? __ldcs(F + i) : 0;
      }
    }
    // survival test: the key's bit in A_d is 0
    bool keep[kCompactKPT];
#pragma unroll
    for (int k = 0; k < kCompactKPT; k++) {
      keep[k] = false;
      if (valid[k]) {
        u64 p = level_pos(x[k], s_d, m);
        keep[k] = !((__ldg(Alev + (p >> 6)) >> (p & 63)) & 1ull);
      }
    }
    unsigned cnt = 0;
#pragma unroll
    for (int k = 0; k < kCompactKPT; k++) {
      unsigned b = __ballot_sync(0xffffffffu, keep[k]);
      if (keep[k]) seg[cnt + __popc(b & lt_mask)] = x[k];
      cnt += __popc(b);
    }
    u64 base = 0;
    if (lane == 0 && cnt) base = atomicAdd(&meta->out_count[d], (u64)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    if (base + cnt > cap && lane == 0) atomicExch(&meta->status, (unsigned)MPHF_EINTERNAL);
    for (unsigned i = lane; i < cnt; i += 32) {
      u64 y = seg[i];
      if (base + i >= cap) break;  // never write past F_{d+1}; status is already set
      Fout[base + i] = y;
      if (m_next) fill_position(ACnext, level_pos(y, s_next, m_next));
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Slab order.  When a level's AC array is far larger than L2, random atomics
// on it go to HBM one sector at a time.  Its keys are then first grouped by
// slab (2^27 consecutive positions, a 32 MB stretch of AC): a count
// per slab, then a multisplit into exact slab ranges.  The fill and the
// compaction stream the grouped keys in order, so all CTAs work inside one or
// two slabs at any moment and the atomics and bit tests hit L2.  The grouping
// changes no result: ArrayFill and the compaction depend on the key set only.
// ---------------------------------------------------------------------------
static unsigned g_slab_shift = 27;           // positions per slab: 2^27
static u64 g_slab_min_ac = 64ull << 20;       // group levels whose AC exceeds this (bytes)
static constexpr unsigned kSlabMax = (unsigned)kBmax; // slabs a multisplit can take
static constexpr int kSlabCountThreads = 256;

__global__ void __launch_bounds__(kSlabCountThreads)
k_slab_count(const u64 *__restrict__ keys, u64 n, u64 s, u64 m, u64 base, unsigned shift,
             unsigned nslab, u64 *__restrict__ counts) {
  __shared__ unsigned hist[kSlabMax];
  for (unsigned i = threadIdx.x; i < nslab; i += kSlabCountThreads) hist[i] = 0;
  __syncthreads();
  const u64 stride = (u64)gridDim.x * kSlabCountThreads;
  for (u64 i = (u64)blockIdx.x * kSlabCountThreads + threadIdx.x; i < n; i += stride)
    atomicAdd(&hist[(unsigned)((level_pos(__ldcs(keys + i), s, m) - base) >> shift)], 1u);
  __syncthreads();
  for (unsigned i = threadIdx.x; i < nslab; i += kSlabCountThreads)
    if (hist[i]) atomicAdd(counts + i, (u64)hist[i]);
}

// Destination slab i of the multisplit: cursor[i] starts at the slab's first
// index and end[i] is one past its last.
struct SlabDest {
  u64 *cursor;
  const u64 *end;
  __device__ __forceinline__ DestRun operator()(unsigned i) const {
    return DestRun{cursor + i, 0, end[i]};
  }
};

// The next tile's keys are staged in shared memory by cp.async while the
// current tile is split (each thread owns kKPT consecutive keys of a tile;
// ALIGNED: the keys are 16-byte aligned, so they move in 16-byte copies).
// WITH_POS: each key's position within its slab (below 2^20) goes to pout
// beside it (the fine slabs' fill and compaction then need no hash).  ONE: at
// most kTT slabs, one per thread in the multisplit.
template <bool ALIGNED, bool WITH_POS, bool ONE>
__global__ void __launch_bounds__(kTT, 2)
k_slab_scatter(const u64 *__restrict__ keys, u64 n, u64 s, u64 m, u64 base, unsigned shift,
               unsigned nslab, u64 *__restrict__ cursor, const u64 *__restrict__ end, u64 *__restrict__ out,
               unsigned *__restrict__ pout, unsigned *__restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  SplitSmem sm = carve_split(smem, nslab);
  split_clear(sm, nslab);
  __syncthreads();
  u64 *inbuf = reinterpret_cast<u64 *>(smem + split_smem_bytes(nslab));
  auto slot = [&](int k) -> u64 * { return inbuf + 2 * ((k >> 1) * kTT + threadIdx.x) + (k & 1); };
  const u64 ntiles = (n + kTile - 1) / kTile;
  const unsigned tb = threadIdx.x * kKPT;
  auto prefetch = [&](u64 t) {
    if (t < ntiles) {
      const u64 *src = keys + t * kTile;
      const u64 rem = n - t * kTile;
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
    cp_async_wait0();  // this thread's copies of tile t have landed
    const u64 rem = n - t * kTile;
    const unsigned nt = rem < (u64)kTile ? (unsigned)rem : (unsigned)kTile;
    u64 x[kKPT];
    unsigned dst[kKPT], lp[kKPT];
    bool ok[kKPT];
#pragma unroll
    for (int k = 0; k < kKPT; k += 2) {
      const uint4 v = *reinterpret_cast<const uint4 *>(slot(k));
      x[k] = ((u64)v.y << 32) | v.x;
      x[k + 1] = ((u64)v.w << 32) | v.z;
    }
    // the slots are read (into registers) before the next tile's copies are
    // issued: each thread copies into and reads only its own slots
    prefetch(t + gridDim.x);
#pragma unroll
    for (int k = 0; k < kKPT; k++) {
      ok[k] = tb + k < nt;
      if (!ok[k]) x[k] = 0;
      const u64 r = ok[k] ? level_pos(x[k], s, m) - base : 0;
      dst[k] = (unsigned)(r >> shift);
      lp[k] = WITH_POS ? (unsigned)r & ((1u << shift) - 1u) : 0u;
    }
    if (ONE)
      multisplit_write_one<WITH_POS>(x, lp, dst, ok, nslab, sm, out, pout, SlabDest{cursor, end},
                                     status);
    else
      multisplit_write<WITH_POS>(x, lp, dst, ok, nslab, sm, out, pout, SlabDest{cursor, end},
                                 status);
  }
  cp_async_wait0();
}

// ArrayFill and compaction of one fine slab of a grouped level, in shared
// memory: CTA f takes the entries [fstart[f], fend[f]) of T (keys) and TP
// (their positions within the fine slab) for positions [p0, min(p0 +
// 2^kFineShift, lim)), p0 = base + f 2^kFineShift.  Pass 1 sets the hit and
// collision bits from the stored positions (Algorithm 2, the same three
// implications as fill_position); A_d's words of the range are written and
// their ones added to weight(A_d).  Every key hashed into these positions is
// in this CTA, so its bits are final: pass 2 reads the keys, hashes each to
// its position again (level seed s_d, size m_d: one memory round trip a step
// instead of a position load and then a key load) and keeps those whose A_d
// bit is 0 (F_{d+1}, Algorithm 1), staged per warp and written to Fout in
// runs reserved with one atomicAdd on out_count.  A run past `cap` is not
// written and raises bit 0 of fuse_status.
static constexpr unsigned kFineShift = 18;
static constexpr int kFineThreads = 512;
static constexpr int kFineStage = 256;  // survivors a warp stages before writing them
static constexpr size_t kFineSmem =
    2 * ((size_t)1 << kFineShift) / 8 + (size_t)(kFineThreads / 32) * kFineStage * 8;

__global__ void __launch_bounds__(kFineThreads, 2)
k_fine_fill(const u64 *__restrict__ T, const unsigned *__restrict__ TP,
            const u64 *__restrict__ fstart, const u64 *__restrict__ fend,
            const u64 *__restrict__ fcap, u64 base, u64 lim, u64 *__restrict__ Alev,
            u64 *__restrict__ weight, u64 *__restrict__ Fout, u64 cap,
            u64 *__restrict__ out_count, unsigned *__restrict__ fuse_status, u64 s_d, u64 m_d) {
  extern __shared__ __align__(16) unsigned fsm[];
  __shared__ u64 red[kFineThreads / 32];
  constexpr unsigned kWords = (1u << kFineShift) / 32;
  unsigned *hit = fsm, *col = fsm + kWords;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 *stage = reinterpret_cast<u64 *>(fsm + 2 * kWords) + warp * kFineStage;
  const u64 p0 = base + ((u64)blockIdx.x << kFineShift);
  const u64 np = min((u64)1 << kFineShift, lim - p0);  // lim: end of the slab, a multiple of 64
  for (unsigned i = threadIdx.x; i < 2 * kWords; i += kFineThreads) fsm[i] = 0;
  __syncthreads();
  const u64 i0 = fstart[blockIdx.x];
  const u64 i1 = min(fend[blockIdx.x], fcap[blockIdx.x]);  // an overflowed range stops at its end
  // [ia, ib): the 16-byte aligned part of the range, read four positions at a
  // time; the at most 3 + 3 entries around it are read one by one
  const u64 ia = min((i0 + 3) & ~3ull, i1);
  const u64 ib = max(ia, i1 & ~3ull);
  auto fill_one = [&](unsigned q) {
    const unsigned bit = 1u << (q & 31);
    const unsigned old = atomicOr(hit + (q >> 5), bit);
    if (old & bit) atomicOr(col + (q >> 5), bit);
  };
  // pass 1: ArrayFill, four 16-byte position loads per thread in flight
  {
    const uint4 *TP4 = reinterpret_cast<const uint4 *>(TP);
    const u64 va = ia >> 2, vb = ib >> 2;
    constexpr int kU = 4;
    u64 v = va + threadIdx.x;
    for (; v + (u64)(kU - 1) * kFineThreads < vb; v += (u64)kU * kFineThreads) {
      uint4 q[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) q[u] = TP4[v + (u64)u * kFineThreads];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        fill_one(q[u].x);
        fill_one(q[u].y);
        fill_one(q[u].z);
        fill_one(q[u].w);
      }
    }
    for (; v < vb; v += kFineThreads) {
      const uint4 q = TP4[v];
      fill_one(q.x);
      fill_one(q.y);
      fill_one(q.z);
      fill_one(q.w);
    }
    const u64 e = threadIdx.x < ia - i0 ? i0 + threadIdx.x
                  : (threadIdx.x < (ia - i0) + (i1 - ib) ? ib + (threadIdx.x - (ia - i0)) : i1);
    if (e < i1) fill_one(TP[e]);
  }
  __syncthreads();
  u64 wsum = 0;
  for (unsigned w = threadIdx.x; w < (unsigned)(np >> 6); w += kFineThreads) {
    const u64 a = (u64)(hit[2 * w] & ~col[2 * w]) | ((u64)(hit[2 * w + 1] & ~col[2 * w + 1]) << 32);
    Alev[(p0 >> 6) + w] = a;
    wsum += __popcll(a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_down_sync(0xffffffffu, wsum, o);
  if (lane == 0) red[warp] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < kFineThreads / 32; w++) t += red[w];
    if (t) atomicAdd(weight, t);
  }
  // pass 2: compaction; a warp step takes kC chunks of 128 entries, each lane
  // four consecutive entries of a chunk (its keys in two 16-byte loads)
  const unsigned lt = (1u << lane) - 1u;
  unsigned cnt = 0;
  auto flush = [&]() {
    u64 b0 = 0;
    if (lane == 0 && cnt) b0 = atomicAdd(out_count, (u64)cnt);
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (lane == 0 && b0 + cnt > cap) atomicOr(fuse_status, 1u);
    __syncwarp();
    for (unsigned j = lane; j < cnt; j += 32)
      if (b0 + j < cap) Fout[b0 + j] = stage[j];
    __syncwarp();
    cnt = 0;
  };
  auto kept = [&](unsigned q) { return !(((hit[q >> 5] & ~col[q >> 5]) >> (q & 31)) & 1u); };
  auto put = [&](bool keep, u64 x) {
    const unsigned bb = __ballot_sync(0xffffffffu, keep);
    if (keep) stage[cnt + __popc(bb & lt)] = x;
    cnt += __popc(bb);
    if (cnt > (unsigned)(kFineStage - 32)) flush();
  };
  {
    const uint4 *T4 = reinterpret_cast<const uint4 *>(T);  // T is 16-byte aligned like TP
    const u64 va = ia >> 2, vb = ib >> 2;
    constexpr int kC = 2;
    // each lane's four keys of a chunk in two 16-byte loads; their positions
    // in the fine slab come from the level hash (no second read of TP)
    auto qpos = [&](u64 x) { return (unsigned)(level_pos(x, s_d, m_d) - p0); };
    constexpr u64 kStep = (u64)kC * kFineThreads;
    const u64 nsteps = (vb - va + kStep - 1) / kStep;
    for (u64 st = 0; st < nsteps; st++) {
      const u64 c0 = va + st * kStep + (u64)warp * 32;
      uint4 x01[kC], x23[kC];
      bool ok[kC];
#pragma unroll
      for (int c = 0; c < kC; c++) {
        const u64 v = c0 + (u64)c * kFineThreads + lane;
        ok[c] = v < vb;
        x01[c] = ok[c] ? __ldcs(T4 + 2 * v) : make_uint4(0, 0, 0, 0);
        x23[c] = ok[c] ? __ldcs(T4 + 2 * v + 1) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int c = 0; c < kC; c++) {
        const u64 y0 = ((u64)x01[c].y << 32) | x01[c].x, y1 = ((u64)x01[c].w << 32) | x01[c].z;
        const u64 y2 = ((u64)x23[c].y << 32) | x23[c].x, y3 = ((u64)x23[c].w << 32) | x23[c].z;
        put(ok[c] && kept(qpos(y0)), y0);
        put(ok[c] && kept(qpos(y1)), y1);
        put(ok[c] && kept(qpos(y2)), y2);
        put(ok[c] && kept(qpos(y3)), y3);
      }
    }
    // the entries around the aligned part (at most 6): warp 0, one per lane
    if (warp == 0) {
      const u64 nh = ia - i0, nt = i1 - ib;
      const u64 e = lane < nh ? i0 + lane : (lane < nh + nt ? ib + (lane - nh) : i1);
      const bool keep = e < i1 && kept(TP[e]);
      put(keep, keep ? T[e] : 0);
    }
  }
  flush();
}

// Fine slab f of a slab takes T[f cap, (f + 1) cap): a cap of mean + 8 sigma
// + 64 keys, so no count pass is needed; a slab whose keys overflow a range
// (raised in status by the multisplit) is redone with exact counts.
__global__ void k_fine_ranges(u64 *__restrict__ cursor, u64 *__restrict__ end,
                              u64 *__restrict__ start, unsigned nf, u64 cap) {
  const unsigned f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < nf) {
    start[f] = cursor[f] = (u64)f * cap;
    end[f] = (u64)(f + 1) * cap;
  }
}

// ---------------------------------------------------------------------------
// Host orchestration.
// ---------------------------------------------------------------------------
struct Scratch {
  DevBuf meta, AC0, AC1, A0, arena, F1, F2, dupflag, R, slab, T, TP;
  void release(cudaStream_t s) {
    dev_free(meta, s); dev_free(AC0, s); dev_free(AC1, s); dev_free(A0, s);
    dev_free(arena, s); dev_free(F1, s); dev_free(F2, s); dev_free(dupflag, s);
    dev_free(R, s); dev_free(slab, s); dev_free(T, s); dev_free(TP, s);
  }
};

// Slabs of a level of m positions, or 0 if its keys are left in their order.
static unsigned slab_count_for(u64 m) {
  if (m / 4 <= g_slab_min_ac) return 0;  // the AC array (2 bits a position) is L2-sized
  const u64 ns = (m + (1ull << g_slab_shift) - 1) >> g_slab_shift;
  return ns <= kSlabMax ? (unsigned)ns : 0u;
}

using SlabScatterFn = void (*)(const u64 *, u64, u64, u64, u64, unsigned, unsigned, u64 *,
                               const u64 *, u64 *, unsigned *, unsigned *);
static SlabScatterFn slab_scatter_fn(bool al, bool pos, bool one) {
  if (one) {
    if (pos) return al ? k_slab_scatter<true, true, true> : k_slab_scatter<false, true, true>;
    return al ? k_slab_scatter<true, false, true> : k_slab_scatter<false, false, true>;
  }
  if (pos) return al ? k_slab_scatter<true, true, false> : k_slab_scatter<false, true, false>;
  return al ? k_slab_scatter<true, false, false> : k_slab_scatter<false, false, false>;
}

// out <- the n keys of F grouped by slab: position p of level (s, m) goes to
// slab (p - base) >> shift, nslab slabs; se[i], se[nslab + i] receive slab i's
// range of out.  slab: 4 * kSlabMax u64 of device scratch.
static int slab_attrs() {
  static bool attr = false;
  if (!attr) {
    const int sb = (int)(split_smem_bytes(kSlabMax) + kTile * 8);
    for (int v = 0; v < 8; v++)
      MPHF_CUDA(cudaFuncSetAttribute(slab_scatter_fn(v & 1, v & 2, v & 4),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, sb));
    MPHF_CUDA(cudaFuncSetAttribute(k_fine_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kFineSmem));
    attr = true;
  }
  return MPHF_OK;
}

// One launch of the slab multisplit: keys F (n) into the ranges cursor[i] ..
// end[i] of out (and, with pout, their in-slab positions into pout).
static void launch_slab_scatter(const u64 *F, u64 n, u64 s, u64 m, u64 base, unsigned shift,
                                unsigned nslab, u64 *cursor, const u64 *end, u64 *out,
                                unsigned *pout, unsigned *status, cudaStream_t st) {
  LaunchScope ls("slab_scatter", st);
  const unsigned g = grid_for(n, kTile, (unsigned)sm_count() * 2);
  const size_t sb = split_smem_bytes(nslab) + kTile * 8;
  const bool al = ((uintptr_t)F & 15) == 0;
  slab_scatter_fn(al, pout != nullptr, nslab <= (unsigned)kTT)<<<g, kTT, sb, st>>>(
      F, n, s, m, base, shift, nslab, cursor, end, out, pout, status);
}

static int group_keys(const u64 *F, u64 n, u64 s, u64 m, u64 base, unsigned shift,
                      unsigned nslab, u64 *out, unsigned *pout, u64 *slab, unsigned *status,
                      std::vector<u64> &se, cudaStream_t st) {
  int rc0 = slab_attrs();
  if (rc0 != MPHF_OK) return rc0;
  u64 *counts = slab, *cursor = slab + kSlabMax, *end = slab + 2 * kSlabMax;
  MPHF_CUDA(cudaMemsetAsync(counts, 0, nslab * 8, st));
  {
    LaunchScope ls("slab_count", st);
    k_slab_count<<<grid_for(n, kSlabCountThreads * 16, (unsigned)sm_count() * 8),
                   kSlabCountThreads, 0, st>>>(F, n, s, m, base, shift, nslab, counts);
  }
  std::vector<u64> c(nslab);
  se.assign(2 * (size_t)nslab, 0);
  MPHF_CUDA(cudaMemcpyAsync(c.data(), counts, nslab * 8, cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaStreamSynchronize(st));
  u64 run = 0;
  for (unsigned i = 0; i < nslab; i++) {
    se[i] = run;
    run += c[i];
    se[nslab + i] = run;
  }
  if (run != n) return MPHF_EINTERNAL;
  // pageable copies: the host data is staged before each call returns
  MPHF_CUDA(cudaMemcpyAsync(cursor, se.data(), nslab * 8, cudaMemcpyHostToDevice, st));
  MPHF_CUDA(cudaMemcpyAsync(end, se.data() + nslab, nslab * 8, cudaMemcpyHostToDevice, st));
  launch_slab_scatter(F, n, s, m, base, shift, nslab, cursor, end, out, pout, status, st);
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

// Capacity of slab c of a level's coarse grouping when n keys spread over m
// positions: its share of the keys plus 8 standard deviations and 64 keys, a
// multiple of 4 (so every slab starts 32-byte aligned).
static u64 slab_cap(u64 n, u64 m, unsigned c) {
  const u64 lo = (u64)c << g_slab_shift;
  const u64 range = std::min((u64)1 << g_slab_shift, m - lo);
  const double mean = (double)n * (double)range / (double)m;
  const u64 cap = (u64)(g_cap_scale * (mean + 8.0 * sqrt(mean) + 64.0));  // scale: tests only
  return (cap + 3) & ~3ull;
}

// Room the coarse grouping of n keys over m positions (nslab slabs) needs:
// the sum of the slab capacities, and at least n (the exact redo).
static u64 grouped_room(u64 n, u64 m, unsigned nslab) {
  u64 t = 0;
  for (unsigned c = 0; c < nslab; c++) t += slab_cap(n, m, c);
  return std::max(t, n);
}

// The coarse grouping of a level (slabs of 2^g_slab_shift positions): keys
// go to fixed-capacity slab ranges of out (slab_cap), so no count pass is
// needed; se receives the ranges actually filled.  If a range overflows
// (thousands of equal keys), the grouping is done again with exact counts.
static int group_level(const u64 *F, u64 n, u64 s, u64 m, unsigned nslab, u64 *out, u64 *slab,
                       unsigned *status, std::vector<u64> &se, cudaStream_t st) {
  int rc0 = slab_attrs();
  if (rc0 != MPHF_OK) return rc0;
  u64 *cursor = slab + kSlabMax, *end = slab + 2 * kSlabMax;
  std::vector<u64> lo(2 * (size_t)nslab);
  u64 run = 0;
  for (unsigned c = 0; c < nslab; c++) {
    lo[c] = run;
    run += slab_cap(n, m, c);
    lo[nslab + c] = run;
  }
  // pageable copies: the host data is staged before each call returns
  MPHF_CUDA(cudaMemcpyAsync(cursor, lo.data(), nslab * 8, cudaMemcpyHostToDevice, st));
  MPHF_CUDA(cudaMemcpyAsync(end, lo.data() + nslab, nslab * 8, cudaMemcpyHostToDevice, st));
  launch_slab_scatter(F, n, s, m, 0, g_slab_shift, nslab, cursor, end, out, nullptr, status, st);
  MPHF_CUDA(cudaGetLastError());
  std::vector<u64> cur(nslab);
  unsigned flag = 0;
  MPHF_CUDA(cudaMemcpyAsync(cur.data(), cursor, nslab * 8, cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaMemcpyAsync(&flag, status, 4, cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    MPHF_CUDA(cudaMemsetAsync(status, 0, 4, st));
    return group_keys(F, n, s, m, 0, g_slab_shift, nslab, out, nullptr, slab, status, se, st);
  }
  se.assign(2 * (size_t)nslab, 0);
  u64 total = 0;
  for (unsigned c = 0; c < nslab; c++) {
    se[c] = lo[c];
    se[nslab + c] = cur[c];
    total += cur[c] - lo[c];
  }
  return total == n ? MPHF_OK : MPHF_EINTERNAL;
}

// ArrayFill and compaction of a level whose keys R are grouped by slab
// (ranges se): each slab's keys are grouped again into fine slabs of
// 2^kFineShift positions (into T, with their positions in TP), then each fine
// slab is filled in shared memory and compacted there (k_fine_fill): A_d and
// weight(A_d) are written, and F_{d+1} goes to Fout (cap keys; out_count[d]
// counts them; a run past cap raises bit 0 of *fuse_status).  Then level d+1
// is sized.
static int fill_grouped(const u64 *R, u64 s, u64 m, unsigned nslab, const std::vector<u64> &se,
                        Scratch &sc, u64 *Alev, BuildMeta *meta, int d, int L, double gamma,
                        u64 *Fout, u64 cap, unsigned *fuse_status, unsigned *status,
                        cudaStream_t st) {
  int rc0 = slab_attrs();
  if (rc0 != MPHF_OK) return rc0;
  const u64 fine = (u64)1 << kFineShift;
  auto fine_count = [&](unsigned c) -> unsigned {
    const u64 base = (u64)c << g_slab_shift;
    const u64 range = std::min((u64)1 << g_slab_shift, m - base);
    return (unsigned)((range + fine - 1) >> kFineShift);
  };
  auto fine_cap = [&](unsigned c) -> u64 {
    // keys expected in a whole fine slab: the slab's keys spread over its range
    const u64 base = (u64)c << g_slab_shift;
    const u64 range = std::min((u64)1 << g_slab_shift, m - base);
    const double mean = (double)(se[nslab + c] - se[c]) * (double)std::min(fine, range) /
                        (double)range;
    const u64 cap = (u64)(g_cap_scale * (mean + 8.0 * sqrt(mean) + 64.0));  // scale: tests only
    return (cap + 3) & ~3ull;
  };
  // T / TP hold one slab's keys and positions in either form: fixed-capacity
  // ranges, or the exact ranges of a redo
  u64 need = 0;
  for (unsigned c = 0; c < nslab; c++)
    if (se[nslab + c] > se[c])
      need = std::max(need, std::max((u64)fine_count(c) * fine_cap(c), se[nslab + c] - se[c]));
  if (sc.T.bytes < need * 8) {
    dev_free(sc.T, st);
    int rc = dev_alloc(sc.T, need * 8, st);
    if (rc != MPHF_OK) return rc;
  }
  if (sc.TP.bytes < need * 4) {
    dev_free(sc.TP, st);
    int rc = dev_alloc(sc.TP, need * 4, st);
    if (rc != MPHF_OK) return rc;
  }
  u64 *T = (u64 *)sc.T.p;
  unsigned *TP = (unsigned *)sc.TP.p;
  u64 *cursor = (u64 *)sc.slab.p + kSlabMax, *end = (u64 *)sc.slab.p + 2 * kSlabMax;
  u64 *fstart = (u64 *)sc.slab.p + 3 * kSlabMax;
  std::vector<u64> fse;
  // exact = false: fine ranges of a fixed capacity; true: counted first
  for (int exact = 0; exact < 2; exact++) {
    for (unsigned c = 0; c < nslab; c++) {
      const u64 a = se[c], b = se[nslab + c];
      const u64 base = (u64)c << g_slab_shift;
      const u64 range = std::min((u64)1 << g_slab_shift, m - base);
      if (a == b) {  // no key in the slab: its stretch of A_d is all zero
        MPHF_CUDA(cudaMemsetAsync(Alev + (base >> 6), 0, range / 8, st));
        continue;
      }
      const unsigned nf = fine_count(c);
      if (exact) {
        int rc = group_keys(R + a, b - a, s, m, base, kFineShift, nf, T, TP, (u64 *)sc.slab.p,
                            status, fse, st);
        if (rc != MPHF_OK) return rc;
        MPHF_CUDA(cudaMemcpyAsync(fstart, fse.data(), nf * 8, cudaMemcpyHostToDevice, st));
      } else {
        {
          LaunchScope lr("slab_ranges", st);
          k_fine_ranges<<<(nf + 255) / 256, 256, 0, st>>>(cursor, end, fstart, nf, fine_cap(c));
        }
        launch_slab_scatter(R + a, b - a, s, m, base, kFineShift, nf, cursor, end, T, TP, status,
                            st);
      }
      {
        LaunchScope ls("fine_fill", st);
        k_fine_fill<<<nf, kFineThreads, kFineSmem, st>>>(T, TP, fstart, cursor, end, base,
                                                         base + range, Alev, &meta->weight[d],
                                                         Fout, cap, &meta->out_count[d],
                                                         fuse_status, s, m);
      }
      MPHF_CUDA(cudaGetLastError());
    }
    if (exact) break;
    // a fixed-capacity range overflowed (duplicate-heavy input): redo the
    // level, fill and compaction, from its grouped keys
    unsigned flag = 0;
    MPHF_CUDA(cudaMemcpyAsync(&flag, status, 4, cudaMemcpyDeviceToHost, st));
    MPHF_CUDA(cudaStreamSynchronize(st));
    if (!flag) break;
    MPHF_CUDA(cudaMemsetAsync(status, 0, 4, st));
    MPHF_CUDA(cudaMemsetAsync(&meta->weight[d], 0, 8, st));
    MPHF_CUDA(cudaMemsetAsync(&meta->out_count[d], 0, 8, st));
    MPHF_CUDA(cudaMemsetAsync(fuse_status, 0, 4, st));
  }
  {
    LaunchScope ls("extract", st);
    k_level_done<<<1, 1, 0, st>>>(meta, d, L, gamma);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

static void release_handle(mphf_t *h, cudaStream_t s) {
  if (!h) return;
  dev_free(h->S, s);
  dev_free(h->SB, s);
  dev_free(h->fb, s);
  handle_delete(h);
}

static int launch_fill0(const u64 *keys, u64 n, u64 s0, u64 m0, u64 *AC, cudaStream_t st) {
  unsigned maxb = (unsigned)sm_count() * 8;
  if (((uintptr_t)keys & 15) == 0) {
    u64 npairs = n >> 1;
    if (npairs) {
      unsigned g = grid_for(npairs, kFillThreads * kFillUnroll, maxb);
      LaunchScope ls("fill", st);
      k_fill_vec<<<g, kFillThreads, 0, st>>>(reinterpret_cast<const uint4 *>(keys), npairs, s0,
                                              m0, AC);
    }
    if (n & 1) {
      LaunchScope ls("fill", st);
      k_fill_scalar<<<1, kFillThreads, 0, st>>>(keys + (n - 1), 1, s0, m0, AC);
    }
  } else {
    unsigned g = grid_for(n, kFillThreads * 4, maxb);
    LaunchScope ls("fill", st);
    k_fill_scalar<<<g, kFillThreads, 0, st>>>(keys, n, s0, m0, AC);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

static int launch_extract(u64 *AC, u64 m_bound, u64 *A0, u64 *arena, BuildMeta *meta, int d,
                          int L, double gamma, cudaStream_t st) {
  unsigned g = grid_for(m_bound / 64, kExtractThreads * 4, (unsigned)sm_count() * 8);
  LaunchScope ls("extract", st);
  k_extract<<<g, kExtractThreads, 0, st>>>(AC, A0, arena, meta, d, L, gamma);
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

static int launch_compact(const u64 *F, u64 n_bound, u64 *Fout, u64 cap, const u64 *A0,
                          const u64 *arena, u64 *ACnext, BuildMeta *meta, int d, u64 s_d,
                          u64 s_next, int do_fill, cudaStream_t st, u64 n_in = ~0ull) {
  unsigned g = grid_for(n_bound, kCompactTile, (unsigned)sm_count() * 4);
  LaunchScope ls("compact", st);
  if (((uintptr_t)F & 15) == 0)
    k_compact<true><<<g, kCompactThreads, 0, st>>>(F, n_in, Fout, A0, arena, ACnext, meta, d,
                                                   s_d, s_next, do_fill, cap);
  else
    k_compact<false><<<g, kCompactThreads, 0, st>>>(F, n_in, Fout, A0, arena, ACnext, meta, d,
                                                    s_d, s_next, do_fill, cap);
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

static int read_meta(const DevBuf &meta, BuildMeta *hm, cudaStream_t st) {
  MPHF_CUDA(cudaMemcpyAsync(hm, meta.p, sizeof(BuildMeta), cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaStreamSynchronize(st));
  return MPHF_OK;
}

static int read_u64(const u64 *d_ptr, u64 *out, cudaStream_t st) {
  MPHF_CUDA(cudaMemcpyAsync(out, d_ptr, sizeof(u64), cudaMemcpyDeviceToHost, st));
  MPHF_CUDA(cudaStreamSynchronize(st));
  return MPHF_OK;
}

// Unbucketed construction: L2 atomics for ArrayFill, one host round trip per
// level.  Used when a bound of the bucketed path (fastbuild.cu) is exceeded.
static int robust_build(const u64 *keys, u64 N, double gamma, uint32_t L, u64 seed,
                        cudaStream_t st, mphf_t *h) {
  int rc = MPHF_OK;
  Scratch sc;
  BuildMeta hm;
  memset(&hm, 0, sizeof(hm));
  const u64 m0 = level_bits(N, gamma);
  hm.n[0] = N;
  hm.m[0] = m0;
  hm.off[0] = 0;
  u64 n1 = 0, last_level = 0, n_fb = 0;
  u64 *Ffb = nullptr;
  BuildMeta *meta = nullptr;
  unsigned int *dflag = nullptr;
  unsigned nslab0 = 0;
  unsigned *slab_status = nullptr;
  unsigned *fuse_status = nullptr;
  u64 ac_cap = 0;       // bytes of each hit/collision array
  std::vector<u64> se;  // slab ranges of the grouped keys

#define TRY(x)                  \
  do {                          \
    rc = (x);                   \
    if (rc != MPHF_OK) goto fail; \
  } while (0)

  TRY(dev_alloc(sc.meta, sizeof(BuildMeta), st));
  meta = (BuildMeta *)sc.meta.p;
  TRY(dev_alloc(sc.A0, m0 / 64 * 8, st));
  TRY(dev_alloc(sc.dupflag, 32, st));  // dup flag, rank total, slab and F1 overflow
  dflag = (unsigned int *)sc.dupflag.p;
  if ((rc = cudaMemcpyAsync(meta, &hm, sizeof(hm), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    rc = cuda_fail((cudaError_t)rc, "cudaMemcpyAsync(meta)");
    goto fail;
  }
  if (cudaMemsetAsync(dflag, 0, 32, st) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    goto fail;
  }
  // Levels too large for L2 are grouped by slab first (levels only shrink, so
  // they are a prefix of the levels).  R holds the grouped keys; without room
  // for it the keys stay in their order.
  nslab0 = slab_count_for(m0);
  if (nslab0) {
    if (dev_alloc(sc.R, grouped_room(N, m0, nslab0) * 8, st) != MPHF_OK ||
        dev_alloc(sc.slab, 4 * kSlabMax * 8, st) != MPHF_OK) {
      cudaGetLastError();
      dev_free(sc.R, st);
      dev_free(sc.slab, st);
      nslab0 = 0;
    }
  }
  // The hit/collision arrays (2 bits a position) serve the ungrouped levels
  // only.  Once level 0 is grouped, a level is ungrouped only when its array
  // is at most g_slab_min_ac bytes (or it is the fallback), so that bounds
  // both arrays.  The extraction zeroes an array behind it: one memset here.
  ac_cap = nslab0 ? std::min(m0 / 32 * 8, ((g_slab_min_ac + 15) & ~(u64)15) + 16) : m0 / 32 * 8;
  TRY(dev_alloc(sc.AC0, ac_cap, st));
  if (cudaMemsetAsync(sc.AC0.p, 0, sc.AC0.bytes, st) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    goto fail;
  }
  slab_status = (unsigned *)((u64 *)sc.dupflag.p + 2);
  fuse_status = (unsigned *)((u64 *)sc.dupflag.p + 3);
  if (nslab0) {
    // Level 0 grouped: fill and compaction run together, F_1 going to F1,
    // allocated for a bound on |F_1| (8 standard deviations above its mean).
    const double mean = (double)N * (1.0 - pow(1.0 - 1.0 / (double)m0, (double)N - 1.0));
    u64 n1_hi = (u64)(mean + 8.0 * sqrt((double)N) + 1024.0);
    if (n1_hi > N) n1_hi = N;
    TRY(dev_alloc(sc.F1, n1_hi * 8, st));
    TRY(group_level(keys, N, h->s[0], m0, nslab0, (u64 *)sc.R.p, (u64 *)sc.slab.p, slab_status,
                    se, st));
    TRY(fill_grouped((const u64 *)sc.R.p, h->s[0], m0, nslab0, se, sc, (u64 *)sc.A0.p, meta, 0,
                     (int)L, gamma, (u64 *)sc.F1.p, n1_hi, fuse_status, slab_status, st));
    TRY(read_u64(&meta->n[1], &n1, st));
    u64 fflag = 0;
    TRY(read_u64((const u64 *)fuse_status, &fflag, st));
    if ((unsigned)fflag) {
      // |F_1| above the bound (thousands of equal keys): F1 at its exact size
      // and the compaction of level 0 again, from the grouped keys in R
      dev_free(sc.F1, st);
      TRY(dev_alloc(sc.F1, n1 * 8, st));
      if (cudaMemsetAsync(&meta->out_count[0], 0, 8, st) != cudaSuccess ||
          cudaMemsetAsync(fuse_status, 0, 4, st) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
        goto fail;
      }
      for (unsigned c = 0; c < nslab0; c++)  // slab by slab: the ranges of R have gaps
        if (se[nslab0 + c] > se[c])
          TRY(launch_compact((const u64 *)sc.R.p + se[c], se[nslab0 + c] - se[c],
                             (u64 *)sc.F1.p, n1, (const u64 *)sc.A0.p, nullptr, nullptr, meta, 0,
                             h->s[0], 0, 0, st, se[nslab0 + c] - se[c]));
    }
  } else {
    TRY(launch_fill0(keys, N, h->s[0], m0, (u64 *)sc.AC0.p, st));
    TRY(launch_extract((u64 *)sc.AC0.p, m0, (u64 *)sc.A0.p, nullptr, meta, 0, (int)L, gamma,
                       st));
    TRY(read_u64(&meta->n[1], &n1, st));
  }

  if (n1 > 0) {
    // Every later level holds at most n1 keys, so these bounds are exact worst cases.
    const u64 m1 = level_bits(n1, gamma);
    if (!sc.F1.p) TRY(dev_alloc(sc.F1, n1 * 8, st));
    // with grouped levels, R (N keys) is the second buffer of the level loop
    if (L > 1 && !nslab0) TRY(dev_alloc(sc.F2, n1 * 8, st));
    if (L > 1) {
      TRY(dev_alloc(sc.AC1, std::min(m1 / 32 * 8, ac_cap), st));
      TRY(dev_alloc(sc.arena, (u64)(L - 1) * (m1 / 64) * 8, st));
      if (cudaMemsetAsync(sc.AC1.p, 0, sc.AC1.bytes, st) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
        goto fail;
      }
    }
  }

  {
    // Level loop.  An ungrouped level d is compacted here (with level d+1's
    // fill when that level is ungrouped too); a grouped level was compacted
    // by its fill, F_{d+1} already in F1.  Then level d+1: grouped (group,
    // fill and compact) or ungrouped (fill unless done, extract).
    u64 n_next = n1;  // |F_{d+1}|
    u64 off_next = 0;
    const u64 *Fin = keys;          // keys of level d, for a compaction here
    bool compacted = nslab0 != 0;   // F_{d+1} written by level d's fill
    u64 *F1 = (u64 *)sc.F1.p;
    int d = 0;
    for (;;) {
      if (n_next == 0) {
        last_level = d;
        break;
      }
      const bool to_fallback = (uint32_t)(d + 1) == L;
      const u64 m_next = to_fallback ? 0 : level_bits(n_next, gamma);
      unsigned nslab = (nslab0 && !to_fallback) ? slab_count_for(m_next) : 0u;
      u64 *ACnext = ((d + 1) & 1) ? (u64 *)sc.AC1.p : (u64 *)sc.AC0.p;
      u64 *Fnext;  // F_{d+1}
      bool filled_next = false;
      if (compacted) {
        Fnext = F1;
      } else {
        // F_{d+1} goes to the buffer F_d is not read from: F1 and F2, or F1 and R
        u64 *other = nslab0 ? (u64 *)sc.R.p : (u64 *)sc.F2.p;
        Fnext = (Fin == F1) ? other : F1;
        if (Fnext != F1) nslab = 0;  // grouped levels are a prefix: cannot happen
        const int fuse = (to_fallback || nslab) ? 0 : 1;
        TRY(launch_compact(Fin, d == 0 ? N : n1, Fnext, n1, (const u64 *)sc.A0.p,
                           (const u64 *)sc.arena.p, fuse ? ACnext : nullptr, meta, d, h->s[d],
                           fuse ? h->s[d + 1] : 0, fuse, st));
        filled_next = fuse != 0;
      }
      if (to_fallback) {
        last_level = d;
        Ffb = Fnext;
        n_fb = n_next;
        break;
      }
      if (nslab) {
        // level d+1 grouped: F_{d+1} into R by slab, then fill and compaction,
        // F_{d+2} written back into F1 (read entirely by the grouping)
        if (grouped_room(n_next, m_next, nslab) * 8 > sc.R.bytes) {  // cannot happen: n shrinks
          rc = MPHF_EINTERNAL;
          goto fail;
        }
        TRY(group_level(Fnext, n_next, h->s[d + 1], m_next, nslab, (u64 *)sc.R.p,
                        (u64 *)sc.slab.p, slab_status, se, st));
        TRY(read_u64(&meta->off[d + 1], &off_next, st));
        TRY(fill_grouped((const u64 *)sc.R.p, h->s[d + 1], m_next, nslab, se, sc,
                         (u64 *)sc.arena.p + ((off_next - m0) >> 6), meta, d + 1, (int)L, gamma,
                         F1, n1, fuse_status, slab_status, st));
        compacted = true;
      } else {
        if (!filled_next) TRY(launch_fill0(Fnext, n_next, h->s[d + 1], m_next, ACnext, st));
        TRY(launch_extract(ACnext, level_bits(n1, gamma), (u64 *)sc.A0.p, (u64 *)sc.arena.p,
                           meta, d + 1, (int)L, gamma, st));
        Fin = Fnext;
        compacted = false;
      }
      TRY(read_u64(&meta->n[d + 2], &n_next, st));
      d++;
    }
  }

  TRY(read_meta(sc.meta, &hm, st));
  if (hm.status) {
    rc = (int)hm.status;
    goto fail;
  }
  h->L_used = (uint32_t)last_level + 1;
  for (uint32_t d = 0; d < h->L_used; d++) {
    h->n[d] = hm.n[d];
    h->m[d] = hm.m[d];
    h->off[d] = hm.off[d];
    // every compaction must have written exactly |F_{d+1}| keys
    if (d + 1 < h->L_used || n_fb) {
      if (hm.out_count[d] != hm.n[d + 1]) {
        rc = MPHF_EINTERNAL;
        goto fail;
      }
    }
  }
  h->n[h->L_used] = n_fb;
  h->M = hm.off[h->L_used - 1] + hm.m[h->L_used - 1];
  h->n_rank = (h->M + MPHF_RANK_BLOCK - 1) / MPHF_RANK_BLOCK;
  h->n_fb = n_fb;

  // Final A = A_0 || arena, stored as sectors with their ranks.
  TRY(make_sectors(h, ASrc{(const u64 *)sc.A0.p, m0 / 64, (const u64 *)sc.arena.p, h->M / 64},
                   (u64 *)sc.dupflag.p + 1, st));

  // Fallback (Sec. 3.5): sorted leftover keys; equal neighbours mean duplicates.
  if (n_fb) {
    TRY(sort_fallback(Ffb, n_fb, dflag, st));
    TRY(dev_alloc(h->fb, n_fb * 8, st));
    if (cudaMemcpyAsync(h->fb.p, Ffb, n_fb * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "cudaMemcpyAsync(fb)");
      goto fail;
    }
  }
  {
    u64 flags[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(flags, sc.dupflag.p, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "dup flag");
      goto fail;
    }
    if ((unsigned)flags[2] || (unsigned)flags[3]) {  // a slab range or F1 overflowed: cannot happen
      rc = MPHF_EINTERNAL;
      goto fail;
    }
    if ((unsigned)flags[0]) {
      rc = MPHF_EDUPLICATE;
      goto fail;
    }
    // rank total must equal the number of placed keys
    if (flags[1] != N - n_fb) {
      rc = MPHF_EINTERNAL;
      goto fail;
    }
  }
  sc.release(st);
  return MPHF_OK;

fail:
  cudaGetLastError();
  sc.release(st);
  dev_free(h->S, st);
  dev_free(h->SB, st);
  dev_free(h->fb, st);
  cudaStreamSynchronize(st);
  return rc;
#undef TRY
}

int g_build_path = 0;  // 0: bucketed, unbucketed on overflow; 1: unbucketed only

// feed (optional): the keys are still arriving from the host; fast_build
// consumes them chunk by chunk, every other step waits for all of them.
static int build_impl(const u64 *keys, u64 N, double gamma, uint32_t L, u64 seed, cudaStream_t st,
                      mphf_t **out, KeyFeed *feed = nullptr) {
  mphf_t *h = handle_new();
  if (!h) return MPHF_ENOMEM;
  cudaGetDevice(&h->device);
  h->N = N;
  h->gamma = gamma;
  h->L = L;
  h->seed = seed;
  for (uint32_t d = 0; d < L; d++) h->s[d] = level_seed(seed, d);
  if (N == 0) {
    *out = h;
    return MPHF_OK;
  }
  int rc = MPHF_OK;
  bool redo = true;
  if (g_build_path == 0) {
    rc = fast_build(keys, N, gamma, L, seed, st, h, &redo, feed);
    if (rc == MPHF_OK && feed) rc = feed->ensure(N, st);
    if (rc != MPHF_OK) {
      release_handle(h, st);
      cudaStreamSynchronize(st);
      return rc;
    }
    h->path = 1;
  }
  if (redo) {
    if (feed) rc = feed->ensure(N, st);
    if (rc == MPHF_OK) rc = robust_build(keys, N, gamma, L, seed, st, h);
    if (rc != MPHF_OK) {
      release_handle(h, st);
      cudaStreamSynchronize(st);
      return rc;
    }
    h->path = 2;
  }
  *out = h;
  return MPHF_OK;
}

int build_single(const u64 *keys, u64 N, double gamma, uint32_t L, u64 seed, cudaStream_t st,
                 mphf_t **out) {
  return build_impl(keys, N, gamma, L, seed, st, out);
}

}  // namespace bbh

using namespace bbh;

extern "C" int mphf_build(const uint64_t *d_keys, uint64_t n, double gamma, uint32_t levels,
                          uint64_t seed, void *stream, mphf_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (!(gamma >= 1.0) || isinf(gamma) || levels < 1 || levels > MPHF_MAX_LEVELS ||
      (n > 0 && !d_keys) || ((uintptr_t)d_keys & 7))
    return MPHF_EINVAL;
  return build_impl((const u64 *)d_keys, n, gamma, levels, seed, (cudaStream_t)stream, out);
}

extern "C" int mphf_build_host(const uint64_t *h_keys, uint64_t n, double gamma, uint32_t levels,
                               uint64_t seed, void *stream, mphf_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (!(gamma >= 1.0) || isinf(gamma) || levels < 1 || levels > MPHF_MAX_LEVELS ||
      (n > 0 && !h_keys))
    return MPHF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf kb;
  int rc = dev_alloc(kb, n * 8, st);
  if (rc != MPHF_OK) return rc;
  const u64 chunk = feed_chunk(n);
  if (!chunk) {
    if (n) {
      cudaError_t e = cudaMemcpyAsync(kb.p, h_keys, n * 8, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) {
        dev_free(kb, st);
        return cuda_fail(e, "cudaMemcpyAsync(H2D keys)");
      }
    }
    rc = build_impl((const u64 *)kb.p, n, gamma, levels, seed, st, out);
    dev_free(kb, st);
    return rc;
  }
  // Large sets: the level-0 partition runs chunk by chunk behind the copy.
  KeyFeed f;
  f.h = (const u64 *)h_keys;
  f.d = (u64 *)kb.p;
  f.n = n;
  f.chunk = chunk;
  SideSet ss;
  rc = side_set(1, &ss);
  if (rc != MPHF_OK) {
    dev_free(kb, st);
    return rc;
  }
  f.cs = ss.s[0];
  f.ev = ss.ev[0];
  // the copies must not start before the buffer's allocation in st's order
  cudaError_t e = cudaEventRecord(f.ev, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(f.cs, f.ev, 0);
  if (e == cudaSuccess) {
    rc = build_impl((const u64 *)kb.p, n, gamma, levels, seed, st, out, &f);
    // every copy ever enqueued is ordered before the buffer's release
    cudaEventRecord(f.ev, f.cs);
    cudaStreamWaitEvent(st, f.ev, 0);
  } else {
    rc = cuda_fail(e, "mphf_build_host (copy stream)");
    cudaStreamSynchronize(f.cs);
  }
  dev_free(kb, st);
  return rc;
}

// Build and query in one call, with every transfer on the host link kept
// busy: the keys stream in chunk by chunk behind the level-0 partition (as in
// mphf_build_host), the queries follow them on the same copy stream while
// the remaining levels are built, and once the function exists the lookup of
// query chunk c runs as soon as that chunk has landed while the indices of
// chunk c-1 stream back on a third stream.
extern "C" int mphf_build_lookup_host(const uint64_t *h_keys, uint64_t n, double gamma,
                                      uint32_t levels, uint64_t seed, const uint64_t *h_queries,
                                      uint64_t nq, uint64_t *h_out, void *stream, mphf_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (!(gamma >= 1.0) || isinf(gamma) || levels < 1 || levels > MPHF_MAX_LEVELS ||
      (n > 0 && !h_keys) || (nq > 0 && (!h_queries || !h_out)))
    return MPHF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const u64 qchunk = nq ? (feed_chunk(nq) ? feed_chunk(nq) : nq) : 1;
  const u64 nqc = nq ? (nq + qchunk - 1) / qchunk : 0;
  DevBuf kb, qb, ob;
  KeyFeed f;
  SideSet ss;
  cudaStream_t co = nullptr;
  cudaEvent_t ev_k = nullptr;
  cudaError_t e = cudaSuccess;
  int rc = side_set((size_t)nqc + 2, &ss);
  if (rc != MPHF_OK) return rc;
  rc = dev_alloc(kb, n * 8, st);
  if (rc == MPHF_OK) rc = dev_alloc(qb, nq * 8, st);
  if (rc == MPHF_OK) rc = dev_alloc(ob, nq * 8, st);
  f.cs = ss.s[0];
  co = ss.s[1];
  f.ev = ss.ev[0];
  ev_k = ss.ev[1];
  if (rc == MPHF_OK) {
    f.h = (const u64 *)h_keys;
    f.d = (u64 *)kb.p;
    f.n = n;
    f.chunk = feed_chunk(n);
    f.hq = (const u64 *)h_queries;
    f.dq = (u64 *)qb.p;
    f.nq = nq;
    f.qchunk = qchunk;
    f.qev = ss.ev + 2;
    // the copies must not start before the buffers' allocation in st's order
    e = cudaEventRecord(f.ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(f.cs, f.ev, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "mphf_build_lookup_host (streams)");
  }
  if (rc == MPHF_OK) rc = build_impl((const u64 *)kb.p, n, gamma, levels, seed, st, out, &f);
  if (rc == MPHF_OK && !f.q_issued) rc = f.issue_queries();
  if (rc == MPHF_OK && nq) {
    // chunk c: wait for its copy, look it up; its indices leave on co after
    // the lookup of chunk c+1 is queued
    u64 prev0 = 0, prevn = 0, i = 0;
    u64 *dq = (u64 *)qb.p, *dout = (u64 *)ob.p;
    for (u64 c0 = 0; c0 < nq && rc == MPHF_OK && e == cudaSuccess; c0 += qchunk, i++) {
      const u64 cn = nq - c0 < qchunk ? nq - c0 : qchunk;
      e = cudaStreamWaitEvent(st, f.qev[i], 0);
      if (e != cudaSuccess) break;
      rc = mphf_lookup(*out, (const uint64_t *)(dq + c0), cn, (uint64_t *)(dout + c0), stream);
      if (rc != MPHF_OK) break;
      e = cudaEventRecord(ev_k, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(co, ev_k, 0);
      if (e == cudaSuccess && prevn)
        e = cudaMemcpyAsync(h_out + prev0, dout + prev0, prevn * 8, cudaMemcpyDeviceToHost, co);
      prev0 = c0;
      prevn = cn;
    }
    if (e == cudaSuccess && rc == MPHF_OK && prevn)
      e = cudaMemcpyAsync(h_out + prev0, dout + prev0, prevn * 8, cudaMemcpyDeviceToHost, co);
    if (e != cudaSuccess && rc == MPHF_OK) rc = cuda_fail(e, "mphf_build_lookup_host");
  }
  // everything enqueued on the side streams is ordered before the frees
  cudaEventRecord(f.ev, f.cs);
  cudaStreamWaitEvent(st, f.ev, 0);
  cudaEventRecord(ev_k, co);
  cudaStreamWaitEvent(st, ev_k, 0);
  dev_free(ob, st);
  dev_free(qb, st);
  dev_free(kb, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (rc == MPHF_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "mphf_build_lookup_host");
  if (rc != MPHF_OK && *out) {
    mphf_free(*out);
    *out = nullptr;
  }
  return rc;
}

extern "C" int mphf_debug_config(int path, double cap_scale) {
  if (path < 0 || path > 1 || !(cap_scale > 0.0) || cap_scale > 16.0) return MPHF_EINVAL;
  bbh::g_build_path = path;
  bbh::g_cap_scale = cap_scale;
  return MPHF_OK;
}

extern "C" int mphf_build_path(const mphf_t *h) { return h ? h->path : 0; }

extern "C" int mphf_debug_slabs(uint32_t shift, uint64_t min_ac_bytes) {
  if (shift < 6 || shift > 29) return MPHF_EINVAL;  // at most 2048 fine slabs of 2^18 a slab
  bbh::g_slab_shift = shift;
  bbh::g_slab_min_ac = min_ac_bytes;
  return MPHF_OK;
}
