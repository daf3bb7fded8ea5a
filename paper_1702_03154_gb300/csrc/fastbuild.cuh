// fastbuild.cuh -- device state of the bucketed construction path (fastbuild.cu)
// and of the single-CTA level loop shared with the batched builder.
#pragma once

#include "common.cuh"

namespace bbh {

// Where the keys of level d live.
enum LevelMode : unsigned {
  LM_NONE = 0,
  LM_BUCKETED = 1,  // in position-range buckets of arena (d & 1)
  LM_FLAT = 2,      // contiguous in the flat buffer (input of the tail, or the fallback if d == L)
  LM_DONE = 3       // no keys left: the function ends at level d - 1
};

// Status bits raised on the device.
enum : unsigned {
  ST_OVERFLOW = 1u,   // a bucket / buffer bound was exceeded: rebuild with the unbucketed path
  ST_DUPLICATE = 2u,  // equal keys in the fallback
  ST_INTERNAL = 4u,   // a consistency check failed
  ST_TIMEOUT = 8u
};

struct FLevel {
  u64 n, m, off;   // |F_d|, |A_d| bits, first bit of A_d in A
  u64 P, B, cap;   // positions per bucket (multiple of 64), buckets, key capacity per bucket
  u64 weight;      // ones of A_d
  unsigned mode;
  unsigned done;   // fill blocks finished
};

struct FastMeta {
  FLevel lv[MPHF_MAX_LEVELS + 1];
  u64 seen[MPHF_MAX_LEVELS + 1];  // keys found in the buckets of level d (consistency check)
  u64 n_flat;            // keys appended to the flat buffer
  u64 n_fb;              // fallback keys
  u64 rank_total;        // ones of A, from the rank table
  unsigned status;
  unsigned levels_used;
  unsigned tail_done;    // 1 once the level loop has finished; 2 if the fallback is left unsorted
  unsigned dup;          // equal neighbours in a fallback sorted outside the tail
};

// Build-wide constants of the bucketed path.
struct FastCfg {
  double gamma;
  uint32_t L;
  u64 seed;
  u64 *X, *Y;           // bucket arenas: levels with even / odd d
  unsigned *XP, *YP;    // in-bucket position of each key of X / Y
  u64 capX, capY;       // their capacities in keys
  u64 *cntX, *cntY;     // per-bucket key counts
  u64 Bmax;             // capacity of the count arrays
  u64 *flat;            // flat buffer (tail input / fallback)
  u64 flat_cap;
  u64 *A0;              // A_0 (m_0 bits)
  u64 *arena;           // A_1, A_2, ... back to back
  u64 m0;
  u64 arena_words;
  u64 T;                // levels with at most T keys run in the single-CTA tail
  u64 Pmax, Pmin, Btarget;
  double cap_scale;     // bucket capacity multiplier (1 in production; < 1 only in tests)
  unsigned *upre;       // [Bmax + 1] compaction units (kIn-entry slices) before each bucket
  u64 nbcap;            // compaction: capacity of its per-destination-bucket arrays
};

__host__ __device__ inline u64 ceil_div(u64 a, u64 b) { return (a + b - 1) / b; }

static constexpr int kTT = 512;            // threads of partition / compaction / fill CTAs
static constexpr int kKPT = 8;             // keys per thread per tile
static constexpr int kTile = kTT * kKPT;   // 4096 keys
static constexpr int kInPT = 4;            // compaction: entries per thread per input unit
static constexpr int kIn = kTT * kInPT;    // 2048 entries per compaction unit
static constexpr u64 kPmax = 256 * 1024;   // positions per bucket at most (64 KB of bits)
static constexpr int kTailThreads = 1024;
static constexpr u64 kTailMaxKeys = 16384;
static constexpr u64 kBmax = 2048;

// ---------------------------------------------------------------------------
// Level sizing (device side, by the last block of a fill).
// ---------------------------------------------------------------------------
__host__ __device__ inline unsigned ilog2_u64(u64 v) {
  unsigned r = 0;
  while ((v >> r) > 1) r++;
  return r;
}

__host__ __device__ inline void size_bucketed(FLevel &lv, u64 n, double gamma, u64 Pmin, u64 Pmax,
                                              u64 Btarget, double cap_scale) {
  lv.n = n;
  lv.m = level_bits(n, gamma);
  u64 want = ceil_div(lv.m, Btarget);
  u64 P = Pmin;
  while (P < want && P < Pmax) P <<= 1;
  lv.P = P;
  lv.B = ceil_div(lv.m, P);
  double mean = (double)n * (double)P / (double)lv.m;
  u64 cap = (u64)(cap_scale * (mean + 8.0 * sqrt(mean) + 64.0));
  lv.cap = (cap + 3) & ~3ull;  // multiple of 4: every bucket starts 16-byte aligned
}

// ---------------------------------------------------------------------------
// Block-wide helpers (kTT threads).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ u64 block_sum(u64 v, u64 *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  u64 s = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT / 32; i++) s += red[i];
    red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// Exclusive scan of NT values (one per thread); returns the prefix, *total = sum.
template <int NT>
__device__ __forceinline__ unsigned block_scan_u32(unsigned v, unsigned *red, unsigned *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned w = lane < NT / 32 ? red[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) red[lane] = w;
  }
  __syncthreads();
  unsigned before = warp ? red[warp - 1] : 0u;
  *total = red[NT / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// The same scan with two barriers instead of four, for callers that put a
// block barrier between one call's reads of red and the next call's writes.
template <int NT>
__device__ __forceinline__ unsigned block_scan_u32_fenced(unsigned v, unsigned *red,
                                                          unsigned *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned w = lane < NT / 32 ? red[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) red[lane] = w;
  }
  __syncthreads();
  *total = red[NT / 32 - 1];
  return (warp ? red[warp - 1] : 0u) + x - v;
}

// Shared memory of the multisplit writer.
struct SplitSmem {
  unsigned *cnt;         // [nb] entries per destination in this tile (zero between calls)
  unsigned short *start; // [nb] multisplit_write_one: local index of each destination's
                         // first entry; multisplit_write: its local limit
  u64 *run;              // [nb] multisplit_write_one: (local limit << 44) | (arena index of
                         // local entry 0, mod 2^44); multisplit_write: that arena index
  u64 *sorted;           // [kTile] keys in destination order (also the survivor staging area)
  unsigned *stag;        // [kTile] (destination << 20) | in-bucket position
  unsigned *red;         // [kTT / 32 + 2]
};

// Destination of a multisplit: where destination bucket i of the tile lives.
struct DestRun {
  u64 *counter;  // keys already in the bucket (atomically advanced)
  u64 base;      // arena index of the bucket's slot 0
  u64 cap;       // slots in the bucket
};

// Plain layout: bucket i at arena[i * cap], counters gcnt[i].
struct UniformDest {
  u64 *gcnt;
  u64 cap;
  __device__ __forceinline__ DestRun operator()(unsigned i) const {
    return DestRun{gcnt + i, (u64)i * cap, cap};
  }
};

static constexpr unsigned kRunShift = 44;  // arena indices below 2^44
static constexpr u64 kRunMask = (1ull << kRunShift) - 1;

// Write the valid entries of a tile into their destination buckets: key to
// arena[base_b + slot] and (WITH_POS) its in-bucket position lp (< 2^20) to
// parena[base_b + slot], where dest(b) gives the bucket's counter, base and
// capacity.  Slots are reserved with one atomicAdd per non-empty destination;
// the entries of one destination leave as one contiguous run.  Entries past a
// bucket's capacity are dropped and ST_OVERFLOW is raised.  sm.cnt[0, nb) is
// zero on entry and on return (split_clear before a kernel's first call).
//
// Up to kTT destinations (one per thread): four block barriers a call (after
// the rank atomics, in the scan, before the scatter into destination order,
// before the write-out), the reservation atomics in flight during the
// scatter, and no barrier at the end: the owner zeroes a destination's count
// as soon as the scan has read it, and the next call writes `start`,
// `sorted`, `stag`, `run` and `red` only after barriers that every thread
// reaches after its write-out.  A caller that itself writes `sorted` (a
// survivor stage) right after the call puts a block barrier in between.
template <bool WITH_POS, class Dest>
__device__ __forceinline__ void multisplit_write_one(const u64 (&x)[kKPT], const unsigned (&lp)[kKPT],
                                                     const unsigned (&dst)[kKPT], const bool (&ok)[kKPT],
                                                     unsigned nb, const SplitSmem &sm,
                                                     u64 *__restrict__ arena,
                                                     unsigned *__restrict__ parena, const Dest &dest,
                                                     unsigned *__restrict__ status) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned rk[kKPT], tag[kKPT];
#pragma unroll
  for (int k = 0; k < kKPT; k++) {
    tag[k] = (dst[k] << 20) | lp[k];
    rk[k] = ok[k] ? atomicAdd(&sm.cnt[dst[k]], 1u) : 0u;
  }
  __syncthreads();
  const unsigned i0 = threadIdx.x;  // the destination this thread owns
  unsigned c = 0;
  if (i0 < nb) {
    c = sm.cnt[i0];
    sm.cnt[i0] = 0;
  }
  // exclusive scan of the counts: each warp scans its own, lane 31 posts the
  // warp's total, and every warp scans the posted totals itself
  unsigned incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) sm.red[warp] = incl;
  __syncthreads();
  unsigned wv = lane < kTT / 32 ? sm.red[lane] : 0u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, wv, o);
    if (lane >= (unsigned)o) wv += y;
  }
  const unsigned wbefore = __shfl_sync(0xffffffffu, wv, (warp + 31) & 31);
  const unsigned total = __shfl_sync(0xffffffffu, wv, kTT / 32 - 1);
  const unsigned pre = (warp ? wbefore : 0u) + incl - c;
  const u64 b0 = c ? atomicAdd(dest(i0).counter, (u64)c) : 0;  // waited for after the scatter
  if (i0 < nb) sm.start[i0] = (unsigned short)pre;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kKPT; k++)
    if (ok[k]) {
      const unsigned pos = sm.start[tag[k] >> 20] + rk[k];
      sm.sorted[pos] = x[k];
      sm.stag[pos] = tag[k];
    }
  // the write-out's limit and arena index of this thread's destination
  if (c) {
    const DestRun r = dest(i0);
    const u64 room = b0 < r.cap ? r.cap - b0 : 0;
    const unsigned lim = pre + (unsigned)(room < c ? room : c);
    sm.run[i0] = ((u64)lim << kRunShift) | ((r.base + b0 - pre) & kRunMask);
  }
  __syncthreads();
  // write-out, four entries a thread at a time: a group's loads are issued
  // before its stores
#pragma unroll
  for (int k0 = 0; k0 < kKPT; k0 += 4) {
    unsigned tg[4];
    u64 v[4], rr[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const unsigned i = threadIdx.x + (unsigned)(k0 + u) * kTT;
      tg[u] = 0;
      v[u] = 0;
      if (i < total) {
        tg[u] = sm.stag[i];
        v[u] = sm.sorted[i];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const unsigned i = threadIdx.x + (unsigned)(k0 + u) * kTT;
      rr[u] = i < total ? sm.run[tg[u] >> 20] : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const unsigned i = threadIdx.x + (unsigned)(k0 + u) * kTT;
      if (i < total) {
        if (i < (unsigned)(rr[u] >> kRunShift)) {
          const u64 j = (rr[u] + i) & kRunMask;
          arena[j] = v[u];
          if (WITH_POS) parena[j] = tg[u] & 0xfffffu;
        } else {
          atomicOr(status, ST_OVERFLOW);
        }
      }
    }
  }
}

// Any number of destinations up to kBmax: each thread owns up to kBmax / kTT
// consecutive ones and issues their reservations together.  Here `start`
// holds each destination's local limit and `run` the arena index of its local
// entry 0; the counts hold the local starts until the write-out, which clears
// them behind a final barrier.
template <bool WITH_POS, class Dest>
__device__ __forceinline__ void multisplit_write(const u64 (&x)[kKPT], const unsigned (&lp)[kKPT],
                                                 const unsigned (&dst)[kKPT], const bool (&ok)[kKPT],
                                                 unsigned nb, const SplitSmem &sm, u64 *__restrict__ arena,
                                                 unsigned *__restrict__ parena, const Dest &dest,
                                                 unsigned *__restrict__ status) {
  constexpr unsigned kPer = (unsigned)(kBmax / kTT);
  static_assert(kBmax % kTT == 0, "destinations per thread");
  unsigned rk[kKPT];
#pragma unroll
  for (int k = 0; k < kKPT; k++) rk[k] = ok[k] ? atomicAdd(&sm.cnt[dst[k]], 1u) : 0u;
  __syncthreads();
  const unsigned per = (nb + kTT - 1) / kTT;
  const unsigned lo = threadIdx.x * per;
  const unsigned hi = min(lo + per, nb);
  unsigned c[kPer], s = 0;
#pragma unroll
  for (unsigned k = 0; k < kPer; k++) {
    c[k] = lo + k < hi ? sm.cnt[lo + k] : 0u;
    s += c[k];
  }
  unsigned total;
  unsigned pre = block_scan_u32_fenced<kTT>(s, sm.red, &total);
  u64 b0[kPer];
#pragma unroll
  for (unsigned k = 0; k < kPer; k++) b0[k] = c[k] ? atomicAdd(dest(lo + k).counter, (u64)c[k]) : 0;
#pragma unroll
  for (unsigned k = 0; k < kPer; k++) {
    if (lo + k < hi) {
      const DestRun r = dest(lo + k);
      const u64 room = c[k] && b0[k] < r.cap ? r.cap - b0[k] : 0;
      sm.cnt[lo + k] = pre;
      sm.start[lo + k] = (unsigned short)(pre + (unsigned)(room < c[k] ? room : c[k]));
      sm.run[lo + k] = (c[k] ? r.base + b0[k] : 0) - pre;
      pre += c[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kKPT; k++) {
    if (ok[k]) {
      const unsigned pos = sm.cnt[dst[k]] + rk[k];
      sm.sorted[pos] = x[k];
      sm.stag[pos] = (dst[k] << 20) | lp[k];
    }
  }
  __syncthreads();
  for (unsigned i = threadIdx.x; i < total; i += kTT) {
    const unsigned tg = sm.stag[i];
    const unsigned b = tg >> 20;
    if (i < sm.start[b]) {
      const u64 j = sm.run[b] + i;
      arena[j] = sm.sorted[i];
      if (WITH_POS) parena[j] = tg & 0xfffffu;
    } else {
      atomicOr(status, ST_OVERFLOW);
    }
  }
  for (unsigned i = threadIdx.x; i < nb; i += kTT) sm.cnt[i] = 0;  // last read before the scatter
  __syncthreads();
}
// Zero the destination counts before a kernel's first multisplit_write (the
// caller synchronises the block before that call).
__device__ __forceinline__ void split_clear(const SplitSmem &sm, unsigned nb_cap) {
  for (unsigned i = threadIdx.x; i < nb_cap; i += kTT) sm.cnt[i] = 0;
}

// sorted_cap >= kTile entries of `sorted` (a caller may stage more keys there
// than one multisplit takes; the multisplit itself uses the first kTile).
__device__ __forceinline__ SplitSmem carve_split(unsigned char *smem, unsigned nb_cap,
                                                 unsigned sorted_cap = kTile) {
  SplitSmem s;
  s.sorted = reinterpret_cast<u64 *>(smem);
  s.run = s.sorted + sorted_cap;
  s.stag = reinterpret_cast<unsigned *>(s.run + nb_cap);
  s.cnt = s.stag + kTile;
  s.red = s.cnt + nb_cap;
  s.start = reinterpret_cast<unsigned short *>(s.red + kTT / 32 + 2);
  return s;
}

static constexpr size_t split_smem_bytes(unsigned nb_cap, unsigned sorted_cap = kTile) {
  // a multiple of 16 bytes: callers place 16-byte staging buffers after it
  return ((size_t)sorted_cap * 8 + (size_t)nb_cap * 8 + (size_t)kTile * 4 + (size_t)nb_cap * 4 +
          (kTT / 32 + 2) * 4 + (size_t)nb_cap * 2 + 8 + 15) & ~(size_t)15;
}

// ---------------------------------------------------------------------------
// Level 0: partition the caller's keys into position buckets of A_0; each key
// is stored with its position inside the bucket, so the fill needs no hash.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }


// ---------------------------------------------------------------------------
// Single-CTA level loop: levels d0.. of a key set of at most kTailMaxKeys keys,
// keys and bit arrays in shared memory.
// ---------------------------------------------------------------------------
struct TailSmem {
  u64 *keys;      // [kTailMaxKeys]
  unsigned *hit;  // [mcap / 32]
  unsigned *col;
  unsigned *red;  // [32 + 2]
  u64 *red64;     // [32]
};

static __device__ void bitonic_sort_smem(u64 *a, unsigned n) {
  unsigned P = 1;
  while (P < n) P <<= 1;
  for (unsigned i = n + threadIdx.x; i < P; i += blockDim.x) a[i] = ~0ull;
  __syncthreads();
  for (unsigned k = 2; k <= P; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned l = i ^ j;
        if (l > i) {
          u64 x = a[i], y = a[l];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Returns the number of levels used.  lvs: level records (n/m/off/weight/mode)
// of this key set; A0 / arena / m0 locate A_d; fb_out receives the sorted
// fallback (n_fb keys).  NT threads, at most MAXK keys (MAXK / NT <= 32).
template <int NT, int MAXK>
static __device__ unsigned cta_levels(const TailSmem &sm, u64 n, int d0, u64 off, FLevel *lvs,
                                      double gamma, uint32_t L, u64 seed, u64 *A0, u64 *arena,
                                      u64 m0, u64 arena_words, u64 *fb_out, u64 *n_fb_out,
                                      unsigned *status) {
  static_assert(MAXK % NT == 0 && MAXK / NT <= 32, "keys per thread must fit a 32-bit mask");
  int d = d0;
  for (;;) {
    if (n == 0) {
      if (threadIdx.x == 0) lvs[d].mode = LM_DONE;
      return (unsigned)d;
    }
    if ((uint32_t)d == L) {
      bitonic_sort_smem(sm.keys, (unsigned)n);
      for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
        u64 v = sm.keys[i];
        fb_out[i] = v;
        if (i + 1 < n && v == sm.keys[i + 1]) atomicOr(status, ST_DUPLICATE);
      }
      if (threadIdx.x == 0) {
        *n_fb_out = n;
        lvs[d].mode = LM_FLAT;
        lvs[d].n = n;
      }
      __syncthreads();
      return L;
    }
    const u64 m = level_bits(n, gamma);
    const u64 s = level_seed(seed, (uint32_t)d);
    const unsigned mw = (unsigned)(m >> 5);
    for (unsigned i = threadIdx.x; i < mw; i += blockDim.x) {
      sm.hit[i] = 0;
      sm.col[i] = 0;
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
      const u64 p = level_pos(sm.keys[i], s, m);
      const unsigned bit = 1u << (p & 31);
      const unsigned old = atomicOr(sm.hit + (p >> 5), bit);
      if (old & bit) atomicOr(sm.col + (p >> 5), bit);
    }
    __syncthreads();
    u64 *Alev = (d == 0) ? A0 : arena + ((off - m0) >> 6);
    // A_d must fit in the space reserved for the levels after the first
    const bool fits = d == 0 || ((off - m0) >> 6) + (m >> 6) <= arena_words;
    if (!fits && threadIdx.x == 0) atomicOr(status, ST_OVERFLOW);
    u64 wsum = 0;
    for (unsigned w = threadIdx.x; w < (unsigned)(m >> 6); w += blockDim.x) {
      const u64 a = (u64)(sm.hit[2 * w] & ~sm.col[2 * w]) |
                    ((u64)(sm.hit[2 * w + 1] & ~sm.col[2 * w + 1]) << 32);
      if (fits) Alev[w] = a;
      wsum += __popcll(a);
    }
    // compaction in place: each thread keeps its contiguous run of keys in registers
    constexpr unsigned KMAX = (unsigned)(MAXK / NT);
    const unsigned per = (unsigned)((n + blockDim.x - 1) / blockDim.x);
    const unsigned lo = threadIdx.x * per;
    u64 mine[KMAX];
    unsigned keepmask = 0, c = 0;
#pragma unroll
    for (unsigned k = 0; k < KMAX; k++) {
      mine[k] = 0;
      const unsigned i = lo + k;
      if (k < per && i < n) {
        const u64 x = sm.keys[i];
        const u64 p = level_pos(x, s, m);
        const unsigned bit = 1u << (p & 31);
        const bool placed = (sm.hit[p >> 5] & ~sm.col[p >> 5]) & bit;
        if (!placed) {
          mine[k] = x;
          keepmask |= 1u << k;
          c++;
        }
      }
    }
    unsigned total;
    unsigned pre = block_scan_u32<NT>(c, sm.red, &total);
    // every thread has read its keys (block_scan synchronises)
#pragma unroll
    for (unsigned k = 0; k < KMAX; k++) {
      if (keepmask & (1u << k)) sm.keys[pre++] = mine[k];
    }
    const u64 wt = block_sum<NT>(wsum, sm.red64);
    if (threadIdx.x == 0) {
      if (wt + total != n) atomicOr(status, ST_INTERNAL);
      lvs[d].n = n;
      lvs[d].m = m;
      lvs[d].off = off;
      lvs[d].weight = wt;
      lvs[d].mode = LM_FLAT;
    }
    n = total;
    off += m;
    d++;
    if (threadIdx.x == 0) {
      lvs[d].n = n;
      lvs[d].off = off;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ TailSmem carve_tail(unsigned char *smem, u64 mcap,
                                               u64 maxk = kTailMaxKeys) {
  TailSmem t;
  t.keys = reinterpret_cast<u64 *>(smem);
  t.hit = reinterpret_cast<unsigned *>(smem + maxk * 8);
  t.col = t.hit + (mcap >> 5);
  t.red64 = reinterpret_cast<u64 *>(t.col + (mcap >> 5));
  t.red = reinterpret_cast<unsigned *>(t.red64 + 32);
  return t;
}

static inline size_t tail_smem_bytes(u64 mcap, u64 maxk = kTailMaxKeys) {
  return maxk * 8 + 2 * (mcap >> 5) * 4 + 32 * 8 + 40 * 4;
}


}  // namespace bbh
