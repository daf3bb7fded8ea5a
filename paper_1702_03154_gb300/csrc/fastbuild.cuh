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
};

__host__ __device__ inline u64 ceil_div(u64 a, u64 b) { return (a + b - 1) / b; }

}  // namespace bbh
