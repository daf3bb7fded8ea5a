// sector.cuh -- the lookup layout of A and its ranks.
//
// The query of Algorithm 3 ends, for a key placed at bit g of the
// concatenated array A (Sec. 2.2.3), with the number of ones of A before g
// (Sec. 3.1).  Kept apart, bit g and the count before it are two random
// memory requests.  Here they share one 32-byte sector:
//
//   word 0 of sector t   ones of A in the sectors of t's superblock before t
//   words 1..7           A's 32-bit words 7t .. 7t+6 (224 bits of A)
//
// A superblock is 2^24 sectors; SB[k] (64-bit) holds the ones before
// superblock k, so word 0 stays 32-bit for any size of A and SB[0] = 0.  A
// probe loads the one sector that holds g with a single 256-bit load; its A
// word and its rank arrive together.  The layout costs 32 bits per 224 bits
// of A (1/7); checkpoints every 512 bits with in-block counts cost 1/4.
//
// The count of ones before bit 512 b (the paper's checkpoint b) and the plain
// A both follow from the sectors, so the introspection entry points return
// exactly the paper's arrays.
#pragma once

#include "common.cuh"

namespace bbh {

static constexpr unsigned kSectWords = 7;                // A words (32-bit) per sector
static constexpr unsigned kSectBits = 32 * kSectWords;   // 224
static constexpr unsigned kSBShift = 24;                 // 2^24 sectors per superblock

__host__ __device__ inline u64 n_sectors(u64 M) {
  return (M / 32 + kSectWords - 1) / kSectWords;
}
__host__ __device__ inline u64 n_superblocks(u64 nsect) {
  return (nsect + (1ull << kSBShift) - 1) >> kSBShift;
}

// One sector in registers: r = word 0, w[i] = word i + 1.
struct Sect {
  unsigned r, w[kSectWords];
};

// Sector t of S (S is 32-byte aligned): one 256-bit load, not kept in L1 (a
// probe's sector is rarely touched again by the same SM).
__device__ __forceinline__ Sect sect_load(const unsigned *__restrict__ S, u64 t) {
  Sect v;
  asm("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v.r), "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3]), "=r"(v.w[4]),
        "=r"(v.w[5]), "=r"(v.w[6])
      : "l"(S + 8 * t));
  return v;
}

// Where bit g lives: sector t, A word j (0..6) of the sector, bit b of the word.
struct SectPos {
  u64 t;
  unsigned j, b;
};
__device__ __forceinline__ SectPos sect_pos(u64 g) {
  const u64 q = g >> 5;
  const u64 t = q / kSectWords;
  return SectPos{t, (unsigned)(q - t * kSectWords), (unsigned)g & 31u};
}

__device__ __forceinline__ unsigned sect_word(const Sect &v, unsigned j) {
  unsigned x = v.w[0];
#pragma unroll
  for (unsigned i = 1; i < kSectWords; i++) x = (j == i) ? v.w[i] : x;
  return x;
}

// Ones of A before bit (t, j, b), given the sector and SB.
__device__ __forceinline__ u64 sect_rank(const Sect &v, const SectPos &p, unsigned word,
                                         const u64 *__restrict__ SB) {
  unsigned c = v.r;
#pragma unroll
  for (unsigned i = 0; i + 1 < kSectWords; i++) c += (i < p.j) ? __popc(v.w[i]) : 0u;
  c += __popc(word & ((1u << p.b) - 1u));
  const u64 k = p.t >> kSBShift;
  return (k ? __ldg(SB + k) : 0ull) + c;
}

// A as 64-bit words in two pieces: words [0, w0) at a0, [w0, W) at a1.
struct ASrc {
  const u64 *a0;
  u64 w0;
  const u64 *a1;
  u64 W;
};

// Build the sectors S (n_sectors(M) * 8 words) and SB (n_superblocks words)
// of the M-bit array src; *d_total receives the number of ones.
int build_sectors(const ASrc &src, u64 M, unsigned *S, u64 *SB, u64 *d_total, cudaStream_t s);
// Allocate h->S / h->SB for h->M bits and build them from src.
int make_sectors(mphf_t *h, const ASrc &src, u64 *d_total, cudaStream_t s);
// The paper's checkpoints: out[b] = ones before bit 512 b, b < n_rank.
int sector_checkpoints(const unsigned *S, const u64 *SB, u64 n_rank, u64 *d_out, cudaStream_t s);

}  // namespace bbh
