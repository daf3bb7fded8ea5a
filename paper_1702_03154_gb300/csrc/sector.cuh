// sector.cuh -- the lookup layout of A and its ranks.
//
// The query of Algorithm 3 ends, for a key placed at bit g of the
// concatenated array A (Sec. 2.2.3), with the number of ones of A before g
// (Sec. 3.1).  Kept apart, bit g and the count before it are two random
// memory requests.  Here they share one sector of W + 1 32-bit words:
//
//   word 0 of sector t   ones of A in the sectors of t's superblock before t
//   words 1..W           A's 32-bit words W t .. W t + W - 1
//
// A superblock is 2^24 sectors; SB[k] (64-bit) holds the ones before
// superblock k, so word 0 stays 32-bit for any size of A and SB[0] = 0.
//
// Two sector sizes give the rank-sampling trade-off of Sec. 3.1 / Sec. 4.3:
//   W = 7  (32 bytes, the default): a probe is one 256-bit load holding both
//          the A word and its count; the counts cost 1/7 of A (the paper's
//          64-bit counter per 512 bits costs 1/8).
//   W = 15 (64 bytes, "minirank"): one count per 480 bits of A, 1/15 of A
//          (the paper's counter per 1024 bits: 1/16); a probe loads both
//          halves of the sector, so queries hold twice the registers.
//
// The count of ones before bit 512 b (the paper's checkpoint b) and the plain
// A both follow from the sectors, so the introspection entry points return
// exactly the paper's arrays.
#pragma once

#include "common.cuh"

namespace bbh {

static constexpr unsigned kSectWords = 7;       // default A words per sector
static constexpr unsigned kSectWordsMini = 15;  // minirank
static constexpr unsigned kSBShift = 24;        // 2^24 sectors per superblock
// Third layout: 8-byte units of 48 bits of A (bits 0-47) and a 16-bit count
// (bits 48-63) of the ones in the unit's block of 1024 units before the unit;
// SB[k] holds the ones before block k.  A probe is one 8-byte load (fewer
// registers in flight, cheaper requests) at the price of counts costing 1/3 of
// A.  The layout id stored in a handle is the 48.
static constexpr unsigned kUnitBits = 48;
static constexpr unsigned kUnitBlockShift = 10;

__host__ __device__ inline bool layout_ok(unsigned W) {
  return W == kSectWords || W == kSectWordsMini || W == kUnitBits;
}
// sectors (or units) holding M bits of A
__host__ __device__ inline u64 n_sectors(u64 M, unsigned W) {
  if (W == kUnitBits) return (M + kUnitBits - 1) / kUnitBits;
  return (M / 32 + W - 1) / W;
}
__host__ __device__ inline u64 n_superblocks(u64 nsect) {
  return (nsect + (1ull << kSBShift) - 1) >> kSBShift;
}
// entries of SB for nsect sectors (units) of layout W
__host__ __device__ inline u64 n_sb_entries(u64 nsect, unsigned W) {
  if (W == kUnitBits) return (nsect + (1ull << kUnitBlockShift) - 1) >> kUnitBlockShift;
  return n_superblocks(nsect);
}
__host__ __device__ inline u64 sector_bytes(unsigned W) { return W == kUnitBits ? 8 : 4ull * (W + 1); }

// Where A's bytes sit in the stored array: `full` records of `width` bytes of A
// at `pitch`-byte steps starting `offset` bytes in, then `rest` bytes of A in
// the next record -- so one strided copy gathers the plain A back.
struct AGather {
  u64 pitch, width, offset, full, rest;
};
__host__ inline AGather a_gather(u64 M, unsigned W) {
  const u64 bytes = M / 8;  // A is whole 64-bit words
  AGather g;
  if (W == kUnitBits) {
    g.pitch = 8;
    g.width = 6;
    g.offset = 0;
  } else {
    g.pitch = 4ull * (W + 1);
    g.width = 4ull * W;
    g.offset = 4;
  }
  g.full = bytes / g.width;
  g.rest = bytes - g.full * g.width;
  return g;
}

// One sector in registers: r = word 0, w[i] = word i + 1.
template <int W>
struct Sect {
  unsigned r, w[W];
};

__device__ __forceinline__ void ld256(const unsigned *p, unsigned (&v)[8]) {
  asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "l"(p));
}

// Sector t of S (sectors are 32-byte aligned): 256-bit non-coherent loads (the
// sectors are read-only while a lookup runs).
template <int W>
__device__ __forceinline__ Sect<W> sect_load(const unsigned *__restrict__ S, u64 t) {
  static_assert(W == 7 || W == 15, "sector sizes: 32 or 64 bytes");
  Sect<W> v;
  unsigned a[8];
  ld256(S + (u64)(W + 1) * t, a);
  v.r = a[0];
#pragma unroll
  for (int i = 0; i < 7; i++) v.w[i] = a[i + 1];
  if (W == 15) {
    unsigned b[8];
    ld256(S + (u64)(W + 1) * t + 8, b);
#pragma unroll
    for (int i = 0; i < 8; i++) v.w[(7 + i) % W] = b[i];
  }
  return v;
}

// Where bit g lives: sector t, A word j (0..W-1) of the sector, bit b of the word.
struct SectPos {
  u64 t;
  unsigned j, b;
};
// q / W for q < 2^32 by a multiply-high (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): for 7 the 33-bit
// magic 2^35/7 is applied as m' = 0x24924925 plus one add-and-shift fixup; for
// 15, 0x88888889 = ceil(2^35 / 15) is exact for every 32-bit q.
template <int W>
__device__ __forceinline__ unsigned div_sector(unsigned q) {
  if (W == 7) {
    const unsigned t = __umulhi(q, 0x24924925u);
    return (t + ((q - t) >> 1)) >> 2;
  }
  return __umulhi(q, 0x88888889u) >> 3;
}

template <int W>
__device__ __forceinline__ SectPos sect_pos(u64 g) {
  const u64 q = g >> 5;
  if ((q >> 32) == 0) {  // A below 2^37 bits: 32-bit arithmetic
    const unsigned q32 = (unsigned)q;
    const unsigned t = div_sector<W>(q32);
    return SectPos{t, q32 - t * (unsigned)W, (unsigned)g & 31u};
  }
  const u64 t = q / W;
  return SectPos{t, (unsigned)(q - t * W), (unsigned)g & 31u};
}

// Element j (< N, N a power of two) of a[0..N-1] by a tree of selects on j's
// bits: N - 1 selects, where comparing j with every index costs a compare
// and a select per element.
template <int N>
__device__ __forceinline__ unsigned select_tree(const unsigned (&a)[N], unsigned j) {
  unsigned x[N];
#pragma unroll
  for (int i = 0; i < N; i++) x[i] = a[i];
#pragma unroll
  for (int h = 1; h < N; h <<= 1) {
    const bool bit = (j & (unsigned)h) != 0u;
#pragma unroll
    for (int i = 0; i < N / (2 * h); i++) x[i] = bit ? x[2 * i + 1] : x[2 * i];
  }
  return x[0];
}

template <int W>
__device__ __forceinline__ unsigned sect_word(const Sect<W> &v, unsigned j) {
  unsigned a[W + 1];
#pragma unroll
  for (int i = 0; i < W; i++) a[i] = v.w[i];
  a[W] = v.w[W - 1];
  return select_tree<W + 1>(a, j);
}

// Ones of A before bit (t, j, b), given the sector and SB: the count of the
// sector plus the prefix counts of its words, the one before word j picked by
// the same select tree.
template <int W>
__device__ __forceinline__ u64 sect_rank(const Sect<W> &v, const SectPos &p, unsigned word,
                                         const u64 *__restrict__ SB) {
  unsigned pre[W + 1];
  pre[0] = v.r;
#pragma unroll
  for (int i = 0; i + 1 < W; i++) pre[i + 1] = pre[i] + __popc(v.w[i]);
  pre[W] = pre[W - 1];
  unsigned c = select_tree<W + 1>(pre, p.j);
  c += __popc(word & ((1u << p.b) - 1u));
  const u64 k = p.t >> kSBShift;
  return (k ? __ldg(SB + k) : 0ull) + c;
}

// ---------------------------------------------------------------------------
// The probe of a lookup through one interface for every layout:
//   Pos p = Lay<W>::pos(g);          where bit g lives
//   Data v = Lay<W>::load(S, p);     the one memory request of the probe
//   Lay<W>::hit(v, p, w)             bit g of A (w: the A word, for rank)
//   Lay<W>::rank(v, p, w, SB)        ones of A before bit g
// ---------------------------------------------------------------------------
//   Pos p = Lay<W>::pos_q(q, lo);    the same for g = q 2^kQShift + lo, q < 2^32
template <int W>
struct Lay {
  using Pos = SectPos;
  using Data = Sect<W>;
  static constexpr unsigned kQShift = 5;  // q: the 32-bit word of A holding bit g
  static __device__ __forceinline__ Pos pos(u64 g) { return sect_pos<W>(g); }
  static __device__ __forceinline__ Pos pos_q(unsigned q, unsigned lo) {
    const unsigned t = div_sector<W>(q);
    return SectPos{t, q - t * (unsigned)W, lo};
  }
  static __device__ __forceinline__ Data load(const unsigned *__restrict__ S, const Pos &p) {
    return sect_load<W>(S, p.t);
  }
  static __device__ __forceinline__ bool hit(const Data &v, const Pos &p, unsigned &w) {
    w = sect_word<W>(v, p.j);
    return (w >> p.b) & 1u;
  }
  static __device__ __forceinline__ u64 rank(const Data &v, const Pos &p, unsigned w,
                                             const u64 *__restrict__ SB) {
    return sect_rank<W>(v, p, w, SB);
  }
};

struct UnitPos {
  u64 u;       // unit
  unsigned b;  // bit within the unit's 48 bits of A
};
template <>
struct Lay<(int)kUnitBits> {
  using Pos = UnitPos;
  using Data = u64;
  // g / 48 = (g / 16) / 3; for g / 16 < 2^32, q / 3 = umulhi(q, 0xAAAAAAAB) >> 1
  // exactly (Granlund and Montgomery, as for the sector widths above)
  static __device__ __forceinline__ Pos pos(u64 g) {
    const u64 q = g >> 4;
    const u64 u = (q >> 32) == 0 ? (u64)(__umulhi((unsigned)q, 0xAAAAAAABu) >> 1) : q / 3;
    return UnitPos{u, (unsigned)(g - u * kUnitBits)};
  }
  static constexpr unsigned kQShift = 4;  // q: the 16-bit piece of A holding bit g
  static __device__ __forceinline__ Pos pos_q(unsigned q, unsigned lo) {
    const unsigned u = __umulhi(q, 0xAAAAAAABu) >> 1;
    return UnitPos{u, 16u * (q - 3u * u) + lo};
  }
  // an ordinary cached load: measured on a GB300, the same 8-byte probes with
  // an L1 no-allocate hint ran 1.6x slower
  static __device__ __forceinline__ Data load(const unsigned *__restrict__ S, const Pos &p) {
    return __ldg(reinterpret_cast<const u64 *>(S) + p.u);
  }
  static __device__ __forceinline__ bool hit(const Data &v, const Pos &p, unsigned &) {
    return (v >> p.b) & 1ull;
  }
  static __device__ __forceinline__ u64 rank(const Data &v, const Pos &p, unsigned,
                                             const u64 *__restrict__ SB) {
    return __ldg(SB + (p.u >> kUnitBlockShift)) + (v >> 48) + __popcll(v & ((1ull << p.b) - 1ull));
  }
};

// A as 64-bit words in two pieces: words [0, w0) at a0, [w0, W) at a1.
struct ASrc {
  const u64 *a0;
  u64 w0;
  const u64 *a1;
  u64 W;
};

// Build the sectors S (n_sectors(M, W) of them) and SB (n_sb_entries words)
// of the M-bit array src; *d_total receives the number of ones.
int build_sectors(const ASrc &src, u64 M, unsigned W, unsigned *S, u64 *SB, u64 *d_total,
                  cudaStream_t s);
// Allocate h->S / h->SB in h->sw's sector size for h->M bits and build them.
int make_sectors(mphf_t *h, const ASrc &src, u64 *d_total, cudaStream_t s);
// The paper's checkpoints: out[b] = ones before bit 512 b, b < n_rank.
int sector_checkpoints(const unsigned *S, const u64 *SB, unsigned W, u64 n_rank, u64 *d_out,
                       cudaStream_t s);

}  // namespace bbh
