// rank.cu -- the ranks of Sec. 3.1 over the concatenated bit array A.
//
// Every function's A is stored in one of the layouts of sector.cuh (A's words
// interleaved with counts of the ones before them); build_sectors writes
// sectors in three passes: (1) each thread popcounts one sector and each CTA
// sums its sectors, (2) one CTA scans the per-CTA sums, (3) each sector is
// written with its count relative to its superblock; 8-byte units in two:
// one CTA per 1024-unit block writes the units with their in-block counts,
// then one CTA scans the block sums into the block table.
// sector_checkpoints evaluates the paper's checkpoints (ones before bit
// 512 b) in any layout.
//
// The file also holds a standalone rank-table builder over caller-supplied
// words (mphf_rank_table_noalloc): one 64-bit checkpoint per 512 bits, stored
// next to a word of seven 9-bit in-block prefix counts -- the "rank9" layout of
// Vigna ("Broadword implementation of rank/select queries", WEA 2008) -- in
// three passes: per-block counts with a CTA scan, a scan of the CTA totals,
// and the addition of each CTA's prefix.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "sector.cuh"

namespace bbh {

static constexpr int kRankThreads = 256;
static constexpr int kScanThreads = 1024;

__device__ __forceinline__ u64 block_exclusive_scan(u64 v, u64 *total) {
  __shared__ u64 warp_sums[kRankThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    u64 w = lane < kRankThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u64 y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kRankThreads / 32) warp_sums[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  u64 before = warp ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kRankThreads / 32 - 1];
  return before + x - v;
}

__global__ void __launch_bounds__(kRankThreads)
k_rank_blocks(const u64 *__restrict__ A, u64 nwords, u64 *__restrict__ rank2, u64 nrank,
              u64 *__restrict__ cta_sums) {
  u64 b = (u64)blockIdx.x * kRankThreads + threadIdx.x;
  u64 c = 0, rel = 0;
  if (b < nrank) {
    u64 w0 = b * 8;
    unsigned pc[8];
    if (w0 + 8 <= nwords) {
      const uint4 *p = reinterpret_cast<const uint4 *>(A + w0);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        uint4 v = __ldg(p + j);
        pc[2 * j] = __popc(v.x) + __popc(v.y);
        pc[2 * j + 1] = __popc(v.z) + __popc(v.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; j++) pc[j] = (w0 + j < nwords) ? __popcll(__ldg(A + w0 + j)) : 0u;
    }
    unsigned run = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (j) rel |= (u64)run << (9 * (j - 1));
      run += pc[j];
    }
    c = run;
  }
  u64 total;
  u64 ex = block_exclusive_scan(c, &total);
  if (b < nrank) {
    rank2[2 * b] = ex;
    rank2[2 * b + 1] = rel;
  }
  if (threadIdx.x == 0) cta_sums[blockIdx.x] = total;
}

// Exclusive scan of `count` CTA totals in one CTA; grand total to *d_total.
__global__ void __launch_bounds__(kScanThreads)
k_scan_sums(u64 *__restrict__ sums, u64 count, u64 *__restrict__ d_total) {
  __shared__ u64 part[kScanThreads];
  const u64 per = (count + kScanThreads - 1) / kScanThreads;
  const u64 lo = threadIdx.x * per;
  const u64 hi = lo + per < count ? lo + per : count;
  u64 s = 0;
  for (u64 i = lo; i < hi; i++) s += sums[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over kScanThreads partials
  for (int o = 1; o < kScanThreads; o <<= 1) {
    u64 add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  u64 run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (u64 i = lo; i < hi; i++) {
    u64 v = sums[i];
    sums[i] = run;
    run += v;
  }
  if (threadIdx.x == kScanThreads - 1 && d_total) *d_total = part[kScanThreads - 1];
}

__global__ void __launch_bounds__(kRankThreads)
k_rank_add(u64 *__restrict__ rank2, u64 nrank, const u64 *__restrict__ cta_prefix) {
  u64 b = (u64)blockIdx.x * kRankThreads + threadIdx.x;
  if (b < nrank) rank2[2 * b] += cta_prefix[blockIdx.x];
}

// ---------------------------------------------------------------------------
// Sector layout (sector.cuh): one thread per sector of W A-words, 256 sectors
// per CTA, so a superblock (2^24 sectors) is exactly 2^16 CTAs.  Pass 1 sums
// the ones of each CTA's sectors, k_scan_sums turns the sums into exclusive
// prefixes, pass 2 reads A again and writes every sector with its count
// relative to the start of its superblock.
// ---------------------------------------------------------------------------
static constexpr int kSectThreads = kRankThreads;
static_assert(((1u << kSBShift) % kSectThreads) == 0, "a CTA must not straddle superblocks");

__device__ __forceinline__ u64 a_word(const ASrc &a, u64 k) {
  if (k < a.w0) return __ldg(a.a0 + k);
  return k < a.W ? __ldg(a.a1 + (k - a.w0)) : 0ull;
}

// A's 32-bit words W t .. W t + W - 1 (zero past the end of A).
template <int W>
__device__ __forceinline__ void sect_words(const ASrc &a, u64 t, unsigned (&w)[W]) {
  constexpr int K = W / 2 + 1;  // 64-bit words covering W + 1 32-bit words
  const u64 q0 = t * W;
  const u64 k0 = q0 >> 1;
  unsigned h[2 * K];
#pragma unroll
  for (int i = 0; i < K; i++) {
    const u64 u = a_word(a, k0 + i);
    h[2 * i] = (unsigned)u;
    h[2 * i + 1] = (unsigned)(u >> 32);
  }
  const bool odd = q0 & 1;
#pragma unroll
  for (int i = 0; i < W; i++) w[i] = odd ? h[i + 1] : h[i];
}

template <int W>
__global__ void __launch_bounds__(kSectThreads)
k_sect_sums(ASrc a, u64 nsect, u64 *__restrict__ cta_sums) {
  const u64 t = (u64)blockIdx.x * kSectThreads + threadIdx.x;
  unsigned c = 0;
  if (t < nsect) {
    unsigned w[W];
    sect_words<W>(a, t, w);
#pragma unroll
    for (int i = 0; i < W; i++) c += __popc(w[i]);
  }
  u64 total;
  block_exclusive_scan(c, &total);
  if (threadIdx.x == 0) cta_sums[blockIdx.x] = total;
}

template <int W>
__global__ void __launch_bounds__(kSectThreads)
k_sect_write(ASrc a, u64 nsect, unsigned *__restrict__ S, const u64 *__restrict__ cta_prefix,
             u64 *__restrict__ SB) {
  const u64 t = (u64)blockIdx.x * kSectThreads + threadIdx.x;
  unsigned w[W];
  unsigned c = 0;
  if (t < nsect) {
    sect_words<W>(a, t, w);
#pragma unroll
    for (int i = 0; i < W; i++) c += __popc(w[i]);
  }
  u64 total;
  const u64 ex = block_exclusive_scan(c, &total);
  constexpr unsigned kCtaPerSB = (1u << kSBShift) / kSectThreads;
  const u64 sb_cta = (u64)blockIdx.x / kCtaPerSB * kCtaPerSB;  // first CTA of the superblock
  if (t < nsect) {
    const unsigned rel = (unsigned)(cta_prefix[blockIdx.x] - cta_prefix[sb_cta] + ex);
    uint4 *dst = reinterpret_cast<uint4 *>(S + (u64)(W + 1) * t);
    dst[0] = make_uint4(rel, w[0], w[1], w[2]);
#pragma unroll
    for (int k = 1; k < (W + 1) / 4; k++)
      dst[k] = make_uint4(w[4 * k - 1], w[4 * k], w[4 * k + 1], w[4 * k + 2]);
  }
  if (threadIdx.x == 0 && (u64)blockIdx.x == sb_cta)
    SB[blockIdx.x / kCtaPerSB] = cta_prefix[blockIdx.x];
}

// 8-byte units: one CTA per block of 1024 units, 4 units per thread.  The
// counts restart at every block, so each CTA writes its block alone; the
// per-block sums then become SB by one exclusive scan.
static constexpr int kUnitThreads = 256;
static constexpr int kUnitsPerThread = (1 << kUnitBlockShift) / kUnitThreads;

__device__ __forceinline__ u64 a_bits48(const ASrc &a, u64 u) {
  const u64 bit = u * kUnitBits, k = bit >> 6;
  const unsigned sh = (unsigned)(bit & 63);
  u64 v = a_word(a, k) >> sh;
  if (sh > 64 - kUnitBits) v |= a_word(a, k + 1) << (64 - sh);
  return v & ((1ull << kUnitBits) - 1ull);
}

__global__ void __launch_bounds__(kUnitThreads)
k_unit_write(ASrc a, u64 nunits, u64 *__restrict__ S8, u64 *__restrict__ block_sums) {
  const u64 u0 = ((u64)blockIdx.x << kUnitBlockShift) + (u64)threadIdx.x * kUnitsPerThread;
  u64 v[kUnitsPerThread];
  unsigned c[kUnitsPerThread], run = 0;
#pragma unroll
  for (int i = 0; i < kUnitsPerThread; i++) {
    v[i] = u0 + i < nunits ? a_bits48(a, u0 + i) : 0;
    c[i] = run;
    run += __popcll(v[i]);
  }
  u64 total;
  const u64 ex = block_exclusive_scan(run, &total);
#pragma unroll
  for (int i = 0; i < kUnitsPerThread; i++)
    if (u0 + i < nunits) S8[u0 + i] = v[i] | ((ex + c[i]) << kUnitBits);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

int build_sectors(const ASrc &src, u64 M, unsigned W, unsigned *S, u64 *SB, u64 *d_total,
                  cudaStream_t s) {
  if (!layout_ok(W)) return MPHF_EINVAL;
  if (W == kUnitBits) {
    const u64 nunits = n_sectors(M, W);
    if (nunits == 0) {
      if (d_total) MPHF_CUDA(cudaMemsetAsync(d_total, 0, sizeof(u64), s));
      return MPHF_OK;
    }
    const u64 blocks = n_sb_entries(nunits, W);
    if (blocks > 0x7fffffffull) return MPHF_EINVAL;
    {
      LaunchScope ls("unit_write", s);
      k_unit_write<<<(unsigned)blocks, kUnitThreads, 0, s>>>(src, nunits, (u64 *)S, SB);
    }
    {
      LaunchScope ls("sect_scan", s);
      k_scan_sums<<<1, kScanThreads, 0, s>>>(SB, blocks, d_total);
    }
    MPHF_CUDA(cudaGetLastError());
    return MPHF_OK;
  }
  const u64 nsect = n_sectors(M, W);
  if (nsect == 0) {
    if (d_total) MPHF_CUDA(cudaMemsetAsync(d_total, 0, sizeof(u64), s));
    return MPHF_OK;
  }
  const u64 ctas = (nsect + kSectThreads - 1) / kSectThreads;
  if (ctas > 0x7fffffffull) return MPHF_EINVAL;
  DevBuf sums;
  int rc = dev_alloc(sums, ctas * sizeof(u64), s);
  if (rc != MPHF_OK) return rc;
  {
    LaunchScope ls("sect_sums", s);
    if (W == kSectWords)
      k_sect_sums<kSectWords><<<(unsigned)ctas, kSectThreads, 0, s>>>(src, nsect, (u64 *)sums.p);
    else
      k_sect_sums<kSectWordsMini><<<(unsigned)ctas, kSectThreads, 0, s>>>(src, nsect,
                                                                          (u64 *)sums.p);
  }
  {
    LaunchScope ls("sect_scan", s);
    k_scan_sums<<<1, kScanThreads, 0, s>>>((u64 *)sums.p, ctas, d_total);
  }
  {
    LaunchScope ls("sect_write", s);
    if (W == kSectWords)
      k_sect_write<kSectWords><<<(unsigned)ctas, kSectThreads, 0, s>>>(src, nsect, S,
                                                                       (const u64 *)sums.p, SB);
    else
      k_sect_write<kSectWordsMini><<<(unsigned)ctas, kSectThreads, 0, s>>>(
          src, nsect, S, (const u64 *)sums.p, SB);
  }
  cudaError_t e = cudaGetLastError();
  dev_free(sums, s);
  if (e != cudaSuccess) return cuda_fail(e, "sector kernels");
  return MPHF_OK;
}

int make_sectors(mphf_t *h, const ASrc &src, u64 *d_total, cudaStream_t s) {
  h->n_sect = n_sectors(h->M, h->sw);
  int rc = dev_alloc(h->S, h->n_sect * sector_bytes(h->sw), s);
  if (rc == MPHF_OK) rc = dev_alloc(h->SB, n_sb_entries(h->n_sect, h->sw) * 8, s);
  if (rc == MPHF_OK)
    rc = build_sectors(src, h->M, h->sw, (unsigned *)h->S.p, (u64 *)h->SB.p, d_total, s);
  return rc;
}

template <int W>
__global__ void __launch_bounds__(256)
k_checkpoints(const unsigned *__restrict__ S, const u64 *__restrict__ SB, u64 n_rank,
              u64 *__restrict__ out) {
  const u64 b = (u64)blockIdx.x * 256 + threadIdx.x;
  if (b >= n_rank) return;
  using LW = Lay<W>;
  const typename LW::Pos p = LW::pos(b * MPHF_RANK_BLOCK);
  const typename LW::Data v = LW::load(S, p);
  unsigned w = 0;
  LW::hit(v, p, w);
  out[b] = LW::rank(v, p, w, SB);
}

int sector_checkpoints(const unsigned *S, const u64 *SB, unsigned W, u64 n_rank, u64 *d_out,
                       cudaStream_t s) {
  if (n_rank == 0) return MPHF_OK;
  const u64 ctas = (n_rank + 255) / 256;
  if (ctas > 0x7fffffffull || !layout_ok(W)) return MPHF_EINVAL;
  {
    LaunchScope ls("checkpoints", s);
    if (W == kSectWords)
      k_checkpoints<kSectWords><<<(unsigned)ctas, 256, 0, s>>>(S, SB, n_rank, d_out);
    else if (W == kSectWordsMini)
      k_checkpoints<kSectWordsMini><<<(unsigned)ctas, 256, 0, s>>>(S, SB, n_rank, d_out);
    else
      k_checkpoints<kUnitBits><<<(unsigned)ctas, 256, 0, s>>>(S, SB, n_rank, d_out);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

}  // namespace bbh

// ---------------------------------------------------------------------------
// Allocation-free variant of the rank-table build, for callers that cannot
// allocate device memory.  The per-CTA partial sums that build_rank_table
// allocates live instead in this file-scope device array.  It is sized for at
// most kNoAllocMaxCtas CTAs, i.e. 2^24 rank blocks of 512 bits (2^27 words of
// A, 2^33 bits).  Every process that loads the library holds it on every GPU
// it uses, until exit.
// ---------------------------------------------------------------------------
namespace bbh {

static constexpr u64 kNoAllocMaxCtas = 65536;
static __device__ __align__(256) u64 g_rank_scratch[kNoAllocMaxCtas];

static std::mutex g_noalloc_mu;
// Device address of g_rank_scratch, per device, looked up on the first call
// there.  The cache assumes the device is never reset while the library is
// loaded (cudaDeviceReset unloads the module that holds the array).
static u64 *g_noalloc_ptr[64] = {nullptr};

}  // namespace bbh

extern "C" int mphf_rank_table_noalloc(const uint64_t *d_words, uint64_t nwords,
                                       uint64_t *d_rank2, uint64_t *d_total, void *stream) {
  using namespace bbh;
  const u64 nrank = (nwords + 7) / 8;
  if (nwords > 0 && (!d_words || !d_rank2)) return MPHF_EINVAL;
  if (((uintptr_t)d_words & 15) || ((uintptr_t)d_rank2 & 15) || ((uintptr_t)d_total & 7))
    return MPHF_EINVAL;
  const u64 ctas = (nrank + kRankThreads - 1) / kRankThreads;
  if (ctas > kNoAllocMaxCtas) return MPHF_EINVAL;  // beyond the fixed scratch
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  MPHF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return MPHF_EINVAL;
  u64 *scratch;
  {
    // First call on a device: look up the array's device address (the host
    // symbol g_rank_scratch is only a stand-in and must not be passed).
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_rank_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(rank scratch)");
      g_noalloc_ptr[dev] = (u64 *)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (nrank == 0) {
    if (d_total) MPHF_CUDA(cudaMemsetAsync(d_total, 0, sizeof(u64), s));
    return MPHF_OK;
  }
  // every used entry of the scratch is written by k_rank_blocks before it is
  // read, so nothing needs clearing between calls
  {
    LaunchScope ls("rank_blocks", s);
    k_rank_blocks<<<(unsigned)ctas, kRankThreads, 0, s>>>((const u64 *)d_words, nwords,
                                                          (u64 *)d_rank2, nrank, scratch);
  }
  {
    LaunchScope ls("rank_scan", s);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(scratch, ctas, (u64 *)d_total);
  }
  if (ctas > 1) {
    LaunchScope ls("rank_add", s);
    k_rank_add<<<(unsigned)ctas, kRankThreads, 0, s>>>((u64 *)d_rank2, nrank, scratch);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}
