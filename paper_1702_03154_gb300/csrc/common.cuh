// common.cuh -- shared internals of libmphf (device hash, level sizing, launch
// accounting, error plumbing).  Internal to the CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mphf.h"

namespace bbh {

typedef unsigned long long u64;

// ---------------------------------------------------------------------------
// Level hash (Sec. 3.3 only says the hash is a fast one built on xor-shifts;
// this library uses the SplitMix64 finalizer, a xor-shift-multiply mixer).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Seed of h_d: a different hash function per level (Sec. 2.1).
__host__ __device__ __forceinline__ u64 level_seed(u64 seed, uint32_t d) {
  return mix64(mix64(seed) + (u64)d);
}

// floor(h * m / 2^64): maps the 64-bit hash onto [0, m) without a division.
// For m < 2^32 (every level below ~2^31 keys) the same value comes from two
// 32x32-bit products: with h = hi 2^32 + lo,
//   floor(h m / 2^64) = floor((hi m + floor(lo m / 2^32)) / 2^32),
// since the dropped fraction of lo m / 2^32 is below 1 and hi m + lo m / 2^32
// stays below 2^64.
__device__ __forceinline__ u64 reduce_range(u64 h, u64 m) {
  if ((m >> 32) == 0) {
    const unsigned m32 = (unsigned)m;
    const u64 t = ((u64)(unsigned)h * m32) >> 32;
    return ((u64)(unsigned)(h >> 32) * m32 + t) >> 32;
  }
  return __umul64hi(h, m);
}

// Position of key x in A_d (m_d bits).
__device__ __forceinline__ u64 level_pos(u64 x, u64 s_d, u64 m_d) {
  return reduce_range(mix64(x ^ s_d), m_d);
}

// |A_d| for n keys (Sec. 2.2.4: gamma * |F_d| bits), in whole 64-bit words, >= 64.
// ceil(gamma * n) comes from one IEEE double multiply (no fused operation).
__host__ __device__ __forceinline__ u64 level_bits(u64 n, double gamma) {
#ifdef __CUDA_ARCH__
  double t = __dmul_rn(gamma, (double)n);
#else
  volatile double t = gamma * (double)n;
#endif
  u64 c = (u64)t;
  if ((double)c < t) c += 1;
  c = (c + 63) & ~63ull;
  return c < 64 ? 64 : c;
}

// ---------------------------------------------------------------------------
// Per-build device metadata.  The build kernels read level sizes from here and
// the last block of each extract writes the next level's sizes, so the level
// loop needs no host round trip to size its launches.
// ---------------------------------------------------------------------------
struct BuildMeta {
  u64 n[MPHF_MAX_LEVELS + 1];   // n[d] = |F_d|
  u64 m[MPHF_MAX_LEVELS + 1];   // m[d] = |A_d| bits (0 past the last level)
  u64 off[MPHF_MAX_LEVELS + 1]; // bit offset of A_d in A
  u64 weight[MPHF_MAX_LEVELS];  // ones in A_d
  u64 out_count[MPHF_MAX_LEVELS + 1];  // keys written to F_{d+1} by compaction d
  unsigned int done[MPHF_MAX_LEVELS];  // extract blocks finished
  unsigned int status;          // 0 or an MPHF_E* code raised on the device
  unsigned int levels_used;     // set by extract when a level leaves no keys
};

// ---------------------------------------------------------------------------
// Host-side plumbing.
// ---------------------------------------------------------------------------
void set_cuda_error(cudaError_t e, const char *where);
int cuda_fail(cudaError_t e, const char *where);  // records and returns MPHF_ECUDA

#define MPHF_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::bbh::cuda_fail(e_, #call); \
  } while (0)

// Kernel launch accounting + optional event timing.  Every launch in the
// library goes through LaunchScope so that mphf_launch_count() and the
// per-kernel profile see it.
void launch_begin(const char *name, cudaStream_t s);
void launch_end(cudaStream_t s);
void add_launches(u64 n);  // kernels replayed inside a recorded graph

struct LaunchScope {
  cudaStream_t s;
  LaunchScope(const char *name, cudaStream_t st) : s(st) { launch_begin(name, st); }
  ~LaunchScope() { launch_end(s); }
};

// Current device, clamped to the 64 slots of the per-device caches below.
inline int cur_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    dev = 0;
  }
  return dev;
}

// SM count of the current device (cached per device; racing writers store
// the same value).
inline int sm_count() {
  static int cache[64] = {0};
  const int dev = cur_device();
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

// CTAs of `kernel` (block threads, dynamic smem bytes) that fit on the whole
// GPU at once: a grid of this size runs in a single wave.
template <class K>
inline unsigned int resident_grid(K kernel, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (unsigned int)(per_sm * sm_count());
}

// Keys a lookup warp takes from its batch at a time: 2048 once the batch has
// that many for every resident warp, otherwise fewer (a multiple of 64, at
// least 128), so that a small batch still spreads over the whole GPU instead
// of queueing on a few warps.
inline u64 lookup_chunk(u64 n, u64 resident_warps) {
  u64 c = (n + resident_warps - 1) / (resident_warps ? resident_warps : 1);
  c = (c + 63) & ~63ull;
  return c < 128 ? 128 : c > 2048 ? 2048 : c;
}

inline unsigned int grid_for(u64 items, unsigned int per_block, unsigned int max_blocks) {
  u64 b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (unsigned int)b;
}

// Device memory owned by a handle or a build.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};
int dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s);
void dev_free(DevBuf &b, cudaStream_t s);

// Host keys copied to a device buffer in chunks on a side stream, so that the
// consumer's kernels on the main stream can start on chunk c while chunk c+1
// is still crossing the host link.  ensure(upto, st) enqueues the copies of
// keys [issued, upto) and makes st wait for them; ensure(n, st) therefore makes
// the whole buffer visible to st.  The copies of one call share one event
// record, and cudaStreamWaitEvent binds the record current at the call, so a
// single event serves every chunk.
struct KeyFeed {
  const u64 *h = nullptr;  // host keys (pinned or pageable)
  u64 *d = nullptr;        // device buffer of n keys, allocated on the main stream
  u64 n = 0;
  u64 chunk = 0;           // keys per copy; a multiple of 4096 keeps chunk starts 16-B aligned
  u64 issued = 0;          // keys whose copy is enqueued (and awaited by the main stream)
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  // Optional second array copied on cs right behind the last key chunk, one
  // event per chunk (mphf_build_lookup_host: the queries cross the host link
  // while the levels are built).  The main stream never waits for them here.
  const u64 *hq = nullptr;
  u64 *dq = nullptr;
  u64 nq = 0, qchunk = 0;        // qchunk: keys per query chunk (> 0)
  cudaEvent_t *qev = nullptr;    // ceil(nq / qchunk) events
  bool q_issued = false;
  int ensure(u64 upto, cudaStream_t st);
  int issue_queries();
};
// Keys per chunk for n keys (0 = copy in one piece: too few keys to pipeline).
u64 feed_chunk(u64 n);

// Side streams and events of the host-buffer entry points, created once per
// host thread and device and reused by every call (creating and destroying
// them per call cost about as much as copying a chunk).  A call joins all it
// enqueued on them into its own stream before it returns, so one thread's
// consecutive calls never overlap on them.
struct SideSet {
  cudaStream_t s[2];
  cudaEvent_t *ev;  // n_events events (timing disabled)
};
int side_set(size_t n_events, SideSet *out);

// Sort n keys ascending in place and flag equal neighbours (sort.cu).
int sort_fallback(u64 *keys, u64 n, unsigned int *d_dup_flag, cudaStream_t s);

}  // namespace bbh

struct mphf_shared;  // one device arena shared by the handles of a batched build
namespace bbh {
void release_shared(mphf_shared *sh);
}

// The handle.  Host copies of the level metadata plus the device arrays.
struct mphf {
  uint64_t N = 0;
  double gamma = 2.0;
  uint32_t L = 25;
  uint64_t seed = 0;
  uint32_t L_used = 0;
  uint64_t M = 0;        // total bits
  uint64_t n_rank = 0;   // ceil(M / 512)
  uint64_t n_fb = 0;
  uint32_t sw = 7;       // layout: A words per sector, 7 (32 B) or 15 (64 B); 48 = 8-byte units
  uint64_t n_sect = 0;   // sectors holding A and its ranks (sector.cuh)
  bbh::DevBuf S;        // n_sect * (sw + 1) 32-bit words
  bbh::DevBuf SB;       // ones before each superblock of 2^24 sectors
  bbh::DevBuf fb;       // n_fb keys
  int device = 0;
  int path = 0;          // 1 bucketed, 2 unbucketed, 3 batched, 4 loaded, 5 without stored F_d
  mphf_shared *shared = nullptr;  // set: S/SB/fb live in a batched arena
  bbh::DevBuf ldesc;     // device descriptor for multi-function lookups (made on first use)
  // level tables (last, so that a record can be reset without them): entries
  // past L_used (n: past L_used + 1; s: past L) are never read
  uint64_t n[MPHF_MAX_LEVELS + 1] = {0};
  uint64_t m[MPHF_MAX_LEVELS] = {0};
  uint64_t off[MPHF_MAX_LEVELS] = {0};
  uint64_t s[MPHF_MAX_LEVELS] = {0};
};

namespace bbh {
// Every level below 2^32 bits and A below 2^36 bits: a probe's position
// arithmetic fits 32 bits (word index g >> 5 or piece index g >> 4 < 2^32).
extern int g_lookup_wide;  // test hook: 1 sends every lookup through the 64-bit kernels
inline bool narrow_positions(const mphf *h) {
  if (g_lookup_wide) return false;
  bool narrow = (h->M >> 36) == 0;
  for (uint32_t d = 0; d < h->L_used; d++) narrow = narrow && (h->m[d] >> 32) == 0;
  return narrow;
}

// Handle records come from a process-wide free list: a batched build makes
// thousands at once, and fresh heap pages for them (each record is ~2 KB of
// level tables) cost a page fault per page.  handle_new returns a zeroed
// record or nullptr; handle_new_n fills out[0..n) under one lock (all or
// none; zero_tables = false leaves a reused record's level tables as they
// were, for a caller that writes every entry it reads); handle_delete takes
// back a record whose device memory is released.
mphf *handle_new();
bool handle_new_n(unsigned n, mphf **out, bool zero_tables = true);
void handle_delete(mphf *h);
}  // namespace bbh
