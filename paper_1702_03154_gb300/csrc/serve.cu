// serve.cu -- a request loop that keeps many functions resident in HBM.
//
// Lookup requests (any resident handle, any batch size) are admitted into a
// pending queue; a scheduler thread coalesces whatever is pending into one
// launch of a multi-function lookup kernel (k_lookup_multi) as soon as a
// launch slot is free (continuous batching: requests that arrive while other
// batches run join the next batch, up to kMaxInflight batches on two
// alternating lookup streams).  Build requests are admitted when their memory
// footprint fits the free device memory (sampled by the build workers, not by
// the scheduler) minus a reserve, and run on their own
// streams in worker threads, so they overlap the lookups.  Completion times
// are taken when the scheduler sees a batch's event complete; latency is
// submit -> completion on the host clock.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "parts.cuh"
#include "sector.cuh"

namespace bbh {

// Device descriptor of a handle for the multi-function lookup.
struct LookupDev {
  const unsigned *S;  // sectors (sector.cuh)
  const u64 *SB, *fb;
  u64 n_fb, N;
  uint32_t L_used, sw;  // levels, A words per sector
  u64 s[MPHF_MAX_LEVELS], m[MPHF_MAX_LEVELS], off[MPHF_MAX_LEVELS];
  // for functions with narrow_positions: m_d and off_d >> kQShift in 32 bits
  unsigned m32[MPHF_MAX_LEVELS], oq[MPHF_MAX_LEVELS];
};

struct ReqDev {
  const LookupDev *h;
  const u64 *keys;
  u64 *out;
  u64 start;  // first index of this request in the batch's key space
};

static std::mutex g_desc_mu;

int ensure_lookup_desc(mphf_t *h) {
  std::lock_guard<std::mutex> lk(g_desc_mu);
  if (h->ldesc.p) return MPHF_OK;
  LookupDev d;
  memset(&d, 0, sizeof(d));
  d.S = (const unsigned *)h->S.p;
  d.SB = (const u64 *)h->SB.p;
  d.fb = (const u64 *)h->fb.p;
  d.n_fb = h->n_fb;
  d.N = h->N;
  d.L_used = h->L_used;
  d.sw = h->sw;
  for (uint32_t i = 0; i < h->L_used; i++) {
    d.s[i] = h->s[i];
    d.m[i] = h->m[i];
    d.off[i] = h->off[i];
    d.m32[i] = (unsigned)h->m[i];
    d.oq[i] = (unsigned)(h->off[i] >> (h->sw == kUnitBits ? Lay<(int)kUnitBits>::kQShift
                                                          : Lay<(int)kSectWords>::kQShift));
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(d));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc(lookup descriptor)");
  }
  e = cudaMemcpy(p, &d, sizeof(d), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_fail(e, "cudaMemcpy(lookup descriptor)");
  }
  h->ldesc.p = p;
  h->ldesc.bytes = sizeof(d);
  return MPHF_OK;
}

__device__ __forceinline__ u64 fallback_index_m(const LookupDev *h, u64 x) {
  u64 lo = 0, hi = h->n_fb;
  while (lo < hi) {
    u64 mid = lo + ((hi - lo) >> 1);
    if (__ldg(h->fb + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  if (lo < h->n_fb && __ldg(h->fb + lo) == x) return h->N - h->n_fb + lo;
  return MPHF_NOT_FOUND;
}

static constexpr int kMultiThreads = 256;
static constexpr int kMultiSlots = 2;

// Lookups of a batch of requests against different functions: the keys of all
// requests form one index space [0, total); warps take chunks of it and keep
// kMultiSlots query slots per lane, each slot carrying its request's function.
// NARROW: every function of the batch has narrow_positions (32-bit probe
// arithmetic, as in k_lookup).
template <int W, bool NARROW>
__global__ void __launch_bounds__(kMultiThreads)
k_lookup_multi(const ReqDev *__restrict__ reqs, unsigned nreq, u64 total, u64 csz) {
  using LW = Lay<W>;
  const unsigned lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const u64 nchunks = (total + csz - 1) / csz;
  const u64 nwarps = ((u64)gridDim.x * kMultiThreads) >> 5;
  u64 chunk = ((u64)blockIdx.x * kMultiThreads + threadIdx.x) >> 5;
  u64 cursor = chunk * csz;
  u64 cend = chunk < nchunks ? min(cursor + csz, total) : cursor;
  bool more = chunk < nchunks;
  unsigned rcur = 0;  // request holding `cursor` (warp-uniform), found by search
  auto find_req = [&](u64 i, unsigned from) -> unsigned {
    unsigned r = from;
    if (r + 1 < nreq && reqs[r + 1].start <= i) {  // jump: binary search
      unsigned lo = r, hi = nreq - 1;
      while (lo < hi) {
        unsigned mid = (lo + hi + 1) >> 1;
        if (reqs[mid].start <= i) lo = mid;
        else hi = mid - 1;
      }
      r = lo;
    }
    return r;
  };
  if (more) rcur = find_req(cursor, 0);

  u64 x[kMultiSlots];
  u64 *optr[kMultiSlots];
  const LookupDev *hd[kMultiSlots];
  unsigned lvl[kMultiSlots];
  bool act[kMultiSlots];
#pragma unroll
  for (int s = 0; s < kMultiSlots; s++) {
    act[s] = false;
    lvl[s] = 0;
    x[s] = 0;
    optr[s] = nullptr;
    hd[s] = nullptr;
  }
  for (;;) {
    // free slots ranked lane by lane, slot 0 first, filled in one pass while
    // the chunk holds a key for each; the rest by the loop below
    unsigned rk[kMultiSlots], nfree = 0;
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) {
      const unsigned need = __ballot_sync(0xffffffffu, !act[s]);
      rk[s] = nfree + __popc(need & lt);
      nfree += __popc(need);
    }
    if (nfree && cend - cursor >= nfree) {
#pragma unroll
      for (int s = 0; s < kMultiSlots; s++) {
        if (!act[s]) {
          const u64 gi = cursor + rk[s];
          unsigned q = rcur;
          while (q + 1 < nreq && reqs[q + 1].start <= gi) q++;
          const ReqDev rd = reqs[q];
          x[s] = __ldcs(rd.keys + (gi - rd.start));
          optr[s] = rd.out + (gi - rd.start);
          hd[s] = rd.h;
          lvl[s] = 0;
          act[s] = true;
        }
      }
      cursor += nfree;
      if (cursor < total) {
        unsigned q = rcur;
        while (q + 1 < nreq && reqs[q + 1].start <= cursor) q++;
        rcur = q;
      }
    }
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) {
      unsigned need = __ballot_sync(0xffffffffu, !act[s]);
      while (need && more) {
        if (cursor >= cend) {
          chunk += nwarps;
          if (chunk >= nchunks) {
            more = false;
            break;
          }
          cursor = chunk * csz;
          cend = min(cursor + csz, total);
          rcur = find_req(cursor, rcur);
        }
        const u64 avail = cend - cursor;
        const unsigned r = __popc(need & lt);
        const bool mine = ((need >> lane) & 1u) && (u64)r < avail;
        if (mine) {
          const u64 gi = cursor + r;
          unsigned q = rcur;
          while (q + 1 < nreq && reqs[q + 1].start <= gi) q++;
          const ReqDev rd = reqs[q];
          x[s] = __ldcs(rd.keys + (gi - rd.start));
          optr[s] = rd.out + (gi - rd.start);
          hd[s] = rd.h;
          lvl[s] = 0;
          act[s] = true;
        }
        const unsigned taken = __ballot_sync(0xffffffffu, mine);
        need &= ~taken;
        cursor += __popc(taken);
        if (more && cursor < total) {
          // keep rcur at the request holding the cursor
          unsigned q = rcur;
          while (q + 1 < nreq && reqs[q + 1].start <= cursor) q++;
          rcur = q;
        }
      }
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) any |= act[s];
    if (!__any_sync(0xffffffffu, any)) break;
    typename LW::Pos p[kMultiSlots];
    typename LW::Data v[kMultiSlots];
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) {
      if (act[s]) {
        const unsigned d = lvl[s];
        const LookupDev *h = hd[s];
        if (NARROW) {
          const u64 hh = mix64(x[s] ^ __ldg(h->s + d));
          const unsigned m32 = __ldg(h->m32 + d);
          const u64 lo = ((u64)(unsigned)hh * m32) >> 32;
          const unsigned pd = (unsigned)(((u64)(unsigned)(hh >> 32) * m32 + lo) >> 32);
          p[s] = LW::pos_q(__ldg(h->oq + d) + (pd >> LW::kQShift),
                           pd & ((1u << LW::kQShift) - 1u));
        } else {
          p[s] = LW::pos(__ldg(h->off + d) + level_pos(x[s], __ldg(h->s + d), __ldg(h->m + d)));
        }
        v[s] = LW::load(h->S, p[s]);
      }
    }
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) {
      if (act[s]) {
        const LookupDev *h = hd[s];
        unsigned w = 0;
        if (LW::hit(v[s], p[s], w)) {
          *optr[s] = LW::rank(v[s], p[s], w, h->SB);
          act[s] = false;
        } else if (++lvl[s] >= h->L_used) {
          *optr[s] = h->n_fb ? fallback_index_m(h, x[s]) : MPHF_NOT_FOUND;
          act[s] = false;
        }
      }
    }
  }
}

// Lookups against the K functions of a split, without routing the keys: a
// refilled slot takes its key's part from the part hash, that part's
// function, and adds the part's offset to the answer.  Slots and probes as in
// k_lookup_multi (one index space: the n keys).
template <int W, bool NARROW>
__global__ void __launch_bounds__(kMultiThreads)
k_lookup_parts(const u64 *__restrict__ keys, u64 n, u64 csz, u64 *__restrict__ out,
               const LookupDev *const *__restrict__ fns, const u64 *__restrict__ prefix,
               uint32_t K, u64 sp) {
  using LW = Lay<W>;
  const unsigned lane = threadIdx.x & 31;
  const u64 nchunks = (n + csz - 1) / csz;
  const u64 nwarps = ((u64)gridDim.x * kMultiThreads) >> 5;
  u64 chunk = ((u64)blockIdx.x * kMultiThreads + threadIdx.x) >> 5;
  u64 cursor = chunk * csz;
  u64 cend = chunk < nchunks ? min(cursor + csz, n) : cursor;
  bool more = chunk < nchunks;
  const unsigned lt = (1u << lane) - 1u;
  u64 x[kMultiSlots], idx[kMultiSlots];
  const LookupDev *hd[kMultiSlots];
  unsigned part[kMultiSlots], lvl[kMultiSlots];
  bool act[kMultiSlots];
#pragma unroll
  for (int s = 0; s < kMultiSlots; s++) {
    act[s] = false;
    lvl[s] = 0;
    x[s] = 0;
    idx[s] = 0;
    part[s] = 0;
    hd[s] = nullptr;
  }
  auto take = [&](int s, u64 i) {
    x[s] = __ldcs(keys + i);
    idx[s] = i;
    part[s] = part_index(x[s], sp, K);
    hd[s] = fns[part[s]];
    lvl[s] = 0;
    act[s] = true;
  };
  for (;;) {
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) {
      unsigned need = __ballot_sync(0xffffffffu, !act[s]);
      while (need && more) {
        if (cursor >= cend) {
          chunk += nwarps;
          if (chunk >= nchunks) {
            more = false;
            break;
          }
          cursor = chunk * csz;
          cend = min(cursor + csz, n);
        }
        const u64 avail = cend - cursor;
        const unsigned r = __popc(need & lt);
        const bool mine = ((need >> lane) & 1u) && (u64)r < avail;
        if (mine) take(s, cursor + r);
        const unsigned taken = __ballot_sync(0xffffffffu, mine);
        need &= ~taken;
        cursor += __popc(taken);
      }
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) any |= act[s];
    if (!__any_sync(0xffffffffu, any)) break;
    typename LW::Pos p[kMultiSlots];
    typename LW::Data v[kMultiSlots];
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) {
      if (act[s]) {
        const unsigned d = lvl[s];
        const LookupDev *h = hd[s];
        if (NARROW) {
          const u64 hh = mix64(x[s] ^ __ldg(h->s + d));
          const unsigned m32 = __ldg(h->m32 + d);
          const u64 lo = ((u64)(unsigned)hh * m32) >> 32;
          const unsigned pd = (unsigned)(((u64)(unsigned)(hh >> 32) * m32 + lo) >> 32);
          p[s] = LW::pos_q(__ldg(h->oq + d) + (pd >> LW::kQShift),
                           pd & ((1u << LW::kQShift) - 1u));
        } else {
          p[s] = LW::pos(__ldg(h->off + d) + level_pos(x[s], __ldg(h->s + d), __ldg(h->m + d)));
        }
        v[s] = LW::load(h->S, p[s]);
      }
    }
#pragma unroll
    for (int s = 0; s < kMultiSlots; s++) {
      if (act[s]) {
        const LookupDev *h = hd[s];
        unsigned w = 0;
        u64 r = MPHF_NOT_FOUND;
        bool done = false;
        if (LW::hit(v[s], p[s], w)) {
          r = LW::rank(v[s], p[s], w, h->SB);
          done = true;
        } else if (++lvl[s] >= h->L_used) {
          r = h->n_fb ? fallback_index_m(h, x[s]) : MPHF_NOT_FOUND;
          done = true;
        }
        if (done) {
          __stcs(out + idx[s], r == MPHF_NOT_FOUND ? r : r + __ldg(prefix + part[s]));
          act[s] = false;
        }
      }
    }
  }
}

template <int W, bool NARROW>
static int launch_parts_wn(const LookupDev *const *d_fns, const u64 *prefix, uint32_t K, u64 sp,
                           const u64 *keys, u64 n, u64 *out, cudaStream_t s) {
  static u64 maxb_dev[64] = {0};  // one wave of resident CTAs, per device
  u64 &maxb = maxb_dev[cur_device()];
  if (!maxb) maxb = resident_grid(k_lookup_parts<W, NARROW>, kMultiThreads, 0);
  const u64 csz = lookup_chunk(n, maxb * (kMultiThreads / 32));
  const u64 chunks = (n + csz - 1) / csz;
  u64 grid = (chunks + (kMultiThreads / 32) - 1) / (kMultiThreads / 32);
  if (grid > maxb) grid = maxb;
  if (grid < 1) grid = 1;
  LaunchScope ls("lookup_parts", s);
  k_lookup_parts<W, NARROW><<<(unsigned)grid, kMultiThreads, 0, s>>>(keys, n, csz, out, d_fns,
                                                                      prefix, K, sp);
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

template <int W>
static int launch_parts_w(const LookupDev *const *d_fns, const u64 *prefix, uint32_t K, u64 sp,
                          const u64 *keys, u64 n, u64 *out, bool narrow, cudaStream_t s) {
  return narrow ? launch_parts_wn<W, true>(d_fns, prefix, K, sp, keys, n, out, s)
                : launch_parts_wn<W, false>(d_fns, prefix, K, sp, keys, n, out, s);
}

int lookup_parts_direct(mphf *const *fs, uint32_t K, u64 sp, const u64 *d_prefix,
                        const u64 *keys, u64 n, u64 *out, cudaStream_t s) {
  if (K == 0 || !fs[0]) return MPHF_EINVAL;
  const unsigned sw = fs[0]->sw;
  bool narrow = true;
  for (uint32_t k = 0; k < K; k++) {
    if (!fs[k] || fs[k]->sw != sw || fs[k]->L_used == 0) return MPHF_EINVAL;
    narrow = narrow && narrow_positions(fs[k]);
  }
  std::vector<const LookupDev *> t(K);
  for (uint32_t k = 0; k < K; k++) {
    int rc = ensure_lookup_desc(fs[k]);
    if (rc != MPHF_OK) return rc;
    t[k] = (const LookupDev *)fs[k]->ldesc.p;
  }
  DevBuf d;
  int rc = dev_alloc(d, sizeof(void *) * K, s);
  if (rc != MPHF_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(d.p, t.data(), sizeof(void *) * K, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    dev_free(d, s);
    return cuda_fail(e, "cudaMemcpyAsync(part functions)");
  }
  const LookupDev *const *dt = (const LookupDev *const *)d.p;
  if (sw == kSectWords) rc = launch_parts_w<kSectWords>(dt, d_prefix, K, sp, keys, n, out, narrow, s);
  else if (sw == kSectWordsMini)
    rc = launch_parts_w<kSectWordsMini>(dt, d_prefix, K, sp, keys, n, out, narrow, s);
  else rc = launch_parts_w<kUnitBits>(dt, d_prefix, K, sp, keys, n, out, narrow, s);
  dev_free(d, s);  // stream-ordered: released after the kernel (the pageable copy has taken t)
  return rc;
}

template <int W, bool NARROW>
static int launch_multi_wn(const ReqDev *d_reqs, unsigned nreq, u64 total, cudaStream_t s) {
  static u64 maxb_dev[64] = {0};  // one wave of resident CTAs, per device
  u64 &maxb = maxb_dev[cur_device()];
  if (!maxb) maxb = resident_grid(k_lookup_multi<W, NARROW>, kMultiThreads, 0);
  const u64 csz = lookup_chunk(total, maxb * (kMultiThreads / 32));
  const u64 chunks = (total + csz - 1) / csz;
  u64 grid = (chunks + (kMultiThreads / 32) - 1) / (kMultiThreads / 32);
  if (grid > maxb) grid = maxb;
  if (grid < 1) grid = 1;
  LaunchScope ls("lookup_multi", s);
  k_lookup_multi<W, NARROW><<<(unsigned)grid, kMultiThreads, 0, s>>>(d_reqs, nreq, total,
                                                                      csz);
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

template <int W>
static int launch_multi_w(const ReqDev *d_reqs, unsigned nreq, u64 total, bool narrow,
                          cudaStream_t s) {
  if (total == 0 || nreq == 0) return MPHF_OK;
  return narrow ? launch_multi_wn<W, true>(d_reqs, nreq, total, s)
                : launch_multi_wn<W, false>(d_reqs, nreq, total, s);
}

// Request table of a batch, grouped by layout: the default-layout requests
// first (index space [0, g.total[0])), then the minirank ones, then those in
// 8-byte units (each group with its own index space from 0), so that each
// group runs in the kernel compiled for its layout.
static constexpr int kLayouts = 3;  // 32-byte sectors, 64-byte sectors, 8-byte units
__host__ inline int layout_group(unsigned sw) {
  return sw == kSectWords ? 0 : sw == kSectWordsMini ? 1 : 2;
}
struct TableGroups {
  unsigned n[kLayouts] = {0, 0, 0};
  u64 total[kLayouts] = {0, 0, 0};
  bool narrow[kLayouts] = {true, true, true};  // every function of the group
};
template <class GetH, class GetKeys, class GetOut, class GetN>
static TableGroups fill_table(ReqDev *t, size_t nreq, GetH geth, GetKeys getk, GetOut geto,
                              GetN getn) {
  TableGroups g;
  unsigned placed = 0;
  for (int grp = 0; grp < kLayouts; grp++) {
    for (size_t i = 0; i < nreq; i++) {
      const mphf_t *h = geth(i);
      if (layout_group(h->sw) != grp) continue;
      ReqDev &r = t[placed++];
      r.h = (const LookupDev *)h->ldesc.p;
      r.keys = getk(i);
      r.out = geto(i);
      r.start = g.total[grp];
      g.total[grp] += getn(i);
      g.n[grp]++;
      g.narrow[grp] = g.narrow[grp] && narrow_positions(h);
    }
  }
  return g;
}

static int launch_lookup_multi(const ReqDev *d_reqs, const TableGroups &g, cudaStream_t s) {
  int rc = launch_multi_w<kSectWords>(d_reqs, g.n[0], g.total[0], g.narrow[0], s);
  if (rc == MPHF_OK)
    rc = launch_multi_w<kSectWordsMini>(d_reqs + g.n[0], g.n[1], g.total[1], g.narrow[1], s);
  if (rc == MPHF_OK)
    rc = launch_multi_w<kUnitBits>(d_reqs + g.n[0] + g.n[1], g.n[2], g.total[2], g.narrow[2], s);
  return rc;
}

// ---------------------------------------------------------------------------
// Server.
// ---------------------------------------------------------------------------
using clk = std::chrono::steady_clock;

static double now_s() {
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id;
  int kind;  // 0 lookup, 1 build
  mphf_t *h;
  const u64 *keys;
  u64 *out;
  u64 n;
  double gamma;
  uint32_t L;
  u64 seed;
  double t_submit = 0, t_done = 0;
  double t_launch = 0;  // lookups: when the batch holding it was launched
  int status = MPHF_OK;
  mphf_t *built = nullptr;
  bool done = false;
};

struct Batch {
  std::vector<Req *> reqs;
  cudaEvent_t ev;       // after the batch (completion)
  cudaEvent_t ev0;      // before the batch (GPU time of the batch, with ev)
  int slot;
};

}  // namespace bbh

struct mphf_server {
  // parameters
  uint64_t max_batch_keys, max_batch_reqs;
  int max_inflight, build_workers;
  uint64_t mem_reserve;
  // state
  std::mutex mu;
  std::condition_variable cv_done;
  std::deque<bbh::Req *> pending_lookups, pending_builds;
  std::unordered_map<uint64_t, bbh::Req *> reqs;
  uint64_t next_id = 1;
  std::atomic<bool> stop{false};
  std::thread sched;
  std::vector<std::thread> workers;
  std::deque<bbh::Req *> build_queue;  // admitted, waiting for a worker
  std::condition_variable cv_build;
  std::atomic<uint64_t> build_reserved{0};
  // device
  int device = 0;
  cudaStream_t lstream[2] = {nullptr, nullptr};
  std::vector<bbh::DevBuf> dtab;           // request tables, one per launch slot
  std::vector<bbh::ReqDev *> htab;         // pinned staging
  std::vector<bool> slot_busy;
  std::vector<cudaEvent_t> slot_ev0, slot_ev;  // timing events of each launch slot, made once
  // free device memory, sampled by the build workers (never by the scheduler,
  // whose loop must not wait on a device query)
  std::atomic<uint64_t> free_mem{0};
  std::deque<bbh::Batch> inflight;
  // statistics
  std::atomic<uint64_t> batches{0}, batched_reqs{0}, batched_keys{0}, builds_done{0};
  // per completed lookup: queue wait (submit -> launch of its batch), GPU time
  // of its batch, and the rest (launch -> completion seen, minus GPU time)
  std::vector<double> part_queue, part_gpu, part_rest;
};

namespace bbh {

static u64 build_footprint(u64 n, double gamma) {
  // bucket arenas (key + position, two levels), A, rank table, small metadata
  const double m = (double)level_bits(n ? n : 1, gamma);
  return (u64)(n * 12.0 * 1.10 + n * 12.0 * 0.70 + m / 8.0 * 3.0 + (64 << 20));
}

static void scheduler(mphf_server *sv) {
  cudaSetDevice(sv->device);
  std::vector<Req *> take;
  int rr = 0;
  while (!sv->stop.load()) {
    bool worked = false;
    // 1. completions, in any order: batches alternate between two streams,
    // so a short batch may finish behind a longer one launched before it
    for (auto it = sv->inflight.begin(); it != sv->inflight.end();) {
      Batch &b = *it;
      cudaError_t q = cudaEventQuery(b.ev);
      if (q == cudaErrorNotReady) {
        ++it;
        continue;
      }
      const double t = now_s();
      float gpu_ms = 0.f;
      if (cudaEventElapsedTime(&gpu_ms, b.ev0, b.ev) != cudaSuccess) {
        cudaGetLastError();
        gpu_ms = 0.f;
      }
      {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (Req *r : b.reqs) {
          r->t_done = t;
          r->status = q == cudaSuccess ? MPHF_OK : MPHF_ECUDA;
          r->done = true;
          sv->part_queue.push_back(r->t_launch - r->t_submit);
          sv->part_gpu.push_back(gpu_ms * 1e-3);
          sv->part_rest.push_back(t - r->t_launch - gpu_ms * 1e-3);
        }
      }
      sv->cv_done.notify_all();
      sv->slot_busy[b.slot] = false;
      it = sv->inflight.erase(it);
      worked = true;
    }
    // 2. a new lookup batch from everything pending (continuous batching)
    if ((int)sv->inflight.size() < sv->max_inflight) {
      int slot = -1;
      for (int i = 0; i < (int)sv->slot_busy.size(); i++)
        if (!sv->slot_busy[i]) {
          slot = i;
          break;
        }
      take.clear();
      u64 keys = 0;
      if (slot >= 0) {
        std::lock_guard<std::mutex> lk(sv->mu);
        while (!sv->pending_lookups.empty() && take.size() < sv->max_batch_reqs) {
          Req *r = sv->pending_lookups.front();
          if (!take.empty() && keys + r->n > sv->max_batch_keys) break;
          take.push_back(r);
          keys += r->n;
          sv->pending_lookups.pop_front();
        }
      }
      if (!take.empty()) {
        ReqDev *ht = sv->htab[slot];
        const TableGroups g = fill_table(
            ht, take.size(), [&](size_t i) { return (const mphf_t *)take[i]->h; },
            [&](size_t i) { return take[i]->keys; }, [&](size_t i) { return take[i]->out; },
            [&](size_t i) { return take[i]->n; });
        cudaStream_t s = sv->lstream[rr++ & 1];
        Batch b;
        b.reqs = take;
        b.slot = slot;
        b.ev0 = sv->slot_ev0[slot];
        b.ev = sv->slot_ev[slot];
        const double tl = now_s();
        for (Req *r : take) r->t_launch = tl;
        cudaEventRecord(b.ev0, s);
        cudaMemcpyAsync(sv->dtab[slot].p, ht, sizeof(ReqDev) * take.size(),
                        cudaMemcpyHostToDevice, s);
        launch_lookup_multi((const ReqDev *)sv->dtab[slot].p, g, s);
        cudaEventRecord(b.ev, s);
        sv->slot_busy[slot] = true;
        sv->inflight.push_back(b);
        sv->batches++;
        sv->batched_reqs += take.size();
        sv->batched_keys += g.total[0] + g.total[1];
        worked = true;
      }
    }
    // 3. build admission by free device memory (as last sampled: at start
    // and after every build)
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      while (!sv->pending_builds.empty()) {
        Req *r = sv->pending_builds.front();
        const u64 free_b = sv->free_mem.load();
        const u64 need = build_footprint(r->n, r->gamma);
        const u64 held = sv->build_reserved.load();
        if (free_b < held + need + sv->mem_reserve) break;  // wait for memory
        sv->build_reserved += need;
        sv->pending_builds.pop_front();
        sv->build_queue.push_back(r);
        sv->cv_build.notify_one();
        worked = true;
      }
    }
    if (!worked) std::this_thread::yield();
  }
}

static void build_worker(mphf_server *sv) {
  cudaSetDevice(sv->device);
  // builds run at the lowest stream priority: when SMs free up, the block
  // scheduler takes the pending CTAs of lookup batches first
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  cudaStream_t s;
  cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, least);
  for (;;) {
    Req *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_build.wait(lk, [&] { return sv->stop.load() || !sv->build_queue.empty(); });
      if (sv->build_queue.empty()) break;
      r = sv->build_queue.front();
      sv->build_queue.pop_front();
    }
    mphf_t *h = nullptr;
    int rc = mphf_build((const uint64_t *)r->keys, r->n, r->gamma, r->L, r->seed, s, &h);
    const double t = now_s();
    {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) sv->free_mem.store(free_b);
      else cudaGetLastError();
    }
    sv->build_reserved -= build_footprint(r->n, r->gamma);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      r->status = rc;
      r->built = h;
      r->t_done = t;
      r->done = true;
    }
    sv->builds_done++;
    sv->cv_done.notify_all();
  }
  cudaStreamDestroy(s);
}

}  // namespace bbh

using namespace bbh;

extern "C" {

int mphf_server_create(uint64_t max_batch_keys, uint32_t max_batch_reqs, int max_inflight,
                       int build_workers, uint64_t mem_reserve_bytes, mphf_server_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (max_batch_keys == 0 || max_batch_reqs == 0 || max_inflight < 1 || max_inflight > 16 ||
      build_workers < 0 || build_workers > 16)
    return MPHF_EINVAL;
  mphf_server *sv = new (std::nothrow) mphf_server();
  if (!sv) return MPHF_ENOMEM;
  sv->max_batch_keys = max_batch_keys;
  sv->max_batch_reqs = max_batch_reqs;
  sv->max_inflight = max_inflight;
  sv->build_workers = build_workers;
  sv->mem_reserve = mem_reserve_bytes;
  cudaGetDevice(&sv->device);
  int rc = MPHF_OK;
  // lookup batches at the highest stream priority (builds take the lowest)
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  for (int i = 0; i < 2 && rc == MPHF_OK; i++)
    if (cudaStreamCreateWithPriority(&sv->lstream[i], cudaStreamNonBlocking, greatest) !=
        cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "cudaStreamCreate");
  sv->dtab.resize(max_inflight);
  sv->htab.resize(max_inflight, nullptr);
  sv->slot_busy.assign(max_inflight, false);
  sv->slot_ev0.assign(max_inflight, nullptr);
  sv->slot_ev.assign(max_inflight, nullptr);
  for (int i = 0; i < max_inflight && rc == MPHF_OK; i++)
    if (cudaEventCreate(&sv->slot_ev0[i]) != cudaSuccess ||
        cudaEventCreate(&sv->slot_ev[i]) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "server events");
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) sv->free_mem.store(free_b);
    else cudaGetLastError();
  }
  for (int i = 0; i < max_inflight && rc == MPHF_OK; i++) {
    if (cudaMalloc(&sv->dtab[i].p, sizeof(ReqDev) * max_batch_reqs) != cudaSuccess ||
        cudaMallocHost((void **)&sv->htab[i], sizeof(ReqDev) * max_batch_reqs) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "server tables");
  }
  if (rc != MPHF_OK) {
    mphf_server_destroy(sv);
    return rc;
  }
  sv->sched = std::thread(scheduler, sv);
  for (int i = 0; i < build_workers; i++) sv->workers.emplace_back(build_worker, sv);
  *out = sv;
  return MPHF_OK;
}

void mphf_server_destroy(mphf_server_t *sv) {
  if (!sv) return;
  sv->stop = true;
  sv->cv_build.notify_all();
  if (sv->sched.joinable()) sv->sched.join();
  for (auto &t : sv->workers)
    if (t.joinable()) t.join();
  for (auto &b : sv->inflight) cudaEventSynchronize(b.ev);
  for (auto e : sv->slot_ev0)
    if (e) cudaEventDestroy(e);
  for (auto e : sv->slot_ev)
    if (e) cudaEventDestroy(e);
  for (auto &kv : sv->reqs) {  // requests never waited for: their builds are released
    if (kv.second->built) mphf_free(kv.second->built);
    delete kv.second;
  }
  for (auto &d : sv->dtab)
    if (d.p) cudaFree(d.p);
  for (auto *h : sv->htab)
    if (h) cudaFreeHost(h);
  for (auto s : sv->lstream)
    if (s) cudaStreamDestroy(s);
  delete sv;
}

int mphf_server_submit_lookup(mphf_server_t *sv, mphf_t *h, const uint64_t *d_keys, uint64_t n,
                              uint64_t *d_out, uint64_t *req_id) {
  if (!sv || !h || !req_id || (n && (!d_keys || !d_out))) return MPHF_EINVAL;
  if (h->L_used == 0 && n) return MPHF_EINVAL;  // empty function: nothing to look up
  int rc = ensure_lookup_desc(h);
  if (rc != MPHF_OK) return rc;
  Req *r = new (std::nothrow) Req();
  if (!r) return MPHF_ENOMEM;
  r->kind = 0;
  r->h = h;
  r->keys = (const u64 *)d_keys;
  r->out = (u64 *)d_out;
  r->n = n;
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->id = sv->next_id++;
  sv->reqs[r->id] = r;
  if (n == 0) {
    r->done = true;
    r->t_done = r->t_submit;
  } else {
    sv->pending_lookups.push_back(r);
  }
  *req_id = r->id;
  return MPHF_OK;
}

int mphf_server_submit_build(mphf_server_t *sv, const uint64_t *d_keys, uint64_t n, double gamma,
                             uint32_t levels, uint64_t seed, uint64_t *req_id) {
  if (!sv || !req_id || sv->build_workers == 0) return MPHF_EINVAL;
  if (!(gamma >= 1.0) || isinf(gamma) || levels < 1 || levels > MPHF_MAX_LEVELS ||
      (n && !d_keys))
    return MPHF_EINVAL;
  Req *r = new (std::nothrow) Req();
  if (!r) return MPHF_ENOMEM;
  r->kind = 1;
  r->keys = (const u64 *)d_keys;
  r->n = n;
  r->gamma = gamma;
  r->L = levels;
  r->seed = seed;
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->id = sv->next_id++;
  sv->reqs[r->id] = r;
  sv->pending_builds.push_back(r);
  *req_id = r->id;
  return MPHF_OK;
}

int mphf_server_wait(mphf_server_t *sv, uint64_t req_id, double timeout_s, int *status,
                     double *latency_s, mphf_t **built) {
  if (!sv) return MPHF_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(req_id);
  if (it == sv->reqs.end()) return MPHF_EINVAL;
  Req *r = it->second;
  const auto deadline = clk::now() + std::chrono::duration<double>(timeout_s);
  while (!r->done) {
    if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
      return MPHF_ETIMEOUT;
  }
  if (status) *status = r->status;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  if (built) *built = r->built;
  else if (r->built) mphf_free(r->built);  // a build nobody takes is released here
  sv->reqs.erase(it);
  delete r;
  return MPHF_OK;
}

int mphf_server_stats(mphf_server_t *sv, uint64_t *batches, uint64_t *requests, uint64_t *keys,
                      uint64_t *builds) {
  if (!sv) return MPHF_EINVAL;
  if (batches) *batches = sv->batches.load();
  if (requests) *requests = sv->batched_reqs.load();
  if (keys) *keys = sv->batched_keys.load();
  if (builds) *builds = sv->builds_done.load();
  return MPHF_OK;
}

int mphf_server_latency_parts(mphf_server_t *sv, double *p50, double *p99) {
  if (!sv || !p50 || !p99) return MPHF_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  std::vector<double> *parts[3] = {&sv->part_queue, &sv->part_gpu, &sv->part_rest};
  for (int k = 0; k < 3; k++) {
    std::vector<double> &v = *parts[k];
    p50[k] = p99[k] = 0.0;
    if (v.empty()) continue;
    std::vector<double> w = v;
    std::sort(w.begin(), w.end());
    p50[k] = w[(size_t)(0.50 * (w.size() - 1))];
    p99[k] = w[(size_t)(0.99 * (w.size() - 1))];
    v.clear();
  }
  return MPHF_OK;
}

// Open-loop synthetic load: Poisson arrivals at `rate_hz` for `duration_s`;
// each lookup picks one of `nh` handles uniformly and a batch size
// log-uniform in [bmin, bmax] of consecutive member keys at a random offset of
// that handle's key array (keys[i], count[i]); outputs go to a device scratch
// array of `out_cap` words used as a ring.  A fraction `build_frac` of the
// arrivals are builds over a prefix of size log-uniform in [nbmin, nbmax] of
// build_keys (device, n_build_keys available).  Latencies of completed
// lookups are written to lat_out (up to lat_cap); counts go to *_out.
int mphf_server_loadgen(mphf_server_t *sv, mphf_t *const *hs, const uint64_t *const *keys,
                        const uint64_t *count, uint32_t nh, double rate_hz, double duration_s,
                        double bmin, double bmax, uint64_t *d_out, uint64_t out_cap,
                        double build_frac, const uint64_t *build_keys, uint64_t n_build_keys,
                        double nbmin, double nbmax, double gamma, uint64_t seed, double *lat_out,
                        uint64_t lat_cap, uint64_t *n_lookups_out, uint64_t *n_keys_out,
                        uint64_t *n_builds_out, double *elapsed_out) {
  if (!sv || !hs || !keys || !count || nh == 0 || !(rate_hz > 0) || !(duration_s > 0) ||
      !d_out || out_cap < (uint64_t)bmax || !(bmin >= 1) || bmax < bmin)
    return MPHF_EINVAL;
  for (uint32_t i = 0; i < nh; i++) {
    int rc = ensure_lookup_desc(hs[i]);
    if (rc != MPHF_OK) return rc;
  }
  std::mt19937_64 rng(seed);
  std::exponential_distribution<double> gap(rate_hz);
  std::uniform_real_distribution<double> u01(0.0, 1.0);
  struct Pending {
    uint64_t id;
    int kind;
    u64 n;
  };
  std::vector<Pending> ids;
  ids.reserve((size_t)(rate_hz * duration_s * 1.2) + 16);
  const double t0 = now_s();
  double next = t0;
  u64 ring = 0, nk = 0, nl = 0, nb = 0;
  while (next - t0 < duration_s) {
    while (now_s() < next) {
    }
    uint64_t id = 0;
    if (build_frac > 0 && build_keys && u01(rng) < build_frac) {
      u64 n = (u64)floor(exp(u01(rng) * (log(nbmax) - log(nbmin)) + log(nbmin)));
      if (n > n_build_keys) n = n_build_keys;
      if (mphf_server_submit_build(sv, build_keys, n, gamma, 25, seed, &id) == MPHF_OK) {
        ids.push_back({id, 1, n});
        nb++;
      }
    } else {
      const uint32_t h = (uint32_t)(u01(rng) * nh) % nh;
      u64 b = (u64)floor(exp(u01(rng) * (log(bmax) - log(bmin)) + log(bmin)));
      if (b > count[h]) b = count[h];
      if (b == 0) b = 1;
      const u64 off = (u64)(u01(rng) * (double)(count[h] - b + 1));
      if (ring + b > out_cap) ring = 0;
      if (mphf_server_submit_lookup(sv, hs[h], keys[h] + off, b, d_out + ring, &id) == MPHF_OK) {
        ids.push_back({id, 0, b});
        nl++;
        nk += b;
      }
      ring += b;
    }
    next += gap(rng);
  }
  u64 nlat = 0;
  int rc = MPHF_OK;
  for (auto &p : ids) {
    int st = 0;
    double lat = 0;
    mphf_t *built = nullptr;
    int w = mphf_server_wait(sv, p.id, 600.0, &st, &lat, &built);
    if (w != MPHF_OK) {
      rc = w;
      continue;
    }
    if (st != MPHF_OK) rc = st;
    if (p.kind == 0 && lat_out && nlat < lat_cap) lat_out[nlat++] = lat;
    if (built) mphf_free(built);
  }
  if (elapsed_out) *elapsed_out = now_s() - t0;
  if (n_lookups_out) *n_lookups_out = nl;
  if (n_keys_out) *n_keys_out = nk;
  if (n_builds_out) *n_builds_out = nb;
  return rc;
}

int mphf_lookup_multi(mphf_t *const *hs, const uint64_t *const *d_keys, uint64_t *const *d_out,
                      const uint64_t *counts, uint32_t nreq, void *stream) {
  if (nreq == 0) return MPHF_OK;
  if (!hs || !d_keys || !d_out || !counts) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<ReqDev> t(nreq);
  for (uint32_t i = 0; i < nreq; i++) {
    if (!hs[i] || (counts[i] && (!d_keys[i] || !d_out[i]))) return MPHF_EINVAL;
    if (hs[i]->L_used == 0 && counts[i]) return MPHF_EINVAL;
    int rc = ensure_lookup_desc(hs[i]);
    if (rc != MPHF_OK) return rc;
  }
  const TableGroups g = fill_table(
      t.data(), nreq, [&](size_t i) { return (const mphf_t *)hs[i]; },
      [&](size_t i) { return (const u64 *)d_keys[i]; }, [&](size_t i) { return (u64 *)d_out[i]; },
      [&](size_t i) { return (u64)counts[i]; });
  DevBuf d;
  int rc = dev_alloc(d, sizeof(ReqDev) * nreq, s);
  if (rc != MPHF_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(d.p, t.data(), sizeof(ReqDev) * nreq, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) rc = launch_lookup_multi((const ReqDev *)d.p, g, s);
  else rc = cuda_fail(e, "cudaMemcpyAsync(requests)");
  dev_free(d, s);  // stream-ordered: released after the kernel
  return rc;        // (a pageable copy has taken the table before returning)
}

}  // extern "C"
