// lookup.cu -- batched queries (Algorithm 3 with the minimal index of
// Sec. 2.2.3 and the ranks of Sec. 3.1).
//
// A key needs e^{1/gamma} level probes on average but up to L; a warp that
// kept 32 keys in lock-step would idle most lanes while its slowest key walks
// down the levels.  Instead every lane owns kSlots independent query slots,
// each with its own (key, output index, level).  Each round every active slot
// probes its current level with one load of the record holding its bit (a
// 256-bit sector or an 8-byte unit, sector.cuh: the A word and a count of the
// ones before it come together); a slot whose bit is set finishes its rank
// from those registers and retires, the others move to the next level, and
// retired slots are refilled from the warp's stream of input keys.  So lanes
// stay busy, each lane keeps kSlots independent loads in flight, and a placed
// key costs one memory request per level probed.
#include <cuda_runtime.h>
#include <stdlib.h>

#include "common.cuh"
#include "sector.cuh"

namespace bbh {

static constexpr int kLookupThreads = 256;

struct LevelTable {
  u64 s[MPHF_MAX_LEVELS];
  u64 m[MPHF_MAX_LEVELS];
  u64 off[MPHF_MAX_LEVELS];
};

struct LookupArgs {
  const unsigned *S;  // sectors: A with its ranks
  const u64 *SB;      // ones before each superblock
  const u64 *fb;
  u64 n_fb;
  u64 N;
  uint32_t L_used;
};

__device__ __forceinline__ u64 fallback_index(const LookupArgs &a, u64 x) {
  u64 lo = 0, hi = a.n_fb;
  while (lo < hi) {
    u64 mid = lo + ((hi - lo) >> 1);
    if (__ldg(a.fb + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  if (lo < a.n_fb && __ldg(a.fb + lo) == x) return a.N - a.n_fb + lo;
  return MPHF_NOT_FOUND;
}

// kNarrow: every m_d < 2^32 and A short enough that bit g's word index
// g >> kQShift is below 2^32 (A below 2^36 bits); then a probe's position
// arithmetic is 32-bit: with off_d a multiple of 64,
//   g >> kQShift = (off_d >> kQShift) + (p >> kQShift),  g & mask = p & mask.
template <int kSlots, int W, bool kNarrow>
__global__ void __launch_bounds__(kLookupThreads)
k_lookup(const u64 *__restrict__ keys, u64 n, u64 csz, u64 *__restrict__ out, LookupArgs a,
         LevelTable t) {
  using LW = Lay<W>;
  __shared__ u64 ts[MPHF_MAX_LEVELS], tm[MPHF_MAX_LEVELS], toff[MPHF_MAX_LEVELS];
  __shared__ unsigned tm32[MPHF_MAX_LEVELS], toq[MPHF_MAX_LEVELS];
  for (unsigned i = threadIdx.x; i < a.L_used; i += kLookupThreads) {
    ts[i] = t.s[i];
    tm[i] = t.m[i];
    toff[i] = t.off[i];
    tm32[i] = (unsigned)t.m[i];
    toq[i] = (unsigned)(t.off[i] >> LW::kQShift);
  }
  __syncthreads();

  const unsigned lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const u64 nchunks = (n + csz - 1) / csz;
  const u64 warp_id = ((u64)blockIdx.x * kLookupThreads + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * kLookupThreads) >> 5;
  u64 chunk = warp_id;
  u64 cursor = chunk * csz;
  u64 cend = chunk < nchunks ? min(cursor + csz, n) : cursor;
  bool more = chunk < nchunks;

  u64 x[kSlots], idx[kSlots];
  unsigned lvl[kSlots];
  bool act[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; s++) {
    act[s] = false;
    lvl[s] = 0;
    x[s] = 0;
    idx[s] = 0;
  }

  for (;;) {
    // refill retired slots from the warp's input stream (warp-uniform
    // control); while the current chunk holds a key for every free slot they
    // are ranked lane by lane, slot 0 first, and filled in one pass
    unsigned rk[kSlots], nfree = 0;
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      const unsigned need = __ballot_sync(0xffffffffu, !act[s]);
      rk[s] = nfree + __popc(need & lt);
      nfree += __popc(need);
    }
    if (nfree && cend - cursor >= nfree) {
#pragma unroll
      for (int s = 0; s < kSlots; s++) {
        if (!act[s]) {
          const u64 i = cursor + rk[s];
          idx[s] = i;
          x[s] = __ldcs(keys + i);
          lvl[s] = 0;
          act[s] = true;
        }
      }
      cursor += nfree;
    }
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
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
        if (mine) {
          idx[s] = cursor + r;
          x[s] = __ldcs(keys + cursor + r);
          lvl[s] = 0;
          act[s] = true;
        }
        const unsigned taken = __ballot_sync(0xffffffffu, mine);
        need &= ~taken;
        cursor += __popc(taken);
      }
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < kSlots; s++) any |= act[s];
    if (!__any_sync(0xffffffffu, any)) break;

    // one probe per active slot: issue all loads, then resolve
    typename LW::Pos p[kSlots];
    typename LW::Data v[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      if (act[s]) {
        const unsigned d = lvl[s];
        if (kNarrow) {
          // reduce_range for m < 2^32, kept in 32 bits
          const u64 h = mix64(x[s] ^ ts[d]);
          const unsigned m32 = tm32[d];
          const u64 lo = ((u64)(unsigned)h * m32) >> 32;
          const unsigned pd = (unsigned)(((u64)(unsigned)(h >> 32) * m32 + lo) >> 32);
          p[s] = LW::pos_q(toq[d] + (pd >> LW::kQShift), pd & ((1u << LW::kQShift) - 1u));
        } else {
          p[s] = LW::pos(toff[d] + level_pos(x[s], ts[d], tm[d]));
        }
        v[s] = LW::load(a.S, p[s]);
      }
    }
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      if (act[s]) {
        unsigned w = 0;
        if (LW::hit(v[s], p[s], w)) {
          __stcs(out + idx[s], LW::rank(v[s], p[s], w, a.SB));
          act[s] = false;
        } else if (++lvl[s] >= a.L_used) {
          __stcs(out + idx[s], a.n_fb ? fallback_index(a, x[s]) : MPHF_NOT_FOUND);
          act[s] = false;
        }
      }
    }
  }
}

static void fill_tables(const mphf_t *h, LookupArgs &a, LevelTable &t) {
  a.S = (const unsigned *)h->S.p;
  a.SB = (const u64 *)h->SB.p;
  a.fb = (const u64 *)h->fb.p;
  a.n_fb = h->n_fb;
  a.N = h->N;
  a.L_used = h->L_used;
  for (uint32_t d = 0; d < MPHF_MAX_LEVELS; d++) {
    t.s[d] = d < h->L_used ? h->s[d] : 0;
    t.m[d] = d < h->L_used ? h->m[d] : 0;
    t.off[d] = d < h->L_used ? h->off[d] : 0;
  }
}

// Query slots per lane: 2 for every layout.  (8-byte units would leave room
// for more, but measured on a GB300 3, 4 or 6 slots run slower than 2.)
static constexpr int kUnitSlots = 2;

template <int SLOTS, int W, bool NARROW>
static int launch_lookup(const u64 *keys, u64 n, u64 *out, const LookupArgs &a,
                         const LevelTable &t, cudaStream_t s) {
  // one wave of resident CTAs: warps take chunks in a fixed order, so a
  // second wave would only start after the first has drained
  static unsigned mb_dev[64] = {0};  // per device
  unsigned &mb = mb_dev[cur_device()];
  if (!mb) mb = resident_grid(k_lookup<SLOTS, W, NARROW>, kLookupThreads, 0);
  const u64 csz = lookup_chunk(n, (u64)mb * (kLookupThreads / 32));
  const u64 nwarps_needed = (n + csz - 1) / csz;
  const unsigned per_block = kLookupThreads / 32;
  u64 grid = (nwarps_needed + per_block - 1) / per_block;
  if (grid > mb) grid = mb;
  if (grid < 1) grid = 1;
  LaunchScope ls("lookup", s);
  k_lookup<SLOTS, W, NARROW><<<(unsigned)grid, kLookupThreads, 0, s>>>(keys, n, csz, out, a,
                                                                       t);
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

int lookup_impl(const mphf_t *h, const u64 *keys, u64 n, u64 *out, cudaStream_t s) {
  LookupArgs a;
  LevelTable t;
  fill_tables(h, a, t);
  const bool narrow = narrow_positions(h);
  if (h->sw == kSectWordsMini)
    return narrow ? launch_lookup<2, kSectWordsMini, true>(keys, n, out, a, t, s)
                  : launch_lookup<2, kSectWordsMini, false>(keys, n, out, a, t, s);
  if (h->sw == kUnitBits)
    return narrow ? launch_lookup<kUnitSlots, kUnitBits, true>(keys, n, out, a, t, s)
                  : launch_lookup<kUnitSlots, kUnitBits, false>(keys, n, out, a, t, s);
  return narrow ? launch_lookup<2, kSectWords, true>(keys, n, out, a, t, s)
                : launch_lookup<2, kSectWords, false>(keys, n, out, a, t, s);
}

}  // namespace bbh

int bbh::g_lookup_wide = 0;

using namespace bbh;

extern "C" int mphf_debug_lookup_wide(int on) {
  g_lookup_wide = on ? 1 : 0;
  return MPHF_OK;
}

extern "C" int mphf_lookup(const mphf_t *h, const uint64_t *d_keys, uint64_t n, uint64_t *d_out,
                           void *stream) {
  if (!h) return MPHF_EINVAL;
  if (n == 0) return MPHF_OK;
  if (!d_keys || !d_out || (((uintptr_t)d_keys | (uintptr_t)d_out) & 7)) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->L_used == 0 && h->n_fb == 0) {  // empty function: every key is a miss
    MPHF_CUDA(cudaMemsetAsync(d_out, 0xff, n * 8, s));
    return MPHF_OK;
  }
  return lookup_impl(h, (const u64 *)d_keys, n, (u64 *)d_out, s);
}

// Large batches run as a three-stage pipeline over chunks of the batch: the
// copy in of chunk c+1 (side stream ci), the lookup of chunk c (the caller's
// stream) and the copy out of chunk c-1 (side stream co) overlap, so the
// batch costs about one pass over the host link instead of two plus the
// kernel.  The D2H copy of chunk c is enqueued after the lookup of chunk c+1,
// so that a pageable h_out (whose copy blocks the host) still leaves the next
// lookup queued.
extern "C" int mphf_lookup_host(const mphf_t *h, const uint64_t *h_keys, uint64_t n,
                                uint64_t *h_out, void *stream) {
  if (!h) return MPHF_EINVAL;
  if (n == 0) return MPHF_OK;
  if (!h_keys || !h_out) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf kb, ob;
  int rc = dev_alloc(kb, n * 8, s);
  if (rc != MPHF_OK) return rc;
  rc = dev_alloc(ob, n * 8, s);
  if (rc != MPHF_OK) {
    dev_free(kb, s);
    return rc;
  }
  const u64 chunk = feed_chunk(n);
  cudaError_t e = cudaSuccess;
  if (!chunk) {
    e = cudaMemcpyAsync(kb.p, h_keys, n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      rc = mphf_lookup(h, (const uint64_t *)kb.p, n, (uint64_t *)ob.p, stream);
      if (rc == MPHF_OK) e = cudaMemcpyAsync(h_out, ob.p, n * 8, cudaMemcpyDeviceToHost, s);
    }
  } else {
    SideSet ss;
    rc = side_set(2, &ss);
    if (rc != MPHF_OK) {
      dev_free(kb, s);
      dev_free(ob, s);
      return rc;
    }
    cudaStream_t ci = ss.s[0], co = ss.s[1];
    cudaEvent_t ev_in = ss.ev[0], ev_k = ss.ev[1];
    u64 *dk = (u64 *)kb.p, *dout = (u64 *)ob.p;
    // both buffers were allocated in s's order: the side streams start after
    e = cudaEventRecord(ev_in, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ci, ev_in, 0);
    u64 prev0 = 0, prevn = 0;  // chunk whose copy out is still to be enqueued
    for (u64 c0 = 0; c0 < n && e == cudaSuccess && rc == MPHF_OK; c0 += chunk) {
      const u64 cn = n - c0 < chunk ? n - c0 : chunk;
      e = cudaMemcpyAsync(dk + c0, (const u64 *)h_keys + c0, cn * 8, cudaMemcpyHostToDevice, ci);
      if (e == cudaSuccess) e = cudaEventRecord(ev_in, ci);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_in, 0);
      if (e != cudaSuccess) break;
      rc = mphf_lookup(h, (const uint64_t *)(dk + c0), cn, (uint64_t *)(dout + c0), stream);
      if (rc != MPHF_OK) break;
      e = cudaEventRecord(ev_k, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(co, ev_k, 0);
      if (e == cudaSuccess && prevn)
        e = cudaMemcpyAsync((u64 *)h_out + prev0, dout + prev0, prevn * 8, cudaMemcpyDeviceToHost, co);
      prev0 = c0;
      prevn = cn;
    }
    if (e == cudaSuccess && rc == MPHF_OK && prevn)
      e = cudaMemcpyAsync((u64 *)h_out + prev0, dout + prev0, prevn * 8, cudaMemcpyDeviceToHost, co);
    // everything enqueued on the side streams is ordered before the frees
    cudaEventRecord(ev_in, ci);
    cudaStreamWaitEvent(s, ev_in, 0);
    cudaEventRecord(ev_k, co);
    cudaStreamWaitEvent(s, ev_k, 0);
  }
  dev_free(kb, s);
  dev_free(ob, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "mphf_lookup_host");
  return rc;
}
