// api.cu -- handle lifetime, introspection, error text, device memory,
// launch accounting / per-kernel event timing, and the synthetic key generator.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stddef.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "sector.cuh"

namespace bbh {

static std::mutex g_err_mu;
static char g_err_text[512] = "no error";

void set_cuda_error(cudaError_t e, const char *where) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  snprintf(g_err_text, sizeof(g_err_text), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
}

int cuda_fail(cudaError_t e, const char *where) {
  set_cuda_error(e, where);
  return MPHF_ECUDA;
}

// ---------------------------------------------------------------------------
// Launch accounting and optional per-kernel event timing.
// ---------------------------------------------------------------------------
static std::atomic<u64> g_launches{0};
static std::atomic<int> g_profile_on{0};
static std::mutex g_prof_mu;
struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof;           // recorded launches
static std::vector<cudaEvent_t> g_event_pool; // reusable events
static thread_local int t_open = -1;          // index of the open record of this thread

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void launch_begin(const char *name, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_profile_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{name, take_event(), take_event()};
  cudaEventRecord(r.a, s);
  g_prof.push_back(r);
  t_open = (int)g_prof.size() - 1;
}

void add_launches(u64 n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void launch_end(cudaStream_t s) {
  if (t_open < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (t_open < (int)g_prof.size()) cudaEventRecord(g_prof[t_open].b, s);
  t_open = -1;
}

// Device memory comes from the device's default stream-ordered pool, which
// keeps every block it has mapped once the library has used it (release
// threshold: unlimited), so a build that needs 120 GB of scratch (1e10 keys)
// finds it again on its next call instead of mapping it from the driver anew.
// A threshold at the most memory held at once is not enough: the cached
// blocks of one workload do not match the sizes another asks for, the pool
// then holds more than that peak and releases (and re-maps) tens of GB at
// every synchronisation.  mphf_pool_trim returns the unused part.
static std::atomic<int> g_pool_set[64];

static void pool_keep(int dev, u64 bytes) {
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    u64 thr = bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  } else {
    cudaGetLastError();
  }
}

int dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s) {
  b.p = nullptr;
  b.bytes = bytes;
  if (bytes == 0) return MPHF_OK;
  const int dev = cur_device();
  if (g_pool_set[dev].load() == 0) {
    int z = 0;
    if (g_pool_set[dev].compare_exchange_strong(z, 1)) pool_keep(dev, ~0ull);
  }
  cudaError_t e = cudaMallocAsync(&b.p, bytes, s);
  if (e != cudaSuccess) {
    b.p = nullptr;
    b.bytes = 0;
    cudaGetLastError();
    set_cuda_error(e, "cudaMallocAsync");
    return MPHF_ENOMEM;
  }
  return MPHF_OK;
}

static std::mutex g_handle_mu;
static const size_t kHandleFreeMax = 1u << 16;
static mphf *g_handle_free[kHandleFreeMax];
static size_t g_handle_nfree = 0;

mphf *handle_new() {
  mphf *h = nullptr;
  if (!handle_new_n(1, &h)) return nullptr;
  return h;
}

bool handle_new_n(unsigned n, mphf **out, bool zero_tables) {
  static const mphf proto;
  unsigned got = 0;
  {
    std::lock_guard<std::mutex> lk(g_handle_mu);
    while (got < n && g_handle_nfree) out[got++] = g_handle_free[--g_handle_nfree];
  }
  for (unsigned i = 0; i < got; i++) {
    if (zero_tables) new (out[i]) mphf();
    else memcpy((void *)out[i], (const void *)&proto, offsetof(mphf, n));
  }
  for (; got < n; got++) {
    out[got] = new (std::nothrow) mphf();
    if (!out[got]) {
      for (unsigned i = 0; i < got; i++) handle_delete(out[i]);
      return false;
    }
  }
  return true;
}

void handle_delete(mphf *h) {
  if (!h) return;
  {
    std::lock_guard<std::mutex> lk(g_handle_mu);
    if (g_handle_nfree < kHandleFreeMax) {
      g_handle_free[g_handle_nfree++] = h;
      return;
    }
  }
  delete h;
}

void dev_free(DevBuf &b, cudaStream_t s) {
  if (b.p) cudaFreeAsync(b.p, s);
  b.p = nullptr;
  b.bytes = 0;
}

}  // namespace bbh

extern "C" int mphf_pool_trim(void) {
  using namespace bbh;
  const int dev = cur_device();
  cudaMemPool_t pool;
  MPHF_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  MPHF_CUDA(cudaDeviceSynchronize());
  MPHF_CUDA(cudaMemPoolTrimTo(pool, 0));
  return MPHF_OK;
}

namespace bbh {

// About 16 chunks of at least 2^20 keys: the first chunk's copy is the
// pipeline's fill time, so chunks stay small next to the whole copy, but each
// still carries far more than a launch's worth of work.
u64 feed_chunk(u64 n) {
  const u64 kMin = 1ull << 20;
  if (n < 4 * kMin) return 0;
  u64 c = (n + 15) / 16;
  c = (c + 4095) & ~4095ull;
  return c < kMin ? kMin : c;
}

int side_set(size_t n_events, SideSet *out) {
  struct Pool {
    cudaStream_t s[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev;
  };
  thread_local std::vector<Pool> pools;  // by device; kept for the thread's life
  int dev = 0;
  MPHF_CUDA(cudaGetDevice(&dev));
  if ((int)pools.size() <= dev) pools.resize(dev + 1);
  Pool &p = pools[dev];
  for (cudaStream_t &x : p.s)
    if (!x) MPHF_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  while (p.ev.size() < n_events) {
    cudaEvent_t e = nullptr;
    MPHF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    p.ev.push_back(e);
  }
  out->s[0] = p.s[0];
  out->s[1] = p.s[1];
  out->ev = p.ev.data();
  return MPHF_OK;
}

int KeyFeed::ensure(u64 upto, cudaStream_t st) {
  if (upto > n) upto = n;
  if (issued >= upto) return MPHF_OK;
  while (issued < upto) {
    const u64 c = chunk && upto - issued > chunk ? chunk : upto - issued;
    MPHF_CUDA(cudaMemcpyAsync(d + issued, h + issued, c * 8, cudaMemcpyHostToDevice, cs));
    issued += c;
  }
  MPHF_CUDA(cudaEventRecord(ev, cs));
  MPHF_CUDA(cudaStreamWaitEvent(st, ev, 0));
  if (issued == n && hq && !q_issued) return issue_queries();
  return MPHF_OK;
}

int KeyFeed::issue_queries() {
  q_issued = true;
  u64 i = 0;
  for (u64 c0 = 0; c0 < nq; c0 += qchunk, i++) {
    const u64 c = nq - c0 < qchunk ? nq - c0 : qchunk;
    MPHF_CUDA(cudaMemcpyAsync(dq + c0, hq + c0, c * 8, cudaMemcpyHostToDevice, cs));
    MPHF_CUDA(cudaEventRecord(qev[i], cs));
  }
  return MPHF_OK;
}

// ---------------------------------------------------------------------------
// Synthetic keys: output j of SplitMix64 started at `seed` is
// fin(seed + (j + 1) * 0x9E3779B97F4A7C15), fin = the generator's finalizer.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_keygen(u64 *__restrict__ out, u64 n, u64 seed, u64 start) {
  const u64 G = 0x9E3779B97F4A7C15ull;
  u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    out[i] = mix64(seed + (start + i + 1) * G);
  }
}

}  // namespace bbh

using namespace bbh;

extern "C" {

const char *mphf_strerror(int code) {
  switch (code) {
    case MPHF_OK: return "ok";
    case MPHF_EINVAL: return "invalid argument";
    case MPHF_ENOMEM: return "out of memory";
    case MPHF_EDUPLICATE: return "duplicate keys";
    case MPHF_ECUDA: return "CUDA error";
    case MPHF_ETIMEOUT: return "device wait timed out";
    case MPHF_EINTERNAL: return "internal consistency check failed";
    default: return "unknown error";
  }
}

const char *mphf_last_cuda_error(void) { return g_err_text; }

int mphf_abi_version(void) { return 2; }

void mphf_free(mphf_t *h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  if (h->ldesc.p) cudaFree(h->ldesc.p);
  if (h->shared) {
    release_shared(h->shared);
  } else {
    dev_free(h->S, 0);
    dev_free(h->SB, 0);
    dev_free(h->fb, 0);
  }
  if (prev != h->device) cudaSetDevice(prev);
  handle_delete(h);
}

// Sec. 3.1's size with one 64-bit counter per 512 bits of A, or per 1024
// bits for the minirank layout (Sec. 4.3).
double mphf_bits_per_key(const mphf_t *h) {
  if (!h || h->N == 0) return 0.0;
  const u64 block = h->sw == kSectWordsMini ? 2 * MPHF_RANK_BLOCK : MPHF_RANK_BLOCK;
  const u64 counters = (h->M + block - 1) / block;
  double bits = (double)h->M + 64.0 * (double)counters + 64.0 * (double)h->n_fb;
  return bits / (double)h->N;
}

uint64_t mphf_num_keys(const mphf_t *h) { return h ? h->N : 0; }
int mphf_num_levels(const mphf_t *h, uint32_t *levels) {
  if (!h || !levels) return MPHF_EINVAL;
  *levels = h->L_used;
  return MPHF_OK;
}
uint64_t mphf_total_bits(const mphf_t *h) { return h ? h->M : 0; }
uint64_t mphf_num_rank(const mphf_t *h) { return h ? h->n_rank : 0; }
uint64_t mphf_num_fallback(const mphf_t *h) { return h ? h->n_fb : 0; }

int mphf_level_info(const mphf_t *h, uint32_t d, uint64_t *n_d, uint64_t *m_d, uint64_t *off_d,
                    uint64_t *s_d) {
  if (!h || d >= h->L_used) return MPHF_EINVAL;
  if (n_d) *n_d = h->n[d];
  if (m_d) *m_d = h->m[d];
  if (off_d) *off_d = h->off[d];
  if (s_d) *s_d = h->s[d];
  return MPHF_OK;
}

static int copy_out(const mphf_t *h, const DevBuf &b, uint64_t *dst, uint64_t count,
                    uint64_t expect) {
  if (!h || (count && !dst) || count != expect) return MPHF_EINVAL;
  if (!count) return MPHF_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  cudaError_t e = cudaMemcpy(dst, b.p, count * sizeof(uint64_t), cudaMemcpyDeviceToHost);
  if (prev != h->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(D2H)");
  return MPHF_OK;
}

// A comes back out of the sectors: each sector (unit) holds a run of whole
// bytes of A at a fixed offset, so one strided copy gathers them.
int mphf_copy_bits(const mphf_t *h, uint64_t *h_words, uint64_t count) {
  if (!h || (count && !h_words) || count != h->M / 64) return MPHF_EINVAL;
  if (!count) return MPHF_OK;
  const AGather g = a_gather(h->M, h->sw);
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  const char *src = (const char *)h->S.p + g.offset;
  char *dst = (char *)h_words;
  cudaError_t e = cudaSuccess;
  if (g.full) e = cudaMemcpy2D(dst, g.width, src, g.pitch, g.width, g.full, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && g.rest)
    e = cudaMemcpy(dst + g.full * g.width, src + g.full * g.pitch, g.rest, cudaMemcpyDeviceToHost);
  if (prev != h->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2D(A from sectors)");
  return MPHF_OK;
}

// The paper's checkpoints (ones before bit 512 b), evaluated from the sectors.
int mphf_copy_rank(const mphf_t *h, uint64_t *h_rank, uint64_t count) {
  if (!h || (count && !h_rank) || count != h->n_rank) return MPHF_EINVAL;
  if (!count) return MPHF_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  DevBuf tmp;
  int rc = dev_alloc(tmp, count * 8, 0);
  if (rc == MPHF_OK) {
    rc = sector_checkpoints((const unsigned *)h->S.p, (const u64 *)h->SB.p, h->sw, count,
                            (u64 *)tmp.p, 0);
    cudaError_t e = cudaSuccess;
    if (rc == MPHF_OK) e = cudaMemcpy(h_rank, tmp.p, count * 8, cudaMemcpyDeviceToHost);
    dev_free(tmp, 0);
    cudaError_t e2 = cudaStreamSynchronize(0);
    if (e == cudaSuccess) e = e2;
    if (rc == MPHF_OK && e != cudaSuccess) rc = cuda_fail(e, "mphf_copy_rank");
  }
  if (prev != h->device) cudaSetDevice(prev);
  return rc;
}

// Re-store A and its ranks in the other sector size (the rank-sampling choice
// of Sec. 4.3): A is gathered out of the old sectors with one strided copy on
// the device and the new sectors are built from it.
int mphf_set_layout(mphf_t *h, uint32_t sector_bytes_, void *stream) {
  if (!h || (sector_bytes_ != 8 && sector_bytes_ != 32 && sector_bytes_ != 64)) return MPHF_EINVAL;
  const unsigned W = sector_bytes_ == 32 ? kSectWords
                     : sector_bytes_ == 64 ? kSectWordsMini : kUnitBits;
  if (W == h->sw) return MPHF_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  mphf_t nh;  // the new arrays, built beside the old ones
  nh.M = h->M;
  nh.sw = W;
  DevBuf A, fb;
  const AGather g = a_gather(h->M, h->sw);
  const char *src = (const char *)h->S.p + g.offset;
  int rc = dev_alloc(A, h->M / 8, s);
  cudaError_t e = cudaSuccess;
  if (rc == MPHF_OK && g.full)
    e = cudaMemcpy2DAsync(A.p, g.width, src, g.pitch, g.width, g.full, cudaMemcpyDeviceToDevice, s);
  if (rc == MPHF_OK && e == cudaSuccess && g.rest)
    e = cudaMemcpyAsync((char *)A.p + g.full * g.width, src + g.full * g.pitch, g.rest,
                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) rc = cuda_fail(e, "mphf_set_layout (gather A)");
  if (rc == MPHF_OK && h->M)
    rc = make_sectors(&nh, ASrc{(const u64 *)A.p, h->M / 64, nullptr, h->M / 64}, nullptr, s);
  // a handle of a batched build gets arrays of its own
  if (rc == MPHF_OK && h->shared && h->n_fb) {
    rc = dev_alloc(fb, h->n_fb * 8, s);
    if (rc == MPHF_OK &&
        (e = cudaMemcpyAsync(fb.p, h->fb.p, h->n_fb * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      rc = cuda_fail(e, "mphf_set_layout (fallback)");
  }
  dev_free(A, s);
  e = cudaStreamSynchronize(s);
  if (rc == MPHF_OK && e != cudaSuccess) rc = cuda_fail(e, "mphf_set_layout");
  if (rc != MPHF_OK) {
    dev_free(nh.S, s);
    dev_free(nh.SB, s);
    dev_free(fb, s);
    cudaStreamSynchronize(s);
    if (prev != h->device) cudaSetDevice(prev);
    return rc;
  }
  if (h->ldesc.p) {  // multi-lookup descriptor of the old arrays
    cudaFree(h->ldesc.p);
    h->ldesc = DevBuf();
  }
  if (h->shared) {
    if (h->n_fb) h->fb = fb;
    else h->fb = DevBuf();
    release_shared(h->shared);
    h->shared = nullptr;
  } else {
    dev_free(h->S, s);
    dev_free(h->SB, s);
  }
  h->S = nh.S;
  h->SB = nh.SB;
  h->sw = W;
  h->n_sect = nh.n_sect;
  nh.S = DevBuf();
  nh.SB = DevBuf();
  if (prev != h->device) cudaSetDevice(prev);
  return MPHF_OK;
}

uint32_t mphf_sector_bytes(const mphf_t *h) { return h ? (uint32_t)sector_bytes(h->sw) : 0; }

uint64_t mphf_device_bytes(const mphf_t *h) {
  return h ? (uint64_t)(h->S.bytes + h->SB.bytes + h->fb.bytes) : 0;
}
int mphf_copy_fallback(const mphf_t *h, uint64_t *h_keys, uint64_t count) {
  return copy_out(h, h->fb, h_keys, count, h ? h->n_fb : 0);
}

int mphf_keygen(uint64_t *d_out, uint64_t n, uint64_t seed, uint64_t start, void *stream) {
  if (n == 0) return MPHF_OK;
  if (!d_out) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int grid = grid_for(n, 256 * 8, (unsigned)sm_count() * 8);
  {
    LaunchScope ls("keygen", s);
    k_keygen<<<grid, 256, 0, s>>>((u64 *)d_out, n, seed, start);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

uint64_t mphf_launch_count(void) { return g_launches.load(); }

int mphf_profile_enable(int on) {
  g_profile_on.store(on ? 1 : 0);
  return MPHF_OK;
}

int mphf_profile_report(char *buf, uint64_t buflen) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::map<std::string, std::pair<u64, double>> agg;
  std::vector<std::string> order;
  int rc = MPHF_OK;
  for (auto &r : g_prof) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaEventElapsedTime");
      rc = MPHF_ECUDA;
      cudaGetLastError();
    }
    std::string k(r.name);
    if (!agg.count(k)) order.push_back(k);
    agg[k].first += 1;
    agg[k].second += ms;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.clear();
  std::string out;
  for (auto &k : order) {
    char line[256];
    snprintf(line, sizeof(line), "%s %llu %.6f\n", k.c_str(), (unsigned long long)agg[k].first,
             agg[k].second);
    out += line;
  }
  if (buf && buflen) {
    size_t n = out.size() < buflen - 1 ? out.size() : (size_t)buflen - 1;
    memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return rc;
}

}  // extern "C"
