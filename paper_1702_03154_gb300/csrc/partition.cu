// partition.cu -- the key set split into K parts, one independent function
// per part (Sec. 4.3: the partitioning other tools put in front of their
// construction applies to this method too).  Key x belongs to part
//   p = floor(mix(x XOR mix(part_seed)) * K / 2^64);
// part p's function is built over its keys alone, and the global index of a
// key is the number of keys of parts 0 .. p-1 plus its index within part p.
// With one part per GPU this is the multi-GPU form of the method: routing the
// keys is one all-to-all, the prefix of the part sizes one all-gather, and
// each part's build needs no exchange at all.
//
// Kernels: a per-part count, a routing multisplit (each tile ranks its keys
// by part in shared memory, reserves one run per part with one global atomic,
// then writes the keys and their source positions), and the scatter back.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "parts.cuh"

namespace bbh {

static constexpr int kPartThreads = 256;
static constexpr int kPartPerThread = 8;
static constexpr int kPartTile = kPartThreads * kPartPerThread;
static constexpr uint32_t kMaxParts = 1024;

__device__ __forceinline__ uint32_t part_of(u64 x, u64 sp, uint32_t K) {
  return part_index(x, sp, K);
}

__global__ void __launch_bounds__(kPartThreads)
k_part_count(const u64 *__restrict__ keys, u64 n, uint32_t K, u64 sp, u64 *__restrict__ counts) {
  __shared__ unsigned hist[kMaxParts];
  for (uint32_t k = threadIdx.x; k < K; k += kPartThreads) hist[k] = 0;
  __syncthreads();
  const u64 stride = (u64)gridDim.x * kPartThreads;
  for (u64 i = (u64)blockIdx.x * kPartThreads + threadIdx.x; i < n; i += stride)
    atomicAdd(&hist[part_of(keys[i], sp, K)], 1u);
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < K; k += kPartThreads)
    if (hist[k]) atomicAdd(&counts[k], (u64)hist[k]);
}

// One tile of kPartTile keys per iteration: rank by part in shared memory,
// reserve one run per part, write.  cursor[k] starts at part k's offset.
__global__ void __launch_bounds__(kPartThreads)
k_part_route(const u64 *__restrict__ keys, u64 n, uint32_t K, u64 sp, u64 *__restrict__ cursor,
             u64 *__restrict__ routed, u64 *__restrict__ src) {
  __shared__ unsigned hist[kMaxParts];
  __shared__ u64 base[kMaxParts];
  const u64 ntiles = (n + kPartTile - 1) / kPartTile;
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (uint32_t k = threadIdx.x; k < K; k += kPartThreads) hist[k] = 0;
    __syncthreads();
    const u64 t0 = t * kPartTile;
    u64 x[kPartPerThread];
    uint32_t part[kPartPerThread];
    unsigned rank[kPartPerThread];
#pragma unroll
    for (int j = 0; j < kPartPerThread; j++) {
      const u64 i = t0 + (u64)j * kPartThreads + threadIdx.x;
      if (i < n) {
        x[j] = keys[i];
        part[j] = part_of(x[j], sp, K);
        rank[j] = atomicAdd(&hist[part[j]], 1u);
      }
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < K; k += kPartThreads)
      if (hist[k]) base[k] = atomicAdd(&cursor[k], (u64)hist[k]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPartPerThread; j++) {
      const u64 i = t0 + (u64)j * kPartThreads + threadIdx.x;
      if (i < n) {
        const u64 o = base[part[j]] + rank[j];
        routed[o] = x[j];
        if (src) src[o] = i;
      }
    }
    __syncthreads();
  }
}

// out[src[i]] = vals[i]
__global__ void k_unroute(const u64 *__restrict__ vals, const u64 *__restrict__ src, u64 n,
                          u64 *__restrict__ out) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[src[i]] = vals[i];
}

// vals[i] += offset unless it is MPHF_NOT_FOUND
__global__ void k_add_offset(u64 *__restrict__ vals, u64 n, u64 offset) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 v = vals[i];
    if (v != MPHF_NOT_FOUND) vals[i] = v + offset;
  }
}

// out[src[i]] = local[i] + prefix[part of routed[i]] (NOT_FOUND stays)
__global__ void k_part_finish(const u64 *__restrict__ routed, const u64 *__restrict__ local,
                              const u64 *__restrict__ src, u64 n, uint32_t K, u64 sp,
                              const u64 *__restrict__ prefix, u64 *__restrict__ out) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 v = local[i];
    out[src[i]] = v == MPHF_NOT_FOUND ? v : v + prefix[part_of(routed[i], sp, K)];
  }
}

// Routes n keys into K parts: counts on the device, offsets on the host.
static int route_impl(const u64 *keys, u64 n, uint32_t K, u64 part_seed, u64 *routed, u64 *src,
                      u64 *h_off, cudaStream_t s) {
  const u64 sp = mix64(part_seed);
  DevBuf cnt;
  int rc = dev_alloc(cnt, 2 * (size_t)K * sizeof(u64), s);
  if (rc != MPHF_OK) return rc;
  u64 *counts = (u64 *)cnt.p, *cursor = counts + K;
  cudaError_t e = cudaMemsetAsync(counts, 0, K * sizeof(u64), s);
  if (e == cudaSuccess && n) {
    LaunchScope ls("part_count", s);
    k_part_count<<<grid_for(n, kPartThreads * 16, (unsigned)sm_count() * 8), kPartThreads, 0, s>>>(
        keys, n, K, sp, counts);
    e = cudaGetLastError();
  }
  std::vector<u64> c(K);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c.data(), counts, K * sizeof(u64), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(cnt, s);
    return cuda_fail(e, "route: count");
  }
  h_off[0] = 0;
  for (uint32_t k = 0; k < K; k++) h_off[k + 1] = h_off[k] + c[k];
  if (h_off[K] != n) {
    dev_free(cnt, s);
    return MPHF_EINTERNAL;
  }
  // pageable copy: staged before the call returns
  e = cudaMemcpyAsync(cursor, h_off, K * sizeof(u64), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n) {
    LaunchScope ls("part_route", s);
    k_part_route<<<grid_for(n, kPartTile, (unsigned)sm_count() * 4), kPartThreads, 0, s>>>(
        keys, n, K, sp, cursor, routed, src);
    e = cudaGetLastError();
  }
  dev_free(cnt, s);
  if (e != cudaSuccess) return cuda_fail(e, "route: scatter");
  return MPHF_OK;
}

}  // namespace bbh

struct mphf_part {
  uint32_t K = 0;
  uint64_t part_seed = 0;
  std::vector<mphf_t *> f;          // one function per part
  std::vector<uint64_t> off;        // K + 1 global offsets (prefix of the part sizes)
  bbh::DevBuf d_off;                // the same on the device
};

using namespace bbh;

extern "C" int mphf_route(const uint64_t *d_keys, uint64_t n, uint32_t K, uint64_t part_seed,
                          uint64_t *d_routed, uint64_t *d_src, uint64_t *h_offsets, void *stream) {
  if (K == 0 || K > kMaxParts || !h_offsets) return MPHF_EINVAL;
  if (n && (!d_keys || !d_routed || ((uintptr_t)d_keys & 7) || ((uintptr_t)d_routed & 7) ||
            ((uintptr_t)d_src & 7)))
    return MPHF_EINVAL;
  return route_impl((const u64 *)d_keys, n, K, part_seed, (u64 *)d_routed, (u64 *)d_src,
                    (u64 *)h_offsets, (cudaStream_t)stream);
}

extern "C" int mphf_unroute(const uint64_t *d_vals, const uint64_t *d_src, uint64_t n,
                            uint64_t *d_out, void *stream) {
  if (n == 0) return MPHF_OK;
  if (!d_vals || !d_src || !d_out) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  {
    LaunchScope ls("unroute", s);
    k_unroute<<<grid_for(n, 256 * 4, (unsigned)sm_count() * 8), 256, 0, s>>>(
        (const u64 *)d_vals, (const u64 *)d_src, n, (u64 *)d_out);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

extern "C" int mphf_add_offset(uint64_t *d_vals, uint64_t n, uint64_t offset, void *stream) {
  if (n == 0) return MPHF_OK;
  if (!d_vals) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  {
    LaunchScope ls("add_offset", s);
    k_add_offset<<<grid_for(n, 256 * 4, (unsigned)sm_count() * 8), 256, 0, s>>>((u64 *)d_vals, n,
                                                                                 offset);
  }
  MPHF_CUDA(cudaGetLastError());
  return MPHF_OK;
}

extern "C" void mphf_part_free(mphf_part_t *p) {
  if (!p) return;
  for (mphf_t *h : p->f) mphf_free(h);
  dev_free(p->d_off, 0);
  delete p;
}

extern "C" int mphf_build_partitioned(const uint64_t *d_keys, uint64_t n, uint32_t K,
                                      uint64_t part_seed, double gamma, uint32_t levels,
                                      uint64_t seed, void *stream, mphf_part_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (K == 0 || K > kMaxParts || !(gamma >= 1.0) || isinf(gamma) || levels < 1 ||
      levels > MPHF_MAX_LEVELS)
    return MPHF_EINVAL;
  if (n && (!d_keys || ((uintptr_t)d_keys & 7))) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  mphf_part *p = new mphf_part;
  p->K = K;
  p->part_seed = part_seed;
  p->off.assign((size_t)K + 1, 0);
  p->f.assign(K, nullptr);
  DevBuf routed;
  int rc = dev_alloc(routed, (n ? n : 1) * sizeof(u64), s);
  if (rc == MPHF_OK)
    rc = route_impl((const u64 *)d_keys, n, K, part_seed, (u64 *)routed.p, nullptr, (u64 *)p->off.data(),
                    s);
  // Parts of up to 2^24 keys: all at once, by the batched construction over
  // the routed sets; larger parts one by one, each by mphf_build's own path.
  u64 largest = 0;
  for (uint32_t k = 0; rc == MPHF_OK && k < K; k++)
    largest = std::max<u64>(largest, p->off[k + 1] - p->off[k]);
  if (rc == MPHF_OK && K > 1 && largest <= (1ull << 24)) {
    rc = mphf_build_batched_host_offsets((const uint64_t *)routed.p, p->off.data(), K, gamma,
                                         levels, seed, stream, p->f.data());
  } else {
    for (uint32_t k = 0; rc == MPHF_OK && k < K; k++)
      rc = mphf_build((const uint64_t *)routed.p + p->off[k], p->off[k + 1] - p->off[k], gamma,
                      levels, seed, stream, &p->f[k]);
  }
  dev_free(routed, s);
  if (rc == MPHF_OK) rc = dev_alloc(p->d_off, ((size_t)K + 1) * sizeof(u64), s);
  if (rc == MPHF_OK) {
    cudaError_t e = cudaMemcpyAsync(p->d_off.p, p->off.data(), ((size_t)K + 1) * sizeof(u64),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "partitioned build: offsets");
  }
  if (rc != MPHF_OK) {
    mphf_part_free(p);
    return rc;
  }
  *out = p;
  return MPHF_OK;
}

extern "C" int mphf_part_lookup(const mphf_part_t *p, const uint64_t *d_keys, uint64_t n,
                                uint64_t *d_out, void *stream) {
  if (!p) return MPHF_EINVAL;
  if (n == 0) return MPHF_OK;
  if (!d_keys || !d_out || ((uintptr_t)d_keys & 7) || ((uintptr_t)d_out & 7)) return MPHF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // one pass: each key's part from its hash, no routing (when the parts share
  // a layout and none is empty)
  if (lookup_parts_direct(p->f.data(), p->K, mix64(p->part_seed), (const u64 *)p->d_off.p,
                          (const u64 *)d_keys, n, (u64 *)d_out, s) == MPHF_OK)
    return MPHF_OK;
  DevBuf buf;
  int rc = dev_alloc(buf, 3 * n * sizeof(u64), s);
  if (rc != MPHF_OK) return rc;
  u64 *routed = (u64 *)buf.p, *src = routed + n, *local = src + n;
  std::vector<u64> qoff((size_t)p->K + 1);
  rc = route_impl((const u64 *)d_keys, n, p->K, p->part_seed, routed, src, qoff.data(), s);
  if (rc == MPHF_OK) {
    std::vector<const uint64_t *> kk(p->K);
    std::vector<uint64_t *> oo(p->K);
    std::vector<uint64_t> cc(p->K);
    for (uint32_t k = 0; k < p->K; k++) {
      kk[k] = (const uint64_t *)(routed + qoff[k]);
      oo[k] = (uint64_t *)(local + qoff[k]);
      cc[k] = qoff[k + 1] - qoff[k];
    }
    rc = mphf_lookup_multi(const_cast<mphf_t *const *>(p->f.data()), kk.data(), oo.data(),
                           cc.data(), p->K, stream);
  }
  if (rc == MPHF_OK) {
    {
      LaunchScope ls("part_finish", s);
      k_part_finish<<<grid_for(n, 256 * 4, (unsigned)sm_count() * 8), 256, 0, s>>>(
          routed, local, src, n, p->K, mix64(p->part_seed), (const u64 *)p->d_off.p,
          (u64 *)d_out);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "partitioned lookup: finish");
  }
  dev_free(buf, s);
  return rc;
}

extern "C" int mphf_part_info(const mphf_part_t *p, uint32_t *K, uint64_t *h_offsets) {
  if (!p || !K) return MPHF_EINVAL;
  *K = p->K;
  if (h_offsets)
    for (uint32_t k = 0; k <= p->K; k++) h_offsets[k] = p->off[k];
  return MPHF_OK;
}

extern "C" const mphf_t *mphf_part_function(const mphf_part_t *p, uint32_t k) {
  if (!p || k >= p->K) return nullptr;
  return p->f[k];
}
