// parts.cuh -- the split of a key set into K parts (Sec. 4.3's partitioning)
// shared by the routing kernels and the one-launch partitioned lookup.
#pragma once

#include "common.cuh"

namespace bbh {

// Part of key x in a split into K parts (Sec. 4.3's partitioning): the top of
// fastrange over the mixed key; sp = mix64(part seed).
__host__ __device__ __forceinline__ uint32_t part_index(u64 x, u64 sp, uint32_t K) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__umul64hi(mix64(x ^ sp), (u64)K);
#else
  return (uint32_t)(((unsigned __int128)mix64(x ^ sp) * K) >> 64);
#endif
}

// Lookup of n keys against the K functions of a split: each key's function
// is fs[part_index(key)] and its answer gets that part's offset prefix[part].
// Returns MPHF_EINVAL without launching anything when the parts do not share
// one storage layout or a part is empty (the caller routes instead).
int lookup_parts_direct(mphf *const *fs, uint32_t K, u64 sp, const u64 *d_prefix,
                        const u64 *keys, u64 n, u64 *out, cudaStream_t s);

}  // namespace bbh
