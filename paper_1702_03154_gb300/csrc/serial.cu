// serial.cu -- a handle as a self-contained byte image (save / load).
//
// The image holds what a query needs (Algorithm 3): the level table
// (n_d, m_d, off_d; the seeds follow from the seed, Sec. 2.1), the sectors
// holding A with its ranks (sector.cuh), the superblock counts and the sorted
// fallback (Sec. 3.5).  Loading checks the header against the sizing rules
// (m_d from n_d and gamma, off_d as the running sum, M, the sector counts)
// and a checksum of the payload, so an image that does not describe a valid
// function is rejected rather than queried.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "sector.cuh"

namespace bbh {

static const char kMagic[8] = {'B', 'B', 'H', 'G', 'B', '3', '0', '0'};
static constexpr uint32_t kVersion = 1;
static constexpr uint64_t kHeader = 128;

struct Header {
  char magic[8];
  uint32_t version, header_bytes;
  uint64_t N;
  double gamma;
  uint32_t L, L_used;
  uint64_t seed, M, n_fb, n_sect, n_sb, total_bytes, checksum;
  uint32_t sector_words, pad;  // layout: A words per sector (7 or 15), or 48 (8-byte units)
  uint64_t reserved[3];
};
static_assert(sizeof(Header) == kHeader, "header layout");

// 64-bit checksum of n 8-byte words: each word is folded in with the
// SplitMix64 finalizer, then the word count.
static uint64_t checksum(const unsigned char *p, uint64_t nwords) {
  uint64_t h = 0x6a09e667f3bcc908ull;
  for (uint64_t i = 0; i < nwords; i++) {
    uint64_t w;
    memcpy(&w, p + 8 * i, 8);
    h = mix64(h + w);
  }
  return mix64(h ^ nwords);
}

static uint64_t level_table_bytes(uint32_t L_used) { return (3ull * L_used + 1) * 8; }

static uint64_t image_bytes(uint32_t L_used, uint64_t n_sect, unsigned W, uint64_t n_sb,
                            uint64_t n_fb) {
  return kHeader + level_table_bytes(L_used) + n_sect * sector_bytes(W) + n_sb * 8 + n_fb * 8;
}

}  // namespace bbh

using namespace bbh;

extern "C" int mphf_serialized_size(const mphf_t *h, uint64_t *bytes) {
  if (!h || !bytes) return MPHF_EINVAL;
  *bytes = image_bytes(h->L_used, h->n_sect, h->sw, n_sb_entries(h->n_sect, h->sw), h->n_fb);
  return MPHF_OK;
}

extern "C" int mphf_serialize(const mphf_t *h, void *h_buf, uint64_t bytes) {
  if (!h || !h_buf) return MPHF_EINVAL;
  const uint64_t n_sb = n_sb_entries(h->n_sect, h->sw);
  const uint64_t total = image_bytes(h->L_used, h->n_sect, h->sw, n_sb, h->n_fb);
  const uint64_t sbytes = h->n_sect * sector_bytes(h->sw);
  if (bytes < total) return MPHF_EINVAL;
  unsigned char *b = (unsigned char *)h_buf;
  uint64_t *lv = (uint64_t *)malloc(level_table_bytes(h->L_used));
  if (!lv) return MPHF_ENOMEM;
  for (uint32_t d = 0; d < h->L_used; d++) {
    lv[3 * d] = h->n[d];
    lv[3 * d + 1] = h->m[d];
    lv[3 * d + 2] = h->off[d];
  }
  lv[3 * h->L_used] = h->n[h->L_used];
  uint64_t at = kHeader;
  memcpy(b + at, lv, level_table_bytes(h->L_used));
  free(lv);
  at += level_table_bytes(h->L_used);
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  cudaError_t e = cudaSuccess;
  if (h->n_sect) e = cudaMemcpy(b + at, h->S.p, sbytes, cudaMemcpyDeviceToHost);
  at += sbytes;
  if (e == cudaSuccess && n_sb) e = cudaMemcpy(b + at, h->SB.p, n_sb * 8, cudaMemcpyDeviceToHost);
  at += n_sb * 8;
  if (e == cudaSuccess && h->n_fb)
    e = cudaMemcpy(b + at, h->fb.p, h->n_fb * 8, cudaMemcpyDeviceToHost);
  if (prev != h->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "mphf_serialize");
  Header hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.header_bytes = (uint32_t)kHeader;
  hd.N = h->N;
  hd.gamma = h->gamma;
  hd.L = h->L;
  hd.L_used = h->L_used;
  hd.seed = h->seed;
  hd.M = h->M;
  hd.n_fb = h->n_fb;
  hd.n_sect = h->n_sect;
  hd.n_sb = n_sb;
  hd.sector_words = h->sw;
  hd.total_bytes = total;
  hd.checksum = checksum(b + kHeader, (total - kHeader) / 8);
  memcpy(b, &hd, sizeof(hd));
  return MPHF_OK;
}

extern "C" int mphf_deserialize(const void *h_buf, uint64_t bytes, void *stream, mphf_t **out) {
  if (!out) return MPHF_EINVAL;
  *out = nullptr;
  if (!h_buf || bytes < kHeader) return MPHF_EINVAL;
  const unsigned char *b = (const unsigned char *)h_buf;
  Header hd;
  memcpy(&hd, b, sizeof(hd));
  if (memcmp(hd.magic, kMagic, 8) != 0 || hd.version != kVersion || hd.header_bytes != kHeader)
    return MPHF_EINVAL;
  if (!(hd.gamma >= 1.0) || isinf(hd.gamma) || hd.L < 1 || hd.L > MPHF_MAX_LEVELS ||
      hd.L_used > hd.L)
    return MPHF_EINVAL;
  // sizes, before reading anything they locate
  const unsigned W = hd.sector_words;
  if (!layout_ok(W)) return MPHF_EINVAL;
  if (hd.M > (1ull << 56) || hd.n_fb > hd.N) return MPHF_EINVAL;
  if (hd.n_sect != n_sectors(hd.M, W) || hd.n_sb != n_sb_entries(hd.n_sect, W)) return MPHF_EINVAL;
  if (hd.total_bytes != image_bytes(hd.L_used, hd.n_sect, W, hd.n_sb, hd.n_fb) ||
      hd.total_bytes > bytes)
    return MPHF_EINVAL;
  if (checksum(b + kHeader, (hd.total_bytes - kHeader) / 8) != hd.checksum) return MPHF_EINVAL;
  // the level table must follow the sizing rules of Sec. 2.2.4
  std::vector<uint64_t> lv(3 * (size_t)hd.L_used + 1);
  memcpy(lv.data(), b + kHeader, level_table_bytes(hd.L_used));
  if (hd.N == 0) {
    if (hd.L_used || hd.M || hd.n_fb) return MPHF_EINVAL;
  } else {
    if (hd.L_used == 0 || lv[0] != hd.N) return MPHF_EINVAL;
    uint64_t off = 0;
    for (uint32_t d = 0; d < hd.L_used; d++) {
      const uint64_t n = lv[3 * d], m = lv[3 * d + 1], o = lv[3 * d + 2];
      const uint64_t nn = lv[3 * d + 3];
      // a level may place no key at all (every position collided), so n_{d+1} <= n_d
      if (n == 0 || m != level_bits(n, hd.gamma) || o != off || nn > n) return MPHF_EINVAL;
      off += m;
    }
    if (off != hd.M) return MPHF_EINVAL;
    const uint64_t left = lv[3 * hd.L_used];
    if (left != hd.n_fb || (hd.n_fb && hd.L_used != hd.L)) return MPHF_EINVAL;
  }
  mphf_t *h = handle_new();
  if (!h) return MPHF_ENOMEM;
  cudaGetDevice(&h->device);
  h->N = hd.N;
  h->gamma = hd.gamma;
  h->L = hd.L;
  h->seed = hd.seed;
  h->L_used = hd.L_used;
  for (uint32_t d = 0; d < hd.L; d++) h->s[d] = level_seed(hd.seed, d);
  for (uint32_t d = 0; d < hd.L_used; d++) {
    h->n[d] = lv[3 * d];
    h->m[d] = lv[3 * d + 1];
    h->off[d] = lv[3 * d + 2];
  }
  h->n[hd.L_used] = lv[3 * hd.L_used];
  h->M = hd.M;
  h->n_rank = (hd.M + MPHF_RANK_BLOCK - 1) / MPHF_RANK_BLOCK;
  h->n_fb = hd.n_fb;
  h->n_sect = hd.n_sect;
  h->sw = W;
  h->path = 4;  // loaded from an image
  cudaStream_t st = (cudaStream_t)stream;
  uint64_t at = kHeader + level_table_bytes(hd.L_used);
  const uint64_t sbytes = hd.n_sect * sector_bytes(W);
  int rc = dev_alloc(h->S, sbytes, st);
  if (rc == MPHF_OK) rc = dev_alloc(h->SB, hd.n_sb * 8, st);
  if (rc == MPHF_OK) rc = dev_alloc(h->fb, hd.n_fb * 8, st);
  cudaError_t e = cudaSuccess;
  if (rc == MPHF_OK && hd.n_sect)
    e = cudaMemcpyAsync(h->S.p, b + at, sbytes, cudaMemcpyHostToDevice, st);
  at += sbytes;
  if (rc == MPHF_OK && e == cudaSuccess && hd.n_sb)
    e = cudaMemcpyAsync(h->SB.p, b + at, hd.n_sb * 8, cudaMemcpyHostToDevice, st);
  at += hd.n_sb * 8;
  if (rc == MPHF_OK && e == cudaSuccess && hd.n_fb)
    e = cudaMemcpyAsync(h->fb.p, b + at, hd.n_fb * 8, cudaMemcpyHostToDevice, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (rc == MPHF_OK && e != cudaSuccess) rc = cuda_fail(e, "mphf_deserialize");
  if (rc != MPHF_OK) {
    dev_free(h->S, st);
    dev_free(h->SB, st);
    dev_free(h->fb, st);
    cudaStreamSynchronize(st);
    handle_delete(h);
    return rc;
  }
  *out = h;
  return MPHF_OK;
}
