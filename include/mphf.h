/*
 * mphf.h -- C ABI of the GB300 (sm_103a) cascading-bit-array minimal perfect
 * hash function library (libmphf.so).
 *
 * The method is BBhash (Limasset, Rizk, Chikhi, Peterlongo, "Fast and scalable
 * minimal perfect hashing for massive key sets", arXiv 1702.03154): keys are
 * hashed level by level into bit arrays A_d of gamma*|F_d| bits; a key that is
 * alone at its position sets its bit, colliding keys move on to F_{d+1}
 * (Sec. 2.1, Algorithms 1-2); the index of a key is the rank of its bit in the
 * concatenation A = A_0 || A_1 || ... (Sec. 2.2.3, Algorithm 3), with 64-bit
 * rank checkpoints every 512 bits (Sec. 3.1); keys left after L levels go to a
 * fallback table (Sec. 3.5).
 *
 * Conventions fixed by this library (the paper leaves them open):
 *   - level seed s_d = mix(mix(seed) + d), h_d(x) = mix(x ^ s_d), where mix is
 *     the SplitMix64 finalizer; position p = floor(h_d(x) * m_d / 2^64);
 *   - m_d = |A_d| = max(64, ceil(gamma * n_d) rounded up to a multiple of 64);
 *   - indices are 0-based, in [0, N); rank is exclusive (ones before the bit);
 *   - bit g of A is bit (g % 64) of 64-bit word g / 64; level d starts at bit
 *     off_d = m_0 + ... + m_{d-1};
 *   - rank[b] = number of ones of A in bits [0, 512 b), ceil(M / 512) entries;
 *   - the fallback is the sorted array of leftover keys; the key at sorted
 *     position i has index N - n_fb + i;
 *   - a key that is not in the set gets what Algorithm 3 yields: the rank at
 *     the first level whose bit is 1, else its fallback index, else
 *     MPHF_NOT_FOUND.
 *
 * Memory and streams.  Pointers named d_* are device pointers (CUDA global
 * memory of the current device); h_* are host pointers.  A `stream` argument
 * is a cudaStream_t passed as void* (NULL = the legacy default stream).  All
 * device memory a handle owns is allocated by the library and released by
 * mphf_free.  Functions return MPHF_OK or an error code; none aborts.  Every
 * function taking a handle is safe to call from one host thread at a time per
 * handle; lookups on one handle from several streams may overlap.
 */
#ifndef MPHF_H
#define MPHF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mphf mphf_t;
typedef struct mphf_server mphf_server_t;
typedef struct mphf_part mphf_part_t;

#define MPHF_NOT_FOUND UINT64_MAX
#define MPHF_MAX_LEVELS 64
#define MPHF_RANK_BLOCK 512

enum {
    MPHF_OK = 0,
    MPHF_EINVAL = 1,      /* bad argument: gamma < 1 or not finite, levels not in [1,64], NULL */
    MPHF_ENOMEM = 2,      /* a device or host allocation failed */
    MPHF_EDUPLICATE = 3,  /* the key set holds two equal keys */
    MPHF_ECUDA = 4,       /* a CUDA runtime call failed (the message is in mphf_last_cuda_error) */
    MPHF_ETIMEOUT = 5,    /* a bounded device wait gave up */
    MPHF_EINTERNAL = 6    /* a device-side consistency check failed */
};

/* Text for an error code (static storage). */
const char *mphf_strerror(int code);
/* Last CUDA runtime error text seen by this library (static storage). */
const char *mphf_last_cuda_error(void);
/* ABI version of this header. */
int mphf_abi_version(void);

/*
 * Build the function over n distinct keys (Algorithm 1 with ArrayFill,
 * Algorithm 2; rank checkpoints, Sec. 3.1; fallback, Sec. 3.5).
 *   d_keys  device array of n uint64 keys; read only, owned by the caller, may
 *           be released as soon as the call returns; any 8-byte alignment.
 *   n       number of keys (0 gives a valid empty function).
 *   gamma   |A_d| / |F_d| (Sec. 2.2.4), finite and >= 1.
 *   levels  level budget L in [1, 64] (D = 25 in the paper).
 *   seed    selects the hash functions h_d.
 *   stream  work is issued on this stream; the call returns when it is done.
 *   out     receives the new handle (NULL on error).
 * Errors: MPHF_EINVAL, MPHF_ENOMEM, MPHF_EDUPLICATE (nothing is leaked),
 * MPHF_ECUDA, MPHF_EINTERNAL.
 */
int mphf_build(const uint64_t *d_keys, uint64_t n, double gamma, uint32_t levels, uint64_t seed,
               void *stream, mphf_t **out);

/* As mphf_build, with the keys in host memory (copied to the device inside the call;
 * page-locked memory makes the copy asynchronous and faster). */
int mphf_build_host(const uint64_t *h_keys, uint64_t n, double gamma, uint32_t levels,
                    uint64_t seed, void *stream, mphf_t **out);

/*
 * mphf_build_host followed by mphf_lookup_host in one call (construction,
 * Algorithms 1-2; query, Algorithm 3 with the ranks of Sec. 3.1), with the host
 * link kept busy: the queries are copied right behind the keys while the
 * levels after the first are built, and each chunk of queries is looked up
 * as soon as it has landed while the indices of the previous chunk are
 * copied back.  Same results as the two calls.
 *   h_keys, n        the key set (host memory; page-locked is faster)
 *   h_queries, nq    the keys to look up (host), h_out receives nq indices
 *                    (host), as mphf_lookup writes them
 *   out              receives the function (release with mphf_free)
 * Waits for the results.  Errors as mphf_build and mphf_lookup; on error
 * nothing is leaked and *out is NULL.
 */
int mphf_build_lookup_host(const uint64_t *h_keys, uint64_t n, double gamma, uint32_t levels,
                           uint64_t seed, const uint64_t *h_queries, uint64_t nq,
                           uint64_t *h_out, void *stream, mphf_t **out);

/*
 * Build S independent functions at once, one per key set (the same method
 * and conventions as mphf_build, applied to each set separately; set s gets
 * exactly the function mphf_build would give it with the same arguments).
 *   d_keys     device array holding the sets back to back (8-byte aligned).
 *   d_offsets  device array of S + 1 non-decreasing indices into d_keys
 *              (8-byte aligned): set s is d_keys[d_offsets[s] ..
 *              d_offsets[s+1]).  Read back to the host at the start of the
 *              call (the plan of the build depends on the set sizes).
 *   S          number of sets, >= 1.
 *   out        host array of S handles, each released with mphf_free (their
 *              device memory is one shared block, returned when the last is
 *              freed).
 * All sets advance level by level together (one launch per phase per level
 * for all sets, recorded once as a CUDA graph and replayed); sets of at most
 * 16384 keys run every level in one thread block.  Synchronous w.r.t. stream.
 * Errors as mphf_build, and MPHF_EINVAL for decreasing offsets; on error no
 * handle is returned (every out[s] is NULL).  Builds through this call are
 * serialised within a process (they share a device workspace, kept between
 * calls; see mphf_workspace_release).
 */
int mphf_build_batched(const uint64_t *d_keys, const uint64_t *d_offsets, uint32_t S, double gamma,
                       uint32_t levels, uint64_t seed, void *stream, mphf_t **out);

/* As mphf_build_batched with the S + 1 offsets in host memory (h_offsets),
 * for callers that planned the sets on the host; nothing is read back. */
int mphf_build_batched_host_offsets(const uint64_t *d_keys, const uint64_t *h_offsets, uint32_t S,
                                    double gamma, uint32_t levels, uint64_t seed, void *stream,
                                    mphf_t **out);

/* Time the candidate bucket widths of mphf_build_batched on this input and keep
 * the fastest for inputs of the same size class (process-wide).  The functions
 * built do not depend on the choice.  *best_ms receives the winning time. */
int mphf_autotune_batched(const uint64_t *d_keys, const uint64_t *h_offsets, uint32_t S,
                          double gamma, uint32_t levels, uint64_t seed, void *stream,
                          double *best_ms);

/* The choice mphf_autotune_batched made for S sets of total_keys keys: the
 * largest bucket width (positions), the most buckets per set and the tail
 * shape (keys handed to the single-CTA tail: 4096 on 256 threads or 8192 on
 * 512).  MPHF_EINVAL (and the defaults) if that size class was never tuned. */
int mphf_batched_tuning(uint32_t S, uint64_t total_keys, uint64_t *pmax, uint64_t *bset_max,
                        uint64_t *tail_keys);

/* Sets the choice for the size class of S sets of total_keys keys (both
 * rounded up to powers of two), e.g. one saved from an earlier
 * mphf_autotune_batched: pmax a power of two in [4096, 262144], bset_max in
 * [1, 2048], tail_keys 4096 or 8192.  Results never depend on it; a choice
 * whose buckets overflow costs a re-build of the sets concerned.
 * MPHF_EINVAL for values out of range. */
int mphf_batched_set_tuning(uint32_t S, uint64_t total_keys, uint64_t pmax, uint64_t bset_max,
                            uint64_t tail_keys);

/* Test hooks, host arithmetic only (no device work).  mphf_debug_size_level:
 * the bucketed construction's choice for a level of n keys with a target of
 * btarget buckets: B buckets of P positions (a power of two) and cap key slots
 * each.  mphf_debug_level1_bound: for a bucketed build of N keys, the bound
 * n1_hi on |F_1| and the slots capY (and buckets Bb) of level 1's arena,
 * allocated before level 0 runs: every level size of n <= n1_hi keys must fit
 * (B <= Bb, B cap <= capY).  MPHF_EINVAL for NULL outputs, gamma < 1 or
 * btarget = 0. */
int mphf_debug_size_level(uint64_t n, double gamma, uint64_t btarget, uint64_t *B, uint64_t *cap,
                          uint64_t *P);
int mphf_debug_level1_bound(uint64_t N, double gamma, uint64_t btarget, uint64_t *n1_hi,
                            uint64_t *capY, uint64_t *Bb);

/* Test hook: nonzero sends every lookup through the kernels with 64-bit
 * position arithmetic, which otherwise only functions with a level of 2^32
 * bits or more, or 2^36 bits of A, take.  Results never depend on it. */
int mphf_debug_lookup_wide(int on);

/* Test hook for the unbucketed construction: a level whose hit/collision
 * array (2 bits a position) exceeds min_ac_bytes has its keys grouped by slabs
 * of 2^shift positions, and each slab's keys by fine slabs of 2^18 positions
 * filled in shared memory (defaults 27 and 64 MiB); no result changes.
 * shift in [6, 29]; MPHF_EINVAL otherwise. */
int mphf_debug_slabs(uint32_t shift, uint64_t min_ac_bytes);

/* Test hook: scales the bucket capacities of mphf_build_batched (default 1;
 * values < 1 make sets overflow and exercise their individual rebuild). */
int mphf_batched_debug_config(double cap_scale);

/* Free the device workspace kept by mphf_build_batched. */
void mphf_workspace_release(void);

/*
 * Query n keys (Algorithm 3, minimal index of Sec. 2.2.3).
 *   d_keys  device array of n keys, any 8-byte alignment.
 *   d_out   device array of n uint64 results (caller-allocated).
 * Asynchronous: returns once the kernel is queued on `stream`.  n = 0 is a no-op.
 */
int mphf_lookup(const mphf_t *h, const uint64_t *d_keys, uint64_t n, uint64_t *d_out,
                void *stream);

/* As mphf_lookup with host arrays: copies in, queries, copies out, and waits. */
int mphf_lookup_host(const mphf_t *h, const uint64_t *h_keys, uint64_t n, uint64_t *h_out,
                     void *stream);

/* Size of the function in bits per key: (M + 64 ceil(M/512) + 64 n_fb) / N with M the
 * total bits of A (Sec. 3.1's (1 + 64/512) gamma e^{1/gamma}); 1024 in place of 512
 * for the minirank layout (mphf_set_layout); level metadata excluded.
 * 0 for an empty function or NULL. */
double mphf_bits_per_key(const mphf_t *h);

/* Device memory the handle holds, in bytes.  A and its ranks are stored
 * together (by default in 32-byte sectors: 224 bits of A and a 32-bit count of
 * the ones before the sector within its superblock of 2^24 sectors, plus one
 * 64-bit count per superblock; see mphf_set_layout for the other layouts),
 * and the fallback keys.  A query then reads one sector per level it probes.
 * The default counts cost 1/7 of A, where Sec. 3.1's 64-bit checkpoint per
 * 512 bits costs 1/8 (mphf_bits_per_key counts the paper's).  0 for NULL. */
uint64_t mphf_device_bytes(const mphf_t *h);

/*
 * Rank sampling (Sec. 3.1; the "minirank" setting of Sec. 4.3).  A and its
 * ranks live in one of three layouts, chosen by sector_bytes:
 *   32  sectors of 224 bits of A + one 32-bit count (the default): every probe
 *       is one 256-bit load; the counts cost 1/7 of A;
 *   64  sectors of 480 bits of A + one count ("minirank"): counts cost 1/15 of
 *       A, at gamma = 1 the size drops from 3.1 to 2.9 bits/key as in the
 *       paper, and a probe loads both halves of its sector;
 *   8   units of 48 bits of A + a 16-bit count within blocks of 1024 units (a
 *       64-bit count per block): every probe is one 8-byte load (lookups as
 *       fast as with 32-byte sectors), at the price of counts costing 1/3 of A.
 * Builds make 32-byte sectors; mphf_set_layout re-stores a function in
 * another layout, keeping every index unchanged; a handle of a batched build
 * then gets arrays of its own.  mphf_bits_per_key counts one 64-bit counter
 * per 512 bits of A (per 1024 bits for the 64-byte layout: the paper's two
 * settings); mphf_device_bytes gives the memory actually held.  Waits for the
 * device before returning.
 */
int mphf_set_layout(mphf_t *h, uint32_t sector_bytes, void *stream);
uint32_t mphf_sector_bytes(const mphf_t *h);   /* 32, 64 or 8; 0 for NULL */

/* Release a handle and its device memory; NULL is a no-op. */
void mphf_free(mphf_t *h);

/* ---- introspection (host copies; for tests and tools) ------------------ */
uint64_t mphf_num_keys(const mphf_t *h);
/* Levels built (index of the last level + 1) into *levels; MPHF_EINVAL for NULL. */
int mphf_num_levels(const mphf_t *h, uint32_t *levels);
uint64_t mphf_total_bits(const mphf_t *h);      /* M */
uint64_t mphf_num_rank(const mphf_t *h);        /* ceil(M / 512) */
uint64_t mphf_num_fallback(const mphf_t *h);    /* n_fb */
/* n_d = |F_d|, m_d = |A_d|, off_d = first bit of A_d in A, s_d = level seed. */
int mphf_level_info(const mphf_t *h, uint32_t d, uint64_t *n_d, uint64_t *m_d, uint64_t *off_d,
                    uint64_t *s_d);
/* Copy A (M/64 words, gathered out of the storage layout), the rank checkpoints
 * (evaluated from the stored counts: ones before bit 512 b) or the sorted
 * fallback to host memory; `count` must equal the size reported above.  These
 * wait for the device. */
int mphf_copy_bits(const mphf_t *h, uint64_t *h_words, uint64_t count);
int mphf_copy_rank(const mphf_t *h, uint64_t *h_rank, uint64_t count);
int mphf_copy_fallback(const mphf_t *h, uint64_t *h_keys, uint64_t count);

/* Which construction path built h: 1 = bucketed (shared-memory ArrayFill),
 * 2 = unbucketed (L2 atomics; taken when a bound of the bucketed path is
 * exceeded, e.g. many duplicate keys), 3 = mphf_build_batched, 4 = loaded by
 * mphf_deserialize, 5 = mphf_build_nodisk / mphf_build_generated.  All give
 * identical results. */
int mphf_build_path(const mphf_t *h);
/* Test hook, process-wide: path 0 = bucketed with automatic fallback (default),
 * 1 = unbucketed only; cap_scale (default 1) scales the bucket capacities, so a
 * value < 1 forces the fallback.  Not thread-safe against concurrent builds. */
int mphf_debug_config(int path, double cap_scale);

/*
 * Rank table of a bit array without allocating device memory.  The paper has
 * no counterpart: the output is one 64-bit count of ones per 512 bits of the
 * array, next to seven 9-bit in-block counts.  It is for callers that must
 * not call cudaMalloc: code that records work into a CUDA graph (cudaMalloc
 * cannot be captured), serving loops that run under a fixed device-memory
 * budget, and hosts whose own allocator owns the device memory (a direct
 * cudaMalloc there fragments that pool and stalls the device).
 *   d_words  device array of nwords 64-bit words (16-byte aligned).
 *   d_rank2  device output of 2 * ceil(nwords / 8) words (16-byte aligned):
 *            d_rank2[2b] = ones of the array in bits [0, 512 b), d_rank2[2b+1]
 *            = seven 9-bit in-block prefix counts (ones of words 0..k-1 of the
 *            block in bits 9(k-1) .. 9k-1, k = 1..7).
 *   d_total  optional device word receiving the total number of ones.
 * Scratch lives in a fixed array inside the library: at most 2^27 words
 * (2^33 bits) per call; larger inputs return MPHF_EINVAL.  The first call on
 * each device looks up that array's device address (make it before any stream
 * capture that should contain later calls; the address is kept until the
 * library is unloaded, so the device must not be reset meanwhile).  All calls
 * share the array: calls whose work may overlap on the GPU (different streams
 * without ordering) race and must be avoided.  Asynchronous on `stream`.
 */
int mphf_rank_table_noalloc(const uint64_t *d_words, uint64_t nwords, uint64_t *d_rank2,
                            uint64_t *d_total, void *stream);

/* ---- construction without stored key sets ---------------------------------- */
/*
 * Build without storing F_d (Sec. 3.4, the second strategy; Sec. 4.5): level d
 * re-reads every input key, asks levels 0..d-1 whether it was placed there
 * (the query of Algorithm 3), and fills A_d with the keys that were not.  The
 * device holds the bit arrays only, until |F_d| <= keep_fraction * n; then F_d
 * is collected once and the remaining levels run on that list (Sec. 4.5
 * keeps keys in memory below 2%: keep_fraction = 0.02).  The function equals
 * mphf_build's on the same keys, bit for bit.
 *   mphf_build_nodisk     keys in a caller-owned device array (8-byte aligned),
 *                         read again at every streamed level, never copied.
 *   mphf_build_generated  keys are key(j) = mix(key_seed + (key_start + j + 1)
 *                         * 0x9E3779B97F4A7C15), j in [0, n) -- the stream of
 *                         mphf_keygen -- computed on the fly and never stored,
 *                         so n is bounded by the bit arrays (about 2 gamma bits
 *                         per key at level 0) instead of 8 bytes per key.
 * keep_fraction must lie in [0, 1]; other arguments as mphf_build.  Waits for
 * the device before returning.
 */
int mphf_build_nodisk(const uint64_t *d_keys, uint64_t n, double gamma, uint32_t levels,
                      uint64_t seed, double keep_fraction, void *stream, mphf_t **out);
int mphf_build_generated(uint64_t n, uint64_t key_seed, uint64_t key_start, double gamma,
                         uint32_t levels, uint64_t seed, double keep_fraction, void *stream,
                         mphf_t **out);

/* ---- string keys ------------------------------------------------------------ */
/*
 * 64-bit keys of n byte strings (Sec. 4.4 / Table 2 run the method on n-grams
 * and random words; the paper does not fix how a string becomes a key).
 * String i is d_bytes[d_offsets[i] .. d_offsets[i+1]); its key is
 *   h = mix(seed + (len + 1) * 0x9E3779B97F4A7C15), then for each group of 8
 *   bytes in order (the last padded with zero bytes) h = mix(h ^ w), w the
 *   group read as a little-endian integer; key = h  (mix = SplitMix64's
 *   finalizer).
 * The keys then go to mphf_build / mphf_lookup like any others.
 *   d_bytes     device array of total_bytes bytes, any alignment.
 *   d_offsets   device array of n + 1 offsets (8-byte aligned), non-decreasing,
 *               at most total_bytes.
 *   d_out       device array of n keys (8-byte aligned).
 * A string whose offsets fall outside [0, total_bytes] or decrease is not read;
 * the call then returns MPHF_EINVAL.  Waits for the device before returning.
 */
int mphf_string_keys(const uint8_t *d_bytes, uint64_t total_bytes, const uint64_t *d_offsets,
                     uint64_t n, uint64_t seed, uint64_t *d_out, void *stream);

/* ---- serialization -------------------------------------------------------- */
/*
 * A handle as a self-contained byte image (host memory), so that a function
 * built once can be stored and loaded again, on this or another GPU.  Format
 * (little-endian): a 128-byte header -- magic "BBHGB300", format version,
 * N, gamma, L, levels used, seed, M, fallback size, sector and superblock
 * counts, a 64-bit checksum of everything after the header, and the layout
 * (A words per sector: 7 or 15; 48 for 8-byte units) -- then the
 * per-level (n_d, m_d, off_d) triples and n_L, then the sectors, the
 * superblock counts and the sorted fallback keys.
 *   mphf_serialized_size  bytes the image of h takes.
 *   mphf_serialize        writes the image to h_buf (bytes >= that size);
 *                         waits for the device.
 *   mphf_deserialize      builds a new handle on the current device from an
 *                         image; a wrong magic, version, size, checksum or an
 *                         inconsistent header returns MPHF_EINVAL and no handle.
 */
int mphf_serialized_size(const mphf_t *h, uint64_t *bytes);
int mphf_serialize(const mphf_t *h, void *h_buf, uint64_t bytes);
int mphf_deserialize(const void *h_buf, uint64_t bytes, void *stream, mphf_t **out);

/* ---- many functions, many requests --------------------------------------- */
/*
 * One launch answering nreq lookup requests against different functions:
 * request i queries counts[i] keys d_keys[i] of function hs[i] into d_out[i]
 * (Algorithm 3 for each).  Asynchronous on `stream`; the arrays are host
 * arrays read before return.  Results equal mphf_lookup's for each request.
 */
int mphf_lookup_multi(mphf_t *const *hs, const uint64_t *const *d_keys, uint64_t *const *d_out,
                      const uint64_t *counts, uint32_t nreq, void *stream);

/*
 * Serving loop for functions resident in HBM (current device).  Lookup
 * requests are queued and, whenever one of `max_inflight` launch slots is
 * free, everything pending (up to max_batch_keys keys / max_batch_reqs
 * requests) is answered by one mphf_lookup_multi-style launch; requests that
 * arrive meanwhile join the next launch.  Build requests run on
 * `build_workers` worker threads, each with its own stream, admitted once
 * their memory footprint plus that of the builds already running fits the
 * free device memory minus mem_reserve_bytes (free memory as sampled when
 * the server was made and after every build: the loop that launches lookups
 * never waits on a device query).  Handles passed to lookups must stay alive until their
 * requests complete; keys and outputs are device arrays owned by the caller.
 */
int mphf_server_create(uint64_t max_batch_keys, uint32_t max_batch_reqs, int max_inflight,
                       int build_workers, uint64_t mem_reserve_bytes, mphf_server_t **out);
/* Stops the loop after the launched work has finished; pending requests are dropped. */
void mphf_server_destroy(mphf_server_t *srv);
int mphf_server_submit_lookup(mphf_server_t *srv, mphf_t *h, const uint64_t *d_keys, uint64_t n,
                              uint64_t *d_out, uint64_t *req_id);
int mphf_server_submit_build(mphf_server_t *srv, const uint64_t *d_keys, uint64_t n, double gamma,
                             uint32_t levels, uint64_t seed, uint64_t *req_id);
/* Wait for a request (at most timeout_s, else MPHF_ETIMEOUT); returns its status,
 * its latency from submission to completion in seconds and, for a build, the
 * new handle (owned by the caller; with built == NULL it is released here).
 * A request can be waited for once; mphf_server_destroy releases the builds
 * of requests never waited for. */
int mphf_server_wait(mphf_server_t *srv, uint64_t req_id, double timeout_s, int *status,
                     double *latency_s, mphf_t **built);
int mphf_server_stats(mphf_server_t *srv, uint64_t *batches, uint64_t *requests, uint64_t *keys,
                      uint64_t *builds);
/* Where the time of the lookups completed since the last call went: p50[k]
 * and p99[k] (seconds) of k = 0 the queue wait (submission to the launch of
 * the request's batch), 1 the batch's GPU time (events around its table copy
 * and kernel), 2 the rest (launch to completion seen by the scheduler, minus
 * the GPU time: stream wait behind other work and detection).  Clears the
 * record. */
int mphf_server_latency_parts(mphf_server_t *srv, double *p50, double *p99);
/*
 * Measurement driver: an open-loop Poisson stream of requests at rate_hz for
 * duration_s against the server.  Each lookup picks one of the nh handles
 * uniformly and a batch of log-uniform size in [bmin, bmax] of consecutive
 * member keys at a random offset of keys[h] (count[h] keys), writing into the
 * device ring d_out (out_cap words >= bmax).  A fraction build_frac of the
 * arrivals are builds over a prefix of build_keys of log-uniform size in
 * [nbmin, nbmax].  Latencies of the lookups (seconds) go to lat_out.
 */
int mphf_server_loadgen(mphf_server_t *srv, mphf_t *const *hs, const uint64_t *const *keys,
                        const uint64_t *count, uint32_t nh, double rate_hz, double duration_s,
                        double bmin, double bmax, uint64_t *d_out, uint64_t out_cap,
                        double build_frac, const uint64_t *build_keys, uint64_t n_build_keys,
                        double nbmin, double nbmax, double gamma, uint64_t seed, double *lat_out,
                        uint64_t lat_cap, uint64_t *n_lookups_out, uint64_t *n_keys_out,
                        uint64_t *n_builds_out, double *elapsed_out);

/* ---- partitioned functions (one independent function per part) ----------- */
/*
 * Sec. 4.3 notes that other tools split the key set into partitions and
 * build one small function per partition, and that the split applies to this
 * method too.  Key x belongs to part
 *   p = floor(mix(x ^ mix(part_seed)) * K / 2^64)      (mix: SplitMix64's finalizer)
 * of K parts (1 <= K <= 1024).  Part p's function is built over its keys
 * alone (seed, gamma, L as for mphf_build), and the global index of a key is
 * the number of keys of parts 0 .. p-1 plus its index within part p: a
 * bijection onto [0, N) again.  With one part per GPU this is the multi-GPU
 * form of the method (routing is one all-to-all of keys, the prefix of the
 * part sizes one all-gather, each part's build needs no exchange); the
 * routing and scatter steps are exposed for that use.
 *
 *   mphf_route        writes d_keys (n, 8-byte aligned) grouped by part into
 *                     d_routed (n words): part k's keys are
 *                     d_routed[h_offsets[k] .. h_offsets[k+1]), in no fixed
 *                     order within the part; d_src (n words, optional) gets
 *                     each routed key's position in d_keys; h_offsets (host,
 *                     K + 1) the part boundaries.  Waits for the counts.
 *   mphf_unroute      d_out[d_src[i]] = d_vals[i] for i < n (the inverse
 *                     placement of mphf_route's output).  Asynchronous.
 *   mphf_add_offset   d_vals[i] += offset for every entry that is not
 *                     MPHF_NOT_FOUND (a part's local indices made global).
 *   mphf_build_partitioned  routes the keys and builds every part (parts of
 *                     up to 2^24 keys together by the batched construction,
 *                     larger ones one by one); the handle owns the K functions.
 *   mphf_part_lookup  writes each key's global index (or MPHF_NOT_FOUND) at
 *                     its own position of d_out.  When the K functions share
 *                     one storage layout and none is empty, one launch
 *                     answers every key with the function of its part (part
 *                     hash per key, no routing; asynchronous on `stream`).
 *                     Otherwise it routes the queries (24 bytes per query of
 *                     scratch; waits for the routing counts), answers every
 *                     part's queries in one multi-function launch and scatters
 *                     the answers back.
 *   mphf_part_info    K and the K + 1 global offsets (h_offsets may be NULL).
 *   mphf_part_function  part k's function (owned by the handle), NULL if k >= K.
 * Errors: MPHF_EINVAL for K outside [1, 1024], bad gamma / levels, NULL or
 * misaligned arrays; otherwise as mphf_build and mphf_lookup.
 */
int mphf_route(const uint64_t *d_keys, uint64_t n, uint32_t K, uint64_t part_seed,
               uint64_t *d_routed, uint64_t *d_src, uint64_t *h_offsets, void *stream);
int mphf_unroute(const uint64_t *d_vals, const uint64_t *d_src, uint64_t n, uint64_t *d_out,
                 void *stream);
int mphf_add_offset(uint64_t *d_vals, uint64_t n, uint64_t offset, void *stream);
int mphf_build_partitioned(const uint64_t *d_keys, uint64_t n, uint32_t K, uint64_t part_seed,
                           double gamma, uint32_t levels, uint64_t seed, void *stream,
                           mphf_part_t **out);
int mphf_part_lookup(const mphf_part_t *p, const uint64_t *d_keys, uint64_t n, uint64_t *d_out,
                     void *stream);
int mphf_part_info(const mphf_part_t *p, uint32_t *K, uint64_t *h_offsets);
const mphf_t *mphf_part_function(const mphf_part_t *p, uint32_t k);
void mphf_part_free(mphf_part_t *p);

/* ---- synthetic keys ------------------------------------------------------ */
/*
 * d_out[i] = output (start + i) of the SplitMix64 generator started at state
 * `seed` (Steele, Lea, Flood, OOPSLA 2014): distinct 64-bit keys, the paper's
 * workload of unique pseudo-random integers (Sec. 4).  Asynchronous on `stream`.
 */
int mphf_keygen(uint64_t *d_out, uint64_t n, uint64_t seed, uint64_t start, void *stream);

/* ---- device memory -------------------------------------------------------- */
/*
 * Scratch and handle memory come from the current device's default
 * stream-ordered memory pool, which keeps the blocks it has mapped (the
 * library sets its release threshold to unlimited): repeated builds over 1e10
 * keys reuse their ~125 GB of scratch instead of mapping it again each time.
 * Memory cached this way is not available to other allocators of the process
 * (torch's, cudaMalloc); mphf_pool_trim waits for the device and returns every
 * unused block of the pool to the driver.
 */
int mphf_pool_trim(void);

/* ---- measurement ---------------------------------------------------------- */
/* Number of kernels this library has launched in this process. */
uint64_t mphf_launch_count(void);
/*
 * Per-kernel timing: while enabled, every kernel the library launches is
 * bracketed by CUDA events on its own stream.  mphf_profile_report waits for
 * the recorded work, then writes lines "name launches total_ms\n" into buf
 * (NUL-terminated, truncated to buflen) and clears the record.
 */
int mphf_profile_enable(int on);
int mphf_profile_report(char *buf, uint64_t buflen);

/*
 * Ceiling measurements: the throughput the memory system gives the accesses
 * the method makes, for rooflines taken in the same run as the kernels they
 * judge.  A lookup probe is one random 32-byte sector load per level
 * (Algorithm 3 with the ranks of Sec. 3.1 stored beside A); ArrayFill marks
 * hits and collisions with random atomic ORs (Sec. 3.2: construction is bound
 * by these random accesses).  Each call launches one kernel on `stream` (time
 * it with events) doing about n random accesses, 8 independent ones in flight
 * per thread, 8 blocks of 256 threads per SM; *performed receives the exact
 * count.  Slot indices come from a per-thread linear congruential stream.
 *   mphf_ceiling_random_loads    loads of `width` bytes (8 or 32) at random
 *                                aligned offsets of d_buf (bytes long, 32-byte
 *                                aligned, at most 2^32 - 1 slots).
 *   mphf_ceiling_random_atomics  atomicOr of one random bit into a random
 *                                word of d_buf (words long, < 2^32); with
 *                                with_return != 0 the old value is used (as
 *                                ArrayFill's hit test does), else not.
 *   d_sink                       device array of 1024 words (rarely written;
 *                                keeps the accesses live).
 * The buffer decides the level measured: an array of tens of MB stays in L2,
 * one of many GB exercises HBM.  MPHF_EINVAL for bad sizes or alignment.
 */
int mphf_ceiling_random_loads(const void *d_buf, uint64_t bytes, uint32_t width, uint64_t n_loads,
                              uint64_t seed, uint64_t *d_sink, uint64_t *performed, void *stream);
int mphf_ceiling_random_atomics(uint64_t *d_buf, uint64_t words, int with_return, uint64_t n_ops,
                                uint64_t seed, uint64_t *d_sink, uint64_t *performed,
                                void *stream);
/* Streaming copy of `bytes` (a multiple of 16, both arrays 16-byte aligned)
 * from d_src to d_dst: the HBM bandwidth a kernel streaming its keys reaches
 * (read + write bytes over the launch's time).  One launch on `stream`. */
int mphf_ceiling_copy(const void *d_src, void *d_dst, uint64_t bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPHF_H */
