/*
 * mphf_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of the cascading-bit-array
 * minimal perfect hash function (BBhash) of Limasset, Rizk, Chikhi and
 * Peterlongo, "Fast and scalable minimal perfect hashing for massive key
 * sets" (arXiv 1702.03154).  It exists to check the CUDA library against:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no source with the CUDA path.
 *
 * The oracle follows the paper's algorithms step by step, in the paper's
 * notation (F_d, A_d, C_d, h_d, gamma, last = L-1), with the conventions the
 * paper leaves open fixed as follows:
 *
 *   mix(z)      the SplitMix64 finalizer (Steele, Lea, Flood, OOPSLA 2014);
 *               the paper only says its hash is built on xor-shifts (Sec. 3.3).
 *   s_d         level seed  = mix(mix(seed) + d).
 *   h_d(x)      = mix(x XOR s_d).
 *   position    p = floor(h_d(x) * m_d / 2^64) (Lemire's fastrange reduction,
 *               in place of the modulo of Algorithms 1-3).
 *   m_d = |A_d| = |C_d| = max(64, ceil(gamma * |F_d|) rounded up to a multiple
 *               of 64), gamma >= 1 real (Sec. 2.2.4); ceil(gamma*n) is taken
 *               from one IEEE-754 double multiply.
 *   indices     0-based: [0, N) instead of the paper's [1, N] (Sec. 1).
 *   rank        exclusive: rank(g) = number of ones of A in bits [0, g)
 *               (Sec. 2.2.3), checkpointed every 512 bits with 64-bit
 *               counters (Sec. 3.1): rank[b] = ones in bits [0, 512 b).
 *   levels      L levels numbered 0 .. L-1 (D = 25 by default, Sec. 3.5);
 *               keys still colliding after level L-1 go to the fallback.
 *   fallback    the table of leftover keys of Sec. 3.5 is a sorted array of
 *               the leftover keys; key at sorted position i gets index
 *               N - n_fb + i (the range Algorithm 1 gives it).
 *   duplicates  identical keys collide at every level, so they reach the
 *               fallback; two equal neighbours there -> ORACLE_EDUPLICATE.
 *   non-members Algorithm 3 run as is: the first level whose bit is 1 gives
 *               the rank, else a fallback hit, else UINT64_MAX.
 *   strings     byte-string keys (Sec. 4.4) become 64-bit keys by the rule of
 *               oracle_string_key below, then take the same path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2
#define ORACLE_EDUPLICATE 3

#define ORACLE_MAX_LEVELS 64
#define ORACLE_RANK_BLOCK 512 /* Sec. 3.1: one 64-bit counter every 512 bits */

/* Optional test hook: replaces the position of key x at level d (must be < m). */
typedef uint64_t (*oracle_pos_hook)(void *user, uint32_t level, uint64_t key, uint64_t m);

typedef struct oracle_mphf {
    uint64_t N;
    double gamma;
    uint32_t L;          /* level budget */
    uint32_t L_used;     /* levels actually built (index of the last one + 1) */
    uint64_t seed;
    uint64_t n[ORACLE_MAX_LEVELS + 1]; /* n[d] = |F_d|; n[L_used] = |fallback| */
    uint64_t m[ORACLE_MAX_LEVELS];     /* |A_d| in bits */
    uint64_t off[ORACLE_MAX_LEVELS];   /* first bit of A_d inside A */
    uint64_t s[ORACLE_MAX_LEVELS];     /* level seeds s_d */
    uint64_t M;                        /* total bits of A = sum m_d */
    unsigned char *bitA;               /* A as one byte per bit, M entries */
    unsigned char *bitC[ORACLE_MAX_LEVELS]; /* C_d kept for the invariant checks */
    uint64_t *rank;                    /* ceil(M / 512) checkpoints */
    uint64_t n_fb;
    uint64_t *fb;                      /* sorted leftover keys */
    oracle_pos_hook hook;
    void *hook_user;
} oracle_mphf;

/* ---- hash pieces ------------------------------------------------------- */

/* SplitMix64 finalizer: the published mixing function of SplitMix64. */
uint64_t oracle_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* s_d: seed of the level-d hash function h_d (Sec. 2.1: every level hashes with its own function). */
uint64_t oracle_level_seed(uint64_t seed, uint32_t d)
{
    return oracle_mix(oracle_mix(seed) + (uint64_t)d);
}

/* h_d(x) (Sec. 3.3). */
uint64_t oracle_hash(uint64_t x, uint64_t s_d)
{
    return oracle_mix(x ^ s_d);
}

/* Reduction of a 64-bit hash onto [0, m): floor(h * m / 2^64). */
uint64_t oracle_fastrange(uint64_t h, uint64_t m)
{
    return (uint64_t)(((unsigned __int128)h * (unsigned __int128)m) >> 64);
}

/* |A_d| for |F_d| = n keys (Sec. 2.2.4: |A_d| = gamma |F_d|). */
uint64_t oracle_level_bits(uint64_t n, double gamma)
{
    double t = gamma * (double)n;
    uint64_t c = (uint64_t)t;
    if ((double)c < t)
        c += 1;                      /* ceil(gamma * n) */
    c = (c + 63) / 64 * 64;          /* whole 64-bit words */
    if (c < 64)
        c = 64;
    return c;
}

static uint64_t position(const oracle_mphf *h, uint32_t d, uint64_t x)
{
    if (h->hook)
        return h->hook(h->hook_user, d, x, h->m[d]);
    return oracle_fastrange(oracle_hash(x, h->s[d]), h->m[d]);
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

void oracle_free(oracle_mphf *h)
{
    if (!h)
        return;
    free(h->bitA);
    for (uint32_t d = 0; d < ORACLE_MAX_LEVELS; d++)
        free(h->bitC[d]);
    free(h->rank);
    free(h->fb);
    free(h);
}

/*
 * Algorithm 2 (ArrayFill) for level d: hash every key of F into A_d / C_d,
 * read as an if / else-if chain on (A[p], C[p]) so that exactly one branch
 * fires per key, which is what the three implications of Sec. 2.2.1 state:
 *   (0,0) -> A=1;   (1,0) -> A=0, C=1;   (0,1) -> skip.
 */
static void fill_one(unsigned char *A, unsigned char *C, uint64_t p)
{
    if (A[p] == 0 && C[p] == 0) {
        A[p] = 1;
    } else if (A[p] == 1 && C[p] == 0) {
        A[p] = 0;
        C[p] = 1;
    } else {
        /* A[p] == 0 and C[p] == 1: skip.  (1,1) never happens. */
    }
}

static void array_fill(const oracle_mphf *h, uint32_t d, const uint64_t *F, uint64_t n,
                       unsigned char *A, unsigned char *C)
{
    for (uint64_t i = 0; i < n; i++)
        fill_one(A, C, position(h, d, F[i]));
}

/*
 * Algorithm 1 (MPHF construction) followed by the rank checkpoints of
 * Sec. 3.1 and the fallback table of Sec. 3.5.
 */
int oracle_build_hooked(const uint64_t *keys, uint64_t N, double gamma, uint32_t L, uint64_t seed,
                        oracle_pos_hook hook, void *hook_user, oracle_mphf **out)
{
    *out = NULL;
    if (!(gamma >= 1.0) || isinf(gamma) || L < 1 || L > ORACLE_MAX_LEVELS || (N > 0 && !keys))
        return ORACLE_EINVAL;
    oracle_mphf *h = (oracle_mphf *)calloc(1, sizeof(oracle_mphf));
    if (!h)
        return ORACLE_ENOMEM;
    h->N = N;
    h->gamma = gamma;
    h->L = L;
    h->seed = seed;
    h->hook = hook;
    h->hook_user = hook_user;

    /* F_0 = the key set; F_{i+1} gets the keys of F_i whose bit ended at 0. */
    uint64_t *F = (uint64_t *)malloc((N ? N : 1) * sizeof(uint64_t));
    uint64_t *Fnext = (uint64_t *)malloc((N ? N : 1) * sizeof(uint64_t));
    unsigned char **Alev = (unsigned char **)calloc(ORACLE_MAX_LEVELS, sizeof(unsigned char *));
    if (!F || !Fnext || !Alev) {
        free(F); free(Fnext); free(Alev); oracle_free(h);
        return ORACLE_ENOMEM;
    }
    if (N)
        memcpy(F, keys, N * sizeof(uint64_t));
    uint64_t n = N;
    uint32_t i = 0;
    uint64_t off = 0;
    while (n > 0 && i < L) {           /* levels go on while keys remain, at most L of them */
        h->n[i] = n;
        h->s[i] = oracle_level_seed(seed, i);
        h->m[i] = oracle_level_bits(n, gamma);
        h->off[i] = off;
        unsigned char *A = (unsigned char *)calloc(h->m[i], 1);
        unsigned char *C = (unsigned char *)calloc(h->m[i], 1);
        if (!A || !C) {
            free(A); free(C);
            for (uint32_t d = 0; d < i; d++) free(Alev[d]);
            free(F); free(Fnext); free(Alev); oracle_free(h);
            return ORACLE_ENOMEM;
        }
        array_fill(h, i, F, n, A, C);   /* level i's bit array from its keys (Algorithm 2) */
        uint64_t nn = 0;
        for (uint64_t k = 0; k < n; k++) {
            uint64_t p = position(h, i, F[k]);
            if (A[p] == 0)
                Fnext[nn++] = F[k];      /* not placed: the key goes on to level i+1 */
        }
        Alev[i] = A;
        h->bitC[i] = C;
        off += h->m[i];
        uint64_t *t = F; F = Fnext; Fnext = t;
        n = nn;
        i++;
    }
    h->L_used = i;
    h->n[i] = n;
    h->M = off;

    /* A = A_0 || A_1 || ... || A_last (Sec. 2.1). */
    h->bitA = (unsigned char *)malloc(h->M ? h->M : 1);
    if (!h->bitA) {
        for (uint32_t d = 0; d < i; d++) free(Alev[d]);
        free(F); free(Fnext); free(Alev); oracle_free(h);
        return ORACLE_ENOMEM;
    }
    for (uint32_t d = 0; d < h->L_used; d++) {
        memcpy(h->bitA + h->off[d], Alev[d], h->m[d]);
        free(Alev[d]);
    }
    free(Alev);

    /* Rank checkpoints (Sec. 3.1): rank[b] = ones of A in bits [0, 512 b). */
    uint64_t R = (h->M + ORACLE_RANK_BLOCK - 1) / ORACLE_RANK_BLOCK;
    h->rank = (uint64_t *)malloc((R ? R : 1) * sizeof(uint64_t));
    if (!h->rank) {
        free(F); free(Fnext); oracle_free(h);
        return ORACLE_ENOMEM;
    }
    uint64_t ones = 0;
    for (uint64_t g = 0; g < h->M; g++) {
        if (g % ORACLE_RANK_BLOCK == 0)
            h->rank[g / ORACLE_RANK_BLOCK] = ones;
        ones += h->bitA[g];
    }

    /* Fallback H (Sec. 3.5): the keys left in F_{last+1}, sorted. */
    h->n_fb = n;
    h->fb = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!h->fb) {
        free(F); free(Fnext); oracle_free(h);
        return ORACLE_ENOMEM;
    }
    if (n)
        memcpy(h->fb, F, n * sizeof(uint64_t));
    free(F);
    free(Fnext);
    qsort(h->fb, n, sizeof(uint64_t), cmp_u64);
    for (uint64_t k = 1; k < n; k++) {
        if (h->fb[k] == h->fb[k - 1]) {
            oracle_free(h);
            return ORACLE_EDUPLICATE;
        }
    }
    *out = h;
    return ORACLE_OK;
}

int oracle_build(const uint64_t *keys, uint64_t N, double gamma, uint32_t L, uint64_t seed,
                 oracle_mphf **out)
{
    return oracle_build_hooked(keys, N, gamma, L, seed, NULL, NULL, out);
}

/* rank(g): ones of A strictly before global bit g, from checkpoint + the bits in between. */
static uint64_t rank_at(const oracle_mphf *h, uint64_t g)
{
    uint64_t b = g / ORACLE_RANK_BLOCK;
    uint64_t r = h->rank[b];
    for (uint64_t t = b * ORACLE_RANK_BLOCK; t < g; t++)
        r += h->bitA[t];
    return r;
}

/* Algorithm 3 (MPHF query), minimal form of Sec. 2.2.3, 0-based. */
uint64_t oracle_query(const oracle_mphf *h, uint64_t x)
{
    for (uint32_t i = 0; i < h->L_used; i++) {
        uint64_t p = position(h, i, x);
        if (h->bitA[h->off[i] + p] == 1)
            return rank_at(h, h->off[i] + p);
    }
    /* H[x]: binary search of the sorted fallback. */
    uint64_t lo = 0, hi = h->n_fb;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (h->fb[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (lo < h->n_fb && h->fb[lo] == x)
        return h->N - h->n_fb + lo;
    return UINT64_MAX;
}

void oracle_lookup(const oracle_mphf *h, const uint64_t *keys, uint64_t n, uint64_t *out)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = oracle_query(h, keys[i]);
}

/* Level of a key: the d that answers it, L_used for the fallback / a miss. */
uint32_t oracle_key_level(const oracle_mphf *h, uint64_t x)
{
    for (uint32_t i = 0; i < h->L_used; i++) {
        uint64_t p = position(h, i, x);
        if (h->bitA[h->off[i] + p] == 1)
            return i;
    }
    return h->L_used;
}

/* ---- introspection ------------------------------------------------------ */

uint32_t oracle_num_levels(const oracle_mphf *h) { return h->L_used; }
uint64_t oracle_total_bits(const oracle_mphf *h) { return h->M; }
uint64_t oracle_num_fallback(const oracle_mphf *h) { return h->n_fb; }
uint64_t oracle_num_rank(const oracle_mphf *h) { return (h->M + ORACLE_RANK_BLOCK - 1) / ORACLE_RANK_BLOCK; }

int oracle_level_info(const oracle_mphf *h, uint32_t d, uint64_t *n_d, uint64_t *m_d, uint64_t *off_d,
                      uint64_t *s_d)
{
    if (d >= h->L_used)
        return ORACLE_EINVAL;
    *n_d = h->n[d];
    *m_d = h->m[d];
    *off_d = h->off[d];
    *s_d = h->s[d];
    return ORACLE_OK;
}

/* A packed into 64-bit words: global bit g is bit (g % 64) of word g / 64. */
void oracle_copy_bits(const oracle_mphf *h, uint64_t *words)
{
    uint64_t W = h->M / 64;
    for (uint64_t w = 0; w < W; w++) {
        uint64_t v = 0;
        for (uint64_t b = 0; b < 64; b++)
            if (h->bitA[w * 64 + b])
                v |= 1ULL << b;
        words[w] = v;
    }
}

/* C_d packed the same way (m_d / 64 words). */
int oracle_copy_collision_bits(const oracle_mphf *h, uint32_t d, uint64_t *words)
{
    if (d >= h->L_used)
        return ORACLE_EINVAL;
    uint64_t W = h->m[d] / 64;
    for (uint64_t w = 0; w < W; w++) {
        uint64_t v = 0;
        for (uint64_t b = 0; b < 64; b++)
            if (h->bitC[d][w * 64 + b])
                v |= 1ULL << b;
        words[w] = v;
    }
    return ORACLE_OK;
}

void oracle_copy_rank(const oracle_mphf *h, uint64_t *out)
{
    uint64_t R = oracle_num_rank(h);
    for (uint64_t b = 0; b < R; b++)
        out[b] = h->rank[b];
}

void oracle_copy_fallback(const oracle_mphf *h, uint64_t *out)
{
    for (uint64_t i = 0; i < h->n_fb; i++)
        out[i] = h->fb[i];
}

/*
 * Size of the function in bits per key with the rank structure of Sec. 3.1
 * ((1 + 64/512) per bit of A) and 64 bits per fallback key; level metadata
 * (a few words per level) is not counted.
 */
/*
 * The same with one 64-bit counter every rank_block bits: Sec. 3.1's default
 * is 512; the minirank setting of Sec. 4.3 (Table 1) samples every 1024.
 */
double oracle_bits_per_key_sampled(const oracle_mphf *h, uint64_t rank_block)
{
    if (h->N == 0 || rank_block == 0)
        return 0.0;
    uint64_t counters = (h->M + rank_block - 1) / rank_block;
    double bits = (double)h->M + 64.0 * (double)counters + 64.0 * (double)h->n_fb;
    return bits / (double)h->N;
}

double oracle_bits_per_key(const oracle_mphf *h)
{
    return oracle_bits_per_key_sampled(h, ORACLE_RANK_BLOCK);
}

/*
 * String keys (Sec. 4.4, Table 2: the method run on n-grams and random words
 * of 18 characters).  The method itself takes 64-bit keys; a string is first
 * turned into one by this library's convention (the paper does not give its
 * string hash):
 *
 *   h = mix(seed + (len + 1) * 0x9E3779B97F4A7C15)
 *   for each group of 8 bytes of the string, in order (the last group padded
 *   with zero bytes): w = the 8 bytes read as a little-endian integer,
 *   h = mix(h XOR w)
 *   key = h
 *
 * The length enters the first state, so a string and the same string with
 * zero bytes appended give different keys (len + 1 keeps the empty string
 * away from mix's fixed point mix(0) = 0).  For a fixed length and fixed
 * leading groups the last step is a bijection of the last group (mix is one),
 * so strings that differ only in their last 8-byte group never collide.
 */
uint64_t oracle_string_key(const uint8_t *s, uint64_t len, uint64_t seed)
{
    uint64_t h = oracle_mix(seed + (len + 1) * 0x9E3779B97F4A7C15ULL);
    for (uint64_t k = 0; k < len; k += 8) {
        uint64_t w = 0;
        for (uint64_t i = 0; i < 8; i++) {
            uint64_t byte = (k + i < len) ? (uint64_t)s[k + i] : 0;
            w |= byte << (8 * i);
        }
        h = oracle_mix(h ^ w);
    }
    return h;
}

/* Keys of n strings: string i is bytes[off[i] .. off[i+1]). */
void oracle_string_keys(const uint8_t *bytes, const uint64_t *off, uint64_t n, uint64_t seed,
                        uint64_t *out)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = oracle_string_key(bytes + off[i], off[i + 1] - off[i], seed);
}

/*
 * One level's ArrayFill over an arbitrary key set, outside a build: keys are
 * hashed with h_d (seed s_d) onto m positions and Algorithm 2 runs on the
 * byte arrays A, C (m entries, zeroed by the caller).  A rank of a
 * multi-GPU build holding a shard of F_d would compute exactly this.
 */
void oracle_fill_level(const uint64_t *keys, uint64_t n, uint64_t s_d, uint64_t m,
                       unsigned char *A, unsigned char *C)
{
    for (uint64_t i = 0; i < n; i++)
        fill_one(A, C, oracle_fastrange(oracle_hash(keys[i], s_d), m));
}

/*
 * The keys whose level position p = fastrange(h_d(x), m) falls inside the
 * window [lo, lo + W) of a level of m positions; they are copied, in input
 * order, to out (room for n keys).  Returns how many there are.  ArrayFill
 * decides every position from the keys hashed to it alone, so these keys
 * and nothing else fix A_d and C_d inside the window.
 */
uint64_t oracle_select_window(const uint64_t *keys, uint64_t n, uint64_t s_d, uint64_t m,
                              uint64_t lo, uint64_t W, uint64_t *out)
{
    uint64_t c = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t p = oracle_fastrange(oracle_hash(keys[i], s_d), m);
        if (p >= lo && p - lo < W)
            out[c++] = keys[i];
    }
    return c;
}

/*
 * Algorithm 2 (ArrayFill) restricted to the window [lo, lo + W) of a level of
 * m positions: A and C hold W entries (position lo + t at entry t, zeroed by
 * the caller); keys hashed outside the window are skipped.
 */
void oracle_fill_window(const uint64_t *keys, uint64_t n, uint64_t s_d, uint64_t m, uint64_t lo,
                        uint64_t W, unsigned char *A, unsigned char *C)
{
    for (uint64_t i = 0; i < n; i++) {
        uint64_t p = oracle_fastrange(oracle_hash(keys[i], s_d), m);
        if (p >= lo && p - lo < W)
            fill_one(A, C, p - lo);
    }
}

/*
 * Exclusive rank inside a window (Sec. 2.2.3 restricted to [lo, lo + W) of a
 * level of m positions whose window bits are A, W entries): for each key whose
 * position p lies in the window with A[p - lo] = 1, out = ones of A in
 * [lo, p); other keys get UINT64_MAX.  For the window at the very start of
 * the concatenated bit array this is the key's index.
 */
int oracle_window_ranks(const uint64_t *keys, uint64_t n, uint64_t s_d, uint64_t m, uint64_t lo,
                        uint64_t W, const unsigned char *A, uint64_t *out)
{
    uint64_t *before = (uint64_t *)malloc((W + 1) * sizeof(uint64_t));
    if (!before)
        return ORACLE_ENOMEM;
    before[0] = 0;
    for (uint64_t t = 0; t < W; t++)
        before[t + 1] = before[t] + A[t];
    for (uint64_t i = 0; i < n; i++) {
        uint64_t p = oracle_fastrange(oracle_hash(keys[i], s_d), m);
        if (p >= lo && p - lo < W && A[p - lo] == 1)
            out[i] = before[p - lo];
        else
            out[i] = UINT64_MAX;
    }
    free(before);
    return ORACLE_OK;
}

/*
 * Combine the fills of two disjoint key sets into the fill of their union
 * (the exchange step of a monolithic multi-GPU level).  Per position, A says
 * "exactly one key" and C says "two or more", so the union has two or more
 * if either side has, or if both sides have exactly one; it has exactly one
 * if one side has one and the union has no collision:
 *   C = C1 | C2 | (A1 & A2),   A = (A1 | A2) & ~C.
 * The result is written to (A1, C1).
 */
void oracle_merge_fill(unsigned char *A1, unsigned char *C1, const unsigned char *A2,
                       const unsigned char *C2, uint64_t m)
{
    for (uint64_t p = 0; p < m; p++) {
        unsigned char c = (unsigned char)(C1[p] | C2[p] | (A1[p] & A2[p]));
        A1[p] = (unsigned char)((A1[p] | A2[p]) & !c);
        C1[p] = c;
    }
}

/*
 * Partitioned use of the method.  Sec. 4.3 notes that other tools split the
 * key set into partitions and build one small function per partition, and
 * that the same split could be put in front of this method.  Here key x goes
 * to part p = floor(mix(x XOR mix(part_seed)) * K / 2^64) of K parts; part p
 * gets its own function, built over its keys alone; the global index of a key
 * is the number of keys of parts 0 .. p-1 plus its index within part p.
 */
uint32_t oracle_part_of(uint64_t x, uint32_t K, uint64_t part_seed)
{
    return (uint32_t)oracle_fastrange(oracle_mix(x ^ oracle_mix(part_seed)), (uint64_t)K);
}

void oracle_parts(const uint64_t *keys, uint64_t n, uint32_t K, uint64_t part_seed, uint32_t *out)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = oracle_part_of(keys[i], K, part_seed);
}
