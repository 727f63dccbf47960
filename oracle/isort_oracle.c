/*
 * ORACLE — test infrastructure only.
 *
 * A plain, serial, obviously-correct CPU restatement of what the integer-sort
 * hot path computes. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Definition of the result (every entry point): the stable sort of the
 * (key, payload) pairs by unsigned key, i.e. ascending by (key, original
 * index). Integer keys have exactly one such output.
 *
 * Functions and the passages they follow (Gerbessiotis, "Integer sorting on
 * multicores: some (experiments and) observations", arXiv:1708.09495):
 *   oracle_count_round_*  one count-sort round: count, prefix, ordered output
 *                         (Section 3, "Serial radix-r radix-sort", eq. Ts)
 *   oracle_lsd_*          SR4 generalised: ceil(key_bits / radix_bits) rounds,
 *                         least significant digit first (Section 3, eq. Ts;
 *                         fewer rounds for a known key range, Section 1 and
 *                         Section 2's remarks on bounded key values)
 *   oracle_digit_hist_*   the count step of every round, for all rounds
 *   oracle_btn_u32        BTN: p sorted blocks + lg p (lg p + 1)/2 merge-split
 *                         stages of a p-input bitonic network (Section 2; Section 3
 *                         "Bitonic Sort", eq. Tb)
 *   oracle_oet_u32        OET: p sorted blocks + p rounds of odd-even
 *                         transposition with merge-split (Section 2; Section 3
 *                         "Odd-even transposition sort", eq. To)
 *   oracle_insertion_*    brute force: stable insertion sort (a pin, not the
 *                         paper's method)
 *   oracle_segmented_u32  the LSD sort applied to each CSR segment on its own
 *   oracle_partition_*    the routing step of a sample sort across p processors:
 *                         splitters chosen regularly from a sorted sample
 *                         (Section 2, the sample sorts with regular sampling),
 *                         every key routed to the range of its splitters by one
 *                         count-sort round on that range (Section 3, eq. Tp's
 *                         key routing)
 *   invariant checkers    non-decreasing, stability (payload = index), 64-bit
 *                         commutative multiset hash
 *
 * Readings where the paper is silent:
 *   - lg r need not divide the key width: the last digit is narrower.
 *   - BTN/OET compare (key, original index) so that the unique stable order
 *     comes out; blocks are padded with (max key, index >= n) pads.
 *   - OET round t pairs blocks (j, j+1) with j = t mod 2, t = 0..p-1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0 /* >0 only in the tests' deliberately broken builds */
#endif

static int num_rounds(int key_bits, int radix_bits) { return (key_bits + radix_bits - 1) / radix_bits; }

/* ------------------------------------------------------------------------
 * One count-sort round over digit (key >> shift) & (2^width - 1).
 * Count, exclusive prefix, then the output written in input order, which makes
 * the round stable (Section 3, Serial radix-r: read for counting, read again
 * for output, write the output).
 * ---------------------------------------------------------------------- */
#define DEFINE_COUNT_ROUND(NAME, KT)                                                                 \
    int NAME(const KT* kin, const uint32_t* vin, KT* kout, uint32_t* vout, size_t n, int shift,    \
             int width) {                                                                           \
        size_t nb = (size_t)1 << width;                                                             \
        KT mask = (KT)(nb - 1);                                                                     \
        size_t* count = (size_t*)calloc(nb, sizeof(size_t));                                        \
        if (!count) return -1;                                                                      \
        for (size_t i = 0; i < n; ++i) count[(size_t)((kin[i] >> shift) & mask)]++;                  \
        size_t run = 0;                                                                             \
        for (size_t b = 0; b < nb; ++b) { size_t c = count[b]; count[b] = run; run += c; }          \
        if (ORACLE_MUTANT == 1) { /* planted: ties placed from the bucket end (unstable) */        \
            for (size_t b = 0; b + 1 < nb; ++b) count[b] = count[b + 1];                            \
            count[nb - 1] = n;                                                                      \
            for (size_t i = 0; i < n; ++i) {                                                        \
                size_t d = (size_t)((kin[i] >> shift) & mask);                                      \
                size_t o = --count[d];                                                              \
                kout[o] = kin[i];                                                                   \
                if (vin) vout[o] = vin[i];                                                          \
            }                                                                                       \
        } else {                                                                                    \
            for (size_t i = 0; i < n; ++i) {                                                        \
                size_t d = (size_t)((kin[i] >> shift) & mask);                                      \
                size_t o = count[d]++;                                                              \
                kout[o] = kin[i];                                                                   \
                if (vin && ORACLE_MUTANT != 2) vout[o] = vin[i];                                    \
                if (vin && ORACLE_MUTANT == 2) vout[i] = vin[i]; /* planted: payload left behind */ \
            }                                                                                       \
        }                                                                                           \
        free(count);                                                                                \
        return 0;                                                                                   \
    }

DEFINE_COUNT_ROUND(oracle_count_round_u32, uint32_t)
DEFINE_COUNT_ROUND(oracle_count_round_u64, uint64_t)

/* ------------------------------------------------------------------------
 * LSD radix sort: rounds d = 0..P-1 over digits of radix_bits bits, starting at
 * the least significant one; P = ceil(key_bits / radix_bits) (Section 3, eq. Ts
 * with 32/lg r rounds; fewer rounds when keys are known to be < 2^key_bits).
 * The result overwrites keys/vals. Returns 0, or -1 on bad arguments / memory.
 * ---------------------------------------------------------------------- */
#define DEFINE_LSD(NAME, ROUND, KT, KBITS)                                                          \
    int NAME(KT* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits) {                   \
        if (key_bits == 0) key_bits = KBITS;                                                        \
        if (key_bits < 1 || key_bits > KBITS || radix_bits < 1 || radix_bits > 16) return -1;      \
        if (n <= 1) return 0;                                                                       \
        KT* k2 = (KT*)malloc(n * sizeof(KT));                                                       \
        uint32_t* v2 = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;                       \
        if (!k2 || (vals && !v2)) { free(k2); free(v2); return -1; }                                \
        KT *ka = keys, *kb = k2;                                                                    \
        uint32_t *va = vals, *vb = v2;                                                              \
        int P = num_rounds(key_bits, radix_bits);                                                   \
        if (ORACLE_MUTANT == 3) P = key_bits / radix_bits; /* planted: short last digit dropped */  \
        for (int d = 0; d < P; ++d) {                                                               \
            int shift = d * radix_bits;                                                             \
            int width = key_bits - shift < radix_bits ? key_bits - shift : radix_bits;              \
            if (ROUND(ka, va, kb, vb, n, shift, width)) { P = -1; break; }                          \
            KT* tk = ka; ka = kb; kb = tk;                                                          \
            uint32_t* tv = va; va = vb; vb = tv;                                                    \
        }                                                                                           \
        if (ka != keys) {                                                                           \
            memcpy(keys, ka, n * sizeof(KT));                                                       \
            if (vals) memcpy(vals, va, n * sizeof(uint32_t));                                       \
        }                                                                                           \
        free(k2); free(v2);                                                                         \
        return P < 0 ? -1 : 0;                                                                      \
    }

DEFINE_LSD(oracle_lsd_u32, oracle_count_round_u32, uint32_t, 32)
DEFINE_LSD(oracle_lsd_u64, oracle_count_round_u64, uint64_t, 64)

/* ------------------------------------------------------------------------
 * Sample-sort partition into `parts` ranges. Splitter j (1 <= j < parts) is
 * sorted_sample[floor(j m / parts)] (a regular choice among the m sorted
 * sample keys); the range of key k is the number of splitters <= k, so keys
 * equal to a splitter go to the range that splitter opens. The keys are then
 * routed by one stable count-sort round whose digit is the range: count,
 * exclusive prefix, output in input order. counts[r] = keys in range r.
 * Returns 0, or -1 on bad arguments / memory.
 * ---------------------------------------------------------------------- */
#define DEFINE_PARTITION(NAME, KT)                                                                  \
    int NAME(const KT* keys, const uint32_t* vals, KT* kout, uint32_t* vout, size_t n,              \
             const KT* sorted_sample, size_t m, int parts, uint64_t* counts) {                      \
        if (parts < 1 || parts > 256 || (parts > 1 && m < 1)) return -1;                            \
        KT spl[256];                                                                                \
        const int ns = parts - 1;                                                                   \
        for (int j = 1; j < parts; ++j) spl[j - 1] = sorted_sample[(size_t)((uint64_t)j * m / (uint64_t)parts)]; \
        uint8_t* r = (uint8_t*)malloc(n ? n : 1);                                                   \
        if (!r) return -1;                                                                          \
        memset(counts, 0, sizeof(uint64_t) * (size_t)parts);                                        \
        for (size_t i = 0; i < n; ++i) {                                                            \
            int q = 0;                                                                              \
            if (ORACLE_MUTANT == 7) { while (q < ns && spl[q] < keys[i]) ++q; } /* planted: < */    \
            else { while (q < ns && spl[q] <= keys[i]) ++q; }                                       \
            r[i] = (uint8_t)q;                                                                      \
            counts[q]++;                                                                            \
        }                                                                                           \
        uint64_t start[256], run = 0;                                                               \
        for (int q = 0; q < parts; ++q) { start[q] = run; run += counts[q]; }                       \
        for (size_t i = 0; i < n; ++i) {                                                            \
            const uint64_t o = start[r[i]]++;                                                       \
            kout[o] = keys[i];                                                                      \
            if (vals) vout[o] = vals[i];                                                            \
        }                                                                                           \
        free(r);                                                                                    \
        return 0;                                                                                   \
    }

DEFINE_PARTITION(oracle_partition_u32, uint32_t)
DEFINE_PARTITION(oracle_partition_u64, uint64_t)

/* Per-round digit histograms of the input: hist[d * 2^radix_bits + b] = number
 * of keys whose round-d digit equals b (the count step of Section 3's
 * count-sort, taken for all rounds at once; counts are invariant under the
 * permutations the earlier rounds apply). */
#define DEFINE_HIST(NAME, KT, KBITS)                                                                \
    int NAME(const KT* keys, size_t n, int key_bits, int radix_bits, uint64_t* hist) {             \
        if (key_bits == 0) key_bits = KBITS;                                                        \
        if (key_bits < 1 || key_bits > KBITS || radix_bits < 1 || radix_bits > 16) return -1;      \
        int P = num_rounds(key_bits, radix_bits);                                                   \
        size_t nb = (size_t)1 << radix_bits;                                                        \
        memset(hist, 0, sizeof(uint64_t) * nb * (size_t)P);                                         \
        for (int d = 0; d < P; ++d) {                                                               \
            int shift = d * radix_bits;                                                             \
            int width = key_bits - shift < radix_bits ? key_bits - shift : radix_bits;              \
            KT mask = (KT)(((uint64_t)1 << width) - 1);                                             \
            for (size_t i = 0; i < n; ++i) hist[(size_t)d * nb + (size_t)((keys[i] >> shift) & mask)]++; \
        }                                                                                           \
        return P;                                                                                   \
    }

DEFINE_HIST(oracle_digit_hist_u32, uint32_t, 32)
DEFINE_HIST(oracle_digit_hist_u64, uint64_t, 64)

/* ------------------------------------------------------------------------
 * Brute force: stable insertion sort (a pin for the oracle, not the method).
 * ---------------------------------------------------------------------- */
#define DEFINE_INSERTION(NAME, KT)                                                                  \
    void NAME(KT* keys, uint32_t* vals, size_t n) {                                                 \
        for (size_t i = 1; i < n; ++i) {                                                            \
            KT k = keys[i];                                                                         \
            uint32_t v = vals ? vals[i] : 0;                                                        \
            size_t j = i;                                                                           \
            while (j > 0 && keys[j - 1] > k) {                                                      \
                keys[j] = keys[j - 1];                                                              \
                if (vals) vals[j] = vals[j - 1];                                                    \
                --j;                                                                                \
            }                                                                                       \
            keys[j] = k;                                                                            \
            if (vals) vals[j] = v;                                                                  \
        }                                                                                           \
    }

DEFINE_INSERTION(oracle_insertion_u32, uint32_t)
DEFINE_INSERTION(oracle_insertion_u64, uint64_t)

/* ------------------------------------------------------------------------
 * BTN and OET (Section 2; Section 3 eqs. Tb and To).
 *
 * Items are (key, original index) pairs compared lexicographically, so ties
 * resolve to input order and the output is the unique stable order. The n
 * items are padded to p * m (m = ceil(n/p)) with pads (2^32-1, n + j) that sort
 * after every real item, split into p blocks of m, and each block is sorted on
 * its own (the paper's SR4 local sort: here the oracle's LSD round applied to
 * the composite (key << 32 | index), which sorts by key then index).
 * Then the network runs with "compare-exchange" replaced by merge-split: the
 * two sorted blocks are merged and the lower-indexed block keeps the m smallest
 * (or, for a descending comparator, the m largest).
 * ---------------------------------------------------------------------- */
static void merge_split(uint64_t* lo_blk, uint64_t* hi_blk, size_t m, uint64_t* tmp, int lower_keeps_small) {
    size_t a = 0, b = 0;
    for (size_t t = 0; t < 2 * m; ++t) {
        if (b >= m || (a < m && lo_blk[a] <= hi_blk[b])) tmp[t] = lo_blk[a++];
        else tmp[t] = hi_blk[b++];
    }
    if (lower_keeps_small) {
        memcpy(lo_blk, tmp, m * sizeof(uint64_t));
        memcpy(hi_blk, tmp + m, m * sizeof(uint64_t));
    } else {
        memcpy(lo_blk, tmp + m, m * sizeof(uint64_t));
        memcpy(hi_blk, tmp, m * sizeof(uint64_t));
    }
}

static uint64_t* make_blocks(const uint32_t* keys, size_t n, int p, size_t* m_out) {
    size_t m = (n + (size_t)p - 1) / (size_t)p;
    if (m == 0) m = 1;
    size_t tot = m * (size_t)p;
    uint64_t* it = (uint64_t*)malloc(tot * sizeof(uint64_t));
    if (!it) return NULL;
    for (size_t i = 0; i < tot; ++i)
        it[i] = i < n ? ((uint64_t)keys[i] << 32) | (uint64_t)i : (0xFFFFFFFFULL << 32) | (uint64_t)i;
    /* local sort of each block (SR4 over the 64-bit composite) */
    for (int j = 0; j < p; ++j)
        if (oracle_lsd_u64(it + (size_t)j * m, NULL, m, 64, 8)) { free(it); return NULL; }
    *m_out = m;
    return it;
}

static void unblock(const uint64_t* it, const uint32_t* keys_in_copy, uint32_t* keys, uint32_t* vals,
                    const uint32_t* vals_in_copy, size_t n) {
    /* pads sort last, so the first n items are the real ones */
    for (size_t i = 0; i < n; ++i) {
        uint32_t idx = (uint32_t)(it[i] & 0xFFFFFFFFu);
        keys[i] = keys_in_copy[idx];
        if (vals) vals[i] = vals_in_copy[idx];
    }
}

static int is_pow2(int p) { return p > 0 && (p & (p - 1)) == 0; }

/* BTN: p a power of two. *stages receives the number of merge-split stages
 * executed, lg p (lg p + 1) / 2. n must be < 2^32. */
int oracle_btn_u32(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages) {
    if (!is_pow2(p) || n >= ((size_t)1 << 32) - (size_t)p) return -1;
    uint64_t st = 0;
    if (n == 0) { if (stages) *stages = 0; return 0; }
    size_t m;
    uint64_t* it = make_blocks(keys, n, p, &m);
    uint32_t* kc = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* vc = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    uint64_t* tmp = (uint64_t*)malloc(2 * m * sizeof(uint64_t));
    if (!it || !kc || (vals && !vc) || !tmp) { free(it); free(kc); free(vc); free(tmp); return -1; }
    memcpy(kc, keys, n * sizeof(uint32_t));
    if (vals) memcpy(vc, vals, n * sizeof(uint32_t));
    /* Bitonic network on p blocks: for merge size k = 2, 4, ..., p and
     * distance j = k/2, ..., 1, block i pairs with block i ^ j; the pair is in
     * an ascending comparator iff (i & k) == 0. */
    for (int k = 2; k <= p; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = 0; i < p; ++i) {
                int l = i ^ j;
                if (l <= i) continue;
                int asc = (i & k) == 0;
                if (ORACLE_MUTANT == 4) asc = 1; /* planted: direction ignored */
                merge_split(it + (size_t)i * m, it + (size_t)l * m, m, tmp, asc);
            }
            ++st;
        }
    }
    unblock(it, kc, keys, vals, vc, n);
    if (stages) *stages = st;
    free(it); free(kc); free(vc); free(tmp);
    return 0;
}

/* OET: any p >= 1. *rounds receives the number of transposition rounds, p. */
int oracle_oet_u32(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* rounds) {
    if (p < 1 || n >= ((size_t)1 << 32) - (size_t)p) return -1;
    uint64_t rd = 0;
    if (n == 0) { if (rounds) *rounds = 0; return 0; }
    size_t m;
    uint64_t* it = make_blocks(keys, n, p, &m);
    uint32_t* kc = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* vc = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    uint64_t* tmp = (uint64_t*)malloc(2 * m * sizeof(uint64_t));
    if (!it || !kc || (vals && !vc) || !tmp) { free(it); free(kc); free(vc); free(tmp); return -1; }
    memcpy(kc, keys, n * sizeof(uint32_t));
    if (vals) memcpy(vc, vals, n * sizeof(uint32_t));
    int R = p;
    if (ORACLE_MUTANT == 5) R = p - 1; /* planted: one round short */
    for (int t = 0; t < R; ++t) {
        for (int j = t & 1; j + 1 < p; j += 2) merge_split(it + (size_t)j * m, it + (size_t)(j + 1) * m, m, tmp, 1);
        ++rd;
    }
    unblock(it, kc, keys, vals, vc, n);
    if (rounds) *rounds = rd;
    free(it); free(kc); free(vc); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------
 * Segmented: segment s is [off[s], off[s+1]); each is LSD-sorted on its own.
 * ---------------------------------------------------------------------- */
int oracle_segmented_u32(uint32_t* keys, uint32_t* vals, const uint64_t* off, size_t nseg, int key_bits,
                         int radix_bits) {
    for (size_t s = 0; s < nseg; ++s) {
        if (off[s + 1] < off[s]) return -1;
        size_t len = (size_t)(off[s + 1] - off[s]);
        if (oracle_lsd_u32(keys + off[s], vals ? vals + off[s] : NULL, len, key_bits, radix_bits)) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Invariant checkers.
 * ---------------------------------------------------------------------- */
int oracle_is_sorted_u32(const uint32_t* k, size_t n) {
    for (size_t i = 1; i < n; ++i)
        if (k[i - 1] > k[i]) return 0;
    return 1;
}
int oracle_is_sorted_u64(const uint64_t* k, size_t n) {
    for (size_t i = 1; i < n; ++i)
        if (k[i - 1] > k[i]) return 0;
    return 1;
}

/* With payload = original index, a stable sorted output has strictly
 * increasing payloads inside every run of equal keys. */
int oracle_is_stable_u32(const uint32_t* k, const uint32_t* v, size_t n) {
    for (size_t i = 1; i < n; ++i)
        if (k[i - 1] == k[i] && v[i - 1] >= v[i]) return 0;
    return 1;
}
int oracle_is_stable_u64(const uint64_t* k, const uint32_t* v, size_t n) {
    for (size_t i = 1; i < n; ++i)
        if (k[i - 1] == k[i] && v[i - 1] >= v[i]) return 0;
    return 1;
}

/* Commutative multiset hash: sum over items of mix(key ^ rotl(val, 32)) mod
 * 2^64, mix being SplitMix64's bijective finaliser (Steele, Lea & Flood 2014).
 * Equal multisets of (key, val) pairs give equal sums. */
static inline uint64_t fmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t rotl32(uint64_t v) { return (v << 32) | (v >> 32); }

uint64_t oracle_multiset_hash_u32(const uint32_t* k, const uint32_t* v, size_t n) {
    uint64_t h = 0;
    for (size_t i = 0; i < n; ++i) {
        uint64_t val = v ? (uint64_t)v[i] : 0;
        if (ORACLE_MUTANT == 6) val = 0; /* planted: payload ignored */
        h += fmix((uint64_t)k[i] ^ rotl32(val));
    }
    return h;
}
uint64_t oracle_multiset_hash_u64(const uint64_t* k, const uint32_t* v, size_t n) {
    uint64_t h = 0;
    for (size_t i = 0; i < n; ++i) h += fmix(k[i] ^ rotl32(v ? (uint64_t)v[i] : 0));
    return h;
}

/* ------------------------------------------------------------------------
 * Learned-bucket sort (no counterpart in the paper; its output is still the
 * stable sort above). These restate the model's definitions for checking.
 * ---------------------------------------------------------------------- */
#include <math.h>

#define PWL_SEG 256
#define PWL_KNOTS 257

/* Sample indices: index_j = floor(r_j * n / 2^64), r_j the j-th output of
 * SplitMix64 (Steele, Lea & Flood 2014) started from state seed. */
static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void oracle_sample_indices(uint64_t n, uint32_t m, uint64_t seed, uint64_t* idx) {
    for (uint32_t j = 0; j < m; ++j) {
        uint64_t r = sm_mix(seed + (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ULL);
        idx[j] = (uint64_t)(((unsigned __int128)r * n) >> 64);
    }
}

/* The bucket model in float, every operation rounded to nearest in this order
 * (the definition the sort uses; monotone in the key by construction):
 *   u = float(key) * 2^-kb;
 *   j = the largest j < 256 with X[j] <= u (j = 255 when u >= X[256]);
 *   slope_j = (Y[j+1] - Y[j]) / (X[j+1] - X[j]), 0 when X[j+1] = X[j],
 *             at most 1e30;
 *   f = Y[j] + (u - X[j]) * slope_j, then clamped to [Y[j], Y[j+1]];
 *   bucket = min(B - 1, trunc(f * B)).
 * Within a segment f grows with u (each operation is monotone) and the clamp
 * keeps segment j below segment j+1, so the bucket never decreases as the key
 * grows. */
static int pwl_segment_f32(const float* X, float u) {
    if (!(u < X[PWL_SEG])) return PWL_SEG - 1;
    int lo = 0, hi = PWL_SEG;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (X[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

static float pwl_slope_f32(const float* X, const float* Y, int j) {
    float dx = X[j + 1] - X[j];
    if (!(dx > 0.f)) return 0.f;
    float sl = (Y[j + 1] - Y[j]) / dx;
    return sl < 1e30f ? sl : 1e30f;
}

static float norm_key(uint64_t k, int key_width, float scale) {
    float fk = key_width == 32 ? (float)(uint32_t)k : (float)k;
    return fk * scale;
}

static uint32_t bucket_model(const float* X, const float* Y, int B, float u) {
    int j = pwl_segment_f32(X, u);
    float sl = pwl_slope_f32(X, Y, j);
    float f = Y[j] + (u - X[j]) * sl;
    if (f < Y[j]) f = Y[j];
    if (f > Y[j + 1]) f = Y[j + 1];
    float fb = f * (float)B;
    uint32_t b = (uint32_t)fb; /* f >= 0: truncation is the floor */
    return b > (uint32_t)(B - 1) ? (uint32_t)(B - 1) : b;
}

uint32_t oracle_bucket_of(const float* X, const float* Y, int key_width, int key_bits, int B, uint64_t key) {
    return bucket_model(X, Y, B, norm_key(key, key_width, ldexpf(1.0f, -key_bits)));
}

/* The model's bucket of every key. */
void oracle_bucket_ids(const void* keys, int key_width, size_t n, int key_bits, const float* X, const float* Y,
                       int B, uint32_t* ids) {
    float scale = ldexpf(1.0f, -key_bits);
    for (size_t i = 0; i < n; ++i) {
        uint64_t k = key_width == 32 ? (uint64_t)((const uint32_t*)keys)[i] : ((const uint64_t*)keys)[i];
        ids[i] = bucket_model(X, Y, B, norm_key(k, key_width, scale));
    }
}

/* Splitter table (the buckets' lower key bounds): s_0 = 0; for b = 1..B-1,
 * s_b = the first key in [0, 2^kb) whose bucket is at least b (the largest key
 * if none), by bisection over the keys. */
void oracle_splitters(const float* X, const float* Y, int key_width, int key_bits, int B, uint64_t* s) {
    float scale = ldexpf(1.0f, -key_bits);
    s[0] = 0;
    for (int b = 1; b < B; ++b) {
        uint64_t lo = 0, hi = key_bits >= 64 ? ~0ULL : ((1ULL << key_bits) - 1ULL);
        while (lo < hi) {
            uint64_t mid = lo + ((hi - lo) >> 1);
            if (bucket_model(X, Y, B, norm_key(mid, key_width, scale)) >= (uint32_t)b) hi = mid;
            else lo = mid + 1;
        }
        s[b] = lo;
    }
}

/* The model's knots from theta (double): V_j = sum_{i<j} sp(theta_i) / sum_i sp(theta_i),
 * sp = softplus; theta[0..255] -> X, theta[256..511] -> Y. */
static double softplus_d(double t) { return t > 30.0 ? t : log1p(exp(t)); }

void oracle_cdf_knots(const double* theta, double* X, double* Y) {
    for (int which = 0; which < 2; ++which) {
        double* V = which == 0 ? X : Y;
        double S = 0.0;
        for (int i = 0; i < PWL_SEG; ++i) S += softplus_d(theta[which * PWL_SEG + i]);
        double run = 0.0;
        V[0] = 0.0;
        for (int j = 1; j < PWL_SEG; ++j) {
            run += softplus_d(theta[which * PWL_SEG + j - 1]);
            V[j] = run / S;
        }
        V[PWL_SEG] = 1.0;
    }
}

/* Loss L = (1/m) sum_i (F(u_i) - (i + 1/2)/m)^2 over sorted sample values u,
 * and its gradient with respect to theta (grad may be NULL), in double. The
 * gradient is the chain rule written out: dF/dY_j, dF/dX_j from the segment
 * formula, then dV_j/dtheta_i = sp'(theta_i) (1[i < j] - V_j) / S. */
double oracle_cdf_loss_grad(const double* u, uint32_t m, const double* theta, double* grad) {
    double X[PWL_KNOTS], Y[PWL_KNOTS], gX[PWL_KNOTS], gY[PWL_KNOTS];
    oracle_cdf_knots(theta, X, Y);
    for (int j = 0; j < PWL_KNOTS; ++j) gX[j] = gY[j] = 0.0;
    double loss = 0.0;
    for (uint32_t i = 0; i < m; ++i) {
        double x = u[i];
        int j = PWL_SEG - 1;
        if (x < X[PWL_SEG]) {
            j = 0;
            while (j + 1 < PWL_SEG && X[j + 1] <= x) ++j;
        }
        double dx = X[j + 1] - X[j], dy = Y[j + 1] - Y[j];
        double w = dx > 0 ? (x - X[j]) / dx : 0.0;
        if (w < 0) w = 0;
        if (w > 1) w = 1;
        double f = Y[j] + dy * w;
        double e = f - ((double)i + 0.5) / m;
        loss += e * e / m;
        double ge = 2.0 * e / m;
        gY[j] += ge * (1.0 - w);
        gY[j + 1] += ge * w;
        if (dx > 0 && x < X[j + 1]) {
            double k = ge * dy / (dx * dx);
            gX[j] += k * (x - X[j + 1]);
            gX[j + 1] += -k * (x - X[j]);
        }
    }
    if (grad) {
        for (int which = 0; which < 2; ++which) {
            const double* V = which == 0 ? X : Y;
            const double* g = which == 0 ? gX : gY;
            double S = 0.0, A = 0.0;
            for (int i = 0; i < PWL_SEG; ++i) S += softplus_d(theta[which * PWL_SEG + i]);
            for (int j = 0; j < PWL_KNOTS; ++j) A += g[j] * V[j];
            for (int i = 0; i < PWL_SEG; ++i) {
                double suffix = 0.0;
                for (int j = i + 1; j < PWL_KNOTS; ++j) suffix += g[j];
                double t = theta[which * PWL_SEG + i];
                double sig = 1.0 / (1.0 + exp(-t));
                grad[which * PWL_SEG + i] = sig / S * (suffix - A);
            }
        }
    }
    return loss;
}

/* ---- The alternative model: a 1-32-1 monotone MLP CDF, in double.
 * Parameters p[0..31] = a1 (W1_j = softplus(a1_j)), p[32..63] = b1,
 * p[64..95] = a2 (W2_j = softplus(a2_j)), p[96] = b2, sigmoid hidden units:
 *   z(u) = sum_j W2_j sigma(W1_j u + b1_j) + b2,
 *   F(u) = (z(u) - z(0)) / (z(1) - z(0)).
 * Positive weights and an increasing sigma make F increasing, with F(0) = 0 and
 * F(1) = 1 (b2 cancels). Loss as for the PWL model. */
#define MLP_H 32
#define MLP_P (3 * MLP_H + 1)

static double sigmoid_d(double x) { return 1.0 / (1.0 + exp(-x)); }

static double mlp_z(const double* p, double u) {
    double z = p[3 * MLP_H];
    for (int j = 0; j < MLP_H; ++j) z += softplus_d(p[2 * MLP_H + j]) * sigmoid_d(softplus_d(p[j]) * u + p[MLP_H + j]);
    return z;
}

double oracle_mlp_cdf(const double* p, double u) {
    double z0 = mlp_z(p, 0.0), z1 = mlp_z(p, 1.0);
    return (mlp_z(p, u) - z0) / (z1 - z0);
}

/* d z(u) / d(W1_j, b1_j, W2_j) for every j */
static void mlp_dz(const double* p, double u, double* dW1, double* db1, double* dW2) {
    for (int j = 0; j < MLP_H; ++j) {
        double w1 = softplus_d(p[j]), w2 = softplus_d(p[2 * MLP_H + j]);
        double h = sigmoid_d(w1 * u + p[MLP_H + j]);
        double s = w2 * h * (1.0 - h);
        dW1[j] = s * u;
        db1[j] = s;
        dW2[j] = h;
    }
}

/* Loss (1/m) sum_i (F(u_i) - (i + 1/2)/m)^2 and its gradient with respect to
 * p (grad may be NULL), by the chain rule through the normalisation:
 * dF/dz(u) = 1/D, dF/dz(0) = (F - 1)/D, dF/dz(1) = -F/D, D = z(1) - z(0);
 * then through softplus for a1 and a2. */
double oracle_mlp_loss_grad(const double* u, uint32_t m, const double* p, double* grad) {
    double z0 = mlp_z(p, 0.0), z1 = mlp_z(p, 1.0), D = z1 - z0;
    double gW1[MLP_H] = {0}, gb1[MLP_H] = {0}, gW2[MLP_H] = {0};
    double dW1[MLP_H], db1[MLP_H], dW2[MLP_H];
    double c0 = 0.0, c1 = 0.0, loss = 0.0;
    for (uint32_t i = 0; i < m; ++i) {
        double F = (mlp_z(p, u[i]) - z0) / D;
        double e = F - ((double)i + 0.5) / m;
        loss += e * e / m;
        if (!grad) continue;
        double g = 2.0 * e / m;
        mlp_dz(p, u[i], dW1, db1, dW2);
        for (int j = 0; j < MLP_H; ++j) {
            gW1[j] += g / D * dW1[j];
            gb1[j] += g / D * db1[j];
            gW2[j] += g / D * dW2[j];
        }
        c0 += g * (F - 1.0) / D;
        c1 += -g * F / D;
    }
    if (grad) {
        mlp_dz(p, 0.0, dW1, db1, dW2);
        for (int j = 0; j < MLP_H; ++j) {
            gW1[j] += c0 * dW1[j];
            gb1[j] += c0 * db1[j];
            gW2[j] += c0 * dW2[j];
        }
        mlp_dz(p, 1.0, dW1, db1, dW2);
        for (int j = 0; j < MLP_H; ++j) {
            gW1[j] += c1 * dW1[j];
            gb1[j] += c1 * db1[j];
            gW2[j] += c1 * dW2[j];
        }
        for (int j = 0; j < MLP_H; ++j) {
            grad[j] = gW1[j] / (1.0 + exp(-p[j]));
            grad[MLP_H + j] = gb1[j];
            grad[2 * MLP_H + j] = gW2[j] / (1.0 + exp(-p[2 * MLP_H + j]));
        }
        grad[3 * MLP_H] = 0.0; /* b2 cancels in F */
    }
    return loss;
}

/* ---- Typed keys: signed integers and IEEE 754 floats, sorted stably by the
 * order of their type (the paper sorts unsigned integers from a known range;
 * signed and floating-point keys are the usual extension). The order is
 * written out as a comparison on the key's bits:
 *   signed integers (two's complement): by value;
 *   floats (binary32, binary64): IEEE 754 totalOrder: keys with the sign bit
 *   set come first, ordered by decreasing magnitude bits (all bits but the
 *   sign); then keys with the sign bit clear, by increasing magnitude bits.
 *   So -NaN < -Inf < ... < -0 < +0 < ... < +Inf < +NaN, NaNs by payload.
 * The sort is a top-down stable merge sort driven by that comparison.
 * type: 1 = i32, 2 = f32, 4 = i64, 5 = f64 (keys given as raw bits). */
static int typed_less(uint64_t a, uint64_t b, int type) {
    int width = (type == 1 || type == 2) ? 32 : 64;
    uint64_t sign = (uint64_t)1 << (width - 1);
    uint64_t mag = sign - 1;
    int sa = (a & sign) != 0, sb = (b & sign) != 0;
    if (type == 1 || type == 4) {
        if (sa != sb) return sa; /* the negative one is smaller */
        return (a & (sign | mag)) < (b & (sign | mag)); /* same sign: two's complement order is bit order */
    }
    if (sa != sb) return sa;
    if (sa) return (a & mag) > (b & mag);
    return (a & mag) < (b & mag);
}

static void typed_merge_sort(uint64_t* k, uint32_t* v, size_t n, uint64_t* tk, uint32_t* tv, int type) {
    if (n < 2) return;
    size_t h = n / 2;
    typed_merge_sort(k, v, h, tk, tv, type);
    typed_merge_sort(k + h, v ? v + h : NULL, n - h, tk, tv, type);
    size_t i = 0, j = h, o = 0;
    while (i < h || j < n) {
        /* take from the right only when strictly smaller: equal keys keep input order */
        int right = j < n && (i >= h || typed_less(k[j], k[i], type));
        size_t s = right ? j++ : i++;
        tk[o] = k[s];
        if (v) tv[o] = v[s];
        ++o;
    }
    memcpy(k, tk, n * sizeof(uint64_t));
    if (v) memcpy(v, tv, n * sizeof(uint32_t));
}

int oracle_sort_typed(void* keys, int type, uint32_t* vals, size_t n) {
    if (type != 1 && type != 2 && type != 4 && type != 5) return -1;
    int w32 = type == 1 || type == 2;
    uint64_t* k = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* tk = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint32_t* tv = vals ? (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t)) : NULL;
    if (!k || !tk || (vals && !tv)) {
        free(k);
        free(tk);
        free(tv);
        return -2;
    }
    for (size_t i = 0; i < n; ++i) k[i] = w32 ? (uint64_t)((uint32_t*)keys)[i] : ((uint64_t*)keys)[i];
    typed_merge_sort(k, vals, n, tk, tv, type);
    for (size_t i = 0; i < n; ++i) {
        if (w32) ((uint32_t*)keys)[i] = (uint32_t)k[i];
        else ((uint64_t*)keys)[i] = k[i];
    }
    free(k);
    free(tk);
    free(tv);
    return 0;
}
