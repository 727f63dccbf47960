/*
 * Seeded synthetic key generators for the integer-sort workloads.
 *
 * This module holds no sorting arithmetic: it only turns (seed, stream, index)
 * into input keys, payloads and segment lengths. Both the oracle side and the
 * CUDA side consume its output, so it must stay free of anything either side
 * computes.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used counter-based: the i-th 64-bit draw of
 * stream s under seed S is
 *     R(S, s, i) = mix(x0 + (i + 1) * GAMMA),   x0 = mix((S << 32) + s + GAMMA)
 * where mix() is SplitMix64's output finaliser and GAMMA its golden-ratio
 * increment. Being counter-based, any index range can be produced by any
 * thread, so the output is identical for every thread count.
 *
 * Distributions (the paper draws "random uniformly drawn integers" for every
 * algorithm, Section 4; the skewed and 64-bit families are synthetic stand-ins
 * for the learned-bucket and wide-key workloads):
 *   uniform  [0, 2^b)      : the top b bits of one draw.
 *   log-uniform lengths    : L = round(exp(U(ln lo, ln hi))).
 *   Zipf(s) truncated      : ranks 1..N by rejection-inversion (Hoermann &
 *                            Derflinger 1996), key = bijective 32-bit mix of rank.
 *   lognormal(mu, sigma)   : floor(exp(mu + sigma Z)), draws >= 2^32 redrawn.
 *   Gaussian mixture       : equal weights, means uniform on [0,2^32),
 *                            floor(clamp(mean + sigma Z, 0, 2^32-1)).
 * Rejection sampling uses a fixed window of WINDOW draws per key so that key i
 * never depends on how many draws key i-1 consumed.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GAMMA 0x9E3779B97F4A7C15ULL
#define WINDOW 64u /* draws reserved per key for rejection loops */

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_origin(uint64_t seed, uint64_t stream) {
    return mix64((seed << 32) + stream + GAMMA);
}

static inline uint64_t draw(uint64_t x0, uint64_t i) { return mix64(x0 + (i + 1) * GAMMA); }

/* U in [0,1) with 53 random bits. */
static inline double unit53(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* Bijective 32-bit mixer (xorshift-multiply; constants from C. Wellons'
 * public "hash prospector" search, "lowbias32"). Each step is invertible:
 * xorshift by a non-zero amount and multiplication by an odd constant. */
static inline uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

uint32_t isort_gen_mix32(uint32_t x) { return mix32(x); }
/* The i-th output of plain SplitMix64 started from state x (for test vectors). */
uint64_t isort_gen_splitmix_raw(uint64_t x, uint64_t i) { return draw(x, i); }
uint64_t isort_gen_draw(uint64_t seed, uint64_t stream, uint64_t i) {
    return draw(stream_origin(seed, stream), i);
}

/* ---------------------------------------------------------------- threading */

typedef void (*range_fn)(void* ctx, size_t lo, size_t hi);
typedef struct { range_fn fn; void* ctx; size_t lo, hi; } range_job;

static void* run_job(void* p) {
    range_job* j = (range_job*)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static int g_threads = 0;
void isort_gen_set_threads(int t) { g_threads = t; }

static void parallel_for(size_t n, range_fn fn, void* ctx) {
    int t = g_threads;
    if (t <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        t = (int)(c > 0 ? c : 1);
    }
    if (t > 64) t = 64;
    if (n < (size_t)1 << 16 || t == 1) { fn(ctx, 0, n); return; }
    pthread_t th[64];
    range_job jobs[64];
    size_t chunk = (n + (size_t)t - 1) / (size_t)t;
    int started = 0;
    for (int k = 0; k < t; ++k) {
        size_t lo = (size_t)k * chunk, hi = lo + chunk;
        if (lo >= n) break;
        if (hi > n) hi = n;
        jobs[k].fn = fn; jobs[k].ctx = ctx; jobs[k].lo = lo; jobs[k].hi = hi;
        if (pthread_create(&th[k], NULL, run_job, &jobs[k]) != 0) { run_job(&jobs[k]); th[k] = 0; }
        started = k + 1;
    }
    for (int k = 0; k < started; ++k)
        if (th[k]) pthread_join(th[k], NULL);
}

/* ---------------------------------------------------------------- uniform */

typedef struct { uint64_t x0; int bits; void* out; } uni_ctx;

static void uni32_body(void* c, size_t lo, size_t hi) {
    uni_ctx* u = (uni_ctx*)c;
    uint32_t* out = (uint32_t*)u->out;
    int sh = 64 - u->bits;
    for (size_t i = lo; i < hi; ++i) out[i] = (uint32_t)(draw(u->x0, i) >> sh);
}

static void uni64_body(void* c, size_t lo, size_t hi) {
    uni_ctx* u = (uni_ctx*)c;
    uint64_t* out = (uint64_t*)u->out;
    int sh = 64 - u->bits;
    for (size_t i = lo; i < hi; ++i) {
        uint64_t r = draw(u->x0, i);
        out[i] = sh == 0 ? r : (r >> sh);
    }
}

/* Keys uniform on [0, 2^bits), bits in 1..32. Returns 0 on success. */
int isort_gen_uniform_u32(uint64_t seed, uint64_t stream, size_t n, int bits, uint32_t* out) {
    if (bits < 1 || bits > 32 || (!out && n)) return -1;
    uni_ctx c = {stream_origin(seed, stream), bits, out};
    parallel_for(n, uni32_body, &c);
    return 0;
}

/* Keys uniform on [0, 2^bits), bits in 1..64. */
int isort_gen_uniform_u64(uint64_t seed, uint64_t stream, size_t n, int bits, uint64_t* out) {
    if (bits < 1 || bits > 64 || (!out && n)) return -1;
    uni_ctx c = {stream_origin(seed, stream), bits, out};
    parallel_for(n, uni64_body, &c);
    return 0;
}

typedef struct { uint32_t* out; } iota_ctx;
static void iota_body(void* c, size_t lo, size_t hi) {
    uint32_t* out = ((iota_ctx*)c)->out;
    for (size_t i = lo; i < hi; ++i) out[i] = (uint32_t)i;
}
/* Payload = original index (the stability witness). */
void isort_gen_iota_u32(size_t n, uint32_t* out) {
    iota_ctx c = {out};
    parallel_for(n, iota_body, &c);
}

/* ---------------------------------------------------------------- lengths */

/* Segment lengths log-uniform on [lo, hi]: L = round(exp(U(ln lo, ln hi))). */
int isort_gen_loguniform_lengths(uint64_t seed, uint64_t stream, size_t nseg, double lo, double hi,
                                 uint64_t* out) {
    if (!(lo >= 1.0) || !(hi >= lo)) return -1;
    uint64_t x0 = stream_origin(seed, stream);
    double a = log(lo), b = log(hi);
    for (size_t i = 0; i < nseg; ++i) {
        double u = unit53(draw(x0, i));
        double L = floor(exp(a + (b - a) * u) + 0.5);
        if (L < lo) L = lo;
        if (L > hi) L = hi;
        out[i] = (uint64_t)L;
    }
    return 0;
}

/* ---------------------------------------------------------------- Zipf */

/* Rejection-inversion for P(k) proportional to k^-s on k = 1..N.
 * Hat: the continuous density h(x) = x^-s. Because h is convex, the area of h
 * over [k-1/2, k+1/2] is at least h(k); each integer k owns that interval of the
 * integrated hat H, and a uniform point u in it is accepted iff it falls in the
 * top h(k) of the interval: u >= H(k+1/2) - h(k). For k = 1 the interval is
 * started at H(3/2) - h(1), so that its whole area equals h(1) and k = 1 is
 * always accepted. H and its inverse are written with expm1/log1p for
 * accuracy near s = 1. */
typedef struct {
    double s, one_minus_s, H_lo, H_hi;
    double N;
    uint64_t x0;
    uint32_t* out;
    int bad;
} zipf_ctx;

static inline double zipf_H(const zipf_ctx* z, double x) {
    double lx = log(x);
    return expm1(z->one_minus_s * lx) / z->one_minus_s;
}
static inline double zipf_Hinv(const zipf_ctx* z, double u) {
    double t = u * z->one_minus_s;
    if (t < -1.0) t = -1.0;
    return exp(log1p(t) / z->one_minus_s);
}
static inline double zipf_h(const zipf_ctx* z, double k) { return exp(-z->s * log(k)); }

static void zipf_body(void* c, size_t lo, size_t hi) {
    zipf_ctx* z = (zipf_ctx*)c;
    for (size_t i = lo; i < hi; ++i) {
        uint64_t rank = 0;
        for (uint32_t a = 0; a < WINDOW; ++a) {
            double u01 = unit53(draw(z->x0, (uint64_t)i * WINDOW + a));
            double u = z->H_hi + u01 * (z->H_lo - z->H_hi); /* in (H_lo, H_hi] */
            double x = zipf_Hinv(z, u);
            double k = floor(x + 0.5);
            if (k < 1.0) k = 1.0;
            if (k > z->N) k = z->N;
            if (k == 1.0 || u >= zipf_H(z, k + 0.5) - zipf_h(z, k)) { rank = (uint64_t)k; break; }
        }
        if (rank == 0) { z->bad = 1; rank = 1; }
        z->out[i] = mix32((uint32_t)rank);
    }
}

/* Zipf(s) ranks truncated to 1..2^32-1, hashed by the bijective mix32. */
int isort_gen_zipf_u32(uint64_t seed, uint64_t stream, size_t n, double s, uint32_t* out) {
    if (!(s > 0.0) || s == 1.0) return -1;
    zipf_ctx z;
    z.s = s;
    z.one_minus_s = 1.0 - s;
    z.N = 4294967295.0;
    z.x0 = stream_origin(seed, stream);
    z.out = out;
    z.bad = 0;
    z.H_lo = zipf_H(&z, 1.5) - 1.0; /* h(1) = 1 */
    z.H_hi = zipf_H(&z, z.N + 0.5);
    parallel_for(n, zipf_body, &z);
    return z.bad ? -2 : 0;
}

/* ---------------------------------------------------------------- normal */

/* One standard normal from two draws (Box-Muller, cosine branch). */
static inline double normal_from(uint64_t r1, uint64_t r2) {
    double u1 = 1.0 - unit53(r1); /* (0, 1] */
    double u2 = unit53(r2);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

typedef struct { double mu, sigma; uint64_t x0; uint32_t* out; int bad; } logn_ctx;

static void logn_body(void* c, size_t lo, size_t hi) {
    logn_ctx* L = (logn_ctx*)c;
    for (size_t i = lo; i < hi; ++i) {
        double v = -1.0;
        for (uint32_t a = 0; a + 1 < WINDOW; a += 2) {
            uint64_t base = (uint64_t)i * WINDOW + a;
            double z = normal_from(draw(L->x0, base), draw(L->x0, base + 1));
            double x = exp(L->mu + L->sigma * z);
            if (x < 4294967296.0) { v = x; break; }
        }
        if (v < 0) { L->bad = 1; v = 0; }
        L->out[i] = (uint32_t)floor(v);
    }
}

/* lognormal(mu, sigma) truncated to uint32: draws >= 2^32 are redrawn. */
int isort_gen_lognormal_u32(uint64_t seed, uint64_t stream, size_t n, double mu, double sigma, uint32_t* out) {
    if (!(sigma > 0)) return -1;
    logn_ctx L = {mu, sigma, stream_origin(seed, stream), out, 0};
    parallel_for(n, logn_body, &L);
    return L.bad ? -2 : 0;
}

typedef struct { const double* means; int ncomp; double sigma; uint64_t x0; uint32_t* out; } gmm_ctx;

static void gmm_body(void* c, size_t lo, size_t hi) {
    gmm_ctx* g = (gmm_ctx*)c;
    for (size_t i = lo; i < hi; ++i) {
        uint64_t base = (uint64_t)i * 3;
        int comp = (int)(unit53(draw(g->x0, base)) * g->ncomp);
        if (comp >= g->ncomp) comp = g->ncomp - 1;
        double x = g->means[comp] + g->sigma * normal_from(draw(g->x0, base + 1), draw(g->x0, base + 2));
        if (x < 0) x = 0;
        if (x > 4294967295.0) x = 4294967295.0;
        g->out[i] = (uint32_t)floor(x);
    }
}

/* Equal-weight Gaussian mixture; component means uniform on [0,2^32) drawn
 * from stream (stream + 1); values clipped to [0, 2^32-1]. */
int isort_gen_gmm_u32(uint64_t seed, uint64_t stream, size_t n, int ncomp, double sigma, uint32_t* out) {
    if (ncomp < 1 || ncomp > 4096 || !(sigma > 0)) return -1;
    double* means = (double*)malloc(sizeof(double) * (size_t)ncomp);
    if (!means) return -3;
    uint64_t xm = stream_origin(seed, stream + 1);
    for (int c = 0; c < ncomp; ++c) means[c] = unit53(draw(xm, (uint64_t)c)) * 4294967296.0;
    gmm_ctx g = {means, ncomp, sigma, stream_origin(seed, stream), out};
    parallel_for(n, gmm_body, &g);
    free(means);
    return 0;
}

/* ---------------------------------------------------------------- digest */

/* FNV-1a over bytes: a fingerprint for golden generator fixtures. */
uint64_t isort_gen_fnv1a(const void* data, size_t nbytes) {
    const unsigned char* p = (const unsigned char*)data;
    uint64_t h = 0xcbf29ce484222325ULL;
    for (size_t i = 0; i < nbytes; ++i) { h ^= p[i]; h *= 0x100000001b3ULL; }
    return h;
}
