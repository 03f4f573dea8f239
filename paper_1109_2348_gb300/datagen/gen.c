/*
 * Seeded synthetic block sources for the BWT block sort.
 *
 * This module draws random bytes only. It holds none of the transform's
 * arithmetic, and both the CUDA path and the CPU oracle consume its output.
 * The paper runs no experiments and ships no datasets, so every workload is a
 * synthetic stand-in with the shape of a bzip2 input block (900,000 bytes, the
 * "-9" block size) and with the statistics named for each source below.
 *
 * Random numbers: xoshiro256** (Blackman and Vigna, "Scrambled linear
 * pseudorandom number generators", 2018), its 256-bit state filled from
 * SplitMix64 (Steele, Lea and Flood, 2014), both written here from their
 * published definitions.
 *
 * Build: plain C99 + pthreads, no architecture-specific code, so the output is
 * the same on x86-64 and aarch64 hosts given the same libm pow()/log().
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- PRNG --- */

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* uniform integer in [0, m), m >= 1 (multiply-high mapping; bias < 2^-40) */
static uint32_t rng_below(rng_t *r, uint32_t m) {
    return (uint32_t)(((unsigned __int128)rng_next(r) * m) >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* ------------------------------------------------------ Zipf + Markov --- */

/* Cumulative table of P(rank r) proportional to r^-s, r = 1..A, scaled to
 * 2^53 so a 53-bit uniform draw selects a rank by binary search. */
typedef struct {
    int A;
    uint64_t cdf[256];
} zipf_t;

static void zipf_init(zipf_t *z, int A, double s) {
    double w[256], tot = 0.0;
    for (int r = 1; r <= A; ++r) { w[r - 1] = pow((double)r, -s); tot += w[r - 1]; }
    double acc = 0.0;
    z->A = A;
    for (int r = 0; r < A; ++r) {
        acc += w[r];
        double c = acc / tot * 9007199254740992.0; /* 2^53 */
        z->cdf[r] = (uint64_t)c;
    }
    z->cdf[A - 1] = 9007199254740992ull;
}

/* 0-based rank drawn from the Zipf table */
static int zipf_draw(const zipf_t *z, rng_t *r) {
    uint64_t u = rng_next(r) >> 11;
    int lo = 0, hi = z->A - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (u < z->cdf[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* An order-k Markov source over A symbols (bytes base..base+A-1). For each
 * context ctx (the previous k symbols as a base-A number) the next symbol is
 * sigma_ctx(r) with r Zipf-distributed; sigma_ctx is a Fisher-Yates shuffle of
 * 0..A-1 seeded from (model_seed, ctx). The model (the permutations) is fixed
 * per source; the block seed only drives the sampling, so blocks with
 * different seeds are independent draws from one distribution. */
typedef struct {
    int k, A, base;
    uint32_t nctx;
    uint8_t *perm; /* nctx * A */
    zipf_t z;
} markov_t;

static void markov_build(markov_t *m, int k, int A, int base, double s, uint64_t model_seed) {
    m->k = k; m->A = A; m->base = base;
    uint32_t nctx = 1;
    for (int i = 0; i < k; ++i) nctx *= (uint32_t)A;
    m->nctx = nctx;
    m->perm = (uint8_t *)malloc((size_t)nctx * (size_t)A);
    zipf_init(&m->z, A, s);
    for (uint32_t c = 0; c < nctx; ++c) {
        uint8_t *p = m->perm + (size_t)c * A;
        uint64_t x = model_seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(c + 1));
        rng_t r;
        rng_seed(&r, splitmix64(&x));
        for (int i = 0; i < A; ++i) p[i] = (uint8_t)i;
        for (int i = A - 1; i > 0; --i) {
            int j = (int)rng_below(&r, (uint32_t)(i + 1));
            uint8_t t = p[i]; p[i] = p[j]; p[j] = t;
        }
    }
}

static void markov_sample(const markov_t *m, rng_t *r, uint8_t *out, uint64_t n) {
    uint32_t ctx = 0, mod = m->nctx;
    for (uint64_t i = 0; i < n; ++i) {
        int sym;
        if (i < (uint64_t)m->k) {
            sym = (int)rng_below(r, (uint32_t)m->A);
        } else {
            sym = m->perm[(size_t)ctx * m->A + zipf_draw(&m->z, r)];
        }
        out[i] = (uint8_t)(m->base + sym);
        ctx = (uint32_t)(((uint64_t)ctx * m->A + (uint64_t)sym) % mod);
    }
}

static markov_t g_markov2, g_markov3;
static pthread_once_t g_once2 = PTHREAD_ONCE_INIT, g_once3 = PTHREAD_ONCE_INIT;
static void init_markov2(void) { markov_build(&g_markov2, 2, 64, 0x20, 1.1, 0x6D61726B6F763231ull); }
static void init_markov3(void) { markov_build(&g_markov3, 3, 96, 0x20, 1.2, 0x6D61726B6F763331ull); }

/* --------------------------------------------------------- sources ---- */

enum {
    SRC_UNIFORM = 0,      /* i.i.d. bytes 0..255 */
    SRC_MARKOV2_Z64 = 1,  /* order 2, 64 symbols 0x20..0x5F, Zipf(1.1) */
    SRC_MARKOV3_Z96 = 2,  /* order 3, 96 symbols 0x20..0x7F, Zipf(1.2) */
    SRC_RUNS16 = 3,       /* geometric runs, mean 50, 16 symbols 0x00..0x0F */
    SRC_CONST = 4,        /* every byte 0x61 */
    SRC_PERIOD7 = 5,      /* random primitive 7-byte unit, repeated, truncated */
    SRC_PERIOD1000 = 6,   /* random primitive 1000-byte unit, repeated, truncated */
    SRC_FIBONACCI = 7,    /* Fibonacci word over {a,b}: f1=b, f2=a, fk=f(k-1)f(k-2) */
    SRC_MUTATED_UNIT = 8, /* random 4096-byte unit repeated, 5% single-byte mutations */
    SRC_COUNT = 9
};

/* smallest period p of u (p divides len, u = rotation of itself by p) */
static int is_primitive(const uint8_t *u, int len) {
    for (int p = 1; p < len; ++p) {
        if (len % p) continue;
        int same = 1;
        for (int i = 0; i < len && same; ++i) same = (u[i] == u[(i + p) % len]);
        if (same) return 0;
    }
    return 1;
}

static void periodic(rng_t *r, int unit, uint8_t *out, uint64_t n) {
    uint8_t *u = (uint8_t *)malloc((size_t)unit);
    do {
        for (int i = 0; i < unit; ++i) u[i] = (uint8_t)rng_below(r, 256);
    } while (!is_primitive(u, unit));
    for (uint64_t i = 0; i < n; ++i) out[i] = u[i % (uint64_t)unit];
    free(u);
}

int gen_block(int source, uint64_t seed, uint8_t *out, uint64_t n) {
    rng_t r;
    uint64_t x = seed;
    rng_seed(&r, splitmix64(&x));
    switch (source) {
    case SRC_UNIFORM:
        for (uint64_t i = 0; i < n; ++i) out[i] = (uint8_t)(rng_next(&r) >> 56);
        return 0;
    case SRC_MARKOV2_Z64:
        pthread_once(&g_once2, init_markov2);
        markov_sample(&g_markov2, &r, out, n);
        return 0;
    case SRC_MARKOV3_Z96:
        pthread_once(&g_once3, init_markov3);
        markov_sample(&g_markov3, &r, out, n);
        return 0;
    case SRC_RUNS16: {
        const double lq = log(1.0 - 1.0 / 50.0);
        int sym = (int)rng_below(&r, 16);
        uint64_t i = 0;
        while (i < n) {
            double u = 1.0 - rng_unit(&r); /* (0, 1] */
            uint64_t len = 1 + (uint64_t)floor(log(u) / lq);
            for (uint64_t j = 0; j < len && i < n; ++j) out[i++] = (uint8_t)sym;
            sym = (sym + 1 + (int)rng_below(&r, 15)) & 15;
        }
        return 0;
    }
    case SRC_CONST:
        memset(out, 0x61, (size_t)n);
        return 0;
    case SRC_PERIOD7:
        periodic(&r, 7, out, n);
        return 0;
    case SRC_PERIOD1000:
        periodic(&r, 1000, out, n);
        return 0;
    case SRC_FIBONACCI: {
        /* f_k = f_{k-1} f_{k-2} with f_1 = "b", f_2 = "a": every f_k (k >= 2)
         * is a prefix of f_{k+1}, so the infinite word is grown in place. */
        if (n == 0) return 0;
        out[0] = 'a';            /* f_2 */
        if (n > 1) out[1] = 'b'; /* f_3 = f_2 f_1 = "ab" */
        uint64_t len_prev = 1, len = 2; /* |f_2|, |f_3| */
        while (len < n) {
            /* f_{k+1} = f_k f_{k-1}; f_{k-1} is the prefix of length len_prev */
            for (uint64_t j = 0; j < len_prev && len + j < n; ++j) out[len + j] = out[j];
            uint64_t nl = len + len_prev;
            len_prev = len;
            len = nl;
        }
        return 0;
    }
    case SRC_MUTATED_UNIT: {
        uint8_t u[4096];
        for (int i = 0; i < 4096; ++i) u[i] = (uint8_t)rng_below(&r, 256);
        for (uint64_t i = 0; i < n; ++i) {
            uint8_t c = u[i & 4095];
            if (rng_unit(&r) < 0.05) c = (uint8_t)((c + 1 + rng_below(&r, 255)) & 255);
            out[i] = c;
        }
        return 0;
    }
    default:
        return 1;
    }
}

/* ------------------------------------------------------- batches ------ */

typedef struct {
    int nb, next;
    const int *src;
    const uint64_t *seed, *off;
    uint8_t *out;
    int err;
    pthread_mutex_t mu;
} batch_job_t;

static void *batch_worker(void *arg) {
    batch_job_t *j = (batch_job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int b = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (b >= j->nb) break;
        if (gen_block(j->src[b], j->seed[b], j->out + j->off[b], j->off[b + 1] - j->off[b])) j->err = 1;
    }
    return NULL;
}

/* Fill out[off[b] .. off[b+1]) with gen_block(src[b], seed[b]) for every b,
 * using up to `threads` host threads. Returns 0 on success. */
int gen_batch(int nb, const int *src, const uint64_t *seed, const uint64_t *off, uint8_t *out,
              int threads) {
    batch_job_t j;
    j.nb = nb; j.next = 0; j.src = src; j.seed = seed; j.off = off; j.out = out; j.err = 0;
    pthread_mutex_init(&j.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (threads > nb) threads = nb > 0 ? nb : 1;
    pthread_t th[256];
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, batch_worker, &j);
    batch_worker(&j);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j.mu);
    return j.err;
}

/* count uniform integers in [lo, hi] (inclusive) from one seeded stream */
void gen_uniform_ints(uint64_t seed, int count, uint64_t lo, uint64_t hi, uint64_t *out) {
    rng_t r;
    uint64_t x = seed;
    rng_seed(&r, splitmix64(&x));
    uint64_t span = hi - lo + 1;
    for (int i = 0; i < count; ++i)
        out[i] = lo + (uint64_t)(((unsigned __int128)rng_next(&r) * span) >> 64);
}

/* count uniform doubles in [0, 1) from one seeded stream */
void gen_uniform_unit(uint64_t seed, int64_t count, double *out) {
    rng_t r;
    uint64_t x = seed;
    rng_seed(&r, splitmix64(&x));
    for (int64_t i = 0; i < count; ++i) out[i] = rng_unit(&r);
}

/* first 8 outputs of xoshiro256** seeded through SplitMix64: lets tests pin
 * the generator against the published reference sequence */
void gen_rng_probe(uint64_t seed, uint64_t *out8) {
    rng_t r;
    uint64_t x = seed;
    rng_seed(&r, splitmix64(&x));
    for (int i = 0; i < 8; ++i) out8[i] = rng_next(&r);
}

/* SplitMix64 outputs from a raw state (for pinning against its definition) */
void gen_splitmix_probe(uint64_t state, int count, uint64_t *out) {
    uint64_t x = state;
    for (int i = 0; i < count; ++i) out[i] = splitmix64(&x);
}

/* A uniformly random permutation of 0..n-1 (Fisher-Yates) from one seeded
 * stream: minibatch orders for training are drawn here, not in the trainer. */
void gen_permutation(uint64_t seed, uint32_t n, uint32_t *out) {
    rng_t r;
    uint64_t x = seed;
    rng_seed(&r, splitmix64(&x));
    for (uint32_t i = 0; i < n; ++i) out[i] = i;
    for (uint32_t i = n; i > 1; --i) {
        uint32_t j = rng_below(&r, i);
        uint32_t t = out[i - 1]; out[i - 1] = out[j]; out[j] = t;
    }
}
