/*
 * CPU ORACLE for the forward Burrows-Wheeler block sort -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline arm may
 * load this library. The product path (the CUDA library and its binding)
 * neither links nor calls it, and shares no code with it.
 *
 * What it computes (Section 3.1 of the paper: the forward transform sorts the
 * rotations of the block, citing Burrows and Wheeler 1994):
 *   for a block S[0..n-1], rotation i is S[i..n-1] S[0..i-1];
 *   SA = the permutation of 0..n-1 ordered by (rotation i compared as unsigned
 *        bytes, then i ascending) -- identical rotations keep index order;
 *   L[k] = S[(SA[k] + n - 1) mod n]   (the last column of the sorted matrix);
 *   primary = the row k with SA[k] = 0 (where the original block sits).
 *
 * Two routines reach that result:
 *   oracle_bwt_bruteforce -- the definition written out: a comparison sort of
 *     the n rotations with a full n-byte cyclic compare. Quadratic; tiny n only.
 *   oracle_bwt_block -- prefix doubling (Manber and Myers 1990), the textbook
 *     way to sort rotations, with the C library qsort as its sort step:
 *     rank_1[i] = S[i]; each round sorts the triples
 *     (rank_h[i], rank_h[(i+h) mod n], i) and renames equal pairs to one rank,
 *     giving rank_2h; it stops once all ranks differ or 2h >= n (then equal
 *     ranks mean identical rotations, already in index order by the third key).
 *
 * Also here: the inverse transform by the LF walk (Section 3.1 notes the
 * inverse can start from any row), and a double-precision reference of the
 * small MLP used by the learned bucketing (forward, MSE loss, backward, Adam).
 *
 * Parity pins (tests/test_oracle_pins.py): brute force over every {a,b}
 * string up to length 12 and random strings, hand-checked words, the inverse
 * round trip, permutation invariants, closed forms for constant blocks and
 * exact powers; the MLP by central finite differences.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------ brute force ---- */

static __thread const uint8_t *bf_S;
static __thread int64_t bf_n;

/* full cyclic comparison of rotations a and b, then index */
static int bf_cmp(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    for (int64_t j = 0; j < bf_n; ++j) {
        uint8_t ca = bf_S[(a + j) % bf_n], cb = bf_S[(b + j) % bf_n];
        if (ca != cb) return ca < cb ? -1 : 1;
    }
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Definition of the transform, written out. Returns 0, or 1 for n < 1. */
int oracle_bwt_bruteforce(const uint8_t *S, int64_t n, uint8_t *L, int32_t *primary, int32_t *SA) {
    if (n < 1) return 1;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    bf_S = S;
    bf_n = n;
    qsort(idx, (size_t)n, sizeof(int64_t), bf_cmp);
    for (int64_t k = 0; k < n; ++k) {
        L[k] = S[(idx[k] + n - 1) % n];
        if (idx[k] == 0) *primary = (int32_t)k;
        if (SA) SA[k] = (int32_t)idx[k];
    }
    free(idx);
    return 0;
}

/* ------------------------------------------------- prefix doubling ---- */

typedef struct { uint32_t r1, r2, i; } triple_t;

static int triple_cmp(const void *pa, const void *pb) {
    const triple_t *a = (const triple_t *)pa, *b = (const triple_t *)pb;
    if (a->r1 != b->r1) return a->r1 < b->r1 ? -1 : 1;
    if (a->r2 != b->r2) return a->r2 < b->r2 ? -1 : 1;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    return 0;
}

/* Sorted rotations of one block by prefix doubling. n < 2^32 - 1.
 * Writes L, *primary and (if non-NULL) SA. Returns 0, or 1 for n < 1. */
int oracle_bwt_block(const uint8_t *S, int64_t n, uint8_t *L, int32_t *primary, int32_t *SA) {
    if (n < 1) return 1;
    uint32_t *rank = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    triple_t *t = (triple_t *)malloc(sizeof(triple_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) rank[i] = S[i]; /* rank_1: the first byte */
    int64_t h = 1;                                   /* rank holds rank_h */
    for (;;) {
        for (int64_t i = 0; i < n; ++i) {
            t[i].r1 = rank[i];
            t[i].r2 = rank[(i + h) % n];
            t[i].i = (uint32_t)i;
        }
        qsort(t, (size_t)n, sizeof(triple_t), triple_cmp);
        /* rename: equal (r1, r2) pairs share the rank of the first row */
        int64_t distinct = 1;
        rank[t[0].i] = 0;
        for (int64_t k = 1; k < n; ++k) {
            int same = (t[k].r1 == t[k - 1].r1) && (t[k].r2 == t[k - 1].r2);
            if (!same) ++distinct;
            rank[t[k].i] = same ? rank[t[k - 1].i] : (uint32_t)k;
        }
        h *= 2; /* rank now holds rank_h for the doubled h */
        if (distinct == n || h >= n) break;
    }
    for (int64_t k = 0; k < n; ++k) {
        int64_t sa = t[k].i;
        L[k] = S[(sa + n - 1) % n];
        if (sa == 0) *primary = (int32_t)k;
        if (SA) SA[k] = (int32_t)sa;
    }
    free(t);
    free(rank);
    return 0;
}

/* ---------------------------------------------------------- batches --- */

typedef struct {
    const uint8_t *S;
    const uint64_t *off;
    int nb, next, err;
    uint8_t *L;
    int32_t *primary;
    pthread_mutex_t mu;
} oracle_job_t;

static void *oracle_worker(void *arg) {
    oracle_job_t *j = (oracle_job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int b = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (b >= j->nb) break;
        uint64_t o = j->off[b], n = j->off[b + 1] - o;
        if (oracle_bwt_block(j->S + o, (int64_t)n, j->L + o, j->primary + b, NULL)) j->err = 1;
    }
    return NULL;
}

/* Every block of a batch (block b = S[off[b] .. off[b+1])), parallel over
 * blocks with up to `threads` host threads. Returns 0, or 1 on an empty block. */
int oracle_bwt_batch(const uint8_t *S, const uint64_t *off, int nb, uint8_t *L, int32_t *primary,
                     int threads) {
    oracle_job_t j;
    j.S = S; j.off = off; j.nb = nb; j.next = 0; j.err = 0; j.L = L; j.primary = primary;
    pthread_mutex_init(&j.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (threads > nb) threads = nb > 0 ? nb : 1;
    pthread_t th[256];
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, oracle_worker, &j);
    oracle_worker(&j);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j.mu);
    return j.err;
}

/* ---------------------------------------------------------- inverse --- */

/* Inverse transform by the LF walk from the primary row: row r holds rotation
 * SA[r]; LF(r) = C[L[r]] + (occurrences of L[r] in L[0..r-1]) is the row of
 * rotation SA[r] - 1, so walking from the primary row emits S backwards.
 * Returns 0, or 1 on bad arguments. */
int oracle_inverse_bwt(const uint8_t *L, int64_t n, int32_t primary, uint8_t *out) {
    if (n < 1 || primary < 0 || primary >= n) return 1;
    int64_t C[257] = {0};
    uint32_t *lf = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    for (int64_t k = 0; k < n; ++k) C[L[k] + 1]++;
    for (int c = 0; c < 256; ++c) C[c + 1] += C[c];
    int64_t seen[256] = {0};
    for (int64_t k = 0; k < n; ++k) lf[k] = (uint32_t)(C[L[k]] + seen[L[k]]++);
    int64_t r = primary;
    for (int64_t i = n - 1; i >= 0; --i) {
        out[i] = L[r];
        r = lf[r];
    }
    free(lf);
    return 0;
}

/* ------------------------------------------------- MLP (double) ------- */
/*
 * The learned CDF model: x in R^8 (the 8 prefix bytes / 255) ->
 * h1 = relu(W1 x + b1) in R^32 -> h2 = relu(W2 h1 + b2) in R^32 ->
 * y = W3 h2 + b3 in R. Loss over a batch = mean over samples of (y - t)^2.
 * Parameter vector layout (1,377 values):
 *   W1[32][8] | b1[32] | W2[32][32] | b2[32] | W3[32] | b3[1]   (row-major).
 */
enum { MLP_IN = 8, MLP_H = 32, MLP_NPARAM = 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1 };

int oracle_mlp_nparams(void) { return MLP_NPARAM; }

static void mlp_sample(const double *p, const double *x, double *h1, double *h2, double *y) {
    const double *W1 = p, *b1 = W1 + 256, *W2 = b1 + 32, *b2 = W2 + 1024, *W3 = b2 + 32, *b3 = W3 + 32;
    for (int j = 0; j < MLP_H; ++j) {
        double a = b1[j];
        for (int i = 0; i < MLP_IN; ++i) a += W1[j * MLP_IN + i] * x[i];
        h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_H; ++j) {
        double a = b2[j];
        for (int i = 0; i < MLP_H; ++i) a += W2[j * MLP_H + i] * h1[i];
        h2[j] = a > 0.0 ? a : 0.0;
    }
    double o = b3[0];
    for (int i = 0; i < MLP_H; ++i) o += W3[i] * h2[i];
    *y = o;
}

/* y[s] = f(x[s]) for s < B; x is row-major [B][8]. */
void oracle_mlp_forward(const double *p, const double *x, int64_t B, double *y) {
    double h1[MLP_H], h2[MLP_H];
    for (int64_t s = 0; s < B; ++s) mlp_sample(p, x + s * MLP_IN, h1, h2, y + s);
}

/* Loss = mean_s (f(x_s) - t_s)^2 and its gradient with respect to every
 * parameter (chain rule through the two ReLU layers; the ReLU derivative at 0
 * is taken as 0). Returns the loss. */
double oracle_mlp_loss_grad(const double *p, const double *x, const double *t, int64_t B, double *g) {
    const double *W2 = p + 256 + 32, *W3 = W2 + 1024 + 32;
    double *gW1 = g, *gb1 = gW1 + 256, *gW2 = gb1 + 32, *gb2 = gW2 + 1024, *gW3 = gb2 + 32, *gb3 = gW3 + 32;
    memset(g, 0, sizeof(double) * MLP_NPARAM);
    double loss = 0.0;
    double h1[MLP_H], h2[MLP_H], d2[MLP_H], d1[MLP_H];
    for (int64_t s = 0; s < B; ++s) {
        const double *xs = x + s * MLP_IN;
        double y;
        mlp_sample(p, xs, h1, h2, &y);
        double e = y - t[s];
        loss += e * e;
        double dy = 2.0 * e / (double)B;
        gb3[0] += dy;
        for (int i = 0; i < MLP_H; ++i) {
            gW3[i] += dy * h2[i];
            d2[i] = h2[i] > 0.0 ? dy * W3[i] : 0.0;
        }
        for (int j = 0; j < MLP_H; ++j) {
            gb2[j] += d2[j];
            for (int i = 0; i < MLP_H; ++i) gW2[j * MLP_H + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double a = 0.0;
            for (int j = 0; j < MLP_H; ++j) a += W2[j * MLP_H + i] * d2[j];
            d1[i] = h1[i] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < MLP_H; ++j) {
            gb1[j] += d1[j];
            for (int i = 0; i < MLP_IN; ++i) gW1[j * MLP_IN + i] += d1[j] * xs[i];
        }
    }
    return loss / (double)B;
}

/* One Adam update (Kingma and Ba 2015, Algorithm 1) at step t >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void oracle_adam_step(double *p, const double *g, double *m, double *v, int64_t count, int t, double lr,
                      double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < count; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
