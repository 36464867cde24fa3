/*
 * Seeded synthetic sparse-vector generator.
 *
 * This module only draws inputs: it holds none of the search method's
 * arithmetic (no inner products, pruning, windows or selection). Both the
 * CPU oracle and the GPU path consume the CSR arrays it writes.
 *
 * Randomness is counter-based: every row r of a matrix owns an independent
 * SplitMix64 stream whose state is derived from (seed, r), so rows can be
 * generated in any order or in parallel and always come out the same.
 * SplitMix64 follows its published definition (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014).
 *
 * Row layout: CSR with int64 indptr[n+1], int32 indices[nnz] (dims,
 * ascending within each row, unique), float values[nnz].
 *
 * Distributions (the paper's workloads are real SPLADE / BGE-M3 embeddings
 * that are not available; these stand in for them):
 *   nnz per row : Poisson(mu) | round(lognormal) clipped | uniform int
 *   dims        : truncated Zipf over ranks 1..d (p_r ~ r^-s), drawn without
 *                 replacement by rejecting repeats; dim = rank - 1
 *                 (or uniform over [0, d) when s == 0)
 *   values      : lognormal(0, sigma) as float, or uniform (0, 1]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GEN_NNZ_POISSON 0
#define GEN_NNZ_LOGNORMAL 1
#define GEN_NNZ_UNIFORM 2

#define GEN_VAL_LOGNORMAL 0
#define GEN_VAL_UNIFORM 1

typedef struct {
    int64_t n_rows;
    int32_t dim;
    int32_t nnz_kind;   /* GEN_NNZ_* */
    double nnz_a;       /* Poisson mean | lognormal target mean | uniform low  */
    double nnz_b;       /* unused       | lognormal sigma_ln    | uniform high */
    int32_t nnz_min;    /* clip low  (applied after the draw) */
    int32_t nnz_max;    /* clip high (applied after the draw; also <= dim) */
    double zipf_s;      /* 0 => uniform dims */
    int32_t val_kind;   /* GEN_VAL_* */
    double val_sigma;   /* lognormal sigma */
    uint64_t seed;
} gen_params;

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } sm64;

static inline uint64_t sm64_next(sm64* g) {
    g->s += 0x9E3779B97F4A7C15ULL;
    return sm64_mix(g->s);
}

/* uniform in [0, 1) with 53 random bits */
static inline double u01(sm64* g) { return (double)(sm64_next(g) >> 11) * 0x1.0p-53; }
/* uniform in (0, 1] */
static inline double u01_open0(sm64* g) { return 1.0 - u01(g); }

static inline sm64 row_stream(uint64_t seed, int64_t row, uint64_t salt) {
    sm64 g;
    g.s = sm64_mix(seed ^ sm64_mix((uint64_t)row * 0xD1B54A32D192ED03ULL + salt));
    return g;
}

static double std_normal(sm64* g) {
    /* Box-Muller, one output per pair of uniforms */
    double u1 = u01_open0(g), u2 = u01(g);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* Box-Muller, both outputs of one pair of uniforms */
static void std_normal2(sm64* g, double* z0, double* z1) {
    double u1 = u01_open0(g), u2 = u01(g);
    double r = sqrt(-2.0 * log(u1)), t = 6.283185307179586476925 * u2;
    *z0 = r * cos(t);
    *z1 = r * sin(t);
}

static int64_t poisson(sm64* g, double mu) {
    /* Knuth's multiplication method; fine for the small means used here */
    double L = exp(-mu), p = 1.0;
    int64_t k = 0;
    do { k++; p *= u01(g); } while (p > L);
    return k - 1;
}

static int64_t draw_nnz(const gen_params* P, sm64* g) {
    int64_t n;
    if (P->nnz_kind == GEN_NNZ_POISSON) {
        n = poisson(g, P->nnz_a);
    } else if (P->nnz_kind == GEN_NNZ_LOGNORMAL) {
        /* lognormal with E[n] = nnz_a: mu_ln = ln(mean) - sigma^2 / 2 */
        double s = P->nnz_b, mu = log(P->nnz_a) - 0.5 * s * s;
        n = (int64_t)llround(exp(mu + s * std_normal(g)));
    } else {
        int64_t lo = (int64_t)P->nnz_a, hi = (int64_t)P->nnz_b;
        n = lo + (int64_t)(u01(g) * (double)(hi - lo + 1));
        if (n > hi) n = hi;
    }
    if (n < P->nnz_min) n = P->nnz_min;
    if (n > P->nnz_max) n = P->nnz_max;
    if (n > P->dim) n = P->dim;
    if (n < 0) n = 0;
    return n;
}

/* cumulative Zipf table over ranks 1..d, normalised to cdf[d-1] = 1 */
static double* zipf_cdf(int32_t d, double s) {
    double* c = (double*)malloc(sizeof(double) * (size_t)d);
    if (!c) return NULL;
    double acc = 0.0;
    for (int32_t r = 0; r < d; r++) { acc += pow((double)(r + 1), -s); c[r] = acc; }
    for (int32_t r = 0; r < d; r++) c[r] /= acc;
    c[d - 1] = 1.0;
    return c;
}

/* Guide table for the inverse-CDF draw (Chen and Asau's cutpoint method):
   guide[b] = first rank r with cdf[r] > b / nb, so a draw starts its linear
   search near the answer. */
typedef struct { const double* cdf; int32_t* guide; int32_t d, nb; } zipf_table;

static int zipf_table_init(zipf_table* z, const double* cdf, int32_t d) {
    z->cdf = cdf; z->d = d; z->nb = d;
    z->guide = (int32_t*)malloc(sizeof(int32_t) * (size_t)(d + 1));
    if (!z->guide) return -1;
    int32_t r = 0;
    for (int32_t b = 0; b <= d; b++) {
        double t = (double)b / (double)d;
        while (r < d - 1 && cdf[r] <= t) r++;
        z->guide[b] = r;
    }
    return 0;
}

static int32_t zipf_draw(const zipf_table* z, sm64* g) {
    double u = u01(g);
    int32_t b = (int32_t)(u * (double)z->nb);
    if (b > z->nb) b = z->nb;
    int32_t r = z->guide[b];
    while (r < z->d - 1 && z->cdf[r] <= u) r++;   /* first r with cdf[r] > u */
    return r;
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Pass 1: nnz of every row (cheap, sequential stream per row, salt 1). */
int gen_row_nnz(const gen_params* P, int64_t* nnz_out) {
    if (!P || !nnz_out || P->n_rows < 0 || P->dim <= 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < P->n_rows; r++) {
        sm64 g = row_stream(P->seed, r, 1);
        nnz_out[r] = draw_nnz(P, &g);
    }
    return 0;
}

/* Pass 2: fill dims and values given indptr (from the prefix sum of pass 1). */
int gen_fill(const gen_params* P, const int64_t* indptr, int32_t* indices, float* values) {
    if (!P || !indptr || P->dim <= 0) return -1;
    double* cdf = NULL;
    zipf_table zt = {0};
    if (P->zipf_s > 0.0) {
        cdf = zipf_cdf(P->dim, P->zipf_s);
        if (!cdf || zipf_table_init(&zt, cdf, P->dim) != 0) { free(cdf); return -2; }
    }
    int err = 0;
#pragma omp parallel
    {
        int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)P->dim);
        if (!mark) {
#pragma omp atomic write
            err = -2;
        } else {
            /* mark[j] == (row & 0x3fffffff) + 1 means dim j is taken in this row;
               tags repeat only every 2^30 rows, far beyond any row count used */
            memset(mark, 0, sizeof(int32_t) * (size_t)P->dim);
#pragma omp for schedule(dynamic, 1024)
            for (int64_t r = 0; r < P->n_rows; r++) {
                int64_t b = indptr[r], n = indptr[r + 1] - indptr[r];
                int32_t tag = (int32_t)((r & 0x3fffffff) + 1);
                sm64 g = row_stream(P->seed, r, 2);
                int64_t got = 0, tries = 0;
                while (got < n) {
                    int32_t j;
                    if (cdf) j = zipf_draw(&zt, &g);
                    else { j = (int32_t)(u01(&g) * (double)P->dim); if (j >= P->dim) j = P->dim - 1; }
                    tries++;
                    if (tries > 64 * (n + 16)) {
                        /* pathological rejection rate: take the lowest free dim */
                        j = 0;
                        while (mark[j] == tag) j++;
                    }
                    if (mark[j] == tag) continue;
                    mark[j] = tag;
                    indices[b + got] = j;
                    got++;
                }
                qsort(indices + b, (size_t)n, sizeof(int32_t), cmp_i32);
                sm64 gv = row_stream(P->seed, r, 3);
                double zpair[2];
                for (int64_t t = 0; t < n; t++) {
                    double v;
                    if (P->val_kind == GEN_VAL_LOGNORMAL) {
                        if ((t & 1) == 0) std_normal2(&gv, &zpair[0], &zpair[1]);
                        v = exp(P->val_sigma * zpair[t & 1]);
                    } else {
                        v = u01_open0(&gv);
                    }
                    float f = (float)v;
                    if (f == 0.0f) f = 0x1.0p-126f;   /* keep every stored entry non-zero */
                    values[b + t] = f;
                }
            }
        }
        free(mark);
    }
    free(zt.guide);
    free(cdf);
    return err;
}
