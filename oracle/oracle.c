/*
 * SINDI oracle: a plain, slow, single-threaded CPU reference in FP64.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls
 * it.
 *
 * What it computes, and where the paper defines it (arXiv 2509.08395):
 *   - sparse vector, non-zero entries only ............ Definition 1 (Sec. 2.1)
 *   - inner product over the common dims Omega ........ Definition 2
 *   - exact MIPS / top-k by brute force ............... Definition 3
 *   - mass and the alpha-mass subvector ............... Definitions "Mass of a
 *                                                       Vector" and "alpha-Mass
 *                                                       Subvector" (Sec. 4.1)
 *   - value-storing inverted lists I_{j,w} ............ Sec. 3.1, 3.3.1, Algorithm 1
 *   - pruned construction (keeps D for reordering) .... Algorithm 3
 *   - the other pruning methods the paper compares ...... Sec. 4.1 (List
 *     Pruning, Vector Number Pruning) and the ablation of Sec. 5 (List
 *     Pruning combined with Mass Ratio Pruning)
 *   - window-accumulation search with a min-heap ...... Algorithm 2
 *   - beta-mass query + gamma candidates + reorder .... Algorithm 4, Sec. 4.2
 *   - FP16 / FP8-E4M3 posting values (reduced-precision form; the paper has
 *     no quantisation, so these follow IEEE 754 binary16 and the OCP FP8 E4M3
 *     definition)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - ties are broken by lower document id: order = (score desc, id asc);
 *   - window slots whose global id is >= N are not candidates;
 *   - gamma == 0 means "no reordering": the coarse top-k is the answer;
 *   - alpha == 1 keeps every non-zero entry (the exact-arithmetic reading of
 *     the alpha-mass definition, so FP64 rounding cannot drop tail entries);
 *   - explicit zeros in the input are not entries (Definition 1) and are
 *     dropped; duplicate dims in a row and dims outside [0, d) are errors;
 *   - the terms of a query are visited in ascending dim order;
 *   - within a list I_{j,w}, postings are kept in ascending document id;
 *   - Vector Number Pruning keeps the first vn entries in the alpha-mass
 *     order pi (|x| desc, equal |x| by lower dim); List Pruning keeps the
 *     l' entries of largest |x| of each list I_j over all windows, equal |x|
 *     by lower document id; the combination applies alpha-mass first and
 *     List Pruning to the lists it leaves.
 *
 * Arithmetic: every input is FP32 and is widened exactly to FP64; all sums,
 * products and comparisons below are FP64, evaluated in the order written
 * (the build uses -ffp-contract=off so no FMA changes the rounding).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------ */
/* Dataset: the canonical form of D (Definition 1). Rows sorted by dim,      */
/* explicit zeros removed, values widened to FP64.                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;          /* ||D||                      */
    int32_t d;          /* dimension                   */
    int64_t* ptr;       /* [n + 1]                     */
    int32_t* dim;       /* [nnz] ascending in each row */
    double* val;        /* [nnz]                       */
} orc_dataset;

typedef struct { int32_t j; double v; } orc_entry;

static int cmp_entry_dim(const void* a, const void* b) {
    int32_t x = ((const orc_entry*)a)->j, y = ((const orc_entry*)b)->j;
    return (x > y) - (x < y);
}

void orc_dataset_free(orc_dataset* D) {
    if (!D) return;
    free(D->ptr); free(D->dim); free(D->val); free(D);
}

/* Canonicalise one CSR matrix. Returns NULL and sets *err on failure:
   -1 malformed indptr / dim out of range / duplicate dim / non-finite value. */
orc_dataset* orc_dataset_create(const int64_t* indptr, const int32_t* indices, const float* values,
                                int64_t n, int32_t d, int* err) {
    *err = ORC_OK;
    if (n < 0 || d <= 0 || !indptr || indptr[0] != 0) { *err = ORC_EINVAL; return NULL; }
    for (int64_t i = 0; i < n; i++)
        if (indptr[i + 1] < indptr[i]) { *err = ORC_EINVAL; return NULL; }
    int64_t nnz = indptr[n];
    orc_dataset* D = (orc_dataset*)calloc(1, sizeof(orc_dataset));
    if (!D) { *err = ORC_ENOMEM; return NULL; }
    D->n = n; D->d = d;
    D->ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    D->dim = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    D->val = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!D->ptr || !D->dim || !D->val) { orc_dataset_free(D); *err = ORC_ENOMEM; return NULL; }
    int64_t maxrow = 0;
    for (int64_t i = 0; i < n; i++)
        if (indptr[i + 1] - indptr[i] > maxrow) maxrow = indptr[i + 1] - indptr[i];
    orc_entry* row = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)(maxrow > 0 ? maxrow : 1));
    if (!row) { orc_dataset_free(D); *err = ORC_ENOMEM; return NULL; }
    int64_t out = 0;
    D->ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t m = 0;
        for (int64_t t = indptr[i]; t < indptr[i + 1]; t++) {
            float v = values[t];
            int32_t j = indices[t];
            if (j < 0 || j >= d || !isfinite(v)) { free(row); orc_dataset_free(D); *err = ORC_EINVAL; return NULL; }
            row[m].j = j; row[m].v = (double)v; m++;
        }
        qsort(row, (size_t)m, sizeof(orc_entry), cmp_entry_dim);
        for (int64_t t = 1; t < m; t++)
            if (row[t].j == row[t - 1].j) { free(row); orc_dataset_free(D); *err = ORC_EINVAL; return NULL; }
        for (int64_t t = 0; t < m; t++) {
            if (row[t].v == 0.0) continue;            /* Definition 1: x^j != 0 only */
            D->dim[out] = row[t].j; D->val[out] = row[t].v; out++;
        }
        D->ptr[i + 1] = out;
    }
    free(row);
    return D;
}

int64_t orc_dataset_nnz(const orc_dataset* D) { return D->ptr[D->n]; }

/* Copy out the canonical rows (for tests). */
void orc_dataset_export(const orc_dataset* D, int64_t* ptr, int32_t* dim, double* val) {
    memcpy(ptr, D->ptr, sizeof(int64_t) * (size_t)(D->n + 1));
    memcpy(dim, D->dim, sizeof(int32_t) * (size_t)D->ptr[D->n]);
    memcpy(val, D->val, sizeof(double) * (size_t)D->ptr[D->n]);
}

/* ------------------------------------------------------------------------ */
/* Definition 2: delta(x, q) = sum over j in Omega(x, q) of x^j * q^j.       */
/* Both rows are canonical (ascending dims); the sum runs over Omega in      */
/* ascending dim order.                                                      */
/* ------------------------------------------------------------------------ */
static double inner_product(const int32_t* xd, const double* xv, int64_t xn,
                            const int32_t* qd, const double* qv, int64_t qn) {
    double s = 0.0;
    int64_t a = 0, b = 0;
    while (a < xn && b < qn) {
        if (xd[a] < qd[b]) a++;
        else if (xd[a] > qd[b]) b++;
        else { s += xv[a] * qv[b]; a++; b++; }
    }
    return s;
}

double orc_inner_product(const orc_dataset* X, int64_t i, const orc_dataset* Q, int64_t r) {
    return inner_product(X->dim + X->ptr[i], X->val + X->ptr[i], X->ptr[i + 1] - X->ptr[i],
                         Q->dim + Q->ptr[r], Q->val + Q->ptr[r], Q->ptr[r + 1] - Q->ptr[r]);
}

/* ------------------------------------------------------------------------ */
/* Result order: a is better than b when it has the larger score, or the     */
/* same score and the lower id.                                              */
/* ------------------------------------------------------------------------ */
typedef struct { double s; int64_t id; } orc_hit;

static int better(orc_hit a, orc_hit b) { return a.s > b.s || (a.s == b.s && a.id < b.id); }

static int cmp_hit_best_first(const void* pa, const void* pb) {
    orc_hit a = *(const orc_hit*)pa, b = *(const orc_hit*)pb;
    if (better(a, b)) return -1;
    if (better(b, a)) return 1;
    return 0;
}

/* A bounded heap whose root is the worst kept hit (the "min-heap" H of
   Algorithm 2 and, with distance = -score, the max-heap R of Algorithm 4). */
typedef struct { orc_hit* h; int64_t len, cap; } orc_heap;

static void heap_sift_up(orc_heap* H, int64_t i) {
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (better(H->h[p], H->h[i])) {       /* parent better than child: swap (root = worst) */
            orc_hit t = H->h[p]; H->h[p] = H->h[i]; H->h[i] = t; i = p;
        } else break;
    }
}

static void heap_sift_down(orc_heap* H, int64_t i) {
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, w = i;
        if (l < H->len && better(H->h[w], H->h[l])) w = l;
        if (r < H->len && better(H->h[w], H->h[r])) w = r;
        if (w == i) break;
        orc_hit t = H->h[w]; H->h[w] = H->h[i]; H->h[i] = t; i = w;
    }
}

static void heap_insert(orc_heap* H, orc_hit x) { H->h[H->len++] = x; heap_sift_up(H, H->len - 1); }

static orc_hit heap_pop(orc_heap* H) {
    orc_hit top = H->h[0];
    H->h[0] = H->h[--H->len];
    if (H->len > 0) heap_sift_down(H, 0);
    return top;
}

/* Offer x to a heap that keeps the best `k` hits: insert when the heap has
   fewer than k hits or x beats the worst one; pop when it grows past k. */
static void heap_offer(orc_heap* H, int64_t k, orc_hit x) {
    if (k <= 0) return;
    if (H->len < k || better(x, H->h[0])) {
        heap_insert(H, x);
        if (H->len > k) (void)heap_pop(H);
    }
}

/* Drain a heap into best-first order. Returns the count. */
static int64_t heap_drain_sorted(orc_heap* H, int64_t* ids, double* scores) {
    int64_t n = H->len;
    qsort(H->h, (size_t)n, sizeof(orc_hit), cmp_hit_best_first);
    for (int64_t t = 0; t < n; t++) { ids[t] = H->h[t].id; scores[t] = H->h[t].s; }
    H->len = 0;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Definition 3 (and its top-k form): exact brute-force MIPS.                */
/* Scores every document by Definition 2 and keeps the best min(k, N).       */
/* Returns the number of results written.                                    */
/* ------------------------------------------------------------------------ */
int64_t orc_brute_force(const orc_dataset* D, const orc_dataset* Q, int64_t r, int64_t k,
                        int64_t* out_ids, double* out_scores) {
    orc_heap H;
    int64_t cap = (k < D->n ? k : D->n) + 1;
    H.h = (orc_hit*)malloc(sizeof(orc_hit) * (size_t)(cap > 0 ? cap : 1)); H.len = 0; H.cap = cap;
    if (!H.h) return ORC_ENOMEM;
    for (int64_t i = 0; i < D->n; i++) {
        orc_hit x = { orc_inner_product(D, i, Q, r), i };
        heap_offer(&H, k, x);
    }
    int64_t n = heap_drain_sorted(&H, out_ids, out_scores);
    free(H.h);
    return n;
}

/* Exact scores of every document for query r (Definition 2), for tests. */
void orc_all_scores(const orc_dataset* D, const orc_dataset* Q, int64_t r, double* out) {
    for (int64_t i = 0; i < D->n; i++) out[i] = orc_inner_product(D, i, Q, r);
}

/* ------------------------------------------------------------------------ */
/* Mass (Definition "Mass of a Vector") and the alpha-mass subvector          */
/* (Definition "alpha-Mass Subvector"):                                      */
/*   pi orders the entries by non-increasing |x| (ties: lower dim first);    */
/*   mass = sum of |x^j| (accumulated in pi order);                          */
/*   r = the smallest r >= 1 with sum_{t<=r} |x^{pi_t}| >= alpha * mass.     */
/* Writes the r kept positions (indices into the row, in pi order).          */
/* ------------------------------------------------------------------------ */
typedef struct { double a; int32_t j; int64_t pos; } orc_mag;

static int cmp_mag(const void* pa, const void* pb) {
    const orc_mag* a = (const orc_mag*)pa;
    const orc_mag* b = (const orc_mag*)pb;
    if (a->a > b->a) return -1;
    if (a->a < b->a) return 1;
    return (a->j > b->j) - (a->j < b->j);
}

static int64_t alpha_mass(const int32_t* dim, const double* val, int64_t n, double alpha,
                          int64_t* kept_pos, orc_mag* work) {
    if (n == 0) return 0;
    for (int64_t t = 0; t < n; t++) { work[t].a = fabs(val[t]); work[t].j = dim[t]; work[t].pos = t; }
    qsort(work, (size_t)n, sizeof(orc_mag), cmp_mag);
    int64_t r;
    if (alpha >= 1.0) {
        r = n;
    } else {
        double mass = 0.0;
        for (int64_t t = 0; t < n; t++) mass += work[t].a;
        double target = alpha * mass;
        double prefix = 0.0;
        r = n;
        for (int64_t t = 0; t < n; t++) {
            prefix += work[t].a;
            if (prefix >= target) { r = t + 1; break; }
        }
    }
    for (int64_t t = 0; t < r; t++) kept_pos[t] = work[t].pos;
    return r;
}

/* Vector Number Pruning (Sec. 4.1): the first min(vn, n) entries of the row
   in pi order. kept_pos receives their positions, in that order. */
static int64_t vector_number(const int32_t* dim, const double* val, int64_t n, int64_t vn, int64_t* kept_pos,
                             orc_mag* work) {
    if (n == 0) return 0;
    for (int64_t t = 0; t < n; t++) { work[t].a = fabs(val[t]); work[t].j = dim[t]; work[t].pos = t; }
    qsort(work, (size_t)n, sizeof(orc_mag), cmp_mag);
    int64_t r = n < vn ? n : vn;
    for (int64_t t = 0; t < r; t++) kept_pos[t] = work[t].pos;
    return r;
}

/* List Pruning order: |x| descending, then lower document id. */
typedef struct { double a; int64_t doc; int64_t pos; } orc_lmag;
static int cmp_lmag(const void* pa, const void* pb) {
    const orc_lmag* a = (const orc_lmag*)pa;
    const orc_lmag* b = (const orc_lmag*)pb;
    if (a->a > b->a) return -1;
    if (a->a < b->a) return 1;
    return (a->doc < b->doc) ? -1 : (a->doc > b->doc);
}

/* alpha-mass of one raw row (FP32 values), positions refer to the input row. */
int64_t orc_alpha_mass(const int32_t* dim, const float* val, int64_t n, double alpha, int64_t* kept_pos) {
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_mag* w = (orc_mag*)malloc(sizeof(orc_mag) * (size_t)(n > 0 ? n : 1));
    if (!v || !w) { free(v); free(w); return ORC_ENOMEM; }
    for (int64_t t = 0; t < n; t++) v[t] = (double)val[t];
    int64_t r = alpha_mass(dim, v, n, alpha, kept_pos, w);
    free(v); free(w);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision posting values.                                          */
/* binary16: IEEE 754 round-to-nearest-even from FP32.                        */
/* E4M3 (OCP FP8): 1 sign, 4 exponent (bias 7), 3 mantissa bits; no            */
/* infinities; largest finite 448; S.1111.111 is NaN. Encoding rounds to       */
/* nearest even and saturates to +-448.                                       */
/* Both encoders work on the exact FP64 value of the FP32 input.              */
/* ------------------------------------------------------------------------ */
static double f16_decode_d(uint16_t h) {
    int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(1024 + m), e - 25);
    return s ? -v : v;
}

float orc_f16_decode(uint16_t h) { return (float)f16_decode_d(h); }

/* nearest-even choice between the two neighbours lo < x < hi of a grid,
   given their codes (codes of neighbours differ by 1, the even code wins) */
static uint32_t pick_rne(double x, double lo, double hi, uint32_t code_lo) {
    double dl = x - lo, dh = hi - x;
    if (dl < dh) return code_lo;
    if (dh < dl) return code_lo + 1;
    return (code_lo & 1) ? code_lo + 1 : code_lo;
}

uint16_t orc_f16_encode(float f) {
    double x = (double)f;
    uint16_t sign = signbit(x) ? 0x8000 : 0;
    if (isnan(x)) return 0x7E00;
    double a = fabs(x);
    if (isinf(x)) return sign | 0x7C00;
    /* magnitudes are a monotone grid of codes 0..0x7BFF (65504), then inf */
    /* binary search the largest code whose value <= a */
    uint32_t lo = 0, hi = 0x7BFF;
    if (a >= f16_decode_d(0x7BFF)) {
        /* beyond the largest finite: RNE overflows to inf at >= 65520 */
        if (a >= 65520.0) return sign | 0x7C00;
        return sign | 0x7BFF;
    }
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) / 2;
        if (f16_decode_d((uint16_t)mid) <= a) lo = mid; else hi = mid - 1;
    }
    double vlo = f16_decode_d((uint16_t)lo);
    if (vlo == a) return (uint16_t)(sign | lo);
    double vhi = f16_decode_d((uint16_t)(lo + 1));
    return (uint16_t)(sign | pick_rne(a, vlo, vhi, lo));
}

static double e4m3_decode_d(uint8_t c) {
    int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
    double v;
    if (e == 15 && m == 7) return NAN;
    if (e == 0) v = ldexp((double)m, -9);            /* subnormal: m/8 * 2^-6 */
    else v = ldexp((double)(8 + m), e - 10);        /* (1 + m/8) * 2^(e-7)   */
    return s ? -v : v;
}

float orc_e4m3_decode(uint8_t c) { return (float)e4m3_decode_d(c); }

uint8_t orc_e4m3_encode(float f) {
    double x = (double)f;
    if (isnan(x)) return 0x7F;
    uint8_t sign = signbit(x) ? 0x80 : 0;
    double a = fabs(x);
    if (a >= 448.0) return (uint8_t)(sign | 0x7E);   /* saturate (also +-inf) */
    uint32_t lo = 0, hi = 0x7E;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) / 2;
        if (e4m3_decode_d((uint8_t)mid) <= a) lo = mid; else hi = mid - 1;
    }
    double vlo = e4m3_decode_d((uint8_t)lo);
    if (vlo == a) return (uint8_t)(sign | lo);
    double vhi = e4m3_decode_d((uint8_t)(lo + 1));
    return (uint8_t)(sign | pick_rne(a, vlo, vhi, lo));
}

/* ------------------------------------------------------------------------ */
/* The index: lists I_{j,w} (Sec. 3.3.1) built by Algorithm 1 over the        */
/* pruned dataset D' of Algorithm 3. Stored list by list: list (j, w) is      */
/* seg[j * sigma + w] .. seg[j * sigma + w + 1] in (pid, pval).               */
/* ------------------------------------------------------------------------ */
#define ORC_F32 0
#define ORC_F16 1
#define ORC_E4M3 2

typedef struct {
    const orc_dataset* D;   /* the unpruned dataset, kept for reordering (Alg. 3 returns it) */
    int64_t lambda, sigma;
    int32_t d;
    int32_t dtype;
    int64_t* seg;           /* [d * sigma + 1] */
    int64_t* pid;           /* global document id i */
    double* pval;           /* stored value (FP32 value, or its FP16 / E4M3 dequantised form) */
    float* scale;           /* [d] per-list E4M3 scale (1 otherwise) */
    int64_t* kept_count;    /* [n] r_i of every document */
} orc_index;

void orc_index_free(orc_index* I) {
    if (!I) return;
    free(I->seg); free(I->pid); free(I->pval); free(I->scale); free(I->kept_count); free(I);
}

#define ORC_PRUNE_MASS 0
#define ORC_PRUNE_VECTOR_NUMBER 1
#define ORC_PRUNE_LIST 2
#define ORC_PRUNE_MASS_LIST 3

/* Algorithm 3 (ApproximateSindiConstruction) with Algorithm 1 inside it.
   lambda in [1, ...]; alpha in (0, 1]; dtype ORC_F32 | ORC_F16 | ORC_E4M3.
   prune selects the document pruning (Sec. 4.1): MASS (alpha-mass, the
   method's own), VECTOR_NUMBER (n_keep entries per document), LIST (n_keep
   entries per list I_j) or MASS_LIST (alpha-mass, then LIST). alpha is
   used by MASS and MASS_LIST only; n_keep >= 1 by the other three. */
orc_index* orc_build_ex(const orc_dataset* D, int64_t lambda, double alpha, int32_t dtype, int32_t prune,
                        int64_t n_keep, int* err) {
    *err = ORC_OK;
    if (!D || lambda <= 0 || !(alpha > 0.0 && alpha <= 1.0) || dtype < 0 || dtype > 2) { *err = ORC_EINVAL; return NULL; }
    if (prune < ORC_PRUNE_MASS || prune > ORC_PRUNE_MASS_LIST || (prune != ORC_PRUNE_MASS && n_keep < 1)) {
        *err = ORC_EINVAL; return NULL;
    }
    const double doc_alpha = (prune == ORC_PRUNE_MASS || prune == ORC_PRUNE_MASS_LIST) ? alpha : 1.0;
    orc_index* I = (orc_index*)calloc(1, sizeof(orc_index));
    if (!I) { *err = ORC_ENOMEM; return NULL; }
    I->D = D; I->lambda = lambda; I->d = D->d; I->dtype = dtype;
    I->sigma = (D->n + lambda - 1) / lambda;                 /* sigma = ceil(||D|| / lambda) */
    int64_t n = D->n, d = D->d, sigma = I->sigma;

    /* Alg. 3, pruning step: D' <- { alpha-mass(x_i) }. Kept entries go back in
       ascending dim order (the subvector is a set; canonical order). */
    int64_t nnz = D->ptr[n];
    int64_t* kptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t* kdim = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    double* kval = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    I->kept_count = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t maxrow = 0;
    for (int64_t i = 0; i < n; i++) if (D->ptr[i + 1] - D->ptr[i] > maxrow) maxrow = D->ptr[i + 1] - D->ptr[i];
    orc_mag* work = (orc_mag*)malloc(sizeof(orc_mag) * (size_t)(maxrow > 0 ? maxrow : 1));
    int64_t* kpos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxrow > 0 ? maxrow : 1));
    char* keep = (char*)malloc((size_t)(maxrow > 0 ? maxrow : 1));
    if (!kptr || !kdim || !kval || !I->kept_count || !work || !kpos || !keep) {
        free(kptr); free(kdim); free(kval); free(work); free(kpos); free(keep); orc_index_free(I);
        *err = ORC_ENOMEM; return NULL;
    }
    kptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t b = D->ptr[i], m = D->ptr[i + 1] - b;
        int64_t r = prune == ORC_PRUNE_VECTOR_NUMBER ? vector_number(D->dim + b, D->val + b, m, n_keep, kpos, work)
                                                     : alpha_mass(D->dim + b, D->val + b, m, doc_alpha, kpos, work);
        I->kept_count[i] = r;
        memset(keep, 0, (size_t)(m > 0 ? m : 1));
        for (int64_t t = 0; t < r; t++) keep[kpos[t]] = 1;
        int64_t o = kptr[i];
        for (int64_t t = 0; t < m; t++)
            if (keep[t]) { kdim[o] = D->dim[b + t]; kval[o] = D->val[b + t]; o++; }
        kptr[i + 1] = o;
    }
    free(work); free(kpos); free(keep);

    /* Alg. 1: for every dim j, X = { x'_i : x'^j_i != 0 } (ascending i), and
       every x'^j_i is appended to I_{j, floor(i / lambda)}. X for all j is
       collected first (a transpose by counting), then the loop runs j-major. */
    int64_t P = kptr[n];
    int64_t* xptr = (int64_t*)calloc((size_t)(d + 1), sizeof(int64_t));
    int64_t* xdoc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P > 0 ? P : 1));
    double* xval = (double*)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1));
    I->seg = (int64_t*)calloc((size_t)(d * sigma + 1), sizeof(int64_t));
    I->pid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P > 0 ? P : 1));
    I->pval = (double*)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1));
    I->scale = (float*)malloc(sizeof(float) * (size_t)d);
    if (!xptr || !xdoc || !xval || !I->seg || !I->pid || !I->pval || !I->scale) {
        free(kptr); free(kdim); free(kval); free(xptr); free(xdoc); free(xval); orc_index_free(I);
        *err = ORC_ENOMEM; return NULL;
    }
    for (int64_t t = 0; t < P; t++) xptr[kdim[t] + 1]++;
    for (int64_t j = 0; j < d; j++) xptr[j + 1] += xptr[j];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)d);
        if (!fill) { free(kptr); free(kdim); free(kval); free(xptr); free(xdoc); free(xval); orc_index_free(I); *err = ORC_ENOMEM; return NULL; }
        memcpy(fill, xptr, sizeof(int64_t) * (size_t)d);
        for (int64_t i = 0; i < n; i++)
            for (int64_t t = kptr[i]; t < kptr[i + 1]; t++) {
                int64_t j = kdim[t];
                xdoc[fill[j]] = i; xval[fill[j]] = kval[t]; fill[j]++;
            }
        free(fill);
    }
    free(kptr); free(kdim); free(kval);

    /* List Pruning (Sec. 4.1): list I_j (all windows) keeps its n_keep
       entries of largest |x|, equal |x| by lower document id; the kept ones
       stay in ascending document order. */
    if (prune == ORC_PRUNE_LIST || prune == ORC_PRUNE_MASS_LIST) {
        int64_t maxlen = 0;
        for (int64_t j = 0; j < d; j++) if (xptr[j + 1] - xptr[j] > maxlen) maxlen = xptr[j + 1] - xptr[j];
        orc_lmag* lw = (orc_lmag*)malloc(sizeof(orc_lmag) * (size_t)(maxlen > 0 ? maxlen : 1));
        char* lkeep = (char*)malloc((size_t)(maxlen > 0 ? maxlen : 1));
        if (!lw || !lkeep) {
            free(lw); free(lkeep); free(xptr); free(xdoc); free(xval); orc_index_free(I);
            *err = ORC_ENOMEM; return NULL;
        }
        int64_t wpos = 0;
        for (int64_t j = 0; j < d; j++) {
            const int64_t b = xptr[j], e = xptr[j + 1], len = e - b;
            for (int64_t t = 0; t < len; t++) {
                lw[t].a = fabs(xval[b + t]); lw[t].doc = xdoc[b + t]; lw[t].pos = t; lkeep[t] = 0;
            }
            qsort(lw, (size_t)len, sizeof(orc_lmag), cmp_lmag);
            for (int64_t t = 0; t < len; t++) {
                if (t < n_keep) lkeep[lw[t].pos] = 1;
                else I->kept_count[lw[t].doc]--;
            }
            xptr[j] = wpos;
            for (int64_t t = 0; t < len; t++)
                if (lkeep[t]) { xdoc[wpos] = xdoc[b + t]; xval[wpos] = xval[b + t]; wpos++; }
        }
        xptr[d] = wpos;
        free(lw); free(lkeep);
    }

    /* lengths of every I_{j,w}, then appends in (j, ascending i) order */
    for (int64_t j = 0; j < d; j++)
        for (int64_t t = xptr[j]; t < xptr[j + 1]; t++) {
            int64_t w = xdoc[t] / lambda;
            I->seg[j * sigma + w + 1]++;
        }
    for (int64_t s = 0; s < d * sigma; s++) I->seg[s + 1] += I->seg[s];
    {
        int64_t o = 0;
        for (int64_t j = 0; j < d; j++)
            for (int64_t t = xptr[j]; t < xptr[j + 1]; t++) {
                /* appending in ascending i keeps each I_{j,w} contiguous */
                I->pid[o] = xdoc[t]; I->pval[o] = xval[t]; o++;
            }
    }

    /* Reduced-precision values: each stored value becomes its dequantised
       FP16 value, or q * scale_j with scale_j = (max |x| over list I_j) / 448
       computed in FP32 and q = E4M3(x / scale_j) with the division in FP32. */
    for (int64_t j = 0; j < d; j++) I->scale[j] = 1.0f;
    if (dtype == ORC_F16) {
        for (int64_t t = 0; t < P; t++) I->pval[t] = (double)orc_f16_decode(orc_f16_encode((float)I->pval[t]));
    } else if (dtype == ORC_E4M3) {
        for (int64_t j = 0; j < d; j++) {
            float amax = 0.0f;
            for (int64_t t = xptr[j]; t < xptr[j + 1]; t++) {
                float a = fabsf((float)xval[t]);
                if (a > amax) amax = a;
            }
            volatile float sc = amax / 448.0f;
            if (!(sc > 0.0f)) sc = 1.0f;
            I->scale[j] = sc;
            for (int64_t t = I->seg[j * sigma]; t < I->seg[(j + 1) * sigma]; t++) {
                volatile float ratio = (float)I->pval[t] / sc;
                uint8_t code = orc_e4m3_encode(ratio);
                volatile float deq = orc_e4m3_decode(code) * sc;
                I->pval[t] = (double)deq;
            }
        }
    }
    free(xptr); free(xdoc); free(xval);
    return I;
}

orc_index* orc_build(const orc_dataset* D, int64_t lambda, double alpha, int32_t dtype, int* err) {
    return orc_build_ex(D, lambda, alpha, dtype, ORC_PRUNE_MASS, 0, err);
}

int64_t orc_index_sigma(const orc_index* I) { return I->sigma; }
int64_t orc_index_postings(const orc_index* I) { return I->seg[(int64_t)I->d * I->sigma]; }

/* The largest |stored value| of every list I_j over all its windows (0 for
   an empty list): out[j] = max |pval[p]|, p in seg[j*sigma] .. seg[(j+1)*sigma].
   It bounds every product q^j * x^j_i that a window adds for term j. */
void orc_list_vmax(const orc_index* I, double* out) {
    for (int64_t j = 0; j < I->d; j++) {
        double m = 0.0;
        for (int64_t p = I->seg[j * I->sigma]; p < I->seg[(j + 1) * I->sigma]; p++)
            if (fabs(I->pval[p]) > m) m = fabs(I->pval[p]);
        out[j] = m;
    }
}

/* Export the lists (for comparing a device-built index): seg[d*sigma + 1],
   pid[P], pval[P] (FP64), scale[d], kept_count[n]. */
void orc_index_export(const orc_index* I, int64_t* seg, int64_t* pid, double* pval, float* scale, int64_t* kept) {
    int64_t S = (int64_t)I->d * I->sigma, P = I->seg[S];
    memcpy(seg, I->seg, sizeof(int64_t) * (size_t)(S + 1));
    memcpy(pid, I->pid, sizeof(int64_t) * (size_t)P);
    memcpy(pval, I->pval, sizeof(double) * (size_t)P);
    memcpy(scale, I->scale, sizeof(float) * (size_t)I->d);
    memcpy(kept, I->kept_count, sizeof(int64_t) * (size_t)I->D->n);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 (PreciseSindiSearch) for one query (given as its entries in    */
/* ascending dim order): per window w, A[i mod lambda] += q^j * x^j_i over     */
/* every posting of every I_{j,w}; then every slot m of the window (with      */
/* global id < N) is offered to the heap H of the best `k`; A[m] is reset.    */
/* Writes up to k hits best-first; returns the count.                        */
/* ------------------------------------------------------------------------ */
static int64_t precise_search(const orc_index* I, const int32_t* qd, const double* qv, int64_t qn,
                              int64_t k, int64_t* out_ids, double* out_scores) {
    int64_t lambda = I->lambda, sigma = I->sigma, N = I->D->n;
    double* A = (double*)malloc(sizeof(double) * (size_t)lambda);
    int64_t cap = (k < N ? k : N) + 1;
    orc_heap H;
    H.h = (orc_hit*)malloc(sizeof(orc_hit) * (size_t)(cap > 0 ? cap : 1)); H.len = 0; H.cap = cap;
    if (!A || !H.h) { free(A); free(H.h); return ORC_ENOMEM; }
    for (int64_t m = 0; m < lambda; m++) A[m] = 0.0;
    for (int64_t w = 0; w < sigma; w++) {
        for (int64_t t = 0; t < qn; t++) {
            int64_t j = qd[t];
            double q = qv[t];
            int64_t s0 = I->seg[j * sigma + w], s1 = I->seg[j * sigma + w + 1];
            for (int64_t p = s0; p < s1; p++) {
                double prod = q * I->pval[p];         /* the product P^j[t] */
                int64_t m = I->pid[p] % lambda;
                A[m] = A[m] + prod;
            }
        }
        for (int64_t m = 0; m < lambda; m++) {
            int64_t id = m + lambda * w;
            if (id < N) {
                orc_hit x = { A[m], id };
                heap_offer(&H, k, x);
            }
            A[m] = 0.0;
        }
    }
    int64_t n = heap_drain_sorted(&H, out_ids, out_scores);
    free(A); free(H.h);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 4 (ApproximateSindiSearch) for query row r of Q:                 */
/*   q' = beta-mass(q); H = Algorithm 2 (q', I, gamma);                        */
/*   every candidate i gets the exact delta(x_i, q) from the unpruned x_i and  */
/*   the unpruned q; R keeps the best k (ranking by delta descending is the   */
/*   same order as the paper's 1 - delta ascending).                          */
/* gamma == 0: no reordering; the answer is Algorithm 2 (q', I, k).          */
/* If coarse_ids != NULL, the gamma coarse candidates (best-first) and their  */
/* coarse scores are written there as well; *n_coarse gets their count.      */
/* Returns the number of results written.                                    */
/* ------------------------------------------------------------------------ */
int64_t orc_search(const orc_index* I, const orc_dataset* Q, int64_t r, double beta, int64_t gamma, int64_t k,
                   int64_t* out_ids, double* out_scores,
                   int64_t* coarse_ids, double* coarse_scores, int64_t* n_coarse) {
    const int32_t* qd = Q->dim + Q->ptr[r];
    const double* qv = Q->val + Q->ptr[r];
    int64_t qn = Q->ptr[r + 1] - Q->ptr[r];
    if (k < 0 || gamma < 0 || !(beta > 0.0 && beta <= 1.0)) return ORC_EINVAL;

    /* q' = beta-mass(q), kept entries back in ascending dim order */
    int64_t* kpos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(qn > 0 ? qn : 1));
    orc_mag* work = (orc_mag*)malloc(sizeof(orc_mag) * (size_t)(qn > 0 ? qn : 1));
    char* keep = (char*)calloc((size_t)(qn > 0 ? qn : 1), 1);
    int32_t* pd = (int32_t*)malloc(sizeof(int32_t) * (size_t)(qn > 0 ? qn : 1));
    double* pv = (double*)malloc(sizeof(double) * (size_t)(qn > 0 ? qn : 1));
    if (!kpos || !work || !keep || !pd || !pv) { free(kpos); free(work); free(keep); free(pd); free(pv); return ORC_ENOMEM; }
    int64_t rq = alpha_mass(qd, qv, qn, beta, kpos, work);
    for (int64_t t = 0; t < rq; t++) keep[kpos[t]] = 1;
    int64_t pn = 0;
    for (int64_t t = 0; t < qn; t++) if (keep[t]) { pd[pn] = qd[t]; pv[pn] = qv[t]; pn++; }
    free(kpos); free(work); free(keep);

    int64_t result;
    if (gamma == 0) {
        result = precise_search(I, pd, pv, pn, k, out_ids, out_scores);
        if (n_coarse) *n_coarse = 0;
    } else {
        int64_t N = I->D->n;
        int64_t gcap = gamma < N ? gamma : N;
        int64_t* hid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(gcap > 0 ? gcap : 1));
        double* hs = (double*)malloc(sizeof(double) * (size_t)(gcap > 0 ? gcap : 1));
        int64_t rcap = (k < gcap ? k : gcap) + 1;
        orc_heap R;
        R.h = (orc_hit*)malloc(sizeof(orc_hit) * (size_t)(rcap > 0 ? rcap : 1)); R.len = 0; R.cap = rcap;
        if (!hid || !hs || !R.h) { free(hid); free(hs); free(R.h); free(pd); free(pv); return ORC_ENOMEM; }
        int64_t nh = precise_search(I, pd, pv, pn, gamma, hid, hs);
        if (nh < 0) { free(hid); free(hs); free(R.h); free(pd); free(pv); return nh; }
        if (coarse_ids) {
            for (int64_t t = 0; t < nh; t++) { coarse_ids[t] = hid[t]; coarse_scores[t] = hs[t]; }
        }
        if (n_coarse) *n_coarse = nh;
        for (int64_t t = 0; t < nh; t++) {
            int64_t i = hid[t];
            orc_hit x = { orc_inner_product(I->D, i, Q, r), i };
            heap_offer(&R, k, x);
        }
        result = heap_drain_sorted(&R, out_ids, out_scores);
        free(hid); free(hs); free(R.h);
    }
    free(pd); free(pv);
    return result;
}
