/*
 * Double-double (FP64x2) GEMM oracle: C := A B, every entry a scalar
 * double-double dot product.  TEST INFRASTRUCTURE ONLY: it is called by
 * tests/, by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py,
 * never by the CUDA product path.  It shares no code with that path.
 *
 * What it follows (Parikh, van de Geijn, Henry, "Cascading GEMM: High
 * Precision from Low Precision"):
 *   - Section 2.4 (FP64 and FP64x2 numbers, eq. "doubledouble"): a value is
 *     the exact real hi + lo, hi and lo both FP64.
 *   - Section 2.2 (Basics): an FP64x2 multiply is one FMA plus ordinary
 *     multiplies (TwoProd), an FP64x2 add is a chain of dependent adds
 *     (TwoSum).  The FP64x2 triple-nested loop of Section 5 (the accuracy
 *     competitor) is this computation.
 * It is NOT the cascade: it is the quantity the cascade approximates.
 *
 * Building blocks (textbook error-free transformations):
 *   two_sum      Knuth's TwoSum: s = fl(a+b), e = (a+b) - s exactly.
 *   fast_two_sum Dekker's FastTwoSum, valid when |a| >= |b| (or a = 0).
 *   two_prod     p = fl(a*b), e = a*b - p exactly, via a single FMA.
 * Compile with -ffp-contract=off and without fast-math so that every
 * operation below is one IEEE round-to-nearest-even operation.
 */
#include <math.h>
#include <stddef.h>

static inline void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

static inline void fast_two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    *s = x;
    *e = b - (x - a);
}

static inline void two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* (ah + al) * (bh + bl) rounded to a double-double.  The al*bl term is kept. */
static inline void dd_mul(double ah, double al, double bh, double bl,
                          double *rh, double *rl) {
    double p, e;
    two_prod(ah, bh, &p, &e);
    e += ah * bl + al * bh + al * bl;
    fast_two_sum(p, e, rh, rl);
}

/* Accurate double-double addition: two TwoSums, then renormalise twice. */
static inline void dd_add(double ah, double al, double bh, double bl,
                          double *rh, double *rl) {
    double s, e, t, f;
    two_sum(ah, bh, &s, &e);
    two_sum(al, bl, &t, &f);
    e += t;
    fast_two_sum(s, e, &s, &e);
    e += f;
    fast_two_sum(s, e, rh, rl);
}

/* One entry: sum over l = 0..k-1 of A[i,l] * B[l,j], in order, in FP64x2. */
static void dd_dot(int k, const double *Ahi, const double *Alo, int lda,
                   const double *Bhi, const double *Blo, int ldb, int i, int j,
                   double *ch, double *cl) {
    double sh = 0.0, sl = 0.0;
    for (int l = 0; l < k; ++l) {
        double ph, pl;
        size_t ia = (size_t)i * lda + l, ib = (size_t)l * ldb + j;
        dd_mul(Ahi[ia], Alo[ia], Bhi[ib], Blo[ib], &ph, &pl);
        dd_add(sh, sl, ph, pl, &sh, &sl);
    }
    *ch = sh;
    *cl = sl;
}

/* Row-major A (m x k, leading dim lda), B (k x n, ldb), C (m x n, ldc). */
void oracle_ddgemm(int m, int n, int k,
                   const double *Ahi, const double *Alo, int lda,
                   const double *Bhi, const double *Blo, int ldb,
                   double *Chi, double *Clo, int ldc) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j)
            dd_dot(k, Ahi, Alo, lda, Bhi, Blo, ldb, i, j,
                   &Chi[(size_t)i * ldc + j], &Clo[(size_t)i * ldc + j]);
}

/* The same definition, for `count` chosen entries (rows[t], cols[t]). */
void oracle_ddgemm_entries(int k,
                           const double *Ahi, const double *Alo, int lda,
                           const double *Bhi, const double *Blo, int ldb,
                           int count, const int *rows, const int *cols,
                           double *out_hi, double *out_lo) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < count; ++t)
        dd_dot(k, Ahi, Alo, lda, Bhi, Blo, ldb, rows[t], cols[t],
               &out_hi[t], &out_lo[t]);
}

/* Element-wise building blocks, exposed so that tests can pin them alone. */
void oracle_two_sum(double a, double b, double *s, double *e) { two_sum(a, b, s, e); }
void oracle_two_prod(double a, double b, double *p, double *e) { two_prod(a, b, p, e); }
void oracle_dd_add(double ah, double al, double bh, double bl, double *rh, double *rl) {
    dd_add(ah, al, bh, bl, rh, rl);
}
void oracle_dd_mul(double ah, double al, double bh, double bl, double *rh, double *rl) {
    dd_mul(ah, al, bh, bl, rh, rl);
}

/* Threads OpenMP will use (1 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
#else
int oracle_num_threads(void) { return 1; }
#endif
