/*
 * Plain, slow CPU oracle (FP64) for the emulated complex GEMM of
 * "Quantum Circuit Simulation by SGEMM Emulation on Tensor Cores and
 * Automatic Precision Selection" (Ootomo, Manabe, Harada, Yokota, 2023).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * code with the CUDA library and neither includes nor links it.
 *
 * Matrices are BLAS column-major complex64 (interleaved float re, im) with a
 * leading dimension; results are complex128 (interleaved double).
 * op codes: 0 = N (as stored), 1 = T (transpose), 2 = C (conjugate transpose).
 *
 * Every function cites the passage of the paper it follows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double re, im;
} cd;

/* Element (r, c) of op(X), X column-major with leading dimension ldx. */
static inline cd op_elem(const float *X, int op, int64_t r, int64_t c, int64_t ldx) {
    int64_t idx = (op == 0) ? (r + c * ldx) : (c + r * ldx);
    cd v;
    v.re = (double)X[2 * idx];
    v.im = (double)X[2 * idx + 1];
    if (op == 2) v.im = -v.im;
    return v;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * C = alpha * op(A) * op(B) + beta * C_in, in complex128, by the textbook
 * triple loop.  This is the definition the emulated CGEMM approximates
 * (Section 3, the CGEMM unit test compares against the FP64 result).
 * op(A) is m x k, op(B) is k x n.  C_in (complex64, ld ldc_in) may be NULL
 * when beta is zero.  C_out is complex128, column-major, leading dim m.
 */
int oracle_cgemm_naive(int opA, int opB, int64_t m, int64_t n, int64_t k,
                       const double *alpha, const float *A, int64_t lda,
                       const float *B, int64_t ldb, const double *beta,
                       const float *C_in, int64_t ldc_in, double *C_out) {
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double sr = 0.0, si = 0.0;
            for (int64_t l = 0; l < k; ++l) {
                cd a = op_elem(A, opA, i, l, lda);
                cd b = op_elem(B, opB, l, j, ldb);
                sr += a.re * b.re - a.im * b.im;
                si += a.re * b.im + a.im * b.re;
            }
            double cr = alpha[0] * sr - alpha[1] * si;
            double ci = alpha[0] * si + alpha[1] * sr;
            if (C_in && (beta[0] != 0.0 || beta[1] != 0.0)) {
                double xr = (double)C_in[2 * (i + j * ldc_in)];
                double xi = (double)C_in[2 * (i + j * ldc_in) + 1];
                cr += beta[0] * xr - beta[1] * xi;
                ci += beta[0] * xi + beta[1] * xr;
            }
            C_out[2 * (i + j * m)] = cr;
            C_out[2 * (i + j * m) + 1] = ci;
        }
    }
    return 0;
}

/*
 * Same product restricted to the output rows listed in ``rows`` (nrows of
 * them), parallel over output columns with OpenMP.  Used to check and time
 * large GEMMs on a row sample.  C_out is complex128 nrows x n, column-major
 * (leading dim nrows).  The k loop is outermost per column so that the
 * sampled rows of op(A), copied once to FP64, stream contiguously.
 */
int oracle_cgemm_rows(int opA, int opB, int64_t m, int64_t n, int64_t k,
                      const double *alpha, const float *A, int64_t lda,
                      const float *B, int64_t ldb, const double *beta,
                      const float *C_in, int64_t ldc_in, const int64_t *rows,
                      int64_t nrows, double *C_out) {
    (void)m;
    double *Ar = (double *)malloc(sizeof(double) * 2 * (size_t)nrows * (size_t)(k > 0 ? k : 1));
    if (!Ar) return -1;
    for (int64_t l = 0; l < k; ++l)
        for (int64_t r = 0; r < nrows; ++r) {
            cd a = op_elem(A, opA, rows[r], l, lda);
            Ar[2 * (l * nrows + r)] = a.re;
            Ar[2 * (l * nrows + r) + 1] = a.im;
        }
    int err = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)(nrows > 0 ? nrows : 1));
        if (!acc) {
#pragma omp atomic write
            err = -1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t j = 0; j < n; ++j) {
                for (int64_t r = 0; r < 2 * nrows; ++r) acc[r] = 0.0;
                for (int64_t l = 0; l < k; ++l) {
                    cd b = op_elem(B, opB, l, j, ldb);
                    const double *ar = Ar + 2 * l * nrows;
                    for (int64_t r = 0; r < nrows; ++r) {
                        acc[2 * r] += ar[2 * r] * b.re - ar[2 * r + 1] * b.im;
                        acc[2 * r + 1] += ar[2 * r] * b.im + ar[2 * r + 1] * b.re;
                    }
                }
                for (int64_t r = 0; r < nrows; ++r) {
                    double sr = acc[2 * r], si = acc[2 * r + 1];
                    double cr = alpha[0] * sr - alpha[1] * si;
                    double ci = alpha[0] * si + alpha[1] * sr;
                    if (C_in && (beta[0] != 0.0 || beta[1] != 0.0)) {
                        int64_t ix = rows[r] + j * ldc_in;
                        double xr = (double)C_in[2 * ix], xi = (double)C_in[2 * ix + 1];
                        cr += beta[0] * xr - beta[1] * xi;
                        ci += beta[0] * xi + beta[1] * xr;
                    }
                    C_out[2 * (r + j * nrows)] = cr;
                    C_out[2 * (r + j * nrows) + 1] = ci;
                }
            }
            free(acc);
        }
    }
    free(Ar);
    return err;
}

/* ------------------------------------------------------------------------
 * Conversions to the low-precision tensor-core input types ("toLow" of
 * Eq. 1 in Section 2.1), restated from the IEEE 754 binary16 definition and
 * from the TF32 format (8-bit exponent, 10-bit fraction), both with
 * round-to-nearest, ties to even.
 * ---------------------------------------------------------------------- */

static inline uint32_t f32_bits(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
}
static inline float bits_f32(uint32_t u) {
    float x;
    memcpy(&x, &u, 4);
    return x;
}

/* Round the non-negative integer significand ``sig`` right by ``shift``
 * bits, nearest with ties to even.  shift >= 1. */
static inline uint64_t rne_shift(uint64_t sig, int shift) {
    if (shift >= 64) return 0;
    uint64_t keep = sig >> shift;
    uint64_t rest = sig & ((1ull << shift) - 1ull);
    uint64_t half = 1ull << (shift - 1);
    if (rest > half || (rest == half && (keep & 1ull))) keep += 1;
    return keep;
}

/* binary32 -> binary16 bit pattern, round to nearest even. */
uint16_t oracle_f32_to_f16(float x) {
    uint32_t u = f32_bits(x);
    uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
    uint32_t ex = (u >> 23) & 0xFFu;
    uint32_t fr = u & 0x7FFFFFu;
    if (ex == 0xFFu) return (uint16_t)(sign | 0x7C00u | (fr ? 0x200u : 0u));
    if (ex == 0u) return sign; /* |x| < 2^-126, far below half the least FP16 subnormal */
    int e = (int)ex - 127;     /* |x| = (1 + fr/2^23) 2^e */
    uint64_t sig = 0x800000ull | fr; /* 24-bit significand, |x| = sig 2^(e-23) */
    if (e >= -14) {
        /* normal range: keep 11 significant bits */
        uint64_t r = rne_shift(sig, 13); /* in [2^10, 2^11] */
        int eb = e + 15;
        if (r == 0x800ull) { r = 0x400ull; eb += 1; }
        if (eb >= 31) return (uint16_t)(sign | 0x7C00u); /* overflow to infinity */
        return (uint16_t)(sign | ((uint32_t)eb << 10) | (uint32_t)(r - 0x400ull));
    }
    /* subnormal: |x| / 2^-24 = sig 2^(e+1), rounded to an integer */
    uint64_t r = rne_shift(sig, -(e + 1));
    return (uint16_t)(sign | (uint32_t)r); /* r == 0x400 is the least normal, encoded alike */
}

float oracle_f16_to_f32(uint16_t h) {
    int sign = (h >> 15) & 1;
    int ex = (h >> 10) & 0x1F;
    int fr = h & 0x3FF;
    double v;
    if (ex == 0x1F) {
        v = fr ? NAN : INFINITY;
    } else if (ex == 0) {
        v = ldexp((double)fr, -24);
    } else {
        v = ldexp((double)(0x400 | fr), ex - 25);
    }
    return (float)(sign ? -v : v);
}

/* binary32 -> TF32 (value kept in a binary32 container), round to nearest
 * even at the 10th fraction bit. */
float oracle_f32_to_tf32(float x) {
    uint32_t u = f32_bits(x);
    uint32_t ex = (u >> 23) & 0xFFu;
    if (ex == 0xFFu) return x;
    uint32_t sign = u & 0x80000000u;
    uint32_t mag = u & 0x7FFFFFFFu; /* exponent and fraction as one integer */
    /* The 13 dropped bits are below the last kept fraction bit; rounding the
     * magnitude integer rounds the value (a carry out of the fraction bumps
     * the exponent, and out of the largest finite value gives infinity). */
    uint64_t r = rne_shift((uint64_t)mag, 13) << 13;
    return bits_f32(sign | (uint32_t)r);
}

/* binary32 -> bfloat16 (kept in a binary32 container), nearest even. */
float oracle_f32_to_bf16(float x) {
    uint32_t u = f32_bits(x);
    uint32_t ex = (u >> 23) & 0xFFu;
    if (ex == 0xFFu) return x;
    uint32_t sign = u & 0x80000000u;
    uint32_t mag = u & 0x7FFFFFFFu;
    uint64_t r = rne_shift((uint64_t)mag, 16) << 16;
    return bits_f32(sign | (uint32_t)r);
}

/*
 * The split of Eq. 1 (Section 2.1), applied after an optional power-of-two
 * scaling 2^s (the FP16TCEC-with-scaling mode of Section 4):
 *   xs = x * 2^s,  hi = toLow(xs),  lo = toLow((xs - toF32(hi)) * 2^11).
 * kind: 0 = FP16, 1 = TF32, 2 = BF16.  hi and lo are returned as the exact
 * binary32 values of the low-precision numbers.  The subtraction and the
 * scalings are exact in binary32, so this is also the value a binary32
 * implementation computes.
 */
void oracle_split(int kind, int s, int64_t count, const float *x, float *hi, float *lo) {
    for (int64_t i = 0; i < count; ++i) {
        float xs = (float)ldexp((double)x[i], s);
        float h, l;
        if (kind == 0) {
            h = oracle_f16_to_f32(oracle_f32_to_f16(xs));
            float r = (float)((double)xs - (double)h);
            l = oracle_f16_to_f32(oracle_f32_to_f16((float)ldexp((double)r, 11)));
        } else if (kind == 1) {
            h = oracle_f32_to_tf32(xs);
            float r = (float)((double)xs - (double)h);
            l = oracle_f32_to_tf32((float)ldexp((double)r, 11));
        } else {
            h = oracle_f32_to_bf16(xs);
            float r = (float)((double)xs - (double)h);
            l = oracle_f32_to_bf16((float)ldexp((double)r, 11));
        }
        hi[i] = h;
        lo[i] = l;
    }
}

/*
 * Exponent statistics of Section 4.1 over every real and imaginary scalar of
 * a column-major complex64 matrix (rows x cols, leading dim ldx).  For each
 * non-zero scalar, e = floor(log2 |x|); the histogram bin is e + 127 for
 * normal binary32 numbers, 0 for subnormals (e < -126) and 255 for Inf/NaN.
 * Zeros are counted apart in *n_zero and enter no bin.  hist has 256 slots.
 */
void oracle_exp_stats(int64_t rows, int64_t cols, const float *X, int64_t ldx,
                      int64_t *hist, int64_t *n_zero) {
    for (int b = 0; b < 256; ++b) hist[b] = 0;
    *n_zero = 0;
    for (int64_t c = 0; c < cols; ++c)
        for (int64_t r = 0; r < rows; ++r)
            for (int p = 0; p < 2; ++p) {
                float v = X[2 * (r + c * ldx) + p];
                if (!isfinite(v)) {
                    hist[255]++;
                } else if (v == 0.0f) {
                    (*n_zero)++;
                } else {
                    int ex;
                    (void)frexp((double)v, &ex); /* |v| = f 2^ex, f in [0.5, 1) */
                    int e = ex - 1;              /* floor(log2|v|) */
                    int bin = e + 127;
                    if (bin < 1) bin = 0;
                    hist[bin]++;
                }
            }
}

/*
 * The emulated product in exact arithmetic: Eq. 1's compensated sum
 *   hi_A hi_B + (lo_A hi_B + hi_A lo_B) / 2^11
 * for each of the four real products of the complex expansion in Section 3
 * (Re = Ar Br - Ai Bi, Im = Ar Bi + Ai Br), with the scalings 2^sA, 2^sB
 * undone on the result, then alpha * P + beta * C_in.  Summation in FP64.
 * The tensor-core kernel differs from this only by FP32 accumulation
 * rounding.  kind: 0 FP16, 1 TF32, 2 BF16.  Output as oracle_cgemm_naive.
 */
int oracle_tcec_cgemm(int kind, int sA, int sB, int opA, int opB, int64_t m, int64_t n,
                      int64_t k, const double *alpha, const float *A, int64_t lda,
                      const float *B, int64_t ldb, const double *beta, const float *C_in,
                      int64_t ldc_in, double *C_out) {
    size_t na = (size_t)m * (size_t)k, nb = (size_t)k * (size_t)n;
    float *a = (float *)malloc(sizeof(float) * 2 * (na ? na : 1));
    float *b = (float *)malloc(sizeof(float) * 2 * (nb ? nb : 1));
    float *ah = (float *)malloc(sizeof(float) * 2 * (na ? na : 1));
    float *al = (float *)malloc(sizeof(float) * 2 * (na ? na : 1));
    float *bh = (float *)malloc(sizeof(float) * 2 * (nb ? nb : 1));
    float *bl = (float *)malloc(sizeof(float) * 2 * (nb ? nb : 1));
    if (!a || !b || !ah || !al || !bh || !bl) {
        free(a); free(b); free(ah); free(al); free(bh); free(bl);
        return -1;
    }
    /* op(A) as an m x k interleaved array, index (i + l m) */
    for (int64_t l = 0; l < k; ++l)
        for (int64_t i = 0; i < m; ++i) {
            cd v = op_elem(A, opA, i, l, lda);
            a[2 * (i + l * m)] = (float)v.re;
            a[2 * (i + l * m) + 1] = (float)v.im;
        }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t l = 0; l < k; ++l) {
            cd v = op_elem(B, opB, l, j, ldb);
            b[2 * (l + j * k)] = (float)v.re;
            b[2 * (l + j * k) + 1] = (float)v.im;
        }
    oracle_split(kind, sA, 2 * (int64_t)na, a, ah, al);
    oracle_split(kind, sB, 2 * (int64_t)nb, b, bh, bl);
    double unscale = ldexp(1.0, -(sA + sB));
    double corr = ldexp(1.0, -11);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            double r0 = 0, i0 = 0, r1 = 0, i1 = 0;
            for (int64_t l = 0; l < k; ++l) {
                size_t ia = 2 * (size_t)(i + l * m), ib = 2 * (size_t)(l + j * k);
                double arh = ah[ia], aih = ah[ia + 1], arl = al[ia], ail = al[ia + 1];
                double brh = bh[ib], bih = bh[ib + 1], brl = bl[ib], bil = bl[ib + 1];
                r0 += arh * brh - aih * bih;
                i0 += arh * bih + aih * brh;
                r1 += (arl * brh + arh * brl) - (ail * bih + aih * bil);
                i1 += (arl * bih + arh * bil) + (ail * brh + aih * brl);
            }
            double sr = (r0 + corr * r1) * unscale;
            double si = (i0 + corr * i1) * unscale;
            double cr = alpha[0] * sr - alpha[1] * si;
            double ci = alpha[0] * si + alpha[1] * sr;
            if (C_in && (beta[0] != 0.0 || beta[1] != 0.0)) {
                double xr = (double)C_in[2 * (i + j * ldc_in)];
                double xi = (double)C_in[2 * (i + j * ldc_in) + 1];
                cr += beta[0] * xr - beta[1] * xi;
                ci += beta[0] * xi + beta[1] * xr;
            }
            C_out[2 * (i + j * m)] = cr;
            C_out[2 * (i + j * m) + 1] = ci;
        }
    free(a); free(b); free(ah); free(al); free(bh); free(bl);
    return 0;
}

/*
 * Gauss's three-product form of the emulated complex product (a variant
 * beyond the paper): with ar, ai the parts of op(A) and br, bi those of
 * op(B) (conjugation applied),
 *   T1 = ar br,  T2 = ai bi,  T3 = (ar + ai)(br + bi),
 *   Re = T1 - T2,  Im = T3 - T1 - T2,
 * where each real product is Eq. 1's compensated product in exact
 * arithmetic, the operand sums are binary32 additions, and for the FP16 kind
 * (kind 0) the sums are scaled by 2^(sA - 1), 2^(sB - 1) instead of 2^sA,
 * 2^sB.  Then alpha P + beta C_in.  Output as oracle_cgemm_naive.
 */
int oracle_tcec_cgemm_3m(int kind, int sA, int sB, int opA, int opB, int64_t m, int64_t n,
                         int64_t k, const double *alpha, const float *A, int64_t lda,
                         const float *B, int64_t ldb, const double *beta, const float *C_in,
                         int64_t ldc_in, double *C_out) {
    size_t na = (size_t)m * (size_t)k, nb = (size_t)k * (size_t)n;
    size_t ta = 3 * (na ? na : 1), tb = 3 * (nb ? nb : 1);
    float *a = (float *)malloc(sizeof(float) * ta), *b = (float *)malloc(sizeof(float) * tb);
    float *ah = (float *)malloc(sizeof(float) * ta), *al = (float *)malloc(sizeof(float) * ta);
    float *bh = (float *)malloc(sizeof(float) * tb), *bl = (float *)malloc(sizeof(float) * tb);
    if (!a || !b || !ah || !al || !bh || !bl) {
        free(a); free(b); free(ah); free(al); free(bh); free(bl);
        return -1;
    }
    /* part p of op(A) at a + p na, index (i + l m); likewise for op(B), (l + j k) */
    for (int64_t l = 0; l < k; ++l)
        for (int64_t i = 0; i < m; ++i) {
            cd v = op_elem(A, opA, i, l, lda);
            float re = (float)v.re, im = (float)v.im;
            a[i + l * m] = re;
            a[na + i + l * m] = im;
            a[2 * na + i + l * m] = re + im;
        }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t l = 0; l < k; ++l) {
            cd v = op_elem(B, opB, l, j, ldb);
            float re = (float)v.re, im = (float)v.im;
            b[l + j * k] = re;
            b[nb + l + j * k] = im;
            b[2 * nb + l + j * k] = re + im;
        }
    const int s3A = (kind == 0) ? sA - 1 : sA, s3B = (kind == 0) ? sB - 1 : sB;
    oracle_split(kind, sA, 2 * (int64_t)na, a, ah, al);
    oracle_split(kind, s3A, (int64_t)na, a + 2 * na, ah + 2 * na, al + 2 * na);
    oracle_split(kind, sB, 2 * (int64_t)nb, b, bh, bl);
    oracle_split(kind, s3B, (int64_t)nb, b + 2 * nb, bh + 2 * nb, bl + 2 * nb);
    const double corr = ldexp(1.0, -11);
    const double un12 = ldexp(1.0, -(sA + sB)), un3 = ldexp(1.0, -(s3A + s3B));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            double T[3];
            for (int p = 0; p < 3; ++p) {
                double p0 = 0, p1 = 0;
                for (int64_t l = 0; l < k; ++l) {
                    size_t ia = p * na + (size_t)(i + l * m), ib = p * nb + (size_t)(l + j * k);
                    p0 += (double)ah[ia] * (double)bh[ib];
                    p1 += (double)al[ia] * (double)bh[ib] + (double)ah[ia] * (double)bl[ib];
                }
                T[p] = (p0 + corr * p1) * (p == 2 ? un3 : un12);
            }
            double sr = T[0] - T[1];
            double si = T[2] - T[0] - T[1];
            double cr = alpha[0] * sr - alpha[1] * si;
            double ci = alpha[0] * si + alpha[1] * sr;
            if (C_in && (beta[0] != 0.0 || beta[1] != 0.0)) {
                double xr = (double)C_in[2 * (i + j * ldc_in)];
                double xi = (double)C_in[2 * (i + j * ldc_in) + 1];
                cr += beta[0] * xr - beta[1] * xi;
                ci += beta[0] * xi + beta[1] * xr;
            }
            C_out[2 * (i + j * m)] = cr;
            C_out[2 * (i + j * m) + 1] = ci;
        }
    free(a); free(b); free(ah); free(al); free(bh); free(bl);
    return 0;
}

/* ------------------------------------------------------------------------
 * Real matrices (the SGEMM that Section 2.1 emulates).  Column-major
 * binary32 with a leading dimension; op 0 = N, 1 or 2 = T.  Results are
 * binary64, column-major.
 * ---------------------------------------------------------------------- */

/* Element (r, c) of op(X). */
static inline double op_elem_real(const float *X, int op, int64_t r, int64_t c, int64_t ldx) {
    return (double)X[(op == 0) ? (r + c * ldx) : (c + r * ldx)];
}

/*
 * C = alpha op(A) op(B) + beta C_in for the output rows listed in ``rows``
 * (all m rows, in order, when rows is NULL), by the textbook sum over l in
 * binary64, parallel over output columns.  C_in (binary32, ld ldc_in) may
 * be NULL when beta is zero.  C_out is nrows x n, leading dim nrows.
 */
int oracle_sgemm_rows(int opA, int opB, int64_t m, int64_t n, int64_t k, double alpha,
                      const float *A, int64_t lda, const float *B, int64_t ldb, double beta,
                      const float *C_in, int64_t ldc_in, const int64_t *rows, int64_t nrows,
                      double *C_out) {
    if (!rows) nrows = m;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t r = 0; r < nrows; ++r) {
            const int64_t i = rows ? rows[r] : r;
            double acc = 0.0;
            for (int64_t l = 0; l < k; ++l)
                acc += op_elem_real(A, opA, i, l, lda) * op_elem_real(B, opB, l, j, ldb);
            double c = alpha * acc;
            if (C_in && beta != 0.0) c += beta * (double)C_in[i + j * ldc_in];
            C_out[r + j * nrows] = c;
        }
    }
    return err;
}

/*
 * The emulated real product of Eq. 1 in exact arithmetic:
 *   2^-(sA+sB) (hi_A hi_B + (lo_A hi_B + hi_A lo_B) / 2^11)
 * summed over l in binary64, then alpha P + beta C_in.  The tensor-core
 * kernel differs from this only by binary32 accumulation rounding.
 * kind: 0 FP16, 1 TF32, 2 BF16.  Output as oracle_sgemm_rows (all rows).
 */
int oracle_tcec_sgemm(int kind, int sA, int sB, int opA, int opB, int64_t m, int64_t n, int64_t k,
                      double alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                      double beta, const float *C_in, int64_t ldc_in, double *C_out) {
    size_t na = (size_t)m * (size_t)k, nb = (size_t)k * (size_t)n;
    float *a = (float *)malloc(sizeof(float) * (na ? na : 1));
    float *b = (float *)malloc(sizeof(float) * (nb ? nb : 1));
    float *ah = (float *)malloc(sizeof(float) * (na ? na : 1));
    float *al = (float *)malloc(sizeof(float) * (na ? na : 1));
    float *bh = (float *)malloc(sizeof(float) * (nb ? nb : 1));
    float *bl = (float *)malloc(sizeof(float) * (nb ? nb : 1));
    if (!a || !b || !ah || !al || !bh || !bl) {
        free(a); free(b); free(ah); free(al); free(bh); free(bl);
        return -1;
    }
    for (int64_t l = 0; l < k; ++l)
        for (int64_t i = 0; i < m; ++i) a[i + l * m] = (float)op_elem_real(A, opA, i, l, lda);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t l = 0; l < k; ++l) b[l + j * k] = (float)op_elem_real(B, opB, l, j, ldb);
    oracle_split(kind, sA, (int64_t)na, a, ah, al);
    oracle_split(kind, sB, (int64_t)nb, b, bh, bl);
    double unscale = ldexp(1.0, -(sA + sB));
    double corr = ldexp(1.0, -11);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            double p0 = 0, p1 = 0;
            for (int64_t l = 0; l < k; ++l) {
                size_t ia = (size_t)(i + l * m), ib = (size_t)(l + j * k);
                p0 += (double)ah[ia] * (double)bh[ib];
                p1 += (double)al[ia] * (double)bh[ib] + (double)ah[ia] * (double)bl[ib];
            }
            double c = alpha * ((p0 + corr * p1) * unscale);
            if (C_in && beta != 0.0) c += beta * (double)C_in[i + j * ldc_in];
            C_out[i + j * m] = c;
        }
    free(a); free(b); free(ah); free(al); free(bh); free(bl);
    return 0;
}

/*
 * Exponent statistics of Section 4.1 over the scalars of a real matrix
 * (rows x cols, leading dim ldx); bins as oracle_exp_stats.
 */
void oracle_exp_stats_real(int64_t rows, int64_t cols, const float *X, int64_t ldx,
                           int64_t *hist, int64_t *n_zero) {
    for (int b = 0; b < 256; ++b) hist[b] = 0;
    *n_zero = 0;
    for (int64_t c = 0; c < cols; ++c)
        for (int64_t r = 0; r < rows; ++r) {
            float v = X[r + c * ldx];
            if (!isfinite(v)) {
                hist[255]++;
            } else if (v == 0.0f) {
                (*n_zero)++;
            } else {
                int ex;
                (void)frexp((double)v, &ex);
                int bin = ex - 1 + 127;
                if (bin < 1) bin = 0;
                hist[bin]++;
            }
        }
}

/*
 * Pairwise tensor contraction by nested loops (Section 2.2: connected edges
 * are summed, Einstein convention), with no reshaping to a GEMM.  Tensors
 * are complex128, row-major (last index fastest).  Each label is a
 * non-negative integer; a label of C must occur in A or B; labels of A and B
 * absent from C are summed.  The dimension of each label is taken from the
 * operand it appears in.  C (rc labels) is overwritten.
 */
int oracle_contract_pair(int ra, const int *la, const int64_t *da, const double *A,
                         int rb, const int *lb, const int64_t *db, const double *B,
                         int rc, const int *lc, double *C) {
    int lab[64];
    int64_t dim[64];
    int nl = 0;
    const int *ls[2] = {la, lb};
    const int64_t *ds[2] = {da, db};
    int rs[2] = {ra, rb};
    for (int t = 0; t < 2; ++t)
        for (int q = 0; q < rs[t]; ++q) {
            int f = -1;
            for (int u = 0; u < nl; ++u)
                if (lab[u] == ls[t][q]) f = u;
            if (f < 0) {
                if (nl >= 64) return -1;
                lab[nl] = ls[t][q];
                dim[nl] = ds[t][q];
                ++nl;
            } else if (dim[f] != ds[t][q]) {
                return -2;
            }
        }
    /* position of each operand/output index in the label list */
    int pa[64], pb[64], pc[64];
    int64_t dc[64];
    for (int q = 0; q < ra; ++q)
        for (int u = 0; u < nl; ++u) if (lab[u] == la[q]) pa[q] = u;
    for (int q = 0; q < rb; ++q)
        for (int u = 0; u < nl; ++u) if (lab[u] == lb[q]) pb[q] = u;
    for (int q = 0; q < rc; ++q) {
        pc[q] = -1;
        for (int u = 0; u < nl; ++u) if (lab[u] == lc[q]) pc[q] = u;
        if (pc[q] < 0) return -3;
        dc[q] = dim[pc[q]];
    }
    int64_t csize = 1;
    for (int q = 0; q < rc; ++q) csize *= dc[q];
    for (int64_t t = 0; t < 2 * csize; ++t) C[t] = 0.0;
    int64_t idx[64];
    for (int u = 0; u < nl; ++u) idx[u] = 0;
    for (;;) {
        int64_t ia = 0, ib = 0, ic = 0;
        for (int q = 0; q < ra; ++q) ia = ia * da[q] + idx[pa[q]];
        for (int q = 0; q < rb; ++q) ib = ib * db[q] + idx[pb[q]];
        for (int q = 0; q < rc; ++q) ic = ic * dc[q] + idx[pc[q]];
        double ar = A[2 * ia], ai = A[2 * ia + 1], br = B[2 * ib], bi = B[2 * ib + 1];
        C[2 * ic] += ar * br - ai * bi;
        C[2 * ic + 1] += ar * bi + ai * br;
        int u = nl - 1;
        while (u >= 0) {
            if (++idx[u] < dim[u]) break;
            idx[u] = 0;
            --u;
        }
        if (u < 0) break;
    }
    return 0;
}

/*
 * State-vector method (Section 1; the state of Section 2.2 as a 2^n complex
 * vector), in place and in FP64, for circuits too large for a copy per
 * gate.  psi holds 2^n complex128 amplitudes; qubit q is bit (n-1-q) of the
 * basis index (qubit 0 most significant).  A one-qubit gate g (2x2, row =
 * output) updates each pair of amplitudes that differ in that bit; a
 * two-qubit gate (4x4, basis index 2 b(q0) + b(q1)) each quadruple.
 */
void oracle_sv_apply1(int n, double *psi, int q, const double *g) {
    const int64_t N = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << (n - 1 - q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        if (i & bit) continue;
        const int64_t j = i | bit;
        const double a0r = psi[2 * i], a0i = psi[2 * i + 1];
        const double a1r = psi[2 * j], a1i = psi[2 * j + 1];
        psi[2 * i] = g[0] * a0r - g[1] * a0i + g[2] * a1r - g[3] * a1i;
        psi[2 * i + 1] = g[0] * a0i + g[1] * a0r + g[2] * a1i + g[3] * a1r;
        psi[2 * j] = g[4] * a0r - g[5] * a0i + g[6] * a1r - g[7] * a1i;
        psi[2 * j + 1] = g[4] * a0i + g[5] * a0r + g[6] * a1i + g[7] * a1r;
    }
}

void oracle_sv_apply2(int n, double *psi, int q0, int q1, const double *g) {
    const int64_t N = (int64_t)1 << n;
    const int64_t b0 = (int64_t)1 << (n - 1 - q0);
    const int64_t b1 = (int64_t)1 << (n - 1 - q1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        if ((i & b0) || (i & b1)) continue;
        const int64_t idx[4] = {i, i | b1, i | b0, i | b0 | b1};
        double ar[4], ai[4];
        for (int u = 0; u < 4; ++u) {
            ar[u] = psi[2 * idx[u]];
            ai[u] = psi[2 * idx[u] + 1];
        }
        for (int r = 0; r < 4; ++r) {
            double sr = 0.0, si = 0.0;
            for (int c = 0; c < 4; ++c) {
                const double gr = g[2 * (4 * r + c)], gi = g[2 * (4 * r + c) + 1];
                sr += gr * ar[c] - gi * ai[c];
                si += gr * ai[c] + gi * ar[c];
            }
            psi[2 * idx[r]] = sr;
            psi[2 * idx[r] + 1] = si;
        }
    }
}
