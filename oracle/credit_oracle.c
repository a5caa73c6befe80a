/*
 * credit_oracle.c -- plain FP64 CPU oracle for the reduction-reuse row ops.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or constant table with the
 * CUDA library; the two meet only at the seeded input bytes.
 *
 * What it computes (CREDIT, Sec. III-B, Eq. 1): every op reduces a row of N
 * elements to a few statistics and then applies an elementwise function h to
 * every element of the same row.  Because the cluster split of Eq. 2 is only a
 * re-association of the same reductions, the oracle is the plain definition of
 * each op, one row at a time, in double precision, with no blocking, slicing
 * or reordering:
 *
 *   softmax   m = max_i x_i,  S = sum_i exp(x_i - m),  y_i = exp(x_i - m) / S
 *   logsumexp m + ln S                                (one value per row)
 *   layernorm mu = sum x / N, var = sum (x - mu)^2 / N  (biased, two passes),
 *             y_i = (x_i - mu) / sqrt(var + eps) * gamma_i + beta_i
 *   rmsnorm   y_i = x_i / sqrt(sum x^2 / N + eps) * gamma_i
 *
 * and the input gradients of softmax, LayerNorm and RMSNorm (their
 * vector-Jacobian products with an upstream gradient dy, given the forward's
 * saved row statistics; see the backward section below).
 *
 * Sums use Neumaier compensation so that the oracle's own rounding stays far
 * below every tolerance the GPU path is held to.
 *
 * Inputs are decoded EXACTLY to double: BF16 widens exactly; an FP8-E4M3 code
 * times its FP32 per-row scale is exact in double (4 + 24 significant bits).
 * Output rounding (BF16 round-to-nearest-even, E4M3 round-to-nearest-even with
 * saturation to +-448) is written here from the two formats' definitions.
 *
 * FP8 output uses a per-row scale s = amax_i |y_i| / 448, codes q_i =
 * RNE_sat(y_i / s); a row whose outputs are all zero gets s = 1 and q = 0.
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared -ffp-contract=off (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <float.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_F32 = 0, OR_BF16 = 1, OR_E4M3 = 2 };
enum { OR_SOFTMAX = 0, OR_LOGSUMEXP = 1, OR_LAYERNORM = 2, OR_RMSNORM = 3 };
enum { OR_SOFTMAX_LOGITS = 7, OR_XENT = 8 };  /* backward batch only */

/* ------------------------------------------------------------------ */
/* Compensated (Neumaier) summation                                    */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } nsum_t;

static inline void nsum_add(nsum_t *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else                       a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nsum_get(const nsum_t *a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* Number formats, from their definitions                              */
/* ------------------------------------------------------------------ */

/* bfloat16: 1 sign, 8 exponent (bias 127), 7 fraction bits; the upper half
 * of an IEEE binary32. */
double oracle_bf16_to_double(uint16_t b) {
    int sign = (b >> 15) & 1;
    int e = (b >> 7) & 0xFF;
    int f = b & 0x7F;
    double v;
    if (e == 0xFF) v = f ? NAN : INFINITY;
    else if (e == 0) v = ldexp((double)f, -126 - 7);          /* subnormal */
    else v = ldexp(1.0 + (double)f / 128.0, e - 127);
    return sign ? -v : v;
}

/* FP8 E4M3 ("fn" variant): 1 sign, 4 exponent (bias 7), 3 fraction bits; no
 * infinities; S.1111.111 is NaN; largest finite magnitude 1.75 * 2^8 = 448. */
double oracle_e4m3_to_double(uint8_t b) {
    int sign = (b >> 7) & 1;
    int e = (b >> 3) & 0xF;
    int f = b & 0x7;
    double v;
    if (e == 0xF && f == 0x7) return NAN;
    if (e == 0) v = ldexp((double)f, -6 - 3);                 /* subnormal */
    else v = ldexp(1.0 + (double)f / 8.0, e - 7);
    return sign ? -v : v;
}

/* Round v to a multiple of 2^k, ties to even (exact for the magnitudes used:
 * v / 2^k is an exact power-of-two scaling). */
static double round_to_quantum(double v, int k) {
    double t = ldexp(v, -k);
    double r = nearbyint(t);           /* default rounding mode: ties to even */
    return ldexp(r, k);
}

uint16_t oracle_double_to_bf16(double v) {
    if (isnan(v)) return 0x7FC0;
    uint16_t sign = signbit(v) ? 0x8000 : 0;
    double a = fabs(v);
    if (a == 0.0) return sign;
    int e;
    frexp(a, &e);                      /* a = m * 2^e, m in [0.5, 1) */
    int ex = e - 1;                    /* a in [2^ex, 2^(ex+1)) */
    if (ex < -126) ex = -126;          /* subnormal quantum 2^-133 */
    double q = round_to_quantum(a, ex - 7);
    /* largest finite bf16 = (2 - 2^-7) * 2^127; overflow rounds to inf */
    if (q >= ldexp(2.0, 127)) return sign | 0x7F80;
    if (q == 0.0) return sign;
    int qe;
    frexp(q, &qe);
    int qx = qe - 1;
    if (qx < -126) {                   /* subnormal encoding */
        int f = (int)ldexp(q, 133);
        return sign | (uint16_t)f;
    }
    int f = (int)(ldexp(q, -qx) * 128.0 - 128.0 + 0.5);
    return sign | (uint16_t)((qx + 127) << 7) | (uint16_t)f;
}

uint8_t oracle_double_to_e4m3_sat(double v) {
    if (isnan(v)) return 0x7F;
    uint8_t sign = signbit(v) ? 0x80 : 0;
    double a = fabs(v);
    if (a == 0.0) return sign;
    int e;
    frexp(a, &e);
    int ex = e - 1;
    if (ex < -6) ex = -6;              /* subnormal quantum 2^-9 */
    double q = round_to_quantum(a, ex - 3);
    if (q > 448.0) q = 448.0;          /* saturate (satfinite) */
    if (q == 0.0) return sign;
    int qe;
    frexp(q, &qe);
    int qx = qe - 1;
    if (qx < -6) {
        int f = (int)ldexp(q, 9);
        return sign | (uint8_t)f;
    }
    int f = (int)(ldexp(q, -qx) * 8.0 - 8.0 + 0.5);
    return sign | (uint8_t)((qx + 7) << 3) | (uint8_t)f;
}

/* ------------------------------------------------------------------ */
/* The four ops on one row of doubles (Eq. 1, plain definitions)        */
/* ------------------------------------------------------------------ */

void oracle_softmax_row(const double *x, int64_t n, double *y) {
    double m = -INFINITY;
    for (int64_t i = 0; i < n; ++i) m = x[i] > m ? x[i] : m;
    nsum_t S = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&S, exp(x[i] - m));
    double s = nsum_get(&S);
    for (int64_t i = 0; i < n; ++i) y[i] = exp(x[i] - m) / s;
}

double oracle_lse_row(const double *x, int64_t n) {
    double m = -INFINITY;
    for (int64_t i = 0; i < n; ++i) m = x[i] > m ? x[i] : m;
    nsum_t S = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&S, exp(x[i] - m));
    return m + log(nsum_get(&S));
}

void oracle_layernorm_row(const double *x, int64_t n, const double *gamma,
                          const double *beta, double eps, double *y) {
    nsum_t S = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&S, x[i]);
    double mu = nsum_get(&S) / (double)n;
    nsum_t V = {0, 0};
    for (int64_t i = 0; i < n; ++i) { double d = x[i] - mu; nsum_add(&V, d * d); }
    double var = nsum_get(&V) / (double)n;
    double r = 1.0 / sqrt(var + eps);
    for (int64_t i = 0; i < n; ++i) {
        double g = gamma ? gamma[i] : 1.0;
        double b = beta ? beta[i] : 0.0;
        y[i] = (x[i] - mu) * r * g + b;
    }
}

void oracle_rmsnorm_row(const double *x, int64_t n, const double *gamma,
                        double eps, double *y) {
    nsum_t S = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&S, x[i] * x[i]);
    double r = 1.0 / sqrt(nsum_get(&S) / (double)n + eps);
    for (int64_t i = 0; i < n; ++i) {
        double g = gamma ? gamma[i] : 1.0;
        y[i] = x[i] * r * g;
    }
}

/* ------------------------------------------------------------------ */
/* Input gradients (the backward members of the workload suite,        */
/* Sec. IV-A): the vector-Jacobian product of each forward op above    */
/* with the upstream gradient dy, by the chain rule through the row    */
/* statistics.  With g_i = dy_i * gamma_i (gamma = 1 when absent):      */
/*   softmax   s = sum_j y_j dy_j,                  dx_i = y_i (dy_i - s) */
/*             (y is the forward output)                              */
/*   layernorm xh_i = (x_i - mean) * rstd,                            */
/*             dx_i = rstd (g_i - sum_j g_j / N - xh_i sum_j g_j xh_j / N) */
/*   rmsnorm   xh_i = x_i * rstd,                                     */
/*             dx_i = rstd (g_i - xh_i sum_j g_j xh_j / N)            */
/* mean and rstd are the forward's saved row statistics (rstd =       */
/* 1/sqrt(var + eps) and 1/sqrt(sum x^2 / N + eps)); they are taken as */
/* given, so the result is exact for the statistics the caller holds.  */
/* The derivation: d mean / d x_k = 1/N, d rstd / d x_k = -rstd^2 xh_k / N */
/* (layernorm; the mean's own term cancels because sum (x - mean) = 0) */
/* and -rstd^2 xh_k / N (rmsnorm).                                    */
/* ------------------------------------------------------------------ */

void oracle_softmax_bwd_row(const double *y, const double *dy, int64_t n, double *dx) {
    nsum_t S = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&S, y[i] * dy[i]);
    double s = nsum_get(&S);
    for (int64_t i = 0; i < n; ++i) dx[i] = y[i] * (dy[i] - s);
}

void oracle_layernorm_bwd_row(const double *x, const double *dy, int64_t n, const double *gamma,
                              double mean, double rstd, double *dx) {
    nsum_t A = {0, 0}, B = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double g = dy[i] * (gamma ? gamma[i] : 1.0);
        double xh = (x[i] - mean) * rstd;
        nsum_add(&A, g);
        nsum_add(&B, g * xh);
    }
    double a = nsum_get(&A) / (double)n, b = nsum_get(&B) / (double)n;
    for (int64_t i = 0; i < n; ++i) {
        double g = dy[i] * (gamma ? gamma[i] : 1.0);
        double xh = (x[i] - mean) * rstd;
        dx[i] = rstd * (g - a - xh * b);
    }
}

void oracle_rmsnorm_bwd_row(const double *x, const double *dy, int64_t n, const double *gamma,
                            double rstd, double *dx) {
    nsum_t B = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&B, dy[i] * (gamma ? gamma[i] : 1.0) * x[i] * rstd);
    double b = nsum_get(&B) / (double)n;
    for (int64_t i = 0; i < n; ++i) {
        double g = dy[i] * (gamma ? gamma[i] : 1.0);
        dx[i] = rstd * (g - x[i] * rstd * b);
    }
}

/* Gradients with respect to the logits z of a softmax (the "softmax-logits */
/* backward" workload of Sec. IV-A), where y = softmax(z) is recomputed    */
/* from z rather than read:                                               */
/*   through the softmax, given dy:   dz_i = y_i (dy_i - sum_j y_j dy_j)   */
/*   of the cross entropy L = -sum_j t_j log y_j with target weights t    */
/*   (soft labels), times a per-row upstream scale w:                     */
/*                                    dz_i = w (y_i sum_j t_j - t_i)      */
/* (dL/dz_k = -sum_i t_i (delta_ik - y_k)).                               */
void oracle_softmax_logits_bwd_row(const double *z, const double *dy, int64_t n, double *dz) {
    double *y = (double *)malloc((size_t)n * sizeof(double));
    if (!y) { for (int64_t i = 0; i < n; ++i) dz[i] = NAN; return; }
    oracle_softmax_row(z, n, y);
    oracle_softmax_bwd_row(y, dy, n, dz);
    free(y);
}

void oracle_xent_bwd_row(const double *z, const double *t, int64_t n, double w, double *dz) {
    oracle_softmax_row(z, n, dz);
    nsum_t T = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&T, t[i]);
    double tt = nsum_get(&T);
    for (int64_t i = 0; i < n; ++i) dz[i] = w * (dz[i] * tt - t[i]);
}

/* Two-input statistics and their gradients (the "weighted-variance      */
/* backward" and "Pearson-correlation backward" workloads of Sec. IV-A). */
/* Weighted variance of x with weights w:                                 */
/*   W = sum w, mu = sum w x / W, v = sum w (x - mu)^2 / W;               */
/*   given the upstream gradient g of v:                                  */
/*   dx_i = g 2 w_i (x_i - mu) / W,   dw_i = g ((x_i - mu)^2 - v) / W     */
/*   (the mean's own terms vanish because sum w (x - mu) = 0).            */
/* Pearson correlation of x and y with centred sums                       */
/*   Sxy = sum (x - xb)(y - yb), Sxx = sum (x - xb)^2, Syy likewise:      */
/*   r = Sxy / sqrt(Sxx Syy);  given the upstream gradient g of r:        */
/*   dx_i = g ((y_i - yb) / sqrt(Sxx Syy) - r (x_i - xb) / Sxx), dy_i     */
/*   symmetrically (the means' own terms vanish because the centred       */
/*   values sum to zero).                                                 */
double oracle_wvar_row(const double *x, const double *w, int64_t n) {
    nsum_t W = {0, 0}, A = {0, 0};
    for (int64_t i = 0; i < n; ++i) { nsum_add(&W, w[i]); nsum_add(&A, w[i] * x[i]); }
    double ww = nsum_get(&W), mu = nsum_get(&A) / ww;
    nsum_t V = {0, 0};
    for (int64_t i = 0; i < n; ++i) { double d = x[i] - mu; nsum_add(&V, w[i] * d * d); }
    return nsum_get(&V) / ww;
}

void oracle_wvar_bwd_row(const double *x, const double *w, int64_t n, double g, double *dx, double *dw) {
    nsum_t W = {0, 0}, A = {0, 0};
    for (int64_t i = 0; i < n; ++i) { nsum_add(&W, w[i]); nsum_add(&A, w[i] * x[i]); }
    double ww = nsum_get(&W), mu = nsum_get(&A) / ww;
    nsum_t V = {0, 0};
    for (int64_t i = 0; i < n; ++i) { double d = x[i] - mu; nsum_add(&V, w[i] * d * d); }
    double v = nsum_get(&V) / ww;
    for (int64_t i = 0; i < n; ++i) {
        double d = x[i] - mu;
        dx[i] = g * 2.0 * w[i] * d / ww;
        dw[i] = g * (d * d - v) / ww;
    }
}

static void pearson_sums(const double *x, const double *y, int64_t n, double *xb, double *yb, double *sxx,
                         double *syy, double *sxy) {
    nsum_t X = {0, 0}, Y = {0, 0};
    for (int64_t i = 0; i < n; ++i) { nsum_add(&X, x[i]); nsum_add(&Y, y[i]); }
    *xb = nsum_get(&X) / (double)n;
    *yb = nsum_get(&Y) / (double)n;
    nsum_t A = {0, 0}, B = {0, 0}, C = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double dxv = x[i] - *xb, dyv = y[i] - *yb;
        nsum_add(&A, dxv * dxv);
        nsum_add(&B, dyv * dyv);
        nsum_add(&C, dxv * dyv);
    }
    *sxx = nsum_get(&A);
    *syy = nsum_get(&B);
    *sxy = nsum_get(&C);
}

double oracle_pearson_row(const double *x, const double *y, int64_t n) {
    double xb, yb, sxx, syy, sxy;
    pearson_sums(x, y, n, &xb, &yb, &sxx, &syy, &sxy);
    return sxy / sqrt(sxx * syy);
}

void oracle_pearson_bwd_row(const double *x, const double *y, int64_t n, double g, double *dx, double *dy) {
    double xb, yb, sxx, syy, sxy;
    pearson_sums(x, y, n, &xb, &yb, &sxx, &syy, &sxy);
    double den = sqrt(sxx * syy), r = sxy / den;
    for (int64_t i = 0; i < n; ++i) {
        double cx = x[i] - xb, cy = y[i] - yb;
        dx[i] = g * (cy / den - r * cx / sxx);
        dy[i] = g * (cx / den - r * cy / syy);
    }
}

/* Row-wise int8 quantisation (the "row-wise int8 quantization" workload */
/* of Sec. IV-A): s = amax_i |x_i| / 127 (1 for an all-zero row) and     */
/* q_i = the integer nearest to x_i / s (ties to even), clamped to       */
/* [-127, 127].  The quotients are taken in FP32 as a kernel takes them: */
/* s = fl32(amax / 127) and fl32(x_i / s), each computed in double and   */
/* rounded once to FP32, which equals the correctly rounded FP32         */
/* quotient (53 >= 2 * 24 + 2 bits, so the double rounding is harmless). */
/* Returns s; q receives the codes.                                      */
float oracle_quant_int8_row(const float *x, int64_t n, int8_t *q) {
    double amax = 0.0;
    for (int64_t i = 0; i < n; ++i) { double a = fabs((double)x[i]); amax = a > amax ? a : amax; }
    float s = amax > 0.0 ? (float)(amax / 127.0) : 1.0f;
    for (int64_t i = 0; i < n; ++i) {
        float r = (float)((double)x[i] / (double)s);
        double k = nearbyint((double)r);   /* default rounding mode: ties to even */
        if (k > 127.0) k = 127.0;
        if (k < -127.0) k = -127.0;
        q[i] = (int8_t)k;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Negative controls of the screening rule (Sec. III-D; Sec. IV-C): row  */
/* ops that read and write a row once but lack the reduction-reuse       */
/* pattern, so the rule rejects the cluster path for them.               */
/* Row scan (inclusive prefix sum): y_i = sum_{j <= i} x_j, the running  */
/* sum kept with Neumaier compensation.                                  */
void oracle_scan_row(const double *x, int64_t n, double *y) {
    nsum_t S = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        nsum_add(&S, x[i]);
        y[i] = nsum_get(&S);
    }
}

/* Row stencil of radius r: y_i = sum_{k=-r..r} w[k + r] x_{i+k}, with    */
/* x_j = 0 outside the row (zero padding at both ends).                   */
void oracle_stencil_row(const double *x, int64_t n, const double *w, int r, double *y) {
    for (int64_t i = 0; i < n; ++i) {
        nsum_t S = {0, 0};
        for (int k = -r; k <= r; ++k) {
            int64_t j = i + k;
            if (j >= 0 && j < n) nsum_add(&S, w[k + r] * x[j]);
        }
        y[i] = nsum_get(&S);
    }
}

/* ------------------------------------------------------------------ */
/* Batch driver: decode -> op -> (exact doubles, encoded output)        */
/* ------------------------------------------------------------------ */

static double decode_one(const void *base, int dtype, int64_t idx) {
    switch (dtype) {
    case OR_F32:  return (double)((const float *)base)[idx];
    case OR_BF16: return oracle_bf16_to_double(((const uint16_t *)base)[idx]);
    default:      return oracle_e4m3_to_double(((const uint8_t *)base)[idx]);
    }
}

static void *malloc_row(int64_t n) { return malloc((size_t)n * sizeof(double)); }
static void free_row(void *p) { free(p); }

static int dtype_size(int dtype) { return dtype == OR_F32 ? 4 : (dtype == OR_BF16 ? 2 : 1); }

/* Decode `rows` rows of `cols` elements (row stride ld elements) to doubles.
 * For E4M3 input the per-row FP32 scale multiplies the decoded code. */
void oracle_decode(int dtype, const void *in, const float *in_scale, int64_t rows,
                   int64_t cols, int64_t ld, double *x) {
    for (int64_t r = 0; r < rows; ++r) {
        const char *row = (const char *)in + r * ld * dtype_size(dtype);
        double sc = (dtype == OR_E4M3 && in_scale) ? (double)in_scale[r] : 1.0;
        for (int64_t i = 0; i < cols; ++i) x[r * cols + i] = decode_one(row, dtype, i) * sc;
    }
}

/*
 * Full batch.  y64 (may be NULL) receives the exact result: rows*cols doubles,
 * or `rows` doubles for logsumexp.  out (may be NULL) receives the result
 * rounded to out_dtype with row stride ld_out; for E4M3 output out_scale gets
 * the per-row scale (amax/448, or 1 for an all-zero row).  Logsumexp always
 * writes FP32.  nthreads <= 0 uses the OpenMP default.  Returns 0, or -1 on a
 * bad argument.
 */
int oracle_run(int op, int in_dtype, int out_dtype, const void *in,
               const float *in_scale, int64_t rows, int64_t cols, int64_t ld_in,
               const float *gamma, const float *beta, double eps, double *y64,
               void *out, int64_t ld_out, float *out_scale, int nthreads) {
    if (rows < 0 || cols <= 0 || !in) return -1;
    if (op < 0 || op > 3 || in_dtype < 0 || in_dtype > 2 || out_dtype < 0 || out_dtype > 2) return -1;
    if (ld_in <= 0) ld_in = cols;
    if (ld_out <= 0) ld_out = cols;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int bad = 0;
#pragma omp parallel
    {
        double *x = (double *)malloc_row(cols);
        double *y = (double *)malloc_row(cols);
        double *g = gamma ? (double *)malloc_row(cols) : NULL;
        double *b = beta ? (double *)malloc_row(cols) : NULL;
        if (!x || !y || (gamma && !g) || (beta && !b)) {
#pragma omp atomic write
            bad = 1;
        } else {
            if (g) for (int64_t i = 0; i < cols; ++i) g[i] = (double)gamma[i];
            if (b) for (int64_t i = 0; i < cols; ++i) b[i] = (double)beta[i];
#pragma omp for schedule(dynamic, 1)
            for (int64_t r = 0; r < rows; ++r) {
                const char *row = (const char *)in + r * ld_in * dtype_size(in_dtype);
                double sc = (in_dtype == OR_E4M3 && in_scale) ? (double)in_scale[r] : 1.0;
                for (int64_t i = 0; i < cols; ++i) x[i] = decode_one(row, in_dtype, i) * sc;
                if (op == OR_LOGSUMEXP) {
                    double v = oracle_lse_row(x, cols);
                    if (y64) y64[r] = v;
                    if (out) ((float *)out)[r] = (float)v;
                    continue;
                }
                if (op == OR_SOFTMAX) oracle_softmax_row(x, cols, y);
                else if (op == OR_LAYERNORM) oracle_layernorm_row(x, cols, g, b, eps, y);
                else oracle_rmsnorm_row(x, cols, g, eps, y);
                if (y64) memcpy(y64 + r * cols, y, (size_t)cols * sizeof(double));
                if (!out) continue;
                char *orow = (char *)out + r * ld_out * dtype_size(out_dtype);
                if (out_dtype == OR_F32) {
                    for (int64_t i = 0; i < cols; ++i) ((float *)orow)[i] = (float)y[i];
                } else if (out_dtype == OR_BF16) {
                    for (int64_t i = 0; i < cols; ++i) ((uint16_t *)orow)[i] = oracle_double_to_bf16(y[i]);
                } else {
                    double amax = 0.0;
                    for (int64_t i = 0; i < cols; ++i) amax = fabs(y[i]) > amax ? fabs(y[i]) : amax;
                    double s = amax > 0.0 ? amax / 448.0 : 1.0;
                    if (out_scale) out_scale[r] = (float)s;
                    for (int64_t i = 0; i < cols; ++i) ((uint8_t *)orow)[i] = oracle_double_to_e4m3_sat(y[i] / s);
                }
            }
        }
        free_row(x); free_row(y); free_row(g); free_row(b);
    }
    return bad ? -1 : 0;
}

/*
 * Backward batch.  op: 0 softmax, 2 layernorm, 3 rmsnorm (the forward op's
 * code), 7 softmax from logits, 8 cross entropy from logits.  a (softmax:
 * the forward output y; norms: the forward input x; 7 and 8: the logits z)
 * and dy (8: the target weights t) hold rows x cols elements of dtype (F32
 * or BF16) with row stride ld; gamma (cols FP32, NULL = 1), mean (rows FP32,
 * layernorm) and rstd (rows FP32, norms; for 8 the per-row upstream scale w,
 * NULL = 1) are decoded exactly.  dx64 (may be NULL) receives the exact
 * rows*cols result, dx (may be NULL) the result rounded to dtype with row
 * stride ld.  Returns 0, or -1 on a bad argument.
 */
int oracle_run_bwd(int op, int dtype, const void *a, const void *dy, int64_t rows, int64_t cols, int64_t ld,
                   const float *gamma, const float *mean, const float *rstd, double *dx64, void *dx,
                   int nthreads) {
    if (rows < 0 || cols <= 0 || !a || !dy) return -1;
    if (!(op == OR_SOFTMAX || op == OR_LAYERNORM || op == OR_RMSNORM || op == OR_SOFTMAX_LOGITS ||
          op == OR_XENT) || dtype < 0 || dtype > 1)
        return -1;
    if (op == OR_LAYERNORM && (!mean || !rstd)) return -1;
    if (op == OR_RMSNORM && !rstd) return -1;
    if (ld <= 0) ld = cols;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int bad = 0;
#pragma omp parallel
    {
        double *x = (double *)malloc_row(cols);
        double *d = (double *)malloc_row(cols);
        double *o = (double *)malloc_row(cols);
        double *g = gamma ? (double *)malloc_row(cols) : NULL;
        if (!x || !d || !o || (gamma && !g)) {
#pragma omp atomic write
            bad = 1;
        } else {
            if (g) for (int64_t i = 0; i < cols; ++i) g[i] = (double)gamma[i];
#pragma omp for schedule(dynamic, 1)
            for (int64_t r = 0; r < rows; ++r) {
                const char *ar = (const char *)a + r * ld * dtype_size(dtype);
                const char *dr = (const char *)dy + r * ld * dtype_size(dtype);
                for (int64_t i = 0; i < cols; ++i) {
                    x[i] = decode_one(ar, dtype, i);
                    d[i] = decode_one(dr, dtype, i);
                }
                if (op == OR_SOFTMAX) oracle_softmax_bwd_row(x, d, cols, o);
                else if (op == OR_SOFTMAX_LOGITS) oracle_softmax_logits_bwd_row(x, d, cols, o);
                else if (op == OR_XENT) oracle_xent_bwd_row(x, d, cols, rstd ? (double)rstd[r] : 1.0, o);
                else if (op == OR_LAYERNORM)
                    oracle_layernorm_bwd_row(x, d, cols, g, (double)mean[r], (double)rstd[r], o);
                else oracle_rmsnorm_bwd_row(x, d, cols, g, (double)rstd[r], o);
                if (dx64) memcpy(dx64 + r * cols, o, (size_t)cols * sizeof(double));
                if (!dx) continue;
                char *orow = (char *)dx + r * ld * dtype_size(dtype);
                if (dtype == OR_F32) {
                    for (int64_t i = 0; i < cols; ++i) ((float *)orow)[i] = (float)o[i];
                } else {
                    for (int64_t i = 0; i < cols; ++i) ((uint16_t *)orow)[i] = oracle_double_to_bf16(o[i]);
                }
            }
        }
        free_row(x); free_row(d); free_row(o); free_row(g);
    }
    return bad ? -1 : 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
