/*
 * dsfft_oracle.c — CPU oracle for the dual-select FMA radix-2 FFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * It is deliberately plain and slow: every floating-point step is written out
 * in the order the paper states it, and every rounding to FP32/FP16/BF16 is a
 * single correctly rounded (round-to-nearest-even) operation, emulated in FP64.
 *
 * Contents (paper references are to "Dual-Select FMA Butterfly for FFT"):
 *   orc_round      — RN-even rounding of an FP64 value to FP32/FP16/BF16.
 *   orc_fma/orc_mul— correctly rounded fused multiply-add / multiply in those
 *                    formats (exact product, TwoSum, round-to-odd in FP64,
 *                    then one RN-even rounding: Boldo & Melquiond, "Emulation
 *                    of FMA and correctly rounded sums: proved algorithms using
 *                    rounding to odd", IEEE Trans. Computers 57(4), 2008).
 *   orc_dft        — direct DFT in FP64, W = exp(-j 2 pi k/N) (Eq. 1 sign).
 *   orc_fft_fp64   — radix-2 Stockham FFT in FP64 with the 10-op butterfly of
 *                    Eqs. 2-3 (m = log2 N passes, Section IV).
 *   orc_table      — twiddle table of Algorithm 1 (dual-select), of the
 *                    Linzer-Feig factorization (Eqs. 4-6, ratio cot, with the
 *                    epsilon clamp of Section I) and of the cosine
 *                    factorization (Eqs. 7-9, ratio tan); FP64 arithmetic,
 *                    then the ratio and multiplier rounded once.
 *   orc_emulate_fft— the m-pass Stockham FFT whose butterflies are the 6-FMA
 *                    forms of Eqs. 4-9, branching on the table flag as the
 *                    Implementation paragraph of Section III describes, each
 *                    FMA rounded once in the target format.
 *   orc_table_range— the same table rules for any k in [0, count) (the
 *                    radix-4 passes need W^k for k < 3N/4).
 *   orc_emulate_fft_r4 — the radix-4 extension the Discussion proposes
 *                    (dual-select in radix-4 passes): radix-4 Stockham DIT
 *                    passes, preceded by one radix-2 pass when log2 N is odd,
 *                    each of the three twiddle products in the 6-FMA form of
 *                    its own table entry; the operation sequence is spelled
 *                    out at orc_emulate_fft_r4.
 *
 * Readings where the paper is silent or misprinted:
 *   - Eq. 4 prints s2 = (w_r/w_i) b_r + b_i; that does not reproduce Eq. 2
 *     (s2 * w_i must equal w_i b_r + w_r b_i).  The sine path here uses
 *     s2 = b_r + (w_r/w_i) b_i.  The tests show the printed form fails.
 *   - Ties |w_r| == |w_i| go to the cosine path (Algorithm 1 uses >=).
 *   - theta = (-2 pi k)/N evaluated in FP64 exactly in that order.
 *   - Linzer-Feig clamp: if |w_i| < eps then w_i := -eps (forward sign).
 *   - Inverse transform: conjugate twiddles (w_i -> -w_i), taken exactly
 *     from the forward FP64 values before rounding.
 *   - Optional exact x0.5 per pass: a' = RN(0.5 a), multiplier stored as
 *     RN(m/2); A = a' + m' u, B = a' - m' u.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_FP64 = 0, ORC_FP32 = 1, ORC_FP16 = 2, ORC_BF16 = 3 };
enum { ORC_LF = 0, ORC_COS = 1, ORC_DS = 2 };
enum { ORC_PATH_COS = 0, ORC_PATH_SIN = 1 };

/* significand bits p (with hidden bit), minimum normal exponent, maximum
 * exponent of each binary format */
static int fmt_params(int fmt, int *p, int *emin, int *emax) {
    switch (fmt) {
    case ORC_FP32: *p = 24; *emin = -126; *emax = 127; return 0;
    case ORC_FP16: *p = 11; *emin = -14;  *emax = 15;  return 0;
    case ORC_BF16: *p = 8;  *emin = -126; *emax = 127; return 0;
    default: return -1;
    }
}

/* Round x (any double) to the nearest value of the format, ties to even,
 * with gradual underflow and overflow to infinity.  FP64 is the identity. */
double orc_round(double x, int fmt) {
    int p, emin, emax;
    if (fmt == ORC_FP64) return x;
    if (fmt_params(fmt, &p, &emin, &emax) != 0) return NAN;
    if (isnan(x) || isinf(x) || x == 0.0) return x;
    int e;
    frexp(x, &e);              /* |x| = f * 2^e, 0.5 <= f < 1 */
    int lead = e - 1;          /* exponent of the leading bit */
    if (lead < emin) lead = emin;   /* subnormal range: fixed quantum */
    double q = ldexp(1.0, lead - (p - 1));
    double r = nearbyint(x / q) * q;     /* x / q is exact */
    double maxv = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
    if (fabs(r) > maxv) return copysign(INFINITY, x);
    return r;
}

/* round-to-odd of the exact sum s + e (s = fl(s+e)) in FP64 */
static double round_to_odd(double s, double e) {
    if (e == 0.0 || !isfinite(s)) return s;
    uint64_t bits;
    memcpy(&bits, &s, sizeof bits);
    if (bits & 1u) return s;                      /* already odd */
    return nextafter(s, e > 0.0 ? INFINITY : -INFINITY);
}

/* Correctly rounded a*b + c in the format.  a, b, c must be values of the
 * format (then a*b is exact in FP64). */
double orc_fma(double a, double b, double c, int fmt) {
    if (fmt == ORC_FP64) return fma(a, b, c);
    double prod = a * b;          /* exact for FP32/FP16/BF16 operands */
    if (!isfinite(prod) || !isfinite(c)) return orc_round(prod + c, fmt);
    /* TwoSum (Knuth): s + err == prod + c exactly */
    double s = prod + c;
    double bb = s - prod;
    double err = (prod - (s - bb)) + (c - bb);
    if (!isfinite(s)) return orc_round(s, fmt);
    return orc_round(round_to_odd(s, err), fmt);
}

/* Correctly rounded a*b (exact in FP64, then one rounding). */
double orc_mul(double a, double b, int fmt) {
    return orc_round(a * b, fmt);
}

/* ---------------------------------------------------------------------- */
/* Direct DFT, Eq. 1 convention: X[k] = sum_n x[n] exp(sign * j 2 pi kn/N),
 * sign = -1 forward.  The angle uses (k*n mod N) so it stays in [0, 2 pi).
 * x, X: interleaved (re, im), length 2N. */
void orc_dft(int64_t N, const double *x, double *X, int sign) {
    double *c = (double *)malloc(sizeof(double) * (size_t)N);
    double *s = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t r = 0; r < N; r++) {
        double th = (2.0 * M_PI * (double)r) / (double)N;
        c[r] = cos(th);
        s[r] = (double)sign * sin(th);
    }
    for (int64_t k = 0; k < N; k++) {
        double acc_r = 0.0, acc_i = 0.0;
        for (int64_t n = 0; n < N; n++) {
            int64_t r = (int64_t)(((unsigned __int128)k * (unsigned __int128)n) % (unsigned __int128)N);
            double xr = x[2 * n], xi = x[2 * n + 1];
            acc_r += xr * c[r] - xi * s[r];
            acc_i += xr * s[r] + xi * c[r];
        }
        X[2 * k] = acc_r;
        X[2 * k + 1] = acc_i;
    }
    free(c);
    free(s);
}

/* One DFT output bin X[k] of one transform (for sampled checks). */
void orc_dft_bin(int64_t N, const double *x, int64_t k, int sign, double *out2) {
    double acc_r = 0.0, acc_i = 0.0;
    for (int64_t n = 0; n < N; n++) {
        int64_t r = (int64_t)(((unsigned __int128)k * (unsigned __int128)n) % (unsigned __int128)N);
        double th = (2.0 * M_PI * (double)r) / (double)N;
        double cr = cos(th), si = (double)sign * sin(th);
        acc_r += x[2 * n] * cr - x[2 * n + 1] * si;
        acc_i += x[2 * n] * si + x[2 * n + 1] * cr;
    }
    out2[0] = acc_r;
    out2[1] = acc_i;
}

/* ---------------------------------------------------------------------- */
/* Radix-2 Stockham FFT in FP64 (Section IV: m = log2 N passes).  Pass with
 * half-span L: for s in [0, N/2L), j in [0, L):
 *   a = Z[sL + j], b = Z[N/2 + sL + j], W = exp(sign j 2 pi j/(2L))
 *   Y[2sL + j] = a + W b,  Y[2sL + L + j] = a - W b        (Eq. 1)
 * computed with the 10-operation real form of Eqs. 2-3.  Batch-contiguous
 * interleaved data; in and out may alias. */
void orc_fft_fp64(int64_t N, const double *x, double *y, int64_t batch, int sign) {
    double *Z = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *Y = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int64_t bi = 0; bi < batch; bi++) {
        memcpy(Z, x + 2 * N * bi, sizeof(double) * 2 * (size_t)N);
        for (int64_t L = 1; L < N; L *= 2) {
            for (int64_t s = 0; s < N / (2 * L); s++) {
                for (int64_t j = 0; j < L; j++) {
                    int64_t k = j * (N / (2 * L));
                    double th = (-2.0 * M_PI * (double)k) / (double)N;
                    double wr = cos(th), wi = sin(th);
                    if (sign > 0) wi = -wi;
                    double ar = Z[2 * (s * L + j)], ai = Z[2 * (s * L + j) + 1];
                    double br = Z[2 * (N / 2 + s * L + j)], bi2 = Z[2 * (N / 2 + s * L + j) + 1];
                    double pr = wr * br - wi * bi2;   /* Eq. 2 */
                    double pi = wi * br + wr * bi2;
                    Y[2 * (2 * s * L + j)] = ar + pr;
                    Y[2 * (2 * s * L + j) + 1] = ai + pi;
                    Y[2 * (2 * s * L + L + j)] = ar - pr;   /* Eq. 3 */
                    Y[2 * (2 * s * L + L + j) + 1] = ai - pi;
                }
            }
            double *tmp = Z; Z = Y; Y = tmp;
        }
        memcpy(y + 2 * N * bi, Z, sizeof(double) * 2 * (size_t)N);
    }
    free(Z);
    free(Y);
}

/* ---------------------------------------------------------------------- */
/* Twiddle table for a factorization, FP64 arithmetic then one rounding.
 *   ORC_DS : Algorithm 1 — cosine path (m = w_r, t = w_i/w_r) when
 *            |w_r| >= |w_i|, else sine path (m = w_i, t = w_r/w_i).
 *   ORC_LF : Eqs. 4-6 — sine path everywhere; w_i clamped to -eps when
 *            |w_i| < eps (Section I: clamp to a small epsilon).
 *   ORC_COS: Eqs. 7-9 — cosine path everywhere (t = tan theta).
 * dir > 0 conjugates the twiddles (w_i -> -w_i) after the clamp; scaled
 * stores the multiplier as RN(m/2).  Outputs: t, m as the rounded values in
 * double, path as ORC_PATH_COS / ORC_PATH_SIN. */
void orc_table_range(int64_t N, int64_t count, int fac, double eps, int dir, int fmt, double mscale,
                     double *t, double *m, int32_t *path) {
    for (int64_t k = 0; k < count; k++) {
        double th = (-2.0 * M_PI * (double)k) / (double)N;
        double wr = cos(th), wi = sin(th);
        int use_cos;
        if (fac == ORC_DS) {
            use_cos = fabs(wr) >= fabs(wi);
        } else if (fac == ORC_LF) {
            use_cos = 0;
            if (fabs(wi) < eps) wi = -eps;
        } else {
            use_cos = 1;
        }
        if (dir > 0) wi = -wi;
        double tt, mm;
        if (use_cos) { mm = wr; tt = wi / wr; }
        else         { mm = wi; tt = wr / wi; }
        mm = mm * mscale;     /* a power of two: exact */
        t[k] = orc_round(tt, fmt);
        m[k] = orc_round(mm, fmt);
        path[k] = use_cos ? ORC_PATH_COS : ORC_PATH_SIN;
    }
}

/* Algorithm 1 (or Eqs. 4-6 / 7-9) for k in [0, N/2); the multiplier is
 * halved (x0.5 per pass) when `scaled`. */
void orc_table(int64_t N, int fac, double eps, int dir, int fmt, int scaled,
               double *t, double *m, int32_t *path) {
    orc_table_range(N, N / 2, fac, eps, dir, fmt, scaled ? 0.5 : 1.0, t, m, path);
}

/* One butterfly, in the paper's branched form.  Inputs a, b are values of
 * the format; (t, m, path) a rounded table entry.  Writes A, B. */
static void butterfly(int fmt, int scaled, double t, double m, int path,
                      const double a[2], const double b[2], double A[2], double B[2]) {
    double ar = a[0], ai = a[1], br = b[0], bi = b[1];
    if (scaled) {
        ar = orc_mul(ar, 0.5, fmt);
        ai = orc_mul(ai, 0.5, fmt);
    }
    if (path == ORC_PATH_COS) {
        /* Eq. 7: s1 = b_r - t b_i, s2 = t b_r + b_i (t = w_i/w_r) */
        double s1 = orc_fma(-t, bi, br, fmt);
        double s2 = orc_fma(t, br, bi, fmt);
        /* Eqs. 8-9: A = a + s w_r, B = a - s w_r */
        A[0] = orc_fma(s1, m, ar, fmt);
        A[1] = orc_fma(s2, m, ai, fmt);
        B[0] = orc_fma(-s1, m, ar, fmt);
        B[1] = orc_fma(-s2, m, ai, fmt);
    } else {
        /* Eq. 4 with the corrected s2: s1 = b_i - t b_r, s2 = b_r + t b_i
         * (t = w_r/w_i) */
        double s1 = orc_fma(-t, br, bi, fmt);
        double s2 = orc_fma(t, bi, br, fmt);
        /* Eqs. 5-6: A_r = a_r - s1 w_i, A_i = a_i + s2 w_i, B the opposite */
        A[0] = orc_fma(-s1, m, ar, fmt);
        A[1] = orc_fma(s2, m, ai, fmt);
        B[0] = orc_fma(s1, m, ar, fmt);
        B[1] = orc_fma(-s2, m, ai, fmt);
    }
}

/* Exported single butterfly (for the identity tests). */
void orc_butterfly(int fmt, int scaled, double t, double m, int path,
                   const double *a, const double *b, double *A, double *B) {
    butterfly(fmt, scaled, t, m, path, a, b, A, B);
}

/* The m-pass radix-2 Stockham FFT with 6-FMA butterflies, each operation
 * rounded once in the format.  The table (t, m, path) has N/2 entries indexed
 * by k = j * N/(2L) for the butterfly (s, j) of the pass with half-span L.
 * x, y: batch-contiguous interleaved values of the format held in doubles. */
void orc_emulate_fft(int64_t N, int fmt, int scaled,
                     const double *t, const double *m, const int32_t *path,
                     const double *x, double *y, int64_t batch) {
    double *Z = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *Y = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int64_t bi = 0; bi < batch; bi++) {
        memcpy(Z, x + 2 * N * bi, sizeof(double) * 2 * (size_t)N);
        for (int64_t L = 1; L < N; L *= 2) {
            for (int64_t s = 0; s < N / (2 * L); s++) {
                for (int64_t j = 0; j < L; j++) {
                    int64_t k = j * (N / (2 * L));
                    double A[2], B[2];
                    butterfly(fmt, scaled, t[k], m[k], path[k],
                              &Z[2 * (s * L + j)], &Z[2 * (N / 2 + s * L + j)], A, B);
                    Y[2 * (2 * s * L + j)] = A[0];
                    Y[2 * (2 * s * L + j) + 1] = A[1];
                    Y[2 * (2 * s * L + L + j)] = B[0];
                    Y[2 * (2 * s * L + L + j) + 1] = B[1];
                }
            }
            double *tmp = Z; Z = Y; Y = tmp;
        }
        memcpy(y + 2 * N * bi, Z, sizeof(double) * 2 * (size_t)N);
    }
    free(Z);
    free(Y);
}

/* ---------------------------------------------------------------------- */
/* Radix-4 extension.  The paper's Discussion proposes applying the
 * dual-select choice to radix-4 passes, each twiddle product taking the form
 * of its own table entry; it gives no operation order, so this is the
 * definition the library implements (and this emulation checks):
 *
 * Pass with span L (sub-transforms of length L done): for s in [0, N/4L),
 * j in [0, L), inputs a_q = Z[q N/4 + s L + j] (q = 0..3), table entries
 * e_q = T4[q j N/(4L)] for W_4L^(q j), outputs
 *   Y[4 s L + p L + j] = sum_q W_4L^(q j) a_q (-/+ i)^(q p)   (forward -i).
 * Operations (each one correctly rounded in the format):
 *   (s1_q, s2_q) = Eq. 7 (cosine entry) or Eq. 4 corrected (sine entry) of
 *                  b = a_q with the entry's ratio t_q,      q = 1, 2, 3
 *   mr_q = m_q (cosine) or -m_q (sine): W a_q = (mr_q s1_q, m_q s2_q)
 *   [scaled: a_0 <- RN(a_0 / 4); the table multipliers are RN(m / 4)]
 *   b3 = (RN(mr_3 s1_3), RN(m_3 s2_3))
 *   c0 = (fma( mr_2, s1_2, a0r), fma( m_2, s2_2, a0i))      a0 + W^2j a2
 *   c1 = (fma(-mr_2, s1_2, a0r), fma(-m_2, s2_2, a0i))      a0 - W^2j a2
 *   c2 = (fma( mr_1, s1_1, b3r), fma( m_1, s2_1, b3i))      W^j a1 + b3
 *   d3 = (fma(-mr_1, s1_1, b3r), fma(-m_1, s2_1, b3i))      b3 - W^j a1
 *   y0 = c0 + c2, y2 = c0 - c2 (componentwise RN sums)
 *   forward: y1 = c1 + i d3 = (RN(c1r - d3i), RN(c1i + d3r)),
 *            y3 = c1 - i d3 = (RN(c1r + d3i), RN(c1i - d3r));
 *   inverse: y1 and y3 exchanged (W_4 = +i).
 * Passes: spans L = 1, 4, 16, ... when log2 N is even; when it is odd, a
 * radix-2 pass with span 1 first (the butterfly of orc_emulate_fft with the
 * radix-2 entry k = 0, W^0), then spans 2, 8, 32, ....  Scaled transforms
 * therefore divide by 4 per radix-4 pass and 2 in the radix-2 pass: DFT/N. */

/* the pair (s1, s2) of Eq. 7 (cosine) or Eq. 4 with corrected s2 (sine) */
static void pre_products(int fmt, double t, int path, const double b[2], double *s1, double *s2) {
    if (path == ORC_PATH_COS) {
        *s1 = orc_fma(-t, b[1], b[0], fmt);
        *s2 = orc_fma(t, b[0], b[1], fmt);
    } else {
        *s1 = orc_fma(-t, b[0], b[1], fmt);
        *s2 = orc_fma(t, b[1], b[0], fmt);
    }
}

static void butterfly4(int fmt, int scaled, int inverse, const double *t, const double *m, const int32_t *path,
                       const int64_t k[4], const double *a0, const double *a1, const double *a2, const double *a3,
                       double y[4][2]) {
    double s1[4], s2[4], mr[4], mi[4];
    const double *a[4] = {a0, a1, a2, a3};
    for (int q = 1; q < 4; q++) {
        pre_products(fmt, t[k[q]], path[k[q]], a[q], &s1[q], &s2[q]);
        mi[q] = m[k[q]];
        mr[q] = path[k[q]] == ORC_PATH_COS ? m[k[q]] : -m[k[q]];
    }
    double x0r = a0[0], x0i = a0[1];
    if (scaled) {
        x0r = orc_mul(x0r, 0.25, fmt);
        x0i = orc_mul(x0i, 0.25, fmt);
    }
    double b3r = orc_mul(mr[3], s1[3], fmt), b3i = orc_mul(mi[3], s2[3], fmt);
    double c0r = orc_fma(mr[2], s1[2], x0r, fmt), c0i = orc_fma(mi[2], s2[2], x0i, fmt);
    double c1r = orc_fma(-mr[2], s1[2], x0r, fmt), c1i = orc_fma(-mi[2], s2[2], x0i, fmt);
    double c2r = orc_fma(mr[1], s1[1], b3r, fmt), c2i = orc_fma(mi[1], s2[1], b3i, fmt);
    double d3r = orc_fma(-mr[1], s1[1], b3r, fmt), d3i = orc_fma(-mi[1], s2[1], b3i, fmt);
    y[0][0] = orc_fma(c2r, 1.0, c0r, fmt);
    y[0][1] = orc_fma(c2i, 1.0, c0i, fmt);
    y[2][0] = orc_fma(c2r, -1.0, c0r, fmt);
    y[2][1] = orc_fma(c2i, -1.0, c0i, fmt);
    double pr = orc_fma(d3i, -1.0, c1r, fmt), pi = orc_fma(d3r, 1.0, c1i, fmt);   /* c1 + i d3 */
    double nr = orc_fma(d3i, 1.0, c1r, fmt), ni = orc_fma(d3r, -1.0, c1i, fmt);   /* c1 - i d3 */
    int f = inverse ? 3 : 1, g = inverse ? 1 : 3;
    y[f][0] = pr; y[f][1] = pi;
    y[g][0] = nr; y[g][1] = ni;
}

/* The radix-4 (+ one radix-2) FFT defined above.  (t4, m4, path4): the
 * table for k in [0, 3N/4) with multipliers RN(m/4) when scaled (m unscaled
 * otherwise); (t0, m0, path0): the radix-2 entry k = 0 (multiplier RN(m/2)
 * when scaled) used by the radix-2 pass of odd log2 N. */
void orc_emulate_fft_r4(int64_t N, int fmt, int scaled, int inverse,
                        const double *t4, const double *m4, const int32_t *path4,
                        double t0, double m0, int32_t path0,
                        const double *x, double *y, int64_t batch) {
    double *Z = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *Y = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    int log2n = 0;
    while ((int64_t)1 << log2n < N) log2n++;
    for (int64_t bi = 0; bi < batch; bi++) {
        memcpy(Z, x + 2 * N * bi, sizeof(double) * 2 * (size_t)N);
        int64_t L = 1;
        if (log2n & 1) {
            /* radix-2 pass, span 1: a = Z[s], b = Z[N/2 + s] -> Y[2s], Y[2s + 1] */
            for (int64_t s = 0; s < N / 2; s++) {
                double A[2], B[2];
                butterfly(fmt, scaled, t0, m0, path0, &Z[2 * s], &Z[2 * (N / 2 + s)], A, B);
                Y[2 * (2 * s)] = A[0];
                Y[2 * (2 * s) + 1] = A[1];
                Y[2 * (2 * s + 1)] = B[0];
                Y[2 * (2 * s + 1) + 1] = B[1];
            }
            double *tmp = Z; Z = Y; Y = tmp;
            L = 2;
        }
        for (; L < N; L *= 4) {
            for (int64_t s = 0; s < N / (4 * L); s++) {
                for (int64_t j = 0; j < L; j++) {
                    int64_t k1 = j * (N / (4 * L));
                    int64_t k[4] = {0, k1, 2 * k1, 3 * k1};
                    double yv[4][2];
                    butterfly4(fmt, scaled, inverse, t4, m4, path4, k, &Z[2 * (s * L + j)],
                               &Z[2 * (N / 4 + s * L + j)], &Z[2 * (N / 2 + s * L + j)],
                               &Z[2 * (3 * N / 4 + s * L + j)], yv);
                    for (int p = 0; p < 4; p++) {
                        Y[2 * (4 * s * L + p * L + j)] = yv[p][0];
                        Y[2 * (4 * s * L + p * L + j) + 1] = yv[p][1];
                    }
                }
            }
            double *tmp = Z; Z = Y; Y = tmp;
        }
        memcpy(y + 2 * N * bi, Z, sizeof(double) * 2 * (size_t)N);
    }
    free(Z);
    free(Y);
}

/* Elementwise rounding of an array (used to make inputs of a format). */
void orc_round_array(const double *x, double *y, int64_t n, int fmt) {
    for (int64_t i = 0; i < n; i++) y[i] = orc_round(x[i], fmt);
}
