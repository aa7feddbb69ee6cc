/*
 * FP64 CPU oracle for 2-D image resampling (nearest, bilinear, bicubic).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this file; the library's CUDA path never does,
 * and this file shares no code, header or table with it.
 *
 * What it computes (the paper's Sec. II.B, Eqs. 1-5, extended to the two
 * interpolation kernels the paper names but does not define):
 *
 *   Per axis, output index j in [0, m) of a source axis of length n:
 *   1. Map (Eq. 1). The paper's x_p = x_f / scale with scale = m / n taken
 *      from the sizes, so x = j * n / m, held as the exact rational
 *      num / den (ASYMMETRIC). The half-pixel option maps pixel centres:
 *      x = (j + 1/2) * n / m - 1/2 = ((2j + 1) n - m) / (2 m). The
 *      align-corners option (an extension; the paper has one map) pins
 *      the first and last samples of both axes together:
 *      x = j (n - 1) / (m - 1), and x = 0 when m = 1.
 *   2. Base and fraction (Eqs. 2-4): i0 = floor(x), t = x - i0.
 *   3. Taps. nearest: i0 (ASYMMETRIC) or floor(x + 1/2) (HALF_PIXEL and
 *      ALIGN_CORNERS), weight
 *      1. bilinear: i0, i0+1 with weights 1-t, t (Eq. 5 with its second
 *      (1 - offsetY) read as (1 - offsetX)). bicubic: i0-1 .. i0+2 with
 *      weights K(t+1), K(t), K(1-t), K(2-t) for Keys' cubic convolution
 *      kernel K with parameter a (default -1/2).
 *   4. Border: every tap index is clamped to [0, n-1] (edge replicate).
 *   5. 2-D: Y[y,x,c] = sum_p sum_q wy_p wx_q X[iy_p, ix_q, c] in FP64.
 *   The adjoint is the transpose of that linear map: every output sample
 *   scatters w * dY into the input samples its clamped taps name.
 *
 * Storage rounding (applied by the oracle_quantize_* helpers): uint8 clamps
 * to [0, 255] then rounds half to even; FP16 / BF16 round to nearest even
 * directly from FP64; FP32 is the C cast (round to nearest even).
 *
 * Parity pins: every function here is checked by the CPU tests against
 * invariants and independent routines (identity, constants, ramps,
 * quadratics, interpolation of samples, the Catmull-Rom midpoint weights,
 * SciPy linear interpolation, PyTorch's half-pixel kernels, NumPy's FP16
 * rounding, the adjoint dot-product identity and finite differences).
 *
 * Build: gcc -O2 -ffp-contract=off [-fopenmp] -shared -fPIC -lm
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { M_NEAREST = 0, M_BILINEAR = 1, M_BICUBIC = 2 };
enum { C_ASYMMETRIC = 0, C_HALF_PIXEL = 1, C_ALIGN_CORNERS = 2 };

/* floor(num / den) for den > 0 and any sign of num. */
static int64_t floor_div(int64_t num, int64_t den)
{
    int64_t q = num / den;
    if ((num % den != 0) && (num < 0)) q -= 1;
    return q;
}

static int64_t clampi(int64_t i, int64_t n)
{
    if (i < 0) return 0;
    if (i > n - 1) return n - 1;
    return i;
}

/* Keys' cubic convolution kernel with parameter a (piecewise definition). */
static double keys(double u, double a)
{
    double x = fabs(u);
    if (x <= 1.0) return (a + 2.0) * x * x * x - (a + 3.0) * x * x + 1.0;
    if (x < 2.0) return a * x * x * x - 5.0 * a * x * x + 8.0 * a * x - 4.0 * a;
    return 0.0;
}

/*
 * Taps of output index j on an axis resampled from n to m samples.
 * Writes up to 4 clamped source indices and weights; returns the tap count.
 */
static int axis_taps(int64_t j, int64_t n, int64_t m, int method, int coord,
                     double a, int64_t idx[4], double w[4])
{
    int64_t num, den;
    if (coord == C_ASYMMETRIC) {          /* x = j n / m */
        num = j * n;
        den = m;
    } else if (coord == C_HALF_PIXEL) {   /* x = ((2j+1) n - m) / (2m) */
        num = (2 * j + 1) * n - m;
        den = 2 * m;
    } else if (m > 1) {                   /* x = j (n-1) / (m-1) */
        num = j * (n - 1);
        den = m - 1;
    } else {                              /* one output sample: x = 0 */
        num = 0;
        den = 1;
    }
    int64_t i0 = floor_div(num, den);
    double t = (double)(num - i0 * den) / (double)den;

    if (method == M_NEAREST) {
        int64_t i = i0;
        if (coord == C_HALF_PIXEL) {
            /* floor(x + 1/2) = floor((2j+1) n / (2m)) */
            i = floor_div((2 * j + 1) * n, 2 * m);
        } else if (coord == C_ALIGN_CORNERS) {
            /* floor(x + 1/2) = floor((2 num + den) / (2 den)) */
            i = floor_div(2 * num + den, 2 * den);
        }
        idx[0] = clampi(i, n);
        w[0] = 1.0;
        return 1;
    }
    if (method == M_BILINEAR) {
        idx[0] = clampi(i0, n);
        idx[1] = clampi(i0 + 1, n);
        w[0] = 1.0 - t;
        w[1] = t;
        return 2;
    }
    /* bicubic */
    idx[0] = clampi(i0 - 1, n);
    idx[1] = clampi(i0, n);
    idx[2] = clampi(i0 + 1, n);
    idx[3] = clampi(i0 + 2, n);
    w[0] = keys(t + 1.0, a);
    w[1] = keys(t, a);
    w[2] = keys(1.0 - t, a);
    w[3] = keys(2.0 - t, a);
    return 4;
}

/* ---------------------------------------------------------------------- */

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* One output pixel (all C channels) of the 2-D resampling, step 5. */
static void pixel(const double *src, int64_t H, int64_t W, int64_t C,
                  int64_t y, int64_t x, int64_t Ho, int64_t Wo,
                  int method, int coord, double a, double *out)
{
    int64_t iy[4], ix[4];
    double wy[4], wx[4];
    int ny = axis_taps(y, H, Ho, method, coord, a, iy, wy);
    int nx = axis_taps(x, W, Wo, method, coord, a, ix, wx);
    for (int64_t c = 0; c < C; ++c) {
        double acc = 0.0;
        for (int p = 0; p < ny; ++p)
            for (int q = 0; q < nx; ++q)
                acc += wy[p] * wx[q] * src[(iy[p] * W + ix[q]) * C + c];
        out[c] = acc;
    }
}

/*
 * Resample an HWC image src (H x W x C, row-major, FP64) to dst (Ho x Wo x C).
 */
void oracle_resize_f64(const double *src, int64_t H, int64_t W, int64_t C,
                       double *dst, int64_t Ho, int64_t Wo,
                       int method, int coord, double a)
{
    int64_t y;
#pragma omp parallel for schedule(static)
    for (y = 0; y < Ho; ++y)
        for (int64_t x = 0; x < Wo; ++x)
            pixel(src, H, W, C, y, x, Ho, Wo, method, coord, a,
                  dst + (y * Wo + x) * C);
}

/* Same definition evaluated only at the output points (ys[k], xs[k]). */
void oracle_resize_points_f64(const double *src, int64_t H, int64_t W, int64_t C,
                              int64_t Ho, int64_t Wo, int method, int coord, double a,
                              const int64_t *ys, const int64_t *xs, int64_t npts,
                              double *out)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < npts; ++k)
        pixel(src, H, W, C, ys[k], xs[k], Ho, Wo, method, coord, a, out + k * C);
}

/*
 * The paper's bilinear formula (Eqs. 1-5) for one channel (H x W, FP64),
 * written in its four-neighbour form: f(x1,y1), f(x2,y2), f(x3,y3), f(x4,y4)
 * with x1 = x3 = int(x_p), x2 = x4 = int(x_p) + 1, y1 = y2 = int(y_p),
 * y3 = y4 = int(y_p) + 1, each neighbour clamped to the image, and
 *   f = (1 - oy) (ox f2 + (1 - ox) f1) + oy (ox f4 + (1 - ox) f3).
 * Asymmetric map only (Eq. 1).
 */
void oracle_bilinear_eq5_f64(const double *src, int64_t H, int64_t W,
                             double *dst, int64_t Ho, int64_t Wo)
{
    for (int64_t yf = 0; yf < Ho; ++yf) {
        for (int64_t xf = 0; xf < Wo; ++xf) {
            int64_t x1 = floor_div(xf * W, Wo), y1 = floor_div(yf * H, Ho);
            double ox = (double)(xf * W - x1 * Wo) / (double)Wo;
            double oy = (double)(yf * H - y1 * Ho) / (double)Ho;
            int64_t x2 = x1 + 1, y3 = y1 + 1;
            int64_t cx1 = clampi(x1, W), cx2 = clampi(x2, W);
            int64_t cy1 = clampi(y1, H), cy3 = clampi(y3, H);
            double f1 = src[cy1 * W + cx1], f2 = src[cy1 * W + cx2];
            double f3 = src[cy3 * W + cx1], f4 = src[cy3 * W + cx2];
            dst[yf * Wo + xf] = (1.0 - oy) * (ox * f2 + (1.0 - ox) * f1)
                              + oy * (ox * f4 + (1.0 - ox) * f3);
        }
    }
}

/*
 * Adjoint (transpose) of oracle_resize_f64: gx (H x W x C) receives, for
 * every output sample (y, x, c) and every tap pair (p, q), the product
 * wy_p wx_q gy[y, x, c] at the clamped input index (iy_p, ix_q). gx is
 * overwritten. Serial scatter in output order.
 */
void oracle_adjoint_f64(const double *gy, int64_t Ho, int64_t Wo, int64_t C,
                        double *gx, int64_t H, int64_t W,
                        int method, int coord, double a)
{
    memset(gx, 0, sizeof(double) * (size_t)(H * W * C));
    for (int64_t y = 0; y < Ho; ++y) {
        int64_t iy[4];
        double wy[4];
        int ny = axis_taps(y, H, Ho, method, coord, a, iy, wy);
        for (int64_t x = 0; x < Wo; ++x) {
            int64_t ix[4];
            double wx[4];
            int nx = axis_taps(x, W, Wo, method, coord, a, ix, wx);
            for (int64_t c = 0; c < C; ++c) {
                double g = gy[(y * Wo + x) * C + c];
                for (int p = 0; p < ny; ++p)
                    for (int q = 0; q < nx; ++q)
                        gx[(iy[p] * W + ix[q]) * C + c] += wy[p] * wx[q] * g;
            }
        }
    }
}

/* Dense m x n matrix of one axis: A[j][i] = sum of the weights of the taps
 * of output j whose clamped index is i. */
void oracle_axis_matrix(int64_t n, int64_t m, int method, int coord, double a,
                        double *A)
{
    memset(A, 0, sizeof(double) * (size_t)(n * m));
    for (int64_t j = 0; j < m; ++j) {
        int64_t idx[4];
        double w[4];
        int k = axis_taps(j, n, m, method, coord, a, idx, w);
        for (int q = 0; q < k; ++q) A[j * n + idx[q]] += w[q];
    }
}

/* Taps of every output index of one axis (unused slots: index -1, weight 0). */
void oracle_axis_taps(int64_t n, int64_t m, int method, int coord, double a,
                      int64_t *idx, double *w)
{
    for (int64_t j = 0; j < m; ++j) {
        int64_t ii[4] = {-1, -1, -1, -1};
        double ww[4] = {0, 0, 0, 0};
        axis_taps(j, n, m, method, coord, a, ii, ww);
        for (int q = 0; q < 4; ++q) {
            idx[j * 4 + q] = ii[q];
            w[j * 4 + q] = ww[q];
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Storage rounding                                                         */

/* uint8: clamp to [0, 255], then round half to even. NaN maps to 0. */
void oracle_quantize_u8(const double *v, int64_t n, uint8_t *out)
{
    for (int64_t k = 0; k < n; ++k) {
        double x = v[k];
        if (!(x >= 0.0)) x = 0.0;
        if (x > 255.0) x = 255.0;
        out[k] = (uint8_t)nearbyint(x);
    }
}

/*
 * Round d to the nearest value of a binary format with p significand bits
 * and exponent range [emin, emax] (ties to even, gradual underflow,
 * overflow to infinity). The quantum at d's binade is 2^(e - (p-1)) with
 * e = max(exponent of d, emin); d / quantum is exact, nearbyint rounds it
 * half to even.
 */
static double round_format(double d, int p, int emin, int emax)
{
    if (d == 0.0 || !isfinite(d)) return d;
    int e2;
    (void)frexp(d, &e2);
    int lead = e2 - 1;
    if (lead < emin) lead = emin;
    double q = ldexp(1.0, lead - (p - 1));
    double r = nearbyint(d / q) * q;
    double maxv = ldexp(2.0 - ldexp(1.0, -(p - 1)), emax);
    if (fabs(r) > maxv) return copysign(INFINITY, d);
    return r;
}

static uint16_t encode_format(double r, int p, int emin, int ebits)
{
    uint16_t sign = signbit(r) ? (uint16_t)(1u << (p - 1 + ebits)) : 0;
    uint16_t expmask = (uint16_t)((1u << ebits) - 1);
    if (isnan(r)) return (uint16_t)((expmask << (p - 1)) | (1u << (p - 2)));
    if (isinf(r)) return (uint16_t)(sign | (expmask << (p - 1)));
    double x = fabs(r);
    if (x == 0.0) return sign;
    int e2;
    (void)frexp(x, &e2);
    int lead = e2 - 1;
    int bias = -emin + 1;
    if (lead < emin) {   /* subnormal: exponent field 0 */
        uint32_t mant = (uint32_t)ldexp(x, -(emin - (p - 1)));
        return (uint16_t)(sign | mant);
    }
    uint32_t mant = (uint32_t)(ldexp(x, -(lead - (p - 1))) - ldexp(1.0, p - 1));
    return (uint16_t)(sign | ((uint32_t)(lead + bias) << (p - 1)) | mant);
}

/* IEEE binary16: 11 significand bits, exponents -14..15. */
void oracle_to_f16_bits(const double *v, int64_t n, uint16_t *out)
{
    for (int64_t k = 0; k < n; ++k)
        out[k] = encode_format(round_format(v[k], 11, -14, 15), 11, -14, 5);
}

/* bfloat16: 8 significand bits, exponents -126..127. */
void oracle_to_bf16_bits(const double *v, int64_t n, uint16_t *out)
{
    for (int64_t k = 0; k < n; ++k)
        out[k] = encode_format(round_format(v[k], 8, -126, 127), 8, -126, 8);
}

/* ---------------------------------------------------------------------- */
/* Eq. 6: output pixel (px, py) is computed by thread (tx, ty) of block     */
/* (bx, by) for blocks of bw x bh threads.                                  */

void oracle_tile_of_pixel(int64_t px, int64_t py, int64_t bw, int64_t bh,
                          int64_t *bx, int64_t *by, int64_t *tx, int64_t *ty)
{
    *bx = px / bw;
    *tx = px - *bx * bw;
    *by = py / bh;
    *ty = py - *by * bh;
}
