/*
 * ssim_oracle.c -- plain FP64 CPU reference for the SSIM / MS-SSIM hot path of
 * "A Hitchhiker's Guide to Structural Similarity" (arXiv 2101.06354).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the independent checker that the CUDA
 * library is compared against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no source, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Every routine writes the paper's definition out literally in double
 * precision: direct k x k window sums (no separable regrouping, no running
 * sums), except the integral-image routine, whose whole point is to follow the
 * paper's own summed-area-table algorithm (Section "Versions of SSIM",
 * Performance-Efficiency Tradeoffs, Eqs. integral_image_start..corr_from_sum).
 * The only parallelism is an OpenMP split over independent output rows; it
 * does not change any arithmetic.
 *
 * Conventions: images are row-major doubles (H rows, W columns, contiguous)
 * unless a `pitch` is given; window positions are the "valid" ones, i.e. the
 * k x k window W_ij spans rows i..i+k-1 and columns j..j+k-1 (Background
 * section), evaluated at i, j in {0, s, 2s, ...} with i <= H-k, j <= W-k
 * (Section "Effect of stride"); the map is OH x OW with OH = (H-k)/s + 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_BAD_ARG -1

static long out_dim(long n, int k, int s) { return (n < k) ? 0 : (n - k) / s + 1; }

/* 2-D Gaussian window (Background section: "weighting functions sum to unity,
 * and have a finite-extent Gaussian ... shape"; recommended k = 11, sigma = 1.5).
 * w(m,n) = exp(-((m-c)^2 + (n-c)^2) / (2 sigma^2)) / Z, c = (k-1)/2, Z the sum
 * over the k x k support, so that the weights sum to one. */
int oracle_gaussian_window(int k, double sigma, double *w)
{
    if (k < 1 || !(sigma > 0.0) || !w) return ORACLE_BAD_ARG;
    double c = 0.5 * (k - 1), z = 0.0;
    for (int m = 0; m < k; ++m)
        for (int n = 0; n < k; ++n) {
            double dm = m - c, dn = n - c;
            double v = exp(-(dm * dm + dn * dn) / (2.0 * sigma * sigma));
            w[m * k + n] = v;
            z += v;
        }
    for (int i = 0; i < k * k; ++i) w[i] /= z;
    return ORACLE_OK;
}

/* Rectangular window, w(m,n) = 1/k^2 (Section "Performance-Efficiency
 * Tradeoffs": the rectangular weighting used with integral images). */
int oracle_box_window(int k, double *w)
{
    if (k < 1 || !w) return ORACLE_BAD_ARG;
    for (int i = 0; i < k * k; ++i) w[i] = 1.0 / ((double)k * (double)k);
    return ORACLE_OK;
}

/* Local statistics, Eqs. local_means .. local_corr (Background section):
 *   mu1 = sum w I1,  mu2 = sum w I2,
 *   var1 = sum w I1^2 - mu1^2,  var2 = sum w I2^2 - mu2^2,
 *   cov  = sum w I1 I2 - mu1 mu2,
 * each sum running over the k x k window W_ij with weights w (row-major k x k,
 * any values; the paper's windows sum to one).  Outputs are OH x OW maps. */
int oracle_window_stats(const double *x, const double *y, long H, long W,
                        const double *w, int k, int s,
                        double *mu1, double *mu2, double *var1, double *var2,
                        double *cov)
{
    if (!x || !y || !w || k < 1 || s < 1 || H < k || W < k) return ORACLE_BAD_ARG;
    long OH = out_dim(H, k, s), OW = out_dim(W, k, s);
#pragma omp parallel for schedule(dynamic, 1)
    for (long a = 0; a < OH; ++a) {
        for (long b = 0; b < OW; ++b) {
            long i = a * s, j = b * s;
            double s1 = 0, s2 = 0, s11 = 0, s22 = 0, s12 = 0;
            for (int m = 0; m < k; ++m)
                for (int n = 0; n < k; ++n) {
                    double wm = w[m * k + n];
                    double p = x[(i + m) * W + (j + n)];
                    double q = y[(i + m) * W + (j + n)];
                    s1 += wm * p;
                    s2 += wm * q;
                    s11 += wm * p * p;
                    s22 += wm * q * q;
                    s12 += wm * p * q;
                }
            long o = a * OW + b;
            mu1[o] = s1;
            mu2[o] = s2;
            var1[o] = s11 - s1 * s1;
            var2[o] = s22 - s2 * s2;
            cov[o] = s12 - s1 * s2;
        }
    }
    return ORACLE_OK;
}

/* Luminance term (Eq. lum_term) and the combined contrast-structure term with
 * C3 = C2/2 (the cs equation after Eq. cont_term); Q = l * cs.  Any output
 * pointer may be NULL. */
int oracle_ssim_terms(const double *mu1, const double *mu2, const double *var1,
                      const double *var2, const double *cov, long n, double C1,
                      double C2, double *l, double *cs, double *q)
{
    if (!mu1 || !mu2 || !var1 || !var2 || !cov || n < 0) return ORACLE_BAD_ARG;
    for (long i = 0; i < n; ++i) {
        double li = (2.0 * mu1[i] * mu2[i] + C1) / (mu1[i] * mu1[i] + mu2[i] * mu2[i] + C1);
        double ci = (2.0 * cov[i] + C2) / (var1[i] + var2[i] + C2);
        if (l) l[i] = li;
        if (cs) cs[i] = ci;
        if (q) q[i] = li * ci;
    }
    return ORACLE_OK;
}

/* Mean pooling, MSSIM = average of the quality map (Background section).  The
 * average runs over the map elements that exist (valid, strided positions). */
double oracle_mean(const double *v, long n)
{
    double acc = 0.0;
    for (long i = 0; i < n; ++i) acc += v[i];
    return n > 0 ? acc / (double)n : NAN;
}

/* Integer window sums of a uint8 pair by direct summation over each k x k
 * window: out[5*o + {0..4}] = S1_1, S1_2, S2_1, S2_2, S12 (the local sums that
 * Eq. integral_image_end produces).  `pitch` is the row stride in bytes. */
int oracle_box_sums_direct(const uint8_t *x, const uint8_t *y, long H, long W,
                           long pitch, int k, int s, int64_t *out)
{
    if (!x || !y || !out || k < 1 || s < 1 || H < k || W < k || pitch < W) return ORACLE_BAD_ARG;
    long OH = out_dim(H, k, s), OW = out_dim(W, k, s);
#pragma omp parallel for schedule(dynamic, 1)
    for (long a = 0; a < OH; ++a)
        for (long b = 0; b < OW; ++b) {
            int64_t t[5] = {0, 0, 0, 0, 0};
            for (int m = 0; m < k; ++m)
                for (int n = 0; n < k; ++n) {
                    int64_t p = x[(a * s + m) * pitch + b * s + n];
                    int64_t q = y[(a * s + m) * pitch + b * s + n];
                    t[0] += p;
                    t[1] += q;
                    t[2] += p * p;
                    t[3] += q * q;
                    t[4] += p * q;
                }
            memcpy(out + 5 * (a * OW + b), t, sizeof t);
        }
    return ORACLE_OK;
}

/* The paper's integral-image algorithm (Eqs. integral_image_start ..
 * integral_image_end): five summed-area tables I(i,j) = sum_{m<=i, n<=j} of
 * I1, I2, I1^2, I2^2, I1*I2 with 1-based indices and I = 0 when i or j is 0;
 * the sum over the window whose top-left pixel is (i,j) (1-based) is
 *   I(i+k-1, j+k-1) + I(i-1, j-1) - I(i+k-1, j-1) - I(i-1, j+k-1).
 * Output layout as oracle_box_sums_direct. */
int oracle_box_sums_integral(const uint8_t *x, const uint8_t *y, long H, long W,
                             long pitch, int k, int s, int64_t *out)
{
    if (!x || !y || !out || k < 1 || s < 1 || H < k || W < k || pitch < W) return ORACLE_BAD_ARG;
    long SW = W + 1;
    int64_t *I[5];
    for (int t = 0; t < 5; ++t) {
        I[t] = (int64_t *)calloc((size_t)(H + 1) * (size_t)SW, sizeof(int64_t));
        if (!I[t]) {
            for (int u = 0; u < t; ++u) free(I[u]);
            return ORACLE_BAD_ARG;
        }
    }
    for (long i = 1; i <= H; ++i)
        for (long j = 1; j <= W; ++j) {
            int64_t p = x[(i - 1) * pitch + (j - 1)], q = y[(i - 1) * pitch + (j - 1)];
            int64_t v[5] = {p, q, p * p, q * q, p * q};
            for (int t = 0; t < 5; ++t)
                I[t][i * SW + j] = v[t] + I[t][(i - 1) * SW + j] + I[t][i * SW + (j - 1)] -
                                   I[t][(i - 1) * SW + (j - 1)];
        }
    long OH = out_dim(H, k, s), OW = out_dim(W, k, s);
    for (long a = 0; a < OH; ++a)
        for (long b = 0; b < OW; ++b) {
            long i = a * s + 1, j = b * s + 1; /* 1-based top-left pixel */
            for (int t = 0; t < 5; ++t)
                out[5 * (a * OW + b) + t] = I[t][(i + k - 1) * SW + (j + k - 1)] + I[t][(i - 1) * SW + (j - 1)] -
                                            I[t][(i + k - 1) * SW + (j - 1)] - I[t][(i - 1) * SW + (j + k - 1)];
        }
    for (int t = 0; t < 5; ++t) free(I[t]);
    return ORACLE_OK;
}

/* Statistics from local sums, Eqs. mean_from_sum .. corr_from_sum:
 *   mu = S/k^2,  var = S2/k^2 - mu^2,  cov = S12/k^2 - mu1 mu2,
 * then the SSIM terms as in oracle_ssim_terms.  q / cs may be NULL. */
/* SSIM-3D window sums (Section "Spatio-Temporal SSIM"): the five sums of the
 * k x k x Kt rectangular neighbourhood over frames t .. t+Kt-1 (the window
 * ending at frame t+Kt-1), for every valid spatial position and every
 * t = 0 .. T-Kt.  Direct summation.  Frames are `frame_stride` bytes apart,
 * rows `pitch` bytes.  Output: int64[(T-Kt+1) * OH * OW * 5], frame-major. */
int oracle_box3d_sums_direct(const uint8_t *x, const uint8_t *y, long T, long H, long W, long pitch,
                             long frame_stride, int k, int kt, int64_t *out)
{
    if (!x || !y || !out || k < 1 || kt < 1 || T < kt || H < k || W < k || pitch < W ||
        frame_stride < H * pitch) return ORACLE_BAD_ARG;
    long OH = H - k + 1, OW = W - k + 1, OT = T - kt + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (long ta = 0; ta < OT * OH; ++ta) {
        long t = ta / OH, a = ta % OH;
        for (long b = 0; b < OW; ++b) {
            int64_t v[5] = {0, 0, 0, 0, 0};
            for (int o = 0; o < kt; ++o)
                for (int m = 0; m < k; ++m)
                    for (int n = 0; n < k; ++n) {
                        long at = (t + o) * frame_stride + (a + m) * pitch + b + n;
                        int64_t p = x[at], q = y[at];
                        v[0] += p;
                        v[1] += q;
                        v[2] += p * p;
                        v[3] += q * q;
                        v[4] += p * q;
                    }
            memcpy(out + 5 * ((t * OH + a) * OW + b), v, sizeof v);
        }
    }
    return ORACLE_OK;
}

/* Q and cs from window sums over windows of `count` pixels (the local
 * statistics of Eqs. mean_from_sum .. corr_from_sum with the window size
 * k^2 replaced by the number of pixels in the neighbourhood). */
int oracle_box_ssim_from_sums_n(const int64_t *sums, long n, double count, double C1, double C2,
                                double *q, double *cs)
{
    if (!sums || !(count > 0.0) || n < 0) return ORACLE_BAD_ARG;
    for (long o = 0; o < n; ++o) {
        const int64_t *t = sums + 5 * o;
        double mu1 = (double)t[0] / count, mu2 = (double)t[1] / count;
        double var1 = (double)t[2] / count - mu1 * mu1;
        double var2 = (double)t[3] / count - mu2 * mu2;
        double cov = (double)t[4] / count - mu1 * mu2;
        double l = (2.0 * mu1 * mu2 + C1) / (mu1 * mu1 + mu2 * mu2 + C1);
        double c = (2.0 * cov + C2) / (var1 + var2 + C2);
        if (q) q[o] = l * c;
        if (cs) cs[o] = c;
    }
    return ORACLE_OK;
}

int oracle_box_ssim_from_sums(const int64_t *sums, long n, int k, double C1, double C2,
                              double *q, double *cs)
{
    if (!sums || k < 1 || n < 0) return ORACLE_BAD_ARG;
    double kk = (double)k * (double)k;
    for (long o = 0; o < n; ++o) {
        const int64_t *t = sums + 5 * o;
        double mu1 = (double)t[0] / kk, mu2 = (double)t[1] / kk;
        double var1 = (double)t[2] / kk - mu1 * mu1;
        double var2 = (double)t[3] / kk - mu2 * mu2;
        double cov = (double)t[4] / kk - mu1 * mu2;
        double l = (2.0 * mu1 * mu2 + C1) / (mu1 * mu1 + mu2 * mu2 + C1);
        double c = (2.0 * cov + C2) / (var1 + var2 + C2);
        if (q) q[o] = l * c;
        if (cs) cs[o] = c;
    }
    return ORACLE_OK;
}

/* Dyadic downsampling by 2x2 average pooling (MS-SSIM implementations of
 * Daala, Scikit-Video and Tensorflow, Section "Salient Features of SSIM and
 * MS-SSIM Implementations"): out(r,c) = mean of in(2r..2r+1, 2c..2c+1); the
 * output is floor(H/2) x floor(W/2), an odd last row/column is dropped. */
int oracle_downsample2x2(const double *in, long H, long W, double *out)
{
    if (!in || !out || H < 0 || W < 0) return ORACLE_BAD_ARG;
    long OH = H / 2, OW = W / 2;
    for (long r = 0; r < OH; ++r)
        for (long c = 0; c < OW; ++c)
            out[r * OW + c] = 0.25 * (in[(2 * r) * W + 2 * c] + in[(2 * r) * W + 2 * c + 1] +
                                      in[(2 * r + 1) * W + 2 * c] + in[(2 * r + 1) * W + 2 * c + 1]);
    return ORACLE_OK;
}

/* Gradient of the pooled score with respect to the distorted image I2.
 *
 * The paper defines SSIM but not its derivative; this is the chain rule of the
 * Background-section definition.  Treat the five raw window moments of each
 * position p as independent variables: mu1, mu2, m11 = sum w I1^2,
 * m22 = sum w I2^2, m12 = sum w I1 I2, so that var2 = m22 - mu2^2 and
 * cov = m12 - mu1 mu2.  With A1 = 2 mu1 mu2 + C1, B1 = mu1^2 + mu2^2 + C1,
 * A2 = 2 cov + C2, B2 = var1 + var2 + C2, l = A1/B1, cs = A2/B2:
 *   d cs / d m22 = -A2/B2^2,   d cs / d m12 = 2/B2,
 *   d cs / d mu2 = (-A2/B2^2)(-2 mu2) + (2/B2)(-mu1),
 *   d l  / d mu2 = (2 mu1 B1 - 2 mu2 A1) / B1^2,
 * and for Q = l cs: dQ = cs dl + l dcs.  Since d mu2/d I2(q) = w(q-p),
 * d m22/d I2(q) = 2 w(q-p) I2(q), d m12/d I2(q) = w(q-p) I1(q):
 *   d mean / d I2(q) = (1/|map|) sum_p w(q-p) [D_mu2(p) + 2 I2(q) D_m22(p) + I1(q) D_m12(p)],
 * the sum running over the map positions p whose window covers q.
 * which = 0 differentiates mean Q, which = 1 differentiates mean cs.
 * grad is H x W and is overwritten. */
int oracle_ssim_grad(const double *x, const double *y, long H, long W, const double *w,
                     int k, int s, double C1, double C2, int which, double *grad)
{
    if (!x || !y || !w || !grad || k < 1 || s < 1 || H < k || W < k || (which != 0 && which != 1))
        return ORACLE_BAD_ARG;
    long OH = out_dim(H, k, s), OW = out_dim(W, k, s), n = OH * OW;
    double *mu1 = malloc(sizeof(double) * n), *mu2 = malloc(sizeof(double) * n);
    double *v1 = malloc(sizeof(double) * n), *v2 = malloc(sizeof(double) * n);
    double *cv = malloc(sizeof(double) * n);
    double *d_mu2 = malloc(sizeof(double) * n), *d_m22 = malloc(sizeof(double) * n);
    double *d_m12 = malloc(sizeof(double) * n);
    if (!mu1 || !mu2 || !v1 || !v2 || !cv || !d_mu2 || !d_m22 || !d_m12) {
        free(mu1); free(mu2); free(v1); free(v2); free(cv); free(d_mu2); free(d_m22); free(d_m12);
        return ORACLE_BAD_ARG;
    }
    oracle_window_stats(x, y, H, W, w, k, s, mu1, mu2, v1, v2, cv);
    for (long p = 0; p < n; ++p) {
        double A1 = 2.0 * mu1[p] * mu2[p] + C1, B1 = mu1[p] * mu1[p] + mu2[p] * mu2[p] + C1;
        double A2 = 2.0 * cv[p] + C2, B2 = v1[p] + v2[p] + C2;
        double l = A1 / B1, cs = A2 / B2;
        double dcs_m22 = -A2 / (B2 * B2), dcs_m12 = 2.0 / B2;
        double dcs_mu2 = dcs_m22 * (-2.0 * mu2[p]) + dcs_m12 * (-mu1[p]);
        double dl_mu2 = (2.0 * mu1[p] * B1 - 2.0 * mu2[p] * A1) / (B1 * B1);
        if (which == 0) {
            d_mu2[p] = cs * dl_mu2 + l * dcs_mu2;
            d_m22[p] = l * dcs_m22;
            d_m12[p] = l * dcs_m12;
        } else {
            d_mu2[p] = dcs_mu2;
            d_m22[p] = dcs_m22;
            d_m12[p] = dcs_m12;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < H; ++r)
        for (long c = 0; c < W; ++c) {
            double acc = 0.0;
            for (int m = 0; m < k; ++m) {
                long i = r - m; /* window top row of a position covering row r */
                if (i < 0 || i % s != 0 || i / s >= OH) continue;
                for (int nn = 0; nn < k; ++nn) {
                    long j = c - nn;
                    if (j < 0 || j % s != 0 || j / s >= OW) continue;
                    long p = (i / s) * OW + (j / s);
                    acc += w[m * k + nn] * (d_mu2[p] + 2.0 * y[r * W + c] * d_m22[p] + x[r * W + c] * d_m12[p]);
                }
            }
            grad[r * W + c] = acc / (double)n;
        }
    free(mu1); free(mu2); free(v1); free(v2); free(cv); free(d_mu2); free(d_m22); free(d_m12);
    return ORACLE_OK;
}

/* Number of threads the OpenMP split uses (1 when built without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of threads of the OpenMP split (no effect without OpenMP);
 * the CPU baseline times the oracle on one core and on all of them. */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* The same local statistics as oracle_window_stats for a SEPARABLE window
 * w(m,n) = g(m) g(n) (the Gaussian of the Background section, the
 * rectangular window with g = 1/k), computed in two passes the way a plain
 * CPU implementation does: first the five weighted row sums
 *   h_p(r, b) = sum_n g(n) p(r, b s + n)   for p = I1, I2, I1^2, I2^2, I1 I2
 * at every input row r and strided output column b, then the weighted column
 * sums of those at every strided output row, and finally mu and the centred
 * moments exactly as in Eqs. local_means .. local_corr.  Mathematically equal
 * to the direct k x k sums; in FP64 the two agree to rounding (~1e-12
 * relative).  This is the oracle mode the CPU baseline times; the direct mode
 * stays the checker.  g: k taps. */
int oracle_window_stats_separable(const double *x, const double *y, long H, long W,
                                  const double *g, int k, int s,
                                  double *mu1, double *mu2, double *var1, double *var2,
                                  double *cov)
{
    if (!x || !y || !g || k < 1 || s < 1 || H < k || W < k) return ORACLE_BAD_ARG;
    long OH = out_dim(H, k, s), OW = out_dim(W, k, s);
    double *h = (double *)malloc(sizeof(double) * 5 * (size_t)H * (size_t)OW);
    if (!h) return ORACLE_BAD_ARG;
    double *h1 = h, *h2 = h + (size_t)H * OW, *h11 = h + 2 * (size_t)H * OW;
    double *h22 = h + 3 * (size_t)H * OW, *h12 = h + 4 * (size_t)H * OW;
#pragma omp parallel for schedule(dynamic, 8)
    for (long r = 0; r < H; ++r)
        for (long b = 0; b < OW; ++b) {
            double s1 = 0, s2 = 0, s11 = 0, s22 = 0, s12 = 0;
            const double *xr = x + r * W + b * s, *yr = y + r * W + b * s;
            for (int n = 0; n < k; ++n) {
                double p = xr[n], q = yr[n];
                s1 += g[n] * p;
                s2 += g[n] * q;
                s11 += g[n] * p * p;
                s22 += g[n] * q * q;
                s12 += g[n] * p * q;
            }
            long o = r * OW + b;
            h1[o] = s1;
            h2[o] = s2;
            h11[o] = s11;
            h22[o] = s22;
            h12[o] = s12;
        }
#pragma omp parallel for schedule(dynamic, 8)
    for (long a = 0; a < OH; ++a)
        for (long b = 0; b < OW; ++b) {
            double s1 = 0, s2 = 0, s11 = 0, s22 = 0, s12 = 0;
            for (int m = 0; m < k; ++m) {
                long o = (a * s + m) * OW + b;
                s1 += g[m] * h1[o];
                s2 += g[m] * h2[o];
                s11 += g[m] * h11[o];
                s22 += g[m] * h22[o];
                s12 += g[m] * h12[o];
            }
            long o = a * OW + b;
            mu1[o] = s1;
            mu2[o] = s2;
            var1[o] = s11 - s1 * s1;
            var2[o] = s22 - s2 * s2;
            cov[o] = s12 - s1 * s2;
        }
    free(h);
    return ORACLE_OK;
}
