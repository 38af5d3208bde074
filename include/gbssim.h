/*
 * gbssim.h -- C ABI of libgbssim.so, a GB300-native (sm_103a) implementation of
 * the SSIM / MS-SSIM hot path of "A Hitchhiker's Guide to Structural
 * Similarity" (arXiv 2101.06354).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named *_out, `data`, `map`, `workspace`, `grad_y` are DEVICE
 *    pointers owned by the caller.  Descriptor/parameter structs are HOST
 *    memory read during the call only.  The library allocates nothing per call
 *    (gbssim_batch_plan is the one exception and says so).
 *  - Every function is asynchronous on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream): it validates its arguments on the host, enqueues
 *    kernels and returns; results appear in device memory when the stream
 *    reaches them.  Nothing synchronises.
 *  - Return value: GBSSIM_OK (0) or a negative gbssim_status.  Argument errors
 *    are detected before anything is enqueued, so a failed call has no effect.
 *    GBSSIM_ERR_CUDA reports a launch error returned by the CUDA runtime.
 *  - Images are "valid"-bordered: a k x k window W_ij spans rows i..i+k-1 and
 *    columns j..j+k-1 (Background section) and is evaluated at i, j in
 *    {0, s, 2s, ...} with i <= H-k, j <= W-k (Section "Effect of stride"), so
 *    the quality map is OH x OW with OH = (H-k)/s + 1, OW = (W-k)/s + 1.
 *  - Pooled scores are doubles, combined in a fixed order (deterministic:
 *    identical inputs give bit-identical scores).
 */
#ifndef GBSSIM_H
#define GBSSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBSSIM_VERSION 1
#define GBSSIM_MAX_SCALES 8
#define GBSSIM_MAX_K 63
#define GBSSIM_STATIC_SCRATCH_BYTES (1 << 20)
#define GBSSIM_MAX_K_BACKWARD 31

typedef enum gbssim_status {
    GBSSIM_OK = 0,
    GBSSIM_ERR_INVALID_ARG = -1,  /* null pointer, bad enum, stride < 1, ... */
    GBSSIM_ERR_TOO_SMALL = -2,    /* an image (or pyramid level) is smaller than k */
    GBSSIM_ERR_UNSUPPORTED = -3,  /* valid combination the library does not implement */
    GBSSIM_ERR_CUDA = -4,         /* the CUDA runtime reported an error */
    GBSSIM_ERR_DOMAIN = -5,       /* MS-SSIM product with a non-positive pooled term */
    GBSSIM_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
    GBSSIM_ERR_WORKSPACE = -7,    /* workspace missing or smaller than required */
    GBSSIM_ERR_TOO_LARGE = -8     /* problem needs more than the static scratch holds */
} gbssim_status;

typedef enum gbssim_dtype {
    GBSSIM_U8 = 0,   /* 8-bit luminance, nominal range [0, 255] */
    GBSSIM_F16 = 1,
    GBSSIM_BF16 = 2,
    GBSSIM_F32 = 3
} gbssim_dtype;

typedef enum gbssim_window {
    GBSSIM_WIN_GAUSSIAN = 0,  /* w(m,n) = g(m) g(n), g(t) ~ exp(-(t-c)^2 / 2 sigma^2), sum 1 */
    GBSSIM_WIN_BOX = 1        /* w(m,n) = 1/k^2 (integral-image path for uint8) */
} gbssim_window;

typedef enum gbssim_combine {
    GBSSIM_COMBINE_PRODUCT = 0,  /* MS = prod_j m_j^beta_j */
    GBSSIM_COMBINE_SUM = 1       /* MS = sum_j (beta_j / sum beta) m_j  (Scikit-Video "Sum") */
} gbssim_combine;

/* A batch of `count` equally sized images in device memory.  Image b, row r,
 * column c is at element  b*image_stride + r*row_stride + c  of `data`
 * (strides in ELEMENTS, not bytes). */
typedef struct gbssim_plane {
    const void *data;
    int32_t dtype;          /* gbssim_dtype */
    int32_t count;          /* >= 1 */
    int64_t height;         /* H (rows) */
    int64_t width;          /* W (columns) */
    int64_t row_stride;     /* >= width */
    int64_t image_stride;   /* >= height*row_stride when count > 1 */
} gbssim_plane;

/* The problem's knobs as the paper states them.  Fill with
 * gbssim_params_default() and override fields. */
typedef struct gbssim_params {
    int32_t window;   /* gbssim_window */
    int32_t k;        /* window size, 1..GBSSIM_MAX_K (Background: k x k window) */
    double sigma;     /* Gaussian scale (recommended 1.5 with k = 11); ignored for box */
    double K1, K2;    /* C1 = (K1 L)^2, C2 = (K2 L)^2  (Background section) */
    double L;         /* dynamic range, 255 for 8-bit */
    int32_t stride;   /* distance between evaluated windows, >= 1 (Section "Effect of stride") */
    int32_t scales;   /* MS-SSIM scales, 1..GBSSIM_MAX_SCALES (5 in MS-SSIM) */
    double exponents[GBSSIM_MAX_SCALES];  /* beta_j per scale, finest first */
    int32_t combine;  /* gbssim_combine */
    int32_t flags;    /* GBSSIM_FLAG_* (0 = defaults) */
} gbssim_params;

/* uint8 box windows at stride 4 with 16-byte aligned planes: load tiles with
 * double-buffered bulk tensor copies (TMA) instead of per-thread vector loads.
 * Same results (exact integer sums); which is faster depends on the GPU. */
#define GBSSIM_FLAG_BOX_TMA 1
/* MS-SSIM pyramid from the 9/7 biorthogonal wavelet low-pass instead of the
 * 2x2 average (Section "Salient Features of SSIM and MS-SSIM
 * Implementations", the LIBVMAF variant): the CDF 9/7 analysis low-pass
 * (JPEG 2000 irreversible transform, scaled to unit DC gain) along rows and
 * columns with whole-sample symmetric extension, keeping the even samples;
 * level sizes stay floor(H/2) x floor(W/2).  Forward only (the backward and
 * the batch API reject it with GBSSIM_ERR_UNSUPPORTED). */
#define GBSSIM_FLAG_PYRAMID_97 2
/* Border extension (Section "Salient Features of SSIM and MS-SSIM
 * Implementations", border handling): instead of valid windows only, each
 * level's image is extended by floor((k-1)/2) rows / columns before and
 * k-1-floor((k-1)/2) after, with zeros (BORDER_ZERO) or with its mirror image
 * about the border, edge samples repeated (BORDER_REFLECT: x(-1-i) = x(i)),
 * and the valid windows of the extended image make the map: one output per
 * input pixel at stride 1, floor((H-1)/s)+1 x floor((W-1)/s)+1 in general.
 * The MS-SSIM pyramid is formed from the unextended levels.  Every level
 * must be at least ceil((k-1)/2) pixels high and wide (else
 * GBSSIM_ERR_TOO_SMALL).  gbssim_ssim_map and gbssim_msssim only; the other
 * entry points return GBSSIM_ERR_UNSUPPORTED.  At most one of the two. */
#define GBSSIM_FLAG_BORDER_ZERO 4
#define GBSSIM_FLAG_BORDER_REFLECT 8

/* Operation codes for gbssim_workspace_size. */
typedef enum gbssim_op {
    GBSSIM_OP_SSIM = 0,
    GBSSIM_OP_MSSSIM = 1,
    GBSSIM_OP_BACKWARD = 2,
    GBSSIM_OP_BACKWARD_MS = 3,
    GBSSIM_OP_POOL = 4
} gbssim_op;

/* Pooling kinds for gbssim_ssim_pool (Background section for the mean;
 * Section "Spatio-temporal Aggregation of Quality Scores" for the rest).
 * Q is a map value, n the number of values, mu_Q their mean.  `args` (host
 * memory) holds the parameters listed. */
typedef enum gbssim_pool_kind {
    GBSSIM_POOL_MEAN = 0,        /* mean of the map (MSSIM) */
    GBSSIM_POOL_COV = 1,         /* sigma_Q / mu_Q, sigma the population standard deviation */
    GBSSIM_POOL_MINKOWSKI = 2,   /* (1/n) sum (1 - Q)^p;                 args[0] = p >= 0 */
    GBSSIM_POOL_DW = 3,          /* sum (1-Q)^p Q / sum (1-Q)^p;          args[0] = p >= 0 */
    GBSSIM_POOL_MD = 4,          /* ((1/n) sum |Q - mu_Q|^p)^(o/p);       args = p > 0, o */
    GBSSIM_POOL_GM_DSSIM = 5,    /* geometric mean of 1 - Q */
    GBSSIM_POOL_HM_DSSIM = 6,    /* harmonic mean of 1 - Q (0 if some Q = 1) */
    GBSSIM_POOL_PERCENTILE = 7,  /* p-th percentile, linear between order statistics at
                                    h = p/100 (n-1);                      args[0] = p in [0, 100] */
    GBSSIM_POOL_MEDIAN = 8,      /* the 50th percentile */
    GBSSIM_POOL_FNS = 9,         /* five-number summary (min + Q1 + median + Q3 + max) / 5 */
    GBSSIM_POOL_PP = 10,         /* percentile pooling: values at or below the p-th percentile
                                    divided by r, then averaged;          args = p in [0, 100], r > 0 */
    /* series only (gbssim_series_pool): temporal pooling of frame scores */
    GBSSIM_POOL_GM = 11,         /* geometric mean of the scores */
    GBSSIM_POOL_HM = 12,         /* harmonic mean of the scores */
    GBSSIM_POOL_W_AM = 13,       /* mean over the n-k+1 windows of k frames of the window's mean; args[0] = k */
    GBSSIM_POOL_W_GM = 14,       /* ... of the window's geometric mean;  args[0] = k */
    GBSSIM_POOL_W_HM = 15,       /* ... of the window's harmonic mean;   args[0] = k */
    GBSSIM_POOL_W_COV = 16       /* ... of the window's sigma / mean;    args[0] = k */
} gbssim_pool_kind;

/* Human-readable name of a status code (static string, never NULL). */
const char *gbssim_status_string(int status);

/* GBSSIM_VERSION of the loaded library. */
int gbssim_version(void);

/* Recommended defaults (Background section): Gaussian window k = 11,
 * sigma = 1.5, K1 = 0.01, K2 = 0.03, L = 255, stride 1; 5 MS-SSIM scales with
 * exponents 0.0448, 0.2856, 0.3001, 0.2363, 0.1333, product combination. */
void gbssim_params_default(gbssim_params *p);

/* Bytes of device workspace that `op` needs for planes shaped like `x` with
 * parameters `p` (written to *bytes).  The workspace is scratch owned by the
 * caller; it may be reused across calls that do not overlap on the GPU. */
int gbssim_workspace_size(const gbssim_plane *x, const gbssim_params *p, int op, size_t *bytes);

/* SSIM index map and mean-pooled score (MSSIM) of each of the x.count pairs.
 * Eqs. local_means..local_corr (window statistics), lum_term and the
 * C3 = C2/2 contrast-structure term (Q = l * cs), mean pooling (Background
 * section); box windows on uint8 use the integral-image formulation
 * (Eqs. integral_image_start..corr_from_sum) with exact integer sums.
 *   x, y       : reference and distorted batches, identical shape and dtype.
 *   map_out    : nullable; receives Q as float, image b at
 *                map_out + b*map_image_stride, rows map_ld floats apart
 *                (map_ld >= OW, map_image_stride >= OH*map_ld).
 *   mean_out   : nullable; receives x.count doubles (MSSIM per pair).
 *   workspace  : device scratch of at least gbssim_workspace_size(GBSSIM_OP_SSIM).
 */
int gbssim_ssim_map(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                    float *map_out, int64_t map_ld, int64_t map_image_stride, double *mean_out,
                    void *workspace, size_t workspace_bytes, void *stream);

/* Pool `count` float maps (h x w, rows `ld` floats apart, images
 * `image_stride` floats apart) into one double each (device memory `out`).
 * kind is a gbssim_pool_kind; `args` is a host array of its parameters (NULL
 * for the kinds without).  Moment kinds sum fp32 terms per thread with
 * compensation and per block in fp64; order statistics are selected exactly
 * (radix select), so percentiles equal those of the sorted map.  Needs
 * gbssim_workspace_size(GBSSIM_OP_POOL) bytes of workspace computed for a
 * plane of the map's shape (height h, width w, count maps).  Errors:
 * GBSSIM_ERR_INVALID_ARG for a bad kind or parameter, GBSSIM_ERR_UNSUPPORTED
 * for maps of 2^32 values or more. */
int gbssim_ssim_pool(const float *map, int64_t h, int64_t w, int64_t ld, int32_t count,
                     int64_t image_stride, int32_t kind, const double *args, double *out,
                     void *workspace, size_t workspace_bytes, void *stream);

/* Automatic downscaling factor Z (the recommended implementation's "if
 * min(M, N) > 256, resize so that min(M, N) = 256"; Section "Transforming
 * across Various Scales").  rule GBSSIM_DOWNSCALE_ROUND_MIN:
 * max(1, round(min(h, w) / 256)) with halves rounded up (LIBVMAF);
 * GBSSIM_DOWNSCALE_CEIL_H: max(1, ceil(h / 256)).  Host function; returns Z,
 * or GBSSIM_ERR_INVALID_ARG for a bad rule or size. */
#define GBSSIM_DOWNSCALE_ROUND_MIN 0
#define GBSSIM_DOWNSCALE_CEIL_H 1
int gbssim_downscale_factor(int64_t h, int64_t w, int32_t rule);

/* Z x Z block means of each image of `in` (floor size (H / Z) x (W / Z)) into
 * float planes: image b at out + b*out_image_stride, rows out_ld floats apart
 * (out_ld >= W / Z, out_image_stride >= (H / Z) out_ld).  The averaging
 * filter of width Z followed by keeping every Z-th sample, with
 * non-overlapping blocks (Z = 2 is the MS-SSIM 2x2 pyramid step).  1 <= Z <=
 * min(H, W).  Any input dtype; sums in fp32. */
int gbssim_downscale(const gbssim_plane *in, int32_t z, float *out, int64_t out_ld, int64_t out_image_stride,
                     void *stream);

/* BT.709 luma and colour differences of planar RGB images as the paper
 * prints them (Section "Channel-wise SSIM"): Y = 0.213 R + 0.715 G + 0.072 B,
 * Cb = 0.539 (B - Y), Cr = 0.635 (R - Y), on the inputs' own scale (no
 * offset, no clipping; Cb and Cr are signed).  r, g, b: planes of one shape
 * and dtype; outputs: float planes, image i at out + i*out_image_stride,
 * rows out_ld floats apart.  Feed the three planes to gbssim_video (weights
 * e.g. 0.8, 0.1, 0.1, or 1, alpha, beta) for the channel-weighted SSIM. */
int gbssim_rgb_to_ycbcr(const gbssim_plane *r, const gbssim_plane *g, const gbssim_plane *b, float *y_out,
                        float *cb_out, float *cr_out, int64_t out_ld, int64_t out_image_stride, void *stream);

/* Window-weighted local mean of x at every valid (strided) map position, the
 * mu_1 of Eq. local_means, with p's window (Gaussian k, sigma or box k) and
 * stride; float output laid out like a map (rows out_ld floats apart, images
 * out_image_stride apart).  Any input dtype; fp32 sums.  It is the input of
 * luminance-weighted pooling. */
int gbssim_local_mean(const gbssim_plane *x, const gbssim_params *p, float *out, int64_t out_ld,
                      int64_t out_image_stride, void *stream);

/* Luminance-weighted pooling (Section "Spatio-temporal Aggregation of Quality
 * Scores", LW pooling): S_LW = (1/n) sum w(mu_1) Q with w = 0 for mu_1 < a,
 * (mu_1 - a)/b on [a, a + b), 1 from a + b on (b = 0: a step at a); mu_ref
 * holds mu_1 (gbssim_local_mean of the reference) in the map's layout.
 * a = b = 0 is the plain mean.  Workspace: gbssim_workspace_size(GBSSIM_OP_POOL). */
int gbssim_ssim_pool_lw(const float *map, const float *mu_ref, int64_t h, int64_t w, int64_t ld, int32_t count,
                        int64_t image_stride, double a, double b, double *out, void *workspace, size_t workspace_bytes,
                        void *stream);

/* Temporal pooling of `count` series of n frame scores (doubles, device
 * memory, series b at scores + b*stride) into one double each (device `out`),
 * in fp64 (Section "Spatio-temporal Aggregation of Quality Scores").  Every
 * gbssim_pool_kind applies: the map kinds as for gbssim_ssim_pool, plus
 * GM / HM and the windowed means W-AM, W-GM, W-HM, W-CoV over the n-k+1
 * windows of k consecutive frames (args[0] = k, 1 <= k <= n).  `args` is a
 * host array.  n in 1..4096, count in 1..65535, stride >= n; no workspace.
 * Errors: GBSSIM_ERR_INVALID_ARG for a bad kind, size or parameter. */
int gbssim_series_pool(const double *scores, int32_t n, int32_t count, int64_t stride, int32_t kind,
                       const double *args, double *out, void *stream);

/* SSIM-3D of a uint8 video pair (Section "Spatio-Temporal SSIM"): SSIM whose
 * local statistics (mean, variance, covariance) are taken over k x k x kt
 * rectangular spatio-temporal neighbourhoods instead of k x k ones.  The
 * window of output frame t covers input frames t .. t+kt-1 (the window
 * ending at frame t+kt-1); like the spatial map, only windows inside the
 * video count, so there are T-kt+1 output frames of (H-k+1) x (W-k+1)
 * positions.  The window sums are exact integers (int32 or int64, int64
 * numerators).
 *   x, y       : the T frames as a batch (count = T, image_stride = frame stride).
 *   p          : window = GBSSIM_WIN_BOX, k <= 31, stride 1; K1, K2, L as usual.
 *   kt         : frames per window, 1 <= kt <= T, 5 (k^2 kt)^2 255^2 < 2^63
 *                (the exact int64 numerators; int32 window sums while
 *                k^2 kt 510^2 < 2^31, int64 beyond).
 *   frame_out  : nullable; T-kt+1 doubles, the mean Q of each output frame.
 *   score_out  : nullable; one double, the mean over all output frames.
 *   map_out    : nullable; Q of output frame t at map_out + t*map_frame_stride,
 *                rows map_ld floats apart.
 *   workspace  : gbssim_ssim3d_workspace_size bytes.
 * Errors: GBSSIM_ERR_UNSUPPORTED for other dtypes, windows, strides or sizes
 * past the exact-integer range; GBSSIM_ERR_TOO_SMALL if T < kt or a frame is
 * smaller than k. */
int gbssim_ssim3d_workspace_size(const gbssim_plane *x, const gbssim_params *p, int32_t kt, size_t *bytes);
int gbssim_ssim3d(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t kt,
                  double *frame_out, double *score_out, float *map_out, int64_t map_ld, int64_t map_frame_stride,
                  void *workspace, size_t workspace_bytes, void *stream);

/* MS-SSIM-3D of a uint8 video pair (Section "Spatio-Temporal SSIM": the 3-D
 * index computed over several spatial scales).  Every frame has its own 2x2
 * average pyramid (floor sizes, as gbssim_msssim); level j of the video is
 * the T frames at pyramid level j, and gbssim_ssim3d's k x k x kt box
 * statistics on it give the cs and Q maps of the T-kt+1 output frames.  Per
 * output frame, m_j = mean cs_j (j < S) and m_S = mean Q_S are combined like
 * MS-SSIM (product of m_j^beta_j, or the normalised sum); the video score is
 * the mean over output frames.  Pyramid values are multiples of 4^-j: the
 * window sums stay exact (int64 sums of the values times 4^j).
 *   p             : window = GBSSIM_WIN_BOX, k <= 31, stride 1; scales,
 *                   exponents and combine as for gbssim_msssim.
 *   kt            : frames per window, 1 <= kt <= T, with the exact-integer
 *                   range 5 (k^2 kt)^2 (255 4^j)^2 < 2^63 at every level j.
 *   frame_out     : nullable; T-kt+1 doubles, the score of each output frame.
 *   score_out     : nullable; one double, the mean of the frame scores.
 *   per_scale_out : nullable; (T-kt+1) * scales * 2 doubles, (mean cs_j,
 *                   mean Q_j) of each output frame and scale, finest first.
 *   workspace     : gbssim_msssim3d_workspace_size bytes (tile partials and
 *                   the float pyramid, 4/3 of the input's bytes per video).
 * Errors: as gbssim_ssim3d, GBSSIM_ERR_TOO_SMALL if a level is below k x k,
 * GBSSIM_ERR_UNSUPPORTED for T > 65535 with more than one scale. */
int gbssim_msssim3d_workspace_size(const gbssim_plane *x, const gbssim_params *p, int32_t kt, size_t *bytes);
int gbssim_msssim3d(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t kt,
                    double *frame_out, double *score_out, double *per_scale_out, void *workspace,
                    size_t workspace_bytes, void *stream);

/* CMSSIM of `count` pairs of RGB images (Section "CMSSIM"): RGB -> CIE XYZ
 * -> the luminance, red-green and blue-yellow planes (the section's forward
 * matrix) -> Gaussian smoothing of the two chromatic planes -> XYZ (the
 * section's inverse matrix, as printed) -> CIE 1976 L*, a*, b*; the SSIM map
 * of the two L* planes (dynamic range 100) is weighted at every position by
 * (1 - Delta E / 45), Delta E the CIELAB distance of the two images at the
 * window's centre pixel, and mean-pooled.  Readings: linear RGB in [0, 1]
 * (uint8 values / 255, no transfer curve) with the BT.709 / sRGB primaries
 * and D65 white; the smoothing kernel is the params' Gaussian window with one
 * output per pixel (planes extended by mirroring about the border); CIELAB
 * relative to that D65 white.
 *   rgb_x, rgb_y : three planes each (R, G, B), all of one shape and dtype.
 *   p            : window = GBSSIM_WIN_GAUSSIAN (k, sigma), K1, K2, stride;
 *                  L is fixed at 100 (the L* range); no flags.
 *   score_out    : count doubles (device).
 *   map_out      : nullable; the weighted map of each pair, rows map_ld floats
 *                  apart, images map_image_stride floats apart.
 *   workspace    : gbssim_cmssim_workspace_size bytes (r's shape and p).
 * Errors: GBSSIM_ERR_UNSUPPORTED for a box window or border flags;
 * GBSSIM_ERR_TOO_SMALL if the images are smaller than k x k. */
int gbssim_cmssim_workspace_size(const gbssim_plane *r, const gbssim_params *p, size_t *bytes);
int gbssim_cmssim(const gbssim_plane rgb_x[3], const gbssim_plane rgb_y[3], const gbssim_params *p,
                  double *score_out, float *map_out, int64_t map_ld, int64_t map_image_stride, void *workspace,
                  size_t workspace_bytes, void *stream);

/* QSSIM of `count` pairs of colour pictures (Section "Quaternion SSIM"): each
 * pixel of a tristimulus picture (RGB, YUV, ... : the three planes given) is
 * the pure quaternion q = c0 i + c1 j + c2 k; per picture the mean ("DC")
 * mu_q = (1/MN) sum q and the deviations ("AC") ac_q = q - mu_q give
 *   sigma_q^2 = sum |ac_q|^2 / ((M-1)(N-1)),
 *   sigma_{ref,dis} = sum ac_ref conj(ac_dis) / ((M-1)(N-1))  (a quaternion),
 *   QSSIM = |2 mu_ref conj(mu_dis) + C1| / (|mu_ref|^2 + |mu_dis|^2 + C1)
 *         * |2 sigma_{ref,dis} + C2| / (sigma_ref^2 + sigma_dis^2 + C2),
 * |.| the quaternion modulus: one global score per picture, no windows.
 * Readings of the printed (garbled) formula: the contrast uses the squared
 * norm; mu^2, sigma^2 in the denominators are squared moduli; the second
 * factor's denominator is sigma_ref^2 + sigma_dis^2 and its numerator carries
 * the grayscale cs term's factor 2 (so QSSIM(x, x) = 1); the grayscale
 * stabilising constants C1, C2 are added (K1 = K2 = 0 gives the printed
 * constant-free form); the (M-1)(N-1) normalisation is as printed.
 *   tri_x, tri_y : three planes each (the tristimulus components), all six of
 *                  one shape, dtype, count and strides; H, W >= 2.
 *   p            : K1, K2 and L only (window, k, stride, scales are unused).
 *   score_out    : count doubles (device).
 *   terms_out    : nullable; 2 * count doubles (device): the luminance factor
 *                  and the contrast-structure factor of each pair.
 *   workspace    : gbssim_qssim_workspace_size bytes (x's shape and dtype).
 * uint8 pictures take exact integer sums (one pass); float pictures two
 * passes (means, then the deviations' sums), fp64 per CTA, fixed order.
 * Errors: GBSSIM_ERR_TOO_SMALL for H or W < 2. */
int gbssim_qssim_workspace_size(const gbssim_plane *x, size_t *bytes);
int gbssim_qssim(const gbssim_plane tri_x[3], const gbssim_plane tri_y[3], const gbssim_params *p,
                 double *score_out, double *terms_out, void *workspace, size_t workspace_bytes, void *stream);

/* MS-SSIM of each pair (Introduction; Section "Salient Features of SSIM and
 * MS-SSIM Implementations"): scale 1 is the input, scale j+1 the 2x2 average
 * of scale j (floor size); the contrast-structure term is mean-pooled at every
 * scale and the luminance term only at the coarsest, m_j = mean cs_j (j < S),
 * m_S = mean Q_S; score = prod m_j^beta_j (or the normalised sum).
 *   score_out     : x.count doubles.  A product with a non-positive m_j under a
 *                   non-integer exponent yields NaN for that pair (the call
 *                   still returns GBSSIM_OK; the value is checked on device).
 *   per_scale_out : nullable; x.count * scales * 2 doubles, (mean cs_j, mean Q_j)
 *                   for each scale j, finest first.
 * Every pyramid level must be at least k x k (else GBSSIM_ERR_TOO_SMALL). */
int gbssim_msssim(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                  double *score_out, double *per_scale_out, void *workspace,
                  size_t workspace_bytes, void *stream);

/* MS-SSIM of pairs held in HOST memory, with the host-to-device copies
 * overlapped with compute (the computation is gbssim_msssim's; this call only
 * adds the transfers; the paper has no counterpart).  The count images are
 * split into `chunks` chunks of ceil(count / chunks) images; chunk c+1 is
 * copied on `copy_stream` into one of two device stages while chunk c is
 * scored on `stream`, and the scores come back with one device-to-host copy.
 *   x, y         : host planes (any pitch; pinned memory gives the overlap,
 *                  pageable memory is correct but copied synchronously).
 *                  They must stay valid until `stream` has completed.
 *   chunks       : >= 1 (clamped to count); or 0, streamed: every image gets
 *                  its own device slot and one MS-SSIM launch covers them all;
 *                  the copy stream copies the images in up to 16 groups of
 *                  consecutive images and after each group sets that group's
 *                  arrival flag with a stream memory write; the level-0 work
 *                  of an image waits (bounded) for its group's flag, so
 *                  scoring starts as soon as the first group is in.  Work
 *                  items run as a wavefront over the groups (level j of group
 *                  g beside level 0 of group g + j), and the two largest
 *                  levels use shorter items than gbssim_msssim's, so the
 *                  scores agree with it to rounding (another fp32 summation
 *                  order), not bit for bit; chunked mode is bit-identical.
 *                  A wait that gives up yields NaN scores.  Streamed
 *                  mode needs the Gaussian 11-tap window at stride 1 without
 *                  the 9/7 pyramid or border flags (else
 *                  GBSSIM_ERR_UNSUPPORTED) and a copy_stream created with
 *                  cudaStreamNonBlocking (else GBSSIM_ERR_INVALID_ARG: a
 *                  stream that synchronises with `stream` would hold the
 *                  copies behind the launch).
 *   score_host   : x.count doubles in host memory (pinned for an asynchronous
 *                  return), valid once `stream` has completed.
 *   workspace    : device buffer of gbssim_msssim_host_workspace_size bytes;
 *                  every earlier call on `stream` that used it is finished
 *                  before this call's copies overwrite it.
 *   stream, copy_stream : two different streams (GBSSIM_ERR_INVALID_ARG if
 *                  equal); all work of the call, copies included, is ordered
 *                  before the end of `stream` (also when a bounded wait gave
 *                  up before every copy landed).
 *   stream2      : nullable third stream.  When given, odd chunks are scored
 *                  on it (each stage has its own MS-SSIM workspace), so one
 *                  chunk's kernel fills the GPU while the previous one drains;
 *                  it must differ from the other two.  Streamed mode has one
 *                  launch and leaves it unused.
 * Six CUDA events are created per call and released when the streams pass
 * them. */
int gbssim_msssim_host_workspace_size(const gbssim_plane *x, const gbssim_params *p, int32_t chunks,
                                      size_t *bytes);
int gbssim_msssim_host(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t chunks,
                       double *score_host, void *workspace, size_t workspace_bytes, void *stream,
                       void *copy_stream, void *stream2);

/* Gradient of the pooled score with respect to the distorted image y, for
 * SSIM (multiscale = 0: score = MSSIM, Background section) or MS-SSIM
 * (multiscale = 1: score as gbssim_msssim).  The paper defines the score,
 * not its derivative; this is the chain rule of those definitions: each
 * window position p contributes w(q - p) [dQ/dmu_y + 2 (y(q) - mu_y) dQ/ds_y^2
 * + (x(q) - mu_x) dQ/ds_xy] to pixel q, mean pooling divides by the map size,
 * MS-SSIM multiplies level j by d score / d m_j (= score beta_j / m_j for the
 * product) and carries coarser levels to finer ones through the adjoint of
 * 2x2 average pooling (a quarter of each coarse gradient to each of its four
 * pixels).  The window moments are recomputed, nothing from a forward call is
 * reused.
 *   grad_y[b] = grad_scale * g_b * d score_b / d y_b, where g_b = 1 when
 *   grad_out is NULL, else grad_out[grad_out_per_image ? b : 0] (device
 *   doubles, e.g. the incoming gradient of a loss).  grad_y (device) has
 *   dtype grad_dtype (F32, F16 or BF16), rows grad_ld elements apart, images
 *   grad_image_stride apart; every pixel of every image is written.
 *   fwd_score, fwd_per_scale (MS-SSIM only, nullable, both or neither):
 *   device outputs (score_out, per_scale_out) of a gbssim_msssim call on the
 *   same x, y and parameters.  When given, the backward does not re-run the
 *   MS-SSIM forward to pool the scales; it only rebuilds the pyramid planes
 *   (the window moments are still recomputed).  Ignored for SSIM.
 *   score_out: nullable, x.count doubles, the scores themselves.
 *   Requires stride == 1 and k <= GBSSIM_MAX_K_BACKWARD (else
 *   GBSSIM_ERR_UNSUPPORTED); workspace of gbssim_workspace_size with
 *   GBSSIM_OP_BACKWARD (multiscale = 0) or GBSSIM_OP_BACKWARD_MS. */
int gbssim_ssim_backward(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                         int32_t multiscale, double grad_scale, const double *grad_out,
                         int32_t grad_out_per_image, const double *fwd_score, const double *fwd_per_scale,
                         void *grad_y, int32_t grad_dtype, int64_t grad_ld, int64_t grad_image_stride,
                         double *score_out, void *workspace, size_t workspace_bytes, void *stream);

/* The SSIM / MS-SSIM loss split into a forward that keeps what the backward
 * needs and a backward that reuses it (the computation of
 * gbssim_ssim_backward without recomputing the window moments; the paper
 * defines the score only, the gradient is the chain rule of its
 * definitions).  gbssim_loss_forward runs every level once in coefficient
 * mode (moments, Q, cs and the three coefficient maps per output, 2x2 pyramid
 * fused) and writes the scores (score_out, nullable; per_scale_out as for
 * gbssim_msssim, nullable) and, in `saved`, the coefficient maps, pooled
 * values and pyramid planes.  gbssim_loss_backward then writes
 * grad_scale * grad_out * d(score)/dy into grad_y from `saved` alone (x, y and
 * p must be those of the forward; `saved` is not modified except for its
 * coarse-gradient scratch).  `saved` is caller-owned device memory of
 * gbssim_loss_saved_size bytes; it must stay untouched between the two calls.
 * Arguments and restrictions otherwise as gbssim_ssim_backward (stride 1,
 * k <= 31, no 9/7 pyramid). */
int gbssim_loss_saved_size(const gbssim_plane *x, const gbssim_params *p, int32_t multiscale, size_t *bytes);
int gbssim_loss_forward(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t multiscale,
                        double *score_out, double *per_scale_out, void *saved, size_t saved_bytes, void *stream);
int gbssim_loss_backward(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t multiscale,
                         double grad_scale, const double *grad_out, int32_t grad_out_per_image, const void *saved,
                         size_t saved_bytes, void *grad_y, int32_t grad_dtype, int64_t grad_ld,
                         int64_t grad_image_stride, void *stream);

/* Colour and temporal pooling of a YUV video (any chroma subsampling).
 * planes = {x_Y, y_Y, x_U, y_U, x_V, y_V}, each a batch of `frames` images
 * (count = frames, the same for all six); each plane pair is scored at its
 * own resolution with gbssim_ssim_map's MSSIM.  Then (Section "Channel-wise
 * SSIM") frame score F(t) = (w_Y S_Y + w_U S_U + w_V S_V) / (w_Y + w_U + w_V)
 * with weights = {w_Y, w_U, w_V} (e.g. 6, 1, 1 or 0.8, 0.1, 0.1), and
 * (Sections "Spatio-temporal Aggregation of Quality Scores", "Percentile
 * Pooling") video_out[0] = mean_t F, video_out[1] = the `percentile`-th
 * percentile of F (linear interpolation at h = p/100 (frames-1) of the
 * sorted scores), video_out[2] = percentile pooling: the mean of F after the
 * scores at or below that percentile are divided by pp_r.
 *   frame_out (nullable): frames doubles F(t); plane_out (nullable):
 *   3 x frames doubles S_Y(t) | S_U(t) | S_V(t); video_out: 3 doubles (all
 *   device).  frames <= 4096.  Workspace: gbssim_video_workspace_size. */
int gbssim_video_workspace_size(const gbssim_plane planes[6], const gbssim_params *p, size_t *bytes);
int gbssim_video(const gbssim_plane planes[6], const gbssim_params *p, const double weights[3], double percentile,
                 double pp_r, double *frame_out, double *plane_out, double *video_out, void *workspace,
                 size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ ragged batch
 * SSIM or MS-SSIM of many pairs of different sizes in ONE persistent kernel
 * launch (plus a memset and a finaliser), suitable for CUDA-graph capture.
 * Restricted to the fused 11-tap path: k = 11, stride 1 (Gaussian or box
 * window), any input dtype shared by the whole batch. */
typedef struct gbssim_batch gbssim_batch;

/* Tuning knobs of a batch plan (chosen by the Python autotuner); zero = default. */
typedef struct gbssim_tuning {
    int32_t seg_rows;      /* output rows per work item, multiple of 16 (default 256) */
    int32_t ctas_per_sm;   /* resident CTAs per SM of the persistent grid (default: maximum) */
    uint32_t wait_limit;   /* spin iterations before a level dependency wait gives up (default 4M) */
    int32_t flags;         /* GBSSIM_TUNING_* */
    int32_t tile_w;        /* output columns per work item (the strip width): 32, 64 (default) or 128;
                              a CTA runs 4 x tile_w threads, each 4 output rows of one column */
} gbssim_tuning;

/* Test hook: image 0's level-1 items wait for one more level-0 item than
 * exists, so their bounded wait runs out and the run reports
 * GBSSIM_ERR_TIMEOUT through gbssim_batch_status.  Never set in production. */
#define GBSSIM_TUNING_TEST_STALL 1
/* Test hook of gbssim_msssim_host_ex (streamed mode): the last copy group's
 * arrival flag is never written, so the level-0 items of its images wait
 * until their bounded wait runs out; the call then reports
 * GBSSIM_ERR_TIMEOUT in *status_host and NaN scores for those images (the
 * copies themselves still run).  Never set in production. */
#define GBSSIM_TUNING_TEST_DROP_ARRIVAL 2

/* Build a plan for n entries: entry e pairs xs[e] with ys[e] (identical
 * shape; each entry may itself hold count >= 1 equally sized images); all
 * entries share one dtype.  The plan is bound to these device pointers: a run
 * reads whatever they hold at that time.  This call allocates (one device
 * buffer for the work tables) and copies to it synchronously; it is the only
 * allocating call of the library.  multiscale = 0: SSIM; 1: MS-SSIM with
 * p->scales levels.  tuning may be NULL.  Errors: GBSSIM_ERR_UNSUPPORTED
 * unless k = 11 and stride = 1; GBSSIM_ERR_TOO_SMALL if a level is below k. */
int gbssim_batch_plan(const gbssim_plane *xs, const gbssim_plane *ys, int32_t n, const gbssim_params *p,
                      int32_t multiscale, const gbssim_tuning *tuning, gbssim_batch **plan_out);

/* Workspace bytes a run of this plan needs (pyramid levels, pooling slots,
 * work counter, dependency counters, status word). */
int gbssim_batch_workspace_size(const gbssim_batch *plan, size_t *bytes);

/* Images in the plan, work items, persistent grid size, rows per item
 * (any pointer may be NULL). */
int gbssim_batch_info(const gbssim_batch *plan, int32_t *n_images, int32_t *total_items, int32_t *grid,
                      int32_t *seg_rows);

/* Enqueue one run: scores_out receives one double per image (entries
 * expanded in order), per_scale_out (nullable) images x scales x 2 doubles
 * (mean cs_j, mean Q_j).  Asynchronous and graph-capturable. */
int gbssim_batch_run(const gbssim_batch *plan, double *scores_out, double *per_scale_out, void *workspace,
                     size_t workspace_bytes, void *stream);

/* Copy the run's device status word (GBSSIM_OK, or GBSSIM_ERR_TIMEOUT when a
 * bounded dependency wait gave up) to the device int32 *status_out, ordered
 * after the run on `stream`. */
int gbssim_batch_status(const gbssim_batch *plan, const void *workspace, int32_t *status_out, void *stream);

/* Release the plan's device tables (NULL is ignored). */
void gbssim_batch_free(gbssim_batch *plan);

/* gbssim_msssim_host with two more arguments (no counterpart in the paper):
 *   tuning      : nullable; wait_limit (0 = default) bounds the persistent
 *                 launch's device-side waits (a level-j item's wait for its
 *                 image's level j-1, `wait_limit` polls; a level-0 item's wait
 *                 for its copy group's arrival flag, 16 x `wait_limit` polls);
 *                 flags may hold GBSSIM_TUNING_TEST_DROP_ARRIVAL only (else
 *                 GBSSIM_ERR_INVALID_ARG); seg_rows, ctas_per_sm and tile_w are ignored.
 *   status_host : nullable host int32 (pinned for an asynchronous return);
 *                 receives the launch's status word, GBSSIM_OK or
 *                 GBSSIM_ERR_TIMEOUT when a bounded wait gave up (its images
 *                 then score NaN), valid once `stream` has completed.
 * status_host and the test flag need streamed mode (chunks = 0), else
 * GBSSIM_ERR_UNSUPPORTED.  Everything else as gbssim_msssim_host. */
int gbssim_msssim_host_ex(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t chunks,
                          const gbssim_tuning *tuning, double *score_host, int32_t *status_host, void *workspace,
                          size_t workspace_bytes, void *stream, void *copy_stream, void *stream2);

/* gbssim_ssim_map without a workspace argument, for callers that cannot
 * allocate device memory: a plugin inside a host application that owns the
 * GPU allocator and gives it only input and output buffers, or a real-time
 * pipeline that forbids cudaMalloc after start-up because it can block and
 * synchronise the device.  (The paper has no counterpart; this is a calling
 * convention of this library.)
 *   Same arguments, results and errors as gbssim_ssim_map, minus the
 *   workspace.  Scratch comes from a static device array of
 *   GBSSIM_STATIC_SCRATCH_BYTES (1 MiB) that every GPU loading the library
 *   holds until exit; a problem whose gbssim_workspace_size(GBSSIM_OP_SSIM)
 *   exceeds it is rejected with GBSSIM_ERR_TOO_LARGE before any work is
 *   enqueued (about 430 pairs of 1920x1080 fit in one call).
 *   The call allocates nothing.  Its first call on a device (with that
 *   device current) looks up the array's device address once; make that
 *   first call before any stream capture (a lookup that fails returns
 *   GBSSIM_ERR_CUDA and is retried by the next call).  All calls share the array and it
 *   keeps the last call's contents (nothing needs clearing: each call writes
 *   every slot it reads), so calls whose GPU work overlaps race: serialise
 *   them. */
int gbssim_ssim_map_static(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                           float *map_out, int64_t map_ld, int64_t map_image_stride,
                           double *mean_out, void *stream);

/* FP32 fused multiply-add throughput probe (no counterpart in the paper: it
 * measures the peak that the ALU-bound Gaussian kernels are compared with).
 * Enqueues one launch of `blocks` CTAs x 256 threads; every thread performs
 * 256 * iters FMAs = 512 * iters FLOP, as 16 independent scalar FFMA chains
 * (packed = 0) or 8 independent packed f32x2 FFMA2 chains (packed != 0), and
 * writes one float to sink[block * 256 + thread] (device, blocks * 256
 * floats, caller-owned).  Time it with CUDA events on `stream`: FP32 rate =
 * blocks * 256 * 512 * iters / time.  Errors: GBSSIM_ERR_INVALID_ARG for a
 * null sink or blocks, iters < 1. */
int gbssim_fp32_probe(int32_t packed, int32_t blocks, int32_t iters, float *sink, void *stream);

/* Exact integer window sums of a uint8 pair, the quantities the paper's
 * integral images produce (Eqs. integral_image_start..integral_image_end):
 * for every window position, 5 int64 values S1_x, S1_y, S2_x, S2_y, S_xy in
 * row-major map order, image b at sums_out + 5*b*OH*OW.  k <= GBSSIM_MAX_K. */
int gbssim_window_sums(const gbssim_plane *x, const gbssim_plane *y, int32_t k, int32_t stride,
                       int64_t *sums_out, void *stream);
/* As gbssim_window_sums with GBSSIM_FLAG_* flags (GBSSIM_FLAG_BOX_TMA selects
 * the bulk-tensor-copy tile loader for stride 4 on aligned planes). */
int gbssim_window_sums_ex(const gbssim_plane *x, const gbssim_plane *y, int32_t k, int32_t stride, int32_t flags,
                          int64_t *sums_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBSSIM_H */
