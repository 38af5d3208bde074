// common.cuh -- device helpers and launch declarations shared by the gbssim
// kernels.  Internal to libgbssim.so; the public interface is include/gbssim.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/gbssim.h"

namespace gbssim {

// Per-device once-flags of the launchers (a kernel's shared-memory attribute
// set, a device figure cached).  Callers may launch from several host
// threads: a flag read as set (acquire) implies the work before its set
// (release); two threads may both do the (idempotent) work.
struct DeviceOnce {
    std::atomic<bool> done[64];
    bool is_set(int dev) const { return done[dev].load(std::memory_order_acquire); }
    void set(int dev) { done[dev].store(true, std::memory_order_release); }
};

// The correctly rounded fp32 value of an integer |v| < 2^48, the value
// __ll2float_rn gives, without the 64-bit conversion (which runs on the slow
// FP64 pipe): v = hi 2^24 + lo with 0 <= lo < 2^24, both parts exact in
// fp32, and the FMA rounds the exact hi 2^24 + lo once.
__device__ __forceinline__ float i48_to_f32(int64_t v) {
    const int hi = (int)(v >> 24);
    const int lo = (int)(v & 0xffffff);
    return fmaf((float)hi, 16777216.0f, (float)lo);
}

// ---------------------------------------------------------------- element loads

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<uint8_t>(uint8_t v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }

template <typename T>
__device__ __forceinline__ float load_f32(const T *p) { return to_f32<T>(__ldg(p)); }
template <>
__device__ __forceinline__ float load_f32<__half>(const __half *p) {
    return __half2float(__ldg(p));
}
template <>
__device__ __forceinline__ float load_f32<__nv_bfloat16>(const __nv_bfloat16 *p) {
    unsigned short raw = __ldg(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float(((unsigned)raw) << 16);
}

// ---------------------------------------------------------------- shapes

struct ImgDesc {
    const void *data;
    int64_t H, W, row_stride, image_stride;
};

__host__ __device__ inline int64_t out_dim(int64_t n, int k, int s) {
    return n < k ? 0 : (n - k) / s + 1;
}

// 1-D separable taps, passed by value (lives in the kernel-parameter bank).
template <int K>
struct Taps {
    float g[K];
};
struct TapsDyn {
    float g[GBSSIM_MAX_K];
};
// Taps duplicated as (w, w) pairs, the operand form of the packed f32x2
// instructions, so the pair comes straight from the parameter bank.
template <int K>
struct Taps2 {
    float2 g2[K];
};

// SSIM constants of one launch.
struct SsimConst {
    float C1, C2;
    float C1x2, C2x2;  // 2 C1, 2 C2 (the (u, w) form of the formula)
};
// The only constructor: C1 = (K1 L)^2 and C2 = (K2 L)^2 given in double.
inline SsimConst ssim_const(double c1, double c2) {
    return SsimConst{(float)c1, (float)c2, 2.f * (float)c1, 2.f * (float)c2};
}

// ---------------------------------------------------------------- backward coefficients
//
// Derivative of Q (which = 0) or cs (which = 1) at one window position with
// respect to the distorted image.  From the Background-section definitions,
// with A1 = 2 mu_x mu_y + C1, B1 = mu_x^2 + mu_y^2 + C1, A2 = 2 s_xy + C2,
// B2 = s_x^2 + s_y^2 + C2, l = A1/B1, cs = A2/B2:
//   dQ/d mu_y (central moments fixed) = cs * 2 (mu_x - mu_y l) / B1
//   dQ/d s_y^2 = -l cs / B2,    dQ/d s_xy = 2 l / B2
// and a pixel q of the window moves mu_y by w, s_y^2 by 2 w (y(q) - mu_y) and
// s_xy by w (x(q) - mu_x).  Writing y(q) - mu_y = (y(q) - s) - (mu_y - s) for
// a fixed shift s (L/2), the contribution of window p to dQ/dy(q) is
//   w(q - p) [A(p) + (y(q) - s) B(p) + (x(q) - s) C(p)]
// with A = D_mu - 2 (mu_y - s) D_sy - (mu_x - s) D_sxy, B = 2 D_sy, C = D_sxy.
// Row pitch (floats) of the coefficient planes: OW rounded up to 4 so rows
// start on 16-byte boundaries.
__host__ __device__ inline int64_t coef_ld(int64_t OW) { return (OW + 3) & ~(int64_t)3; }

struct CoefOut {
    float *coef;   // nullable: A, B, C planes (OH rows x coef_ld(OW)), image b at coef + 3*b*OH*coef_ld(OW)
    int which;     // 0: Q, 1: cs
    float sx, sy;  // shifts
};

__device__ __forceinline__ void ssim_coef(float ux, float uy, float A1, float B1, float A2, float B2,
                                          int which, float sx, float sy, float &a, float &b, float &c) {
    const float iB1 = __fdividef(1.f, B1), iB2 = __fdividef(1.f, B2);
    const float l = A1 * iB1, cs = A2 * iB2;
    float dmu, dvy, dcv;
    if (which == 0) {
        dmu = cs * 2.f * fmaf(-uy, l, ux) * iB1;
        dvy = -l * cs * iB2;
        dcv = 2.f * l * iB2;
    } else {
        dmu = 0.f;
        dvy = -cs * iB2;
        dcv = 2.f * iB2;
    }
    a = dmu - 2.f * (uy - sy) * dvy - (ux - sx) * dcv;
    b = 2.f * dvy;
    c = dcv;
}

// ---------------------------------------------------------------- block reduction

// Sum two doubles over the CTA; the result is valid in thread 0.
// `scratch` must hold 2 * (blockDim.x / 32) doubles.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        scratch[2 * warp] = a;
        scratch[2 * warp + 1] = b;
    }
    __syncthreads();
    if (warp == 0) {
        a = lane < nw ? scratch[2 * lane] : 0.0;
        b = lane < nw ? scratch[2 * lane + 1] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// ---------------------------------------------------------------- launch API (internal)

// Fast 11-tap stride-1 path (k_gauss.cu).  Writes per-item partial sums
// (sum Q, sum cs) to `partials`; optionally the Q map and, for MS-SSIM, the
// 2x2-average downsampled pair (float) of the input.
struct GaussLaunch {
    ImgDesc x, y;
    int dtype;          // gbssim_dtype of x / y
    int count;
    float *map;         // nullable
    int64_t map_ld, map_is;
    float *ds_x, *ds_y; // nullable: downsampled outputs ((H/2) x (W/2), dense)
    double2 *partials;  // items: count * strips * segments
    Taps<11> taps;
    Taps2<11> taps2;    // filled by the launcher from `taps`
    SsimConst c;
    int seg_rows;       // output rows per work item (multiple of 16)
    bool vec;           // x/y rows aligned for 4-element vector loads (set by the launcher)
    CoefOut co;         // backward: coefficient maps instead of (besides) pooling
};
int gauss11_items(int64_t H, int64_t W, int seg_rows, int *strips, int *segs);
// Strip width (output columns per work item) of the persistent MS-SSIM
// kernel of equally sized images, and its strips per image of width W.
constexpr int kUniformTW = 64;
inline int uniform_strips(int64_t W) { return (int)((W - 10 + kUniformTW - 1) / kUniformTW); }
cudaError_t launch_gauss11(const GaussLaunch &L, cudaStream_t st);

// Ragged persistent batch (k_gauss.cu).  Device tables built by the host
// plan; offsets are relative to the run's workspace base `ws`.
struct BatchLevel {
    const void *x, *y;      // level 0: the caller's planes
    int64_t x_off;          // levels >= 1: x plane (then y plane) in the workspace
    int64_t H, W, rs;
    int64_t ds_off;         // next level's planes in the workspace, -1 at the last level
    int64_t part_off;       // this (image, level)'s item slots in the workspace
    int level, strips, segs, seg_rows, items, vec;
    int wait_target;        // completion count dependants wait for (= items)
    int pad;
};
struct BatchItem {
    int level_index;        // into the BatchLevel array (image-major: image * scales + level)
    int strip, seg, pad;
};
struct BatchTable {
    const BatchLevel *levels;
    const BatchItem *items;
    void *ws;
    int64_t counter_off, done_off, status_off;
    int total_items, n_images, scales, dtype;
    int tile_w;  // strip width of the kernel: 32, 64 or 128 output columns (4 x that many threads a CTA)
    unsigned wait_limit;
};
cudaError_t launch_batch(const BatchTable &B, const Taps<11> &taps, SsimConst cc, int grid, cudaStream_t st);

// Equally sized images (gbssim_msssim's persistent path): no table, the item
// list is arithmetic; offsets are into gbssim_msssim's workspace.
struct UniformLevel {
    int64_t H, W;
    int strips, segs, seg_rows, items_per_image, vec, pad;
    int64_t item_begin;   // first item of this level (level-major order)
    int64_t x_off;        // levels >= 1: x planes of all images, then y planes
    int64_t pitch;        // levels >= 1: row pitch of those planes, in elements
    int64_t part_off;     // pooling slots: image-major, items_per_image each
};
constexpr int kUniformMaxGroups = 16;  // arrival flags (copy groups) of the streamed host mode
constexpr int kUniformMaxWaves = kUniformMaxGroups + GBSSIM_MAX_SCALES - 1;
struct UniformBatch {
    const void *x, *y;
    int64_t rs, image_stride;  // level 0, in elements
    int dtype, count, scales;
    // 1: uint8 input with at most 5 scales; levels >= 1 are uint16 planes
    // holding 4^j times the level's values (exact), row pitch a multiple of
    // 8, read by bulk tensor copies.  0: fp32 planes of the 2x2 means.
    int ipyr;
    // levels j < cs_only_levels pool only mean cs (their mean Q is not
    // asked for: MS-SSIM without per-scale output), the rest both
    int cs_only_levels;
    UniformLevel lv[GBSSIM_MAX_SCALES];
    int64_t total_items;
    void *ws;
    int64_t counter_off, done_off, status_off;
    unsigned wait_limit;
    // nullable: level-0 items of the images of copy group g (images
    // group_begin[g] .. group_begin[g + 1] - 1) wait (bounded) until
    // arrive[g] != 0
    const unsigned *arrive;
    int group_begin[kUniformMaxGroups + 1];
    // waves > 0 (with arrive): items in copy-group wavefront order, wave w
    // holding level j of group w - j for every level (groups of group_begin
    // images); wave_begin[w] is its first item.  waves == 0: level-major.
    int waves, groups;
    int wave_begin[kUniformMaxWaves + 1];
};
cudaError_t launch_uniform(const UniformBatch &U, const Taps<11> &taps, SsimConst cc, int grid, cudaStream_t st);
int gauss11_batch_max_ctas_per_sm(int dtype, bool table, int tile_w = 64);
struct BatchFinalize {
    const BatchLevel *levels;
    const void *ws;
    int n_images, scales, combine;
    double exps[GBSSIM_MAX_SCALES];
    double *score_out, *per_scale_out;
};
cudaError_t launch_finalize_batch(const BatchFinalize &F, cudaStream_t st);

// Generic path: any k <= GBSSIM_MAX_K, any stride, separable taps.
struct GenericLaunch {
    ImgDesc x, y;
    int dtype, count, k, stride;
    float *map;
    int64_t map_ld, map_is;
    double2 *partials;  // items: count * tiles
    TapsDyn taps;
    SsimConst c;
    CoefOut co;
};
int generic_items(int64_t OH, int64_t OW);
cudaError_t launch_generic(const GenericLaunch &L, cudaStream_t st);

// Exact integer box path for uint8 (k_box.cu).
struct BoxLaunch {
    ImgDesc x, y;
    int count, k, stride;
    float *map;
    int64_t map_ld, map_is;
    double2 *partials;  // nullable when sums_out is set
    int64_t *sums_out;  // nullable: 5 int64 per window position
    float C1k4, C2k4;   // C1 * k^4, C2 * k^4
    bool use_tma;       // stride-4 aligned tiles through bulk tensor copies
};
int box_items_ks(int64_t OH, int64_t OW, int k, int s);  // workspace sizing (max over layouts)
bool box_aligned16(const ImgDesc &x, const ImgDesc &y);
int box_path_items(int64_t OH, int64_t OW, int k, int s, bool aligned16, bool tma);  // items of the layout launched
cudaError_t launch_box_u8(const BoxLaunch &L, cudaStream_t st);

// 2x2 average downsample of a batch into dense float planes (k_pool.cu).
cudaError_t launch_downsample(const ImgDesc &in, int dtype, int count, float *out,
                              cudaStream_t st);

// Finalisers (k_pool.cu): deterministic fp64 combination of per-item partials.
cudaError_t launch_finalize_ssim(const double2 *partials, int count, int items_per_image,
                                 double inv_n, double *mean_out, cudaStream_t st);
struct MsLevelInfo {
    const double2 *partials;
    int items_per_image;
    double inv_n;
};
struct MsFinalize {
    MsLevelInfo lv[GBSSIM_MAX_SCALES];
    double exps[GBSSIM_MAX_SCALES];
    int scales, count, combine;
    double *score_out, *per_scale_out;
};
cudaError_t launch_finalize_msssim(const MsFinalize &F, cudaStream_t st);
// Backward gradient pass (k_bwd.cu): full correlation of the coefficient
// maps with the window, combined with the images, plus the 2x2-average
// adjoint of the next coarser level.
struct GradLaunch {
    ImgDesc x, y;          // this level's images
    int dtype, count, k;
    const float *coef;     // A, B, C planes of this level (dense OH x OW)
    TapsDyn taps;
    float sx, sy;
    double base_scale;     // grad_scale / (number of map elements of this level)
    const double *grad_out; // nullable device factor(s)
    int grad_out_per_image;
    const double *ms_score, *ms_per_scale;  // nullable: MS-SSIM forward results
    int ms_scales, ms_level, ms_combine;
    double ms_beta, ms_beta_hat;
    const float *coarse;   // nullable: gradient of the next coarser level, dense (H/2) x (W/2)
    void *out;
    int out_dtype;
    int64_t out_ld, out_is;
};
cudaError_t launch_grad(const GradLaunch &G, cudaStream_t st);

cudaError_t launch_video_pool(const double *sY, const double *sU, const double *sV, int n, const double w[3],
                              double pct, double r, double *frame_out, double *video_out, cudaStream_t st);
constexpr int kVideoMaxFrames = 4096;  // 32 KB of shared memory for the sort

// Pooling family on stored maps (k_poolmap.cu).
constexpr int kPoolMaxRanks = 10;  // order statistics one call selects (five-number summary: 5 x 2)
struct PoolLayout {
    int items;                          // row blocks per map
    size_t partials, center, state, hist;
    size_t fast, vhist, cand;           // value-bin selection: state, bin counts, candidates
    size_t bytes;
};
PoolLayout pool_layout(int64_t h, int64_t w, int count);
// SSIM-3D and MS-SSIM-3D (k_ssim3d.cu): k x k x kt rectangular windows over
// a uint8 video pair (level 0) or one float pyramid level of it (values times
// `scale` are exact integers); int32 or int64 ("wide") window sums.
constexpr int kSsim3dMaxK = 31;  // shared memory per CTA at k = 31: 98 KB (int32), 188 KB (int64)
struct Ssim3dLaunch {
    ImgDesc x, y;           // frames as images: count = T, image_stride = frame stride (elements)
    int T, k, kt;
    float *map;             // nullable: (T-kt+1) maps of Q, frames map_fs floats apart, rows map_ld
    int64_t map_ld, map_fs;
    double2 *partials;      // (T-kt+1) x tiles of (sum Q, sum cs)
    float scale;            // float levels: values times scale are exact integers (4^j at level j)
    float C1x2n2, C2x2n2;   // 2 C1 N^2, 2 C2 N^2 with N = k^2 kt (times scale^2 for a scaled level)
    bool vec4;              // data, row and frame strides allow 4-element vector loads
};
void ssim3d_tiles(int64_t H, int64_t W, int k, bool wide, int *tx, int *ty);
cudaError_t launch_ssim3d_level(const Ssim3dLaunch &L, bool u8_input, bool wide, cudaStream_t st);
// Per-frame combination of the levels' (frame, item) partials.
struct Ms3dFinalize {
    const double2 *partials[GBSSIM_MAX_SCALES];  // level j: frames x items[j] of (sum Q, sum cs)
    int items[GBSSIM_MAX_SCALES];
    double inv_n[GBSSIM_MAX_SCALES];             // 1 / positions of a frame at level j
    double exps[GBSSIM_MAX_SCALES];
    int scales, frames, combine;
};
// frame_scores: frames doubles (written); per_scale_out, score_out nullable.
cudaError_t launch_ssim3d_finalize(const Ms3dFinalize &F, double *frame_scores, double *per_scale_out,
                                   double *score_out, cudaStream_t st);

// Scale handling (k_scale.cu): Z x Z block means and the 9/7 wavelet pyramid step.
cudaError_t launch_block_mean(const ImgDesc &in, int dtype, int count, int z, float *out, int64_t out_ld,
                              int64_t out_is, cudaStream_t st);
cudaError_t launch_pyramid97(const ImgDesc &in, int dtype, int count, float *out, cudaStream_t st);
// Border extension into dense PH x PW planes of the same dtype (mode 0 zero,
// 1 mirror with the edge repeated).
cudaError_t launch_pad(const ImgDesc &in, int dtype, int count, void *out, int64_t PH, int64_t PW, int top,
                       int left, int mode, cudaStream_t st);
cudaError_t launch_rgb_ycbcr(const ImgDesc &r, const ImgDesc &g, const ImgDesc &b, int dtype, int count, float *y,
                             float *cb, float *cr, int64_t out_ld, int64_t out_is, cudaStream_t st);

// CMSSIM colour steps (k_colour.cu).  Planes are dense H x W floats; the
// three channels of a batch are separate arrays (channel stride cs).
cudaError_t launch_rgb_opp(const ImgDesc &r, const ImgDesc &g, const ImgDesc &b, int dtype, int count,
                           const double m[9], float *q1, float *q2, float *q3, cudaStream_t st);
cudaError_t launch_opp_lab(float *p1, float *p2, float *p3, int64_t n, const double inv[9], const double white[3],
                           cudaStream_t st);
cudaError_t launch_cmssim_weight(float *map, int64_t oh, int64_t ow, int64_t map_ld, int64_t map_is, int count,
                                 const float *lab_x, const float *lab_y, int64_t H, int64_t W, int64_t cs, int centre,
                                 int stride, cudaStream_t st);

// QSSIM (k_qssim.cu): the CTA band height, the workspace bytes and the launch
// (x, y: the three planes of each picture, one shape and dtype).
int64_t qssim_rows_per(int64_t H, int64_t W, int count);
size_t qssim_workspace(int dtype, int64_t H, int64_t W, int count);
cudaError_t launch_qssim(const ImgDesc x[3], const ImgDesc y[3], int dtype, int count, double C1, double C2, void *ws,
                         double *score, double *terms, cudaStream_t st);

// Temporal pooling of frame-score series (k_series.cu).
cudaError_t launch_series_pool(const double *scores, int n, int count, int64_t stride, int kind, double a0,
                               double a1, double *out, cudaStream_t st);
constexpr int kPoolLW = 100;       // internal kind: luminance-weighted pooling (aux = mu_1 map)
cudaError_t launch_pool_map(const float *map, int64_t h, int64_t w, int64_t ld, int count, int64_t is, int kind,
                            double a0, double a1, char *ws, double *out, cudaStream_t st, const float *aux = nullptr);
cudaError_t launch_local_mean(const ImgDesc &x, int dtype, int count, const TapsDyn &taps, int k, int s, float *out,
                              int64_t out_ld, int64_t out_is, cudaStream_t st);

}  // namespace gbssim
