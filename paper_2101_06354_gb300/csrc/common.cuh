// common.cuh -- device helpers and launch declarations shared by the gbssim
// kernels.  Internal to libgbssim.so; the public interface is include/gbssim.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbssim.h"

namespace gbssim {

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
};

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
};
int gauss11_items(int64_t H, int64_t W, int seg_rows, int *strips, int *segs);
cudaError_t launch_gauss11(const GaussLaunch &L, cudaStream_t st);

// Generic path: any k <= GBSSIM_MAX_K, any stride, separable taps.
struct GenericLaunch {
    ImgDesc x, y;
    int dtype, count, k, stride;
    float *map;
    int64_t map_ld, map_is;
    double2 *partials;  // items: count * tiles
    TapsDyn taps;
    SsimConst c;
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
};
int box_items_ks(int64_t OH, int64_t OW, int k, int s);
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
cudaError_t launch_pool_mean(const float *map, int64_t h, int64_t w, int64_t ld, int count,
                             int64_t image_stride, double2 *partials, double *out,
                             cudaStream_t st);
int pool_items(int64_t h, int64_t w);

}  // namespace gbssim
