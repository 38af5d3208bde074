// k_pool.cu -- pooling, pyramid and finalisation kernels.
//
//  * finalize_ssim / finalize_msssim: one CTA per image adds the per-item
//    partial sums of the SSIM kernels in a fixed order in fp64, so scores are
//    bit-reproducible, then forms MSSIM (mean pooling, Background section) or
//    MS-SSIM (product prod_j m_j^beta_j, or the normalised sum, with
//    m_j = mean cs_j below the coarsest scale and mean Q at the coarsest).
//  * downsample: dyadic 2x2 average pooling with floor size (the MS-SSIM
//    implementations of Daala, Scikit-Video and Tensorflow) for the paths
//    that do not fuse it into the level kernel.
//  * pool_mean: mean of a stored float map (gbssim_ssim_pool).
#include <math.h>

#include "common.cuh"

namespace gbssim {
namespace {

constexpr int NT = 256;

__global__ void __launch_bounds__(NT) finalize_ssim_kernel(const double2 *partials, int items,
                                                           double inv_n, double *mean_out) {
    __shared__ double red[2 * NT / 32];
    const double2 *p = partials + (int64_t)blockIdx.x * items;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < items; i += NT) {
        a += p[i].x;
        b += p[i].y;
    }
    block_sum2(a, b, red);
    if (threadIdx.x == 0) mean_out[blockIdx.x] = a * inv_n;
}

// One warp per scale: warp j adds level j's partials (fp64, fixed lane
// order), lane 0 forms the scale's factor, thread 0 combines the factors.
__global__ void __launch_bounds__(32 * GBSSIM_MAX_SCALES) finalize_msssim_kernel(const MsFinalize F) {
    __shared__ double term[GBSSIM_MAX_SCALES], mq[GBSSIM_MAX_SCALES], mcs[GBSSIM_MAX_SCALES];
    const int img = blockIdx.x, j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = F.scales;
    if (j < S) {
        const MsLevelInfo &lv = F.lv[j];
        const double2 *p = lv.partials + (int64_t)img * lv.items_per_image;
        double a = 0.0, b = 0.0;
        for (int i = lane; i < lv.items_per_image; i += 32) {
            a += p[i].x;
            b += p[i].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            mq[j] = a * lv.inv_n;
            mcs[j] = b * lv.inv_n;
            const double m = j == S - 1 ? mq[j] : mcs[j];
            if (F.combine == GBSSIM_COMBINE_SUM) {
                double wsum = 0.0;
                for (int t = 0; t < S; ++t) wsum += F.exps[t];
                term[j] = F.exps[j] / wsum * m;
            } else {
                term[j] = pow(m, F.exps[j]);  // NaN for m < 0 under a non-integer exponent
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double score = F.combine == GBSSIM_COMBINE_SUM ? 0.0 : 1.0;
        for (int t = 0; t < S; ++t) score = F.combine == GBSSIM_COMBINE_SUM ? score + term[t] : score * term[t];
        F.score_out[img] = score;
        if (F.per_scale_out)
            for (int t = 0; t < S; ++t) {
                F.per_scale_out[((int64_t)img * S + t) * 2] = mcs[t];
                F.per_scale_out[((int64_t)img * S + t) * 2 + 1] = mq[t];
            }
    }
}

// Ragged batch: one CTA per image, one warp per scale (item counts differ
// per image and level).
__global__ void __launch_bounds__(32 * GBSSIM_MAX_SCALES) finalize_batch_kernel(const BatchFinalize F) {
    __shared__ double term[GBSSIM_MAX_SCALES], mq[GBSSIM_MAX_SCALES], mcs[GBSSIM_MAX_SCALES];
    const int img = blockIdx.x, j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = F.scales;
    if (j < S) {
        const BatchLevel &lv = F.levels[img * S + j];
        const double2 *p = reinterpret_cast<const double2 *>(static_cast<const char *>(F.ws) + lv.part_off);
        double a = 0.0, b = 0.0;
        for (int i = lane; i < lv.items; i += 32) {
            a += p[i].x;
            b += p[i].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            const double inv_n = 1.0 / ((double)(lv.H - 10) * (double)(lv.W - 10));
            mq[j] = a * inv_n;
            mcs[j] = b * inv_n;
            const double m = j == S - 1 ? mq[j] : mcs[j];
            if (F.combine == GBSSIM_COMBINE_SUM) {
                double wsum = 0.0;
                for (int t = 0; t < S; ++t) wsum += F.exps[t];
                term[j] = F.exps[j] / wsum * m;
            } else {
                term[j] = pow(m, F.exps[j]);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double score = F.combine == GBSSIM_COMBINE_SUM ? 0.0 : 1.0;
        for (int t = 0; t < S; ++t) score = F.combine == GBSSIM_COMBINE_SUM ? score + term[t] : score * term[t];
        F.score_out[img] = score;
        if (F.per_scale_out)
            for (int t = 0; t < S; ++t) {
                F.per_scale_out[((int64_t)img * S + t) * 2] = mcs[t];
                F.per_scale_out[((int64_t)img * S + t) * 2 + 1] = mq[t];
            }
    }
}

// 8 consecutive elements as floats, zero past n: one 8- or 16-byte vector
// load when `vec` (the address is aligned for it), else element by element.
template <typename T>
__device__ __forceinline__ void load8(const T *p, int n, bool vec, float (&v)[8]) {
    if (vec && n == 8) {
        if constexpr (sizeof(T) == 1) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                v[e] = (float)((w.x >> (8 * e)) & 255u);
                v[4 + e] = (float)((w.y >> (8 * e)) & 255u);
            }
            return;
        } else if constexpr (sizeof(T) == 4) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(p)), b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
            v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = e < n ? load_f32<T>(p + e) : 0.f;
}

// 2x2 averages, 4 outputs per thread; the sum order (a + b) + (c + d) of
// each 2x2 block is that of the scalar definition.
template <typename T>
__global__ void downsample_kernel(ImgDesc in, float *out, bool vec_in, bool vec_out) {
    const int64_t Hh = in.H >> 1, Wh = in.W >> 1;
    const int img = blockIdx.z;
    const int64_t C = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    const int64_t R = blockIdx.y;
    if (C >= Wh) return;
    const int n = (int)min((int64_t)4, Wh - C);
    const T *b = static_cast<const T *>(in.data) + img * in.image_stride + 2 * R * in.row_stride + 2 * C;
    float r0[8], r1[8];
    load8<T>(b, 2 * n, vec_in, r0);
    load8<T>(b + in.row_stride, 2 * n, vec_in, r1);
    float o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] = 0.25f * ((r0[2 * e] + r0[2 * e + 1]) + (r1[2 * e] + r1[2 * e + 1]));
    float *op = out + img * Hh * Wh + R * Wh + C;
    if (vec_out && n == 4) {
        *reinterpret_cast<float4 *>(op) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
        for (int e = 0; e < n; ++e) op[e] = o[e];
    }
}

}  // namespace

cudaError_t launch_finalize_ssim(const double2 *partials, int count, int items_per_image,
                                 double inv_n, double *mean_out, cudaStream_t st) {
    finalize_ssim_kernel<<<count, NT, 0, st>>>(partials, items_per_image, inv_n, mean_out);
    return cudaGetLastError();
}

cudaError_t launch_finalize_msssim(const MsFinalize &F, cudaStream_t st) {
    finalize_msssim_kernel<<<F.count, 32 * F.scales, 0, st>>>(F);
    return cudaGetLastError();
}

// Colour + temporal pooling of per-plane frame scores (one CTA): frame score
// F(t) = (wY S_Y + wU S_U + wV S_V) / (wY + wU + wV) (Section "Channel-wise
// SSIM"); temporal mean; p-th percentile of F with linear interpolation at
// h = p/100 (n-1) of the sorted scores; percentile pooling S_PP = mean of F
// with the scores at or below that percentile divided by r (Section
// "Percentile Pooling").  Sums run in a fixed tree order (deterministic).
constexpr int VP_THREADS = 1024;

__device__ double vp_block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(VP_THREADS) video_pool_kernel(const double *sY, const double *sU, const double *sV,
                                                                int n, double wY, double wU, double wV, double pct,
                                                                double r, double *frame_out, double *video_out) {
    extern __shared__ double sv[];  // P doubles, P = next power of two >= n
    __shared__ double red[32];
    int P = 1;
    while (P < n) P <<= 1;
    const double wsum = wY + wU + wV;
    double local = 0.0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        double f = INFINITY;
        if (i < n) {
            f = (wY * sY[i] + wU * sU[i] + wV * sV[i]) / wsum;
            if (frame_out) frame_out[i] = f;
            local += f;
        }
        sv[i] = f;
    }
    const double mean = vp_block_sum(local, red) / n;
    // bitonic sort, ascending
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const double a = sv[i], b = sv[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        sv[i] = b;
                        sv[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    const double h = pct / 100.0 * (n - 1);
    const int lo = (int)floor(h);
    const int hi = lo + 1 < n ? lo + 1 : n - 1;
    const double pv = sv[lo] + (h - lo) * (sv[hi] - sv[lo]);
    double lp = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lp += sv[i] <= pv ? sv[i] / r : sv[i];
    const double pp = vp_block_sum(lp, red) / n;
    if (threadIdx.x == 0) {
        video_out[0] = mean;
        video_out[1] = pv;
        video_out[2] = pp;
    }
}

cudaError_t launch_video_pool(const double *sY, const double *sU, const double *sV, int n, const double w[3],
                              double pct, double r, double *frame_out, double *video_out, cudaStream_t st) {
    int P = 1;
    while (P < n) P <<= 1;
    video_pool_kernel<<<1, VP_THREADS, sizeof(double) * P, st>>>(sY, sU, sV, n, w[0], w[1], w[2], pct, r, frame_out,
                                                                  video_out);
    return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const BatchFinalize &F, cudaStream_t st) {
    finalize_batch_kernel<<<F.n_images, 32 * F.scales, 0, st>>>(F);
    return cudaGetLastError();
}

cudaError_t launch_downsample(const ImgDesc &in, int dtype, int count, float *out,
                              cudaStream_t st) {
    const int64_t Hh = in.H >> 1, Wh = in.W >> 1;
    if (Hh == 0 || Wh == 0) return cudaSuccess;
    dim3 grid((unsigned)((Wh + 511) / 512), (unsigned)Hh, count);
    // vector loads: 8 u8 (8 B) or 8 f32 (2 x 16 B) at every even-column group
    // start, which is aligned when the base and both strides are
    const int64_t vb = dtype == GBSSIM_U8 ? 8 : dtype == GBSSIM_F32 ? 16 : 0;
    const int64_t es = dtype == GBSSIM_U8 ? 1 : dtype == GBSSIM_F32 ? 4 : 2;
    const bool vec_in = vb > 0 && (uintptr_t)in.data % vb == 0 && (in.row_stride * es) % vb == 0 &&
                        (in.image_stride * es) % vb == 0;
    const bool vec_out = (uintptr_t)out % 16 == 0 && Wh % 4 == 0;
    switch (dtype) {
    case GBSSIM_U8: downsample_kernel<uint8_t><<<grid, 128, 0, st>>>(in, out, vec_in, vec_out); break;
    case GBSSIM_F16: downsample_kernel<__half><<<grid, 128, 0, st>>>(in, out, false, vec_out); break;
    case GBSSIM_BF16: downsample_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(in, out, false, vec_out); break;
    case GBSSIM_F32: downsample_kernel<float><<<grid, 128, 0, st>>>(in, out, vec_in, vec_out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gbssim
