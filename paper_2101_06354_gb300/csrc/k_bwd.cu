// k_bwd.cu -- gradient of pooled SSIM / MS-SSIM with respect to the
// distorted image.
//
// The forward kernels, run in coefficient mode, recompute the window moments
// and write three maps per window position p (common.cuh, ssim_coef):
//   A(p), B(p), C(p)  with  d score / d y(q) = f * sum_p w(q - p) [A(p) + (y(q) - s) B(p) + (x(q) - s) C(p)],
// the sum running over the positions p whose window covers q, f the pooling
// factor (1 / number of map elements, times the MS-SSIM chain factor and the
// caller's scale).  This kernel evaluates the three sums as full correlations
// of the zero-extended maps with the window (two separable passes through
// shared memory), combines them with x(q), y(q), and adds a quarter of the
// next coarser level's gradient at (q/2): the adjoint of 2x2 average pooling.
#include "common.cuh"

namespace gbssim {
namespace {

constexpr int NT = 256;
constexpr int TH = 32, TW = 64;  // gradient pixels per CTA tile

template <typename T>
__device__ __forceinline__ void store_grad(void *out, int64_t idx, float v);
template <>
__device__ __forceinline__ void store_grad<float>(void *out, int64_t idx, float v) {
    static_cast<float *>(out)[idx] = v;
}
template <>
__device__ __forceinline__ void store_grad<__half>(void *out, int64_t idx, float v) {
    static_cast<__half *>(out)[idx] = __float2half_rn(v);
}
template <>
__device__ __forceinline__ void store_grad<__nv_bfloat16>(void *out, int64_t idx, float v) {
    static_cast<__nv_bfloat16 *>(out)[idx] = __float2bfloat16_rn(v);
}

template <typename T, typename G>
__global__ void __launch_bounds__(NT) grad_kernel(const GradLaunch L) {
    extern __shared__ __align__(16) float sm[];
    const int k = L.k, hk = k - 1;
    const int RH = TH + hk, RW = TW + hk;   // coefficient tile with the leading halo
    float *raw = sm;                        // [3][RH][RW]
    float *hor = sm + 3 * RH * RW;          // [3][RH][TW]
    __shared__ float fac;

    const int img = blockIdx.z;
    const int64_t H = L.x.H, W = L.x.W, OH = H - hk, OW = W - hk;
    const int64_t r0 = (int64_t)blockIdx.y * TH, c0 = (int64_t)blockIdx.x * TW;
    const int64_t plane = OH * OW;
    const float *coef = L.coef + (int64_t)img * 3 * plane;

    if (threadIdx.x == 0) {
        double f = L.base_scale;
        if (L.grad_out) f *= (double)L.grad_out[L.grad_out_per_image ? img : 0];
        if (L.ms_score) {
            if (L.ms_combine == GBSSIM_COMBINE_SUM) {
                f *= L.ms_beta_hat;
            } else {
                const int S = L.ms_scales, j = L.ms_level;
                const double m = L.ms_per_scale[((int64_t)img * S + j) * 2 + (j == S - 1 ? 1 : 0)];
                f *= L.ms_score[img] * L.ms_beta / m;
            }
        }
        fac = (float)f;
    }
    // stage A, B, C for positions [r0 - hk, r0 + TH) x [c0 - hk, c0 + TW), zero outside the map
    for (int t = threadIdx.x; t < 3 * RH * RW; t += NT) {
        const int m = t / (RH * RW), rem = t - m * RH * RW;
        const int r = rem / RW, c = rem - r * RW;
        const int64_t pr = r0 - hk + r, pc = c0 - hk + c;
        float v = 0.f;
        if (pr >= 0 && pr < OH && pc >= 0 && pc < OW) v = __ldg(coef + m * plane + pr * OW + pc);
        raw[t] = v;
    }
    __syncthreads();
    // horizontal: hor[m][r][c] = sum_n w(n) raw[m][r][c + hk - n]
    for (int t = threadIdx.x; t < 3 * RH * TW; t += NT) {
        const int m = t / (RH * TW), rem = t - m * RH * TW;
        const int r = rem / TW, c = rem - r * TW;
        const float *src = raw + (m * RH + r) * RW + c + hk;
        float acc = 0.f;
        for (int n = 0; n < k; ++n) acc = fmaf(L.taps.g[n], src[-n], acc);
        hor[t] = acc;
    }
    __syncthreads();
    // vertical + combine, one gradient pixel per thread-iteration
    const T *xb = static_cast<const T *>(L.x.data) + img * L.x.image_stride;
    const T *yb = static_cast<const T *>(L.y.data) + img * L.y.image_stride;
    const int64_t Hh = H >> 1, Wh = W >> 1;
    const float *coarse = L.coarse ? L.coarse + (int64_t)img * Hh * Wh : nullptr;
    const float f = fac;
    for (int t = threadIdx.x; t < TH * TW; t += NT) {
        const int r = t / TW, c = t - r * TW;
        const int64_t q = r0 + r, qc = c0 + c;
        if (q >= H || qc >= W) continue;
        float ga = 0.f, gb = 0.f, gc = 0.f;
        for (int m = 0; m < k; ++m) {
            const float w = L.taps.g[m];
            const int rr = r + hk - m;
            ga = fmaf(w, hor[(0 * RH + rr) * TW + c], ga);
            gb = fmaf(w, hor[(1 * RH + rr) * TW + c], gb);
            gc = fmaf(w, hor[(2 * RH + rr) * TW + c], gc);
        }
        const float xv = load_f32<T>(xb + q * L.x.row_stride + qc);
        const float yv = load_f32<T>(yb + q * L.y.row_stride + qc);
        float gval = f * fmaf(yv - L.sy, gb, fmaf(xv - L.sx, gc, ga));
        if (coarse && (q >> 1) < Hh && (qc >> 1) < Wh) gval = fmaf(0.25f, coarse[(q >> 1) * Wh + (qc >> 1)], gval);
        store_grad<G>(L.out, img * L.out_is + q * L.out_ld + qc, gval);
    }
}

// ------------------------------------------------------------ 11-tap specialisation
//
// Same computation, register-blocked: (A, B) travel as float2 pairs (packed
// f32x2 instructions), C as a scalar; each thread filters 4 adjacent columns
// of one row in the horizontal pass and 4 adjacent rows of one column in the
// vertical pass, so every shared-memory value loaded feeds up to 4 outputs.
constexpr int K11 = 11, H11 = K11 - 1;
constexpr int RH11 = TH + H11, RW11 = 4 * ((TW + H11 + 3) / 4);  // 42 x 76

struct __align__(16) Grad11Smem {
    float2 ab[RH11][RW11];
    float c[RH11][RW11];
    float2 hab[RH11][TW];
    float hc[RH11][TW];
};

template <typename T, typename G>
__global__ void __launch_bounds__(NT) grad11_kernel(const GradLaunch L, Taps2<K11> t2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Grad11Smem &S = *reinterpret_cast<Grad11Smem *>(smem_raw);
    __shared__ float fac;
    const int img = blockIdx.z;
    const int64_t H = L.x.H, W = L.x.W, OH = H - H11, OW = W - H11;
    const int64_t r0 = (int64_t)blockIdx.y * TH, c0 = (int64_t)blockIdx.x * TW;
    const int64_t plane = OH * OW;
    const float *coef = L.coef + (int64_t)img * 3 * plane;

    if (threadIdx.x == 0) {
        double f = L.base_scale;
        if (L.grad_out) f *= L.grad_out[L.grad_out_per_image ? img : 0];
        if (L.ms_score) {
            if (L.ms_combine == GBSSIM_COMBINE_SUM) {
                f *= L.ms_beta_hat;
            } else {
                const int Sc = L.ms_scales, j = L.ms_level;
                const double m = L.ms_per_scale[((int64_t)img * Sc + j) * 2 + (j == Sc - 1 ? 1 : 0)];
                f *= L.ms_score[img] * L.ms_beta / m;
            }
        }
        fac = (float)f;
    }
    // stage positions [r0 - 10, r0 + TH) x [c0 - 10, c0 + RW11 - 10), zero outside the map
    for (int t = threadIdx.x; t < RH11 * RW11; t += NT) {
        const int r = t / RW11, c = t - r * RW11;
        const int64_t pr = r0 - H11 + r, pc = c0 - H11 + c;
        float a = 0.f, b = 0.f, cc = 0.f;
        if (pr >= 0 && pr < OH && pc >= 0 && pc < OW) {
            const float *src = coef + pr * OW + pc;
            a = __ldg(src);
            b = __ldg(src + plane);
            cc = __ldg(src + 2 * plane);
        }
        S.ab[r][c] = make_float2(a, b);
        S.c[r][c] = cc;
    }
    __syncthreads();
    // horizontal: h(r, c) = sum_n w(n) M(r, c + 10 - n), 4 columns per task
    for (int task = threadIdx.x; task < RH11 * (TW / 4); task += NT) {
        const int r = task >> 4, g4 = (task & 15) * 4;
        float2 pab[14];
        float pc[14];
        const float4 *sab = reinterpret_cast<const float4 *>(&S.ab[r][g4]);
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const float4 v = sab[k];
            pab[2 * k] = make_float2(v.x, v.y);
            pab[2 * k + 1] = make_float2(v.z, v.w);
        }
        const float4 *sc = reinterpret_cast<const float4 *>(&S.c[r][g4]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = sc[k];
            pc[4 * k] = v.x;
            pc[4 * k + 1] = v.y;
            pc[4 * k + 2] = v.z;
            pc[4 * k + 3] = v.w;
        }
        {
            const float2 v = *reinterpret_cast<const float2 *>(&S.c[r][g4 + 12]);
            pc[12] = v.x;
            pc[13] = v.y;
        }
        float2 hab[4];
        float hc[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            hab[o] = make_float2(0.f, 0.f);
            hc[o] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 14; ++i)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int n = H11 + o - i;  // tap applied to column i for output o
                if (n >= 0 && n < K11) {
                    hab[o] = __ffma2_rn(t2.g2[n], pab[i], hab[o]);
                    hc[o] = fmaf(t2.g2[n].x, pc[i], hc[o]);
                }
            }
        float4 *dab = reinterpret_cast<float4 *>(&S.hab[r][g4]);
        dab[0] = make_float4(hab[0].x, hab[0].y, hab[1].x, hab[1].y);
        dab[1] = make_float4(hab[2].x, hab[2].y, hab[3].x, hab[3].y);
        *reinterpret_cast<float4 *>(&S.hc[r][g4]) = make_float4(hc[0], hc[1], hc[2], hc[3]);
    }
    __syncthreads();
    // vertical + combine: 4 rows of one column per task
    const T *xb = static_cast<const T *>(L.x.data) + img * L.x.image_stride;
    const T *yb = static_cast<const T *>(L.y.data) + img * L.y.image_stride;
    const int64_t Hh = H >> 1, Wh = W >> 1;
    const float *coarse = L.coarse ? L.coarse + (int64_t)img * Hh * Wh : nullptr;
    const float f = fac;
    for (int task = threadIdx.x; task < TW * (TH / 4); task += NT) {
        const int c = task & (TW - 1), r4 = (task >> 6) * 4;
        float2 gab[4];
        float gc[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            gab[o] = make_float2(0.f, 0.f);
            gc[o] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 14; ++i) {
            const float2 v = S.hab[r4 + i][c];
            const float vc = S.hc[r4 + i][c];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int n = H11 + o - i;
                if (n >= 0 && n < K11) {
                    gab[o] = __ffma2_rn(t2.g2[n], v, gab[o]);
                    gc[o] = fmaf(t2.g2[n].x, vc, gc[o]);
                }
            }
        }
        const int64_t qc = c0 + c;
        if (qc >= W) continue;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int64_t q = r0 + r4 + o;
            if (q >= H) break;
            const float xv = load_f32<T>(xb + q * L.x.row_stride + qc);
            const float yv = load_f32<T>(yb + q * L.y.row_stride + qc);
            float gval = f * fmaf(yv - L.sy, gab[o].y, fmaf(xv - L.sx, gc[o], gab[o].x));
            if (coarse && (q >> 1) < Hh && (qc >> 1) < Wh) gval = fmaf(0.25f, coarse[(q >> 1) * Wh + (qc >> 1)], gval);
            store_grad<G>(L.out, img * L.out_is + q * L.out_ld + qc, gval);
        }
    }
}

template <typename T, typename G>
cudaError_t launch_grad11(const GradLaunch &L, cudaStream_t st) {
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(grad11_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Grad11Smem));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    Taps2<K11> t2;
    for (int n = 0; n < K11; ++n) t2.g2[n] = make_float2(L.taps.g[n], L.taps.g[n]);
    dim3 grid((unsigned)((L.x.W + TW - 1) / TW), (unsigned)((L.x.H + TH - 1) / TH), L.count);
    grad11_kernel<T, G><<<grid, NT, sizeof(Grad11Smem), st>>>(L, t2);
    return cudaGetLastError();
}

template <typename T, typename G>
cudaError_t launch_grad_tg(const GradLaunch &L, cudaStream_t st) {
    if (L.k == K11) return launch_grad11<T, G>(L, st);
    const int hk = L.k - 1;
    const size_t smem = sizeof(float) * (3 * (TH + hk) * (TW + hk) + 3 * (TH + hk) * TW);
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(grad_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    dim3 grid((unsigned)((L.x.W + TW - 1) / TW), (unsigned)((L.x.H + TH - 1) / TH), L.count);
    grad_kernel<T, G><<<grid, NT, smem, st>>>(L);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad_t(const GradLaunch &L, cudaStream_t st) {
    switch (L.out_dtype) {
    case GBSSIM_F32: return launch_grad_tg<T, float>(L, st);
    case GBSSIM_F16: return launch_grad_tg<T, __half>(L, st);
    case GBSSIM_BF16: return launch_grad_tg<T, __nv_bfloat16>(L, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_grad(const GradLaunch &L, cudaStream_t st) {
    switch (L.dtype) {
    case GBSSIM_U8: return launch_grad_t<uint8_t>(L, st);
    case GBSSIM_F16: return launch_grad_t<__half>(L, st);
    case GBSSIM_BF16: return launch_grad_t<__nv_bfloat16>(L, st);
    case GBSSIM_F32: return launch_grad_t<float>(L, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gbssim
