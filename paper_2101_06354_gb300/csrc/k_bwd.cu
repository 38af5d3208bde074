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
#include "tma.cuh"

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
    const int64_t cld = coef_ld(OW), plane = OH * cld;
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
        if (pr >= 0 && pr < OH && pc >= 0 && pc < OW) v = __ldg(coef + m * plane + pr * cld + pc);
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

// ------------------------------------------------------------ 11-tap strip kernel
//
// The same computation organised like the forward kernel: a CTA owns a strip
// of 64 gradient columns and a segment of rows and walks it in chunks of 16
// rows.  Gradient row q needs coefficient rows q-10..q; numbering coefficient
// rows from the segment start minus 10, output row t uses ring rows t..t+10,
// so each coefficient row is filtered horizontally once per segment.  The
// maps are staged with 16-byte asynchronous copies (cp.async, zero-filled
// outside the map), double-buffered so the next chunk's rows arrive while the
// current chunk is filtered.
constexpr int K11 = 11, H11 = K11 - 1;
constexpr int GCH = 16, GFIRST = GCH + H11;   // rows per chunk / first stage
constexpr int GRING = 32, GDUP = 10, GRROWS = GRING + GDUP;
constexpr int GQ = 20, GSW = 4 * GQ;          // staged quads / floats per row (columns c0-12 .. c0+67)

struct __align__(128) Grad11Smem {
    float st[3][GFIRST + GCH][GSW];   // staging: [map][row][col]; rows 0..25 buffer 0, 26..41 buffer 1
    float h[3][GRROWS][TW];           // ring of horizontal results
    unsigned long long bar[2];        // bulk-copy completion of buffers 0 and 1
};

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Issue the copies of NR coefficient rows starting at map row pr0 into
// staging rows row0..row0+NR-1 (all three maps).  NR is a compile-time
// constant so the task decomposition needs no integer division.
template <int NR>
__device__ __forceinline__ void stage_coef(Grad11Smem &S, const float *coef, int64_t plane, int64_t cld, int64_t OH,
                                           int64_t OW, int64_t pr0, int row0, int64_t pc0) {
    for (int t = threadIdx.x; t < 3 * NR * GQ; t += NT) {
        const int m = t / (NR * GQ), rem = t - m * NR * GQ;
        const int r = rem / GQ, q = rem - r * GQ;
        const int64_t pr = pr0 + r, pc = pc0 + 4 * q;
        int bytes = 0;
        const float *src = coef;
        if (pr >= 0 && pr < OH && pc >= 0 && pc < OW) {
            bytes = (int)(min((int64_t)4, OW - pc) * 4);
            src = coef + m * plane + pr * cld + pc;
        }
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(&S.st[m][row0 + r][4 * q])),
                     "l"(src), "r"(bytes)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Horizontal pass over staged rows row0..row0+NR-1 into ring rows (rel0 + r).
template <int NR>
__device__ __forceinline__ void grad_horizontal(Grad11Smem &S, int row0, int rel0, const TapsDyn &t) {
    for (int task = threadIdx.x; task < 3 * NR * (TW / 4); task += NT) {
        const int m = task / (NR * (TW / 4)), rem = task - m * NR * (TW / 4);
        const int r = rem >> 4, g4 = (rem & 15) * 4;
        float v[16];
        const float4 *src = reinterpret_cast<const float4 *>(&S.st[m][row0 + r][g4]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 a = src[k];
            v[4 * k] = a.x;
            v[4 * k + 1] = a.y;
            v[4 * k + 2] = a.z;
            v[4 * k + 3] = a.w;
        }
        // output column j = g4 + o (gradient column c0 + j) takes staged columns j + 2 .. j + 12:
        // h(j) = sum_n w(n) M(c0 + j - n), staged index j + 12 - n
        float h[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 2; i < 16; ++i)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int n = o + 12 - i;
                if (n >= 0 && n < K11) h[o] = fmaf(t.g[n], v[i], h[o]);
            }
        const int slot = (rel0 + r) & (GRING - 1);
        const float4 hv = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(&S.h[m][slot][g4]) = hv;
        if (slot < GDUP) *reinterpret_cast<float4 *>(&S.h[m][slot + GRING][g4]) = hv;
    }
}

// TMAS: the coefficient rows arrive as per-map 2-D tiles of bulk tensor
// copies (tmA: 26-row tiles for the first chunk, tmB: 16-row tiles) on two
// mbarriers, one thread issuing them; otherwise every thread issues 16-byte
// cp.async copies.  A bulk-copy wait that gives up writes NaN into the rest
// of the CTA's gradient, waits (bounded) for its copies in flight and returns.
template <typename T, typename G, bool TMAS>
__global__ void __launch_bounds__(NT, 3)
    grad11_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const GradLaunch L, int strips, int segs, int seg_rows) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Grad11Smem &S = *reinterpret_cast<Grad11Smem *>(smem_raw);
    __shared__ float fac;
    const int strip = blockIdx.x, seg = blockIdx.y, img = blockIdx.z;
    const int64_t H = L.x.H, W = L.x.W, OH = H - H11, OW = W - H11;
    const int64_t cld = coef_ld(OW), plane = OH * cld;
    const float *coef = L.coef + (int64_t)img * 3 * plane;
    const int64_t c0 = (int64_t)strip * TW, q0 = (int64_t)seg * seg_rows;
    const int64_t qend = min(q0 + (int64_t)seg_rows, H);
    const int nchunks = (int)((qend - q0 + GCH - 1) / GCH);
    const int64_t pr0 = q0 - H11, pc0 = c0 - 12;

    if (threadIdx.x == 0) {
        double f = L.base_scale;
        if (L.grad_out) f *= L.grad_out[L.grad_out_per_image ? img : 0];
        if (L.ms_score) {
            if (L.ms_combine == GBSSIM_COMBINE_SUM) {
                f *= L.ms_beta_hat;
            } else {
                const int Sc = L.ms_scales, j = L.ms_level;
                const double mv = L.ms_per_scale[((int64_t)img * Sc + j) * 2 + (j == Sc - 1 ? 1 : 0)];
                f *= L.ms_score[img] * L.ms_beta / mv;
            }
        }
        fac = (float)f;
    }
    // chunk c's staged rows: c == 0 rows 0..25; c >= 1 rows 0..15 (c even) or 26..41 (c odd)
    auto buf_row = [](int c) { return (c & 1) ? GFIRST : 0; };
    const T *xb = static_cast<const T *>(L.x.data) + img * L.x.image_stride;
    const T *yb = static_cast<const T *>(L.y.data) + img * L.y.image_stride;
    const int64_t Hh = H >> 1, Wh = W >> 1;
    const float *coarse = L.coarse ? L.coarse + (int64_t)img * Hh * Wh : nullptr;
    const int col = threadIdx.x & (TW - 1), grp = threadIdx.x >> 6;
    const int64_t qc = c0 + col;
    // bulk copies of chunk c (thread 0): its NR rows of the three maps
    auto issue = [&](int c) {
        const bool first = c == 0;
        const int row0 = first ? 0 : buf_row(c);
        const int pr = (int)(first ? pr0 : pr0 + GFIRST + (int64_t)GCH * (c - 1));
        unsigned long long *bar = &S.bar[c & 1];
        mbar_expect_tx(bar, 3u * (first ? GFIRST : GCH) * GSW * (unsigned)sizeof(float));
        for (int m = 0; m < 3; ++m) tma_load_3d(&S.st[m][row0][0], first ? &tmA : &tmB, (int)pc0, pr, img * 3 + m, bar);
    };
    // a wait gave up at chunk cf: NaN for this thread's outputs of chunks cf.., drain the copies in flight
    auto give_up = [&](int cf) {
        if (qc < W)
            for (int c = cf; c < nchunks; ++c)
                for (int o = 0; o < 4; ++o) {
                    const int64_t q = q0 + GCH * c + 4 * grp + o;
                    if (q < qend) store_grad<G>(L.out, img * L.out_is + q * L.out_ld + qc, nanf(""));
                }
        if (threadIdx.x == 0)
            for (int c = cf; c < nchunks && c < cf + 2; ++c) mbar_wait_bounded(&S.bar[c & 1], (c >> 1) & 1);
    };
    if constexpr (TMAS) {
        if (threadIdx.x == 0) {
            mbar_init(&S.bar[0], 1);
            mbar_init(&S.bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            issue(0);
            if (nchunks > 1) issue(1);
        }
        const bool ok = mbar_wait_bounded(&S.bar[0], 0);
        if (__syncthreads_or(!ok)) {
            give_up(0);
            return;
        }
    } else {
        stage_coef<GFIRST>(S, coef, plane, cld, OH, OW, pr0, 0, pc0);
        if (nchunks > 1) {
            stage_coef<GCH>(S, coef, plane, cld, OH, OW, pr0 + GFIRST, buf_row(1), pc0);
            asm volatile("cp.async.wait_group %0;" ::"n"(1) : "memory");  // chunk 0 landed, chunk 1 may fly
        } else {
            asm volatile("cp.async.wait_group %0;" ::"n"(0) : "memory");  // the only group must land
        }
        __syncthreads();
    }
    grad_horizontal<GFIRST>(S, 0, 0, L.taps);

    for (int c = 0; c < nchunks; ++c) {
        __syncthreads();  // ring rows of chunk c complete
        {
            const int base = GCH * c + 4 * grp;
            const int b0 = base & (GRING - 1);
            // this chunk's x, y (and coarse-level) values, loaded before the
            // vertical pass so their latency overlaps its arithmetic
            float xv[4], yv[4], cv[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int64_t q = q0 + base + o;
                xv[o] = yv[o] = cv[o] = 0.f;
                if (qc < W && q < qend) {
                    xv[o] = load_f32<T>(xb + q * L.x.row_stride + qc);
                    yv[o] = load_f32<T>(yb + q * L.y.row_stride + qc);
                    if (coarse && (q >> 1) < Hh && (qc >> 1) < Wh) cv[o] = coarse[(q >> 1) * Wh + (qc >> 1)];
                }
            }
            float acc[3][4];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int o = 0; o < 4; ++o) acc[m][o] = 0.f;
#pragma unroll
            for (int i = 0; i < 14; ++i) {
                const float va = S.h[0][b0 + i][col], vb = S.h[1][b0 + i][col], vc = S.h[2][b0 + i][col];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int n = o + H11 - i;
                    if (n >= 0 && n < K11) {
                        const float w = L.taps.g[n];
                        acc[0][o] = fmaf(w, va, acc[0][o]);
                        acc[1][o] = fmaf(w, vb, acc[1][o]);
                        acc[2][o] = fmaf(w, vc, acc[2][o]);
                    }
                }
            }
            const float f = fac;
            if (qc < W) {
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int64_t q = q0 + base + o;
                    if (q >= qend) break;
                    float gval = f * fmaf(yv[o] - L.sy, acc[1][o], fmaf(xv[o] - L.sx, acc[2][o], acc[0][o]));
                    if (coarse) gval = fmaf(0.25f, cv[o], gval);  // 0 outside the coarse level
                    store_grad<G>(L.out, img * L.out_is + q * L.out_ld + qc, gval);
                }
            }
        }
        if (c + 1 < nchunks) {
            if constexpr (TMAS) {
                // chunk c's buffer was last read by its horizontal pass, before this
                // iteration's first barrier: refill it with chunk c+2
                if (threadIdx.x == 0 && c + 2 < nchunks) {
                    fence_proxy_async_smem();
                    issue(c + 2);
                }
                const bool ok = mbar_wait_bounded(&S.bar[(c + 1) & 1], ((c + 1) >> 1) & 1);
                if (__syncthreads_or(!ok)) {  // chunk c+1 staged; ring rows of chunk c consumed
                    give_up(c + 1);
                    return;
                }
            } else {
                if (c + 2 < nchunks) {
                    stage_coef<GCH>(S, coef, plane, cld, OH, OW, pr0 + GFIRST + (int64_t)GCH * (c + 1),
                                    buf_row(c + 2), pc0);
                    asm volatile("cp.async.wait_group %0;" ::"n"(1) : "memory");
                } else {
                    asm volatile("cp.async.wait_group %0;" ::"n"(0) : "memory");
                }
                __syncthreads();  // chunk c+1 staged; ring rows of chunk c consumed
            }
            grad_horizontal<GCH>(S, buf_row(c + 1), GFIRST + GCH * c, L.taps);
        }
    }
}

template <typename T, typename G>
cudaError_t launch_grad11(const GradLaunch &L, cudaStream_t st) {
    static DeviceOnce attr_set;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set.is_set(dev)) {
        cudaError_t e = cudaFuncSetAttribute(grad11_kernel<T, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Grad11Smem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(grad11_kernel<T, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(Grad11Smem));
        if (e != cudaSuccess) return e;
        attr_set.set(dev);
    }
    // the three coefficient planes of every image as one 3-D tensor
    // (columns, rows, image * 3 + map); 80 x 26 and 80 x 16 float tiles
    const int64_t OH = L.x.H - H11, OW = L.x.W - H11, cld = coef_ld(OW);
    CUtensorMap tmA, tmB;
    memset(&tmA, 0, sizeof tmA);
    memset(&tmB, 0, sizeof tmB);
    bool tma = false;
    if (auto fn = tensor_map_encoder()) {
        const cuuint64_t dims[3] = {(cuuint64_t)OW, (cuuint64_t)OH, (cuuint64_t)(3 * L.count)};
        const cuuint64_t strides[2] = {(cuuint64_t)(cld * 4), (cuuint64_t)(OH * cld * 4)};
        const cuuint32_t boxA[3] = {GSW, GFIRST, 1}, boxB[3] = {GSW, GCH, 1}, estr[3] = {1, 1, 1};
        tma = (uintptr_t)L.coef % 16 == 0 &&
              fn(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(L.coef), dims, strides, boxA, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
              fn(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(L.coef), dims, strides, boxB, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const int strips = (int)((L.x.W + TW - 1) / TW);
    int seg_rows = 256;
    while (seg_rows > 32 && (int64_t)strips * ((L.x.H + seg_rows - 1) / seg_rows) * L.count < 4 * 456) seg_rows -= 32;
    const int segs = (int)((L.x.H + seg_rows - 1) / seg_rows);
    dim3 grid(strips, segs, L.count);
    if (tma)
        grad11_kernel<T, G, true><<<grid, NT, sizeof(Grad11Smem), st>>>(tmA, tmB, L, strips, segs, seg_rows);
    else
        grad11_kernel<T, G, false><<<grid, NT, sizeof(Grad11Smem), st>>>(tmA, tmB, L, strips, segs, seg_rows);
    return cudaGetLastError();
}

template <typename T, typename G>
cudaError_t launch_grad_tg(const GradLaunch &L, cudaStream_t st) {
    if (L.k == K11) return launch_grad11<T, G>(L, st);
    const int hk = L.k - 1;
    const size_t smem = sizeof(float) * (3 * (TH + hk) * (TW + hk) + 3 * (TH + hk) * TW);
    static DeviceOnce attr_set;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set.is_set(dev)) {
        cudaError_t e = cudaFuncSetAttribute(grad_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set.set(dev);
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
