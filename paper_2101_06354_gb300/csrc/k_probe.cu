// k_probe.cu -- FP32 fused multiply-add throughput probe.
//
// The Gaussian SSIM kernels are bound by FP32 arithmetic, not by memory, so
// their roofline is the GPU's FP32 FMA rate.  This kernel measures that rate
// instead of deriving it from unit counts: every thread runs 16 independent
// FMA chains (scalar FFMA) or 8 independent packed chains (FFMA2, two lanes
// per instruction), deep enough to hide the pipeline latency at full
// occupancy, and writes one value so nothing is optimised away.  The caller
// times a launch with CUDA events and divides the FLOP count the header
// states by the time.
#include "common.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeInner = 16;  // unrolled steps per iteration

template <bool PACKED>
__global__ void __launch_bounds__(kProbeThreads) ffma_probe_kernel(float *sink, int iters, float b, float c) {
    const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
    float s = 0.f;
    if (PACKED) {
        float2 a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = make_float2(seed + k, seed - k);
        const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kProbeInner; ++u)
#pragma unroll
                for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
    } else {
        float a[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = seed + k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kProbeInner; ++u)
#pragma unroll
                for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) s += a[k];
    }
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int gbssim_fp32_probe(int32_t packed, int32_t blocks, int32_t iters, float *sink, void *stream) {
    if (!sink || blocks < 1 || iters < 1) return GBSSIM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // b slightly below 1 and a small c keep every chain finite and normal
    if (packed) ffma_probe_kernel<true><<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.99999f, 1e-3f);
    else ffma_probe_kernel<false><<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.99999f, 1e-3f);
    return cudaGetLastError() == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}
