// k_series.cu -- temporal pooling of frame-score series (Section
// "Spatio-temporal Aggregation of Quality Scores" of arXiv 2101.06354): the
// pooling kinds of the maps applied to a series of per-frame scores, plus the
// plain geometric and harmonic means and the windowed means (W-AM, W-GM,
// W-HM, W-CoV) over windows of k consecutive frames.
//
// One CTA per series, in fp64 (a series holds at most kVideoMaxFrames
// scores): the series and a bitonic-sorted copy sit in shared memory; sums
// are formed per thread over a fixed index set and combined by a fixed tree,
// so every result is deterministic.
#include "common.cuh"

namespace gbssim {
namespace {

constexpr int ST = 512;  // threads per series

// Deterministic CTA sum: fixed per-thread order, then a fixed smem tree.
__device__ double cta_sum(double v, double *red) {
    __syncthreads();
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = ST / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double pct_of(const double *sv, int n, double p) {
    const double h = p / 100.0 * (n - 1.0);
    const double fl = floor(h);
    const int lo = (int)fl;
    const int hi = lo + 1 < n ? lo + 1 : n - 1;
    return sv[lo] + (h - fl) * (sv[hi] - sv[lo]);
}

// Statistic of one window [t, t + k) for the windowed kinds.
__device__ double window_stat(const double *v, int t, int k, int kind) {
    double a = 0.0;
    switch (kind) {
    case GBSSIM_POOL_W_AM:
        for (int i = 0; i < k; ++i) a += v[t + i];
        return a / k;
    case GBSSIM_POOL_W_GM:
        for (int i = 0; i < k; ++i) a += log(v[t + i]);
        return exp(a / k);
    case GBSSIM_POOL_W_HM:
        for (int i = 0; i < k; ++i) a += 1.0 / v[t + i];
        return k / a;
    default: {  // GBSSIM_POOL_W_COV: population sigma over mean
        for (int i = 0; i < k; ++i) a += v[t + i];
        const double mu = a / k;
        double d = 0.0;
        for (int i = 0; i < k; ++i) d += (v[t + i] - mu) * (v[t + i] - mu);
        return sqrt(d / k) / mu;
    }
    }
}

__global__ void __launch_bounds__(ST) series_pool_kernel(const double *scores, int n, int64_t stride, int kind,
                                                         double a0, double a1, double *out) {
    extern __shared__ double sm[];  // v[n], then the sorted copy sv[P]
    __shared__ double red[ST];
    int P = 1;
    while (P < n) P <<= 1;
    double *v = sm, *sv = sm + n;
    const double *src = scores + (int64_t)blockIdx.x * stride;
    for (int i = threadIdx.x; i < P; i += ST) {
        const double x = i < n ? src[i] : INFINITY;
        if (i < n) v[i] = x;
        sv[i] = x;
    }
    __syncthreads();
    const bool order = kind == GBSSIM_POOL_PERCENTILE || kind == GBSSIM_POOL_MEDIAN || kind == GBSSIM_POOL_FNS ||
                       kind == GBSSIM_POOL_PP;
    if (order) {  // bitonic sort, ascending (+inf padding sinks to the end)
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += ST) {
                    const int l = i ^ j;
                    if (l > i) {
                        const double a = sv[i], b = sv[l];
                        if ((a > b) == ((i & k) == 0)) {
                            sv[i] = b;
                            sv[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
    }
    double res = 0.0;
    if (kind == GBSSIM_POOL_W_AM || kind == GBSSIM_POOL_W_GM || kind == GBSSIM_POOL_W_HM ||
        kind == GBSSIM_POOL_W_COV) {
        const int k = (int)a0, nw = n - k + 1;
        double loc = 0.0;
        for (int t = threadIdx.x; t < nw; t += ST) loc += window_stat(v, t, k, kind);
        res = cta_sum(loc, red) / nw;
    } else if (kind == GBSSIM_POOL_PERCENTILE || kind == GBSSIM_POOL_MEDIAN) {
        res = pct_of(sv, n, kind == GBSSIM_POOL_MEDIAN ? 50.0 : a0);
    } else if (kind == GBSSIM_POOL_FNS) {
        res = (pct_of(sv, n, 0.0) + pct_of(sv, n, 25.0) + pct_of(sv, n, 50.0) + pct_of(sv, n, 75.0) +
               pct_of(sv, n, 100.0)) / 5.0;
    } else {
        // moments: (a, b) per element, a second pass for the deviation kinds
        double mu = 0.0;
        if (kind == GBSSIM_POOL_COV || kind == GBSSIM_POOL_MD) {
            double loc = 0.0;
            for (int i = threadIdx.x; i < n; i += ST) loc += v[i];
            mu = cta_sum(loc, red) / n;
        }
        const double thr = kind == GBSSIM_POOL_PP ? pct_of(sv, n, a0) : 0.0;
        double la = 0.0, lb = 0.0;
        for (int i = threadIdx.x; i < n; i += ST) {
            const double q = v[i];
            switch (kind) {
            case GBSSIM_POOL_MEAN: la += q; break;
            case GBSSIM_POOL_COV: la += (q - mu) * (q - mu); break;
            case GBSSIM_POOL_MINKOWSKI: la += pow(1.0 - q, a0); break;
            case GBSSIM_POOL_DW: {
                const double w = pow(1.0 - q, a0);
                la += w * q;
                lb += w;
            } break;
            case GBSSIM_POOL_MD: la += pow(fabs(q - mu), a0); break;
            case GBSSIM_POOL_GM_DSSIM: la += log(1.0 - q); break;
            case GBSSIM_POOL_HM_DSSIM: la += 1.0 / (1.0 - q); break;
            case GBSSIM_POOL_GM: la += log(q); break;
            case GBSSIM_POOL_HM: la += 1.0 / q; break;
            default: la += q <= thr ? q / a1 : q; break;  // GBSSIM_POOL_PP
            }
        }
        const double sa = cta_sum(la, red), sb = cta_sum(lb, red);
        switch (kind) {
        case GBSSIM_POOL_COV: res = sqrt(sa / n) / mu; break;
        case GBSSIM_POOL_DW: res = sa / sb; break;
        case GBSSIM_POOL_MD: res = pow(pow(sa / n, 1.0 / a0), a1); break;
        case GBSSIM_POOL_GM_DSSIM:
        case GBSSIM_POOL_GM: res = exp(sa / n); break;
        case GBSSIM_POOL_HM_DSSIM:
        case GBSSIM_POOL_HM: res = n / sa; break;
        default: res = sa / n; break;  // MEAN, MINKOWSKI, PP
        }
    }
    if (threadIdx.x == 0) out[blockIdx.x] = res;
}

}  // namespace

size_t series_pool_smem(int n) {
    int P = 1;
    while (P < n) P <<= 1;
    return sizeof(double) * ((size_t)n + P);
}

cudaError_t launch_series_pool(const double *scores, int n, int count, int64_t stride, int kind, double a0,
                               double a1, double *out, cudaStream_t st) {
    const size_t smem = series_pool_smem(n);
    static DeviceOnce attr_set;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set.is_set(dev)) {
        const cudaError_t e = cudaFuncSetAttribute(series_pool_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)series_pool_smem(kVideoMaxFrames));
        if (e != cudaSuccess) return e;
        attr_set.set(dev);
    }
    series_pool_kernel<<<count, ST, smem, st>>>(scores, n, stride, kind, a0, a1, out);
    return cudaGetLastError();
}

}  // namespace gbssim
