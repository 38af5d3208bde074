// k_qssim.cu -- QSSIM (Section "Quaternion SSIM" of arXiv 2101.06354).
//
// Each colour pixel is the pure quaternion q = r i + g j + b k.  The score
// needs, per picture pair, the mean quaternions mu_ref, mu_dis and four sums
// over the deviations ac = q - mu:
//   sum |ac_ref|^2, sum |ac_dis|^2, sum ac_ref . ac_dis, sum ac_ref x ac_dis,
// because for pure quaternions a conj(b) = a . b - a x b, so the quaternion
// correlation sum ac_ref conj(ac_dis) has the dot sum as its real part and
// minus the cross sum as its vector part.  Then
//   l  = |2 mu_ref conj(mu_dis) + C1| / (|mu_ref|^2 + |mu_dis|^2 + C1),
//   cs = |2 sigma_{ref,dis} + C2| / (sigma_ref^2 + sigma_dis^2 + C2),
// with sigma^2 = sum |ac|^2 / ((M-1)(N-1)) and sigma_{ref,dis} the
// correlation sum over (M-1)(N-1), and QSSIM = l cs (the product of the two
// moduli is the modulus of the product: both denominators are real).
//
// The whole picture is one statistic, so this is a reduction bound by HBM
// (6 planes read once).  uint8 pictures: one pass of exact integer sums (the
// 12 raw sums sum r, g, b of both pictures, sum |q|^2 of both, sum q_ref .
// q_dis, sum q_ref x q_dis), int32 per thread, int64 per warp, added into
// per-picture int64 totals with atomics (exact, so the order does not
// matter); the deviations' sums follow in fp64 from the exact totals
// (sum |ac|^2 = sum |q|^2 - |sum q|^2 / MN, ...).  Float pictures: two passes,
// the means first, then the deviations' sums around them; per-thread
// compensated fp32 sums, fp64 per CTA into fixed slots, added in a fixed
// order per picture (deterministic).
#include "common.cuh"

namespace gbssim {
namespace {

constexpr int QT = 256;

struct QssimPlanes {
    const void *x[3], *y[3];
    int64_t H, W, rs, is;
    int count, blocks;  // blocks: CTAs per picture, each a band of rows_per rows
    int64_t rows_per;
};

__device__ __forceinline__ void qssim_factors(const double mr[3], const double md[3], double srr, double sdd,
                                              double dot, const double cr[3], double inv_norm, double C1,
                                              double C2, double &l, double &cs) {
    const double d = mr[0] * md[0] + mr[1] * md[1] + mr[2] * md[2];
    const double c0 = mr[1] * md[2] - mr[2] * md[1], c1 = mr[2] * md[0] - mr[0] * md[2],
                 c2 = mr[0] * md[1] - mr[1] * md[0];
    const double ln = sqrt((2.0 * d + C1) * (2.0 * d + C1) + 4.0 * (c0 * c0 + c1 * c1 + c2 * c2));
    const double ld = (mr[0] * mr[0] + mr[1] * mr[1] + mr[2] * mr[2]) + (md[0] * md[0] + md[1] * md[1] + md[2] * md[2]) +
                      C1;
    const double re = 2.0 * dot * inv_norm + C2;
    const double v2 = 4.0 * inv_norm * inv_norm * (cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    l = ln / ld;
    cs = sqrt(re * re + v2) / ((srr + sdd) * inv_norm + C2);
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ uint8: exact sums

// isum: 12 int64 per picture (as unsigned, two's complement), zeroed first:
// [0..2] sum ref rgb, [3..5] sum dis rgb, [6] sum |ref|^2, [7] sum |dis|^2,
// [8] sum ref . dis, [9..11] sum ref x dis.
__global__ void __launch_bounds__(QT) qssim_u8_kernel(const QssimPlanes P, unsigned long long *isum) {
    const int img = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * P.rows_per;
    const int64_t r1 = min(P.H, r0 + P.rows_per);
    const uint8_t *xr = static_cast<const uint8_t *>(P.x[0]), *xg = static_cast<const uint8_t *>(P.x[1]),
                  *xb = static_cast<const uint8_t *>(P.x[2]);
    const uint8_t *yr = static_cast<const uint8_t *>(P.y[0]), *yg = static_cast<const uint8_t *>(P.y[1]),
                  *yb = static_cast<const uint8_t *>(P.y[2]);
    // each thread adds at most rows_per * ceil(W / QT) <= 8192 pixels: every
    // int32 sum stays below 8192 * 3 * 255^2 < 2^31
    int a[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) a[q] = 0;
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t base = (int64_t)img * P.is + r * P.rs;
        for (int64_t c = threadIdx.x; c < P.W; c += QT) {
            const int64_t o = base + c;
            const int pr = __ldg(xr + o), pg = __ldg(xg + o), pb = __ldg(xb + o);
            const int qr = __ldg(yr + o), qg = __ldg(yg + o), qb = __ldg(yb + o);
            a[0] += pr;
            a[1] += pg;
            a[2] += pb;
            a[3] += qr;
            a[4] += qg;
            a[5] += qb;
            a[6] += pr * pr + pg * pg + pb * pb;
            a[7] += qr * qr + qg * qg + qb * qb;
            a[8] += pr * qr + pg * qg + pb * qb;
            a[9] += pg * qb - pb * qg;
            a[10] += pb * qr - pr * qb;
            a[11] += pr * qg - pg * qr;
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const long long s = warp_sum<long long>((long long)a[q]);
        if (lane == 0 && s != 0) atomicAdd(isum + (int64_t)img * 12 + q, (unsigned long long)s);
    }
}

__global__ void qssim_u8_finalize(const unsigned long long *isum, int count, double npix, double inv_norm, double C1,
                                  double C2, double *score, double *terms) {
    const int img = blockIdx.x * blockDim.x + threadIdx.x;
    if (img >= count) return;
    double s[12];
    for (int q = 0; q < 12; ++q) s[q] = (double)(long long)isum[(int64_t)img * 12 + q];  // exact: |s| < 2^53
    const double mr[3] = {s[0] / npix, s[1] / npix, s[2] / npix}, md[3] = {s[3] / npix, s[4] / npix, s[5] / npix};
    const double srr = s[6] - (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) / npix;
    const double sdd = s[7] - (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]) / npix;
    const double dot = s[8] - (s[0] * s[3] + s[1] * s[4] + s[2] * s[5]) / npix;
    const double cr[3] = {s[9] - (s[1] * s[5] - s[2] * s[4]) / npix, s[10] - (s[2] * s[3] - s[0] * s[5]) / npix,
                          s[11] - (s[0] * s[4] - s[1] * s[3]) / npix};
    double l, cs;
    qssim_factors(mr, md, srr, sdd, dot, cr, inv_norm, C1, C2, l, cs);
    score[img] = l * cs;
    if (terms) {
        terms[2 * img] = l;
        terms[2 * img + 1] = cs;
    }
}

// ------------------------------------------------------------ float: two passes

struct KSumF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float get() const { return s - c; }
};

// Six per-thread values reduced over the CTA (fp32 tree in the warp, fp64
// across warps) and written to part[0..5] by thread 0.
__device__ __forceinline__ void block_sum6(const float (&v)[6], double *part) {
    __shared__ double red[QT / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float s = warp_sum<float>(v[q]);
        if (lane == 0) red[warp][q] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int w = 0; w < QT / 32; ++w) t += red[w][threadIdx.x];
        part[threadIdx.x] = t;
    }
}

// PASS 0: sums of the six channels; PASS 1: the deviations' sums around the
// means (|ac_ref|^2, |ac_dis|^2, ac_ref . ac_dis, ac_ref x ac_dis).
template <typename T, int PASS>
__global__ void __launch_bounds__(QT) qssim_float_kernel(const QssimPlanes P, const double *means, double *part) {
    const int img = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * P.rows_per;
    const int64_t r1 = min(P.H, r0 + P.rows_per);
    float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (PASS == 1)
#pragma unroll
        for (int q = 0; q < 6; ++q) m[q] = (float)means[(int64_t)img * 6 + q];
    KSumF acc[6];
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t base = (int64_t)img * P.is + r * P.rs;
        for (int64_t c = threadIdx.x; c < P.W; c += QT) {
            const int64_t o = base + c;
            float v[6];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                v[ch] = load_f32<T>(static_cast<const T *>(P.x[ch]) + o) - m[ch];
                v[3 + ch] = load_f32<T>(static_cast<const T *>(P.y[ch]) + o) - m[3 + ch];
            }
            if (PASS == 0) {
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[q].add(v[q]);
            } else {
                acc[0].add(fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2])));
                acc[1].add(fmaf(v[3], v[3], fmaf(v[4], v[4], v[5] * v[5])));
                acc[2].add(fmaf(v[0], v[3], fmaf(v[1], v[4], v[2] * v[5])));
                acc[3].add(fmaf(v[1], v[5], -v[2] * v[4]));
                acc[4].add(fmaf(v[2], v[3], -v[0] * v[5]));
                acc[5].add(fmaf(v[0], v[4], -v[1] * v[3]));
            }
        }
    }
    float t[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) t[q] = acc[q].get();
    block_sum6(t, part + ((int64_t)img * P.blocks + blockIdx.x) * 6);
}

// Per picture, the CTA partials added in slot order.  PASS 0 writes the means;
// PASS 1 the score (and the two factors).
template <int PASS>
__global__ void qssim_float_finalize(const double *part, int count, int blocks, double npix, double inv_norm,
                                     double C1, double C2, double *means, double *score, double *terms) {
    const int img = blockIdx.x * blockDim.x + threadIdx.x;
    if (img >= count) return;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < blocks; ++b)
        for (int q = 0; q < 6; ++q) s[q] += part[((int64_t)img * blocks + b) * 6 + q];
    if (PASS == 0) {
        for (int q = 0; q < 6; ++q) means[(int64_t)img * 6 + q] = s[q] / npix;
        return;
    }
    const double *mu = means + (int64_t)img * 6;
    const double mr[3] = {mu[0], mu[1], mu[2]}, md[3] = {mu[3], mu[4], mu[5]}, cr[3] = {s[3], s[4], s[5]};
    double l, cs;
    qssim_factors(mr, md, s[0], s[1], s[2], cr, inv_norm, C1, C2, l, cs);
    score[img] = l * cs;
    if (terms) {
        terms[2 * img] = l;
        terms[2 * img + 1] = cs;
    }
}

template <typename T>
cudaError_t run_float(const QssimPlanes &P, double npix, double inv_norm, double C1, double C2, double *part,
                      double *means, double *score, double *terms, cudaStream_t st) {
    const dim3 grid(P.blocks, P.count);
    const int fb = (P.count + 127) / 128;
    qssim_float_kernel<T, 0><<<grid, QT, 0, st>>>(P, nullptr, part);
    qssim_float_finalize<0><<<fb, 128, 0, st>>>(part, P.count, P.blocks, npix, inv_norm, C1, C2, means, nullptr,
                                                nullptr);
    qssim_float_kernel<T, 1><<<grid, QT, 0, st>>>(P, means, part);
    qssim_float_finalize<1><<<fb, 128, 0, st>>>(part, P.count, P.blocks, npix, inv_norm, C1, C2, means, score,
                                                terms);
    return cudaGetLastError();
}

}  // namespace

// Rows per CTA band: enough CTAs to fill the GPU (about 8 per SM over the
// batch) but at most 8192 pixels per thread (the uint8 path's int32 bound).
int64_t qssim_rows_per(int64_t H, int64_t W, int count) {
    const int64_t cols = (W + QT - 1) / QT;
    int64_t cap = 8192 / cols;
    if (cap < 1) cap = 1;
    int64_t want = (H * count + 1215) / 1216;
    if (want < 1) want = 1;
    return want < cap ? want : cap;
}

size_t qssim_workspace(int dtype, int64_t H, int64_t W, int count) {
    if (dtype == GBSSIM_U8) return sizeof(unsigned long long) * 12 * (size_t)count;
    const int64_t rp = qssim_rows_per(H, W, count), blocks = (H + rp - 1) / rp;
    return sizeof(double) * 6 * (size_t)count * ((size_t)blocks + 1);
}

cudaError_t launch_qssim(const ImgDesc x[3], const ImgDesc y[3], int dtype, int count, double C1, double C2,
                         void *ws, double *score, double *terms, cudaStream_t st) {
    QssimPlanes P;
    for (int c = 0; c < 3; ++c) {
        P.x[c] = x[c].data;
        P.y[c] = y[c].data;
    }
    P.H = x[0].H;
    P.W = x[0].W;
    P.rs = x[0].row_stride;
    P.is = x[0].image_stride;
    P.count = count;
    P.rows_per = qssim_rows_per(P.H, P.W, count);
    P.blocks = (int)((P.H + P.rows_per - 1) / P.rows_per);
    const double npix = (double)P.H * (double)P.W;
    const double inv_norm = 1.0 / ((double)(P.H - 1) * (double)(P.W - 1));
    if (dtype == GBSSIM_U8) {
        unsigned long long *isum = static_cast<unsigned long long *>(ws);
        cudaError_t e = cudaMemsetAsync(isum, 0, sizeof(unsigned long long) * 12 * (size_t)count, st);
        if (e != cudaSuccess) return e;
        qssim_u8_kernel<<<dim3(P.blocks, count), QT, 0, st>>>(P, isum);
        qssim_u8_finalize<<<(count + 127) / 128, 128, 0, st>>>(isum, count, npix, inv_norm, C1, C2, score, terms);
        return cudaGetLastError();
    }
    double *means = static_cast<double *>(ws);
    double *part = means + 6 * (size_t)count;
    switch (dtype) {
    case GBSSIM_F16: return run_float<__half>(P, npix, inv_norm, C1, C2, part, means, score, terms, st);
    case GBSSIM_BF16: return run_float<__nv_bfloat16>(P, npix, inv_norm, C1, C2, part, means, score, terms, st);
    case GBSSIM_F32: return run_float<float>(P, npix, inv_norm, C1, C2, part, means, score, terms, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gbssim
