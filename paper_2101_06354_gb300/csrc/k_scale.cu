// k_scale.cu -- scale handling around SSIM / MS-SSIM (Section "Salient
// Features of SSIM and MS-SSIM Implementations", Section "Transforming across
// Various Scales" of arXiv 2101.06354): Z x Z block-mean downscaling (the
// automatic downscaling of the recommended implementation) and one step of
// the 9/7 biorthogonal wavelet pyramid (the LIBVMAF MS-SSIM variant).
// Both are light, memory-bound passes; one thread per output sample.
#include "common.cuh"

namespace gbssim {
namespace {

// Low-pass analysis filter of the CDF 9/7 wavelet (JPEG 2000 irreversible
// transform), taps -4..4, scaled to sum to one.
__constant__ float kCdf97[9] = {0.026748757410810f, -0.016864118442875f, -0.078223266528990f,
                                0.266864118442875f, 0.602949018236360f,  0.266864118442875f,
                                -0.078223266528990f, -0.016864118442875f, 0.026748757410810f};

template <typename T>
__global__ void block_mean_kernel(ImgDesc in, int z, float inv_zz, float *out, int64_t out_ld, int64_t out_is) {
    const int64_t oh = in.H / z, ow = in.W / z;
    const int img = blockIdx.z;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= ow || r >= oh) return;
    const T *b = static_cast<const T *>(in.data) + img * in.image_stride + r * z * in.row_stride + c * z;
    float s = 0.f;
    for (int m = 0; m < z; ++m)
        for (int n = 0; n < z; ++n) s += load_f32<T>(b + m * in.row_stride + n);
    out[img * out_is + r * out_ld + c] = s * inv_zz;
}

// Whole-sample symmetric extension: ... 2 1 | 0 1 .. n-1 | n-2 ...
__device__ __forceinline__ int64_t sym(int64_t i, int64_t n) {
    if (n == 1) return 0;
    const int64_t period = 2 * (n - 1);
    i %= period;
    if (i < 0) i += period;
    return i < n ? i : period - i;
}

// out(i, j) = sum_s h_s sum_t h_t in(2i + s, 2j + t), rows filtered first.
template <typename T>
__global__ void pyramid97_kernel(ImgDesc in, float *out) {
    const int64_t oh = in.H >> 1, ow = in.W >> 1;
    const int img = blockIdx.z;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= ow || i >= oh) return;
    const T *b = static_cast<const T *>(in.data) + img * in.image_stride;
    int64_t cols[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) cols[t] = sym(2 * j + t - 4, in.W);
    float acc = 0.f;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        const T *row = b + sym(2 * i + s - 4, in.H) * in.row_stride;
        float h = 0.f;
#pragma unroll
        for (int t = 0; t < 9; ++t) h = fmaf(kCdf97[t], load_f32<T>(row + cols[t]), h);
        acc = fmaf(kCdf97[s], h, acc);
    }
    out[img * oh * ow + i * ow + j] = acc;
}

// BT.709 luma and colour differences with the paper's coefficients.
template <typename T>
__global__ void rgb_ycbcr_kernel(ImgDesc r, ImgDesc g, ImgDesc b, float *yo, float *cbo, float *cro, int64_t out_ld,
                                 int64_t out_is) {
    const int img = blockIdx.z;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y;
    if (c >= r.W || row >= r.H) return;
    const float R = load_f32<T>(static_cast<const T *>(r.data) + img * r.image_stride + row * r.row_stride + c);
    const float G = load_f32<T>(static_cast<const T *>(g.data) + img * g.image_stride + row * g.row_stride + c);
    const float B = load_f32<T>(static_cast<const T *>(b.data) + img * b.image_stride + row * b.row_stride + c);
    const float Y = fmaf(0.213f, R, fmaf(0.715f, G, 0.072f * B));
    const int64_t o = img * out_is + row * out_ld + c;
    yo[o] = Y;
    cbo[o] = 0.539f * (B - Y);
    cro[o] = 0.635f * (R - Y);
}

// Border extension of a batch into dense planes (PH x PW per image): the
// source pixel at (r - top, c - left), or 0 outside the image (mode 0), or
// its mirror about the border with the edge repeated (mode 1; the host
// guarantees one reflection suffices).  Elements are copied as raw bits.
template <typename E>
__global__ void pad_kernel(ImgDesc in, E *out, int64_t PH, int64_t PW, int top, int left, int mode) {
    const int img = blockIdx.z;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= PW) return;
    int64_t sr = r - top, sc = c - left;
    bool inside = sr >= 0 && sr < in.H && sc >= 0 && sc < in.W;
    if (!inside && mode == 1) {
        sr = sr < 0 ? -1 - sr : (sr >= in.H ? 2 * in.H - 1 - sr : sr);
        sc = sc < 0 ? -1 - sc : (sc >= in.W ? 2 * in.W - 1 - sc : sc);
        inside = true;
    }
    E v = 0;
    if (inside) v = static_cast<const E *>(in.data)[img * in.image_stride + sr * in.row_stride + sc];
    out[((int64_t)img * PH + r) * PW + c] = v;
}

}  // namespace

cudaError_t launch_rgb_ycbcr(const ImgDesc &r, const ImgDesc &g, const ImgDesc &b, int dtype, int count, float *y,
                             float *cb, float *cr, int64_t out_ld, int64_t out_is, cudaStream_t st) {
    const dim3 grid((unsigned)((r.W + 127) / 128), (unsigned)r.H, count);
    switch (dtype) {
    case GBSSIM_U8: rgb_ycbcr_kernel<uint8_t><<<grid, 128, 0, st>>>(r, g, b, y, cb, cr, out_ld, out_is); break;
    case GBSSIM_F16: rgb_ycbcr_kernel<__half><<<grid, 128, 0, st>>>(r, g, b, y, cb, cr, out_ld, out_is); break;
    case GBSSIM_BF16: rgb_ycbcr_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(r, g, b, y, cb, cr, out_ld, out_is); break;
    case GBSSIM_F32: rgb_ycbcr_kernel<float><<<grid, 128, 0, st>>>(r, g, b, y, cb, cr, out_ld, out_is); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_block_mean(const ImgDesc &in, int dtype, int count, int z, float *out, int64_t out_ld,
                              int64_t out_is, cudaStream_t st) {
    const int64_t oh = in.H / z, ow = in.W / z;
    if (oh == 0 || ow == 0) return cudaSuccess;
    const dim3 grid((unsigned)((ow + 127) / 128), (unsigned)oh, count);
    const float inv = 1.f / (float)(z * z);
    switch (dtype) {
    case GBSSIM_U8: block_mean_kernel<uint8_t><<<grid, 128, 0, st>>>(in, z, inv, out, out_ld, out_is); break;
    case GBSSIM_F16: block_mean_kernel<__half><<<grid, 128, 0, st>>>(in, z, inv, out, out_ld, out_is); break;
    case GBSSIM_BF16: block_mean_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(in, z, inv, out, out_ld, out_is); break;
    case GBSSIM_F32: block_mean_kernel<float><<<grid, 128, 0, st>>>(in, z, inv, out, out_ld, out_is); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pyramid97(const ImgDesc &in, int dtype, int count, float *out, cudaStream_t st) {
    const int64_t oh = in.H >> 1, ow = in.W >> 1;
    if (oh == 0 || ow == 0) return cudaSuccess;
    const dim3 grid((unsigned)((ow + 127) / 128), (unsigned)oh, count);
    switch (dtype) {
    case GBSSIM_U8: pyramid97_kernel<uint8_t><<<grid, 128, 0, st>>>(in, out); break;
    case GBSSIM_F16: pyramid97_kernel<__half><<<grid, 128, 0, st>>>(in, out); break;
    case GBSSIM_BF16: pyramid97_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(in, out); break;
    case GBSSIM_F32: pyramid97_kernel<float><<<grid, 128, 0, st>>>(in, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pad(const ImgDesc &in, int dtype, int count, void *out, int64_t PH, int64_t PW, int top,
                       int left, int mode, cudaStream_t st) {
    if (PH > 65535 || count > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((PW + 255) / 256), (unsigned)PH, count);
    switch (dtype) {
    case GBSSIM_U8: pad_kernel<uint8_t><<<grid, 256, 0, st>>>(in, (uint8_t *)out, PH, PW, top, left, mode); break;
    case GBSSIM_F16:
    case GBSSIM_BF16: pad_kernel<uint16_t><<<grid, 256, 0, st>>>(in, (uint16_t *)out, PH, PW, top, left, mode); break;
    case GBSSIM_F32: pad_kernel<uint32_t><<<grid, 256, 0, st>>>(in, (uint32_t *)out, PH, PW, top, left, mode); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gbssim
