// k_colour.cu -- CMSSIM (Section "CMSSIM" of arXiv 2101.06354): the steps
// around the SSIM kernels.
//
//   rgb_opp_kernel    linear RGB in [0, 1] (uint8 / 255) -> CIE XYZ (BT.709 /
//                     sRGB primaries, D65) -> the luminance, red-green and
//                     blue-yellow planes Q1, Q2, Q3 (the section's forward
//                     matrix);
//   (Q2 and Q3 are then smoothed by the host driver: mirror extension plus
//    the Gaussian window's local mean, one output per pixel)
//   opp_lab_kernel    Q1, smoothed Q2, Q3 -> XYZ (the section's inverse
//                     matrix, as printed) -> CIE 1976 L*, a*, b* in place;
//   (the SSIM map of the L* planes comes from the SSIM kernels, L = 100)
//   weight_kernel     each map value times (1 - Delta E / 45), Delta E the
//                     CIELAB distance of the two images at the window's
//                     centre pixel.
#include "common.cuh"

namespace gbssim {
namespace {

// XYZ_TO_OPP x RGB_TO_XYZ, formed in double on the host.
struct Mat3 {
    float m[9];
};

template <typename T>
__device__ __forceinline__ float unit_value(const T *p);
template <>
__device__ __forceinline__ float unit_value<uint8_t>(const uint8_t *p) {
    return (float)__ldg(p) * (1.f / 255.f);
}
template <>
__device__ __forceinline__ float unit_value<float>(const float *p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ float unit_value<__half>(const __half *p) {
    return load_f32<__half>(p);
}
template <>
__device__ __forceinline__ float unit_value<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return load_f32<__nv_bfloat16>(p);
}

template <typename T>
__global__ void rgb_opp_kernel(ImgDesc r, ImgDesc g, ImgDesc b, Mat3 M, float *q1, float *q2, float *q3) {
    const int img = blockIdx.z;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y;
    if (c >= r.W) return;
    const float R = unit_value<T>(static_cast<const T *>(r.data) + img * r.image_stride + row * r.row_stride + c);
    const float G = unit_value<T>(static_cast<const T *>(g.data) + img * g.image_stride + row * g.row_stride + c);
    const float B = unit_value<T>(static_cast<const T *>(b.data) + img * b.image_stride + row * b.row_stride + c);
    const int64_t o = (img * r.H + row) * r.W + c;
    q1[o] = fmaf(M.m[0], R, fmaf(M.m[1], G, M.m[2] * B));
    q2[o] = fmaf(M.m[3], R, fmaf(M.m[4], G, M.m[5] * B));
    q3[o] = fmaf(M.m[6], R, fmaf(M.m[7], G, M.m[8] * B));
}

// CIE 1976 f(t): cube root above (6/29)^3, the linear segment below.
__device__ __forceinline__ float lab_f(float t) {
    const float d3 = 216.f / 24389.f;  // (6/29)^3
    return t > d3 ? cbrtf(t) : fmaf(t, 841.f / 108.f, 4.f / 29.f);  // t / (3 (6/29)^2) + 4/29
}

__global__ void opp_lab_kernel(float *p1, float *p2, float *p3, int64_t n, Mat3 inv, float3 white_inv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = p1[i], b = p2[i], c = p3[i];
    const float X = fmaf(inv.m[0], a, fmaf(inv.m[1], b, inv.m[2] * c));
    const float Y = fmaf(inv.m[3], a, fmaf(inv.m[4], b, inv.m[5] * c));
    const float Z = fmaf(inv.m[6], a, fmaf(inv.m[7], b, inv.m[8] * c));
    const float fx = lab_f(X * white_inv.x), fy = lab_f(Y * white_inv.y), fz = lab_f(Z * white_inv.z);
    p1[i] = fmaf(116.f, fy, -16.f);
    p2[i] = 500.f * (fx - fy);
    p3[i] = 200.f * (fy - fz);
}

// lx, ly: L*, a*, b* planes of each image, channel c of image n at
// c * cs + n * H * W.
__global__ void weight_kernel(float *map, int64_t oh, int64_t ow, int64_t map_ld, int64_t map_is, const float *lx,
                              const float *ly, int64_t H, int64_t W, int64_t cs, int centre, int stride) {
    const int img = blockIdx.z;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= ow) return;
    const int64_t p = img * H * W + (i * stride + centre) * W + j * stride + centre;
    const float dL = lx[p] - ly[p], da = lx[p + cs] - ly[p + cs], db = lx[p + 2 * cs] - ly[p + 2 * cs];
    const float de = sqrtf(fmaf(dL, dL, fmaf(da, da, db * db)));
    float *m = map + img * map_is + i * map_ld + j;
    *m *= 1.f - de * (1.f / 45.f);
}

}  // namespace

cudaError_t launch_rgb_opp(const ImgDesc &r, const ImgDesc &g, const ImgDesc &b, int dtype, int count,
                           const double m[9], float *q1, float *q2, float *q3, cudaStream_t st) {
    Mat3 M;
    for (int i = 0; i < 9; ++i) M.m[i] = (float)m[i];
    const dim3 grid((unsigned)((r.W + 127) / 128), (unsigned)r.H, count);
    switch (dtype) {
    case GBSSIM_U8: rgb_opp_kernel<uint8_t><<<grid, 128, 0, st>>>(r, g, b, M, q1, q2, q3); break;
    case GBSSIM_F16: rgb_opp_kernel<__half><<<grid, 128, 0, st>>>(r, g, b, M, q1, q2, q3); break;
    case GBSSIM_BF16: rgb_opp_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(r, g, b, M, q1, q2, q3); break;
    case GBSSIM_F32: rgb_opp_kernel<float><<<grid, 128, 0, st>>>(r, g, b, M, q1, q2, q3); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_opp_lab(float *p1, float *p2, float *p3, int64_t n, const double inv[9], const double white[3],
                           cudaStream_t st) {
    Mat3 M;
    for (int i = 0; i < 9; ++i) M.m[i] = (float)inv[i];
    const float3 wi = make_float3((float)(1.0 / white[0]), (float)(1.0 / white[1]), (float)(1.0 / white[2]));
    opp_lab_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p1, p2, p3, n, M, wi);
    return cudaGetLastError();
}

cudaError_t launch_cmssim_weight(float *map, int64_t oh, int64_t ow, int64_t map_ld, int64_t map_is, int count,
                                 const float *lab_x, const float *lab_y, int64_t H, int64_t W, int64_t cs, int centre,
                                 int stride, cudaStream_t st) {
    const dim3 grid((unsigned)((ow + 127) / 128), (unsigned)oh, count);
    weight_kernel<<<grid, 128, 0, st>>>(map, oh, ow, map_ld, map_is, lab_x, lab_y, H, W, cs, centre, stride);
    return cudaGetLastError();
}

}  // namespace gbssim
