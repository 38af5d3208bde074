// k_ssim3d.cu -- SSIM-3D (Section "Spatio-Temporal SSIM" of arXiv
// 2101.06354): SSIM whose local statistics are taken over k x k x Kt
// rectangular spatio-temporal neighbourhoods of a uint8 video pair, the
// window of output frame t covering input frames t .. t+Kt-1 (the window
// ending at frame t+Kt-1).
//
// The paper keeps rolling temporal sums T(i,j,k) of the last Kt frames and
// forms the spatial window sums of T.  Here one CTA owns a tile of 64 x 16
// output positions and walks the video in time: per input frame f it adds
// frame f and subtracts frame f-Kt from the tile's five exact int32 temporal
// sums in shared memory (4-pixel word loads; frame f-Kt was read Kt steps
// earlier by the same CTA and is normally still in L2), sums k rows of T down
// each column (running sums, lanes over consecutive columns), turns each row
// of those column sums into prefix sums with a warp scan, and takes every
// window sum as the difference of two prefix values.  The box formula is
// evaluated with exact int64 numerators over N = k^2 Kt pixels.  Each input
// byte comes from HBM once.  Per (tile, output frame) partial sums of Q are
// combined per frame in a fixed order.  Prefix sums may pass 2^31 for the
// largest windows; they are kept in wrapping unsigned arithmetic, which
// leaves every difference (a window sum below 2^31) exact.
#include "common.cuh"

namespace gbssim {
namespace {

constexpr int NT = 256;
constexpr int OW3 = 64, OH3 = 16;  // output tile
constexpr int RB = 4;              // rows per warp whose loads are in flight together

struct S3Geo {
    int k, iw, ih, pw;  // window, input tile width and height, row pitch of the sums (ints)
};

// Dynamic shared memory: Ts[5][ih][pw] temporal sums of the input tile, then
// Vs[5][OH3][pw] vertical window sums of Ts (turned into row prefix sums in
// place), then the reduction scratch.
__device__ __forceinline__ int *ts_of(int *sm, const S3Geo &g, int q) { return sm + q * g.ih * g.pw; }
__device__ __forceinline__ int *vs_of(int *sm, const S3Geo &g, int q) {
    return sm + 5 * g.ih * g.pw + q * OH3 * g.pw;
}

__global__ void __launch_bounds__(NT) ssim3d_kernel(const Ssim3dLaunch L, int tiles_x, int tiles_y) {
    extern __shared__ __align__(16) int sm[];
    S3Geo g;
    g.k = L.k;
    g.iw = OW3 + L.k - 1;
    g.ih = OH3 + L.k - 1;
    g.pw = (g.iw + 4) & ~3;  // >= iw + 1 (a zero column in front of the prefix sums), multiple of 4
    float *red = reinterpret_cast<float *>(sm + 5 * g.ih * g.pw + 5 * OH3 * g.pw);
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int64_t H = L.x.H, W = L.x.W, rs = L.x.row_stride, fs = L.x.image_stride;
    const int64_t OH = H - L.k + 1, OW = W - L.k + 1;
    const int64_t x0 = (int64_t)tx * OW3, y0 = (int64_t)ty * OH3;
    const uint8_t *xb = static_cast<const uint8_t *>(L.x.data), *yb = static_cast<const uint8_t *>(L.y.data);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 5 * g.ih * g.pw; i += NT) sm[i] = 0;
    const int64_t N = (int64_t)L.k * L.k * L.kt;
    // word loads of 4 pixels when rows and frames are 4-byte aligned (tiles start at multiples of 64)
    const bool words = L.vec4;
    for (int f = 0; f < L.T; ++f) {
        __syncthreads();  // the previous frame's readers of Ts / Vs are done
        // 1. temporal sums: + frame f, - frame f - kt.  Warp w takes rows
        //    w, w+8, ... in groups of RB (all loads of a group issued first);
        //    lane l the 4 pixels at columns 4l .. 4l+3, updated with one
        //    16-byte shared access per quantity (conflict-free).
        const bool old = f >= L.kt;
        for (int rg = warp; rg < g.ih; rg += RB * (NT / 32)) {
            unsigned wx[RB], wy[RB], ox[RB], oy[RB];
            int n4[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                const int r = rg + u * (NT / 32);
                const int c = 4 * lane;
                const int64_t row = y0 + r;
                wx[u] = wy[u] = ox[u] = oy[u] = 0u;
                n4[u] = 0;
                if (r >= g.ih || row >= H || c >= g.iw) continue;
                n4[u] = (int)min((int64_t)4, min((int64_t)(g.iw - c), W - (x0 + c)));
                if (n4[u] <= 0) continue;
                const int64_t o = row * rs + x0 + c;
                if (words && n4[u] == 4) {
                    wx[u] = __ldg(reinterpret_cast<const unsigned *>(xb + f * fs + o));
                    wy[u] = __ldg(reinterpret_cast<const unsigned *>(yb + f * fs + o));
                    if (old) {
                        ox[u] = __ldg(reinterpret_cast<const unsigned *>(xb + (f - L.kt) * fs + o));
                        oy[u] = __ldg(reinterpret_cast<const unsigned *>(yb + (f - L.kt) * fs + o));
                    }
                } else {
                    for (int e = 0; e < n4[u]; ++e) {
                        wx[u] |= (unsigned)__ldg(xb + f * fs + o + e) << (8 * e);
                        wy[u] |= (unsigned)__ldg(yb + f * fs + o + e) << (8 * e);
                        if (old) {
                            ox[u] |= (unsigned)__ldg(xb + (f - L.kt) * fs + o + e) << (8 * e);
                            oy[u] |= (unsigned)__ldg(yb + (f - L.kt) * fs + o + e) << (8 * e);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                if (n4[u] <= 0) continue;  // bytes past n4 are zero: they add nothing
                const int r = rg + u * (NT / 32);
                int d[5][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int p = (wx[u] >> (8 * e)) & 255, q = (wy[u] >> (8 * e)) & 255;
                    const int po = (ox[u] >> (8 * e)) & 255, qo = (oy[u] >> (8 * e)) & 255;
                    d[0][e] = p - po;
                    d[1][e] = q - qo;
                    d[2][e] = p * p - po * po;
                    d[3][e] = q * q - qo * qo;
                    d[4][e] = p * q - po * qo;
                }
                const int at = r * g.pw + 4 * lane;
#pragma unroll
                for (int qd = 0; qd < 5; ++qd) {
                    int4 *t4 = reinterpret_cast<int4 *>(ts_of(sm, g, qd) + at);
                    int4 v = *t4;
                    v.x += d[qd][0];
                    v.y += d[qd][1];
                    v.z += d[qd][2];
                    v.w += d[qd][3];
                    *t4 = v;
                }
            }
        }
        if (f < L.kt - 1) continue;
        const int t = f - L.kt + 1;  // output frame
        __syncthreads();
        // 2. vertical k-sums of Ts for the OH3 output rows: one thread per
        //    (quantity, column), running down the rows; stored one column
        //    to the right (column 0 of Vs stays 0 for the prefix sums)
        for (int task = threadIdx.x; task < 5 * g.iw; task += NT) {
            const int q = task / g.iw, c = task - q * g.iw;
            const int *tc = ts_of(sm, g, q) + c;
            int *vc = vs_of(sm, g, q) + c + 1;
            int s = 0;
            for (int m = 0; m < g.k; ++m) s += tc[m * g.pw];
            vc[0] = s;
            for (int i = 1; i < OH3; ++i) {
                s += tc[(i + g.k - 1) * g.pw] - tc[(i - 1) * g.pw];
                vc[i * g.pw] = s;
            }
        }
        __syncthreads();
        // 3. inclusive prefix sums along each Vs row (5 x OH3 rows), in place:
        //    one warp per row, 3 columns per lane, a shuffle scan of the lane totals
        for (int rr = warp; rr < 5 * OH3; rr += NT / 32) {
            unsigned *vr = reinterpret_cast<unsigned *>(vs_of(sm, g, rr / OH3) + (rr % OH3) * g.pw);
            const int c0 = 1 + 3 * lane;  // columns c0 .. c0+2 (1 .. iw hold data)
            unsigned v0 = c0 <= g.iw ? vr[c0] : 0u, v1 = c0 + 1 <= g.iw ? vr[c0 + 1] : 0u,
                     v2 = c0 + 2 <= g.iw ? vr[c0 + 2] : 0u;
            v1 += v0;
            v2 += v1;
            unsigned incl = v2;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const unsigned excl = incl - v2;
            if (c0 <= g.iw) vr[c0] = v0 + excl;
            if (c0 + 1 <= g.iw) vr[c0 + 1] = v1 + excl;
            if (c0 + 2 <= g.iw) vr[c0 + 2] = v2 + excl;
            if (lane == 0) vr[0] = 0u;
        }
        __syncthreads();
        // 4. window sums = P[j + k] - P[j] (P shifted by the zero column), formula
        float accQ = 0.f;
        for (int o = threadIdx.x; o < OH3 * OW3; o += NT) {
            const int i = o / OW3, j = o - i * OW3;
            const int64_t a = y0 + i, b = x0 + j;
            if (a >= OH || b >= OW) continue;
            int s[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const unsigned *vr = reinterpret_cast<const unsigned *>(vs_of(sm, g, q) + i * g.pw);
                s[q] = (int)(vr[j + g.k] - vr[j]);
            }
            // exact int64 numerators over N pixels (the box formula times N^2)
            const int64_t s1x = s[0], s1y = s[1];
            const int64_t P2 = 2 * s1x * s1y, Q1 = s1x * s1x + s1y * s1y;
            const int64_t Nxy = N * s[4] - s1x * s1y;
            const int64_t T2 = (N * s[2] - s1x * s1x) + (N * s[3] - s1y * s1y);
            const float A1 = __ll2float_rn(P2) + L.C1n2, B1 = __ll2float_rn(Q1) + L.C1n2;
            const float A2 = fmaf(2.f, __ll2float_rn(Nxy), L.C2n2), B2 = __ll2float_rn(T2) + L.C2n2;
            const float qv = __fdividef(A1, B1) * __fdividef(A2, B2);
            accQ += qv;
            if (L.map) L.map[t * L.map_fs + a * L.map_ld + b] = qv;
        }
        // CTA sum -> this (tile, frame) partial
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) accQ += __shfl_down_sync(0xffffffffu, accQ, o);
        if (lane == 0) red[warp] = accQ;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int w = 0; w < NT / 32; ++w) sum += (double)red[w];
            L.partials[(int64_t)t * tiles_x * tiles_y + tile] = sum;
        }
    }
}

// Frame scores (fixed-order sums of the tile partials) and the video mean.
__global__ void ssim3d_finalize_kernel(const double *partials, int tiles, int frames, double inv_n, double *frame_out,
                                       double *score_out) {
    __shared__ double red[256];
    double loc = 0.0;
    for (int t = threadIdx.x; t < frames; t += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < tiles; ++i) s += partials[(int64_t)t * tiles + i];
        s *= inv_n;
        if (frame_out) frame_out[t] = s;
        loc += s;
    }
    red[threadIdx.x] = loc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && score_out) *score_out = red[0] / frames;
}

}  // namespace

void ssim3d_tiles(int64_t H, int64_t W, int k, int *tx, int *ty) {
    *tx = (int)((W - k + 1 + OW3 - 1) / OW3);
    *ty = (int)((H - k + 1 + OH3 - 1) / OH3);
}

size_t ssim3d_smem(int k) {
    const size_t ih = OH3 + k - 1, iw = OW3 + k - 1, pw = (iw + 4) & ~(size_t)3;
    return sizeof(int) * (5 * ih * pw + 5 * OH3 * pw) + sizeof(float) * (NT / 32);
}

cudaError_t launch_ssim3d(const Ssim3dLaunch &L, double *frame_out, double *score_out, cudaStream_t st) {
    int tx, ty;
    ssim3d_tiles(L.x.H, L.x.W, L.k, &tx, &ty);
    const size_t smem = ssim3d_smem(L.k);
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(ssim3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)ssim3d_smem(kSsim3dMaxK));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    ssim3d_kernel<<<tx * ty, NT, smem, st>>>(L, tx, ty);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int frames = L.T - L.kt + 1;
    const double inv_n = 1.0 / ((double)(L.x.H - L.k + 1) * (double)(L.x.W - L.k + 1));
    ssim3d_finalize_kernel<<<1, 256, 0, st>>>(L.partials, tx * ty, frames, inv_n, frame_out, score_out);
    return cudaGetLastError();
}

}  // namespace gbssim
