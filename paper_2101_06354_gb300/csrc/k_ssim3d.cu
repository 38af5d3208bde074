// k_ssim3d.cu -- SSIM-3D and MS-SSIM-3D (Section "Spatio-Temporal SSIM" of
// arXiv 2101.06354): SSIM whose local statistics are taken over k x k x Kt
// rectangular spatio-temporal neighbourhoods of a video pair, the window of
// output frame t covering input frames t .. t+Kt-1 (the window ending at
// frame t+Kt-1); MS-SSIM-3D applies it to every level of each frame's 2x2
// average pyramid.
//
// The paper keeps rolling temporal sums T(i,j,k) of the last Kt frames and
// forms the spatial window sums of T.  Here one CTA owns a tile of 64 x 16
// output positions and walks the video in time: per input frame f it adds
// frame f and subtracts frame f-Kt from the tile's five exact integer
// temporal sums in shared memory (frame f-Kt was read Kt steps earlier by the
// same CTA and is normally still in L2), sums k rows of T down each column
// (running sums, lanes over consecutive columns), turns each row of those
// column sums into prefix sums with a warp scan, and takes every window sum
// as the difference of two prefix values.  The box formula is evaluated with
// exact int64 numerators over N = k^2 Kt pixels.  Each input byte comes from
// HBM once.  Per (tile, output frame) partial sums of Q and cs are combined
// per frame in a fixed order.  Prefix sums may pass the accumulator's range
// for the largest windows; they are kept in wrapping unsigned arithmetic,
// which leaves every difference (a window sum inside the range) exact.
//
// Level 0 of uint8 video runs with int32 sums; pyramid levels j >= 1 hold
// multiples of 4^-j (averages of 4^j pixels), which the kernel scales by 4^j
// to exact integers and sums in int64, with C1 and C2 scaled by 16^j so that
// l and cs are those of the unscaled level.
#include "common.cuh"

namespace gbssim {
namespace {

constexpr int NT = 256;
constexpr int OW3 = 64;  // output tile width
// Output tile height: 16 rows with int32 sums; 8 with int64 sums, so that two
// CTAs fit an SM's shared memory.
template <typename A>
struct TileRows {
    static constexpr int v = sizeof(A) == 4 ? 16 : 8;
};
constexpr int RB = 4;              // rows per warp whose loads are in flight together

template <typename A>
struct Unsigned;
template <>
struct Unsigned<int> {
    using T = unsigned;
};
template <>
struct Unsigned<long long> {
    using T = unsigned long long;
};

struct S3Geo {
    int k, iw, ih, pw;  // window, input tile width and height, row pitch of the sums (elements)
};

// Dynamic shared memory (accumulator type A): Ts[5][ih][pw] temporal sums of
// the input tile, then Vs[5][OH][pw] vertical window sums of Ts (turned into
// row prefix sums in place), then the reduction scratch.
template <typename A>
__device__ __forceinline__ A *ts_of(A *sm, const S3Geo &g, int q) {
    return sm + q * g.ih * g.pw;
}
template <typename A>
__device__ __forceinline__ A *vs_of(A *sm, const S3Geo &g, int q) {
    return sm + 5 * g.ih * g.pw + q * TileRows<A>::v * g.pw;
}

// Up to 4 pixels of one row, raw (a 4-byte word, or a float4), zero past
// n4; unpack() turns them into integers (pixel value times `scale`).
template <typename In>
struct Raw;
template <>
struct Raw<uint8_t> {
    unsigned w;
};
template <>
struct Raw<float> {
    float4 v;
};

__device__ __forceinline__ void load_raw(const uint8_t *p, int n4, bool words, Raw<uint8_t> &r) {
    r.w = 0u;
    if (n4 <= 0) return;
    if (words && n4 == 4) {
        r.w = __ldg(reinterpret_cast<const unsigned *>(p));
    } else {
        for (int e = 0; e < n4; ++e) r.w |= (unsigned)__ldg(p + e) << (8 * e);
    }
}
__device__ __forceinline__ void load_raw(const float *p, int n4, bool words, Raw<float> &r) {
    r.v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n4 <= 0) return;
    if (words && n4 == 4) {
        r.v = __ldg(reinterpret_cast<const float4 *>(p));
    } else {
        r.v.x = __ldg(p);
        if (n4 > 1) r.v.y = __ldg(p + 1);
        if (n4 > 2) r.v.z = __ldg(p + 2);
        if (n4 > 3) r.v.w = __ldg(p + 3);
    }
}
__device__ __forceinline__ int unpack(const Raw<uint8_t> &r, int e, float) { return (r.w >> (8 * e)) & 255; }
__device__ __forceinline__ int unpack(const Raw<float> &r, int e, float scale) {
    const float f = e == 0 ? r.v.x : e == 1 ? r.v.y : e == 2 ? r.v.z : r.v.w;
    return __float2int_rn(f * scale);  // exact: pyramid values are multiples of 1 / scale
}

// 4 consecutive accumulators += d (16-byte accesses: int4, or two longlong2).
__device__ __forceinline__ void add4(int *t, const int (&d)[4]) {
    int4 *t4 = reinterpret_cast<int4 *>(t);
    int4 v = *t4;
    v.x += d[0];
    v.y += d[1];
    v.z += d[2];
    v.w += d[3];
    *t4 = v;
}
__device__ __forceinline__ void add4(long long *t, const long long (&d)[4]) {
    longlong2 *t2 = reinterpret_cast<longlong2 *>(t);
    longlong2 a = t2[0], b = t2[1];
    a.x += d[0];
    a.y += d[1];
    b.x += d[2];
    b.y += d[3];
    t2[0] = a;
    t2[1] = b;
}

template <typename A, typename In>
__global__ void __launch_bounds__(NT, sizeof(A) == 4 ? 3 : 2) ssim3d_kernel(const Ssim3dLaunch L, int tiles_x, int tiles_y) {
    using U = typename Unsigned<A>::T;
    constexpr int OH3 = TileRows<A>::v;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *sm = reinterpret_cast<A *>(smem_raw);
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
    const In *xb = static_cast<const In *>(L.x.data), *yb = static_cast<const In *>(L.y.data);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 5 * g.ih * g.pw; i += NT) sm[i] = 0;
    const int64_t N = (int64_t)L.k * L.k * L.kt;
    const bool words = L.vec4;  // 4-element vector loads (rows and frames aligned; tiles start at multiples of 64)
    const float scale = L.scale;
    for (int f = 0; f < L.T; ++f) {
        __syncthreads();  // the previous frame's readers of Ts / Vs are done
        // 1. temporal sums: + frame f, - frame f - kt.  Warp w takes rows
        //    w, w+8, ... in groups of RB (all loads of a group issued first);
        //    lane l the 4 pixels at columns 4l .. 4l+3, updated with 16-byte
        //    shared accesses (conflict-free).
        const bool old = f >= L.kt;
        for (int rg = warp; rg < g.ih; rg += RB * (NT / 32)) {
            Raw<In> rx[RB], ry[RB], qx[RB], qy[RB];
            int n4[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                const int r = rg + u * (NT / 32);
                const int c = 4 * lane;
                const int64_t row = y0 + r;
                n4[u] = 0;
                if (r < g.ih && row < H && c < g.iw)
                    n4[u] = (int)max((int64_t)0, min((int64_t)4, min((int64_t)(g.iw - c), W - (x0 + c))));
                const int64_t o = row * rs + x0 + c;
                load_raw(xb + f * fs + o, n4[u], words, rx[u]);
                load_raw(yb + f * fs + o, n4[u], words, ry[u]);
                load_raw(xb + (f - L.kt) * fs + o, old ? n4[u] : 0, words, qx[u]);
                load_raw(yb + (f - L.kt) * fs + o, old ? n4[u] : 0, words, qy[u]);
            }
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                if (n4[u] <= 0) continue;  // values past n4 are zero: they add nothing
                const int r = rg + u * (NT / 32);
                A d[5][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const A p = unpack(rx[u], e, scale), q = unpack(ry[u], e, scale);
                    const A po = unpack(qx[u], e, scale), qo = unpack(qy[u], e, scale);
                    d[0][e] = p - po;
                    d[1][e] = q - qo;
                    d[2][e] = p * p - po * po;
                    d[3][e] = q * q - qo * qo;
                    d[4][e] = p * q - po * qo;
                }
                const int at = r * g.pw + 4 * lane;
#pragma unroll
                for (int qd = 0; qd < 5; ++qd) add4(ts_of(sm, g, qd) + at, d[qd]);
            }
        }
        if (f < L.kt - 1) continue;
        const int t = f - L.kt + 1;  // output frame
        __syncthreads();
        // 2. vertical k-sums of Ts for the OH3 output rows: one thread per
        //    (quantity, column), running down the rows; stored one column to
        //    the right (column 0 of Vs stays 0 for the prefix sums)
        for (int task = threadIdx.x; task < 5 * g.iw; task += NT) {
            const int q = task / g.iw, c = task - q * g.iw;
            const A *tc = ts_of(sm, g, q) + c;
            A *vc = vs_of(sm, g, q) + c + 1;
            A s = 0;
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
            U *vr = reinterpret_cast<U *>(vs_of(sm, g, rr / OH3) + (rr % OH3) * g.pw);
            const int c0 = 1 + 3 * lane;  // columns c0 .. c0+2 (1 .. iw hold data)
            U v0 = c0 <= g.iw ? vr[c0] : (U)0, v1 = c0 + 1 <= g.iw ? vr[c0 + 1] : (U)0,
              v2 = c0 + 2 <= g.iw ? vr[c0 + 2] : (U)0;
            v1 += v0;
            v2 += v1;
            U incl = v2;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const U u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const U excl = incl - v2;
            if (c0 <= g.iw) vr[c0] = v0 + excl;
            if (c0 + 1 <= g.iw) vr[c0 + 1] = v1 + excl;
            if (c0 + 2 <= g.iw) vr[c0 + 2] = v2 + excl;
            if (lane == 0) vr[0] = (U)0;
        }
        __syncthreads();
        // 4. window sums = P[j + k] - P[j] (P shifted by the zero column), formula
        float accQ = 0.f, accC = 0.f;
        for (int o = threadIdx.x; o < OH3 * OW3; o += NT) {
            const int i = o / OW3, j = o - i * OW3;
            const int64_t a = y0 + i, b = x0 + j;
            if (a >= OH || b >= OW) continue;
            A s[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const U *vr = reinterpret_cast<const U *>(vs_of(sm, g, q) + i * g.pw);
                s[q] = (A)(vr[j + g.k] - vr[j]);
            }
            // exact int64 numerators over N pixels (the box formula times N^2)
            const int64_t s1x = s[0], s1y = s[1];
            const int64_t P2 = 2 * s1x * s1y, Q1 = s1x * s1x + s1y * s1y;
            const int64_t Nxy = N * (int64_t)s[4] - s1x * s1y;
            const int64_t T2 = (N * (int64_t)s[2] - s1x * s1x) + (N * (int64_t)s[3] - s1y * s1y);
            const float A1 = __ll2float_rn(P2) + L.C1n2, B1 = __ll2float_rn(Q1) + L.C1n2;
            const float A2 = fmaf(2.f, __ll2float_rn(Nxy), L.C2n2), B2 = __ll2float_rn(T2) + L.C2n2;
            const float cs = __fdividef(A2, B2);
            const float qv = __fdividef(A1, B1) * cs;
            accQ += qv;
            accC += cs;
            if (L.map) L.map[t * L.map_fs + a * L.map_ld + b] = qv;
        }
        // CTA sums -> this (tile, frame) partial
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            accQ += __shfl_down_sync(0xffffffffu, accQ, o);
            accC += __shfl_down_sync(0xffffffffu, accC, o);
        }
        if (lane == 0) {
            red[2 * warp] = accQ;
            red[2 * warp + 1] = accC;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sq = 0.0, sc = 0.0;
            for (int w = 0; w < NT / 32; ++w) {
                sq += (double)red[2 * w];
                sc += (double)red[2 * w + 1];
            }
            L.partials[(int64_t)t * tiles_x * tiles_y + tile] = make_double2(sq, sc);
        }
    }
}

// Mean of the frame scores in a fixed order (one CTA).
__global__ void frame_mean_kernel(const double *frames, int n, double *out) {
    __shared__ double red[256];
    double loc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) loc += frames[t];
    red[threadIdx.x] = loc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / n;
}

template <typename A>
size_t smem_bytes(int k) {
    constexpr int OH3 = TileRows<A>::v;
    const size_t ih = OH3 + k - 1, iw = OW3 + k - 1, pw = (iw + 4) & ~(size_t)3;
    return sizeof(A) * (5 * ih * pw + 5 * OH3 * pw) + sizeof(float) * 2 * (NT / 32);
}

template <typename A, typename In>
cudaError_t launch_level(const Ssim3dLaunch &L, cudaStream_t st) {
    int tx, ty;
    ssim3d_tiles(L.x.H, L.x.W, L.k, sizeof(A) == 4, &tx, &ty);
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(ssim3d_kernel<A, In>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem_bytes<A>(kSsim3dMaxK));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    ssim3d_kernel<A, In><<<tx * ty, NT, smem_bytes<A>(L.k), st>>>(L, tx, ty);
    return cudaGetLastError();
}

}  // namespace

void ssim3d_tiles(int64_t H, int64_t W, int k, bool level0, int *tx, int *ty) {
    const int oh = level0 ? TileRows<int>::v : TileRows<long long>::v;
    *tx = (int)((W - k + 1 + OW3 - 1) / OW3);
    *ty = (int)((H - k + 1 + oh - 1) / oh);
}

cudaError_t launch_ssim3d_level(const Ssim3dLaunch &L, bool level0, cudaStream_t st) {
    return level0 ? launch_level<int, uint8_t>(L, st) : launch_level<long long, float>(L, st);
}

cudaError_t launch_frame_mean(const double *frames, int n, double *out, cudaStream_t st) {
    frame_mean_kernel<<<1, 256, 0, st>>>(frames, n, out);
    return cudaGetLastError();
}

}  // namespace gbssim
