// k_ssim3d.cu -- SSIM-3D and MS-SSIM-3D (Section "Spatio-Temporal SSIM" of
// arXiv 2101.06354): SSIM whose local statistics are taken over k x k x Kt
// rectangular spatio-temporal neighbourhoods of a video pair, the window of
// output frame t covering input frames t .. t+Kt-1 (the window ending at
// frame t+Kt-1); MS-SSIM-3D applies it to every level of each frame's 2x2
// average pyramid.
//
// The paper keeps rolling temporal sums T(i,j,k) of the last Kt frames and
// forms the spatial window sums of T.  Here one CTA owns a tile of 64 output
// columns and OH output rows and walks the video in time.  Per input frame f:
//   1. the tile's temporal sums in shared memory gain frame f and lose frame
//      f-Kt (read Kt steps earlier by the same CTA, normally still in L2);
//      each thread owns fixed 4-column groups, so this step needs no barrier
//      between frames;
//   2. once Kt frames are in, running sums down each column give the k-row
//      sums of the OH output rows, stored transposed (column-major);
//   3. running sums along each output row over those column sums give the
//      k x k x Kt window sums of 8 consecutive outputs per thread, and the
//      formula is evaluated right away.
// Two barriers per output frame.  Each input byte comes from HBM once.
//
// The window statistics are carried in the (u, w) = (x + y, x - y) form:
// sums of u, w, u^2, w^2 (four quantities instead of five).  With
// Su = sum u, Sw = sum w, Vu = N sum u^2 - Su^2, Vw = N sum w^2 - Sw^2 over
// N = k^2 Kt pixels, the Background-section factors are exactly
//   l  = (Su^2 - Sw^2 + 2 C1 N^2) / (Su^2 + Sw^2 + 2 C1 N^2),
//   cs = (Vu - Vw + 2 C2 N^2) / (Vu + Vw + 2 C2 N^2),
// since Su^2 - Sw^2 = 4 sx sy, Su^2 + Sw^2 = 2 (sx^2 + sy^2),
// Vu - Vw = 4 (N sxy - sx sy) and Vu + Vw = 2 (N sxx - sx^2 + N syy - sy^2).
// All sums are exact integers; the int64 numerators are rounded to fp32 once
// (with int32 sums, l is formed in fp32 from the exact Su, Sw).
//
// uint8 video runs with int32 sums while N (2 255)^2 < 2^31, else int64;
// pyramid levels j >= 1 hold multiples of 4^-j (averages of 4^j pixels),
// which the kernel scales by 4^j to exact integers and sums in int64, with
// C1 and C2 scaled by 16^j so that l and cs are those of the unscaled level.
#include <type_traits>

#include "tma.cuh"

namespace gbssim {
namespace {

constexpr int NT = 256;
constexpr int OW3 = 64;  // output tile width
constexpr int SEG = 8;   // consecutive outputs of one row per thread in step 3
constexpr int RB = 2;    // 4-column groups per thread whose loads are in flight together

// Tile height (16 rows) and the pitch of the transposed column sums
// (elements).  The pitches make step 3's reads (lanes over rows, then two
// 8-column segments per warp) and step 2's stores (lanes over columns)
// conflict-free: 18 int32 (9 pairs for the paired stores, two segments 16
// banks apart), 17 int64 (8-byte accesses, half a warp per wavefront).
template <typename A>
struct Tile3 {
    static constexpr int OH = 16;
    static constexpr int PV = sizeof(A) == 4 ? 18 : 17;
    static constexpr int TASKS3 = OH * (OW3 / SEG);  // step-3 threads
    static constexpr int WARPS3 = TASKS3 / 32;       // step-3 warps
};

struct S3Geo {
    int k, iw, ih, pw, groups;  // window, input tile width and height, Ts pitch, 4-column groups per row
};

// Dynamic shared memory: Ts[4][ih][pw] temporal sums of the input tile, then
// Vs[4][iw][PV] the k-row column sums (column-major), then the step-3 warp
// sums (double2 per warp; every part starts on a 16-byte boundary); with
// bulk copies (uint8 video) then, from a 128-byte boundary, the four byte
// tiles of the next frame (x, y, x and y of the frame leaving the window),
// ih rows of raw3_width(k) bytes each, and their mbarrier.
// Bytes per bulk-copied tile row: the input tile width rounded up to 16
// (covers every 4-column group, a multiple of 16 as bulk copies need).
__host__ __device__ constexpr int raw3_width(int k) { return ((OW3 + k - 1) + 15) & ~15; }
template <typename A>
__device__ __forceinline__ A *ts_of(A *sm, const S3Geo &g, int q) {
    return sm + q * g.ih * g.pw;
}
template <typename A>
__device__ __forceinline__ A *vs_of(A *sm, const S3Geo &g, int q) {
    return sm + 4 * g.ih * g.pw + q * g.iw * Tile3<A>::PV;
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
__device__ __forceinline__ void add4(unsigned *t, const unsigned (&d)[4]) {
    uint4 *t4 = reinterpret_cast<uint4 *>(t);
    uint4 v = *t4;
    v.x += d[0];
    v.y += d[1];
    v.z += d[2];
    v.w += d[3];
    *t4 = v;
}
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

// Step 2's column of OH k-row sums, stored column-major: int32 as pairs
// (8-byte stores), int64 one by one.
template <int OH>
__device__ __forceinline__ void store_col(int *vc, const int (&v)[OH]) {
#pragma unroll
    for (int i = 0; i < OH; i += 2) *reinterpret_cast<int2 *>(vc + i) = make_int2(v[i], v[i + 1]);
}
template <int OH>
__device__ __forceinline__ void store_col(unsigned *vc, const unsigned (&v)[OH]) {
#pragma unroll
    for (int i = 0; i < OH; i += 2) *reinterpret_cast<uint2 *>(vc + i) = make_uint2(v[i], v[i + 1]);
}
template <int OH>
__device__ __forceinline__ void store_col(long long *vc, const long long (&v)[OH]) {
#pragma unroll
    for (int i = 0; i < OH; ++i) vc[i] = v[i];
}

// BULK (uint8 video): each frame's input tiles arrive by 2-D bulk tensor
// copies (tmx, tmy: ih x 80-byte tiles of frame z) issued by one thread after
// the previous frame's step 1, instead of per-thread loads.  A bulk-copy wait
// that gives up writes NaN partials for the CTA's remaining output frames,
// waits (bounded) for its copies in flight and returns.
// 64 registers a thread (4 CTAs per SM) with 32-bit sums of byte input;
// float input keeps four float4 prefetches per 4-column group in flight and
// gets 80 (3 CTAs); int64 sums 128 (2 CTAs).
template <typename A, typename In>
constexpr int ssim3d_min_ctas() {
    return sizeof(A) == 8 ? 2 : (std::is_same<In, float>::value ? 3 : 4);
}

template <typename A, typename In, bool BULK>
__global__ void __launch_bounds__(NT, (ssim3d_min_ctas<A, In>()))
    ssim3d_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy,
                  const Ssim3dLaunch L, int tiles_x, int tiles_y, int t_chunk) {
    constexpr int OH = Tile3<A>::OH, PV = Tile3<A>::PV;
    // 4-column groups whose loads are in flight together: float input holds
    // a float4 per row and frame, so one group (the byte input's word, two)
    constexpr int RBK = std::is_same<In, float>::value ? 1 : RB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    A *sm = reinterpret_cast<A *>(smem_raw);
    S3Geo g;
    g.k = L.k;
    g.iw = OW3 + L.k - 1;
    g.ih = OH + L.k - 1;
    g.pw = (g.iw + 3) & ~3;
    g.groups = (g.iw + 3) >> 2;
    const int tile = blockIdx.x % (tiles_x * tiles_y);
    // output frames t_begin .. t_end-1 from input frames f_begin .. f_end-1
    const int t_begin = (blockIdx.x / (tiles_x * tiles_y)) * t_chunk;
    const int t_end = min(t_begin + t_chunk, L.T - L.kt + 1);
    const int f_begin = t_begin, f_end = t_end + L.kt - 1;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int64_t H = L.x.H, W = L.x.W, rs = L.x.row_stride, fs = L.x.image_stride;
    const int64_t OHt = H - L.k + 1, OWt = W - L.k + 1;
    const int64_t x0 = (int64_t)tx * OW3, y0 = (int64_t)ty * OH;
    const In *xb = static_cast<const In *>(L.x.data), *yb = static_cast<const In *>(L.y.data);
    const int lane = threadIdx.x & 31;
    // bulk-copy tiles and their mbarrier after the warp sums
    const size_t bulk_off = ((reinterpret_cast<unsigned char *>(vs_of(sm, g, 4) + 0) - smem_raw) +
                             sizeof(double2) * Tile3<A>::WARPS3 + 127) & ~(size_t)127;
    unsigned char *raw = smem_raw + bulk_off;
    const int rw = raw3_width(L.k);
    const unsigned tile_bytes = (unsigned)(g.ih * rw);            // one tile
    const unsigned tile_stride = (tile_bytes + 127u) & ~127u;      // tiles start on 128-byte boundaries
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(raw + 4 * tile_stride);
    // frame ff's tiles (thread 0): x, y of ff, and of ff - kt when it leaves a window of this CTA
    auto issue = [&](int ff) {
        const bool with_old = ff - L.kt >= f_begin;
        mbar_expect_tx(bar, (with_old ? 4u : 2u) * tile_bytes);
        tma_load_3d(raw, &tmx, (int)x0, (int)y0, ff, bar);
        tma_load_3d(raw + tile_stride, &tmy, (int)x0, (int)y0, ff, bar);
        if (with_old) {
            tma_load_3d(raw + 2 * tile_stride, &tmx, (int)x0, (int)y0, ff - L.kt, bar);
            tma_load_3d(raw + 3 * tile_stride, &tmy, (int)x0, (int)y0, ff - L.kt, bar);
        }
    };
    unsigned phase = 0;
    if (BULK && threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        issue(f_begin);
    }
    for (int i = threadIdx.x; i < 4 * g.ih * g.pw; i += NT) sm[i] = 0;
    __syncthreads();
    const int64_t N = (int64_t)L.k * L.k * L.kt;
    const bool words = L.vec4;  // 4-element vector loads (rows and frames aligned; tiles start at multiples of 64)
    const float scale = L.scale;
    const int units = g.ih * g.groups;
    int pending = -1;  // output frame whose warp sums wait in red
    auto flush = [&](int tp) {
        const double2 *red = reinterpret_cast<const double2 *>(vs_of(sm, g, 4));
        double sq = 0.0, sc = 0.0;
#pragma unroll
        for (int w = 0; w < Tile3<A>::WARPS3; ++w) {
            sq += red[w].x;
            sc += red[w].y;
        }
        L.partials[(int64_t)tp * (tiles_x * tiles_y) + tile] = make_double2(sq, sc);
    };
    // the first RBK groups of this thread: offsets and widths hoisted out of
    // the frame loop; their bytes of frame f+1 and of frame f+1-kt (the one
    // leaving the window) are loaded while frame f is in steps 2 and 3
    int64_t o0[RBK];
    int n40[RBK], at0[RBK];
#pragma unroll
    for (int u = 0; u < RBK; ++u) {
        const int unit = threadIdx.x + u * NT;
        const int r = unit / g.groups, c = 4 * (unit - r * g.groups);
        const int64_t row = y0 + r;
        n40[u] = 0;
        if (unit < units && row < H)
            n40[u] = (int)max((int64_t)0, min((int64_t)4, min((int64_t)(g.iw - c), W - (x0 + c))));
        at0[u] = r * g.pw + c;
        o0[u] = row * rs + x0 + c;
    }
    Raw<In> px[RBK], py[RBK], pxo[RBK], pyo[RBK];  // frame f and frame f - kt of those groups
#pragma unroll
    for (int u = 0; u < RBK; ++u) {
        load_raw(xb + f_begin * fs + o0[u], BULK ? 0 : n40[u], words, px[u]);
        load_raw(yb + f_begin * fs + o0[u], BULK ? 0 : n40[u], words, py[u]);
        load_raw(xb, 0, words, pxo[u]);  // no frame leaves the window yet
        load_raw(yb, 0, words, pyo[u]);
    }
    for (int f = f_begin; f < f_end; ++f) {
        // 1. temporal sums: + frame f, - frame f - kt.  Thread t owns the
        //    4-column groups t, t + NT, ... (row-major over the input tile),
        //    RBK of them with their loads in flight together; 16-byte shared
        //    accesses, consecutive across a warp.
        const bool old = f - L.kt >= f_begin;
        bool failed = false;
        if constexpr (BULK) {
            // the tiles of frame f, bulk-copied during the previous frame's steps 2 and 3
            if (!mbar_wait_bounded(bar, phase)) failed = true;
            phase ^= 1u;
            if (!failed)
                for (int unit = threadIdx.x; unit < units; unit += NT) {
                    const int r = unit / g.groups, c = 4 * (unit - r * g.groups);
                    const unsigned char *rp = raw + r * rw + c;
                    Raw<In> ux, uy, ox, oy;
                    ux.w = *reinterpret_cast<const unsigned *>(rp);
                    uy.w = *reinterpret_cast<const unsigned *>(rp + tile_stride);
                    ox.w = old ? *reinterpret_cast<const unsigned *>(rp + 2 * tile_stride) : 0u;
                    oy.w = old ? *reinterpret_cast<const unsigned *>(rp + 3 * tile_stride) : 0u;
                    A d[4][4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int p = unpack(ux, e, scale), q = unpack(uy, e, scale);
                        const int po = unpack(ox, e, scale), qo = unpack(oy, e, scale);
                        const A uu = (A)p + q, ww = (A)p - q, uo = (A)po + qo, wo = (A)po - qo;
                        d[0][e] = uu - uo;
                        d[1][e] = ww - wo;
                        d[2][e] = (uu - uo) * (uu + uo);
                        d[3][e] = (ww - wo) * (ww + wo);
                    }
                    const int at = r * g.pw + c;
#pragma unroll
                    for (int qd = 0; qd < 4; ++qd) add4(ts_of(sm, g, qd) + at, d[qd]);
                }
        } else {
        const In *xf = xb + f * fs, *yf = yb + f * fs;
        const In *xo = xb + (f - L.kt) * fs, *yo = yb + (f - L.kt) * fs;
        for (int u0 = threadIdx.x; u0 < units; u0 += RBK * NT) {
            const bool first = u0 == threadIdx.x;
            Raw<In> rx[RBK], ry[RBK], qx[RBK], qy[RBK];
            int n4[RBK], at[RBK];
#pragma unroll
            for (int u = 0; u < RBK; ++u) {
                if (first) {
                    n4[u] = n40[u];
                    at[u] = at0[u];
                    rx[u] = px[u];
                    ry[u] = py[u];
                    qx[u] = pxo[u];
                    qy[u] = pyo[u];
                } else {
                    const int unit = u0 + u * NT;
                    const int r = unit / g.groups, c = 4 * (unit - r * g.groups);
                    const int64_t row = y0 + r;
                    n4[u] = 0;
                    if (unit < units && row < H)
                        n4[u] = (int)max((int64_t)0, min((int64_t)4, min((int64_t)(g.iw - c), W - (x0 + c))));
                    at[u] = r * g.pw + c;
                    const int64_t o = row * rs + x0 + c;
                    load_raw(xf + o, n4[u], words, rx[u]);
                    load_raw(yf + o, n4[u], words, ry[u]);
                    load_raw(xo + o, old ? n4[u] : 0, words, qx[u]);
                    load_raw(yo + o, old ? n4[u] : 0, words, qy[u]);
                }
            }
            if (first && f + 1 < f_end) {
                const bool old1 = f + 1 - L.kt >= f_begin;
#pragma unroll
                for (int u = 0; u < RBK; ++u) {
                    load_raw(xf + fs + o0[u], n40[u], words, px[u]);
                    load_raw(yf + fs + o0[u], n40[u], words, py[u]);
                    load_raw(xo + fs + o0[u], old1 ? n40[u] : 0, words, pxo[u]);
                    load_raw(yo + fs + o0[u], old1 ? n40[u] : 0, words, pyo[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < RBK; ++u) {
                if (n4[u] <= 0) continue;  // values past n4 are zero: they add nothing
                A d[4][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int p = unpack(rx[u], e, scale), q = unpack(ry[u], e, scale);
                    const int po = unpack(qx[u], e, scale), qo = unpack(qy[u], e, scale);
                    const A uu = (A)p + q, ww = (A)p - q, uo = (A)po + qo, wo = (A)po - qo;
                    d[0][e] = uu - uo;
                    d[1][e] = ww - wo;
                    d[2][e] = (uu - uo) * (uu + uo);  // u^2 - uo^2
                    d[3][e] = (ww - wo) * (ww + wo);
                }
#pragma unroll
                for (int qd = 0; qd < 4; ++qd) add4(ts_of(sm, g, qd) + at[u], d[qd]);
            }
        }
        }  // register path
        const bool out_frame = f >= f_begin + L.kt - 1;
        if constexpr (BULK) {
            // every thread is done with the tiles of frame f: thread 0 refills them with frame f+1
            if (__syncthreads_or(failed)) {
                if (threadIdx.x == 0) {
                    mbar_wait_bounded(bar, phase ^ 1u);  // drain the copy that did not complete (bounded)
                    for (int tt = max(t_begin, f - L.kt + 1); tt < t_end; ++tt)
                        L.partials[(int64_t)tt * (tiles_x * tiles_y) + tile] = make_double2(nan(""), nan(""));
                }
                return;
            }
            if (threadIdx.x == 0 && f + 1 < f_end) {
                fence_proxy_async_smem();
                issue(f + 1);
            }
        }
        if (!out_frame) continue;
        const int t = f - L.kt + 1;  // output frame
        if (!BULK) __syncthreads();  // Ts holds frames t .. f; red holds frame t-1's warp sums
        if (threadIdx.x == 0 && pending >= 0) flush(pending);
        // 2. k-row sums down each column for the OH output rows: one thread
        //    per (quantity, column), lanes over consecutive columns
        for (int task = threadIdx.x; task < 4 * g.iw; task += NT) {
            const int q = task / g.iw, c = task - q * g.iw;
            const A *tc = ts_of(sm, g, q) + c;
            A v[OH];
            A s = 0;
#pragma unroll 4
            for (int m = 0; m < g.k; ++m) s += tc[m * g.pw];
            v[0] = s;
            const A *tn = tc + g.k * g.pw;  // row entering the window
#pragma unroll
            for (int i = 1; i < OH; ++i) {
                s += tn[(i - 1) * g.pw] - tc[(i - 1) * g.pw];
                v[i] = s;
            }
            store_col<OH>(vs_of(sm, g, q) + c * PV, v);
        }
        __syncthreads();  // Vs holds the column sums of frame t
        // 3. row running sums over the column sums (k x k x kt window sums of
        //    SEG outputs per thread, lanes over rows) and the formula
        if (threadIdx.x < Tile3<A>::TASKS3) {
            const int i = threadIdx.x % OH, j0 = (threadIdx.x / OH) * SEG;
            const int64_t a = y0 + i;
            float accQ = 0.f, accC = 0.f;
            if (a < OHt && x0 + j0 < OWt) {
                const A *v0 = vs_of(sm, g, 0) + j0 * PV + i, *v1 = vs_of(sm, g, 1) + j0 * PV + i;
                const A *v2 = vs_of(sm, g, 2) + j0 * PV + i, *v3 = vs_of(sm, g, 3) + j0 * PV + i;
                A su = 0, sw = 0, su2 = 0, sw2 = 0;
#pragma unroll 4
                for (int m = 0; m < g.k; ++m) {
                    su += v0[m * PV];
                    sw += v1[m * PV];
                    su2 += v2[m * PV];
                    sw2 += v3[m * PV];
                }
                const int nout = (int)min((int64_t)SEG, OWt - (x0 + j0));
                float *mrow = L.map ? L.map + t * L.map_fs + a * L.map_ld + x0 + j0 : nullptr;
#pragma unroll
                for (int e = 0; e < SEG; ++e) {
                    if (e > 0) {
                        const int in = (e + g.k - 1) * PV, out = (e - 1) * PV;
                        su += v0[in] - v0[out];
                        sw += v1[in] - v1[out];
                        su2 += v2[in] - v2[out];
                        sw2 += v3[in] - v3[out];
                    }
                    if (e < nout) {
                        float A1, B1;
                        int64_t Vu, Vw;
                        if constexpr (sizeof(A) == 4) {
                            // |Su|, |Sw| < 2^23 (uint8 video: 510 N with N < 8256; the
                            // unsigned level: checked by the launcher): exact in fp32, and
                            // Su^2 - Sw^2 = (Su - Sw)(Su + Sw) rounds once.  Unsigned sums
                            // are modulo 2^32: Sw (may be negative) reads as int32, the
                            // square sums (>= 0, < 2^32) as uint32.
                            const int64_t su_ = (int64_t)(int)su, sw_ = (int64_t)(int)sw;
                            const int64_t su2_ = (int64_t)(unsigned)su2, sw2_ = (int64_t)(unsigned)sw2;
                            const float fu = (float)su_, fw = (float)sw_;
                            A1 = fmaf(fu - fw, fu + fw, L.C1x2n2);
                            B1 = fmaf(fu, fu, fmaf(fw, fw, L.C1x2n2));
                            Vu = N * su2_ - su_ * su_;
                            Vw = N * sw2_ - sw_ * sw_;
                        } else {
                            const int64_t U2 = (int64_t)su * su, W2 = (int64_t)sw * sw;
                            Vu = N * (int64_t)su2 - U2;
                            Vw = N * (int64_t)sw2 - W2;
                            A1 = __ll2float_rn(U2 - W2) + L.C1x2n2;
                            B1 = __ll2float_rn(U2 + W2) + L.C1x2n2;
                        }
                        // variances need the exact int64 differences; with 32-bit sums
                        // |Vu +- Vw| < 2 N^2 (2 x 255 scale)^2 < 2^48 (N < 8256 at scale 1;
                        // the unsigned level's bounds), so the conversion avoids the FP64 pipe
                        float A2, B2;
                        if constexpr (sizeof(A) == 4) {
                            A2 = i48_to_f32(Vu - Vw) + L.C2x2n2;
                            B2 = i48_to_f32(Vu + Vw) + L.C2x2n2;
                        } else {
                            A2 = __ll2float_rn(Vu - Vw) + L.C2x2n2;
                            B2 = __ll2float_rn(Vu + Vw) + L.C2x2n2;
                        }
                        const float cs = __fdividef(A2, B2);
                        const float qv = __fdividef(A1, B1) * cs;
                        accQ += qv;
                        accC += cs;
                        if (mrow) mrow[e] = qv;
                    }
                }
            }
            // warp sums -> red[warp]; thread 0 adds them up after the next
            // barrier (or after the loop) into this (frame, tile) partial
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                accQ += __shfl_down_sync(0xffffffffu, accQ, o);
                accC += __shfl_down_sync(0xffffffffu, accC, o);
            }
            if (lane == 0)
                reinterpret_cast<double2 *>(vs_of(sm, g, 4))[threadIdx.x >> 5] =
                    make_double2((double)accQ, (double)accC);
        }
        pending = t;
    }
    __syncthreads();
    if (threadIdx.x == 0 && pending >= 0) flush(pending);
}

// ----------------------------------------------------------------- uint8, 11 x 11 x kt, int32 sums
//
// The SSIM-3D hot case (uint8 video, k = 11, int32 sums, bulk copies) keeps
// the tile's temporal sums in REGISTERS: thread (q, c) owns quantity q (u, w,
// u^2 or w^2 of (u, w) = (x + y, x - y)) of input column c for all 26 rows,
// adds frame f and subtracts frame f - kt straight from the bulk-copied
// bytes, and forms the 16 k-row sums of its column in registers (running
// sums down the column); only those column sums go to shared memory, double
// buffered, so one barrier per frame separates a frame's column sums from
// the row pass that reads them while the next frame's column pass writes the
// other buffer.  The row pass (running sums over 11 column sums, 4 outputs
// per thread, 256 threads) and the formula are those of ssim3d_kernel.
constexpr int NTC = 320;                 // 4 quantities x 80 column slots (74 used)
constexpr int KC = 11;                   // window width and height
constexpr int OHC = 16;                  // output rows per tile (as Tile3<int>)
constexpr int IHC = OHC + KC - 1;        // 26 input rows
constexpr int IWC = OW3 + KC - 1;        // 74 input columns
constexpr int PVC = 20;                  // pitch of the column sums: 4 PVC = 16 mod 32 (row pass), int4 stores
constexpr int SEGC = 4;                  // outputs per row-pass thread
constexpr int T3C = OHC * (OW3 / SEGC);  // 256 row-pass threads (warps 2..9)
constexpr int RWC = raw3_width(KC);      // 80 bytes per bulk-copied row
constexpr int TILEC = (IHC * RWC + 127) & ~127;
struct __align__(128) S3C {
    unsigned char raw[4][TILEC];   // x, y of frame f; x, y of frame f - kt
    int vs[2][4][IWC][PVC];        // column sums [buffer][quantity][column][row]
    double2 red[2][T3C / 32];      // row-pass warp sums [buffer][warp]
    unsigned long long bar;
};

__global__ void __launch_bounds__(NTC, 3)
    ssim3d_cols_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy,
                       const Ssim3dLaunch L, int tiles_x, int tiles_y, int t_chunk) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S3C &S = *reinterpret_cast<S3C *>(smem_raw);
    const int tiles = tiles_x * tiles_y;
    const int tile = blockIdx.x % tiles;
    const int t_begin = (blockIdx.x / tiles) * t_chunk;
    const int t_end = min(t_begin + t_chunk, L.T - L.kt + 1);
    const int f_begin = t_begin, f_end = t_end + L.kt - 1;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int64_t OHt = L.x.H - KC + 1, OWt = L.x.W - KC + 1;
    const int64_t x0 = (int64_t)tx * OW3, y0 = (int64_t)ty * OHC;
    const int64_t N = (int64_t)KC * KC * L.kt;
    constexpr unsigned tile_bytes = IHC * RWC;
    auto issue = [&](int ff) {  // thread 0: the tiles of frame ff (and of ff - kt once it leaves a window)
        const bool with_old = ff - L.kt >= f_begin;
        mbar_expect_tx(&S.bar, (with_old ? 4u : 2u) * tile_bytes);
        tma_load_3d(S.raw[0], &tmx, (int)x0, (int)y0, ff, &S.bar);
        tma_load_3d(S.raw[1], &tmy, (int)x0, (int)y0, ff, &S.bar);
        if (with_old) {
            tma_load_3d(S.raw[2], &tmx, (int)x0, (int)y0, ff - L.kt, &S.bar);
            tma_load_3d(S.raw[3], &tmy, (int)x0, (int)y0, ff - L.kt, &S.bar);
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
        issue(f_begin);
    }
    __syncthreads();
    // column thread: quantity q (0 u, 1 w, 2 u^2, 3 w^2), input column c
    const int q = threadIdx.x / 80, c = threadIdx.x - 80 * q;
    const bool col = c < IWC;
    const int sgn = (q & 1) ? -1 : 1;  // w = x - y
    const bool sq = q >= 2;
    int T[IHC];
#pragma unroll
    for (int r = 0; r < IHC; ++r) T[r] = 0;
    unsigned phase = 0;
    int pending = -1;  // output frame whose warp sums wait in red[pending_buf]
    int pending_buf = 0;
    for (int f = f_begin; f < f_end; ++f) {
        const bool old = f - L.kt >= f_begin;
        const bool ok = mbar_wait_bounded(&S.bar, phase);
        phase ^= 1u;
        const bool out_frame = f >= f_begin + L.kt - 1;
        const int buf = f & 1;
        if (ok && col) {
            const unsigned char *rx = S.raw[0] + c, *ry = S.raw[1] + c;
            if (old) {
                const unsigned char *ox = S.raw[2] + c, *oy = S.raw[3] + c;
#pragma unroll
                for (int r = 0; r < IHC; ++r) {
                    const int a = (int)rx[r * RWC] + sgn * (int)ry[r * RWC];
                    const int ao = (int)ox[r * RWC] + sgn * (int)oy[r * RWC];
                    const int d = a - ao;
                    T[r] += sq ? d * (a + ao) : d;  // u^2 - uo^2 = (u - uo)(u + uo)
                }
            } else {
#pragma unroll
                for (int r = 0; r < IHC; ++r) {
                    const int a = (int)rx[r * RWC] + sgn * (int)ry[r * RWC];
                    T[r] += sq ? a * a : a;
                }
            }
            if (out_frame) {
                int v[OHC];
                int sum = 0;
#pragma unroll
                for (int m = 0; m < KC; ++m) sum += T[m];
                v[0] = sum;
#pragma unroll
                for (int i = 1; i < OHC; ++i) {
                    sum += T[i + KC - 1] - T[i - 1];
                    v[i] = sum;
                }
                int4 *dst = reinterpret_cast<int4 *>(&S.vs[buf][q][c][0]);
#pragma unroll
                for (int i = 0; i < OHC / 4; ++i) dst[i] = make_int4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                mbar_wait_bounded(&S.bar, phase ^ 1u);  // drain the copy that did not complete (bounded)
                for (int tt = max(t_begin, f - L.kt); tt < t_end; ++tt)
                    L.partials[(int64_t)tt * tiles + tile] = make_double2(nan(""), nan(""));
            }
            return;
        }
        if (threadIdx.x == 0) {
            if (pending >= 0) {
                double sq_ = 0.0, sc_ = 0.0;
#pragma unroll
                for (int w = 0; w < T3C / 32; ++w) {
                    sq_ += S.red[pending_buf][w].x;
                    sc_ += S.red[pending_buf][w].y;
                }
                L.partials[(int64_t)pending * tiles + tile] = make_double2(sq_, sc_);
                pending = -1;
            }
            // every column thread is done with this frame's tiles: refill them
            if (f + 1 < f_end) {
                fence_proxy_async_smem();
                issue(f + 1);
            }
        }
        if (!out_frame) continue;
        const int t = f - L.kt + 1;
        if (threadIdx.x >= NTC - T3C) {
            const int s3 = threadIdx.x - (NTC - T3C);
            const int i = s3 % OHC, j0 = (s3 / OHC) * SEGC;
            const int64_t a = y0 + i;
            float accQ = 0.f, accC = 0.f;
            if (a < OHt && x0 + j0 < OWt) {
                const int *v0 = &S.vs[buf][0][j0][i], *v1 = &S.vs[buf][1][j0][i];
                const int *v2 = &S.vs[buf][2][j0][i], *v3 = &S.vs[buf][3][j0][i];
                int su = 0, sw = 0, su2 = 0, sw2 = 0;
#pragma unroll
                for (int m = 0; m < KC; ++m) {
                    su += v0[m * PVC];
                    sw += v1[m * PVC];
                    su2 += v2[m * PVC];
                    sw2 += v3[m * PVC];
                }
                const int nout = (int)min((int64_t)SEGC, OWt - (x0 + j0));
                float *mrow = L.map ? L.map + t * L.map_fs + a * L.map_ld + x0 + j0 : nullptr;
#pragma unroll
                for (int e = 0; e < SEGC; ++e) {
                    if (e > 0) {
                        const int in = (e + KC - 1) * PVC, out = (e - 1) * PVC;
                        su += v0[in] - v0[out];
                        sw += v1[in] - v1[out];
                        su2 += v2[in] - v2[out];
                        sw2 += v3[in] - v3[out];
                    }
                    if (e < nout) {
                        // |Su|, |Sw| <= 510 N < 2^23: exact in fp32; Su^2 - Sw^2 = (Su - Sw)(Su + Sw) rounds once
                        const float fu = (float)su, fw = (float)sw;
                        const float A1 = fmaf(fu - fw, fu + fw, L.C1x2n2);
                        const float B1 = fmaf(fu, fu, fmaf(fw, fw, L.C1x2n2));
                        const int n32 = (int)N;
                        const int64_t Vu = (int64_t)n32 * su2 - (int64_t)su * su;
                        const int64_t Vw = (int64_t)n32 * sw2 - (int64_t)sw * sw;
                        // |Vu +- Vw| < 2 N^2 510^2 < 2^48: no 64-bit conversion
                        const float A2 = i48_to_f32(Vu - Vw) + L.C2x2n2, B2 = i48_to_f32(Vu + Vw) + L.C2x2n2;
                        const float cs = __fdividef(A2, B2);
                        const float qv = __fdividef(A1, B1) * cs;
                        accQ += qv;
                        accC += cs;
                        if (mrow) mrow[e] = qv;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                accQ += __shfl_down_sync(0xffffffffu, accQ, o);
                accC += __shfl_down_sync(0xffffffffu, accC, o);
            }
            if ((threadIdx.x & 31) == 0) S.red[buf][s3 >> 5] = make_double2((double)accQ, (double)accC);
        }
        pending = t;
        pending_buf = buf;
    }
    __syncthreads();
    if (threadIdx.x == 0 && pending >= 0) {
        double sq_ = 0.0, sc_ = 0.0;
#pragma unroll
        for (int w = 0; w < T3C / 32; ++w) {
            sq_ += S.red[pending_buf][w].x;
            sc_ += S.red[pending_buf][w].y;
        }
        L.partials[(int64_t)pending * tiles + tile] = make_double2(sq_, sc_);
    }
}

// One CTA per output frame: per level, the fixed-order sum of the frame's
// tile partials times 1 / positions -> (mean Q_j, mean cs_j); then the frame
// score (m_j = mean cs_j for j < S, m_S = mean Q_S, combined as in MS-SSIM).
__global__ void __launch_bounds__(256) frame_scores_kernel(const Ms3dFinalize F, double *frame_scores,
                                                           double *per_scale_out) {
    __shared__ double rq[256], rc[256];
    __shared__ double mq[GBSSIM_MAX_SCALES], mc[GBSSIM_MAX_SCALES];
    const int t = blockIdx.x;
    for (int j = 0; j < F.scales; ++j) {
        const double2 *p = F.partials[j] + (int64_t)t * F.items[j];
        double q = 0.0, c = 0.0;
        for (int i = threadIdx.x; i < F.items[j]; i += 256) {
            q += p[i].x;
            c += p[i].y;
        }
        rq[threadIdx.x] = q;
        rc[threadIdx.x] = c;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                rq[threadIdx.x] += rq[threadIdx.x + s];
                rc[threadIdx.x] += rc[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            mq[j] = rq[0] * F.inv_n[j];
            mc[j] = rc[0] * F.inv_n[j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double wsum = 0.0;
        for (int j = 0; j < F.scales; ++j) wsum += F.exps[j];
        double v = F.combine == GBSSIM_COMBINE_SUM ? 0.0 : 1.0;
        for (int j = 0; j < F.scales; ++j) {
            const double m = j == F.scales - 1 ? mq[j] : mc[j];
            if (F.combine == GBSSIM_COMBINE_SUM) v += F.exps[j] / wsum * m;
            else v *= pow(m, F.exps[j]);  // NaN for m < 0 under a non-integer exponent
            if (per_scale_out) {
                per_scale_out[((int64_t)t * F.scales + j) * 2] = mc[j];
                per_scale_out[((int64_t)t * F.scales + j) * 2 + 1] = mq[j];
            }
        }
        frame_scores[t] = v;
    }
}

// Mean of the frame scores in a fixed order (one CTA).
__global__ void __launch_bounds__(256) frame_mean_kernel(const double *frames, int n, double *out) {
    __shared__ double red[256];
    double loc = 0.0;
    for (int t = threadIdx.x; t < n; t += 256) loc += frames[t];
    red[threadIdx.x] = loc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / n;
}

template <typename A>
size_t smem_bytes(int k, bool bulk) {
    const size_t ih = Tile3<A>::OH + k - 1, iw = OW3 + k - 1, pw = (iw + 3) & ~(size_t)3;
    const size_t base = sizeof(A) * (4 * ih * pw + 4 * iw * Tile3<A>::PV) + sizeof(double2) * Tile3<A>::WARPS3;
    if (!bulk) return base;
    return ((base + 127) & ~(size_t)127) + 4 * ((ih * raw3_width(k) + 127) & ~(size_t)127) +
           sizeof(unsigned long long);
}

// Bulk-copy map of a uint8 video (columns, rows, frames) with rw x ih
// tiles; false when rows or frames are not 16-byte aligned.
bool encode_video_map(CUtensorMap *m, const ImgDesc &d, int T, int ih, int rw) {
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    if ((uintptr_t)d.data % 16 != 0 || d.row_stride % 16 != 0 || (T > 1 && d.image_stride % 16 != 0)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)d.W, (cuuint64_t)d.H, (cuuint64_t)T};
    const cuuint64_t strides[2] = {(cuuint64_t)d.row_stride,
                                   (cuuint64_t)(T > 1 ? d.image_stride : d.H * d.row_stride)};
    const cuuint32_t box[3] = {(cuuint32_t)rw, (cuuint32_t)ih, 1}, estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(d.data), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename A, typename In, bool BULK>
cudaError_t launch_level_k(const Ssim3dLaunch &L, const CUtensorMap &mx, const CUtensorMap &my, cudaStream_t st) {
    int tx, ty;
    ssim3d_tiles(L.x.H, L.x.W, L.k, sizeof(A) == 8, &tx, &ty);
    static DeviceOnce attr_set;
    static std::atomic<int> slots[64];  // SMs per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t smem = smem_bytes<A>(L.k, BULK);
    if (!attr_set.is_set(dev)) {
        const cudaError_t e = cudaFuncSetAttribute(ssim3d_kernel<A, In, BULK>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem_bytes<A>(kSsim3dMaxK, BULK));
        if (e != cudaSuccess) return e;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaErrorUnknown;
        slots[dev].store(sms, std::memory_order_relaxed);
        attr_set.set(dev);
    }
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ssim3d_kernel<A, In, BULK>, NT, smem) != cudaSuccess)
        return cudaErrorUnknown;
    // Split the output frames into chunks (each CTA primes its own temporal
    // sums with kt-1 frames) when the tiles alone fill fewer than two waves;
    // chunks keep at least max(2, kt) output frames.  Every output frame is
    // computed by one CTA with exact integer sums: the result does not depend
    // on the split.
    const int tiles = tx * ty, frames = L.T - L.kt + 1;
    const int wave = max(1, per_sm) * slots[dev].load(std::memory_order_relaxed);
    int chunks = 1;
    if (tiles < 2 * wave) {
        const int want = (2 * wave + tiles - 1) / tiles;
        chunks = max(1, min(want, frames / max(2, L.kt)));
    }
    const int t_chunk = (frames + chunks - 1) / chunks;
    chunks = (frames + t_chunk - 1) / t_chunk;
    ssim3d_kernel<A, In, BULK><<<tiles * chunks, NT, smem, st>>>(mx, my, L, tx, ty, t_chunk);
    return cudaGetLastError();
}

// The register-column kernel (uint8, k = 11, int32 sums, bulk copies): same
// tiles and partial layout as ssim3d_kernel<int>, the same frame chunking.
cudaError_t launch_cols(const Ssim3dLaunch &L, const CUtensorMap &mx, const CUtensorMap &my, cudaStream_t st) {
    int tx, ty;
    ssim3d_tiles(L.x.H, L.x.W, L.k, false, &tx, &ty);
    static DeviceOnce attr_set;
    static std::atomic<int> slots[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set.is_set(dev)) {
        const cudaError_t e = cudaFuncSetAttribute(ssim3d_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(S3C));
        if (e != cudaSuccess) return e;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaErrorUnknown;
        slots[dev].store(sms, std::memory_order_relaxed);
        attr_set.set(dev);
    }
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ssim3d_cols_kernel, NTC, sizeof(S3C)) != cudaSuccess)
        return cudaErrorUnknown;
    const int tiles = tx * ty, frames = L.T - L.kt + 1;
    const int wave = max(1, per_sm) * slots[dev].load(std::memory_order_relaxed);
    int chunks = 1;
    if (tiles < 2 * wave) {
        const int want = (2 * wave + tiles - 1) / tiles;
        chunks = max(1, min(want, frames / max(2, L.kt)));
    }
    const int t_chunk = (frames + chunks - 1) / chunks;
    chunks = (frames + t_chunk - 1) / t_chunk;
    ssim3d_cols_kernel<<<tiles * chunks, NTC, sizeof(S3C), st>>>(mx, my, L, tx, ty, t_chunk);
    return cudaGetLastError();
}

// uint8 video with 16-byte aligned rows and frames: bulk-copied tiles.
template <typename A, typename In>
cudaError_t launch_level(const Ssim3dLaunch &L, cudaStream_t st) {
    CUtensorMap mx, my;
    memset(&mx, 0, sizeof mx);
    memset(&my, 0, sizeof my);
    if constexpr (std::is_same<In, uint8_t>::value) {
        const int ih = Tile3<A>::OH + L.k - 1;
        const int rw = raw3_width(L.k);
        if (encode_video_map(&mx, L.x, L.T, ih, rw) && encode_video_map(&my, L.y, L.T, ih, rw)) {
            if constexpr (std::is_same<A, int>::value)
                if (L.k == KC) return launch_cols(L, mx, my, st);
            return launch_level_k<A, In, true>(L, mx, my, st);
        }
    }
    return launch_level_k<A, In, false>(L, mx, my, st);
}

}  // namespace

void ssim3d_tiles(int64_t H, int64_t W, int k, bool wide, int *tx, int *ty) {
    const int oh = wide ? Tile3<long long>::OH : Tile3<int>::OH;
    *tx = (int)((W - k + 1 + OW3 - 1) / OW3);
    *ty = (int)((H - k + 1 + oh - 1) / oh);
}

// Pyramid levels of uint8 video hold multiples of 1 / scale up to 255; as
// integers (times scale) the window sums of u = x + y and its square over
// N = k^2 kt pixels stay below 2 x 255 scale N and N (2 x 255 scale)^2.
// When those fit 2^23 (exact in fp32) and 2^32, the level runs with 32-bit
// sums kept modulo 2^32 (level 1 of an 11 x 11 x 5 window: 1.2 M and
// 2.5e9), else with int64 sums.
bool ssim3d_level_fits_u32(const Ssim3dLaunch &L) {
    const double n = (double)L.k * L.k * L.kt, umax = 2.0 * 255.0 * L.scale;
    return n * umax < 8388608.0 && n * umax * umax < 4294967296.0;
}

cudaError_t launch_ssim3d_level(const Ssim3dLaunch &L, bool u8_input, bool wide, cudaStream_t st) {
    if (!u8_input) return ssim3d_level_fits_u32(L) ? launch_level<unsigned, float>(L, st)
                                                   : launch_level<long long, float>(L, st);
    return wide ? launch_level<long long, uint8_t>(L, st) : launch_level<int, uint8_t>(L, st);
}

cudaError_t launch_ssim3d_finalize(const Ms3dFinalize &F, double *frame_scores, double *per_scale_out,
                                   double *score_out, cudaStream_t st) {
    frame_scores_kernel<<<F.frames, 256, 0, st>>>(F, frame_scores, per_scale_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !score_out) return e;
    frame_mean_kernel<<<1, 256, 0, st>>>(frame_scores, F.frames, score_out);
    return cudaGetLastError();
}

}  // namespace gbssim
