// k_gauss.cu -- fused SSIM kernels for separable windows (Gaussian, or a box
// window on non-integer inputs).
//
// What is computed (Background section of arXiv 2101.06354): for every valid
// window position the local means mu_x, mu_y, variances sigma_x^2, sigma_y^2
// and covariance sigma_xy under weights w(m,n) = g(m) g(n)
// (Eqs. local_means .. local_corr), then l = (2 mu_x mu_y + C1)/(mu_x^2 +
// mu_y^2 + C1) (Eq. lum_term), cs = (2 sigma_xy + C2)/(sigma_x^2 + sigma_y^2
// + C2) (the C3 = C2/2 form) and Q = l cs, mean-pooled per image.
//
// Precision.  sigma^2 = sum w x^2 - mu^2 cancels catastrophically in fp32 on
// flat windows far from zero (x ~ 255: sum w x^2 ~ 65025 with an ulp of
// 0.004, while |dQ/d sigma^2| <= 1/C2 = 0.017), which alone breaks a 1e-5
// per-element bound.  Both passes therefore work on SHIFTED data and combine
// the two directions through the law of total variance:
//   horizontal: for a group of 4 adjacent outputs of one row, subtract one
//     pixel c of that row lying inside all 4 windows (offset <= 2 taps from
//     each centre), and accumulate sum g d, sum g d^2, sum g dx dy with
//     d = x - c; the row-window mean is c + sum g d and its variance
//     sum g d^2 - (sum g d)^2;
//   vertical: for a group of 4 adjacent outputs of one column, subtract the
//     row-window mean b of one row inside all 4 windows and accumulate
//     sum g e, sum g (e^2 + v_row), sum g (ex ey + c_row) with e = mu_row - b;
//     the window variance is sum g (e^2 + v_row) - (sum g e)^2.
// Because the shift lies inside every window of its group, the shifted second
// moment is at most (1 + 1/g_min) times the variance it yields (g_min = the
// tap 2 away from the centre, 0.109 for sigma = 1.5), so rounding error stays
// relative to the local variance instead of to x^2.
//
// Fast kernel (11 taps, stride 1).  One CTA owns a strip of 64 output
// columns and a segment of `seg_rows` output rows.  It walks the segment in
// chunks of 16 rows: the horizontal pass writes its 5 per-row moments into a
// 32-row ring in shared memory, the vertical pass reads 26 ring rows per
// chunk, so every input row is filtered horizontally once per segment (10-row
// overlap between segments).  The next chunk's input rows are prefetched into
// registers while the current chunk is filtered.  For MS-SSIM the same CTA
// also writes the 2x2 average of the input rows/columns it owns (the next
// pyramid level), so the input is read from HBM once per level.
#include "common.cuh"

namespace gbssim {
namespace {

constexpr int K = 11;
constexpr int HALO = K - 1;       // 10
constexpr int TW = 64;            // output columns per strip
constexpr int CH = 16;            // output rows per chunk
constexpr int RING = 32;          // ring rows (>= CH + HALO, power of two)
constexpr int FIRST = CH + HALO;  // input rows staged for the first chunk
constexpr int IW = TW + HALO;     // input columns per strip (74)
constexpr int IWP = 80;           // staged row pitch in floats
constexpr int NT = 256;
constexpr int QUADS = (IW + 3) / 4;             // 4-column staging units per row (19)
constexpr int PFQ = (2 * CH * QUADS + NT - 1) / NT;  // prefetched quads per thread (3)
// The vertical pass of a thread reads ring rows base..base+13 with base a
// multiple of 4 below RING; rows 0..DUP-1 are also stored at RING..RING+DUP-1
// so those reads never wrap.
constexpr int DUP = 10;
constexpr int RROWS = RING + DUP;

struct __align__(16) Smem {
    float in_x[FIRST][IWP];
    float in_y[FIRST][IWP];
    float mu_x[RROWS][TW];
    float mu_y[RROWS][TW];
    float v_x[RROWS][TW];
    float v_y[RROWS][TW];
    float c_xy[RROWS][TW];
    float red[2 * NT / 32];
};

struct Geo {
    const void *xb, *yb;
    int64_t H, W, rs, OH, OW;
    int64_t j0;        // first output / input column of the strip
    int64_t o0, oend;  // output rows [o0, oend)
    int64_t own_r1;    // owned input rows [o0, own_r1) (downsample)
    int64_t own_c1;    // owned input columns [j0, own_c1)
    bool vec;          // rows and strip start aligned for 4-element vector loads
};

// Four consecutive elements (columns c..c+3 of one row) as floats; zero
// outside the image.  `vec`: the row start and c are aligned for one vector
// load of four elements.
__device__ __forceinline__ float u8f(unsigned w, int k) {
    // byte k of w placed in the mantissa of 2^23, minus 2^23: exact for 0..255
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7540u + k)) - 8388608.0f;
}
template <typename T>
__device__ __forceinline__ float4 load_quad(const T *row, int64_t c, int64_t W, bool vec);
template <>
__device__ __forceinline__ float4 load_quad<uint8_t>(const uint8_t *row, int64_t c, int64_t W, bool vec) {
    if (vec && c + 4 <= W) {
        const unsigned w = __ldg(reinterpret_cast<const unsigned *>(row + c));
        return make_float4(u8f(w, 0), u8f(w, 1), u8f(w, 2), u8f(w, 3));
    }
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = c + k < W ? (float)__ldg(row + c + k) : 0.f;
    return make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ float4 load_quad<float>(const float *row, int64_t c, int64_t W, bool vec) {
    if (vec && c + 4 <= W) return __ldg(reinterpret_cast<const float4 *>(row + c));
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = c + k < W ? __ldg(row + c + k) : 0.f;
    return make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ float4 load_quad<__half>(const __half *row, int64_t c, int64_t W, bool vec) {
    if (vec && c + 4 <= W) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(row + c));
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = c + k < W ? load_f32<__half>(row + c + k) : 0.f;
    return make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ float4 load_quad<__nv_bfloat16>(const __nv_bfloat16 *row, int64_t c, int64_t W,
                                                           bool vec) {
    if (vec && c + 4 <= W) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(row + c));
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    }
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = c + k < W ? load_f32<__nv_bfloat16>(row + c + k) : 0.f;
    return make_float4(v[0], v[1], v[2], v[3]);
}

// Staging unit t (of 2*nr*QUADS): image (x or y), row within the block, quad.
template <typename T>
__device__ __forceinline__ float4 fetch_unit(const Geo &g, int t, int nr, int64_t r0, int &which, int &r,
                                             int &u) {
    which = t >= nr * QUADS;
    const int rem = t - which * nr * QUADS;
    r = rem / QUADS;
    u = rem - r * QUADS;
    const int64_t row = r0 + r;
    if (row >= g.H) return make_float4(0.f, 0.f, 0.f, 0.f);
    const T *base = static_cast<const T *>(which ? g.yb : g.xb) + row * g.rs;
    return load_quad<T>(base, g.j0 + 4 * u, g.W, g.vec);
}

__device__ __forceinline__ void put_unit(Smem &S, int which, int r, int u, float4 v) {
    *reinterpret_cast<float4 *>(&(which ? S.in_y : S.in_x)[r][4 * u]) = v;
}

// Stage `nr` input rows starting at absolute row r0 into in_x/in_y rows 0..nr-1.
template <typename T>
__device__ __forceinline__ void stage_direct(Smem &S, const Geo &g, int64_t r0, int nr) {
    for (int t = threadIdx.x; t < 2 * nr * QUADS; t += NT) {
        int which, r, u;
        const float4 v = fetch_unit<T>(g, t, nr, r0, which, r, u);
        put_unit(S, which, r, u, v);
    }
}

// Raw (unconverted) four-element load for the register prefetch: the
// conversion to float happens only when the data is stored to shared memory,
// so the load latency overlaps the barrier and the vertical pass.  `packed`:
// one vector load (element bits packed as in memory); otherwise component k
// holds element k's bits.  Zero outside the image.
template <typename T>
__device__ __forceinline__ uint4 load_raw(const T *p, int ncols, bool packed) {
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (packed) {
        if (sizeof(T) == 1) r.x = __ldg(reinterpret_cast<const unsigned *>(p));
        else if (sizeof(T) == 2) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
            r.x = v.x;
            r.y = v.y;
        } else r = __ldg(reinterpret_cast<const uint4 *>(p));
        return r;
    }
    unsigned v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < ncols) {
            if (sizeof(T) == 1) v[k] = __ldg(reinterpret_cast<const unsigned char *>(p) + k);
            else if (sizeof(T) == 2) v[k] = __ldg(reinterpret_cast<const unsigned short *>(p) + k);
            else v[k] = __ldg(reinterpret_cast<const unsigned *>(p) + k);
        }
    return make_uint4(v[0], v[1], v[2], v[3]);
}

template <typename T>
__device__ __forceinline__ float elem_f32(unsigned bits);
template <>
__device__ __forceinline__ float elem_f32<uint8_t>(unsigned b) { return u8f(b, 0); }
template <>
__device__ __forceinline__ float elem_f32<__half>(unsigned b) {
    return __half2float(__ushort_as_half((unsigned short)b));
}
template <>
__device__ __forceinline__ float elem_f32<__nv_bfloat16>(unsigned b) { return __uint_as_float(b << 16); }
template <>
__device__ __forceinline__ float elem_f32<float>(unsigned b) { return __uint_as_float(b); }

template <typename T>
__device__ __forceinline__ float4 convert_raw(uint4 r, bool packed) {
    if (!packed || sizeof(T) == 4)
        return make_float4(elem_f32<T>(r.x), elem_f32<T>(r.y), elem_f32<T>(r.z), elem_f32<T>(r.w));
    if (sizeof(T) == 1) return make_float4(u8f(r.x, 0), u8f(r.x, 1), u8f(r.x, 2), u8f(r.x, 3));
    return make_float4(elem_f32<T>(r.x & 0xffffu), elem_f32<T>(r.x >> 16), elem_f32<T>(r.y & 0xffffu),
                       elem_f32<T>(r.y >> 16));
}

// Per-thread staging units of a 16-row chunk, fixed for the whole CTA.
struct Units {
    unsigned dst[PFQ];       // byte offset of the shared-memory destination
    const char *src[PFQ];    // global address of the unit in chunk row 0
    int r[PFQ];              // row within the chunk (-1: no unit)
    int ncols[PFQ];          // columns inside the image (0..4)
    bool packed[PFQ];
};

template <typename T>
__device__ __forceinline__ void make_units(Units &U, Smem &S, const Geo &g) {
#pragma unroll
    for (int i = 0; i < PFQ; ++i) {
        const int t = threadIdx.x + i * NT;
        U.r[i] = -1;
        U.ncols[i] = 0;
        U.packed[i] = false;
        U.dst[i] = 0;
        U.src[i] = nullptr;
        if (t < 2 * CH * QUADS) {
            const int which = t >= CH * QUADS;
            const int rem = t - which * CH * QUADS;
            const int r = rem / QUADS, q = rem - r * QUADS;
            const int64_t c = g.j0 + 4 * q;
            U.r[i] = r;
            U.ncols[i] = (int)max((int64_t)0, min((int64_t)4, g.W - c));
            U.packed[i] = g.vec && U.ncols[i] == 4;
            U.dst[i] = (unsigned)(reinterpret_cast<const char *>(&(which ? S.in_y : S.in_x)[r][4 * q]) -
                                  reinterpret_cast<const char *>(&S));
            U.src[i] = reinterpret_cast<const char *>(static_cast<const T *>(which ? g.yb : g.xb) + r * g.rs + c);
        }
    }
}

template <typename T>
__device__ __forceinline__ void prefetch(uint4 (&pf)[PFQ], const Units &U, const Geo &g, int64_t r0) {
    const int64_t off = r0 * g.rs * (int64_t)sizeof(T);
#pragma unroll
    for (int i = 0; i < PFQ; ++i) {
        pf[i] = make_uint4(0u, 0u, 0u, 0u);
        if (U.r[i] >= 0 && r0 + U.r[i] < g.H && U.ncols[i] > 0)
            pf[i] = load_raw<T>(reinterpret_cast<const T *>(U.src[i] + off), U.ncols[i], U.packed[i]);
    }
}

template <typename T>
__device__ __forceinline__ void store_prefetch(Smem &S, const uint4 (&pf)[PFQ], const Units &U) {
#pragma unroll
    for (int i = 0; i < PFQ; ++i)
        if (U.r[i] >= 0)
            *reinterpret_cast<float4 *>(reinterpret_cast<char *>(&S) + U.dst[i]) = convert_raw<T>(pf[i], U.packed[i]);
}

// 2x2 average of the owned part of the staged rows (absolute rows r0..r0+nr-1).
__device__ __forceinline__ void downsample_rows(const Smem &S, const Geo &g, int64_t r0, int nr,
                                                float *dsx, float *dsy) {
    const int64_t Hh = g.H >> 1, Wh = g.W >> 1;
    constexpr int QC = (IW + 1) / 2;  // 37 column pairs staged
    for (int t = threadIdx.x; t < (nr >> 1) * QC; t += NT) {
        const int p = t / QC, q = t - p * QC;
        const int64_t r = r0 + 2 * p, c = g.j0 + 2 * q;
        if (r >= g.own_r1 || c >= g.own_c1) continue;
        const int64_t R = r >> 1, C = c >> 1;
        if (R >= Hh || C >= Wh) continue;
        const float ax = (S.in_x[2 * p][2 * q] + S.in_x[2 * p][2 * q + 1]) +
                         (S.in_x[2 * p + 1][2 * q] + S.in_x[2 * p + 1][2 * q + 1]);
        const float ay = (S.in_y[2 * p][2 * q] + S.in_y[2 * p][2 * q + 1]) +
                         (S.in_y[2 * p + 1][2 * q] + S.in_y[2 * p + 1][2 * q + 1]);
        dsx[R * Wh + C] = 0.25f * ax;
        dsy[R * Wh + C] = 0.25f * ay;
    }
}

// Horizontal pass over staged rows 0..nr-1; results go to ring rows
// (rel0 + r) & (RING-1), where rel0 is the row index relative to the segment.
__device__ __forceinline__ void horizontal(Smem &S, int nr, int rel0, const Taps<K> &t) {
    for (int task = threadIdx.x; task < nr * (TW / 4); task += NT) {
        const int r = task >> 4, g4 = (task & 15) * 4;
        float xv[14], yv[14];
        {
            const float4 a0 = *reinterpret_cast<const float4 *>(&S.in_x[r][g4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&S.in_x[r][g4 + 4]);
            const float4 a2 = *reinterpret_cast<const float4 *>(&S.in_x[r][g4 + 8]);
            const float2 a3 = *reinterpret_cast<const float2 *>(&S.in_x[r][g4 + 12]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&S.in_y[r][g4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&S.in_y[r][g4 + 4]);
            const float4 b2 = *reinterpret_cast<const float4 *>(&S.in_y[r][g4 + 8]);
            const float2 b3 = *reinterpret_cast<const float2 *>(&S.in_y[r][g4 + 12]);
            xv[0] = a0.x; xv[1] = a0.y; xv[2] = a0.z; xv[3] = a0.w;
            xv[4] = a1.x; xv[5] = a1.y; xv[6] = a1.z; xv[7] = a1.w;
            xv[8] = a2.x; xv[9] = a2.y; xv[10] = a2.z; xv[11] = a2.w;
            xv[12] = a3.x; xv[13] = a3.y;
            yv[0] = b0.x; yv[1] = b0.y; yv[2] = b0.z; yv[3] = b0.w;
            yv[4] = b1.x; yv[5] = b1.y; yv[6] = b1.z; yv[7] = b1.w;
            yv[8] = b2.x; yv[9] = b2.y; yv[10] = b2.z; yv[11] = b2.w;
            yv[12] = b3.x; yv[13] = b3.y;
        }
        // shift: pixel 7 lies in the windows of outputs 0..3 (centres 5..8)
        const float cx = xv[7], cy = yv[7];
        float mx[4], my[4], sxx[4], syy[4], sxy[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) mx[o] = my[o] = sxx[o] = syy[o] = sxy[o] = 0.f;
#pragma unroll
        for (int i = 0; i < 14; ++i) {
            const float dx = xv[i] - cx, dy = yv[i] - cy;
            const float pxx = dx * dx, pyy = dy * dy, pxy = dx * dy;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int n = i - o;
                if (n >= 0 && n < K) {
                    const float w = t.g[n];
                    mx[o] = fmaf(w, dx, mx[o]);
                    my[o] = fmaf(w, dy, my[o]);
                    sxx[o] = fmaf(w, pxx, sxx[o]);
                    syy[o] = fmaf(w, pyy, syy[o]);
                    sxy[o] = fmaf(w, pxy, sxy[o]);
                }
            }
        }
        const int slot = (rel0 + r) & (RING - 1);
        float4 o_mx, o_my, o_vx, o_vy, o_c;
        o_mx.x = mx[0] + cx; o_mx.y = mx[1] + cx; o_mx.z = mx[2] + cx; o_mx.w = mx[3] + cx;
        o_my.x = my[0] + cy; o_my.y = my[1] + cy; o_my.z = my[2] + cy; o_my.w = my[3] + cy;
        o_vx.x = fmaf(-mx[0], mx[0], sxx[0]); o_vx.y = fmaf(-mx[1], mx[1], sxx[1]);
        o_vx.z = fmaf(-mx[2], mx[2], sxx[2]); o_vx.w = fmaf(-mx[3], mx[3], sxx[3]);
        o_vy.x = fmaf(-my[0], my[0], syy[0]); o_vy.y = fmaf(-my[1], my[1], syy[1]);
        o_vy.z = fmaf(-my[2], my[2], syy[2]); o_vy.w = fmaf(-my[3], my[3], syy[3]);
        o_c.x = fmaf(-mx[0], my[0], sxy[0]); o_c.y = fmaf(-mx[1], my[1], sxy[1]);
        o_c.z = fmaf(-mx[2], my[2], sxy[2]); o_c.w = fmaf(-mx[3], my[3], sxy[3]);
        *reinterpret_cast<float4 *>(&S.mu_x[slot][g4]) = o_mx;
        *reinterpret_cast<float4 *>(&S.mu_y[slot][g4]) = o_my;
        *reinterpret_cast<float4 *>(&S.v_x[slot][g4]) = o_vx;
        *reinterpret_cast<float4 *>(&S.v_y[slot][g4]) = o_vy;
        *reinterpret_cast<float4 *>(&S.c_xy[slot][g4]) = o_c;
        if (slot < DUP) {
            *reinterpret_cast<float4 *>(&S.mu_x[slot + RING][g4]) = o_mx;
            *reinterpret_cast<float4 *>(&S.mu_y[slot + RING][g4]) = o_my;
            *reinterpret_cast<float4 *>(&S.v_x[slot + RING][g4]) = o_vx;
            *reinterpret_cast<float4 *>(&S.v_y[slot + RING][g4]) = o_vy;
            *reinterpret_cast<float4 *>(&S.c_xy[slot + RING][g4]) = o_c;
        }
    }
}

// Vertical pass + SSIM formula for the 16 output rows starting at rel0
// (relative to the segment); each thread does 4 rows of one column.
__device__ __forceinline__ void vertical(const Smem &S, const Geo &g, int rel0, const Taps<K> &t,
                                         const SsimConst &cc, float *map, int64_t map_ld, bool col_ok,
                                         float &sumQ, float &sumCS) {
    const int col = threadIdx.x & (TW - 1);
    const int base = rel0 + 4 * (threadIdx.x >> 6);
    const int b0 = base & (RING - 1);  // multiple of 4; b0 + 13 < RROWS
    const float bx = S.mu_x[b0 + 7][col], by = S.mu_y[b0 + 7][col];
    float mx[4], my[4], sxx[4], syy[4], sxy[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) mx[o] = my[o] = sxx[o] = syy[o] = sxy[o] = 0.f;
#pragma unroll
    for (int i = 0; i < 14; ++i) {
        const int s = b0 + i;
        const float ex = S.mu_x[s][col] - bx, ey = S.mu_y[s][col] - by;
        const float qxx = fmaf(ex, ex, S.v_x[s][col]);
        const float qyy = fmaf(ey, ey, S.v_y[s][col]);
        const float qxy = fmaf(ex, ey, S.c_xy[s][col]);
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int n = i - o;
            if (n >= 0 && n < K) {
                const float w = t.g[n];
                mx[o] = fmaf(w, ex, mx[o]);
                my[o] = fmaf(w, ey, my[o]);
                sxx[o] = fmaf(w, qxx, sxx[o]);
                syy[o] = fmaf(w, qyy, syy[o]);
                sxy[o] = fmaf(w, qxy, sxy[o]);
            }
        }
    }
    const int rows_left = col_ok ? (int)(g.oend - g.o0) - base : 0;
    float *mrow = map ? map + (g.o0 + base) * map_ld + g.j0 + col : nullptr;
    sumQ = 0.f;
    sumCS = 0.f;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const float ux = mx[o] + bx, uy = my[o] + by;
        const float vx = fmaf(-mx[o], mx[o], sxx[o]);
        const float vy = fmaf(-my[o], my[o], syy[o]);
        const float cv = fmaf(-mx[o], my[o], sxy[o]);
        const float A1 = fmaf(2.f * ux, uy, cc.C1), B1 = fmaf(ux, ux, fmaf(uy, uy, cc.C1));
        const float A2 = fmaf(2.f, cv, cc.C2), B2 = (vx + vy) + cc.C2;
        const float l = __fdividef(A1, B1), cs = __fdividef(A2, B2);
        const float q = l * cs;
        if (o < rows_left) {
            sumQ += q;
            sumCS += cs;
            if (mrow) mrow[o * map_ld] = q;
        }
    }
}

// Compensated (Kahan) fp32 running sum.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Sum (a, b) over the CTA: fp32 pairwise tree inside each warp, fp64 across
// warps; the result is valid in thread 0.
__device__ __forceinline__ void block_sum2f(float a, float b, float *red, double &ra, double &rb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        red[2 * warp] = a;
        red[2 * warp + 1] = b;
    }
    __syncthreads();
    ra = rb = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) {
            ra += (double)red[2 * w];
            rb += (double)red[2 * w + 1];
        }
}

template <typename T>
__global__ void __launch_bounds__(NT, 3) gauss11_kernel(const GaussLaunch L, int strips, int segs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int strip = blockIdx.x, seg = blockIdx.y, img = blockIdx.z;

    Geo g;
    g.H = L.x.H;
    g.W = L.x.W;
    g.rs = L.x.row_stride;
    g.OH = g.H - HALO;
    g.OW = g.W - HALO;
    g.xb = static_cast<const T *>(L.x.data) + img * L.x.image_stride;
    g.yb = static_cast<const T *>(L.y.data) + img * L.y.image_stride;
    g.j0 = (int64_t)strip * TW;
    g.o0 = (int64_t)seg * L.seg_rows;
    g.oend = min(g.o0 + (int64_t)L.seg_rows, g.OH);
    g.own_r1 = (seg == segs - 1) ? g.H : g.o0 + L.seg_rows;
    g.own_c1 = (strip == strips - 1) ? g.W : g.j0 + TW;
    const int nchunks = (int)((g.oend - g.o0 + CH - 1) / CH);
    g.vec = L.vec;
    float *map = L.map ? L.map + img * L.map_is : nullptr;
    const int64_t dsn = (g.H >> 1) * (g.W >> 1);
    float *dsx = L.ds_x ? L.ds_x + img * dsn : nullptr;
    float *dsy = L.ds_y ? L.ds_y + img * dsn : nullptr;

    KSum accQ, accCS;
    uint4 pf[PFQ];
    Units U;
    make_units<T>(U, S, g);
    const bool col_ok = g.j0 + (threadIdx.x & (TW - 1)) < g.OW;

    stage_direct<T>(S, g, g.o0, FIRST);
    __syncthreads();
    if (dsx) downsample_rows(S, g, g.o0, FIRST, dsx, dsy);
    horizontal(S, FIRST, 0, L.taps);
    for (int c = 0; c < nchunks; ++c) {
        const bool more = c + 1 < nchunks;
        const int64_t next_r0 = g.o0 + FIRST + (int64_t)CH * c;
        if (more) prefetch<T>(pf, U, g, next_r0);
        __syncthreads();  // ring rows of chunk c complete; staging free
        float cq, ccs;
        vertical(S, g, CH * c, L.taps, L.c, map, L.map_ld, col_ok, cq, ccs);
        accQ.add(cq);
        accCS.add(ccs);
        if (more) store_prefetch<T>(S, pf, U);
        __syncthreads();  // staging complete; ring rows of chunk c consumed
        if (more) {
            if (dsx) downsample_rows(S, g, next_r0, CH, dsx, dsy);
            horizontal(S, CH, FIRST + CH * c, L.taps);
        }
    }
    double a, b;
    block_sum2f(accQ.s - accQ.c, accCS.s - accCS.c, S.red, a, b);
    if (threadIdx.x == 0)
        L.partials[((int64_t)img * segs + seg) * strips + strip] = make_double2(a, b);
}

// ----------------------------------------------------------------- generic path
//
// One thread per output; any k <= GBSSIM_MAX_K and any stride.  Same shifted
// two-level scheme with one group per output: the horizontal shift is the
// window's centre pixel of that row, the vertical shift the centre row's mean.

constexpr int GT = 16;  // 16 x 16 outputs per CTA

template <typename T>
__device__ __forceinline__ void row_moments(const T *xr, const T *yr, int k, const TapsDyn &t,
                                            float &mx, float &my, float &vx, float &vy,
                                            float &cv) {
    const float cx = load_f32<T>(xr + k / 2), cy = load_f32<T>(yr + k / 2);
    float sx = 0.f, sy = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
    for (int n = 0; n < k; ++n) {
        const float w = t.g[n];
        const float dx = load_f32<T>(xr + n) - cx, dy = load_f32<T>(yr + n) - cy;
        sx = fmaf(w, dx, sx);
        sy = fmaf(w, dy, sy);
        sxx = fmaf(w, dx * dx, sxx);
        syy = fmaf(w, dy * dy, syy);
        sxy = fmaf(w, dx * dy, sxy);
    }
    mx = sx + cx;
    my = sy + cy;
    vx = fmaf(-sx, sx, sxx);
    vy = fmaf(-sy, sy, syy);
    cv = fmaf(-sx, sy, sxy);
}

template <typename T>
__global__ void __launch_bounds__(GT *GT) generic_kernel(const GenericLaunch L, int tiles_x,
                                                         int tiles_y) {
    __shared__ double red[2 * GT * GT / 32];
    const int img = blockIdx.z;
    const int k = L.k, s = L.stride;
    const int64_t OH = out_dim(L.x.H, k, s), OW = out_dim(L.x.W, k, s);
    const int64_t a = (int64_t)blockIdx.y * GT + (threadIdx.x / GT);
    const int64_t b = (int64_t)blockIdx.x * GT + (threadIdx.x % GT);
    float q = 0.f, cs = 0.f;
    if (a < OH && b < OW) {
        const T *xb = static_cast<const T *>(L.x.data) + img * L.x.image_stride;
        const T *yb = static_cast<const T *>(L.y.data) + img * L.y.image_stride;
        const int64_t rs = L.x.row_stride;
        const int64_t i0 = a * s, j0 = b * s;
        float bx, by, d0, d1, d2;
        row_moments<T>(xb + (i0 + k / 2) * rs + j0, yb + (i0 + k / 2) * rs + j0, k, L.taps, bx, by,
                       d0, d1, d2);
        float mx = 0.f, my = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
        for (int m = 0; m < k; ++m) {
            float hx, hy, vx, vy, cv;
            row_moments<T>(xb + (i0 + m) * rs + j0, yb + (i0 + m) * rs + j0, k, L.taps, hx, hy, vx,
                           vy, cv);
            const float w = L.taps.g[m];
            const float ex = hx - bx, ey = hy - by;
            mx = fmaf(w, ex, mx);
            my = fmaf(w, ey, my);
            sxx = fmaf(w, fmaf(ex, ex, vx), sxx);
            syy = fmaf(w, fmaf(ey, ey, vy), syy);
            sxy = fmaf(w, fmaf(ex, ey, cv), sxy);
        }
        const float ux = mx + bx, uy = my + by;
        const float vx = fmaf(-mx, mx, sxx), vy = fmaf(-my, my, syy), cv = fmaf(-mx, my, sxy);
        const float A1 = fmaf(2.f * ux, uy, L.c.C1), B1 = fmaf(ux, ux, fmaf(uy, uy, L.c.C1));
        const float A2 = fmaf(2.f, cv, L.c.C2), B2 = (vx + vy) + L.c.C2;
        const float l = __fdividef(A1, B1);
        cs = __fdividef(A2, B2);
        q = l * cs;
        if (L.map) L.map[img * L.map_is + a * L.map_ld + b] = q;
    }
    double sa = q, sb = cs;
    block_sum2(sa, sb, red);
    if (threadIdx.x == 0)
        L.partials[((int64_t)img * tiles_y + blockIdx.y) * tiles_x + blockIdx.x] = make_double2(sa, sb);
}

template <typename T>
cudaError_t launch_gauss11_t(const GaussLaunch &L, cudaStream_t st) {
    static bool attr_set = false;
    const size_t smem = sizeof(Smem);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(gauss11_kernel<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int strips, segs;
    gauss11_items(L.x.H, L.x.W, L.seg_rows, &strips, &segs);
    GaussLaunch A = L;
    const uintptr_t vbytes = 4 * sizeof(T);  // one 4-element vector
    A.vec = ((uintptr_t)L.x.data % vbytes == 0) && ((uintptr_t)L.y.data % vbytes == 0) &&
            (L.x.row_stride % 4 == 0) && (L.x.image_stride % 4 == 0) && (L.y.image_stride % 4 == 0);
    dim3 grid(strips, segs, L.count);
    gauss11_kernel<T><<<grid, NT, smem, st>>>(A, strips, segs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_generic_t(const GenericLaunch &L, cudaStream_t st) {
    const int64_t OH = out_dim(L.x.H, L.k, L.stride), OW = out_dim(L.x.W, L.k, L.stride);
    const int tx = (int)((OW + GT - 1) / GT), ty = (int)((OH + GT - 1) / GT);
    dim3 grid(tx, ty, L.count);
    generic_kernel<T><<<grid, GT * GT, 0, st>>>(L, tx, ty);
    return cudaGetLastError();
}

}  // namespace

int gauss11_items(int64_t H, int64_t W, int seg_rows, int *strips, int *segs) {
    const int64_t OH = H - HALO, OW = W - HALO;
    *strips = (int)((OW + TW - 1) / TW);
    *segs = (int)((OH + seg_rows - 1) / seg_rows);
    return *strips * *segs;
}

cudaError_t launch_gauss11(const GaussLaunch &L, cudaStream_t st) {
    switch (L.dtype) {
    case GBSSIM_U8: return launch_gauss11_t<uint8_t>(L, st);
    case GBSSIM_F16: return launch_gauss11_t<__half>(L, st);
    case GBSSIM_BF16: return launch_gauss11_t<__nv_bfloat16>(L, st);
    case GBSSIM_F32: return launch_gauss11_t<float>(L, st);
    }
    return cudaErrorInvalidValue;
}

int generic_items(int64_t OH, int64_t OW) {
    return (int)(((OW + GT - 1) / GT) * ((OH + GT - 1) / GT));
}

cudaError_t launch_generic(const GenericLaunch &L, cudaStream_t st) {
    switch (L.dtype) {
    case GBSSIM_U8: return launch_generic_t<uint8_t>(L, st);
    case GBSSIM_F16: return launch_generic_t<__half>(L, st);
    case GBSSIM_BF16: return launch_generic_t<__nv_bfloat16>(L, st);
    case GBSSIM_F32: return launch_generic_t<float>(L, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gbssim
