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
// Four moments instead of five.  The formula needs sigma_x^2 + sigma_y^2 and
// sigma_xy only through A2 = 2 sigma_xy + C2 and B2 = sigma_x^2 + sigma_y^2
// + C2, and mu_x, mu_y only through A1 and B1.  With u = x + y and w = x - y,
// Var u = s_x^2 + s_y^2 + 2 s_xy and Var w = s_x^2 + s_y^2 - 2 s_xy, so
//   cs = (Var u - Var w + 2 C2) / (Var u + Var w + 2 C2),
//   l  = (mu_u^2 - mu_w^2 + 2 C1) / (mu_u^2 + mu_w^2 + 2 C1),
// an exact regrouping of Eq. lum_term and the cs term.  The kernel therefore
// filters the pair (u, w) and its squares: two packed f32x2 moments per
// window, with no scalar cross product.
//
// Precision.  sigma^2 = sum w x^2 - mu^2 cancels catastrophically in fp32 on
// flat windows far from zero (x ~ 255: sum w x^2 ~ 65025 with an ulp of
// 0.004, while |dQ/d sigma^2| <= 1/C2 = 0.017), which alone breaks a 1e-5
// per-element bound.  Both passes therefore work on SHIFTED data and combine
// the two directions through the law of total variance:
//   horizontal: for a group of 4 adjacent outputs of one row, subtract one
//     pixel c of that row lying inside all 4 windows (offset <= 2 taps from
//     each centre), and accumulate sum g d and sum g d^2 with d = p - c
//     (p = u or w); the row-window mean is c + sum g d and its variance
//     sum g d^2 - (sum g d)^2;
//   vertical: for a group of 4 adjacent outputs of one column, subtract the
//     row-window mean b of one row inside all 4 windows and accumulate
//     sum g e and sum g (e^2 + v_row) with e = mu_row - b; the window
//     variance is sum g (e^2 + v_row) - (sum g e)^2.
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
#include <type_traits>

#include "tma.cuh"

namespace gbssim {
namespace {

constexpr int K = 11;
constexpr int HALO = K - 1;       // 10
constexpr int CH = 16;            // output rows per chunk
constexpr int RING = 32;          // ring rows (>= CH + HALO, power of two)
constexpr int FIRST = CH + HALO;  // input rows staged for the first chunk

// Strip geometry: TW output columns per strip (work item), NT = 4 TW threads
// (in the vertical pass each thread takes 4 output rows of one column).  The
// single-image, MS-SSIM and backward kernels use TW = 64; the ragged-batch
// kernel is also built for 32 and 128, a tuning choice.
// Row pitches of the staged rows (IWP pairs) and of the moment ring (RWP
// pairs) are odd in 16-byte slots (39 and 33 at TW = 64): the horizontal
// pass gives each quarter-warp 4 output groups of 2 adjacent rows, whose
// 16-byte accesses then fall on the even and the odd bank groups
// respectively, so no access of the pass conflicts and every tap offset is a
// compile-time constant.
// Chunks of 16 input rows may arrive by bulk tensor copies instead of
// per-thread register prefetch: one 2-D tile of TMA_COLS elements x CH rows
// per image, x then y, into the staging area that follows the shared-memory
// struct (dense rows of TMA_COLS * sizeof(element) bytes), and the staging
// threads then read their units from there.
template <int TW_>
struct Geom {
    static constexpr int TW = TW_;
    static constexpr int NT = 4 * TW;
    static constexpr int IW = TW + HALO;                  // input columns per strip (74)
    static constexpr int QUADS = (IW + 3) / 4;            // 4-column staging units per row (19)
    static constexpr int IWP = 4 * QUADS + 2;             // staged row pitch in (u, w) pairs (78)
    static constexpr int RWP = TW + 2;                    // ring row pitch in pairs (66)
    static constexpr int TMA_COLS = (4 * QUADS + 15) / 16 * 16;  // 16-byte multiple for every dtype (80)
    static_assert(TW % 16 == 0 && (IWP / 2) % 2 == 1 && (RWP / 2) % 2 == 1, "odd row pitches in 16-byte slots");
    static_assert(CH / 2 * QUADS <= NT, "one staging unit per thread per chunk");
    static_assert(4 * QUADS <= TMA_COLS && TMA_COLS <= 256, "bulk-copy box");
};

// u = x + y and w = x - y travel together as float2 pairs so that every
// moment of the pair is one packed f32x2 instruction (FFMA2 / FADD2 / FMUL2
// on sm_100+).
template <int TW>
struct __align__(128) Smem {
    float2 in[FIRST][Geom<TW>::IWP];  // staged input rows, (u, w) per column
    float2 mu[RING][Geom<TW>::RWP];   // row-window means (mu_u, mu_w)
    float2 v[RING][Geom<TW>::RWP];    // row-window variances (v_u, v_w)
    float red[2 * Geom<TW>::NT / 32];
    unsigned long long bar;  // completion of the bulk copies
};
// The vertical pass reads S.v at a fixed offset from S.mu.
static_assert(offsetof(Smem<32>, v) == offsetof(Smem<32>, mu) + sizeof(float2) * RING * Geom<32>::RWP, "mu, v");
static_assert(offsetof(Smem<64>, v) == offsetof(Smem<64>, mu) + sizeof(float2) * RING * Geom<64>::RWP, "mu, v");
static_assert(offsetof(Smem<128>, v) == offsetof(Smem<128>, mu) + sizeof(float2) * RING * Geom<128>::RWP, "mu, v");
// Shared memory of a launch: Smem, then (bulk-copy variants) the staging
// area of two tiles of element size esz.  At TW = 64: 50 KB without it,
// 55 KB with 1- or 2-byte tiles -- four CTAs per SM.
template <int TW>
constexpr size_t raw_off() {
    return (sizeof(Smem<TW>) + 127) / 128 * 128;
}
template <int TW>
constexpr size_t smem_bulk(size_t esz) {
    return raw_off<TW>() + 2 * CH * Geom<TW>::TMA_COLS * esz;
}
template <int TW>
__device__ __forceinline__ unsigned char *raw_tile(Smem<TW> &S, int img, int esz) {
    return reinterpret_cast<unsigned char *>(&S) + raw_off<TW>() + img * (CH * Geom<TW>::TMA_COLS * esz);
}
// Resident CTAs per SM the kernels are compiled for (the register budget;
// 1024 threads an SM at 64 registers a thread): 1024 / NT for 1- and 2-byte
// data, whose shared memory allows it; 768 / NT for fp32 data, for the
// coefficient-writing (backward) variants and for the persistent variant
// that prefetches every chunk through registers (LEAN false), which would
// spill at 64.
template <typename T, bool COEF, bool LEAN = true, int TW = 64>
constexpr int min_ctas() {
    return (sizeof(T) <= 2 && !COEF && LEAN) ? 1024 / Geom<TW>::NT
                                             : (768 / Geom<TW>::NT > 0 ? 768 / Geom<TW>::NT : 1);
}
// The persistent bulk-copy variant of uint8 data also copies uint16 pyramid
// tiles: its staging area is sized for 2-byte elements.
template <typename T, int TW = kUniformTW>
constexpr size_t persistent_smem() {
    return smem_bulk<TW>(sizeof(T) < 2 ? 2 : sizeof(T));
}

__device__ __forceinline__ unsigned dynamic_smem_bytes() {
    unsigned n;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(n));
    return n;
}

// The 11-tap windows (Gaussian, box) are symmetric, g[n] = g[10 - n] (the
// launchers check it): the passes name taps 0..5 only, which keeps six tap
// pairs live in registers instead of eleven.
__host__ __device__ constexpr int sym(int n) { return n <= HALO / 2 ? n : HALO - n; }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

struct Geo {
    const void *xb, *yb;
    int64_t H, W, rs, OH, OW;
    int64_t j0;        // first output / input column of the strip
    int64_t o0, oend;  // output rows [o0, oend)
    int64_t own_r1;    // owned input rows [o0, own_r1) (downsample)
    int64_t own_c1;    // owned input columns [j0, own_c1)
    bool vec;          // rows and strip start aligned for 4-element vector loads
    bool ds16;         // next level as exact uint16 block sums (else fp32 2x2 means)
    int64_t ds_ld;     // row pitch of the next level's planes, in elements
};

// byte k of w placed in the mantissa of 2^23, minus 2^23: exact for 0..255
__device__ __forceinline__ float u8f(unsigned w, int k) {
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7540u + k)) - 8388608.0f;
}

// Raw (unconverted) load of four consecutive elements.  `packed`: one
// vector load, element bits as in memory; otherwise component k holds
// element k's bits (only the first `ncols` are read).  Keeping the data raw
// lets the register prefetch defer the conversion until after the barrier,
// so the load latency overlaps the vertical pass.
// LD = 0: read-only path (__ldg); LD = 1: L2-coherent loads (__ldcg), for
// data written by other CTAs earlier in the same launch.
template <int LD, typename U>
__device__ __forceinline__ U ld(const U *p) {
    if (LD) return __ldcg(p);
    return __ldg(p);
}

template <typename T, int LD = 0>
__device__ __forceinline__ uint4 load_raw(const T *p, int ncols, bool packed) {
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (packed) {
        if (sizeof(T) == 1) r.x = ld<LD>(reinterpret_cast<const unsigned *>(p));
        else if (sizeof(T) == 2) {
            const uint2 v = ld<LD>(reinterpret_cast<const uint2 *>(p));
            r.x = v.x;
            r.y = v.y;
        } else r = ld<LD>(reinterpret_cast<const uint4 *>(p));
        return r;
    }
    unsigned v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < ncols) {
            if (sizeof(T) == 1) v[k] = ld<LD>(reinterpret_cast<const unsigned char *>(p) + k);
            else if (sizeof(T) == 2) v[k] = ld<LD>(reinterpret_cast<const unsigned short *>(p) + k);
            else v[k] = ld<LD>(reinterpret_cast<const unsigned *>(p) + k);
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
// uint16: the exact integer pyramid levels (4^j times the level's values)
template <>
__device__ __forceinline__ float elem_f32<uint16_t>(unsigned b) {
    return __int_as_float(0x4B000000u | (b & 0xffffu)) - 8388608.0f;
}

template <typename T>
__device__ __forceinline__ float4 convert_raw(uint4 r, bool packed) {
    if (!packed || sizeof(T) == 4)
        return make_float4(elem_f32<T>(r.x), elem_f32<T>(r.y), elem_f32<T>(r.z), elem_f32<T>(r.w));
    if (sizeof(T) == 1) return make_float4(u8f(r.x, 0), u8f(r.x, 1), u8f(r.x, 2), u8f(r.x, 3));
    return make_float4(elem_f32<T>(r.x & 0xffffu), elem_f32<T>(r.x >> 16), elem_f32<T>(r.y & 0xffffu),
                       elem_f32<T>(r.y >> 16));
}

// (u, w) = (x + y, x - y).  For uint8 data both come straight from the
// magic floats 2^23 + x and 2^23 + y: (xm - 2^24) + ym = x + y and
// xm - ym = x - y, every step exact.
__device__ __forceinline__ float2 uw_of(float x, float y) { return make_float2(x + y, x - y); }
__device__ __forceinline__ float2 uw_of_magic(float xm, float ym) {
    return make_float2((xm - 16777216.0f) + ym, xm - ym);
}

// byte k of w as the float 2^23 + byte (exact)
__device__ __forceinline__ float u8m(unsigned w, int k) {
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7540u + k));
}

// Convert a raw unit of x and y (four columns each) into four (u, w) pairs.
template <typename T>
__device__ __forceinline__ void convert_uw(uint4 rx, uint4 ry, bool packed, float2 (&o)[4]) {
    if (sizeof(T) == 1) {
        if (packed) {
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = uw_of_magic(u8m(rx.x, k), u8m(ry.x, k));
        } else {
            o[0] = uw_of_magic(u8m(rx.x, 0), u8m(ry.x, 0));
            o[1] = uw_of_magic(u8m(rx.y, 0), u8m(ry.y, 0));
            o[2] = uw_of_magic(u8m(rx.z, 0), u8m(ry.z, 0));
            o[3] = uw_of_magic(u8m(rx.w, 0), u8m(ry.w, 0));
        }
        return;
    }
    const float4 a = convert_raw<T>(rx, packed), b = convert_raw<T>(ry, packed);
    o[0] = uw_of(a.x, b.x);
    o[1] = uw_of(a.y, b.y);
    o[2] = uw_of(a.z, b.z);
    o[3] = uw_of(a.w, b.w);
}

// Integer data (uint8, or the uint16 pyramid levels) is staged as BIASED
// magic floats formed in integer lanes, with no FP32 work: u' = 2^23 + u and
// w' = 2^23 + B + w, B the largest |w| (255 or 65535).  Both lie in
// [2^23, 2^24), where fp32 holds every integer, and the horizontal pass only
// ever forms differences of staged values (exact) and adds the bias back
// once per group of four outputs.
template <typename T>
constexpr bool kBiasedStaging = std::is_same<T, uint8_t>::value || std::is_same<T, uint16_t>::value;
template <typename T>
__device__ __forceinline__ float2 staging_bias() {
    return make_float2(8388608.0f, sizeof(T) == 1 ? 8388863.0f : 8454143.0f);  // 2^23, 2^23 + 255 / 65535
}
__device__ __forceinline__ float magic(unsigned v) { return __int_as_float(0x4B000000u | v); }

// Store one staged unit: columns 4q..4q+3 as (u, w) pairs.
template <typename T, int TW>
__device__ __forceinline__ void put_unit(Smem<TW> &S, int r, int q, uint4 rx, uint4 ry, bool packed) {
    float4 *d = reinterpret_cast<float4 *>(&S.in[r][4 * q]);
    if constexpr (kBiasedStaging<T>) {
        unsigned u[4], w[4];
        if (sizeof(T) == 1 && packed) {
            // even and odd bytes in two 16-bit lanes each: u <= 510 and
            // w + 255 in [0, 510], so no carry or borrow crosses a lane
            const unsigned xe = rx.x & 0x00ff00ffu, xo = (rx.x >> 8) & 0x00ff00ffu;
            const unsigned ye = ry.x & 0x00ff00ffu, yo = (ry.x >> 8) & 0x00ff00ffu;
            const unsigned ue = xe + ye, uo = xo + yo;
            const unsigned we = xe + 0x00ff00ffu - ye, wo = xo + 0x00ff00ffu - yo;
            d[0] = make_float4(__int_as_float(__byte_perm(ue, 0x4B000000u, 0x7510u)),
                               __int_as_float(__byte_perm(we, 0x4B000000u, 0x7510u)),
                               __int_as_float(__byte_perm(uo, 0x4B000000u, 0x7510u)),
                               __int_as_float(__byte_perm(wo, 0x4B000000u, 0x7510u)));
            d[1] = make_float4(__int_as_float(__byte_perm(ue, 0x4B000000u, 0x7532u)),
                               __int_as_float(__byte_perm(we, 0x4B000000u, 0x7532u)),
                               __int_as_float(__byte_perm(uo, 0x4B000000u, 0x7532u)),
                               __int_as_float(__byte_perm(wo, 0x4B000000u, 0x7532u)));
            return;
        }
        unsigned xv[4], yv[4];
        if (sizeof(T) == 2 && packed) {
            xv[0] = rx.x & 0xffffu, xv[1] = rx.x >> 16, xv[2] = rx.y & 0xffffu, xv[3] = rx.y >> 16;
            yv[0] = ry.x & 0xffffu, yv[1] = ry.x >> 16, yv[2] = ry.y & 0xffffu, yv[3] = ry.y >> 16;
        } else {  // one element per component
            xv[0] = rx.x, xv[1] = rx.y, xv[2] = rx.z, xv[3] = rx.w;
            yv[0] = ry.x, yv[1] = ry.y, yv[2] = ry.z, yv[3] = ry.w;
        }
        const unsigned B = sizeof(T) == 1 ? 255u : 65535u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            u[k] = xv[k] + yv[k];
            w[k] = xv[k] + B - yv[k];
        }
        d[0] = make_float4(magic(u[0]), magic(w[0]), magic(u[1]), magic(w[1]));
        d[1] = make_float4(magic(u[2]), magic(w[2]), magic(u[3]), magic(w[3]));
        return;
    }
    float2 o[4];
    convert_uw<T>(rx, ry, packed, o);
    d[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
    d[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
}

// Staging unit: one quad (4 columns) of two adjacent input rows.  Holding
// both rows lets the thread form the 2x2 averages of the next pyramid level
// straight from the raw x and y values before they become (u, w) pairs.
struct Unit {
    int64_t off;  // element offset of the quad in row 2p of the staged block (from the image start)
    int p, q;     // row pair (-1: no unit), quad
    int ncols;    // columns inside the image (0..4)
    bool packed;
};

template <int TW>
__device__ __forceinline__ void make_unit(Unit &U, const Geo &g, int t, int npairs) {
    constexpr int QUADS = Geom<TW>::QUADS;
    U.p = -1;
    U.q = 0;
    U.ncols = 0;
    U.packed = false;
    U.off = 0;
    if (t < npairs * QUADS) {
        const int p = t / QUADS, q = t - p * QUADS;
        const int64_t c = g.j0 + 4 * q;
        U.p = p;
        U.q = q;
        U.ncols = (int)max((int64_t)0, min((int64_t)4, g.W - c));
        U.packed = g.vec && U.ncols == 4;
        U.off = 2 * p * g.rs + c;
    }
}

struct Raw {
    uint4 x0, y0, x1, y1;  // rows 2p and 2p + 1
};

// Raw loads of a unit of the block whose first row is r0 (rows at or past H read as 0).
template <typename T, int LD = 0>
__device__ __forceinline__ void load_unit(Raw &R, const Unit &U, const Geo &g, int64_t r0) {
    R.x0 = R.y0 = R.x1 = R.y1 = make_uint4(0u, 0u, 0u, 0u);
    if (U.p < 0 || U.ncols <= 0) return;
    const int64_t row = r0 + 2 * U.p, o = r0 * g.rs + U.off;
    const T *xp = static_cast<const T *>(g.xb) + o;
    const T *yp = static_cast<const T *>(g.yb) + o;
    if (row < g.H) {
        R.x0 = load_raw<T, LD>(xp, U.ncols, U.packed);
        R.y0 = load_raw<T, LD>(yp, U.ncols, U.packed);
    }
    if (row + 1 < g.H) {
        R.x1 = load_raw<T, LD>(xp + g.rs, U.ncols, U.packed);
        R.y1 = load_raw<T, LD>(yp + g.rs, U.ncols, U.packed);
    }
}

// A unit read from the bulk-copied rows in shared memory (packed layout as
// load_raw's vector form; rows past H and columns past W hold zeros).
template <typename T, int TW>
__device__ __forceinline__ void load_unit_smem(Raw &R, const Unit &U, Smem<TW> &S) {
    R.x0 = R.y0 = R.x1 = R.y1 = make_uint4(0u, 0u, 0u, 0u);
    if (U.p < 0) return;
    constexpr int pitch = Geom<TW>::TMA_COLS * (int)sizeof(T);
    const int off = 2 * U.p * pitch + 4 * U.q * (int)sizeof(T);
    const unsigned char *bx = raw_tile(S, 0, sizeof(T)) + off, *by = raw_tile(S, 1, sizeof(T)) + off;
    if (sizeof(T) == 1) {
        R.x0.x = *reinterpret_cast<const unsigned *>(bx);
        R.y0.x = *reinterpret_cast<const unsigned *>(by);
        R.x1.x = *reinterpret_cast<const unsigned *>(bx + pitch);
        R.y1.x = *reinterpret_cast<const unsigned *>(by + pitch);
    } else if (sizeof(T) == 2) {
        const uint2 a = *reinterpret_cast<const uint2 *>(bx), b = *reinterpret_cast<const uint2 *>(by);
        const uint2 c = *reinterpret_cast<const uint2 *>(bx + pitch), d = *reinterpret_cast<const uint2 *>(by + pitch);
        R.x0 = make_uint4(a.x, a.y, 0u, 0u);
        R.y0 = make_uint4(b.x, b.y, 0u, 0u);
        R.x1 = make_uint4(c.x, c.y, 0u, 0u);
        R.y1 = make_uint4(d.x, d.y, 0u, 0u);
    } else {
        R.x0 = *reinterpret_cast<const uint4 *>(bx);
        R.y0 = *reinterpret_cast<const uint4 *>(by);
        R.x1 = *reinterpret_cast<const uint4 *>(bx + pitch);
        R.y1 = *reinterpret_cast<const uint4 *>(by + pitch);
    }
}

// Sums of the two 2x2 blocks of a unit (columns 0-1 and 2-3 of rows a, b),
// packed as [block 0 | block 1 << 16]: exact integers.  uint8 rows: each
// block sum is at most 4 x 255; uint16 rows (a pyramid level j holding 4^j
// times its values, at most 255 x 4^j): at most 255 x 4^(j+1), which stays
// below 2^16 up to level 4.  Packed uint8 rows hold bytes 0-3 in one word
// (even and odd bytes are added in two 16-bit lanes, no carry can cross);
// packed uint16 rows hold halves 0-1 and 2-3 in two words; unpacked rows hold
// one element per component.
template <typename T>
__device__ __forceinline__ unsigned block_pair(uint4 a, uint4 b, bool packed) {
    if (packed) {
        if (sizeof(T) == 1)
            return (a.x & 0x00ff00ffu) + ((a.x >> 8) & 0x00ff00ffu) + (b.x & 0x00ff00ffu) + ((b.x >> 8) & 0x00ff00ffu);
        const unsigned s0 = (a.x & 0xffffu) + (a.x >> 16) + (b.x & 0xffffu) + (b.x >> 16);
        const unsigned s1 = (a.y & 0xffffu) + (a.y >> 16) + (b.y & 0xffffu) + (b.y >> 16);
        return s0 | (s1 << 16);
    }
    return (a.x + a.y + b.x + b.y) | ((a.z + a.w + b.z + b.w) << 16);
}

// The next pyramid level from the owned blocks of a unit (absolute rows
// r0 + 2p, +1): fp32 2x2 means, or (g.ds16, uint8 / uint16 data) exact
// uint16 block sums, i.e. 4 x the means in the units of this level.
template <typename T>
__device__ __forceinline__ void downsample_unit(const Raw &R, const Unit &U, const Geo &g, int64_t r0, void *dsx,
                                                void *dsy) {
    const int64_t r = r0 + 2 * U.p;  // even: segment and chunk starts are even
    const int64_t Hh = g.H >> 1, Wh = g.W >> 1, Rr = r >> 1;
    if (r >= g.own_r1 || Rr >= Hh) return;
    const int64_t c = g.j0 + 4 * U.q;
    const bool b0 = c < g.own_c1 && (c >> 1) < Wh;
    const bool b1 = c + 2 < g.own_c1 && ((c + 2) >> 1) < Wh;  // implies b0
    const int64_t o = Rr * g.ds_ld + (c >> 1);
    if constexpr (std::is_same<T, uint8_t>::value || std::is_same<T, uint16_t>::value) {
        if (g.ds16) {
            const unsigned sx = block_pair<T>(R.x0, R.x1, U.packed), sy = block_pair<T>(R.y0, R.y1, U.packed);
            uint16_t *px = static_cast<uint16_t *>(dsx) + o, *py = static_cast<uint16_t *>(dsy) + o;
            if (b1) {  // c >> 1 is even and the pitch a multiple of 8: a 4-byte aligned pair
                *reinterpret_cast<unsigned *>(px) = sx;
                *reinterpret_cast<unsigned *>(py) = sy;
            } else if (b0) {
                *px = (uint16_t)(sx & 0xffffu);
                *py = (uint16_t)(sy & 0xffffu);
            }
            return;
        }
    }
    const float4 x0 = convert_raw<T>(R.x0, U.packed), x1 = convert_raw<T>(R.x1, U.packed);
    const float4 y0 = convert_raw<T>(R.y0, U.packed), y1 = convert_raw<T>(R.y1, U.packed);
    float *fx = static_cast<float *>(dsx) + o, *fy = static_cast<float *>(dsy) + o;
    if (b0) {
        fx[0] = 0.25f * ((x0.x + x0.y) + (x1.x + x1.y));
        fy[0] = 0.25f * ((y0.x + y0.y) + (y1.x + y1.y));
    }
    if (b1) {
        fx[1] = 0.25f * ((x0.z + x0.w) + (x1.z + x1.w));
        fy[1] = 0.25f * ((y0.z + y0.w) + (y1.z + y1.w));
    }
}

// Store a unit into staged rows row0 + 2p, row0 + 2p + 1 (and its pyramid blocks).
template <typename T, int TW>
__device__ __forceinline__ void store_unit(Smem<TW> &S, const Raw &R, const Unit &U, const Geo &g, int64_t r0, int row0,
                                           void *dsx, void *dsy) {
    if (U.p < 0) return;
    if (dsx) downsample_unit<T>(R, U, g, r0, dsx, dsy);
    put_unit<T>(S, row0 + 2 * U.p, U.q, R.x0, R.y0, U.packed);
    put_unit<T>(S, row0 + 2 * U.p + 1, U.q, R.x1, R.y1, U.packed);
}

// Stage `nr` (even) input rows starting at absolute row r0 into in rows
// 0..nr-1 (once per segment, for the first FIRST rows).
template <typename T, int LD, int TW>
__device__ __forceinline__ void stage_direct(Smem<TW> &S, const Geo &g, int64_t r0, int nr, void *dsx, void *dsy) {
    for (int t = threadIdx.x; t < (nr >> 1) * Geom<TW>::QUADS; t += Geom<TW>::NT) {
        Unit U;
        make_unit<TW>(U, g, t, nr >> 1);
        Raw R;
        load_unit<T, LD>(R, U, g, r0);
        store_unit<T>(S, R, U, g, r0, 0, dsx, dsy);
    }
}

// Horizontal pass over staged rows 0..NR-1 (NR even); results go to ring
// rows (rel0 + r) & (RING-1), where rel0 is the row index relative to the
// segment.  Tasks come in quarter-warps of 8: quarter-warp Q takes row pair
// Q / (TW / 16) and, within it, 4 consecutive groups of 4 outputs (group
// quad Q % (TW / 16)): lanes 0-3 of the first row, lanes 4-7 of the second.
// At TW = 64 warp w takes rows 2w and 2w + 1.
template <int NR, int TW>
__device__ __forceinline__ void horizontal(Smem<TW> &S, int rel0, const Taps2<K> &t2, float2 bias) {
    static_assert(NR % 2 == 0, "rows come in pairs");
    constexpr int NT = Geom<TW>::NT, TASKS = NR * (TW / 4), QPR = TW / 16;
#pragma unroll 1
    for (int pass = 0; pass < (TASKS + NT - 1) / NT; ++pass) {
        const int task = threadIdx.x + pass * NT;
        if (TASKS % NT != 0 && task >= TASKS) break;
        const int Q = task >> 3, l = task & 7;
        const int r = 2 * (Q / QPR) + ((l >> 2) & 1);
        const int g4 = 4 * (4 * (Q % QPR) + (l & 3));
        float2 p[14];
        const float4 *src = reinterpret_cast<const float4 *>(&S.in[r][g4]);
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const float4 v = src[k];
            p[2 * k] = make_float2(v.x, v.y);
            p[2 * k + 1] = make_float2(v.z, v.w);
        }
        // shift: pixel 7 lies in the windows of outputs 0..3 (centres 5..8)
        const float2 nc = make_float2(-p[7].x, -p[7].y);
        float2 m[4], sq[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) m[o] = sq[o] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 14; ++i) {
            const float2 d = add2(p[i], nc);  // (du, dw)
            const float2 dd = mul2(d, d);     // (du^2, dw^2)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int n = i - o;
                if (n >= 0 && n < K) {
                    m[o] = fma2(t2.g2[sym(n)], d, m[o]);
                    sq[o] = fma2(t2.g2[sym(n)], dd, sq[o]);
                }
            }
        }
        const int slot = (rel0 + r) & (RING - 1);
        const float2 cc = add2(p[7], make_float2(-bias.x, -bias.y));  // the shift, unbiased (exact)
        float2 om[4], ov[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            om[o] = add2(m[o], cc);
            ov[o] = fma2(make_float2(-m[o].x, -m[o].y), m[o], sq[o]);
        }
        const float4 m01 = make_float4(om[0].x, om[0].y, om[1].x, om[1].y);
        const float4 m23 = make_float4(om[2].x, om[2].y, om[3].x, om[3].y);
        const float4 v01 = make_float4(ov[0].x, ov[0].y, ov[1].x, ov[1].y);
        const float4 v23 = make_float4(ov[2].x, ov[2].y, ov[3].x, ov[3].y);
        float4 *dm = reinterpret_cast<float4 *>(&S.mu[slot][g4]);
        float4 *dv = reinterpret_cast<float4 *>(&S.v[slot][g4]);
        dm[0] = m01;
        dm[1] = m23;
        dv[0] = v01;
        dv[1] = v23;
    }
}

// Vertical window sums of 4 output rows of one column over ring rows
// b0..b0+13 (mod RING), b0 a multiple of 4: the window is read as four
// blocks of 4 rows, each contiguous in the ring, so only the block starts
// wrap; b: the shift (the window-centre row's mean, ring row b0 + 7).
template <int TW>
__device__ __forceinline__ void column_sums(const Smem<TW> &S, int b0, int col, const Taps2<K> &t2, float2 &b,
                                            float2 (&m)[4], float2 (&sq)[4]) {
    const float2 *blk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) blk[q] = &S.mu[(b0 + 4 * q) & (RING - 1)][col];
    constexpr int RWP = Geom<TW>::RWP, VOFF = RING * RWP;  // S.v follows S.mu (asserted at Smem)
    b = blk[1][3 * RWP];
    const float2 nb = make_float2(-b.x, -b.y);
#pragma unroll
    for (int o = 0; o < 4; ++o) m[o] = sq[o] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 14; ++i) {
        const float2 *p = blk[i >> 2] + (i & 3) * RWP;
        const float2 e = add2(p[0], nb);     // (eu, ew)
        const float2 q = fma2(e, e, p[VOFF]);  // (eu^2 + v_u, ew^2 + v_w)
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int n = i - o;
            if (n >= 0 && n < K) {
                m[o] = fma2(t2.g2[sym(n)], e, m[o]);
                sq[o] = fma2(t2.g2[sym(n)], q, sq[o]);
            }
        }
    }
}

// Vertical pass + SSIM formula for the 16 output rows starting at rel0
// (relative to the segment); each thread does 4 rows of one column.
// cs_only (no map, no coefficients): the level's Q is not pooled (MS-SSIM
// levels below the last), so only the contrast-structure term is formed and
// sumQ is 0.
template <bool COEF, int TW>
__device__ __forceinline__ void vertical(const Smem<TW> &S, const Geo &g, int rel0, const Taps<K> &t,
                                         const Taps2<K> &t2, const SsimConst &cc, float *map, int64_t map_ld, bool col_ok,
                                         const CoefOut &co, float *coef_img, bool cs_only, float &sumQ, float &sumCS) {
    const int col = threadIdx.x & (TW - 1);
    const int base = rel0 + 4 * (threadIdx.x / TW);
    const int b0 = base & (RING - 1);  // multiple of 4, uniform over the warp
    float2 b, m[4], sq[4];
    column_sums(S, b0, col, t2, b, m, sq);
    const int rows_left = col_ok ? (int)(g.oend - g.o0) - base : 0;
    sumQ = 0.f;
    sumCS = 0.f;
    if (!COEF && cs_only) {
        float css[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const float2 var = fma2(make_float2(-m[o].x, -m[o].y), m[o], sq[o]);  // (Var u, Var w)
            const float t2c = var.x + cc.C2x2;
            css[o] = __fdividef(t2c - var.y, t2c + var.y);
        }
        if (rows_left >= 4) {
            sumCS = (css[0] + css[1]) + (css[2] + css[3]);
        } else {
#pragma unroll
            for (int o = 0; o < 4; ++o)
                if (o < rows_left) sumCS += css[o];
        }
        return;
    }
    float *mrow = map ? map + (g.o0 + base) * map_ld + g.j0 + col : nullptr;
    float qs[4], css[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const float2 u = add2(m[o], b);                                        // (mu_u, mu_w)
        const float2 var = fma2(make_float2(-m[o].x, -m[o].y), m[o], sq[o]);  // (Var u, Var w)
        // 2 A1, 2 B1, 2 A2, 2 B2 of the (x, y) form
        const float A1 = fmaf(u.x, u.x, fmaf(-u.y, u.y, cc.C1x2)), B1 = fmaf(u.x, u.x, fmaf(u.y, u.y, cc.C1x2));
        const float t2c = var.x + cc.C2x2;
        const float A2 = t2c - var.y, B2 = t2c + var.y;
        const float l = __fdividef(A1, B1), cs = __fdividef(A2, B2);
        qs[o] = l * cs;
        css[o] = cs;
        if (COEF && o < rows_left) {
            float ca, cb, ccf;
            ssim_coef(0.5f * (u.x + u.y), 0.5f * (u.x - u.y), 0.5f * A1, 0.5f * B1, 0.5f * A2, 0.5f * B2, co.which,
                      co.sx, co.sy, ca, cb, ccf);
            const int64_t ld = coef_ld(g.OW), plane = g.OH * ld;
            float *dst = coef_img + (g.o0 + base + o) * ld + g.j0 + col;
            dst[0] = ca;
            dst[plane] = cb;
            dst[2 * plane] = ccf;
        }
    }
    if (rows_left >= 4) {  // the common case: all four outputs exist
        sumQ = (qs[0] + qs[1]) + (qs[2] + qs[3]);
        sumCS = (css[0] + css[1]) + (css[2] + css[3]);
    } else {
#pragma unroll
        for (int o = 0; o < 4; ++o)
            if (o < rows_left) {
                sumQ += qs[o];
                sumCS += css[o];
            }
    }
    if (mrow) {
#pragma unroll
        for (int o = 0; o < 4; ++o)
            if (o < rows_left) mrow[o * map_ld] = qs[o];
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
template <int NT>
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

// One work item: a strip of TW output columns x a segment of output rows of
// one image.  Used by the grid kernel (one item per CTA) and by the
// persistent ragged-batch kernel (items pulled from a queue).
struct Item {
    const void *xb, *yb;   // image (or pyramid level) base pointers
    int64_t H, W, rs;
    int strip, seg, strips, segs, seg_rows;
    bool vec;
    float *map;            // image map base (nullable)
    int64_t map_ld;
    void *dsx, *dsy;       // next-level planes of this image (nullable): fp32, or uint16 when ds16
    bool ds16;             // uint8 / uint16 data: the next level as exact uint16 block sums
    int64_t ds_ld;         // row pitch of the next-level planes, in elements
    float cscale;          // C1, C2 scale (16^j for a uint16 level holding 4^j times its values; else 1)
    bool cs_only;          // only the mean cs of the item is pooled (its sum Q slot reads 0)
    float *coef_img;       // COEF mode: A, B, C planes of this image
    double2 *partial;      // this item's (sum Q, sum cs) slot
    const CUtensorMap *tmx, *tmy;  // nullable: bulk-copy maps of the (level-0) x, y planes
    int tz;                        // this image's index in them
};

// BULK: the chunks after the first arrive by bulk tensor copies (it.tmx,
// it.tmy); `phase`: parity of the bulk-copy mbarrier's next phase (the CTA's
// running count of bulk-copied chunks); `tma_ok`: cleared for the rest of
// the CTA's items when a bulk-copy wait gives up (that item's partial then
// reads NaN).
template <typename T, bool COEF, int LD, bool BULK, int TW>
__device__ __forceinline__ void gauss11_item(Smem<TW> &S, const Item &it, const Taps<K> &taps, const Taps2<K> &taps2,
                                             const SsimConst &cc0, const CoefOut &co, unsigned &phase, bool &tma_ok) {
    Geo g;
    g.H = it.H;
    g.W = it.W;
    g.rs = it.rs;
    g.OH = g.H - HALO;
    g.OW = g.W - HALO;
    g.xb = it.xb;
    g.yb = it.yb;
    g.j0 = (int64_t)it.strip * TW;
    g.o0 = (int64_t)it.seg * it.seg_rows;
    g.oend = min(g.o0 + (int64_t)it.seg_rows, g.OH);
    g.own_r1 = (it.seg == it.segs - 1) ? g.H : g.o0 + it.seg_rows;
    g.own_c1 = (it.strip == it.strips - 1) ? g.W : g.j0 + TW;
    g.vec = it.vec;
    g.ds16 = it.ds16;
    g.ds_ld = it.ds_ld;
    const int nchunks = (int)((g.oend - g.o0 + CH - 1) / CH);
    // SSIM is unchanged when x, y scale by a and C1, C2 by a^2; with a a
    // power of two every fp32 step scales exactly, so a uint16 level holding
    // 4^j times its values gives the bits of the unscaled level
    SsimConst cc = cc0;
    if (it.cscale != 1.f) {
        cc.C1 *= it.cscale;
        cc.C2 *= it.cscale;
        cc.C1x2 *= it.cscale;
        cc.C2x2 *= it.cscale;
    }

    KSum accQ, accCS;
    Raw raw;
    Unit U;
    make_unit<TW>(U, g, threadIdx.x, CH / 2);
    const bool col_ok = g.j0 + (threadIdx.x & (TW - 1)) < g.OW;

    if (BULK && !tma_ok) {  // an earlier bulk-copy wait of this CTA gave up
        if (threadIdx.x == 0) *it.partial = make_double2(nan(""), nan(""));
        return;
    }
    Unit Ut = U;
    Ut.packed = true;  // bulk-copied units are complete (zeros past the image)

    stage_direct<T, LD>(S, g, g.o0, FIRST, it.dsx, it.dsy);
    __syncthreads();
    const float2 bias = kBiasedStaging<T> ? staging_bias<T>() : make_float2(0.f, 0.f);
    horizontal<FIRST>(S, 0, taps2, bias);
    if constexpr (!BULK) {
        for (int c = 0; c < nchunks; ++c) {
            const bool more = c + 1 < nchunks;
            const int64_t next_r0 = g.o0 + FIRST + (int64_t)CH * c;
            if (more) load_unit<T, LD>(raw, U, g, next_r0);
            __syncthreads();  // ring rows of chunk c complete; staging free
            float cq, ccs;
            vertical<COEF>(S, g, CH * c, taps, taps2, cc, it.map, it.map_ld, col_ok, co, it.coef_img, it.cs_only, cq,
                           ccs);
            accQ.add(cq);
            accCS.add(ccs);
            if (more) store_unit<T>(S, raw, U, g, next_r0, 0, it.dsx, it.dsy);
            __syncthreads();  // staging complete; ring rows of chunk c consumed
            if (more) horizontal<CH>(S, FIRST + CH * c, taps2, bias);
        }
    } else {
        for (int c = 0; c < nchunks; ++c) {
            const bool more = c + 1 < nchunks;
            const int64_t next_r0 = g.o0 + FIRST + (int64_t)CH * c;
            // raw[] was last read before the previous barrier
            if (more && threadIdx.x == 0) {
                fence_proxy_async_smem();
                mbar_expect_tx(&S.bar, 2u * CH * Geom<TW>::TMA_COLS * (unsigned)sizeof(T));
                tma_load_3d(raw_tile(S, 0, sizeof(T)), it.tmx, (int)g.j0, (int)next_r0, it.tz, &S.bar);
                tma_load_3d(raw_tile(S, 1, sizeof(T)), it.tmy, (int)g.j0, (int)next_r0, it.tz, &S.bar);
            }
            __syncthreads();  // ring rows of chunk c complete; staging free
            float cq, ccs;
            vertical<COEF>(S, g, CH * c, taps, taps2, cc, it.map, it.map_ld, col_ok, co, it.coef_img, it.cs_only, cq,
                           ccs);
            accQ.add(cq);
            accCS.add(ccs);
            bool failed = false;
            if (more) {
                const unsigned ph = phase;
                phase ^= 1u;
                if (mbar_wait_bounded(&S.bar, ph)) {
                    load_unit_smem<T>(raw, U, S);
                    store_unit<T>(S, raw, Ut, g, next_r0, 0, it.dsx, it.dsy);
                } else {
                    failed = true;
                }
            }
            // staging complete; ring rows of chunk c consumed
            if (__syncthreads_or(failed)) {
                if (threadIdx.x == 0) mbar_wait_bounded(&S.bar, phase ^ 1u);  // drain (bounded)
                tma_ok = false;
                if (threadIdx.x == 0) *it.partial = make_double2(nan(""), nan(""));  // the score reads NaN
                __syncthreads();
                return;
            }
            if (more) horizontal<CH>(S, FIRST + CH * c, taps2, bias);
        }
    }
    double a, b;
    block_sum2f<Geom<TW>::NT>(accQ.s - accQ.c, accCS.s - accCS.c, S.red, a, b);
    if (threadIdx.x == 0) *it.partial = make_double2(a, b);
}

template <typename T, bool COEF>
__global__ void __launch_bounds__(Geom<64>::NT, (min_ctas<T, COEF>()))
    gauss11_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy, bool use_tma,
                   const GaussLaunch L, int strips, int segs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<64> &S = *reinterpret_cast<Smem<64> *>(smem_raw);
    if (use_tma && threadIdx.x == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
    }
    const int strip = blockIdx.x, seg = blockIdx.y, img = blockIdx.z;
    Item it;
    it.H = L.x.H;
    it.W = L.x.W;
    it.rs = L.x.row_stride;
    it.xb = static_cast<const T *>(L.x.data) + img * L.x.image_stride;
    it.yb = static_cast<const T *>(L.y.data) + img * L.y.image_stride;
    it.strip = strip;
    it.seg = seg;
    it.strips = strips;
    it.segs = segs;
    it.seg_rows = L.seg_rows;
    it.vec = L.vec;
    it.map = L.map ? L.map + img * L.map_is : nullptr;
    it.map_ld = L.map_ld;
    const int64_t dsn = (it.H >> 1) * (it.W >> 1);
    it.dsx = L.ds_x ? L.ds_x + img * dsn : nullptr;
    it.dsy = L.ds_y ? L.ds_y + img * dsn : nullptr;
    it.ds16 = false;
    it.ds_ld = it.W >> 1;
    it.cscale = 1.f;
    it.cs_only = false;
    it.coef_img = COEF ? L.co.coef + (int64_t)img * 3 * (it.H - HALO) * coef_ld(it.W - HALO) : nullptr;
    it.partial = L.partials + ((int64_t)img * segs + seg) * strips + strip;
    it.tmx = use_tma ? &tmx : nullptr;
    it.tmy = use_tma ? &tmy : nullptr;
    it.tz = img;
    unsigned phase = 0;
    bool tma_ok = true;
    // the item's first barrier orders the mbarrier initialisation before any use
    if (use_tma) gauss11_item<T, COEF, 0, true>(S, it, L.taps, L.taps2, L.c, L.co, phase, tma_ok);
    else gauss11_item<T, COEF, 0, false>(S, it, L.taps, L.taps2, L.c, L.co, phase, tma_ok);
}

// ----------------------------------------------------------------- ragged persistent batch
//
// One launch of (#SMs x CTAs-per-SM) CTAs for a whole ragged batch.  Work
// items (image, level, strip, segment) are listed level-major; each CTA takes
// the next item from an atomic counter.  A level-j item needs the 2x2 pyramid
// of its image written by all of its level-(j-1) items: after an item, thread
// 0 fences and bumps the (image, level) completion counter; before a level-j
// item it waits (bounded) until the counter of level j-1 reaches that level's
// item count.  Items are handed out in order, so every item waited on is held
// by a running CTA that waits only on earlier items: no deadlock.  If a wait
// exceeds its limit the kernel records GBSSIM_ERR_TIMEOUT in the status word
// and carries on (the scores are then meaningless but the launch ends).
// Pooling slots are fixed per item, so scores are deterministic whichever CTA
// ran which item.
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// What one work item needs, from either source below.
struct Resolved {
    Item it;          // all fields but xb / yb
    const void *xb, *yb;
    int img;          // image index (uniform batches; -1 in ragged ones)
    int level;        // pyramid level j
    bool pyramid;     // level >= 1: float planes written earlier in this launch
    int done_index;   // completion counter this item bumps
    int dep_index;    // counter it waits on (-1: none)
    unsigned dep_target;
    const unsigned *arrive;  // nullable: flag its input's arrival sets (non-zero)
};

// Ragged batches: per-(image, level) records and a per-item list built by
// the host plan (gbssim_batch_plan).
struct TableSource {
    BatchTable B;
    __device__ int total() const { return B.total_items; }
    __device__ bool ipyr() const { return false; }
    __device__ void resolve(int item, char *ws, Resolved &R) const {
        const BatchItem bi = B.items[item];
        const BatchLevel &lv = B.levels[bi.level_index];
        Item &it = R.it;
        it.H = lv.H;
        it.W = lv.W;
        it.rs = lv.rs;
        it.strip = bi.strip;
        it.seg = bi.seg;
        it.strips = lv.strips;
        it.segs = lv.segs;
        it.seg_rows = lv.seg_rows;
        it.vec = lv.vec != 0;
        it.map = nullptr;
        it.map_ld = 0;
        float *ds = lv.ds_off >= 0 ? reinterpret_cast<float *>(ws + lv.ds_off) : nullptr;
        it.dsx = ds;
        it.dsy = ds ? ds + (lv.H >> 1) * (lv.W >> 1) : nullptr;
        it.ds16 = false;
        it.ds_ld = lv.W >> 1;
        it.cscale = 1.f;
        it.cs_only = false;
        it.coef_img = nullptr;
        it.partial = reinterpret_cast<double2 *>(ws + lv.part_off) + (int64_t)bi.seg * lv.strips + bi.strip;
        R.pyramid = lv.level > 0;
        R.level = lv.level;
        R.img = -1;
        if (lv.level == 0) {
            R.xb = lv.x;
            R.yb = lv.y;
        } else {
            R.xb = ws + lv.x_off;
            R.yb = ws + lv.x_off + sizeof(float) * lv.H * lv.W;
        }
        R.arrive = nullptr;
        R.done_index = bi.level_index;
        R.dep_index = lv.level > 0 ? bi.level_index - 1 : -1;
        R.dep_target = lv.level > 0 ? (unsigned)B.levels[bi.level_index - 1].wait_target : 0u;
    }
};

// Batches of equally sized images (gbssim_msssim): the item list is
// arithmetic (level-major, then image, segment, strip; or, with arrival
// flags, the copy-group wavefront of UniformBatch::waves), so no table exists;
// the pyramid and pooling slots use gbssim_msssim's workspace layout.
struct UniformSource {
    UniformBatch U;
    __device__ int total() const { return (int)U.total_items; }
    __device__ bool ipyr() const { return U.ipyr != 0; }
    __device__ void resolve(int item, char *ws, Resolved &R) const {
        int j = 0, img, rem, grp = -1;
        if (U.waves > 0) {
            // wave w: level j of copy group w - j, levels in order; a level's
            // dependency (the level below, same group) is one wave earlier
            int w = 0;
            while (w + 1 < U.waves && item >= U.wave_begin[w + 1]) ++w;
            int r = item - U.wave_begin[w];
            j = w - U.groups + 1 > 0 ? w - U.groups + 1 : 0;
            int g = w - j, m;
            for (;; ++j, --g) {
                m = U.group_begin[g + 1] - U.group_begin[g];
                const int c = m * U.lv[j].items_per_image;
                if (r < c || j + 1 >= U.scales || g == 0) break;
                r -= c;
            }
            const int k = r / U.lv[j].items_per_image;
            img = U.group_begin[g] + k;
            grp = g;
            rem = r - k * U.lv[j].items_per_image;
        } else {
            while (j + 1 < U.scales && item >= U.lv[j + 1].item_begin) ++j;
            const int local = item - (int)U.lv[j].item_begin;
            img = local / U.lv[j].items_per_image;
            rem = local - img * U.lv[j].items_per_image;
        }
        const UniformLevel &lv = U.lv[j];
        const int seg = rem / lv.strips, strip = rem - seg * lv.strips;
        Item &it = R.it;
        it.H = lv.H;
        it.W = lv.W;
        it.rs = j == 0 ? U.rs : lv.pitch;
        it.strip = strip;
        it.seg = seg;
        it.strips = lv.strips;
        it.segs = lv.segs;
        it.seg_rows = lv.seg_rows;
        it.vec = lv.vec != 0;
        it.map = nullptr;
        it.map_ld = 0;
        // pyramid planes (levels >= 1): fp32, or uint16 holding 4^j times the
        // level's values (U.ipyr); each x plane of the level, then each y plane
        const int64_t esz_p = U.ipyr ? 2 : 4;
        const int64_t plane = lv.H * lv.pitch;
        it.ds16 = U.ipyr != 0;
        it.cscale = (U.ipyr && j > 0) ? __int_as_float((127 + 4 * j) << 23) : 1.f;  // 16^j
        it.cs_only = j < U.cs_only_levels;
        if (j + 1 < U.scales) {
            const UniformLevel &nv = U.lv[j + 1];
            const int64_t nplane = nv.H * nv.pitch;
            it.dsx = ws + nv.x_off + esz_p * img * nplane;
            it.dsy = ws + nv.x_off + esz_p * (U.count + img) * nplane;
            it.ds_ld = nv.pitch;
        } else {
            it.dsx = it.dsy = nullptr;
            it.ds_ld = 0;
        }
        it.coef_img = nullptr;
        it.partial = reinterpret_cast<double2 *>(ws + lv.part_off) + (int64_t)img * lv.items_per_image + rem;
        R.pyramid = j > 0;
        R.level = j;
        R.img = img;
        if (j == 0) {
            const size_t esz = U.dtype == GBSSIM_U8 ? 1 : U.dtype == GBSSIM_F32 ? 4 : 2;
            R.xb = static_cast<const char *>(U.x) + esz * img * U.image_stride;
            R.yb = static_cast<const char *>(U.y) + esz * img * U.image_stride;
        } else {
            R.xb = ws + lv.x_off + esz_p * img * plane;
            R.yb = ws + lv.x_off + esz_p * (U.count + img) * plane;
        }
        R.arrive = (j == 0 && U.arrive && grp >= 0) ? U.arrive + grp : nullptr;
        R.done_index = img * U.scales + j;
        R.dep_index = j > 0 ? img * U.scales + j - 1 : -1;
        R.dep_target = j > 0 ? (unsigned)U.lv[j - 1].items_per_image : 0u;
    }
};

// Bulk-copy maps of the uint16 pyramid levels 1..4 (x and y planes of all
// images of a level; the image index is the third coordinate).
constexpr int kPyrMaps = 4;
struct PyrMaps {
    CUtensorMap x[kPyrMaps], y[kPyrMaps];
};

// BULK: level-0 items (uniform batches) take their chunks by bulk tensor
// copies (tmx, tmy; the image index is the map's third coordinate).  Pyramid
// levels: with uint8 input and the uint16 pyramid (src.ipyr()), their
// uint16 planes too (pm, written earlier in this launch: the writers fence
// their generic stores against the async proxy before releasing the level's
// completion count, the reader fences after acquiring it); otherwise fp32
// planes by register staging.  After a bulk-copy wait gives up, the CTA's
// remaining bulk-copied items write NaN partials.  Without BULK the launch
// needs no staging area after the shared-memory struct.  TW: the strip width (64 for
// uniform batches; the ragged-batch table also runs at 32 and 128).
template <typename T, typename Src, bool BULK, int TW = 64>
__global__ void __launch_bounds__(Geom<TW>::NT, (min_ctas<T, false, BULK, TW>()))
    gauss11_persistent_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy,
                              const __grid_constant__ PyrMaps pm, const Src src, void *ws_ptr, int64_t counter_off,
                              int64_t done_off, int64_t status_off, unsigned wait_limit, Taps<K> taps, Taps2<K> taps2,
                              SsimConst cc) {
    constexpr bool kIpyr = BULK && std::is_same<T, uint8_t>::value && std::is_same<Src, UniformSource>::value;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<TW> &S = *reinterpret_cast<Smem<TW> *>(smem_raw);
    // a launch shaped for another strip width would index past its shared
    // memory: refuse it (status word, no score) before any access
    if (blockDim.x != (unsigned)Geom<TW>::NT || dynamic_smem_bytes() < (BULK ? persistent_smem<T, TW>() : raw_off<TW>())) {
        if (threadIdx.x == 0) atomicExch(reinterpret_cast<int *>(static_cast<char *>(ws_ptr) + status_off),
                                         (int)GBSSIM_ERR_INVALID_ARG);
        return;
    }
    if (BULK && threadIdx.x == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
    }
    unsigned phase = 0;
    bool tma_ok = true;
    __shared__ int s_item, s_late;
    char *ws = static_cast<char *>(ws_ptr);
    unsigned *counter = reinterpret_cast<unsigned *>(ws + counter_off);
    unsigned *done = reinterpret_cast<unsigned *>(ws + done_off);
    int *status = reinterpret_cast<int *>(ws + status_off);
    CoefOut co;
    co.coef = nullptr;
    co.which = 0;
    co.sx = co.sy = 0.f;
    const int total = src.total();
    for (;;) {
        if (threadIdx.x == 0) {
            const int i = (int)atomicAdd(counter, 1u);
            const int item = i < total ? i : -1;
            int late = 0;
            if (item >= 0) {
                Resolved R;
                src.resolve(item, ws, R);
                // Once any wait of the launch has given up (status set), the
                // others give up at their next check, so a stalled launch
                // ends after one wait limit, not one per item.
                const volatile int *st_word = status;
                if (R.dep_index >= 0) {
                    const unsigned *flag = done + R.dep_index;
                    unsigned spins = 0;
                    while (ld_acquire(flag) < R.dep_target) {
                        if (++spins > wait_limit || ((spins & 63u) == 0 && *st_word != 0)) {
                            atomicExch(status, (int)GBSSIM_ERR_TIMEOUT);
                            late = 1;
                            break;
                        }
                        __nanosleep(256);
                    }
                    // bulk copies below may read the level this wait acquired
                    if (kIpyr) fence_proxy_async_global();
                }
                if (R.arrive) {  // the image's bytes are still being copied in (bounded: 16x the level limit)
                    unsigned long long spins = 0;
                    while (ld_acquire(R.arrive) == 0u) {
                        if (++spins > 16ull * wait_limit || ((spins & 63u) == 0 && *st_word != 0)) {
                            atomicExch(status, (int)GBSSIM_ERR_TIMEOUT);
                            late = 1;
                            break;
                        }
                        __nanosleep(256);
                    }
                    if (BULK) fence_proxy_async_global();  // before this CTA's bulk copies of those bytes
                }
            }
            s_item = item;
            s_late = late;
        }
        __syncthreads();
        const int item = s_item;
        if (item < 0) break;
        Resolved R;
        src.resolve(item, ws, R);
        R.it.xb = R.xb;
        R.it.yb = R.yb;
        R.it.tmx = BULK ? &tmx : nullptr;
        R.it.tmy = BULK ? &tmy : nullptr;
        R.it.tz = R.img;
        if (R.pyramid) {
            if constexpr (kIpyr) {
                if (src.ipyr()) {
                    R.it.tmx = &pm.x[R.level - 1];
                    R.it.tmy = &pm.y[R.level - 1];
                    gauss11_item<uint16_t, false, 1, true>(S, R.it, taps, taps2, cc, co, phase, tma_ok);
                } else {
                    gauss11_item<float, false, 1, false>(S, R.it, taps, taps2, cc, co, phase, tma_ok);
                }
            } else {
                gauss11_item<float, false, 1, false>(S, R.it, taps, taps2, cc, co, phase, tma_ok);
            }
        } else {
            gauss11_item<T, false, BULK ? 1 : 0, BULK>(S, R.it, taps, taps2, cc, co, phase, tma_ok);
        }
        // the next level's planes are read by bulk copies of other CTAs
        if (kIpyr && R.it.dsx) fence_proxy_async_global();
        __syncthreads();  // every thread's partial and pyramid stores issued
        if (threadIdx.x == 0) {
            if (s_late) *R.it.partial = make_double2(nan(""), nan(""));  // the score reads NaN
            __threadfence();
            atomicAdd(done + R.done_index, 1u);
        }
    }
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
        if (L.co.coef) {
            float ca, cb, ccf;
            ssim_coef(ux, uy, A1, B1, A2, B2, L.co.which, L.co.sx, L.co.sy, ca, cb, ccf);
            const int64_t ld = coef_ld(OW), plane = OH * ld;
            float *dst = L.co.coef + (int64_t)img * 3 * plane + a * ld + b;
            dst[0] = ca;
            dst[plane] = cb;
            dst[2 * plane] = ccf;
        }
    }
    double sa = q, sb = cs;
    block_sum2(sa, sb, red);
    if (threadIdx.x == 0)
        L.partials[((int64_t)img * tiles_y + blockIdx.y) * tiles_x + blockIdx.x] = make_double2(sa, sb);
}

template <typename T>
constexpr CUtensorMapDataType tma_dtype() {
    return sizeof(T) == 1                      ? CU_TENSOR_MAP_DATA_TYPE_UINT8
           : sizeof(T) == 4                    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
           : std::is_same<T, uint16_t>::value ? CU_TENSOR_MAP_DATA_TYPE_UINT16
           : std::is_same<T, __half>::value   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

// Bulk-copy map of a batch of planes (columns, rows, image) with
// TMA_COLS x CH tiles of the TW-column strips; false when the planes are not
// 16-byte aligned (base and strides) or no encoder is available -- the
// register path runs then.
template <typename T, int TW>
bool encode_plane_map(CUtensorMap *m, const void *data, int64_t H, int64_t W, int64_t rs, int64_t is, int count) {
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    const int64_t esz = sizeof(T), istr = count > 1 ? is : H * rs;
    if ((uintptr_t)data % 16 != 0 || (rs * esz) % 16 != 0 || (istr * esz) % 16 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)count};
    const cuuint64_t strides[2] = {(cuuint64_t)(rs * esz), (cuuint64_t)(istr * esz)};
    const cuuint32_t box[3] = {Geom<TW>::TMA_COLS, CH, 1}, estr[3] = {1, 1, 1};
    return fn(m, tma_dtype<T>(), 3, const_cast<void *>(data), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, bool COEF>
cudaError_t launch_gauss11_t(const GaussLaunch &L, cudaStream_t st) {
    static DeviceOnce attr_set;
    const size_t smem = smem_bulk<64>(sizeof(T));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set.is_set(dev)) {
        cudaError_t e = cudaFuncSetAttribute(gauss11_kernel<T, COEF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set.set(dev);
    }
    int strips, segs;
    gauss11_items(L.x.H, L.x.W, L.seg_rows, &strips, &segs);
    GaussLaunch A = L;
    for (int n = 0; n < 11; ++n) {
        if (L.taps.g[n] != L.taps.g[sym(n)]) return cudaErrorInvalidValue;  // the passes assume symmetric taps
        A.taps2.g2[n] = make_float2(L.taps.g[n], L.taps.g[n]);
    }
    const uintptr_t vbytes = 4 * sizeof(T);  // one 4-element vector
    A.vec = ((uintptr_t)L.x.data % vbytes == 0) && ((uintptr_t)L.y.data % vbytes == 0) &&
            (L.x.row_stride % 4 == 0) && (L.x.image_stride % 4 == 0) && (L.y.image_stride % 4 == 0);
    dim3 grid(strips, segs, L.count);
    CUtensorMap mx, my;
    memset(&mx, 0, sizeof mx);
    memset(&my, 0, sizeof my);
    const bool tma =
        encode_plane_map<T, 64>(&mx, L.x.data, L.x.H, L.x.W, L.x.row_stride, L.x.image_stride, L.count) &&
        encode_plane_map<T, 64>(&my, L.y.data, L.y.H, L.y.W, L.y.row_stride, L.y.image_stride, L.count);
    gauss11_kernel<T, COEF><<<grid, Geom<64>::NT, smem, st>>>(mx, my, tma, A, strips, segs);
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
    *strips = (int)((OW + 63) / 64);
    *segs = (int)((OH + seg_rows - 1) / seg_rows);
    return *strips * *segs;
}

cudaError_t launch_gauss11(const GaussLaunch &L, cudaStream_t st) {
    const bool coef = L.co.coef != nullptr;
    switch (L.dtype) {
    case GBSSIM_U8: return coef ? launch_gauss11_t<uint8_t, true>(L, st) : launch_gauss11_t<uint8_t, false>(L, st);
    case GBSSIM_F16: return coef ? launch_gauss11_t<__half, true>(L, st) : launch_gauss11_t<__half, false>(L, st);
    case GBSSIM_BF16:
        return coef ? launch_gauss11_t<__nv_bfloat16, true>(L, st) : launch_gauss11_t<__nv_bfloat16, false>(L, st);
    case GBSSIM_F32: return coef ? launch_gauss11_t<float, true>(L, st) : launch_gauss11_t<float, false>(L, st);
    }
    return cudaErrorInvalidValue;
}

// mx, my: nullable level-0 bulk-copy maps (uniform batches only).
template <typename T, typename Src, int TW = 64>
cudaError_t launch_persistent_t(const Src &src, void *ws, int64_t counter_off, int64_t done_off, int64_t status_off,
                                unsigned wait_limit, const Taps<11> &taps, SsimConst cc, int grid, cudaStream_t st,
                                const CUtensorMap *mx = nullptr, const CUtensorMap *my = nullptr,
                                const PyrMaps *pm = nullptr) {
    constexpr bool can_bulk = std::is_same<Src, UniformSource>::value && TW == kUniformTW;
    constexpr size_t smem = persistent_smem<T, TW>(), smem_reg = raw_off<TW>();
    constexpr int NT = Geom<TW>::NT;
    static DeviceOnce attr_set;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set.is_set(dev)) {
        cudaError_t e = cudaFuncSetAttribute(gauss11_persistent_kernel<T, Src, false, TW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_reg);
        if constexpr (can_bulk)
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(gauss11_persistent_kernel<T, Src, true, TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set.set(dev);
    }
    Taps2<11> t2;
    for (int n = 0; n < 11; ++n) {
        if (taps.g[n] != taps.g[sym(n)]) return cudaErrorInvalidValue;  // the passes assume symmetric taps
        t2.g2[n] = make_float2(taps.g[n], taps.g[n]);
    }
    PyrMaps none;
    memset(&none, 0, sizeof none);
    if constexpr (can_bulk) {
        if (mx && my) {
            gauss11_persistent_kernel<T, Src, true, TW><<<grid, NT, smem, st>>>(
                *mx, *my, pm ? *pm : none, src, ws, counter_off, done_off, status_off, wait_limit, taps, t2, cc);
            return cudaGetLastError();
        }
    }
    CUtensorMap zx, zy;
    memset(&zx, 0, sizeof zx);
    memset(&zy, 0, sizeof zy);
    gauss11_persistent_kernel<T, Src, false, TW><<<grid, NT, smem_reg, st>>>(
        zx, zy, none, src, ws, counter_off, done_off, status_off, wait_limit, taps, t2, cc);
    return cudaGetLastError();
}

template <typename Src, int TW = 64>
cudaError_t launch_persistent(int dtype, const Src &src, void *ws, int64_t counter_off, int64_t done_off,
                              int64_t status_off, unsigned wait_limit, const Taps<11> &taps, SsimConst cc, int grid,
                              cudaStream_t st) {
    switch (dtype) {
    case GBSSIM_U8:
        return launch_persistent_t<uint8_t, Src, TW>(src, ws, counter_off, done_off, status_off, wait_limit, taps, cc,
                                                     grid, st);
    case GBSSIM_F16:
        return launch_persistent_t<__half, Src, TW>(src, ws, counter_off, done_off, status_off, wait_limit, taps, cc,
                                                    grid, st);
    case GBSSIM_BF16:
        return launch_persistent_t<__nv_bfloat16, Src, TW>(src, ws, counter_off, done_off, status_off, wait_limit,
                                                           taps, cc, grid, st);
    case GBSSIM_F32:
        return launch_persistent_t<float, Src, TW>(src, ws, counter_off, done_off, status_off, wait_limit, taps, cc,
                                                   grid, st);
    }
    return cudaErrorInvalidValue;
}

// Resident CTAs per SM of the persistent kernel of one dtype: the bulk-copy
// variant of uniform batches, or the table (ragged batch) variant of strip
// width TW; the >48 KB dynamic shared memory attribute must be set before
// the occupancy query sees it.  A uniform batch whose planes admit no
// bulk-copy map runs the register variant on a grid sized for the bulk one:
// the CTAs beyond the resident ones start as others finish and find the
// queue drained or not, either way correct.
template <typename T, int TW>
int max_ctas_t(bool table) {
    int n = 0;
    if (table) {
        auto kern = gauss11_persistent_kernel<T, TableSource, false, TW>;
        constexpr size_t smem = raw_off<TW>();
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Geom<TW>::NT, smem) != cudaSuccess)
            return 0;
    } else {
        auto kern = gauss11_persistent_kernel<T, UniformSource, true, kUniformTW>;
        constexpr size_t smem = persistent_smem<T>();
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Geom<kUniformTW>::NT, smem) != cudaSuccess)
            return 0;
    }
    return n;
}

template <int TW>
int max_ctas_dtype(int dtype, bool table) {
    switch (dtype) {
    case GBSSIM_U8: return max_ctas_t<uint8_t, TW>(table);
    case GBSSIM_F16: return max_ctas_t<__half, TW>(table);
    case GBSSIM_BF16: return max_ctas_t<__nv_bfloat16, TW>(table);
    case GBSSIM_F32: return max_ctas_t<float, TW>(table);
    }
    return 0;
}

int gauss11_batch_max_ctas_per_sm(int dtype, bool table, int tile_w) {
    if (!table) return max_ctas_dtype<kUniformTW>(dtype, false);
    switch (tile_w) {
    case 32: return max_ctas_dtype<32>(dtype, true);
    case 64: return max_ctas_dtype<64>(dtype, true);
    case 128: return max_ctas_dtype<128>(dtype, true);
    }
    return 0;
}

cudaError_t launch_batch(const BatchTable &B, const Taps<11> &taps, SsimConst cc, int grid, cudaStream_t st) {
    TableSource src{B};
    switch (B.tile_w) {
    case 32:
        return launch_persistent<TableSource, 32>(B.dtype, src, B.ws, B.counter_off, B.done_off, B.status_off,
                                                  B.wait_limit, taps, cc, grid, st);
    case 64:
        return launch_persistent<TableSource, 64>(B.dtype, src, B.ws, B.counter_off, B.done_off, B.status_off,
                                                  B.wait_limit, taps, cc, grid, st);
    case 128:
        return launch_persistent<TableSource, 128>(B.dtype, src, B.ws, B.counter_off, B.done_off, B.status_off,
                                                   B.wait_limit, taps, cc, grid, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_uniform_t(const UniformBatch &U0, const Taps<11> &taps, SsimConst cc, int grid, cudaStream_t st) {
    UniformBatch U = U0;
    CUtensorMap mx, my;
    constexpr int TW = kUniformTW;
    const bool bulk = encode_plane_map<T, TW>(&mx, U.x, U.lv[0].H, U.lv[0].W, U.rs, U.image_stride, U.count) &&
                      encode_plane_map<T, TW>(&my, U.y, U.lv[0].H, U.lv[0].W, U.rs, U.image_stride, U.count);
    // Arrival flags need the bulk-copy path: the register path's first rows
    // go through the read-only data cache, which bytes copied in during the
    // launch must not.
    if (U.arrive && !bulk) return cudaErrorNotSupported;
    // The uint16 pyramid is read by bulk copies only: it needs the bulk
    // variant (aligned level-0 planes) and a map per level; else the levels
    // fall back to fp32 planes (the workspace holds either layout).
    PyrMaps pm;
    memset(&pm, 0, sizeof pm);
    bool ipyr = U.ipyr && std::is_same<T, uint8_t>::value && bulk && U.scales - 1 <= kPyrMaps;
    for (int j = 1; ipyr && j < U.scales; ++j) {
        const UniformLevel &l = U.lv[j];
        char *xb = static_cast<char *>(U.ws) + l.x_off;
        const int64_t plane = l.H * l.pitch;
        ipyr = encode_plane_map<uint16_t, TW>(&pm.x[j - 1], xb, l.H, l.W, l.pitch, plane, U.count) &&
               encode_plane_map<uint16_t, TW>(&pm.y[j - 1], xb + 2 * plane * U.count, l.H, l.W, l.pitch, plane,
                                              U.count);
    }
    if (!ipyr && U.ipyr) {
        U.ipyr = 0;
        for (int j = 1; j < U.scales; ++j) {
            U.lv[j].pitch = U.lv[j].W;
            U.lv[j].vec = U.lv[j].W % 4 == 0;
        }
    }
    UniformSource src{U};
    return launch_persistent_t<T, UniformSource, TW>(src, U.ws, U.counter_off, U.done_off, U.status_off,
                                                     U.wait_limit, taps, cc, grid, st, bulk ? &mx : nullptr,
                                                     bulk ? &my : nullptr, ipyr ? &pm : nullptr);
}

cudaError_t launch_uniform(const UniformBatch &U, const Taps<11> &taps, SsimConst cc, int grid, cudaStream_t st) {
    switch (U.dtype) {
    case GBSSIM_U8: return launch_uniform_t<uint8_t>(U, taps, cc, grid, st);
    case GBSSIM_F16: return launch_uniform_t<__half>(U, taps, cc, grid, st);
    case GBSSIM_BF16: return launch_uniform_t<__nv_bfloat16>(U, taps, cc, grid, st);
    case GBSSIM_F32: return launch_uniform_t<float>(U, taps, cc, grid, st);
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
