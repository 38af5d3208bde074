// k_box.cu -- rectangular-window SSIM for 8-bit images with exact integer
// window sums (Section "Performance-Efficiency Tradeoffs" of arXiv 2101.06354,
// Eqs. integral_image_start .. corr_from_sum).
//
// The five local sums S1_x, S1_y, S2_x, S2_y, S_xy of every k x k window are
// formed exactly in integers.  Multiplying the statistics of
// Eqs. mean_from_sum .. corr_from_sum through by k^4 gives integer numerators,
//   l  = (2 S1x S1y + C1 k^4) / (S1x^2 + S1y^2 + C1 k^4)
//   cs = (2 (k^2 Sxy - S1x S1y) + C2 k^4) / ((k^2 S2x - S1x^2) + (k^2 S2y - S1y^2) + C2 k^4),
// whose integer parts are exact in int64 and are rounded to fp32 once each,
// so Q carries only a few fp32 roundings.
//
// Two tile schemes:
//  * block path (stride s a multiple of 4 and k a multiple of s): sums over
//    the non-overlapping s x s blocks, four pixels per dp4a instruction,
//    then each window adds (k/s)^2 block sums.  Every input byte is read
//    once from HBM; this is the HBM-bound configuration (8 x 8 at stride 4).
//  * integral-image path (any k <= 63, any stride): five summed-area tables
//    of a <= 64 x 64 input tile in shared memory (int32, zero first row and
//    column) and the paper's four-corner formula per window.

#include "tma.cuh"

namespace gbssim {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {  // looked up once (thread-safe static)
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    return fn;
}

namespace {

constexpr int NT = 256;
// stride-4 tiles: 64 x 16 blocks of 4 x 4 pixels loaded, VTOW x (17 - m)
// windows produced; VTOW is a multiple of 4 so every tile starts on a
// 16-byte boundary (tile column b starts at pixel 4 * VTOW * b) and
// VTOW + m - 1 <= 64.
constexpr int VBW = 64, VBH = 16, VTOW = 60;

struct BoxOut {
    int64_t s1x, s1y, s2x, s2y, sxy;
};

__device__ __forceinline__ void box_formula(const BoxOut &v, int k, float C1k4, float C2k4, float &q,
                                            float &cs) {
    const int64_t kk = (int64_t)k * k;
    const int64_t P = 2 * v.s1x * v.s1y;
    const int64_t Q1 = v.s1x * v.s1x + v.s1y * v.s1y;
    const int64_t Nxy = kk * v.sxy - v.s1x * v.s1y;
    const int64_t T2 = (kk * v.s2x - v.s1x * v.s1x) + (kk * v.s2y - v.s1y * v.s1y);
    // k <= 63: every term is below 2 k^4 255^2 < 2^48 (exact conversions without the FP64 pipe)
    const float A1 = i48_to_f32(P) + C1k4, B1 = i48_to_f32(Q1) + C1k4;
    const float A2 = fmaf(2.f, i48_to_f32(Nxy), C2k4), B2 = i48_to_f32(T2) + C2k4;
    cs = __fdividef(A2, B2);
    q = __fdividef(A1, B1) * cs;
}

// Same formula from the five window sums held as exact floats (integers below
// 2^24: k <= 12 keeps S2 <= 65025 * 144).  k^2 S2 - S1^2 is formed without
// cancellation: S1^2 = p + e exactly (p = fl(S1 S1), e = fma(S1, S1, -p),
// Dekker's TwoProduct), then fma(k^2, S2, -p) rounds once and e is taken off
// (two roundings in all, relative to the result).
__device__ __forceinline__ float exact_diff(float kk, float s2, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    return fmaf(kk, s2, -p) - e;
}
__device__ __forceinline__ void box_formula_f(float s1x, float s1y, float s2x, float s2y, float sxy, float kk,
                                              float C1k4, float C2k4, float &q, float &cs) {
    const float A1 = fmaf(2.f * s1x, s1y, C1k4), B1 = fmaf(s1x, s1x, fmaf(s1y, s1y, C1k4));
    const float nxy = exact_diff(kk, sxy, s1x, s1y);
    const float nxx = exact_diff(kk, s2x, s1x, s1x), nyy = exact_diff(kk, s2y, s1y, s1y);
    const float A2 = fmaf(2.f, nxy, C2k4), B2 = (nxx + nyy) + C2k4;
    cs = __fdividef(A2, B2);
    q = __fdividef(A1, B1) * cs;
}

// Compensated (Kahan) fp32 running sum.
struct KSumF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Output phase of the TMA stride-4 kernel: M x M blocks per window, block sums
// in shared memory as exact floats.
template <int M>
__device__ __forceinline__ void box_outputs(const float (&Bs)[5][VBH][VBW + 1], const BoxLaunch &L, int img,
                                            int64_t a0, int64_t b0, int tow, int toh, int64_t OH, int64_t OW,
                                            float &accQ, float &accCS) {
    const float kk = (float)(L.k * L.k);
    for (int o = threadIdx.x; o < tow * toh; o += NT) {
        const int oi = o / tow, oj = o - oi * tow;
        const int64_t a = a0 + oi, b = b0 + oj;
        if (a >= OH || b >= OW) continue;
        float acc[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            float sacc = 0.f;
#pragma unroll
            for (int u = 0; u < M; ++u)
#pragma unroll
                for (int v = 0; v < M; ++v) sacc += Bs[q][oi + u][oj + v];
            acc[q] = sacc;
        }
        if (L.sums_out) {
            int64_t *dst = L.sums_out + 5 * (img * OH * OW + a * OW + b);
#pragma unroll
            for (int q = 0; q < 5; ++q) dst[q] = (int64_t)acc[q];
            continue;
        }
        float qv, cs;
        box_formula_f(acc[0], acc[1], acc[2], acc[3], acc[4], kk, L.C1k4, L.C2k4, qv, cs);
        accQ += qv;
        accCS += cs;
        if (L.map) L.map[img * L.map_is + a * L.map_ld + b] = qv;
    }
}

__device__ __forceinline__ void box_outputs_m(int m, const float (&Bs)[5][VBH][VBW + 1], const BoxLaunch &L,
                                              int img, int64_t a0, int64_t b0, int tow, int toh, int64_t OH,
                                              int64_t OW, float &accQ, float &accCS) {
    if (m == 1) box_outputs<1>(Bs, L, img, a0, b0, tow, toh, OH, OW, accQ, accCS);
    else if (m == 2) box_outputs<2>(Bs, L, img, a0, b0, tow, toh, OH, OW, accQ, accCS);
    else box_outputs<3>(Bs, L, img, a0, b0, tow, toh, OH, OW, accQ, accCS);
}

// Sum (a, b) over the CTA: fp32 pairwise tree inside each warp, fp64 across
// warps (thread 0 holds the result).
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
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ra += (double)red[2 * w];
            rb += (double)red[2 * w + 1];
        }
}

// ------------------------------------------------------------------ stride-4 column walk
//
// Stride 4, k = 4M (M <= 3), 16-byte aligned rows.  One warp is one work
// item: a strip of 32 lanes x VB blocks of 4 x 4 pixels walked down a
// segment of block rows.  Per block row each lane loads 4 VB bytes of four
// pixel rows of x and y (one vector load per row and image), forms the five
// sums of its VB blocks with dp4a, takes the first M-1 block sums of the
// next lane by shuffle and adds the M blocks of each of its VB window
// columns (exact int32); the M rows of a window are added from a rolling
// register copy of the previous M-1 block rows.  Lane 31 only feeds lane 30,
// so strips advance by 31 lanes (31 VB window columns; 124 VB pixels keep
// the vector loads aligned).  Every input byte comes from HBM once; the M-1
// halo block rows of a segment are re-read, normally from L2.  Nothing goes
// through shared memory.
constexpr int S4C_VB = 4;                // blocks per lane
constexpr int S4C_STAGES = 2;            // block rows in flight per warp
constexpr int CW_STEP = 31 * S4C_VB;     // window columns per strip

__device__ __forceinline__ float i2f_exact(int v) { return __int2float_rn(v); }  // |v| < 2^24 here

template <int VB>
struct VecOf;
template <>
struct VecOf<4> {
    using T = uint4;
    static __device__ __forceinline__ unsigned get(const uint4 &v, int b) {
        return b == 0 ? v.x : b == 1 ? v.y : b == 2 ? v.z : v.w;
    }
    static __device__ __forceinline__ uint4 make(const unsigned (&w)[4]) { return make_uint4(w[0], w[1], w[2], w[3]); }
};
template <>
struct VecOf<2> {
    using T = uint2;
    static __device__ __forceinline__ unsigned get(const uint2 &v, int b) { return b == 0 ? v.x : v.y; }
    static __device__ __forceinline__ uint2 make(const unsigned (&w)[2]) { return make_uint2(w[0], w[1]); }
};

// Asynchronous copy of `bytes` (8 or 16) from global to shared memory; the
// first src_size bytes are read and the rest of the destination is zeroed
// (src_size 0: nothing is read).
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void *dst, const void *src, int src_size) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_size) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(src_size) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Dynamic shared memory of box_s4c_kernel<M, VB, S>: per warp, S stages of
// (x, y) x 4 pixel rows x 32 lanes of 4 VB bytes.
template <int VB, int S>
constexpr size_t s4c_smem() { return (size_t)(NT / 32) * S * 2 * 4 * 32 * 4 * VB; }

template <int M, int VB, int S>
__global__ void __launch_bounds__(NT) box_s4c_kernel(const BoxLaunch L, int strips, int segs, int seg_rows) {
    static_assert(M - 1 <= VB, "the next lane must hold the M-1 halo blocks");
    static_assert(S >= 2, "at least double buffering");
    using V = VecOf<VB>;
    using VT = typename V::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int MP = M > 1 ? M - 1 : 1;
    const int lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    const int64_t per_img = (int64_t)strips * segs;
    if (item >= per_img * L.count) return;  // whole warps only
    const int img = (int)(item / per_img);
    const int rem = (int)(item - (int64_t)img * per_img);
    const int seg = rem / strips, strip = rem - seg * strips;
    const int64_t H = L.x.H, W = L.x.W, rs = L.x.row_stride;
    const int64_t OH = out_dim(H, 4 * M, 4), OW = out_dim(W, 4 * M, 4);
    const uint8_t *xb = static_cast<const uint8_t *>(L.x.data) + img * L.x.image_stride;
    const uint8_t *yb = static_cast<const uint8_t *>(L.y.data) + img * L.y.image_stride;
    const int64_t bc = (int64_t)strip * (31 * VB) + VB * lane;  // first block (= window) column of the lane
    const int64_t c0 = 4 * bc;                               // its first pixel column
    const int64_t a_begin = (int64_t)seg * seg_rows;
    const int nout = (int)min((int64_t)seg_rows, OH - a_begin);
    const float kk = (float)(16 * M * M);
    int hp[MP][VB][5];  // window-column sums of the previous M-1 block rows
    KSumF accQ, accCS;
    // Per-lane staging ring: block row i lives in stage i % S.  Each lane
    // copies and later reads only its own bytes, so no barrier is needed; the
    // copy of block row i + S - 1 is issued before row i is summed and
    // overwrites the stage of row i - 1, whose values were consumed in the
    // previous iteration.  Ragged right edge: whole 4-pixel blocks only (the
    // rest zero-filled); rows past the image bottom are zero-filled.
    VT *ring = reinterpret_cast<VT *>(smem_raw) + (size_t)(threadIdx.x >> 5) * S * 2 * 4 * 32 + lane;
    const int nrows = nout + M - 1;
    const int nb = (int)max((int64_t)0, min((int64_t)VB, (W - c0) / 4));  // whole blocks inside the image
    auto issue = [&](int i) {
        const int64_t br = a_begin + i;
        VT *st = ring + (size_t)(i % S) * 2 * 4 * 32;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t row = 4 * br + r;
            const bool in = row < H && nb > 0;
            const int bytes = in ? 4 * nb : 0;
            const uint8_t *px = in ? xb + row * rs + c0 : xb, *py = in ? yb + row * rs + c0 : yb;
            cp_async_zfill<4 * VB>(st + r * 32, px, bytes);
            cp_async_zfill<4 * VB>(st + (4 + r) * 32, py, bytes);
        }
    };
#pragma unroll
    for (int i = 0; i < S - 1; ++i) {
        if (i < nrows) issue(i);
        cp_async_commit();
    }
    for (int i = 0; i < nrows; ++i) {
        const int64_t br = a_begin + i;
        if (i + S - 1 < nrows) issue(i + S - 1);
        cp_async_commit();
        cp_async_wait<S - 1>();  // block row i has landed
        const VT *st = ring + (size_t)(i % S) * 2 * 4 * 32;
        VT vx[4], vy[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            vx[r] = st[r * 32];
            vy[r] = st[(4 + r) * 32];
        }
        int B[VB][5];
#pragma unroll
        for (int b = 0; b < VB; ++b) {
            unsigned sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const unsigned wx = V::get(vx[r], b);
                const unsigned wy = V::get(vy[r], b);
                sx = __dp4a(wx, 0x01010101u, sx);
                sy = __dp4a(wy, 0x01010101u, sy);
                sxx = __dp4a(wx, wx, sxx);
                syy = __dp4a(wy, wy, syy);
                sxy = __dp4a(wx, wy, sxy);
            }
            B[b][0] = (int)sx;
            B[b][1] = (int)sy;
            B[b][2] = (int)sxx;
            B[b][3] = (int)syy;
            B[b][4] = (int)sxy;
        }
        int N[MP][5];  // first M-1 blocks of the next lane
#pragma unroll
        for (int j = 0; j < M - 1; ++j)
#pragma unroll
            for (int q = 0; q < 5; ++q) N[j][q] = __shfl_down_sync(0xffffffffu, B[j][q], 1);
        int Hc[VB][5];
#pragma unroll
        for (int t = 0; t < VB; ++t)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                int v = 0;
#pragma unroll
                for (int j = 0; j < M; ++j) v += t + j < VB ? B[t + j][q] : N[t + j - VB][q];
                Hc[t][q] = v;
            }
        if (i >= M - 1) {
            const int64_t a = br - (M - 1);
#pragma unroll
            for (int t = 0; t < VB; ++t) {
                int w[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    int v = Hc[t][q];
#pragma unroll
                    for (int j = 0; j < M - 1; ++j) v += hp[j][t][q];
                    w[q] = v;
                }
                const int64_t b = bc + t;
                if (lane < 31 && b < OW) {
                    if (L.sums_out) {
                        int64_t *dst = L.sums_out + 5 * ((int64_t)img * OH * OW + a * OW + b);
#pragma unroll
                        for (int q = 0; q < 5; ++q) dst[q] = w[q];
                    } else {
                        float qv, cs;
                        box_formula_f(i2f_exact(w[0]), i2f_exact(w[1]), i2f_exact(w[2]), i2f_exact(w[3]),
                                      i2f_exact(w[4]), kk, L.C1k4, L.C2k4, qv, cs);
                        accQ.add(qv);
                        accCS.add(cs);
                        if (L.map) L.map[img * L.map_is + a * L.map_ld + b] = qv;
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j + 1 < M - 1; ++j)
#pragma unroll
            for (int t = 0; t < VB; ++t)
#pragma unroll
                for (int q = 0; q < 5; ++q) hp[j][t][q] = hp[j + 1][t][q];
        if (M > 1) {
#pragma unroll
            for (int t = 0; t < VB; ++t)
#pragma unroll
                for (int q = 0; q < 5; ++q) hp[MP - 1][t][q] = Hc[t][q];
        }
    }
    if (L.partials) {
        double sq = (double)accQ.s - (double)accQ.c, sc = (double)accCS.s - (double)accCS.c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_down_sync(0xffffffffu, sq, o);
            sc += __shfl_down_sync(0xffffffffu, sc, o);
        }
        if (lane == 0) L.partials[item] = make_double2(sq, sc);
    }
}

// ------------------------------------------------------------------ stride-4 TMA path
//
// Persistent CTAs walk their tiles round-robin (tile t = blockIdx.x + k *
// gridDim.x, so the pooling slots stay deterministic).  Per tile one thread
// issues two 3-D bulk tensor copies (x and y: 256 x 64 bytes of image z at
// (x0, y0)) into one of two shared-memory stages and arms that stage's
// mbarrier with the expected byte count; the copy of tile k+2 is in flight
// while tile k is summed.  Out-of-image bytes arrive as zeros and only feed
// windows outside the map.  Every mbarrier wait is bounded: on timeout the
// CTA writes NaN into the pooling slots of its remaining tiles (the score
// then reads NaN), waits (bounded) for its own copies still in flight and
// returns.
constexpr int TMA_W = 256, TMA_H = 64;          // bytes per row, rows per tile
constexpr unsigned TMA_TILE = TMA_W * TMA_H;    // bytes per image per tile

struct __align__(128) TmaSmem {
    unsigned char st[2][2][TMA_H][TMA_W];  // [stage][x|y][row][byte]
    float Bs[5][VBH][VBW + 1];
    float red[2 * NT / 32];
    unsigned long long bar[2];
};

__global__ void __launch_bounds__(NT) box_tma_kernel(const __grid_constant__ CUtensorMap tmx,
                                                     const __grid_constant__ CUtensorMap tmy, const BoxLaunch L,
                                                     int tiles_x, int tiles_y) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaSmem &S = *reinterpret_cast<TmaSmem *>(smem_raw);
    const int m = L.k >> 2;
    const int toh = VBH - m + 1;
    const int64_t OH = out_dim(L.x.H, L.k, 4), OW = out_dim(L.x.W, L.k, 4);
    const int per_img = tiles_x * tiles_y;
    const int total = per_img * L.count;
    const int ntiles = blockIdx.x < total ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int k, int stage) {
        const int t = blockIdx.x + k * gridDim.x;
        const int img = t / per_img, rem = t - img * per_img;
        const int ty = rem / tiles_x, tx = rem - ty * tiles_x;
        const int x0 = tx * VTOW * 4, y0 = ty * toh * 4;
        mbar_expect_tx(&S.bar[stage], 2 * TMA_TILE);
        tma_load_3d(&S.st[stage][0][0][0], &tmx, x0, y0, img, &S.bar[stage]);
        tma_load_3d(&S.st[stage][1][0][0], &tmy, x0, y0, img, &S.bar[stage]);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < 2 && k < ntiles; ++k) issue(k, k);

    const int bi = threadIdx.x >> 4, qd = threadIdx.x & 15;
    for (int k = 0; k < ntiles; ++k) {
        const int stage = k & 1;
        const unsigned parity = (k >> 1) & 1;
        const bool ok = mbar_wait_bounded(&S.bar[stage], parity);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                for (int r = k; r < ntiles; ++r) {
                    const int t = blockIdx.x + r * gridDim.x;
                    if (L.partials) L.partials[t] = make_double2(nan(""), nan(""));
                }
                // drain this CTA's copies still in flight (tiles k and k+1)
                for (int r = k; r < ntiles && r < k + 2; ++r) mbar_wait_bounded(&S.bar[r & 1], (r >> 1) & 1);
            }
            __syncthreads();
            return;
        }
        const int t = blockIdx.x + k * gridDim.x;
        const int img = t / per_img, rem = t - img * per_img;
        const int tyi = rem / tiles_x, txi = rem - tyi * tiles_x;
        // block sums of the four 4x4 blocks (rows 4bi..4bi+3, columns 16qd..16qd+15)
        uint4 vx[4], vy[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            vx[r] = *reinterpret_cast<const uint4 *>(&S.st[stage][0][4 * bi + r][16 * qd]);
            vy[r] = *reinterpret_cast<const uint4 *>(&S.st[stage][1][4 * bi + r][16 * qd]);
        }
        __syncthreads();  // the stage is consumed: refill it with tile k + 2
        if (threadIdx.x == 0 && k + 2 < ntiles) {
            fence_proxy_async_smem();
            issue(k + 2, stage);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            unsigned sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const unsigned wx = b == 0 ? vx[r].x : b == 1 ? vx[r].y : b == 2 ? vx[r].z : vx[r].w;
                const unsigned wy = b == 0 ? vy[r].x : b == 1 ? vy[r].y : b == 2 ? vy[r].z : vy[r].w;
                sx = __dp4a(wx, 0x01010101u, sx);
                sy = __dp4a(wy, 0x01010101u, sy);
                sxx = __dp4a(wx, wx, sxx);
                syy = __dp4a(wy, wy, syy);
                sxy = __dp4a(wx, wy, sxy);
            }
            const int bj = 4 * qd + b;
            S.Bs[0][bi][bj] = (float)sx;
            S.Bs[1][bi][bj] = (float)sy;
            S.Bs[2][bi][bj] = (float)sxx;
            S.Bs[3][bi][bj] = (float)syy;
            S.Bs[4][bi][bj] = (float)sxy;
        }
        __syncthreads();
        const int64_t a0 = (int64_t)tyi * toh, b0 = (int64_t)txi * VTOW;
        float accQ = 0.f, accCS = 0.f;
        box_outputs_m(m, S.Bs, L, img, a0, b0, VTOW, toh, OH, OW, accQ, accCS);
        double da, db;
        block_sum2f(accQ, accCS, S.red, da, db);  // also orders the Bs reads before the next tile's writes
        if (threadIdx.x == 0 && L.partials) L.partials[t] = make_double2(da, db);
    }
}

bool encode_u8_map(CUtensorMap *map, const ImgDesc &d, int count) {
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)d.W, (cuuint64_t)d.H, (cuuint64_t)count};
    const cuuint64_t strides[2] = {(cuuint64_t)d.row_stride, (cuuint64_t)d.image_stride};
    const cuuint32_t box[3] = {TMA_W, TMA_H, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(d.data), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ------------------------------------------------------------------ block path

constexpr int BW = 32, BH = 16;  // blocks per CTA tile

__global__ void __launch_bounds__(NT) box_block_kernel(const BoxLaunch L, int tiles_x, int tiles_y,
                                                       int aligned4) {
    __shared__ unsigned Bs[5][BH][BW + 1];
    __shared__ float red[2 * NT / 32];
    const int s = L.stride, m = L.k / L.stride, wps = s >> 2;
    const int tow = BW - m + 1, toh = BH - m + 1;
    const int img = blockIdx.z;
    const int64_t H = L.x.H, W = L.x.W, rs = L.x.row_stride;
    const int64_t OH = out_dim(H, L.k, s), OW = out_dim(W, L.k, s);
    const int64_t a0 = (int64_t)blockIdx.y * toh, b0 = (int64_t)blockIdx.x * tow;
    const uint8_t *xb = static_cast<const uint8_t *>(L.x.data) + img * L.x.image_stride;
    const uint8_t *yb = static_cast<const uint8_t *>(L.y.data) + img * L.y.image_stride;

    for (int t = threadIdx.x; t < BW * BH; t += NT) {
        const int bi = t / BW, bj = t - bi * BW;
        const int64_t r0 = (a0 + bi) * s, c0 = (b0 + bj) * s;
        unsigned sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
        if (r0 + s <= H && c0 + s <= W) {  // partial blocks feed no valid window
            for (int r = 0; r < s; ++r) {
                const uint8_t *px = xb + (r0 + r) * rs + c0, *py = yb + (r0 + r) * rs + c0;
                for (int w = 0; w < wps; ++w) {
                    unsigned wx, wy;
                    if (aligned4) {
                        wx = __ldg(reinterpret_cast<const unsigned *>(px) + w);
                        wy = __ldg(reinterpret_cast<const unsigned *>(py) + w);
                    } else {
                        wx = wy = 0;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            wx |= (unsigned)__ldg(px + 4 * w + u) << (8 * u);
                            wy |= (unsigned)__ldg(py + 4 * w + u) << (8 * u);
                        }
                    }
                    sx = __dp4a(wx, 0x01010101u, sx);
                    sy = __dp4a(wy, 0x01010101u, sy);
                    sxx = __dp4a(wx, wx, sxx);
                    syy = __dp4a(wy, wy, syy);
                    sxy = __dp4a(wx, wy, sxy);
                }
            }
        }
        Bs[0][bi][bj] = sx;
        Bs[1][bi][bj] = sy;
        Bs[2][bi][bj] = sxx;
        Bs[3][bi][bj] = syy;
        Bs[4][bi][bj] = sxy;
    }
    __syncthreads();

    float accQ = 0.f, accCS = 0.f;
    for (int t = threadIdx.x; t < tow * toh; t += NT) {
        const int oi = t / tow, oj = t - oi * tow;
        const int64_t a = a0 + oi, b = b0 + oj;
        if (a >= OH || b >= OW) continue;
        int64_t acc[5] = {0, 0, 0, 0, 0};
        for (int u = 0; u < m; ++u)
            for (int v = 0; v < m; ++v)
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[q] += Bs[q][oi + u][oj + v];
        BoxOut o{acc[0], acc[1], acc[2], acc[3], acc[4]};
        if (L.sums_out) {
            int64_t *dst = L.sums_out + 5 * (img * OH * OW + a * OW + b);
#pragma unroll
            for (int q = 0; q < 5; ++q) dst[q] = acc[q];
            continue;
        }
        float q, cs;
        box_formula(o, L.k, L.C1k4, L.C2k4, q, cs);
        accQ += q;
        accCS += cs;
        if (L.map) L.map[img * L.map_is + a * L.map_ld + b] = q;
    }
    if (L.partials) {
        double da, db;
        block_sum2f(accQ, accCS, red, da, db);
        if (threadIdx.x == 0)
            L.partials[((int64_t)img * tiles_y + blockIdx.y) * tiles_x + blockIdx.x] = make_double2(da, db);
    }
}

// ------------------------------------------------------------------ integral-image path

constexpr int RMAX = 64;             // input tile rows / columns (max)
constexpr int SP = RMAX + 1;         // SAT pitch (first row/column are zero)

struct SatSmem {
    int sat[5][SP][SP + 1];
    float red[2 * NT / 32];
};

__host__ __device__ inline int sat_tile_outputs(int k, int s) {
    return k > RMAX ? 0 : (RMAX - k) / s + 1;
}

__global__ void __launch_bounds__(NT) box_sat_kernel(const BoxLaunch L, int tiles_x, int tiles_y) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SatSmem &S = *reinterpret_cast<SatSmem *>(smem_raw);
    const int k = L.k, s = L.stride;
    const int to = sat_tile_outputs(k, s);
    const int img = blockIdx.z;
    const int64_t H = L.x.H, W = L.x.W, rs = L.x.row_stride;
    const int64_t OH = out_dim(H, k, s), OW = out_dim(W, k, s);
    const int64_t a0 = (int64_t)blockIdx.y * to, b0 = (int64_t)blockIdx.x * to;
    const int64_t r0 = a0 * s, c0 = b0 * s;
    const int R = (int)min((int64_t)(to - 1) * s + k, H - r0);
    const int C = (int)min((int64_t)(to - 1) * s + k, W - c0);
    const uint8_t *xb = static_cast<const uint8_t *>(L.x.data) + img * L.x.image_stride;
    const uint8_t *yb = static_cast<const uint8_t *>(L.y.data) + img * L.y.image_stride;

    // products at [r+1][c+1]; zero first row and column
    for (int t = threadIdx.x; t < (R + 1) * (C + 1); t += NT) {
        const int r = t / (C + 1), c = t - r * (C + 1);
        int v[5] = {0, 0, 0, 0, 0};
        if (r > 0 && c > 0) {
            const int p = __ldg(xb + (r0 + r - 1) * rs + c0 + c - 1);
            const int q = __ldg(yb + (r0 + r - 1) * rs + c0 + c - 1);
            v[0] = p; v[1] = q; v[2] = p * p; v[3] = q * q; v[4] = p * q;
        }
#pragma unroll
        for (int u = 0; u < 5; ++u) S.sat[u][r][c] = v[u];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 5 * R; t += NT) {  // row prefix sums
        const int u = t / R, r = 1 + t - u * R;
        int acc = 0;
        for (int c = 1; c <= C; ++c) S.sat[u][r][c] = (acc += S.sat[u][r][c]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 5 * C; t += NT) {  // column prefix sums
        const int u = t / C, c = 1 + t - u * C;
        int acc = 0;
        for (int r = 1; r <= R; ++r) S.sat[u][r][c] = (acc += S.sat[u][r][c]);
    }
    __syncthreads();

    float accQ = 0.f, accCS = 0.f;
    for (int t = threadIdx.x; t < to * to; t += NT) {
        const int oi = t / to, oj = t - oi * to;
        const int64_t a = a0 + oi, b = b0 + oj;
        if (a >= OH || b >= OW) continue;
        // 1-based top-left (i, j) = (oi*s + 1, oj*s + 1) inside the tile:
        // S = I(i+k-1, j+k-1) + I(i-1, j-1) - I(i+k-1, j-1) - I(i-1, j+k-1)
        const int i = oi * s + 1, j = oj * s + 1;
        int64_t acc[5];
#pragma unroll
        for (int u = 0; u < 5; ++u)
            acc[u] = (int64_t)S.sat[u][i + k - 1][j + k - 1] + S.sat[u][i - 1][j - 1] -
                     S.sat[u][i + k - 1][j - 1] - S.sat[u][i - 1][j + k - 1];
        if (L.sums_out) {
            int64_t *dst = L.sums_out + 5 * (img * OH * OW + a * OW + b);
#pragma unroll
            for (int u = 0; u < 5; ++u) dst[u] = acc[u];
            continue;
        }
        BoxOut o{acc[0], acc[1], acc[2], acc[3], acc[4]};
        float q, cs;
        box_formula(o, k, L.C1k4, L.C2k4, q, cs);
        accQ += q;
        accCS += cs;
        if (L.map) L.map[img * L.map_is + a * L.map_ld + b] = q;
    }
    if (L.partials) {
        double da, db;
        block_sum2f(accQ, accCS, S.red, da, db);
        if (threadIdx.x == 0)
            L.partials[((int64_t)img * tiles_y + blockIdx.y) * tiles_x + blockIdx.x] = make_double2(da, db);
    }
}

bool use_block_path(int k, int s) { return s % 4 == 0 && k % s == 0 && k <= 16; }
bool use_s4_path(int k, int s) { return s == 4 && k % 4 == 0 && k <= 12 && VTOW + k / 4 - 1 <= VBW; }

// Block rows (= output rows) per warp item of the column-walk kernel.
constexpr int kS4cSeg = 32;

enum BoxLayout { LAYOUT_S4C, LAYOUT_TMA, LAYOUT_BLOCK, LAYOUT_SAT };

BoxLayout box_layout(int k, int s, bool aligned16, bool tma) {
    if (aligned16 && use_s4_path(k, s)) return tma ? LAYOUT_TMA : LAYOUT_S4C;
    return use_block_path(k, s) ? LAYOUT_BLOCK : LAYOUT_SAT;
}

void box_tiles(int64_t OH, int64_t OW, int k, int s, BoxLayout lay, int *tx, int *ty) {
    if (lay == LAYOUT_S4C) {
        *tx = (int)((OW + CW_STEP - 1) / CW_STEP);
        *ty = (int)((OH + kS4cSeg - 1) / kS4cSeg);
    } else if (lay == LAYOUT_TMA) {
        const int m = k / 4;
        *tx = (int)((OW + VTOW - 1) / VTOW);
        *ty = (int)((OH + VBH - m) / (VBH - m + 1));
    } else if (lay == LAYOUT_BLOCK) {
        const int m = k / s;
        const int tow = BW - m + 1, toh = BH - m + 1;
        *tx = (int)((OW + tow - 1) / tow);
        *ty = (int)((OH + toh - 1) / toh);
    } else {
        const int to = sat_tile_outputs(k, s);
        *tx = (int)((OW + to - 1) / to);
        *ty = (int)((OH + to - 1) / to);
    }
}

}  // namespace

// The stride-4 paths need 16-byte aligned rows, and the opt-in TMA kernel
// has its own tiles.  Workspace sizing uses the largest item count of all
// layouts (box_items_ks); a launch uses the layout its pointers and flags
// select, and the host pools box_path_items of that layout.
bool box_aligned16(const ImgDesc &x, const ImgDesc &y) {
    const uintptr_t bx = (uintptr_t)x.data, by = (uintptr_t)y.data;
    return bx % 16 == 0 && by % 16 == 0 && x.row_stride % 16 == 0 && y.row_stride % 16 == 0 &&
           x.image_stride % 16 == 0 && y.image_stride % 16 == 0;
}

int box_path_items(int64_t OH, int64_t OW, int k, int s, bool aligned16, bool tma) {
    int tx, ty;
    box_tiles(OH, OW, k, s, box_layout(k, s, aligned16, tma), &tx, &ty);
    return tx * ty;
}

int box_items_ks(int64_t OH, int64_t OW, int k, int s) {
    int best = 0;
    for (int a = 0; a < 2; ++a)
        for (int t = 0; t < 2; ++t) best = max(best, box_path_items(OH, OW, k, s, a != 0, t != 0));
    return best;
}

template <int M>
cudaError_t launch_s4c(const BoxLaunch &L, int tx, int ty, unsigned ctas, cudaStream_t st) {
    constexpr size_t smem = s4c_smem<S4C_VB, S4C_STAGES>();
    static DeviceOnce attr_set;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set.is_set(dev)) {
        const cudaError_t e = cudaFuncSetAttribute(box_s4c_kernel<M, S4C_VB, S4C_STAGES>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set.set(dev);
    }
    box_s4c_kernel<M, S4C_VB, S4C_STAGES><<<ctas, NT, smem, st>>>(L, tx, ty, kS4cSeg);
    return cudaGetLastError();
}

cudaError_t launch_box_u8(const BoxLaunch &L, cudaStream_t st) {
    const int64_t OH = out_dim(L.x.H, L.k, L.stride), OW = out_dim(L.x.W, L.k, L.stride);
    if (L.count <= 0 || OH <= 0 || OW <= 0) return cudaSuccess;
    const BoxLayout lay = box_layout(L.k, L.stride, box_aligned16(L.x, L.y), L.use_tma);
    int tx, ty;
    box_tiles(OH, OW, L.k, L.stride, lay, &tx, &ty);
    dim3 grid(tx, ty, L.count);
    if (lay == LAYOUT_TMA) {
        CUtensorMap mx, my;
        // the item count was fixed for this layout: no silent fallback
        if (!encode_u8_map(&mx, L.x, L.count) || !encode_u8_map(&my, L.y, L.count)) return cudaErrorInvalidValue;
        static DeviceOnce attr_set;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!attr_set.is_set(dev)) {
            cudaError_t e = cudaFuncSetAttribute(box_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sizeof(TmaSmem));
            if (e != cudaSuccess) return e;
            attr_set.set(dev);
        }
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, box_tma_kernel, NT, sizeof(TmaSmem));
        const int total = tx * ty * L.count;
        const int g = min(total, max(1, sms * max(per_sm, 1)));
        box_tma_kernel<<<g, NT, sizeof(TmaSmem), st>>>(mx, my, L, tx, ty);
    } else if (lay == LAYOUT_S4C) {
        const int64_t warps = (int64_t)tx * ty * L.count;
        const int64_t ctas = (warps + NT / 32 - 1) / (NT / 32);
        if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
        const int m = L.k / 4;
        if (m == 1) return launch_s4c<1>(L, tx, ty, (unsigned)ctas, st);
        if (m == 2) return launch_s4c<2>(L, tx, ty, (unsigned)ctas, st);
        return launch_s4c<3>(L, tx, ty, (unsigned)ctas, st);
    } else if (use_block_path(L.k, L.stride)) {
        const uintptr_t bx = (uintptr_t)L.x.data, by = (uintptr_t)L.y.data;
        const int aligned4 = (bx % 4 == 0) && (by % 4 == 0) && (L.x.row_stride % 4 == 0) &&
                             (L.y.row_stride % 4 == 0) && (L.x.image_stride % 4 == 0) &&
                             (L.y.image_stride % 4 == 0);
        box_block_kernel<<<grid, NT, 0, st>>>(L, tx, ty, aligned4);
    } else {
        static DeviceOnce attr_set;
        const size_t smem = sizeof(SatSmem);
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!attr_set.is_set(dev)) {
            cudaError_t e = cudaFuncSetAttribute(box_sat_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set.set(dev);
        }
        box_sat_kernel<<<grid, NT, smem, st>>>(L, tx, ty);
    }
    return cudaGetLastError();
}

}  // namespace gbssim
