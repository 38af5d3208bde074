// k_poolmap.cu -- the pooling family on stored SSIM maps (Section
// "Spatio-temporal Aggregation of Quality Scores" of arXiv 2101.06354):
// coefficient of variation, Minkowski, distortion-weighted, mean-deviation,
// geometric / harmonic means of 1 - Q, percentiles, median, five-number
// summary and percentile pooling of `count` float maps.
//
// Moment kinds: one pass (two for the kinds that need the mean first) of
// per-item partial sums -- fp32 per element, compensated fp32 per thread,
// fp64 across the CTA -- combined per image in a fixed order in fp64, so the
// result is deterministic.
//
// Order statistics: an exact radix select on the order-preserving 32-bit key
// of each float (sign-magnitude flipped to unsigned order), 8 bits per pass.
// Pass 0 counts the top byte of every key; a one-warp-per-image step finds,
// for every wanted rank, the bin that holds it; passes 1-3 count the next
// byte of the keys inside each wanted bin.  Four reads of the map give the
// exact k-th smallest values, the values a sort would give, so percentiles
// interpolate between the same order statistics as a sorted list (position
// h = p/100 (n-1), linear).  Shared-memory counts are aggregated per warp
// (one atomic per distinct bin), since SSIM values crowd into few bins.
#include "common.cuh"

namespace gbssim {
namespace {

constexpr int NT = 256;
constexpr int PR = 16;          // map rows per item (moment partial sums, select counts)
constexpr int NBIN = 256;       // histogram bins per select pass (8 key bits)
constexpr int UNR = 8;          // loads in flight per thread and row
constexpr int64_t CHK = 32768;  // map elements per item of a dense map (flat chunks)
constexpr int UNR4 = 4;         // float4 loads in flight per thread (dense maps)

// Calls f(q, mu) for every element of one work item: with DENSE (ld == w and
// 16-byte aligned images) the flat chunk [item CHK, (item + 1) CHK) read as
// float4 groups, UNR4 of them in flight per thread; else PR rows, UNR scalar
// loads in flight per thread and row.  `ax` (nullable) is read alongside.
template <bool DENSE, int64_t CHUNK = CHK, typename F>
__device__ __forceinline__ void for_item(const float *m, const float *ax, int64_t h, int64_t w, int64_t ld,
                                         int item, F &&f) {
    if constexpr (DENSE) {
        const int64_t n = h * w, e0 = (int64_t)item * CHUNK, e1 = min(e0 + CHUNK, n);
        for (int64_t g0 = e0 + 4 * threadIdx.x; g0 < e1; g0 += 4 * NT * UNR4) {
            float4 v[UNR4], u[UNR4];
#pragma unroll
            for (int k = 0; k < UNR4; ++k) {  // all loads first
                const int64_t e = g0 + 4 * NT * k;
                v[k] = u[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (e + 4 <= e1) {
                    v[k] = __ldg(reinterpret_cast<const float4 *>(m + e));
                    if (ax) u[k] = __ldg(reinterpret_cast<const float4 *>(ax + e));
                } else if (e < e1) {
                    v[k].x = __ldg(m + e);
                    if (e + 1 < e1) v[k].y = __ldg(m + e + 1);
                    if (e + 2 < e1) v[k].z = __ldg(m + e + 2);
                    if (ax) {
                        u[k].x = __ldg(ax + e);
                        if (e + 1 < e1) u[k].y = __ldg(ax + e + 1);
                        if (e + 2 < e1) u[k].z = __ldg(ax + e + 2);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < UNR4; ++k) {
                const int64_t e = g0 + 4 * NT * k;
                if (e < e1) f(v[k].x, u[k].x);
                if (e + 1 < e1) f(v[k].y, u[k].y);
                if (e + 2 < e1) f(v[k].z, u[k].z);
                if (e + 3 < e1) f(v[k].w, u[k].w);
            }
        }
    } else {
        constexpr int64_t ROWS = PR * (CHUNK / CHK);  // rows per item scale with the chunk
        const int64_t r0 = (int64_t)item * ROWS;
        for (int64_t row = r0; row < min(r0 + ROWS, h); ++row) {
            const float *rp = m + row * ld;
            const float *ap = ax ? ax + row * ld : nullptr;
            for (int64_t c0 = 0; c0 < w; c0 += UNR * NT) {
                float v[UNR], u[UNR];
#pragma unroll
                for (int k = 0; k < UNR; ++k) {  // all loads first
                    const int64_t col = c0 + threadIdx.x + k * NT;
                    v[k] = col < w ? __ldg(rp + col) : 0.f;
                    u[k] = ap && col < w ? __ldg(ap + col) : 0.f;
                }
#pragma unroll
                for (int k = 0; k < UNR; ++k)
                    if (c0 + threadIdx.x + k * NT < w) f(v[k], u[k]);
            }
        }
    }
}

struct KSumP {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float get() const { return s - c; }
};

__device__ __forceinline__ unsigned f2key(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

enum MomentOp { M_SUM = 0, M_SQDEV = 1, M_ABSDEV_P = 2, M_MINK = 3, M_DW = 4, M_LOG_D = 5, M_INV_D = 6, M_PP = 7,
                M_LW = 8 };

// d^p, by multiplication for the small integer exponents (uniform across
// the launch, so the branch costs nothing), else powf.
__device__ __forceinline__ float pow_arg(float d, float p) {
    if (p == 1.f) return d;
    if (p == 2.f) return d * d;
    if (p == 3.f) return d * d * d;
    if (p == 4.f) {
        const float d2 = d * d;
        return d2 * d2;
    }
    return powf(d, p);
}

// Ops whose second sum b is not always zero.
__host__ __device__ constexpr bool has_b(int op) { return op == M_DW || op == M_LOG_D || op == M_INV_D; }

// Per-element contribution (a, b) of moment op `op`; m = the image's mean
// (or the PP threshold), p, r = arguments; mu = the auxiliary map's value
// (luminance-weighted pooling: the reference's local mean, p = a_s, r = b_s).
template <int op>
__device__ __forceinline__ void contrib(float q, float m, float p, float r, float mu, float &a, float &b) {
    b = 0.f;
    switch (op) {
    case M_LW: {
        const float wl = mu < p ? 0.f : (mu < p + r ? (mu - p) / r : 1.f);
        a = wl * q;
    } break;
    case M_SUM: a = q; break;
    case M_SQDEV: { const float d = q - m; a = d * d; } break;
    case M_ABSDEV_P: a = pow_arg(fabsf(q - m), p); break;
    case M_MINK: a = pow_arg(1.f - q, p); break;
    case M_DW: { const float w = pow_arg(1.f - q, p); a = w * q; b = w; } break;
    // a zero dissimilarity is counted in b (its log / reciprocal is infinite,
    // which a compensated sum cannot carry); any such value makes GM / HM 0
    case M_LOG_D: { const float d = 1.f - q; a = d == 0.f ? 0.f : logf(d); b = d == 0.f ? 1.f : 0.f; } break;
    case M_INV_D: { const float d = 1.f - q; a = d == 0.f ? 0.f : 1.f / d; b = d == 0.f ? 1.f : 0.f; } break;
    default: a = q <= m ? q / r : q; break;  // M_PP
    }
}

__device__ __forceinline__ void block_sum2d(double &a, double &b, double *red) {
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
    if (threadIdx.x == 0) {
        a = b = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
            a += red[2 * w];
            b += red[2 * w + 1];
        }
    }
}

template <bool DENSE, int op>
__global__ void __launch_bounds__(NT) moment_kernel(const float *map, int64_t h, int64_t w, int64_t ld, int64_t is,
                                                    int items, const double *center, float p, float r,
                                                    const float *aux, double2 *partials) {
    __shared__ double red[2 * NT / 32];
    const int img = blockIdx.y;
    const float *m = map + img * is;
    const float *ax = aux ? aux + img * is : nullptr;
    float c = 0.f;
    if (center) {
        // the largest float not above the (double) centre: for float q,
        // q <= c holds exactly when q <= centre does (percentile pooling's test)
        const double cd = center[img];
        c = (float)cd;
        if ((double)c > cd) c = nextafterf(c, -INFINITY);
    }
    KSumP sa, sb;
    for_item<DENSE>(m, op == M_LW ? ax : nullptr, h, w, ld, blockIdx.x, [&](float q, float mu) {
        float a, b;
        contrib<op>(q, c, p, r, mu, a, b);
        sa.add(a);
        if constexpr (has_b(op)) sb.add(b);
    });
    double da = (double)sa.get(), db = (double)sb.get();
    block_sum2d(da, db, red);
    if (threadIdx.x == 0) partials[(int64_t)img * items + blockIdx.x] = make_double2(da, db);
}

// One thread per image: fixed-order sum of the image's partials.
__device__ __forceinline__ double2 image_sum(const double2 *partials, int items, int img) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < items; ++i) {
        const double2 v = partials[(int64_t)img * items + i];
        a += v.x;
        b += v.y;
    }
    return make_double2(a, b);
}

// Finish a moment kind.  stage 0 writes the mean into `center` (kinds that
// need a second pass); stage 1 writes the result.
__global__ void moment_finalize_kernel(const double2 *partials, int items, int count, double n, int kind,
                                       double p, double o, int stage, double *center, double *out) {
    const int img = blockIdx.x * blockDim.x + threadIdx.x;
    if (img >= count) return;
    const double2 s = image_sum(partials, items, img);
    if (stage == 0) {
        center[img] = s.x / n;
        return;
    }
    double v;
    switch (kind) {
    case GBSSIM_POOL_MEAN: v = s.x / n; break;
    case GBSSIM_POOL_COV: v = sqrt(s.x / n) / center[img]; break;
    case GBSSIM_POOL_MINKOWSKI: v = s.x / n; break;
    case GBSSIM_POOL_DW: v = s.x / s.y; break;
    case GBSSIM_POOL_MD: v = pow(pow(s.x / n, 1.0 / p), o); break;
    case GBSSIM_POOL_GM_DSSIM: v = s.y > 0.0 ? 0.0 : exp(s.x / n); break;
    case GBSSIM_POOL_HM_DSSIM: v = s.y > 0.0 ? 0.0 : n / s.x; break;
    default: v = s.x / n; break;  // GBSSIM_POOL_PP
    }
    out[img] = v;
}

// ------------------------------------------------------------------ radix select

struct SelState {
    unsigned prefix[kPoolMaxRanks];  // key bits fixed so far (high bits), per wanted rank
    unsigned rank[kPoolMaxRanks];    // rank still to find inside the bucket
    unsigned uprefix[kPoolMaxRanks]; // the distinct prefixes; each value matches at most one
    int slot[kPoolMaxRanks];         // wanted rank -> its prefix's histogram slot
    int nt, nu;
    int skip;                        // 1: the value-bin path found every key (prefix = the full key)
};

// Value-bin selection (the first path tried): the map's min and max, a
// histogram of VB equal-width value bins over [min, max], the bins that hold
// the wanted ranks, a gather of those bins' values (at most `cap` per image
// together), and an exact select among them.  mode 1: non-finite values,
// or more candidates than `cap` -- the radix passes select that image.
constexpr int VB = 4096;
struct FastSel {
    unsigned kmin, kmax;               // keys of the image's min and max
    int mode, nslot;                   // 0 value-bin path, 1 radix passes; distinct wanted bins
    int bin[kPoolMaxRanks];            // wanted rank -> its bin
    int slot[kPoolMaxRanks];           // wanted rank -> its bin's slot
    unsigned below[kPoolMaxRanks];     // values in the bins before it
    int sbin[kPoolMaxRanks];           // slot -> bin
    unsigned soff[kPoolMaxRanks + 1];  // slot -> first candidate in the image's buffer
    unsigned scnt[kPoolMaxRanks];      // slot -> candidates gathered so far
};
// Candidates kept per image: all wanted bins of an image together.
__host__ __device__ inline int64_t vcap(int64_t n) { return n < 65536 ? n : 65536; }

// Rebuild the distinct-prefix table after the prefixes changed.
__device__ void unique_prefixes(SelState &s) {
    s.nu = 0;
    for (int t = 0; t < s.nt; ++t) {
        int u = 0;
        while (u < s.nu && s.uprefix[u] != s.prefix[t]) ++u;
        if (u == s.nu) s.uprefix[s.nu++] = s.prefix[t];
        s.slot[t] = u;
    }
}

// Pass q (0..3) counts key bits 31-8q .. 24-8q of the values whose higher
// 8q bits equal one of the distinct wanted prefixes (pass 0: of all values,
// into slot 0).  Each thread keeps a run-length count of its last (slot, bin)
// and only adds to shared memory when the bin changes: neighbouring SSIM
// values mostly share a bin, so few shared atomics contend.
// The histogram passes take SEL_SCALE times the moment passes' chunks: every
// CTA adds its nonzero bins (up to kPoolMaxRanks x 256) to the image's global
// histogram with atomics, so fewer, longer CTAs contend less.
constexpr int SEL_SCALE = 1;
template <bool DENSE>
__global__ void __launch_bounds__(NT) select_hist_kernel(const float *map, int64_t h, int64_t w, int64_t ld,
                                                         int64_t is, int pass, const SelState *st,
                                                         unsigned *hist) {
    __shared__ unsigned sh[kPoolMaxRanks][NBIN];
    __shared__ unsigned up[kPoolMaxRanks];
    __shared__ unsigned lowmask[NBIN / 32], prange[2];  // quick rejection of values in no wanted bucket
    const int img = blockIdx.y;
    if (st[img].skip) return;  // the value-bin path has the keys (uniform over the CTA)
    const int nu = pass == 0 ? 1 : st[img].nu;
    for (int i = threadIdx.x; i < nu * NBIN; i += NT) (&sh[0][0])[i] = 0u;
    if (threadIdx.x < nu) up[threadIdx.x] = pass == 0 ? 0u : st[img].uprefix[threadIdx.x];
    if (threadIdx.x == 0) {
        // the prefixes' range and the set of their last bytes: a value whose
        // high bits fall outside the range, or whose last prefix byte no
        // prefix has, matches no prefix (most values after pass 1)
        unsigned lo = 0xffffffffu, hi = 0u, mk[NBIN / 32] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        for (int u = 0; u < nu; ++u) {
            const unsigned v = pass == 0 ? 0u : st[img].uprefix[u];
            lo = min(lo, v);
            hi = max(hi, v);
            mk[(v & 255u) >> 5] |= 1u << (v & 31u);
        }
        for (int k = 0; k < NBIN / 32; ++k) lowmask[k] = mk[k];
        prange[0] = lo;
        prange[1] = hi;
    }
    __syncthreads();
    const unsigned plo = prange[0], phi = prange[1];
    unsigned upr[kPoolMaxRanks];  // the prefixes in registers: a branch-free slot search
#pragma unroll
    for (int u = 0; u < kPoolMaxRanks; ++u) upr[u] = u < nu ? up[u] : 0xffffffffu;
    const float *m = map + img * is;
    const int fixed = 32 - 8 * pass;  // bits above `fixed` are already known
    unsigned run_key = 0xffffffffu, run_n = 0u;  // (slot << 8 | bin) of the current run
    auto count = [&](unsigned key) {
        if (key == run_key) {
            ++run_n;
        } else {
            if (run_n) atomicAdd(&(&sh[0][0])[run_key], run_n);
            run_key = key;
            run_n = 1u;
        }
    };
    for_item<DENSE, CHK * SEL_SCALE>(m, nullptr, h, w, ld, blockIdx.x, [&](float q, float) {
        const unsigned key = f2key(q);
        const unsigned bin = (key >> (fixed - 8)) & (NBIN - 1);
        if (pass == 0) {
            count(bin);
        } else {
            const unsigned hb = key >> fixed;
            if (hb < plo || hb > phi) return;
            int slot = -1;  // distinct prefixes: at most one matches
            if (nu <= 2) {  // a percentile, a median, percentile pooling
                slot = hb == upr[0] ? 0 : (hb == upr[1] ? 1 : -1);
            } else {
#pragma unroll
                for (int u = 0; u < kPoolMaxRanks; ++u) slot = hb == upr[u] ? u : slot;
            }
            if (slot >= 0) count(((unsigned)slot << 8) | bin);
        }
    });
    if (run_n) atomicAdd(&(&sh[0][0])[run_key], run_n);
    __syncthreads();
    unsigned *hi = hist + (int64_t)img * kPoolMaxRanks * NBIN;
    for (int i = threadIdx.x; i < nu * NBIN; i += NT) {
        const unsigned v = (&sh[0][0])[i];
        if (v) atomicAdd(&hi[i], v);
    }
}

// One CTA per image, one warp per wanted rank: find the bin of the rank's
// histogram that holds it with a warp scan (each lane sums 8 consecutive
// bins, an inclusive scan over the lanes finds the lane, a walk over its 8
// bins the bin), then extend the prefix by that bin and keep the rank within
// it.  The warp reads its histogram in parallel, once.
constexpr int STEP_T = 32 * kPoolMaxRanks;
__global__ void __launch_bounds__(STEP_T) select_step_kernel(SelState *st, const unsigned *hist, int pass) {
    const int img = blockIdx.x;
    SelState &s = st[img];
    if (s.skip) return;  // uniform over the CTA
    const unsigned *hi = hist + (int64_t)img * kPoolMaxRanks * NBIN;
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t < s.nt) {
        const unsigned *hb = hi + (pass == 0 ? 0 : s.slot[t] * NBIN);
        const unsigned want = s.rank[t];
        constexpr int PER = NBIN / 32;  // 8 bins per lane
        unsigned c[PER], tot = 0u;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            c[k] = hb[lane * PER + k];
            tot += c[k];
        }
        unsigned inc = tot;  // inclusive scan of the lane totals
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const unsigned exc = inc - tot;
        // the lane whose bins hold the rank (the last lane if the counts fall short)
        const unsigned ballot = __ballot_sync(0xffffffffu, inc > want);
        const int L = ballot ? __ffs(ballot) - 1 : 31;
        if (lane == L) {
            unsigned acc = exc;
            int b = 0;
            for (; b < PER - 1; ++b) {
                if (acc + c[b] > want) break;
                acc += c[b];
            }
            const unsigned bin = (unsigned)(L * PER + b);
            s.prefix[t] = pass == 0 ? bin : (s.prefix[t] << 8) | bin;
            s.rank[t] = want - acc;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) unique_prefixes(s);
}

// bin(v) = min(VB - 1, int((v - lo) * inv)) over [lo, hi] = [min, max]: the
// same fp32 steps in every kernel (explicit roundings, no contraction), so a
// value falls in the same bin each time, and bins are monotone in v.
// False when min or max is not finite or the width is not usable.
__device__ __forceinline__ bool vrange(const FastSel &f, float &lo, float &inv) {
    lo = key2f(f.kmin);
    const float hi = key2f(f.kmax);
    if (!isfinite(lo) || !isfinite(hi)) return false;
    inv = hi > lo ? __fdiv_rn((float)VB, __fsub_rn(hi, lo)) : 0.f;
    return isfinite(inv);
}
__device__ __forceinline__ int vbin(float v, float lo, float inv) {
    const float t = __fmul_rn(__fsub_rn(v, lo), inv);
    return t >= (float)(VB - 1) ? VB - 1 : (int)t;  // t >= 0: lo is the minimum
}

// Pass M: the keys of each image's minimum and maximum (order-preserving
// keys: NaN sorts outside +-inf and turns the image over to the radix path).
template <bool DENSE>
__global__ void __launch_bounds__(NT) vminmax_kernel(const float *map, int64_t h, int64_t w, int64_t ld, int64_t is,
                                                     FastSel *fs) {
    __shared__ unsigned smn[NT / 32], smx[NT / 32];
    const int img = blockIdx.y;
    unsigned mn = 0xffffffffu, mx = 0u;
    for_item<DENSE, CHK * SEL_SCALE>(map + img * is, nullptr, h, w, ld, blockIdx.x, [&](float q, float) {
        const unsigned k = f2key(q);
        mn = min(mn, k);
        mx = max(mx, k);
    });
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        smn[warp] = mn;
        smx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < NT / 32; ++k) {
            mn = min(mn, smn[k]);
            mx = max(mx, smx[k]);
        }
        atomicMin(&fs[img].kmin, mn);
        atomicMax(&fs[img].kmax, mx);
    }
}

// Pass H: per-CTA counts of the VB value bins (run-length aggregated, as in
// the radix passes), added to the image's histogram.
template <bool DENSE>
__global__ void __launch_bounds__(NT) vhist_kernel(const float *map, int64_t h, int64_t w, int64_t ld, int64_t is,
                                                   const FastSel *fs, unsigned *vh) {
    __shared__ unsigned sh[VB];
    const int img = blockIdx.y;
    float lo, inv;
    if (!vrange(fs[img], lo, inv)) return;  // uniform over the CTA
    for (int i = threadIdx.x; i < VB; i += NT) sh[i] = 0u;
    __syncthreads();
    int run_bin = -1;
    unsigned run_n = 0u;
    for_item<DENSE, CHK * SEL_SCALE>(map + img * is, nullptr, h, w, ld, blockIdx.x, [&](float q, float) {
        const int b = vbin(q, lo, inv);
        if (b == run_bin) {
            ++run_n;
        } else {
            if (run_n) atomicAdd(&sh[run_bin], run_n);
            run_bin = b;
            run_n = 1u;
        }
    });
    if (run_n) atomicAdd(&sh[run_bin], run_n);
    __syncthreads();
    unsigned *hi = vh + (int64_t)img * VB;
    for (int i = threadIdx.x; i < VB; i += NT) {
        const unsigned v = sh[i];
        if (v) atomicAdd(&hi[i], v);
    }
}

// Step: one CTA of VSTEP_T threads per image.  Prefix sums over the bins
// find each wanted rank's bin and the count below it; the distinct bins get
// slots and buffer ranges; mode 1 when the bins hold more than `cap` values
// together (or the range is unusable).  With mode 0 the radix passes skip
// the image.
constexpr int VSTEP_T = 1024, VPER = VB / VSTEP_T;
__global__ void __launch_bounds__(VSTEP_T) vstep_kernel(SelState *st, FastSel *fs, const unsigned *vh, int64_t cap) {
    __shared__ unsigned part[VSTEP_T];  // exclusive prefix of each thread's VPER bins
    __shared__ unsigned wsum[VSTEP_T / 32];
    const int img = blockIdx.x;
    FastSel &f = fs[img];
    float lo, inv;
    const bool ok = vrange(f, lo, inv);
    if (!ok) {  // uniform over the CTA
        if (threadIdx.x == 0) f.mode = 1;
        return;
    }
    const unsigned *hb = vh + (int64_t)img * VB;
    unsigned c[VPER], tot = 0u;
#pragma unroll
    for (int k = 0; k < VPER; ++k) {
        c[k] = hb[threadIdx.x * VPER + k];
        tot += c[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned v = wsum[lane], x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        wsum[lane] = x - v;  // exclusive over the warps
    }
    __syncthreads();
    part[threadIdx.x] = wsum[warp] + inc - tot;
    __syncthreads();
    const SelState &s = st[img];
    if (threadIdx.x < s.nt) {
        const int t = threadIdx.x;
        const unsigned want = s.rank[t];
        // the last thread whose exclusive prefix is <= want holds the rank
        int a = 0, b = VSTEP_T - 1;
        while (a < b) {
            const int m = (a + b + 1) >> 1;
            if (part[m] <= want) a = m;
            else b = m - 1;
        }
        unsigned acc = part[a];
        int bin = a * VPER;
        for (int k = 0; k < VPER - 1; ++k, ++bin) {
            const unsigned v = hb[bin];
            if (acc + v > want) break;
            acc += v;
        }
        f.bin[t] = bin;
        f.below[t] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ns = 0;
        unsigned off = 0u;
        for (int t = 0; t < s.nt; ++t) {
            int u = 0;
            while (u < ns && f.sbin[u] != f.bin[t]) ++u;
            if (u == ns) {
                f.sbin[ns] = f.bin[t];
                f.soff[ns] = off;
                off += hb[f.bin[t]];
                f.scnt[ns] = 0u;
                ++ns;
            }
            f.slot[t] = u;
        }
        f.soff[ns] = off;
        f.nslot = ns;
        f.mode = (int64_t)off <= cap ? 0 : 1;
        st[img].skip = f.mode == 0 ? 1 : 0;
    }
}

// Pass G: the values of the wanted bins into the image's candidate buffer
// (warp-aggregated slot counters; the order within a slot is arbitrary, the
// select below does not depend on it).
template <bool DENSE>
__global__ void __launch_bounds__(NT) vgather_kernel(const float *map, int64_t h, int64_t w, int64_t ld, int64_t is,
                                                     FastSel *fs, float *cand, int64_t cap) {
    __shared__ signed char slot_of[VB];
    __shared__ unsigned soff[kPoolMaxRanks + 1];
    const int img = blockIdx.y;
    FastSel &f = fs[img];
    float lo, inv;
    if (f.mode != 0 || !vrange(f, lo, inv)) return;  // uniform over the CTA
    for (int i = threadIdx.x; i < VB; i += NT) slot_of[i] = -1;
    __syncthreads();
    const int ns = f.nslot;
    if (threadIdx.x < ns) slot_of[f.sbin[threadIdx.x]] = (signed char)threadIdx.x;
    if (threadIdx.x <= ns) soff[threadIdx.x] = f.soff[threadIdx.x];
    __syncthreads();
    float *cb = cand + (int64_t)img * cap;
    const int lane = threadIdx.x & 31;
    // append the hits of one value per lane: one counter update per
    // distinct slot among the lanes of `am` that hit
    auto append = [&](unsigned am, int sl, float q) {
        unsigned pending = __ballot_sync(am, sl >= 0);
        while (pending) {
            const int leader = __ffs(pending) - 1;
            const int s0 = __shfl_sync(am, sl, leader);
            const unsigned peers = __ballot_sync(am, sl == s0);
            unsigned base = 0u;
            if (lane == leader) base = atomicAdd(&f.scnt[s0], (unsigned)__popc(peers));
            base = __shfl_sync(am, base, leader);
            if (sl == s0) {
                const unsigned idx = soff[s0] + base + (unsigned)__popc(peers & ((1u << lane) - 1u));
                if (idx < soff[s0 + 1]) cb[idx] = q;  // never more than the bin's count
            }
            pending &= ~peers;
        }
    };
    for_item<DENSE, CHK * SEL_SCALE>(map + img * is, nullptr, h, w, ld, blockIdx.x, [&](float q, float) {
        append(__activemask(), slot_of[vbin(q, lo, inv)], q);
    });
}

// Exact select among one bin's candidates: one CTA per (image, wanted
// rank); four 8-bit radix steps over the candidates' keys with run-length
// aggregated shared counts.  The key goes to the rank's prefix, where the
// radix path would leave it.
constexpr int VSEL_T = 1024;
__global__ void __launch_bounds__(VSEL_T) vselect_kernel(SelState *st, const FastSel *fs, const float *cand,
                                                         int64_t cap) {
    __shared__ unsigned hs[NBIN];
    __shared__ unsigned s_prefix, s_want;
    const int img = blockIdx.x, t = blockIdx.y;
    const FastSel &f = fs[img];
    if (f.mode != 0 || t >= st[img].nt) return;  // uniform over the CTA
    const int sl = f.slot[t];
    const float *cb = cand + (int64_t)img * cap + f.soff[sl];
    const int c = (int)(f.soff[sl + 1] - f.soff[sl]);
    if (threadIdx.x == 0) {
        s_prefix = 0u;
        s_want = st[img].rank[t] - f.below[t];
    }
    unsigned mask = 0u;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int i = threadIdx.x; i < NBIN; i += VSEL_T) hs[i] = 0u;
        __syncthreads();
        const unsigned prefix = s_prefix;
        int run_bin = -1;
        unsigned run_n = 0u;
        for (int i = threadIdx.x; i < c; i += VSEL_T) {
            const unsigned k = f2key(cb[i]);
            if ((k & mask) != prefix) continue;
            const int b = (int)((k >> shift) & 255u);
            if (b == run_bin) {
                ++run_n;
            } else {
                if (run_n) atomicAdd(&hs[run_bin], run_n);
                run_bin = b;
                run_n = 1u;
            }
        }
        if (run_n) atomicAdd(&hs[run_bin], run_n);
        __syncthreads();
        if (threadIdx.x < 32) {  // warp scan: 8 bins a lane
            const int lane = threadIdx.x;
            unsigned c[NBIN / 32], tot = 0u;
#pragma unroll
            for (int k = 0; k < NBIN / 32; ++k) {
                c[k] = hs[lane * (NBIN / 32) + k];
                tot += c[k];
            }
            unsigned inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            const unsigned want = s_want;
            const unsigned ballot = __ballot_sync(0xffffffffu, inc > want);
            const int L = ballot ? __ffs(ballot) - 1 : 31;
            if (lane == L) {
                unsigned acc = inc - tot;
                int b = 0;
                for (; b < NBIN / 32 - 1; ++b) {
                    if (acc + c[b] > want) break;
                    acc += c[b];
                }
                s_prefix = prefix | ((unsigned)(L * (NBIN / 32) + b) << shift);
                s_want = want - acc;
            }
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    if (threadIdx.x == 0) st[img].prefix[t] = s_prefix;
}

// Ranks of the order statistics a percentile needs: floor(h) and floor(h)+1
// (clamped), h = p/100 (n-1).
__host__ __device__ inline void pct_ranks(double p, double n, unsigned &lo, unsigned &hi, double &frac) {
    const double hh = p / 100.0 * (n - 1.0);
    const double fl = floor(hh);
    lo = (unsigned)fl;
    hi = (unsigned)fmin(fl + 1.0, n - 1.0);
    frac = hh - fl;
}

__global__ void select_init_kernel(SelState *st, FastSel *fs, int count, double n, int kind, double parg) {
    const int img = blockIdx.x * blockDim.x + threadIdx.x;
    if (img >= count) return;
    SelState s;
    double ps[5];
    int np = 0;
    if (kind == GBSSIM_POOL_FNS) {
        ps[0] = 0.0; ps[1] = 25.0; ps[2] = 50.0; ps[3] = 75.0; ps[4] = 100.0;
        np = 5;
    } else {
        ps[0] = kind == GBSSIM_POOL_MEDIAN ? 50.0 : parg;
        np = 1;
    }
    s.nt = 2 * np;
    for (int i = 0; i < np; ++i) {
        unsigned lo, hi;
        double f;
        pct_ranks(ps[i], n, lo, hi, f);
        s.rank[2 * i] = lo;
        s.rank[2 * i + 1] = hi;
        s.prefix[2 * i] = s.prefix[2 * i + 1] = 0u;
    }
    unique_prefixes(s);
    s.skip = 0;
    st[img] = s;
    FastSel z;
    memset(&z, 0, sizeof z);
    z.kmin = 0xffffffffu;
    fs[img] = z;
}

// Values of the selected order statistics -> percentile interpolation.
// For PP the threshold goes to `center` (stage 0), else the result to `out`.
__global__ void select_finalize_kernel(const SelState *st, int count, double n, int kind, double parg,
                                       double *center, double *out) {
    const int img = blockIdx.x * blockDim.x + threadIdx.x;
    if (img >= count) return;
    const SelState s = st[img];
    auto pct = [&](int i, double p) {
        unsigned lo, hi;
        double f;
        pct_ranks(p, n, lo, hi, f);
        const double a = (double)key2f(s.prefix[2 * i]), b = (double)key2f(s.prefix[2 * i + 1]);
        return a + f * (b - a);
    };
    if (kind == GBSSIM_POOL_FNS) {
        out[img] = (pct(0, 0.0) + pct(1, 25.0) + pct(2, 50.0) + pct(3, 75.0) + pct(4, 100.0)) / 5.0;
    } else if (kind == GBSSIM_POOL_PP) {
        center[img] = pct(0, parg);
    } else {
        out[img] = pct(0, kind == GBSSIM_POOL_MEDIAN ? 50.0 : parg);
    }
}

// Window-weighted local mean of one image per output (Eq. local_means):
// sum_m g_m sum_n g_n x(i s + m, j s + n), the separable weights in fp32.
template <typename T>
__global__ void local_mean_kernel(ImgDesc x, TapsDyn taps, int k, int s, float *out, int64_t out_ld,
                                  int64_t out_is) {
    const int64_t oh = (x.H - k) / s + 1, ow = (x.W - k) / s + 1;
    const int img = blockIdx.z;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= ow || i >= oh) return;
    const T *b = static_cast<const T *>(x.data) + img * x.image_stride + i * s * x.row_stride + j * s;
    float acc = 0.f;
    for (int m = 0; m < k; ++m) {
        float hsum = 0.f;
        for (int n = 0; n < k; ++n) hsum = fmaf(taps.g[n], load_f32<T>(b + m * x.row_stride + n), hsum);
        acc = fmaf(taps.g[m], hsum, acc);
    }
    out[img * out_is + i * out_ld + j] = acc;
}

}  // namespace

cudaError_t launch_local_mean(const ImgDesc &x, int dtype, int count, const TapsDyn &taps, int k, int s, float *out,
                              int64_t out_ld, int64_t out_is, cudaStream_t st) {
    const int64_t oh = (x.H - k) / s + 1, ow = (x.W - k) / s + 1;
    const dim3 grid((unsigned)((ow + 127) / 128), (unsigned)oh, count);
    switch (dtype) {
    case GBSSIM_U8: local_mean_kernel<uint8_t><<<grid, 128, 0, st>>>(x, taps, k, s, out, out_ld, out_is); break;
    case GBSSIM_F16: local_mean_kernel<__half><<<grid, 128, 0, st>>>(x, taps, k, s, out, out_ld, out_is); break;
    case GBSSIM_BF16: local_mean_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(x, taps, k, s, out, out_ld, out_is); break;
    case GBSSIM_F32: local_mean_kernel<float><<<grid, 128, 0, st>>>(x, taps, k, s, out, out_ld, out_is); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Workspace: partials, per-image centre, selection state, histograms.
PoolLayout pool_layout(int64_t h, int64_t w, int count) {
    PoolLayout L;
    // partial slots for either item form (PR rows, or CHK flat elements)
    L.items = (int)max((h + PR - 1) / PR, (h * w + CHK - 1) / CHK);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    };
    L.partials = take(sizeof(double2) * (size_t)L.items * count);
    L.center = take(sizeof(double) * (size_t)count);
    L.state = take(sizeof(SelState) * (size_t)count);
    L.hist = take(sizeof(unsigned) * (size_t)kPoolMaxRanks * NBIN * count);
    L.fast = take(sizeof(FastSel) * (size_t)count);
    L.vhist = take(sizeof(unsigned) * (size_t)VB * count);
    L.cand = take(sizeof(float) * (size_t)vcap(h * w) * count);
    L.bytes = off;
    return L;
}

cudaError_t launch_pool_map(const float *map, int64_t h, int64_t w, int64_t ld, int count, int64_t is, int kind,
                            double a0, double a1, char *ws, double *out, cudaStream_t st, const float *aux) {
    const PoolLayout L = pool_layout(h, w, count);
    double2 *part = reinterpret_cast<double2 *>(ws + L.partials);
    double *center = reinterpret_cast<double *>(ws + L.center);
    SelState *sel = reinterpret_cast<SelState *>(ws + L.state);
    unsigned *hist = reinterpret_cast<unsigned *>(ws + L.hist);
    FastSel *fsel = reinterpret_cast<FastSel *>(ws + L.fast);
    unsigned *vh = reinterpret_cast<unsigned *>(ws + L.vhist);
    float *cand = reinterpret_cast<float *>(ws + L.cand);
    const int64_t cap = vcap(h * w);
    const double n = (double)h * (double)w;
    // dense maps (and mu_1 maps) with 16-byte aligned images: flat chunks
    const bool dense = ld == w && (uintptr_t)map % 16 == 0 && (count == 1 || is % 4 == 0) &&
                       (!aux || (uintptr_t)aux % 16 == 0);
    const int items = dense ? (int)((h * w + CHK - 1) / CHK) : (int)((h + PR - 1) / PR);
    const dim3 grid(items, count);
    const int64_t sel_chk = CHK * SEL_SCALE, sel_rows = (int64_t)PR * SEL_SCALE;
    const dim3 sel_grid(dense ? (int)((h * w + sel_chk - 1) / sel_chk) : (int)((h + sel_rows - 1) / sel_rows), count);
    const int fb = (count + 127) / 128;
    cudaError_t e = cudaSuccess;
    auto moment = [&](int op, const double *c, double p, double r, int kindv, int stage) {
        const float pf = (float)p, rf = (float)r;
#define GBSSIM_MOMENT(OP)                                                                                           \
    case OP:                                                                                                        \
        if (dense)                                                                                                  \
            moment_kernel<true, OP><<<grid, NT, 0, st>>>(map, h, w, ld, is, items, c, pf, rf, aux, part);          \
        else                                                                                                        \
            moment_kernel<false, OP><<<grid, NT, 0, st>>>(map, h, w, ld, is, items, c, pf, rf, aux, part);         \
        break;
        switch (op) {
            GBSSIM_MOMENT(M_SUM)
            GBSSIM_MOMENT(M_SQDEV)
            GBSSIM_MOMENT(M_ABSDEV_P)
            GBSSIM_MOMENT(M_MINK)
            GBSSIM_MOMENT(M_DW)
            GBSSIM_MOMENT(M_LOG_D)
            GBSSIM_MOMENT(M_INV_D)
            GBSSIM_MOMENT(M_PP)
            GBSSIM_MOMENT(M_LW)
        default: return cudaErrorInvalidValue;
        }
#undef GBSSIM_MOMENT
        moment_finalize_kernel<<<fb, 128, 0, st>>>(part, items, count, n, kindv, p, a1, stage, center, out);
        return cudaGetLastError();
    };
    auto select = [&](double parg) {
        select_init_kernel<<<fb, 128, 0, st>>>(sel, fsel, count, n, kind, parg);
        // value bins first: min / max, bin counts, the wanted bins' values,
        // an exact select among them; images it cannot take (non-finite
        // values, crowded bins) go through the radix passes below, which
        // skip the others
        cudaError_t r = cudaMemsetAsync(vh, 0, sizeof(unsigned) * (size_t)VB * count, st);
        if (r != cudaSuccess) return r;
        if (dense) {
            vminmax_kernel<true><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, fsel);
            vhist_kernel<true><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, fsel, vh);
        } else {
            vminmax_kernel<false><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, fsel);
            vhist_kernel<false><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, fsel, vh);
        }
        vstep_kernel<<<count, VSTEP_T, 0, st>>>(sel, fsel, vh, cap);
        if (dense)
            vgather_kernel<true><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, fsel, cand, cap);
        else
            vgather_kernel<false><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, fsel, cand, cap);
        vselect_kernel<<<dim3(count, kPoolMaxRanks), VSEL_T, 0, st>>>(sel, fsel, cand, cap);
        for (int pass = 0; pass < 4; ++pass) {
            r = cudaMemsetAsync(hist, 0, sizeof(unsigned) * (size_t)kPoolMaxRanks * NBIN * count, st);
            if (r != cudaSuccess) return r;
            if (dense)
                select_hist_kernel<true><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, pass, sel, hist);
            else
                select_hist_kernel<false><<<sel_grid, NT, 0, st>>>(map, h, w, ld, is, pass, sel, hist);
            select_step_kernel<<<count, STEP_T, 0, st>>>(sel, hist, pass);
        }
        select_finalize_kernel<<<fb, 128, 0, st>>>(sel, count, n, kind, parg, center, out);
        return cudaGetLastError();
    };
    switch (kind) {
    case GBSSIM_POOL_MEAN: e = moment(M_SUM, nullptr, 0, 0, kind, 1); break;
    case GBSSIM_POOL_COV:
        e = moment(M_SUM, nullptr, 0, 0, kind, 0);
        if (e == cudaSuccess) e = moment(M_SQDEV, center, 0, 0, kind, 1);
        break;
    case GBSSIM_POOL_MD:
        e = moment(M_SUM, nullptr, 0, 0, kind, 0);
        if (e == cudaSuccess) e = moment(M_ABSDEV_P, center, a0, 0, kind, 1);
        break;
    case GBSSIM_POOL_MINKOWSKI: e = moment(M_MINK, nullptr, a0, 0, kind, 1); break;
    case GBSSIM_POOL_DW: e = moment(M_DW, nullptr, a0, 0, kind, 1); break;
    case GBSSIM_POOL_GM_DSSIM: e = moment(M_LOG_D, nullptr, 0, 0, kind, 1); break;
    case GBSSIM_POOL_HM_DSSIM: e = moment(M_INV_D, nullptr, 0, 0, kind, 1); break;
    case GBSSIM_POOL_PERCENTILE:
    case GBSSIM_POOL_MEDIAN:
    case GBSSIM_POOL_FNS: e = select(a0); break;
    case GBSSIM_POOL_PP:
        e = select(a0);
        if (e == cudaSuccess) e = moment(M_PP, center, 0, a1, kind, 1);
        break;
    case kPoolLW: e = moment(M_LW, nullptr, a0, a1, kind, 1); break;  // sum w(mu) Q / n
    default: e = cudaErrorInvalidValue;
    }
    return e;
}

}  // namespace gbssim
