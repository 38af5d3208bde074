// api.cu -- the extern "C" boundary of libgbssim.so (declared in
// include/gbssim.h): argument validation, workspace layout and kernel
// dispatch.  No function here allocates device memory or synchronises.
#include <math.h>
#include <string.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

using namespace gbssim;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

const double kDefaultExps[5] = {0.0448, 0.2856, 0.3001, 0.2363, 0.1333};

int check_plane(const gbssim_plane *p) {
    if (!p || !p->data) return GBSSIM_ERR_INVALID_ARG;
    if (p->dtype < GBSSIM_U8 || p->dtype > GBSSIM_F32) return GBSSIM_ERR_INVALID_ARG;
    if (p->count < 1 || p->height < 1 || p->width < 1) return GBSSIM_ERR_INVALID_ARG;
    if (p->row_stride < p->width) return GBSSIM_ERR_INVALID_ARG;
    if (p->count > 1 && p->image_stride < p->height * p->row_stride) return GBSSIM_ERR_INVALID_ARG;
    if (p->count > 65535) return GBSSIM_ERR_UNSUPPORTED;
    return GBSSIM_OK;
}

int check_pair(const gbssim_plane *x, const gbssim_plane *y) {
    int rc = check_plane(x);
    if (rc) return rc;
    rc = check_plane(y);
    if (rc) return rc;
    if (x->dtype != y->dtype || x->count != y->count || x->height != y->height ||
        x->width != y->width || x->row_stride != y->row_stride ||
        (x->count > 1 && x->image_stride != y->image_stride))
        return GBSSIM_ERR_INVALID_ARG;
    return GBSSIM_OK;
}

int check_params(const gbssim_params *p) {
    if (!p) return GBSSIM_ERR_INVALID_ARG;
    if (p->window != GBSSIM_WIN_GAUSSIAN && p->window != GBSSIM_WIN_BOX) return GBSSIM_ERR_INVALID_ARG;
    if (p->k < 1 || p->k > GBSSIM_MAX_K) return GBSSIM_ERR_INVALID_ARG;
    if (p->window == GBSSIM_WIN_GAUSSIAN && !(p->sigma > 0.0 && isfinite(p->sigma)))
        return GBSSIM_ERR_INVALID_ARG;
    if (!(isfinite(p->K1) && isfinite(p->K2) && p->K1 >= 0.0 && p->K2 >= 0.0)) return GBSSIM_ERR_INVALID_ARG;
    if (!(p->L > 0.0 && isfinite(p->L))) return GBSSIM_ERR_INVALID_ARG;
    if (p->stride < 1) return GBSSIM_ERR_INVALID_ARG;
    if (p->scales < 1 || p->scales > GBSSIM_MAX_SCALES) return GBSSIM_ERR_INVALID_ARG;
    for (int j = 0; j < p->scales; ++j)
        if (!isfinite(p->exponents[j])) return GBSSIM_ERR_INVALID_ARG;
    if (p->combine != GBSSIM_COMBINE_PRODUCT && p->combine != GBSSIM_COMBINE_SUM) return GBSSIM_ERR_INVALID_ARG;
    if (p->flags & ~(GBSSIM_FLAG_BOX_TMA | GBSSIM_FLAG_PYRAMID_97 | GBSSIM_FLAG_BORDER_ZERO |
                     GBSSIM_FLAG_BORDER_REFLECT))
        return GBSSIM_ERR_INVALID_ARG;
    if ((p->flags & GBSSIM_FLAG_BORDER_ZERO) && (p->flags & GBSSIM_FLAG_BORDER_REFLECT))
        return GBSSIM_ERR_INVALID_ARG;
    return GBSSIM_OK;
}

// Border extension mode of the params: 0 valid only, 1 zero, 2 mirror.
int border_mode(const gbssim_params *p) {
    if (p->flags & GBSSIM_FLAG_BORDER_ZERO) return 1;
    if (p->flags & GBSSIM_FLAG_BORDER_REFLECT) return 2;
    return 0;
}

// check_params for the entry points that take valid windows only.
int check_params_valid(const gbssim_params *p) {
    const int rc = check_params(p);
    if (rc) return rc;
    return border_mode(p) ? GBSSIM_ERR_UNSUPPORTED : GBSSIM_OK;
}

void make_taps(const gbssim_params *p, float *g) {
    const int k = p->k;
    if (p->window == GBSSIM_WIN_BOX) {
        for (int t = 0; t < k; ++t) g[t] = (float)(1.0 / k);
        return;
    }
    double v[GBSSIM_MAX_K], z = 0.0, c = 0.5 * (k - 1);
    for (int t = 0; t < k; ++t) {
        v[t] = exp(-((t - c) * (t - c)) / (2.0 * p->sigma * p->sigma));
        z += v[t];
    }
    for (int t = 0; t < k; ++t) g[t] = (float)(v[t] / z);
}

SsimConst make_const(const gbssim_params *p) {
    const double c1 = (p->K1 * p->L) * (p->K1 * p->L), c2 = (p->K2 * p->L) * (p->K2 * p->L);
    return ssim_const(c1, c2);
}

ImgDesc desc_of(const gbssim_plane *p) {
    return ImgDesc{p->data, p->height, p->width, p->row_stride,
                   p->count > 1 ? p->image_stride : p->height * p->row_stride};
}

enum Path { PATH_GAUSS11, PATH_GENERIC, PATH_BOX_U8 };

Path pick_path(int dtype, const gbssim_params *p) {
    if (p->window == GBSSIM_WIN_BOX && dtype == GBSSIM_U8) return PATH_BOX_U8;
    if (p->k == 11 && p->stride == 1) return PATH_GAUSS11;
    return PATH_GENERIC;
}

int pick_seg_rows(int64_t H, int64_t W, int count) {
    int strips, segs;
    int seg = 256;
    while (seg > 32) {
        gauss11_items(H, W, seg, &strips, &segs);
        if ((int64_t)strips * segs * count >= 4 * 456) break;
        seg -= 32;
    }
    return seg;
}

// Items (CTAs producing one partial each) per image for one level.
int level_items(Path path, int64_t H, int64_t W, int count, const gbssim_params *p, int *seg_rows) {
    const int64_t OH = out_dim(H, p->k, p->stride), OW = out_dim(W, p->k, p->stride);
    switch (path) {
    case PATH_GAUSS11: {
        int strips, segs;
        *seg_rows = pick_seg_rows(H, W, count);
        return gauss11_items(H, W, *seg_rows, &strips, &segs);
    }
    case PATH_BOX_U8: return box_items_ks(OH, OW, p->k, p->stride);
    default: return generic_items(OH, OW);
    }
}

// Rows per work item of the persistent MS-SSIM path at pyramid level j
// (OH output rows, strips x count items per segment row).  Items are long
// (every item restages its first 26 rows and pays its fetch), but every
// level has at least about four items per CTA of the 152 SMs x 4 CTAs
// (2432) when it has the rows: at 1080p x 64 that splits level 0 in two
// segments and the upper levels in two to five, which keeps the chain of
// dependent items of the last images short at the end of the launch
// (measured: 0.996 ms a launch, against 1.06 with one level-0 item per
// strip and two waves at the upper levels).  Segments are balanced (no
// short remainder item) and a multiple of 16 rows.
// Streamed launches (inputs still arriving) take short items at the two
// large levels: the chain after the last copy lands is the step's tail,
// while the extra halo rows cost time the copies leave idle.
int persistent_seg_rows(int j, bool streamed, int64_t OH, int64_t strips, int count) {
    static const int streamed_rows[5] = {128, 128, 64, 32, 32};
    if (streamed) return j < 5 ? streamed_rows[j] : streamed_rows[4];
    static const int target[5] = {1100, 384, 192, 96, 48};
    const int64_t t = j < 5 ? target[j] : target[4];
    int64_t n = (OH + t - 1) / t;
    const int64_t want = 2432, per = strips * (int64_t)count;
    if (n * per < want) {
        const int64_t m = (want + per - 1) / per, cap = (OH + 31) / 32;
        n = m < cap ? m : cap;
        if (n < 1) n = 1;
    }
    int64_t r = (OH + n - 1) / n;
    r = (r + 15) / 16 * 16;
    return (int)(r < 16 ? 16 : r);
}

struct Level {
    int64_t H, W;    // the level's image (pyramid level j)
    int64_t RH, RW;  // the image the SSIM kernel runs on: H x W, or extended by k-1 (border modes)
    Path path;
    int items, seg_rows;
    int pitems, pseg_rows;       // the persistent MS-SSIM path's items per image and rows per item
    size_t part_off, plane_off;  // plane_off: x then y planes of this level (j >= 1)
};

struct MsPlan {
    Level lv[GBSSIM_MAX_SCALES];
    size_t counter_off, done_off, status_off, zero_bytes;  // persistent path counters
    size_t pad_off, pad_plane;                             // border modes: extended x then y (scratch)
    size_t bytes;
};

int plan_levels(const gbssim_plane *x, const gbssim_params *p, int scales, MsPlan *P,
                bool float_path = false, bool streamed = false) {
    size_t off = 0;
    int64_t H = x->height, W = x->width;
    const int border = border_mode(p);
    const int64_t ext = border ? p->k - 1 : 0;
    size_t pad_plane = 0;
    for (int j = 0; j < scales; ++j) {
        if (border ? (H < p->k - 1 - (p->k - 1) / 2 || H < 1 || W < p->k - 1 - (p->k - 1) / 2 || W < 1)
                   : (H < p->k || W < p->k))
            return GBSSIM_ERR_TOO_SMALL;
        Level &L = P->lv[j];
        L.H = H;
        L.W = W;
        L.RH = H + ext;
        L.RW = W + ext;
        const int dtype = j == 0 ? x->dtype : GBSSIM_F32;
        if (border) {
            if (L.RH > 65535) return GBSSIM_ERR_UNSUPPORTED;  // the extension grid's y extent
            const size_t esz = dtype == GBSSIM_U8 ? 1 : (dtype == GBSSIM_F32 ? 4 : 2);
            const size_t plane = esz * (size_t)L.RH * L.RW * x->count;
            if (plane > pad_plane) pad_plane = plane;
        }
        L.path = pick_path(dtype, p);
        if (float_path && L.path == PATH_BOX_U8) L.path = PATH_GENERIC;
        L.seg_rows = 0;
        L.items = level_items(L.path, L.RH, L.RW, x->count, p, &L.seg_rows);
        L.pseg_rows = 0;
        L.pitems = 0;
        if (L.path == PATH_GAUSS11 && !border) {
            L.pseg_rows = persistent_seg_rows(j, streamed, H - 10, uniform_strips(W), x->count);
            L.pitems = uniform_strips(W) * (int)((H - 10 + L.pseg_rows - 1) / L.pseg_rows);
        }
        L.part_off = off;  // pooling slots for whichever layout runs
        off = align_up(off + sizeof(double2) * (size_t)(L.items > L.pitems ? L.items : L.pitems) * x->count);
        if (j > 0) {
            L.plane_off = off;
            off = align_up(off + 2 * sizeof(float) * (size_t)H * W * x->count);
        } else {
            L.plane_off = 0;
        }
        H >>= 1;
        W >>= 1;
    }
    P->counter_off = off;
    P->done_off = off + 16;
    P->status_off = P->done_off + sizeof(unsigned) * (size_t)scales * x->count;
    P->zero_bytes = P->status_off + 16 - P->counter_off;
    off = align_up(P->counter_off + P->zero_bytes);
    P->pad_off = off;
    P->pad_plane = align_up(pad_plane);
    off += 2 * P->pad_plane;
    P->bytes = off;
    return GBSSIM_OK;
}

// The uint8 box path's tile layout (and so its item count) depends on the
// alignment of the actual planes; the plan sized the workspace for the larger.
void fix_box_items(Level &L, const ImgDesc &dx, const ImgDesc &dy, const gbssim_params *p) {
    if (L.path != PATH_BOX_U8) return;
    const int64_t OH = out_dim(L.RH, p->k, p->stride), OW = out_dim(L.RW, p->k, p->stride);
    L.items = box_path_items(OH, OW, p->k, p->stride, box_aligned16(dx, dy), (p->flags & GBSSIM_FLAG_BOX_TMA) != 0);
}

// Border modes: the level's images extended into the plan's scratch (dense
// RH x RW planes of the same dtype); valid mode: the images themselves.
cudaError_t extend_level(const Level &L, const MsPlan &P, char *ws, const gbssim_params *p, int dtype, int count,
                         ImgDesc &dx, ImgDesc &dy, cudaStream_t st) {
    const int border = border_mode(p);
    if (!border) return cudaSuccess;
    const int before = (p->k - 1) / 2;
    char *px = ws + P.pad_off, *py = px + P.pad_plane;
    cudaError_t e = launch_pad(dx, dtype, count, px, L.RH, L.RW, before, before, border - 1, st);
    if (e == cudaSuccess) e = launch_pad(dy, dtype, count, py, L.RH, L.RW, before, before, border - 1, st);
    dx = ImgDesc{px, L.RH, L.RW, L.RW, L.RH * L.RW};
    dy = ImgDesc{py, L.RH, L.RW, L.RW, L.RH * L.RW};
    return e;
}

// Launch one SSIM level: `in_x/in_y` describe the level's images (dtype),
// partials/map as given; ds_x/ds_y (nullable) receive the next level.
cudaError_t run_level(const Level &L, const ImgDesc &dx, const ImgDesc &dy, int dtype, int count,
                      const gbssim_params *p, float *map, int64_t map_ld, int64_t map_is,
                      double2 *partials, float *ds_x, float *ds_y, cudaStream_t st,
                      const CoefOut *co = nullptr) {
    const SsimConst cc = make_const(p);
    CoefOut none;
    none.coef = nullptr;
    none.which = 0;
    none.sx = none.sy = 0.f;
    cudaError_t e = cudaSuccess;
    bool fused_ds = false;
    const bool p97 = (p->flags & GBSSIM_FLAG_PYRAMID_97) != 0;  // the 9/7 pyramid is never fused
    if (p97 && L.path == PATH_GAUSS11 && ds_x) {  // the level alone, then the 9/7 step
        e = run_level(L, dx, dy, dtype, count, p, map, map_ld, map_is, partials, nullptr, nullptr, st, co);
        if (e == cudaSuccess && ds_x) e = launch_pyramid97(dx, dtype, count, ds_x, st);
        if (e == cudaSuccess && ds_y) e = launch_pyramid97(dy, dtype, count, ds_y, st);
        return e;
    }
    if (L.path == PATH_GAUSS11) {
        GaussLaunch G;
        G.x = dx;
        G.y = dy;
        G.dtype = dtype;
        G.count = count;
        G.map = map;
        G.map_ld = map_ld;
        G.map_is = map_is;
        G.ds_x = ds_x;
        G.ds_y = ds_y;
        G.partials = partials;
        make_taps(p, G.taps.g);
        G.c = cc;
        G.seg_rows = L.seg_rows;
        G.co = co ? *co : none;
        e = launch_gauss11(G, st);
        fused_ds = true;
    } else if (L.path == PATH_BOX_U8) {
        BoxLaunch B;
        B.x = dx;
        B.y = dy;
        B.count = count;
        B.k = p->k;
        B.stride = p->stride;
        B.map = map;
        B.map_ld = map_ld;
        B.map_is = map_is;
        B.partials = partials;
        B.sums_out = nullptr;
        B.use_tma = (p->flags & GBSSIM_FLAG_BOX_TMA) != 0;
        const double k4 = pow((double)p->k, 4.0);
        const double c1 = (p->K1 * p->L) * (p->K1 * p->L), c2 = (p->K2 * p->L) * (p->K2 * p->L);
        B.C1k4 = (float)(c1 * k4);
        B.C2k4 = (float)(c2 * k4);
        e = launch_box_u8(B, st);
    } else {
        GenericLaunch G;
        G.x = dx;
        G.y = dy;
        G.dtype = dtype;
        G.count = count;
        G.k = p->k;
        G.stride = p->stride;
        G.map = map;
        G.map_ld = map_ld;
        G.map_is = map_is;
        G.partials = partials;
        memset(G.taps.g, 0, sizeof G.taps.g);
        make_taps(p, G.taps.g);
        G.c = cc;
        G.co = co ? *co : none;
        e = launch_generic(G, st);
    }
    if (e != cudaSuccess) return e;
    if (ds_x && !fused_ds && p97) {
        e = launch_pyramid97(dx, dtype, count, ds_x, st);
        if (e != cudaSuccess) return e;
        e = launch_pyramid97(dy, dtype, count, ds_y, st);
    } else if (ds_x && !fused_ds) {
        e = launch_downsample(dx, dtype, count, ds_x, st);
        if (e != cudaSuccess) return e;
        e = launch_downsample(dy, dtype, count, ds_y, st);
    }
    return e;
}

// MS-SSIM forward over a planned workspace: level kernels (pyramid fused
// where the path allows), then the finaliser.  Shared by gbssim_msssim and
// the MS-SSIM backward.

// arrive (nullable, persistent path only): the images come in `groups` copy
// groups, group g holding images group_begin[g] .. group_begin[g + 1] - 1;
// their level-0 items wait (bounded) until arrive[g] != 0, their bytes being
// copied in on another stream.
int msssim_forward(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                          const MsPlan &P, char *ws, double *score_out, double *per_scale_out,
                          cudaStream_t st, const unsigned *arrive = nullptr, const int *group_begin = nullptr,
                          int groups = 0, unsigned wait_limit = 0, bool int_pyramid = true) {
    const int S = p->scales, n = x->count;
    // the persistent path fuses the 2x2 pyramid into valid-window levels
    bool persistent = (p->flags & GBSSIM_FLAG_PYRAMID_97) == 0 && !border_mode(p);
    for (int j = 0; j < S; ++j) persistent = persistent && P.lv[j].path == PATH_GAUSS11;
    if (arrive && !persistent) return GBSSIM_ERR_UNSUPPORTED;  // only the persistent launch waits for arrivals
    if (persistent) {
        // one launch over all levels and images: level-major items, a level-j
        // item of an image waits (bounded) for that image's level-(j-1) items
        UniformBatch U;
        memset(&U, 0, sizeof U);
        U.x = x->data;
        U.y = y->data;
        U.rs = x->row_stride;
        U.image_stride = desc_of(x).image_stride;
        U.dtype = x->dtype;
        U.count = n;
        U.scales = S;
        // uint8 input: pyramid levels 1..4 as exact uint16 planes (4^j times
        // the level's values, at most 255 x 4^4 = 65280), rows padded to 8
        // elements; they fit the workspace planned for fp32 levels
        U.ipyr = int_pyramid && x->dtype == GBSSIM_U8 && S <= 5;
        // the score pools mean cs below the last level and mean Q at it:
        // without per-scale output the lower levels form cs alone
        U.cs_only_levels = per_scale_out ? 0 : S - 1;
        int64_t begin = 0;
        MsFinalize F;
        memset(&F, 0, sizeof F);
        for (int j = 0; j < S; ++j) {
            const Level &L = P.lv[j];
            UniformLevel &u = U.lv[j];
            u.H = L.H;
            u.W = L.W;
            u.seg_rows = L.pseg_rows;
            u.strips = uniform_strips(L.W);
            u.segs = (int)((L.H - 10 + L.pseg_rows - 1) / L.pseg_rows);
            u.items_per_image = u.strips * u.segs;
            if (u.items_per_image != L.pitems) return GBSSIM_ERR_INVALID_ARG;  // plan and launch disagree
            if (j == 0) {
                const size_t esz = x->dtype == GBSSIM_U8 ? 1 : x->dtype == GBSSIM_F32 ? 4 : 2;
                const uintptr_t vb = 4 * esz;
                u.vec = ((uintptr_t)x->data % vb == 0) && ((uintptr_t)y->data % vb == 0) && (U.rs % 4 == 0) &&
                        (U.image_stride % 4 == 0);
            } else {
                u.pitch = U.ipyr ? (L.W + 7) / 8 * 8 : L.W;
                u.vec = u.pitch % 4 == 0;
            }
            u.item_begin = begin;
            begin += (int64_t)u.items_per_image * n;
            u.x_off = j > 0 ? (int64_t)L.plane_off : -1;
            u.part_off = (int64_t)L.part_off;
            const int64_t OH = L.H - 10, OW = L.W - 10;
            F.lv[j].partials = (const double2 *)(ws + L.part_off);
            F.lv[j].items_per_image = u.items_per_image;
            F.lv[j].inv_n = 1.0 / ((double)OH * (double)OW);
            F.exps[j] = p->exponents[j];
        }
        U.total_items = begin;
        U.ws = ws;
        U.counter_off = (int64_t)P.counter_off;
        U.done_off = (int64_t)P.done_off;
        U.status_off = (int64_t)P.status_off;
        U.wait_limit = wait_limit ? wait_limit : 1u << 22;
        if (begin > 0x7fffffff) return GBSSIM_ERR_UNSUPPORTED;
        U.arrive = arrive;
        if (arrive) {
            // wavefront over copy groups: wave w runs level 0 of group w while
            // the upper levels of earlier groups fill the wait for copies
            const int G = groups;
            if (!group_begin || G < 1 || G > kUniformMaxGroups || group_begin[0] != 0 || group_begin[G] != n)
                return GBSSIM_ERR_INVALID_ARG;
            for (int g = 0; g <= G; ++g) {
                if (g < G && group_begin[g + 1] <= group_begin[g]) return GBSSIM_ERR_INVALID_ARG;
                U.group_begin[g] = group_begin[g];
            }
            U.groups = G;
            U.waves = G + S - 1;
            U.wave_begin[0] = 0;
            int64_t at = 0;
            for (int w = 0; w < U.waves; ++w) {
                for (int j = w - G + 1 > 0 ? w - G + 1 : 0; j <= w && j < S; ++j) {
                    const int g = w - j, m = group_begin[g + 1] - group_begin[g];
                    at += (int64_t)m * U.lv[j].items_per_image;
                }
                U.wave_begin[w + 1] = (int)at;
            }
            if (at != begin) return GBSSIM_ERR_INVALID_ARG;  // the waves cover every item once
        }
        if (cudaMemsetAsync(ws + P.counter_off, 0, P.zero_bytes, st) != cudaSuccess) return GBSSIM_ERR_CUDA;
        Taps<11> taps;
        make_taps(p, taps.g);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = gauss11_batch_max_ctas_per_sm(x->dtype, false);
        if (per_sm < 1) return GBSSIM_ERR_CUDA;
        const int64_t want = (int64_t)sms * per_sm;
        const int grid = (int)(want < begin ? want : begin);
        const cudaError_t le = launch_uniform(U, taps, make_const(p), grid, st);
        if (le == cudaErrorNotSupported) return GBSSIM_ERR_UNSUPPORTED;  // arrival flags without bulk-copy maps
        if (le != cudaSuccess) return GBSSIM_ERR_CUDA;
        F.scales = S;
        F.count = n;
        F.combine = p->combine;
        F.score_out = score_out;
        F.per_scale_out = per_scale_out;
        return launch_finalize_msssim(F, st) == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
    }
    ImgDesc dx = desc_of(x), dy = desc_of(y);
    int dtype = x->dtype;
    MsPlan Pl = P;  // level 0 may take the aligned box layout
    const bool border = border_mode(p) != 0;
    if (!border) fix_box_items(Pl.lv[0], dx, dy, p);
    MsFinalize F;
    memset(&F, 0, sizeof F);
    for (int j = 0; j < S; ++j) {
        Level &L = Pl.lv[j];
        float *ds_x = nullptr, *ds_y = nullptr;
        if (j + 1 < S) {
            const Level &N = Pl.lv[j + 1];
            ds_x = (float *)(ws + N.plane_off);
            ds_y = ds_x + (size_t)N.H * N.W * n;
        }
        double2 *part = (double2 *)(ws + L.part_off);
        cudaError_t e;
        if (border) {
            // the level's SSIM on its extended images; the next level from the unextended ones
            ImgDesc ex = dx, ey = dy;
            e = extend_level(L, P, ws, p, dtype, n, ex, ey, st);
            if (e == cudaSuccess) {
                fix_box_items(L, ex, ey, p);
                e = run_level(L, ex, ey, dtype, n, p, nullptr, 0, 0, part, nullptr, nullptr, st);
            }
            if (e == cudaSuccess && ds_x) {
                const bool p97 = (p->flags & GBSSIM_FLAG_PYRAMID_97) != 0;
                e = p97 ? launch_pyramid97(dx, dtype, n, ds_x, st) : launch_downsample(dx, dtype, n, ds_x, st);
                if (e == cudaSuccess)
                    e = p97 ? launch_pyramid97(dy, dtype, n, ds_y, st) : launch_downsample(dy, dtype, n, ds_y, st);
            }
        } else {
            e = run_level(L, dx, dy, dtype, n, p, nullptr, 0, 0, part, ds_x, ds_y, st);
        }
        if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
        const int64_t OH = out_dim(L.RH, p->k, p->stride), OW = out_dim(L.RW, p->k, p->stride);
        F.lv[j].partials = part;
        F.lv[j].items_per_image = L.items;
        F.lv[j].inv_n = 1.0 / ((double)OH * (double)OW);
        F.exps[j] = p->exponents[j];
        if (j + 1 < S) {
            const Level &N = Pl.lv[j + 1];
            dx = ImgDesc{ds_x, N.H, N.W, N.W, N.H * N.W};
            dy = ImgDesc{ds_y, N.H, N.W, N.W, N.H * N.W};
            dtype = GBSSIM_F32;
        }
    }
    F.scales = S;
    F.count = n;
    F.combine = p->combine;
    F.score_out = score_out;
    F.per_scale_out = per_scale_out;
    return launch_finalize_msssim(F, st) == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}


// Backward workspace: [MS-SSIM forward plan][score][per-scale means]
// [coefficient-pass partials][A, B, C maps of level 0 (reused per level)]
// [float gradients of levels 1..S-1].
struct BwdPlan {
    MsPlan fwd;   // forward plan (multiscale only)
    MsPlan coef;  // per-level items of the coefficient pass (float path)
    size_t score_off, per_off, cpart_off, coef_off, grad_off[GBSSIM_MAX_SCALES];
    size_t bytes;
};

int plan_backward(const gbssim_plane *x, const gbssim_params *p, int multiscale, BwdPlan *B) {
    const int S = multiscale ? p->scales : 1;
    int rc;
    size_t off = 0;
    if (multiscale) {
        rc = plan_levels(x, p, S, &B->fwd);
        if (rc) return rc;
        off = B->fwd.bytes;
    }
    rc = plan_levels(x, p, S, &B->coef, true);
    if (rc) return rc;
    B->score_off = off;
    off = align_up(off + sizeof(double) * x->count);
    B->per_off = off;
    off = align_up(off + 2 * sizeof(double) * S * x->count);
    int max_items = 0;
    for (int j = 0; j < S; ++j) max_items = B->coef.lv[j].items > max_items ? B->coef.lv[j].items : max_items;
    B->cpart_off = off;
    off = align_up(off + sizeof(double2) * (size_t)max_items * x->count);
    const int64_t OH = out_dim(x->height, p->k, 1), OW = out_dim(x->width, p->k, 1);
    B->coef_off = off;
    off = align_up(off + 3 * sizeof(float) * (size_t)OH * coef_ld(OW) * x->count);
    B->grad_off[0] = 0;
    for (int j = 1; j < S; ++j) {
        B->grad_off[j] = off;
        off = align_up(off + sizeof(float) * (size_t)B->coef.lv[j].H * B->coef.lv[j].W * x->count);
    }
    B->bytes = off;
    return GBSSIM_OK;
}

// Saved state of the loss path (gbssim_loss_forward -> gbssim_loss_backward):
// per level the coefficient maps, the pooling partials and (levels >= 1) the
// pyramid planes; the scores and per-scale means; the coarse gradients the
// backward passes down the pyramid.
struct SavedPlan {
    MsPlan lv;  // per-level geometry and items (float path)
    size_t coef_off[GBSSIM_MAX_SCALES], part_off[GBSSIM_MAX_SCALES], plane_off[GBSSIM_MAX_SCALES];
    size_t grad_off[GBSSIM_MAX_SCALES], score_off, per_off, bytes;
};

int plan_saved(const gbssim_plane *x, const gbssim_params *p, int multiscale, SavedPlan *Sv) {
    const int S = multiscale ? p->scales : 1;
    int rc = plan_levels(x, p, S, &Sv->lv, true);
    if (rc) return rc;
    const int n = x->count;
    size_t off = 0;
    for (int j = 0; j < S; ++j) {
        const Level &L = Sv->lv.lv[j];
        const int64_t OH = out_dim(L.H, p->k, 1), OW = out_dim(L.W, p->k, 1);
        Sv->coef_off[j] = off;
        off = align_up(off + 3 * sizeof(float) * (size_t)OH * coef_ld(OW) * n);
        Sv->part_off[j] = off;
        off = align_up(off + sizeof(double2) * (size_t)L.items * n);
        Sv->plane_off[j] = 0;
        Sv->grad_off[j] = 0;
        if (j > 0) {
            Sv->plane_off[j] = off;
            off = align_up(off + 2 * sizeof(float) * (size_t)L.H * L.W * n);
            Sv->grad_off[j] = off;
            off = align_up(off + sizeof(float) * (size_t)L.H * L.W * n);
        }
    }
    Sv->score_off = off;
    off = align_up(off + sizeof(double) * n);
    Sv->per_off = off;
    off = align_up(off + 2 * sizeof(double) * (size_t)S * n);
    Sv->bytes = off;
    return GBSSIM_OK;
}

int check_loss(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p) {
    int rc = check_pair(x, y);
    if (rc) return rc;
    rc = check_params_valid(p);
    if (rc) return rc;
    if (p->stride != 1 || p->k > GBSSIM_MAX_K_BACKWARD) return GBSSIM_ERR_UNSUPPORTED;
    if (p->flags & GBSSIM_FLAG_PYRAMID_97) return GBSSIM_ERR_UNSUPPORTED;
    return GBSSIM_OK;
}

// Host-input MS-SSIM: layout of the device buffer.  Two stages of `per`
// images each (x then y, rows padded to 16 bytes), the MS-SSIM workspace for
// one chunk, and the scores of all images.
struct HostPlan {
    int per, chunks;            // chunks == 0: streamed (one launch, images start as they arrive)
    int64_t pitch_elems;        // device row pitch in elements
    size_t esz, stage_bytes, plane_bytes;
    size_t stage_off[2], ws_off[2], score_off, flags_off, bytes;  // stage s computes in workspace s
    MsPlan ms;                  // for a chunk of `per` images
};

// The persistent MS-SSIM path (the one streamed mode runs) takes these params.
bool persistent_params(const gbssim_params *p) {
    return p->window == GBSSIM_WIN_GAUSSIAN && p->k == 11 && p->stride == 1 &&
           (p->flags & (GBSSIM_FLAG_PYRAMID_97 | GBSSIM_FLAG_BORDER_ZERO | GBSSIM_FLAG_BORDER_REFLECT)) == 0;
}

// cuStreamWriteValue32 through the runtime's driver entry point (nullptr if
// unavailable): the copy stream's arrival flags for the streamed mode.
PFN_cuStreamWriteValue32_v11070 stream_write_value32() {
    static const PFN_cuStreamWriteValue32_v11070 fn = [] {  // looked up once (thread-safe static)
        void *q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &q, 12000, cudaEnableDefault, &r) ==
                cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuStreamWriteValue32_v11070>(q);
        return (PFN_cuStreamWriteValue32_v11070) nullptr;
    }();
    return fn;
}

// Copy groups of the streamed host mode (at most kUniformMaxGroups, each with
// its arrival flag): with 32 images or more the last eight groups hold 4, 4,
// 2, 2, 1, 1, 1, 1 images, so the work left after the last copy lands (that
// group's level-0 items and the chain of its upper levels) is short, and the
// first eight split the rest evenly; with fewer, equal groups of
// ceil(n / 16).  begin[0..G] receives the groups' first images; returns G.
int stream_groups(int n, int *begin) {
    static const int tail[8] = {4, 4, 2, 2, 1, 1, 1, 1};
    int G = 0;
    begin[0] = 0;
    if (n >= 32) {
        const int head = n - 16;
        for (int g = 0; g < 8; ++g, ++G) begin[G + 1] = begin[G] + head / 8 + (g < head % 8 ? 1 : 0);
        for (int g = 0; g < 8; ++g, ++G) begin[G + 1] = begin[G] + tail[g];
    } else {
        const int gs = (n + kUniformMaxGroups - 1) / kUniformMaxGroups;
        for (int i0 = 0; i0 < n; i0 += gs, ++G) begin[G + 1] = i0 + gs < n ? i0 + gs : n;
    }
    return G;
}

int plan_host(const gbssim_plane *x, const gbssim_params *p, int32_t chunks, HostPlan *H) {
    if (chunks < 0) return GBSSIM_ERR_INVALID_ARG;
    const int n = x->count;
    if (chunks == 0) {  // streamed: every image resident at once, a flag per copy group (<= one per image)
        if (!persistent_params(p) || p->scales < 1) return GBSSIM_ERR_UNSUPPORTED;
        H->chunks = 0;
        H->per = n;
        H->esz = x->dtype == GBSSIM_U8 ? 1 : x->dtype == GBSSIM_F32 ? 4 : 2;
        const size_t pitch = ((size_t)x->width * H->esz + 15) / 16 * 16;
        H->pitch_elems = (int64_t)(pitch / H->esz);
        H->plane_bytes = pitch * (size_t)x->height * (size_t)n;
        H->stage_bytes = 2 * H->plane_bytes;
        gbssim_plane c = *x;
        c.row_stride = H->pitch_elems;
        c.image_stride = H->pitch_elems * x->height;
        int rc = plan_levels(&c, p, p->scales, &H->ms, false, true);
        if (rc) return rc;
        size_t off = 0;
        H->stage_off[0] = H->stage_off[1] = off;
        off = align_up(off + H->stage_bytes);
        H->ws_off[0] = H->ws_off[1] = off;
        off = align_up(off + H->ms.bytes);
        H->flags_off = off;
        off = align_up(off + sizeof(unsigned) * (size_t)n);
        H->score_off = off;
        off = align_up(off + sizeof(double) * (size_t)n);
        H->bytes = off;
        return GBSSIM_OK;
    }
    H->chunks = chunks < n ? chunks : n;
    H->per = (n + H->chunks - 1) / H->chunks;
    H->chunks = (n + H->per - 1) / H->per;
    H->esz = x->dtype == GBSSIM_U8 ? 1 : x->dtype == GBSSIM_F32 ? 4 : 2;
    const size_t row_bytes = (size_t)x->width * H->esz;
    const size_t pitch = (row_bytes + 15) / 16 * 16;
    H->pitch_elems = (int64_t)(pitch / H->esz);
    H->plane_bytes = pitch * (size_t)x->height * (size_t)H->per;
    H->stage_bytes = 2 * H->plane_bytes;
    gbssim_plane c = *x;
    c.count = H->per;
    c.row_stride = H->pitch_elems;
    c.image_stride = H->pitch_elems * x->height;
    int rc = plan_levels(&c, p, p->scales, &H->ms);
    if (rc) return rc;
    size_t off = 0;
    H->stage_off[0] = off;
    off = align_up(off + H->stage_bytes);
    H->stage_off[1] = off;
    off = align_up(off + H->stage_bytes);
    H->ws_off[0] = off;
    off = align_up(off + H->ms.bytes);
    H->ws_off[1] = off;
    off = align_up(off + H->ms.bytes);
    H->score_off = off;
    off = align_up(off + sizeof(double) * (size_t)n);
    H->flags_off = 0;
    H->bytes = off;
    return GBSSIM_OK;
}

// Copy images [i0, i0 + m) of a host plane into a dense pitched device plane.
cudaError_t copy_images_h2d(const gbssim_plane *h, int i0, int m, const HostPlan &H, char *dst, cudaStream_t cs) {
    const size_t row_bytes = (size_t)h->width * H.esz, pitch = (size_t)H.pitch_elems * H.esz;
    const int64_t img_stride = h->count > 1 ? h->image_stride : h->height * h->row_stride;
    const char *src = static_cast<const char *>(h->data) + (size_t)i0 * img_stride * H.esz;
    if ((size_t)h->row_stride * H.esz == pitch && img_stride == h->height * h->row_stride)
        return cudaMemcpyAsync(dst, src, pitch * (size_t)h->height * m, cudaMemcpyHostToDevice, cs);
    for (int i = 0; i < m; ++i) {
        const cudaError_t e = cudaMemcpy2DAsync(dst + (size_t)i * pitch * h->height, pitch,
                                                src + (size_t)i * img_stride * H.esz, (size_t)h->row_stride * H.esz,
                                                row_bytes, (size_t)h->height, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char *gbssim_status_string(int status) {
    switch (status) {
    case GBSSIM_OK: return "ok";
    case GBSSIM_ERR_INVALID_ARG: return "invalid argument";
    case GBSSIM_ERR_TOO_SMALL: return "image (or pyramid level) smaller than the window";
    case GBSSIM_ERR_UNSUPPORTED: return "unsupported combination";
    case GBSSIM_ERR_CUDA: return "CUDA runtime error";
    case GBSSIM_ERR_DOMAIN: return "non-positive pooled term under a fractional exponent";
    case GBSSIM_ERR_TIMEOUT: return "bounded device wait timed out";
    case GBSSIM_ERR_WORKSPACE: return "workspace missing or too small";
    case GBSSIM_ERR_TOO_LARGE: return "problem exceeds the static scratch of gbssim_ssim_map_static";
    }
    return "unknown status";
}

int gbssim_version(void) { return GBSSIM_VERSION; }

void gbssim_params_default(gbssim_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->window = GBSSIM_WIN_GAUSSIAN;
    p->k = 11;
    p->sigma = 1.5;
    p->K1 = 0.01;
    p->K2 = 0.03;
    p->L = 255.0;
    p->stride = 1;
    p->scales = 5;
    for (int j = 0; j < 5; ++j) p->exponents[j] = kDefaultExps[j];
    p->combine = GBSSIM_COMBINE_PRODUCT;
    p->flags = 0;
}

int gbssim_workspace_size(const gbssim_plane *x, const gbssim_params *p, int op, size_t *bytes) {
    if (!bytes) return GBSSIM_ERR_INVALID_ARG;
    int rc = check_plane(x);
    if (rc) return rc;
    if (op == GBSSIM_OP_POOL) {
        *bytes = pool_layout(x->height, x->width, x->count).bytes;
        return GBSSIM_OK;
    }
    rc = check_params(p);
    if (rc) return rc;
    MsPlan P;
    if (op == GBSSIM_OP_SSIM) {
        rc = plan_levels(x, p, 1, &P);
    } else if (op == GBSSIM_OP_MSSSIM) {
        rc = plan_levels(x, p, p->scales, &P);
    } else if (op == GBSSIM_OP_BACKWARD || op == GBSSIM_OP_BACKWARD_MS) {
        if (p->stride != 1 || p->k > GBSSIM_MAX_K_BACKWARD || border_mode(p)) return GBSSIM_ERR_UNSUPPORTED;
        BwdPlan B;
        rc = plan_backward(x, p, op == GBSSIM_OP_BACKWARD_MS, &B);
        if (rc) return rc;
        *bytes = B.bytes;
        return GBSSIM_OK;
    } else {
        return GBSSIM_ERR_INVALID_ARG;
    }
    if (rc) return rc;
    *bytes = P.bytes;
    return GBSSIM_OK;
}

int gbssim_ssim_map(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                    float *map_out, int64_t map_ld, int64_t map_image_stride, double *mean_out,
                    void *workspace, size_t workspace_bytes, void *stream) {
    int rc = check_pair(x, y);
    if (rc) return rc;
    rc = check_params(p);
    if (rc) return rc;
    MsPlan P;
    rc = plan_levels(x, p, 1, &P);
    if (rc) return rc;
    const int64_t OH = out_dim(P.lv[0].RH, p->k, p->stride), OW = out_dim(P.lv[0].RW, p->k, p->stride);
    if (map_out && (map_ld < OW || (x->count > 1 && map_image_stride < OH * map_ld)))
        return GBSSIM_ERR_INVALID_ARG;
    if (!map_out && !mean_out) return GBSSIM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < P.bytes) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    ImgDesc dx = desc_of(x), dy = desc_of(y);
    if (extend_level(P.lv[0], P, (char *)workspace, p, x->dtype, x->count, dx, dy, st) != cudaSuccess)
        return GBSSIM_ERR_CUDA;
    fix_box_items(P.lv[0], dx, dy, p);
    double2 *part = (double2 *)((char *)workspace + P.lv[0].part_off);
    cudaError_t e = run_level(P.lv[0], dx, dy, x->dtype, x->count, p, map_out, map_ld, map_image_stride, part,
                              nullptr, nullptr, st);
    if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
    if (mean_out) {
        e = launch_finalize_ssim(part, x->count, P.lv[0].items, 1.0 / ((double)OH * (double)OW), mean_out, st);
        if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
    }
    return GBSSIM_OK;
}

int gbssim_ssim_pool(const float *map, int64_t h, int64_t w, int64_t ld, int32_t count,
                     int64_t image_stride, int32_t kind, const double *args, double *out,
                     void *workspace, size_t workspace_bytes, void *stream) {
    if (!map || !out || h < 1 || w < 1 || ld < w || count < 1 || count > 65535) return GBSSIM_ERR_INVALID_ARG;
    if (count > 1 && image_stride < h * ld) return GBSSIM_ERR_INVALID_ARG;
    if (h * w > 0xffffffffLL) return GBSSIM_ERR_UNSUPPORTED;  // ranks are 32-bit
    double a0 = 0.0, a1 = 0.0;
    switch (kind) {
    case GBSSIM_POOL_MEAN:
    case GBSSIM_POOL_COV:
    case GBSSIM_POOL_GM_DSSIM:
    case GBSSIM_POOL_HM_DSSIM:
    case GBSSIM_POOL_MEDIAN:
    case GBSSIM_POOL_FNS: break;
    case GBSSIM_POOL_MINKOWSKI:
    case GBSSIM_POOL_DW:
        if (!args || !(isfinite(args[0]) && args[0] >= 0.0)) return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        break;
    case GBSSIM_POOL_MD:
        if (!args || !(isfinite(args[0]) && args[0] > 0.0 && isfinite(args[1]))) return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        a1 = args[1];
        break;
    case GBSSIM_POOL_PERCENTILE:
        if (!args || !(args[0] >= 0.0 && args[0] <= 100.0)) return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        break;
    case GBSSIM_POOL_PP:
        if (!args || !(args[0] >= 0.0 && args[0] <= 100.0) || !(isfinite(args[1]) && args[1] > 0.0))
            return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        a1 = args[1];
        break;
    default: return GBSSIM_ERR_INVALID_ARG;
    }
    const PoolLayout L = pool_layout(h, w, count);
    if (!workspace || workspace_bytes < L.bytes) return GBSSIM_ERR_WORKSPACE;
    const cudaError_t e = launch_pool_map(map, h, w, ld, count, count > 1 ? image_stride : h * ld, kind, a0, a1,
                                          (char *)workspace, out, (cudaStream_t)stream);
    return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

int gbssim_series_pool(const double *scores, int32_t n, int32_t count, int64_t stride, int32_t kind,
                       const double *args, double *out, void *stream) {
    if (!scores || !out || n < 1 || n > kVideoMaxFrames || count < 1 || count > 65535) return GBSSIM_ERR_INVALID_ARG;
    if (count > 1 && stride < n) return GBSSIM_ERR_INVALID_ARG;
    double a0 = 0.0, a1 = 0.0;
    switch (kind) {
    case GBSSIM_POOL_MEAN:
    case GBSSIM_POOL_COV:
    case GBSSIM_POOL_GM_DSSIM:
    case GBSSIM_POOL_HM_DSSIM:
    case GBSSIM_POOL_MEDIAN:
    case GBSSIM_POOL_FNS:
    case GBSSIM_POOL_GM:
    case GBSSIM_POOL_HM: break;
    case GBSSIM_POOL_MINKOWSKI:
    case GBSSIM_POOL_DW:
        if (!args || !(isfinite(args[0]) && args[0] >= 0.0)) return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        break;
    case GBSSIM_POOL_MD:
        if (!args || !(isfinite(args[0]) && args[0] > 0.0 && isfinite(args[1]))) return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        a1 = args[1];
        break;
    case GBSSIM_POOL_PERCENTILE:
        if (!args || !(args[0] >= 0.0 && args[0] <= 100.0)) return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        break;
    case GBSSIM_POOL_PP:
        if (!args || !(args[0] >= 0.0 && args[0] <= 100.0) || !(isfinite(args[1]) && args[1] > 0.0))
            return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        a1 = args[1];
        break;
    case GBSSIM_POOL_W_AM:
    case GBSSIM_POOL_W_GM:
    case GBSSIM_POOL_W_HM:
    case GBSSIM_POOL_W_COV:
        if (!args || !(args[0] >= 1.0 && args[0] <= n && args[0] == floor(args[0]))) return GBSSIM_ERR_INVALID_ARG;
        a0 = args[0];
        break;
    default: return GBSSIM_ERR_INVALID_ARG;
    }
    const cudaError_t e =
        launch_series_pool(scores, n, count, count > 1 ? stride : n, kind, a0, a1, out, (cudaStream_t)stream);
    return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

namespace {
// Checks shared by SSIM-3D (scales = 1) and MS-SSIM-3D.
int check_ssim3d(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t kt, int scales) {
    int rc = check_pair(x, y);
    if (rc) return rc;
    rc = check_params_valid(p);
    if (rc) return rc;
    if (x->dtype != GBSSIM_U8 || p->window != GBSSIM_WIN_BOX || p->stride != 1 || p->k > kSsim3dMaxK)
        return GBSSIM_ERR_UNSUPPORTED;
    if (kt < 1) return GBSSIM_ERR_INVALID_ARG;
    if (x->count < kt) return GBSSIM_ERR_TOO_SMALL;
    for (int j = 0; j < scales; ++j)
        if ((x->height >> j) < p->k || (x->width >> j) < p->k) return GBSSIM_ERR_TOO_SMALL;
    // exact int64 numerators: at level j the values times 4^j are integers up
    // to M = 255 4^j, |u| <= 2M, |w| <= M, and every numerator is at most
    // 5 N^2 M^2 (Su^2 + Sw^2, Vu + Vw), kept below 2^63
    const double n = (double)p->k * p->k * kt;
    for (int j = 0; j < scales; ++j) {
        const double m = 255.0 * (double)(1 << (2 * j));
        if (5.0 * n * n * m * m >= 9223372036854775808.0) return GBSSIM_ERR_UNSUPPORTED;
    }
    if (scales > 1 && x->count > 65535) return GBSSIM_ERR_UNSUPPORTED;  // pyramid grid's z extent
    return GBSSIM_OK;
}

// uint8 level 0 sums in int32 while N (2 255)^2 < 2^31 (the largest sum of u^2).
bool ssim3d_wide0(const gbssim_params *p, int32_t kt) {
    return (double)p->k * p->k * kt * 260100.0 >= 2147483648.0;
}

struct Ms3dPlan {
    int frames, scales;
    int64_t H[GBSSIM_MAX_SCALES], W[GBSSIM_MAX_SCALES];
    int items[GBSSIM_MAX_SCALES];  // partials (tiles) per output frame
    size_t partials[GBSSIM_MAX_SCALES], pyr_x[GBSSIM_MAX_SCALES], pyr_y[GBSSIM_MAX_SCALES], frame_buf, bytes;
};

// Workspace: per level the (frame, tile) partials, a frame-score buffer,
// then the float pyramid levels 1..S-1 of x and y (T dense frames each).
Ms3dPlan plan_ms3d(const gbssim_plane *x, const gbssim_params *p, int32_t kt, int scales) {
    Ms3dPlan P{};
    P.frames = x->count - kt + 1;
    P.scales = scales;
    size_t off = 0;
    for (int j = 0; j < scales; ++j) {
        P.H[j] = x->height >> j;
        P.W[j] = x->width >> j;
        const bool wide = j > 0 || ssim3d_wide0(p, kt);
        int tx, ty;
        ssim3d_tiles(P.H[j], P.W[j], p->k, wide, &tx, &ty);
        P.items[j] = tx * ty;
        P.partials[j] = off;
        off = align_up(off + sizeof(double2) * (size_t)P.frames * P.items[j]);
    }
    P.frame_buf = off;
    off = align_up(off + sizeof(double) * (size_t)P.frames);
    for (int j = 1; j < scales; ++j) {
        const size_t plane = sizeof(float) * (size_t)P.H[j] * P.W[j] * x->count;
        P.pyr_x[j] = off;
        off = align_up(off + plane);
        P.pyr_y[j] = off;
        off = align_up(off + plane);
    }
    P.bytes = off;
    return P;
}

// SSIM-3D on every level of the frames' 2x2 pyramid, then the per-frame
// combination (the MS-SSIM finaliser over frames) and the video mean.
int run_ms3d(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t kt, int scales,
             const double *exps, int combine, double *frame_out, double *score_out, double *per_scale_out,
             float *map_out, int64_t map_ld, int64_t map_frame_stride, void *workspace, size_t workspace_bytes,
             cudaStream_t st) {
    const Ms3dPlan P = plan_ms3d(x, p, kt, scales);
    if (!workspace || workspace_bytes < P.bytes) return GBSSIM_ERR_WORKSPACE;
    char *ws = static_cast<char *>(workspace);
    const double n = (double)p->k * p->k * kt;
    const double c1 = (p->K1 * p->L) * (p->K1 * p->L), c2 = (p->K2 * p->L) * (p->K2 * p->L);
    Ms3dFinalize F{};
    F.scales = scales;
    F.frames = P.frames;
    F.combine = combine;
    for (int j = 0; j < scales; ++j) {
        F.exps[j] = exps[j];
        Ssim3dLaunch L{};
        const bool level0 = j == 0;
        if (level0) {
            L.x = desc_of(x);
            L.y = desc_of(y);
            L.vec4 = (uintptr_t)x->data % 4 == 0 && (uintptr_t)y->data % 4 == 0 && L.x.row_stride % 4 == 0 &&
                     L.x.image_stride % 4 == 0;
            L.scale = 1.f;
        } else {
            // level j from level j-1: uint8 input or the float level below
            const ImgDesc src_x = j == 1 ? desc_of(x)
                                         : ImgDesc{ws + P.pyr_x[j - 1], P.H[j - 1], P.W[j - 1], P.W[j - 1],
                                                   P.H[j - 1] * P.W[j - 1]};
            const ImgDesc src_y = j == 1 ? desc_of(y)
                                         : ImgDesc{ws + P.pyr_y[j - 1], P.H[j - 1], P.W[j - 1], P.W[j - 1],
                                                   P.H[j - 1] * P.W[j - 1]};
            const int dt = j == 1 ? GBSSIM_U8 : GBSSIM_F32;
            cudaError_t e = launch_downsample(src_x, dt, x->count, (float *)(ws + P.pyr_x[j]), st);
            if (e == cudaSuccess) e = launch_downsample(src_y, dt, x->count, (float *)(ws + P.pyr_y[j]), st);
            if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
            L.x = ImgDesc{ws + P.pyr_x[j], P.H[j], P.W[j], P.W[j], P.H[j] * P.W[j]};
            L.y = ImgDesc{ws + P.pyr_y[j], P.H[j], P.W[j], P.W[j], P.H[j] * P.W[j]};
            L.vec4 = P.W[j] % 4 == 0 && (uintptr_t)L.x.data % 16 == 0 && (uintptr_t)L.y.data % 16 == 0;
            L.scale = (float)(1 << (2 * j));
        }
        const double sc2 = (double)L.scale * L.scale;
        L.T = x->count;
        L.k = p->k;
        L.kt = kt;
        L.map = level0 ? map_out : nullptr;
        L.map_ld = map_ld;
        L.map_fs = map_frame_stride;
        L.partials = (double2 *)(ws + P.partials[j]);
        L.C1x2n2 = (float)(2.0 * c1 * sc2 * n * n);
        L.C2x2n2 = (float)(2.0 * c2 * sc2 * n * n);
        const bool wide = !level0 || ssim3d_wide0(p, kt);
        if (launch_ssim3d_level(L, level0, wide, st) != cudaSuccess) return GBSSIM_ERR_CUDA;
        F.partials[j] = L.partials;
        F.items[j] = P.items[j];
        F.inv_n[j] = 1.0 / ((double)(P.H[j] - p->k + 1) * (double)(P.W[j] - p->k + 1));
    }
    double *frames = frame_out ? frame_out : (double *)(ws + P.frame_buf);
    return launch_ssim3d_finalize(F, frames, per_scale_out, score_out, st) == cudaSuccess
               ? GBSSIM_OK
               : GBSSIM_ERR_CUDA;
}
}  // namespace

int gbssim_ssim3d_workspace_size(const gbssim_plane *x, const gbssim_params *p, int32_t kt, size_t *bytes) {
    const int rc = check_ssim3d(x, x, p, kt, 1);
    if (rc) return rc;
    if (!bytes) return GBSSIM_ERR_INVALID_ARG;
    *bytes = plan_ms3d(x, p, kt, 1).bytes;
    return GBSSIM_OK;
}

int gbssim_ssim3d(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t kt,
                  double *frame_out, double *score_out, float *map_out, int64_t map_ld, int64_t map_frame_stride,
                  void *workspace, size_t workspace_bytes, void *stream) {
    const int rc = check_ssim3d(x, y, p, kt, 1);
    if (rc) return rc;
    const int64_t OH = x->height - p->k + 1, OW = x->width - p->k + 1;
    if (!frame_out && !score_out && !map_out) return GBSSIM_ERR_INVALID_ARG;
    if (map_out && (map_ld < OW || map_frame_stride < OH * map_ld)) return GBSSIM_ERR_INVALID_ARG;
    // one level: the normalised sum with weight 1 is the mean Q itself
    const double one = 1.0;
    return run_ms3d(x, y, p, kt, 1, &one, GBSSIM_COMBINE_SUM, frame_out, score_out, nullptr, map_out, map_ld,
                    map_frame_stride, workspace, workspace_bytes, (cudaStream_t)stream);
}

int gbssim_msssim3d_workspace_size(const gbssim_plane *x, const gbssim_params *p, int32_t kt, size_t *bytes) {
    const int rc = check_params_valid(p);
    if (rc) return rc;
    const int rc2 = check_ssim3d(x, x, p, kt, p->scales);
    if (rc2) return rc2;
    if (!bytes) return GBSSIM_ERR_INVALID_ARG;
    *bytes = plan_ms3d(x, p, kt, p->scales).bytes;
    return GBSSIM_OK;
}

int gbssim_msssim3d(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t kt,
                    double *frame_out, double *score_out, double *per_scale_out, void *workspace,
                    size_t workspace_bytes, void *stream) {
    const int rc = check_params_valid(p);
    if (rc) return rc;
    const int rc2 = check_ssim3d(x, y, p, kt, p->scales);
    if (rc2) return rc2;
    if (!frame_out && !score_out && !per_scale_out) return GBSSIM_ERR_INVALID_ARG;
    return run_ms3d(x, y, p, kt, p->scales, p->exponents, p->combine, frame_out, score_out, per_scale_out, nullptr,
                    0, 0, workspace, workspace_bytes, (cudaStream_t)stream);
}

int gbssim_rgb_to_ycbcr(const gbssim_plane *r, const gbssim_plane *g, const gbssim_plane *b, float *y_out,
                        float *cb_out, float *cr_out, int64_t out_ld, int64_t out_image_stride, void *stream) {
    int rc = check_pair(r, g);
    if (rc) return rc;
    rc = check_pair(r, b);
    if (rc) return rc;
    if (!y_out || !cb_out || !cr_out || out_ld < r->width || (r->count > 1 && out_image_stride < r->height * out_ld))
        return GBSSIM_ERR_INVALID_ARG;
    const cudaError_t e =
        launch_rgb_ycbcr(desc_of(r), desc_of(g), desc_of(b), r->dtype, r->count, y_out, cb_out, cr_out, out_ld,
                         r->count > 1 ? out_image_stride : r->height * out_ld, (cudaStream_t)stream);
    return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

int gbssim_local_mean(const gbssim_plane *x, const gbssim_params *p, float *out, int64_t out_ld,
                      int64_t out_image_stride, void *stream) {
    int rc = check_plane(x);
    if (rc) return rc;
    rc = check_params_valid(p);
    if (rc) return rc;
    if (!out || x->height < p->k || x->width < p->k) return out ? GBSSIM_ERR_TOO_SMALL : GBSSIM_ERR_INVALID_ARG;
    const int64_t OH = out_dim(x->height, p->k, p->stride), OW = out_dim(x->width, p->k, p->stride);
    if (out_ld < OW || (x->count > 1 && out_image_stride < OH * out_ld)) return GBSSIM_ERR_INVALID_ARG;
    TapsDyn taps;
    memset(taps.g, 0, sizeof taps.g);
    make_taps(p, taps.g);
    const cudaError_t e = launch_local_mean(desc_of(x), x->dtype, x->count, taps, p->k, p->stride, out, out_ld,
                                            x->count > 1 ? out_image_stride : OH * out_ld, (cudaStream_t)stream);
    return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

int gbssim_ssim_pool_lw(const float *map, const float *mu_ref, int64_t h, int64_t w, int64_t ld, int32_t count,
                        int64_t image_stride, double a, double b, double *out, void *workspace, size_t workspace_bytes,
                        void *stream) {
    if (!map || !mu_ref || !out || h < 1 || w < 1 || ld < w || count < 1 || count > 65535) return GBSSIM_ERR_INVALID_ARG;
    if (count > 1 && image_stride < h * ld) return GBSSIM_ERR_INVALID_ARG;
    if (!isfinite(a) || !isfinite(b) || b < 0.0) return GBSSIM_ERR_INVALID_ARG;
    const PoolLayout L = pool_layout(h, w, count);
    if (!workspace || workspace_bytes < L.bytes) return GBSSIM_ERR_WORKSPACE;
    const cudaError_t e = launch_pool_map(map, h, w, ld, count, count > 1 ? image_stride : h * ld, kPoolLW, a, b,
                                          (char *)workspace, out, (cudaStream_t)stream, mu_ref);
    return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

namespace {
// CMSSIM's matrices: linear BT.709 / sRGB RGB to XYZ (D65), and the
// section's XYZ -> opponent and opponent -> XYZ matrices as printed.
const double kRgbToXyz[9] = {0.4124, 0.3576, 0.1805, 0.2126, 0.7152, 0.0722, 0.0193, 0.1192, 0.9505};
const double kXyzToOpp[9] = {0.279, 0.72, -0.107, -0.449, 0.29, -0.077, 0.086, -0.59, 0.501};
const double kOppToXyz[9] = {0.6204, -1.8704, -0.1553, 1.3661, 0.9316, 0.4339, 1.5013, 1.4176, 2.5331};

struct CmPlan {
    int64_t H, W, OH, OW, PH, PW, plane;
    size_t lab_off, pad_off, map_off, ssim_off, pool_off, bytes;
    MsPlan ssim;
    gbssim_params ps;  // the SSIM of L*: the caller's window and K1, K2 with L = 100
};

int plan_cmssim(const gbssim_plane *x, const gbssim_params *p, CmPlan *C) {
    int rc = check_params_valid(p);
    if (rc) return rc;
    if (p->window != GBSSIM_WIN_GAUSSIAN) return GBSSIM_ERR_UNSUPPORTED;
    if (x->height < p->k || x->width < p->k) return GBSSIM_ERR_TOO_SMALL;
    const int64_t n = x->count;
    C->H = x->height;
    C->W = x->width;
    C->plane = C->H * C->W;
    C->OH = out_dim(C->H, p->k, p->stride);
    C->OW = out_dim(C->W, p->k, p->stride);
    C->PH = C->H + p->k - 1;
    C->PW = C->W + p->k - 1;
    if (C->PH > 65535 || C->H > 65535) return GBSSIM_ERR_UNSUPPORTED;  // grid y extents
    C->ps = *p;
    C->ps.L = 100.0;
    C->ps.scales = 1;
    C->ps.flags = 0;
    gbssim_plane lp{x->data, GBSSIM_F32, x->count, C->H, C->W, C->W, C->plane};
    rc = plan_levels(&lp, &C->ps, 1, &C->ssim);
    if (rc) return rc;
    size_t off = 0;
    C->lab_off = off;
    off = align_up(off + 6 * sizeof(float) * (size_t)C->plane * n);
    C->pad_off = off;
    off = align_up(off + sizeof(float) * (size_t)C->PH * C->PW * n);
    C->map_off = off;
    off = align_up(off + sizeof(float) * (size_t)C->OH * C->OW * n);
    C->ssim_off = off;
    off = align_up(off + C->ssim.bytes);
    C->pool_off = off;
    off = align_up(off + pool_layout(C->OH, C->OW, x->count).bytes);
    C->bytes = off;
    return GBSSIM_OK;
}
}  // namespace

int gbssim_cmssim_workspace_size(const gbssim_plane *r, const gbssim_params *p, size_t *bytes) {
    int rc = check_plane(r);
    if (rc) return rc;
    if (!bytes) return GBSSIM_ERR_INVALID_ARG;
    CmPlan C;
    rc = plan_cmssim(r, p, &C);
    if (rc) return rc;
    *bytes = C.bytes;
    return GBSSIM_OK;
}

int gbssim_cmssim(const gbssim_plane rgb_x[3], const gbssim_plane rgb_y[3], const gbssim_params *p,
                  double *score_out, float *map_out, int64_t map_ld, int64_t map_image_stride, void *workspace,
                  size_t workspace_bytes, void *stream) {
    if (!rgb_x || !rgb_y || !score_out) return GBSSIM_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c) {
        int rc = check_pair(&rgb_x[0], &rgb_x[c]);
        if (!rc) rc = check_pair(&rgb_x[0], &rgb_y[c]);
        if (rc) return rc;
    }
    CmPlan C;
    int rc = plan_cmssim(&rgb_x[0], p, &C);
    if (rc) return rc;
    const int n = rgb_x[0].count;
    if (map_out && (map_ld < C.OW || (n > 1 && map_image_stride < C.OH * map_ld))) return GBSSIM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < C.bytes) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    const int64_t cs = C.plane * n;  // channel stride of the L*, a*, b* arrays
    float *lab[2] = {(float *)(ws + C.lab_off), (float *)(ws + C.lab_off) + 3 * cs};
    // RGB -> XYZ -> opponent planes, in one matrix product formed in double
    double m[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int t = 0; t < 3; ++t) acc += kXyzToOpp[3 * i + t] * kRgbToXyz[3 * t + j];
            m[3 * i + j] = acc;
        }
    const double white[3] = {kRgbToXyz[0] + kRgbToXyz[1] + kRgbToXyz[2], kRgbToXyz[3] + kRgbToXyz[4] + kRgbToXyz[5],
                             kRgbToXyz[6] + kRgbToXyz[7] + kRgbToXyz[8]};
    TapsDyn taps;
    memset(taps.g, 0, sizeof taps.g);
    make_taps(p, taps.g);
    const int before = (p->k - 1) / 2;
    float *pad = (float *)(ws + C.pad_off);
    for (int s = 0; s < 2; ++s) {
        const gbssim_plane *rgb = s ? rgb_y : rgb_x;
        float *q = lab[s];
        if (launch_rgb_opp(desc_of(&rgb[0]), desc_of(&rgb[1]), desc_of(&rgb[2]), rgb[0].dtype, n, m, q, q + cs,
                           q + 2 * cs, st) != cudaSuccess)
            return GBSSIM_ERR_CUDA;
        // the chromatic planes smoothed in place: mirror extension, then the window mean
        for (int c = 1; c < 3; ++c) {
            const ImgDesc d{q + c * cs, C.H, C.W, C.W, C.plane};
            if (launch_pad(d, GBSSIM_F32, n, pad, C.PH, C.PW, before, before, 1, st) != cudaSuccess)
                return GBSSIM_ERR_CUDA;
            const ImgDesc pd{pad, C.PH, C.PW, C.PW, C.PH * C.PW};
            if (launch_local_mean(pd, GBSSIM_F32, n, taps, p->k, 1, q + c * cs, C.W, C.plane, st) != cudaSuccess)
                return GBSSIM_ERR_CUDA;
        }
        if (launch_opp_lab(q, q + cs, q + 2 * cs, cs, kOppToXyz, white, st) != cudaSuccess) return GBSSIM_ERR_CUDA;
    }
    // SSIM map of the L* planes, weighted by (1 - Delta E / 45), mean-pooled
    float *map = map_out ? map_out : (float *)(ws + C.map_off);
    const int64_t ld = map_out ? map_ld : C.OW;
    const int64_t is = map_out ? (n > 1 ? map_image_stride : C.OH * map_ld) : C.OH * C.OW;
    const ImgDesc lx{lab[0], C.H, C.W, C.W, C.plane}, ly{lab[1], C.H, C.W, C.W, C.plane};
    Level L = C.ssim.lv[0];
    char *sws = ws + C.ssim_off;
    double2 *part = (double2 *)(sws + L.part_off);
    if (run_level(L, lx, ly, GBSSIM_F32, n, &C.ps, map, ld, is, part, nullptr, nullptr, st) != cudaSuccess)
        return GBSSIM_ERR_CUDA;
    if (launch_cmssim_weight(map, C.OH, C.OW, ld, is, n, lab[0], lab[1], C.H, C.W, cs, before, p->stride, st) !=
        cudaSuccess)
        return GBSSIM_ERR_CUDA;
    return launch_pool_map(map, C.OH, C.OW, ld, n, is, GBSSIM_POOL_MEAN, 0.0, 0.0, ws + C.pool_off, score_out, st) ==
                   cudaSuccess
               ? GBSSIM_OK
               : GBSSIM_ERR_CUDA;
}

int gbssim_qssim_workspace_size(const gbssim_plane *x, size_t *bytes) {
    int rc = check_plane(x);
    if (rc) return rc;
    if (!bytes) return GBSSIM_ERR_INVALID_ARG;
    if (x->height < 2 || x->width < 2) return GBSSIM_ERR_TOO_SMALL;
    *bytes = qssim_workspace(x->dtype, x->height, x->width, x->count);
    return GBSSIM_OK;
}

int gbssim_qssim(const gbssim_plane tri_x[3], const gbssim_plane tri_y[3], const gbssim_params *p,
                 double *score_out, double *terms_out, void *workspace, size_t workspace_bytes, void *stream) {
    if (!tri_x || !tri_y || !score_out) return GBSSIM_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c) {
        int rc = check_pair(&tri_x[0], &tri_x[c]);
        if (!rc) rc = check_pair(&tri_x[0], &tri_y[c]);
        if (rc) return rc;
    }
    if (!p) return GBSSIM_ERR_INVALID_ARG;
    if (!(isfinite(p->K1) && isfinite(p->K2) && p->K1 >= 0.0 && p->K2 >= 0.0)) return GBSSIM_ERR_INVALID_ARG;
    if (!(p->L > 0.0 && isfinite(p->L))) return GBSSIM_ERR_INVALID_ARG;
    const gbssim_plane &x = tri_x[0];
    if (x.height < 2 || x.width < 2) return GBSSIM_ERR_TOO_SMALL;
    const size_t need = qssim_workspace(x.dtype, x.height, x.width, x.count);
    if (!workspace || workspace_bytes < need) return GBSSIM_ERR_WORKSPACE;
    ImgDesc dx[3], dy[3];
    for (int c = 0; c < 3; ++c) {
        dx[c] = desc_of(&tri_x[c]);
        dy[c] = desc_of(&tri_y[c]);
    }
    const double c1 = (p->K1 * p->L) * (p->K1 * p->L), c2 = (p->K2 * p->L) * (p->K2 * p->L);
    return launch_qssim(dx, dy, x.dtype, x.count, c1, c2, workspace, score_out, terms_out, (cudaStream_t)stream) ==
                   cudaSuccess
               ? GBSSIM_OK
               : GBSSIM_ERR_CUDA;
}

int gbssim_downscale_factor(int64_t h, int64_t w, int32_t rule) {
    if (h < 1 || w < 1) return GBSSIM_ERR_INVALID_ARG;
    if (rule == GBSSIM_DOWNSCALE_ROUND_MIN) {
        const int64_t z = ((h < w ? h : w) + 128) / 256;
        return (int)(z > 1 ? z : 1);
    }
    if (rule == GBSSIM_DOWNSCALE_CEIL_H) {
        const int64_t z = (h + 255) / 256;
        return (int)(z > 1 ? z : 1);
    }
    return GBSSIM_ERR_INVALID_ARG;
}

int gbssim_downscale(const gbssim_plane *in, int32_t z, float *out, int64_t out_ld, int64_t out_image_stride,
                     void *stream) {
    int rc = check_plane(in);
    if (rc) return rc;
    if (!out || z < 1 || z > in->height || z > in->width) return GBSSIM_ERR_INVALID_ARG;
    const int64_t oh = in->height / z, ow = in->width / z;
    if (out_ld < ow || (in->count > 1 && out_image_stride < oh * out_ld)) return GBSSIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_block_mean(desc_of(in), in->dtype, in->count, z, out, out_ld,
                                            in->count > 1 ? out_image_stride : oh * out_ld, (cudaStream_t)stream);
    return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

int gbssim_msssim(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                  double *score_out, double *per_scale_out, void *workspace,
                  size_t workspace_bytes, void *stream) {
    int rc = check_pair(x, y);
    if (rc) return rc;
    rc = check_params(p);
    if (rc) return rc;
    if (!score_out) return GBSSIM_ERR_INVALID_ARG;
    MsPlan P;
    rc = plan_levels(x, p, p->scales, &P);
    if (rc) return rc;
    if (!workspace || workspace_bytes < P.bytes) return GBSSIM_ERR_WORKSPACE;
    return msssim_forward(x, y, p, P, (char *)workspace, score_out, per_scale_out, (cudaStream_t)stream);
}

int gbssim_msssim_host_workspace_size(const gbssim_plane *x, const gbssim_params *p, int32_t chunks,
                                      size_t *bytes) {
    int rc = check_plane(x);
    if (rc) return rc;
    rc = check_params_valid(p);
    if (rc) return rc;
    if (!bytes) return GBSSIM_ERR_INVALID_ARG;
    HostPlan H;
    rc = plan_host(x, p, chunks, &H);
    if (rc) return rc;
    *bytes = H.bytes;
    return GBSSIM_OK;
}

}  // extern "C"

namespace {

// gbssim_msssim_host and gbssim_msssim_host_ex.  wait_limit: 0 = the default;
// drop_flag: test hook, the last copy group's arrival flag is never set;
// status_host (nullable, streamed mode only): the launch's status word.
int msssim_host_impl(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t chunks,
                     double *score_host, int32_t *status_host, unsigned wait_limit, bool drop_flag,
                     void *workspace, size_t workspace_bytes, void *stream, void *copy_stream, void *stream2) {
    int rc = check_pair(x, y);
    if (rc) return rc;
    rc = check_params_valid(p);
    if (rc) return rc;
    if (!score_host) return GBSSIM_ERR_INVALID_ARG;
    if ((status_host || drop_flag) && chunks != 0) return GBSSIM_ERR_UNSUPPORTED;
    HostPlan H;
    rc = plan_host(x, p, chunks, &H);
    if (rc) return rc;
    if (!workspace || workspace_bytes < H.bytes) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
    cudaStream_t cst[2] = {st, stream2 ? (cudaStream_t)stream2 : st};  // compute stream of stage s
    if (cs == st || cs == cst[1] || (stream2 && cst[1] == st)) return GBSSIM_ERR_INVALID_ARG;
    char *ws = (char *)workspace;
    double *score_dev = (double *)(ws + H.score_off);
    // events: the caller's prior work, per stage "copied" / "consumed", and
    // the second compute stream's end
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (auto &e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            for (auto &f : ev)
                if (f) cudaEventDestroy(f);
            return GBSSIM_ERR_CUDA;
        }
    cudaEvent_t prior = ev[0], copied[2] = {ev[1], ev[2]}, consumed[2] = {ev[3], ev[4]}, done2 = ev[5];
    cudaError_t e = cudaEventRecord(prior, st);  // earlier calls on `stream` may still read the buffers
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, prior, 0);
    if (H.chunks == 0) {
        // streamed: on the copy stream, clear the arrival flags, then per
        // group of images copy x, y and set the group's flag with a stream
        // memory write that orders the copies before it; then the one
        // MS-SSIM launch over all images (its level-0 items wait for their
        // group's flag).  Every copy is enqueued before the launch, so the
        // launch depends on no host call after it (a serialised or blocking
        // launch still finds its inputs arriving).
        auto write32 = stream_write_value32();
        unsigned *flags = (unsigned *)(ws + H.flags_off);
        int gbegin[kUniformMaxGroups + 1];
        const int G = stream_groups(x->count, gbegin);
        char *xs = ws + H.stage_off[0], *ysg = xs + H.plane_bytes;
        if (!write32) e = cudaErrorNotSupported;
        // the copy stream must not wait for the launch (an implicitly
        // synchronising stream would leave the level-0 items waiting)
        unsigned cflags = 0;
        if (e == cudaSuccess && (cudaStreamGetFlags(cs, &cflags) != cudaSuccess || !(cflags & cudaStreamNonBlocking)))
            rc = GBSSIM_ERR_INVALID_ARG;
        if (e == cudaSuccess && rc == GBSSIM_OK) e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)x->count, cs);
        if (e == cudaSuccess && rc == GBSSIM_OK) e = cudaEventRecord(copied[0], cs);
        // one copy of x and one of y per group, then the group's flag
        const size_t img_bytes = (size_t)H.pitch_elems * H.esz * x->height;
        for (int f = 0; f < G && e == cudaSuccess && rc == GBSSIM_OK; ++f) {
            const int i0 = gbegin[f], m = gbegin[f + 1] - gbegin[f];
            e = copy_images_h2d(x, i0, m, H, xs + i0 * img_bytes, cs);
            if (e == cudaSuccess) e = copy_images_h2d(y, i0, m, H, ysg + i0 * img_bytes, cs);
            const bool last = f + 1 == G;
            if (e == cudaSuccess && !(drop_flag && last) &&
                write32(cs, (CUdeviceptr)(flags + f), 1u, CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS)
                e = cudaErrorUnknown;
        }
        // the copy stream's end: `stream` waits for it before the score
        // readback, so every copy of the call (also one whose items' bounded
        // wait gave up before it landed) is ordered before the end of `stream`
        if (e == cudaSuccess && rc == GBSSIM_OK) e = cudaEventRecord(copied[1], cs);
        if (e == cudaSuccess && rc == GBSSIM_OK) e = cudaStreamWaitEvent(st, copied[0], 0);  // flags cleared
        if (e == cudaSuccess && rc == GBSSIM_OK) {
            gbssim_plane dx = *x, dy = *y;
            dx.data = xs;
            dy.data = ysg;
            dx.row_stride = dy.row_stride = H.pitch_elems;
            dx.image_stride = dy.image_stride = H.pitch_elems * x->height;
            rc = msssim_forward(&dx, &dy, p, H.ms, ws + H.ws_off[0], score_dev, nullptr, st, flags, gbegin, G,
                                wait_limit);
        }
        if (e == cudaSuccess && rc == GBSSIM_OK) e = cudaStreamWaitEvent(st, copied[1], 0);
        if (e == cudaSuccess && rc == GBSSIM_OK)
            e = cudaMemcpyAsync(score_host, score_dev, sizeof(double) * (size_t)x->count, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && rc == GBSSIM_OK && status_host)
            e = cudaMemcpyAsync(status_host, ws + H.ws_off[0] + H.ms.status_off, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st);
        for (auto &f : ev) cudaEventDestroy(f);
        if (rc != GBSSIM_OK) return rc;
        if (e == cudaErrorNotSupported) return GBSSIM_ERR_UNSUPPORTED;
        return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
    }
    if (e == cudaSuccess && stream2) e = cudaStreamWaitEvent(cst[1], prior, 0);
    for (int c = 0; c < H.chunks && e == cudaSuccess && rc == GBSSIM_OK; ++c) {
        const int s = c & 1, i0 = c * H.per, m = x->count - i0 < H.per ? x->count - i0 : H.per;
        char *xs = ws + H.stage_off[s], *ysg = xs + H.plane_bytes;
        if (c >= 2) e = cudaStreamWaitEvent(cs, consumed[s], 0);  // chunk c-2 done with this stage
        if (e == cudaSuccess) e = copy_images_h2d(x, i0, m, H, xs, cs);
        if (e == cudaSuccess) e = copy_images_h2d(y, i0, m, H, ysg, cs);
        if (e == cudaSuccess) e = cudaEventRecord(copied[s], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cst[s], copied[s], 0);
        if (e != cudaSuccess) break;
        gbssim_plane dx = *x, dy = *y;
        dx.data = xs;
        dy.data = ysg;
        dx.count = dy.count = m;
        dx.row_stride = dy.row_stride = H.pitch_elems;
        dx.image_stride = dy.image_stride = H.pitch_elems * x->height;
        MsPlan P;  // a short last chunk has fewer items: re-plan its layout (it fits the full one)
        rc = plan_levels(&dx, p, p->scales, &P);
        if (rc == GBSSIM_OK && P.bytes > H.ms.bytes) rc = GBSSIM_ERR_WORKSPACE;
        if (rc == GBSSIM_OK)
            rc = msssim_forward(&dx, &dy, p, P, ws + H.ws_off[s], score_dev + i0, nullptr, cst[s]);
        if (rc == GBSSIM_OK) e = cudaEventRecord(consumed[s], cst[s]);
    }
    if (e == cudaSuccess && rc == GBSSIM_OK && stream2) {  // `stream` ends after the second compute stream
        e = cudaEventRecord(done2, cst[1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, done2, 0);
    }
    if (e == cudaSuccess && rc == GBSSIM_OK)
        e = cudaMemcpyAsync(score_host, score_dev, sizeof(double) * (size_t)x->count, cudaMemcpyDeviceToHost, st);
    for (auto &f : ev) cudaEventDestroy(f);  // released once the streams are past them
    if (rc != GBSSIM_OK) return rc;
    return e == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

}  // namespace

extern "C" {

int gbssim_msssim_host(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t chunks,
                       double *score_host, void *workspace, size_t workspace_bytes, void *stream,
                       void *copy_stream, void *stream2) {
    return msssim_host_impl(x, y, p, chunks, score_host, nullptr, 0, false, workspace, workspace_bytes, stream,
                            copy_stream, stream2);
}

int gbssim_msssim_host_ex(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t chunks,
                          const gbssim_tuning *tuning, double *score_host, int32_t *status_host, void *workspace,
                          size_t workspace_bytes, void *stream, void *copy_stream, void *stream2) {
    if (tuning && (tuning->flags & ~GBSSIM_TUNING_TEST_DROP_ARRIVAL)) return GBSSIM_ERR_INVALID_ARG;
    const unsigned wl = tuning ? tuning->wait_limit : 0u;
    const bool drop = tuning && (tuning->flags & GBSSIM_TUNING_TEST_DROP_ARRIVAL);
    return msssim_host_impl(x, y, p, chunks, score_host, status_host, wl, drop, workspace, workspace_bytes, stream,
                            copy_stream, stream2);
}

int gbssim_ssim_backward(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p,
                         int32_t multiscale, double grad_scale, const double *grad_out,
                         int32_t grad_out_per_image, const double *fwd_score, const double *fwd_per_scale,
                         void *grad_y, int32_t grad_dtype, int64_t grad_ld, int64_t grad_image_stride,
                         double *score_out, void *workspace, size_t workspace_bytes, void *stream) {
    int rc = check_pair(x, y);
    if (rc) return rc;
    rc = check_params_valid(p);
    if (rc) return rc;
    if (p->stride != 1 || p->k > GBSSIM_MAX_K_BACKWARD) return GBSSIM_ERR_UNSUPPORTED;
    if (p->flags & GBSSIM_FLAG_PYRAMID_97) return GBSSIM_ERR_UNSUPPORTED;  // no adjoint of the 9/7 step
    if (!grad_y || (grad_dtype != GBSSIM_F32 && grad_dtype != GBSSIM_F16 && grad_dtype != GBSSIM_BF16))
        return GBSSIM_ERR_INVALID_ARG;
    if (grad_ld < x->width || (x->count > 1 && grad_image_stride < x->height * grad_ld))
        return GBSSIM_ERR_INVALID_ARG;
    if (!isfinite(grad_scale)) return GBSSIM_ERR_INVALID_ARG;
    if ((fwd_score == nullptr) != (fwd_per_scale == nullptr)) return GBSSIM_ERR_INVALID_ARG;
    BwdPlan B;
    rc = plan_backward(x, p, multiscale != 0, &B);
    if (rc) return rc;
    if (!workspace || workspace_bytes < B.bytes) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    const int n = x->count, S = multiscale ? p->scales : 1;
    double *score = (double *)(ws + B.score_off), *per = (double *)(ws + B.per_off);
    const double *ms_score = score, *ms_per = per;
    if (multiscale && fwd_score) {
        // the caller's forward already pooled every scale: only the pyramid
        // planes are rebuilt (2x2 average pooling), the moments are recomputed below
        ms_score = fwd_score;
        ms_per = fwd_per_scale;
        ImgDesc dx = desc_of(x), dy = desc_of(y);
        int dtype = x->dtype;
        for (int j = 1; j < S; ++j) {
            const Level &N = B.fwd.lv[j];
            float *px = (float *)(ws + N.plane_off), *py = px + (size_t)N.H * N.W * n;
            if (launch_downsample(dx, dtype, n, px, st) != cudaSuccess ||
                launch_downsample(dy, dtype, n, py, st) != cudaSuccess)
                return GBSSIM_ERR_CUDA;
            dx = ImgDesc{px, N.H, N.W, N.W, N.H * N.W};
            dy = ImgDesc{py, N.H, N.W, N.W, N.H * N.W};
            dtype = GBSSIM_F32;
        }
    } else if (multiscale) {
        // the coefficient passes below read the fp32 pyramid planes
        rc = msssim_forward(x, y, p, B.fwd, ws, score, per, st, nullptr, nullptr, 0, 0, false);
        if (rc) return rc;
    }
    double esum = 0.0;
    for (int j = 0; j < S; ++j) esum += p->exponents[j];
    float *coef = (float *)(ws + B.coef_off);
    double2 *cpart = (double2 *)(ws + B.cpart_off);
    for (int j = S - 1; j >= 0; --j) {
        const Level &L = B.coef.lv[j];
        ImgDesc dx = desc_of(x), dy = desc_of(y);
        int dtype = x->dtype;
        if (j > 0) {
            const float *px = (const float *)(ws + B.fwd.lv[j].plane_off);
            dx = ImgDesc{px, L.H, L.W, L.W, L.H * L.W};
            dy = ImgDesc{px + (size_t)L.H * L.W * n, L.H, L.W, L.W, L.H * L.W};
            dtype = GBSSIM_F32;
        }
        CoefOut co;
        co.coef = coef;
        co.which = (multiscale && j < S - 1) ? 1 : 0;
        co.sx = co.sy = (float)(0.5 * p->L);
        cudaError_t e = run_level(L, dx, dy, dtype, n, p, nullptr, 0, 0, cpart, nullptr, nullptr, st, &co);
        if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
        const int64_t OH = out_dim(L.H, p->k, 1), OW = out_dim(L.W, p->k, 1);
        if (!multiscale && score_out) {
            e = launch_finalize_ssim(cpart, n, L.items, 1.0 / ((double)OH * (double)OW), score_out, st);
            if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
        }
        GradLaunch G;
        memset(&G, 0, sizeof G);
        G.x = dx;
        G.y = dy;
        G.dtype = dtype;
        G.count = n;
        G.k = p->k;
        G.coef = coef;
        make_taps(p, G.taps.g);
        G.sx = G.sy = co.sx;
        G.base_scale = grad_scale / ((double)OH * (double)OW);
        G.grad_out = grad_out;
        G.grad_out_per_image = grad_out_per_image;
        if (multiscale) {
            G.ms_score = ms_score;
            G.ms_per_scale = ms_per;
            G.ms_scales = S;
            G.ms_level = j;
            G.ms_combine = p->combine;
            G.ms_beta = p->exponents[j];
            G.ms_beta_hat = p->exponents[j] / esum;
        }
        G.coarse = j + 1 < S ? (const float *)(ws + B.grad_off[j + 1]) : nullptr;
        if (j == 0) {
            G.out = grad_y;
            G.out_dtype = grad_dtype;
            G.out_ld = grad_ld;
            G.out_is = x->count > 1 ? grad_image_stride : x->height * grad_ld;
        } else {
            G.out = ws + B.grad_off[j];
            G.out_dtype = GBSSIM_F32;
            G.out_ld = L.W;
            G.out_is = L.H * L.W;
        }
        e = launch_grad(G, st);
        if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
    }
    if (multiscale && score_out &&
        cudaMemcpyAsync(score_out, ms_score, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return GBSSIM_ERR_CUDA;
    return GBSSIM_OK;
}

int gbssim_loss_saved_size(const gbssim_plane *x, const gbssim_params *p, int32_t multiscale, size_t *bytes) {
    int rc = check_loss(x, x, p);
    if (rc) return rc;
    if (!bytes) return GBSSIM_ERR_INVALID_ARG;
    SavedPlan Sv;
    rc = plan_saved(x, p, multiscale != 0, &Sv);
    if (rc) return rc;
    *bytes = Sv.bytes;
    return GBSSIM_OK;
}

int gbssim_loss_forward(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t multiscale,
                        double *score_out, double *per_scale_out, void *saved, size_t saved_bytes, void *stream) {
    int rc = check_loss(x, y, p);
    if (rc) return rc;
    SavedPlan Sv;
    rc = plan_saved(x, p, multiscale != 0, &Sv);
    if (rc) return rc;
    if (!saved || saved_bytes < Sv.bytes) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)saved;
    const int n = x->count, S = multiscale ? p->scales : 1;
    MsFinalize F;
    memset(&F, 0, sizeof F);
    for (int j = 0; j < S; ++j) {
        const Level &L = Sv.lv.lv[j];
        ImgDesc dx = desc_of(x), dy = desc_of(y);
        int dtype = x->dtype;
        if (j > 0) {
            const float *px = (const float *)(ws + Sv.plane_off[j]);
            dx = ImgDesc{px, L.H, L.W, L.W, L.H * L.W};
            dy = ImgDesc{px + (size_t)L.H * L.W * n, L.H, L.W, L.W, L.H * L.W};
            dtype = GBSSIM_F32;
        }
        float *ds_x = nullptr, *ds_y = nullptr;
        if (j + 1 < S) {
            const Level &N = Sv.lv.lv[j + 1];
            ds_x = (float *)(ws + Sv.plane_off[j + 1]);
            ds_y = ds_x + (size_t)N.H * N.W * n;
        }
        CoefOut co;
        co.coef = (float *)(ws + Sv.coef_off[j]);
        co.which = (multiscale && j < S - 1) ? 1 : 0;
        co.sx = co.sy = (float)(0.5 * p->L);
        double2 *part = (double2 *)(ws + Sv.part_off[j]);
        if (run_level(L, dx, dy, dtype, n, p, nullptr, 0, 0, part, ds_x, ds_y, st, &co) != cudaSuccess)
            return GBSSIM_ERR_CUDA;
        const int64_t OH = out_dim(L.H, p->k, 1), OW = out_dim(L.W, p->k, 1);
        F.lv[j].partials = part;
        F.lv[j].items_per_image = L.items;
        F.lv[j].inv_n = 1.0 / ((double)OH * (double)OW);
        F.exps[j] = multiscale ? p->exponents[j] : 1.0;
    }
    double *score = (double *)(ws + Sv.score_off), *per = (double *)(ws + Sv.per_off);
    F.scales = S;
    F.count = n;
    F.combine = multiscale ? p->combine : GBSSIM_COMBINE_PRODUCT;
    F.score_out = score;
    F.per_scale_out = per;
    if (launch_finalize_msssim(F, st) != cudaSuccess) return GBSSIM_ERR_CUDA;
    if (score_out && cudaMemcpyAsync(score_out, score, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return GBSSIM_ERR_CUDA;
    if (per_scale_out &&
        cudaMemcpyAsync(per_scale_out, per, 2 * sizeof(double) * S * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return GBSSIM_ERR_CUDA;
    return GBSSIM_OK;
}

int gbssim_loss_backward(const gbssim_plane *x, const gbssim_plane *y, const gbssim_params *p, int32_t multiscale,
                         double grad_scale, const double *grad_out, int32_t grad_out_per_image, const void *saved,
                         size_t saved_bytes, void *grad_y, int32_t grad_dtype, int64_t grad_ld,
                         int64_t grad_image_stride, void *stream) {
    int rc = check_loss(x, y, p);
    if (rc) return rc;
    if (!grad_y || (grad_dtype != GBSSIM_F32 && grad_dtype != GBSSIM_F16 && grad_dtype != GBSSIM_BF16))
        return GBSSIM_ERR_INVALID_ARG;
    if (grad_ld < x->width || (x->count > 1 && grad_image_stride < x->height * grad_ld)) return GBSSIM_ERR_INVALID_ARG;
    if (!isfinite(grad_scale)) return GBSSIM_ERR_INVALID_ARG;
    SavedPlan Sv;
    rc = plan_saved(x, p, multiscale != 0, &Sv);
    if (rc) return rc;
    if (!saved || saved_bytes < Sv.bytes) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)const_cast<void *>(saved);  // the backward writes only the coarse-gradient planes
    const int n = x->count, S = multiscale ? p->scales : 1;
    double esum = 0.0;
    for (int j = 0; j < S; ++j) esum += p->exponents[j];
    for (int j = S - 1; j >= 0; --j) {
        const Level &L = Sv.lv.lv[j];
        ImgDesc dx = desc_of(x), dy = desc_of(y);
        int dtype = x->dtype;
        if (j > 0) {
            const float *px = (const float *)(ws + Sv.plane_off[j]);
            dx = ImgDesc{px, L.H, L.W, L.W, L.H * L.W};
            dy = ImgDesc{px + (size_t)L.H * L.W * n, L.H, L.W, L.W, L.H * L.W};
            dtype = GBSSIM_F32;
        }
        const int64_t OH = out_dim(L.H, p->k, 1), OW = out_dim(L.W, p->k, 1);
        GradLaunch G;
        memset(&G, 0, sizeof G);
        G.x = dx;
        G.y = dy;
        G.dtype = dtype;
        G.count = n;
        G.k = p->k;
        G.coef = (const float *)(ws + Sv.coef_off[j]);
        make_taps(p, G.taps.g);
        G.sx = G.sy = (float)(0.5 * p->L);
        G.base_scale = grad_scale / ((double)OH * (double)OW);
        G.grad_out = grad_out;
        G.grad_out_per_image = grad_out_per_image;
        if (multiscale) {
            G.ms_score = (const double *)(ws + Sv.score_off);
            G.ms_per_scale = (const double *)(ws + Sv.per_off);
            G.ms_scales = S;
            G.ms_level = j;
            G.ms_combine = p->combine;
            G.ms_beta = p->exponents[j];
            G.ms_beta_hat = p->exponents[j] / esum;
        }
        G.coarse = j + 1 < S ? (const float *)(ws + Sv.grad_off[j + 1]) : nullptr;
        if (j == 0) {
            G.out = grad_y;
            G.out_dtype = grad_dtype;
            G.out_ld = grad_ld;
            G.out_is = x->count > 1 ? grad_image_stride : x->height * grad_ld;
        } else {
            G.out = ws + Sv.grad_off[j];
            G.out_dtype = GBSSIM_F32;
            G.out_ld = L.W;
            G.out_is = L.H * L.W;
        }
        if (launch_grad(G, st) != cudaSuccess) return GBSSIM_ERR_CUDA;
    }
    return GBSSIM_OK;
}

// Workspace of gbssim_video: per-plane SSIM partials, then the per-plane
// frame means (3 x frames doubles).
static int plan_video(const gbssim_plane planes[6], const gbssim_params *p, MsPlan P[3], size_t offs[4],
                      size_t *bytes) {
    size_t off = 0;
    for (int q = 0; q < 3; ++q) {
        int rc = plan_levels(&planes[2 * q], p, 1, &P[q]);
        if (rc) return rc;
        offs[q] = off;
        off = align_up(off + P[q].bytes);
    }
    offs[3] = off;
    off = align_up(off + 3 * sizeof(double) * planes[0].count);
    *bytes = off;
    return GBSSIM_OK;
}

int gbssim_video_workspace_size(const gbssim_plane planes[6], const gbssim_params *p, size_t *bytes) {
    if (!planes || !bytes) return GBSSIM_ERR_INVALID_ARG;
    for (int q = 0; q < 3; ++q) {
        int rc = check_pair(&planes[2 * q], &planes[2 * q + 1]);
        if (rc) return rc;
    }
    int rc = check_params_valid(p);
    if (rc) return rc;
    MsPlan P[3];
    size_t offs[4];
    return plan_video(planes, p, P, offs, bytes);
}

int gbssim_video(const gbssim_plane planes[6], const gbssim_params *p, const double weights[3], double percentile,
                 double pp_r, double *frame_out, double *plane_out, double *video_out, void *workspace,
                 size_t workspace_bytes, void *stream) {
    if (!planes || !weights || !video_out) return GBSSIM_ERR_INVALID_ARG;
    for (int q = 0; q < 3; ++q) {
        int rc = check_pair(&planes[2 * q], &planes[2 * q + 1]);
        if (rc) return rc;
        if (planes[2 * q].count != planes[0].count) return GBSSIM_ERR_INVALID_ARG;
    }
    int rc = check_params_valid(p);
    if (rc) return rc;
    const int n = planes[0].count;
    if (n > kVideoMaxFrames) return GBSSIM_ERR_UNSUPPORTED;
    if (!(percentile >= 0.0 && percentile <= 100.0) || !(pp_r > 0.0) || !isfinite(pp_r)) return GBSSIM_ERR_INVALID_ARG;
    const double wsum = weights[0] + weights[1] + weights[2];
    if (!isfinite(wsum) || wsum == 0.0) return GBSSIM_ERR_INVALID_ARG;
    MsPlan P[3];
    size_t offs[4], need;
    rc = plan_video(planes, p, P, offs, &need);
    if (rc) return rc;
    if (!workspace || workspace_bytes < need) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    double *means = plane_out ? plane_out : (double *)(ws + offs[3]);
    for (int q = 0; q < 3; ++q) {
        const gbssim_plane *x = &planes[2 * q], *y = &planes[2 * q + 1];
        Level L = P[q].lv[0];
        fix_box_items(L, desc_of(x), desc_of(y), p);
        double2 *part = (double2 *)(ws + offs[q] + L.part_off);
        cudaError_t e = run_level(L, desc_of(x), desc_of(y), x->dtype, n, p, nullptr, 0, 0, part, nullptr, nullptr, st);
        if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
        const int64_t OH = out_dim(x->height, p->k, p->stride), OW = out_dim(x->width, p->k, p->stride);
        e = launch_finalize_ssim(part, n, L.items, 1.0 / ((double)OH * (double)OW), means + (size_t)q * n, st);
        if (e != cudaSuccess) return GBSSIM_ERR_CUDA;
    }
    return launch_video_pool(means, means + n, means + 2 * (size_t)n, n, weights, percentile, pp_r, frame_out,
                             video_out, st) == cudaSuccess
               ? GBSSIM_OK
               : GBSSIM_ERR_CUDA;
}

int gbssim_window_sums(const gbssim_plane *x, const gbssim_plane *y, int32_t k, int32_t stride,
                       int64_t *sums_out, void *stream) {
    return gbssim_window_sums_ex(x, y, k, stride, 0, sums_out, stream);
}

int gbssim_window_sums_ex(const gbssim_plane *x, const gbssim_plane *y, int32_t k, int32_t stride, int32_t flags,
                          int64_t *sums_out, void *stream) {
    int rc = check_pair(x, y);
    if (rc) return rc;
    if (x->dtype != GBSSIM_U8) return GBSSIM_ERR_UNSUPPORTED;
    if (!sums_out || k < 1 || k > GBSSIM_MAX_K || stride < 1) return GBSSIM_ERR_INVALID_ARG;
    if (x->height < k || x->width < k) return GBSSIM_ERR_TOO_SMALL;
    BoxLaunch B;
    memset(&B, 0, sizeof B);
    B.x = desc_of(x);
    B.y = desc_of(y);
    B.count = x->count;
    B.k = k;
    B.stride = stride;
    B.sums_out = sums_out;
    B.use_tma = (flags & GBSSIM_FLAG_BOX_TMA) != 0;
    return launch_box_u8(B, (cudaStream_t)stream) == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

}  // extern "C"
