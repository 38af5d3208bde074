// batch.cu -- host side of the ragged persistent batch (gbssim_batch_*).
//
// gbssim_batch_plan builds, once, the device tables the persistent kernel
// walks: one BatchLevel per (image, pyramid level) and one BatchItem per
// (image, level, strip, segment), listed level-major so that every item an
// item depends on is handed out before it.  The tables live in one device
// allocation owned by the plan (the only allocation the library makes, freed
// by gbssim_batch_free).  gbssim_batch_run only enqueues a memset, the
// persistent kernel and the finaliser, so it can be captured in a CUDA graph
// and replayed; the plan is bound to the input pointers it was built with.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"

using namespace gbssim;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

}  // namespace

struct gbssim_batch {
    int device;
    int n_images, scales, dtype, combine;
    double exps[GBSSIM_MAX_SCALES];
    gbssim_params params;
    int seg_rows, ctas_per_sm, grid, tile_w;
    unsigned wait_limit;
    int total_items;
    size_t ws_bytes;
    int64_t counter_off, done_off, status_off, zero_bytes;
    void *d_table;
    BatchLevel *d_levels;
    BatchItem *d_items;
};

extern "C" {

int gbssim_batch_plan(const gbssim_plane *xs, const gbssim_plane *ys, int32_t n, const gbssim_params *p,
                      int32_t multiscale, const gbssim_tuning *tuning, gbssim_batch **plan_out) {
    if (!xs || !ys || !p || !plan_out || n < 1) return GBSSIM_ERR_INVALID_ARG;
    *plan_out = nullptr;
    if (p->window != GBSSIM_WIN_GAUSSIAN && p->window != GBSSIM_WIN_BOX) return GBSSIM_ERR_INVALID_ARG;
    if (p->k != 11 || p->stride != 1) return GBSSIM_ERR_UNSUPPORTED;
    if (p->flags & (GBSSIM_FLAG_PYRAMID_97 | GBSSIM_FLAG_BORDER_ZERO | GBSSIM_FLAG_BORDER_REFLECT))
        return GBSSIM_ERR_UNSUPPORTED;  // the persistent kernel fuses the 2x2 pyramid into valid-window levels
    if (!(p->L > 0.0) || p->K1 < 0.0 || p->K2 < 0.0 || p->flags != 0) return GBSSIM_ERR_INVALID_ARG;
    if (p->window == GBSSIM_WIN_GAUSSIAN && !(p->sigma > 0.0)) return GBSSIM_ERR_INVALID_ARG;
    const int S = multiscale ? p->scales : 1;
    if (S < 1 || S > GBSSIM_MAX_SCALES) return GBSSIM_ERR_INVALID_ARG;
    if (multiscale && (p->combine != GBSSIM_COMBINE_PRODUCT && p->combine != GBSSIM_COMBINE_SUM))
        return GBSSIM_ERR_INVALID_ARG;

    int seg_rows = 256, ctas = 0, tile_w = 64;
    unsigned wait_limit = 1u << 22;
    int flags = 0;
    if (tuning) {
        if (tuning->seg_rows) seg_rows = tuning->seg_rows;
        ctas = tuning->ctas_per_sm;
        if (tuning->wait_limit) wait_limit = tuning->wait_limit;
        flags = tuning->flags;
        if (tuning->tile_w) tile_w = tuning->tile_w;
    }
    if (seg_rows < 16 || seg_rows > 4096 || seg_rows % 16 != 0 || ctas < 0) return GBSSIM_ERR_INVALID_ARG;
    if (tile_w != 32 && tile_w != 64 && tile_w != 128) return GBSSIM_ERR_INVALID_ARG;

    // expand entries into images
    const int dtype = xs[0].dtype;
    std::vector<gbssim_plane> ix, iy;
    for (int e = 0; e < n; ++e) {
        const gbssim_plane &a = xs[e], &b = ys[e];
        if (!a.data || !b.data || a.count < 1 || a.count != b.count) return GBSSIM_ERR_INVALID_ARG;
        if (a.dtype != dtype || b.dtype != dtype) return GBSSIM_ERR_INVALID_ARG;
        if (a.height != b.height || a.width != b.width || a.row_stride != b.row_stride) return GBSSIM_ERR_INVALID_ARG;
        if (a.width < 1 || a.height < 1 || a.row_stride < a.width) return GBSSIM_ERR_INVALID_ARG;
        if (a.count > 1 && (a.image_stride < a.height * a.row_stride || a.image_stride != b.image_stride))
            return GBSSIM_ERR_INVALID_ARG;
        const size_t esz = dtype == GBSSIM_U8 ? 1 : dtype == GBSSIM_F32 ? 4 : 2;
        for (int c = 0; c < a.count; ++c) {
            gbssim_plane pa = a, pb = b;
            pa.data = static_cast<const char *>(a.data) + esz * (size_t)c * a.image_stride;
            pb.data = static_cast<const char *>(b.data) + esz * (size_t)c * b.image_stride;
            pa.count = pb.count = 1;
            ix.push_back(pa);
            iy.push_back(pb);
        }
    }
    const int N = (int)ix.size();
    if (N > 65535) return GBSSIM_ERR_UNSUPPORTED;
    const size_t esz = dtype == GBSSIM_U8 ? 1 : dtype == GBSSIM_F32 ? 4 : 2;

    std::vector<BatchLevel> lv((size_t)N * S);
    size_t off = 0;
    for (int i = 0; i < N; ++i) {
        int64_t H = ix[i].height, W = ix[i].width;
        for (int j = 0; j < S; ++j) {
            if (H < p->k || W < p->k) return GBSSIM_ERR_TOO_SMALL;
            BatchLevel &L = lv[(size_t)i * S + j];
            memset(&L, 0, sizeof L);
            L.level = j;
            L.H = H;
            L.W = W;
            if (j == 0) {
                L.x = ix[i].data;
                L.y = iy[i].data;
                L.rs = ix[i].row_stride;
                const uintptr_t vb = 4 * esz;
                L.vec = ((uintptr_t)L.x % vb == 0) && ((uintptr_t)L.y % vb == 0) && (L.rs % 4 == 0);
                L.x_off = -1;
            } else {
                L.rs = W;
                L.vec = W % 4 == 0;
                L.x_off = (int64_t)off;
                off = align_up(off + 2 * sizeof(float) * (size_t)H * W);
            }
            L.seg_rows = seg_rows;
            L.strips = (int)((W - 10 + tile_w - 1) / tile_w);
            L.segs = (int)((H - 10 + seg_rows - 1) / seg_rows);
            L.items = L.strips * L.segs;
            L.wait_target = L.items;
            H >>= 1;
            W >>= 1;
        }
        for (int j = 0; j < S; ++j) lv[(size_t)i * S + j].ds_off = j + 1 < S ? lv[(size_t)i * S + j + 1].x_off : -1;
    }
    if ((flags & GBSSIM_TUNING_TEST_STALL) && S > 1) lv[0].wait_target = lv[0].items + 1;
    for (auto &L : lv) {
        L.part_off = (int64_t)off;
        off = align_up(off + sizeof(double2) * (size_t)L.items);
    }
    const int64_t counter_off = (int64_t)off;
    const int64_t done_off = counter_off + 16;
    const int64_t status_off = done_off + (int64_t)sizeof(unsigned) * N * S;
    const int64_t zero_bytes = status_off + 16 - counter_off;
    off = align_up((size_t)(counter_off + zero_bytes));

    std::vector<BatchItem> items;
    for (int j = 0; j < S; ++j)
        for (int i = 0; i < N; ++i) {
            const BatchLevel &L = lv[(size_t)i * S + j];
            for (int sg = 0; sg < L.segs; ++sg)
                for (int st = 0; st < L.strips; ++st) items.push_back(BatchItem{i * S + j, st, sg, 0});
        }

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GBSSIM_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GBSSIM_ERR_CUDA;
    const int max_ctas = gauss11_batch_max_ctas_per_sm(dtype, true, tile_w);
    if (max_ctas < 1) return GBSSIM_ERR_CUDA;
    if (ctas == 0 || ctas > max_ctas) ctas = max_ctas;

    gbssim_batch *B = new (std::nothrow) gbssim_batch;
    if (!B) return GBSSIM_ERR_INVALID_ARG;
    memset(B, 0, sizeof *B);
    B->device = dev;
    B->n_images = N;
    B->scales = S;
    B->dtype = dtype;
    B->combine = multiscale ? p->combine : GBSSIM_COMBINE_PRODUCT;
    for (int j = 0; j < S; ++j) B->exps[j] = multiscale ? p->exponents[j] : 1.0;
    B->params = *p;
    B->seg_rows = seg_rows;
    B->tile_w = tile_w;
    B->ctas_per_sm = ctas;
    B->grid = sms * ctas;
    B->wait_limit = wait_limit;
    B->total_items = (int)items.size();
    B->ws_bytes = off;
    B->counter_off = counter_off;
    B->done_off = done_off;
    B->status_off = status_off;
    B->zero_bytes = zero_bytes;
    const size_t lv_bytes = align_up(sizeof(BatchLevel) * lv.size());
    const size_t it_bytes = sizeof(BatchItem) * items.size();
    if (cudaMalloc(&B->d_table, lv_bytes + it_bytes) != cudaSuccess) {
        delete B;
        return GBSSIM_ERR_CUDA;
    }
    B->d_levels = static_cast<BatchLevel *>(B->d_table);
    B->d_items = reinterpret_cast<BatchItem *>(static_cast<char *>(B->d_table) + lv_bytes);
    if (cudaMemcpy(B->d_levels, lv.data(), sizeof(BatchLevel) * lv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_items, items.data(), it_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(B->d_table);
        delete B;
        return GBSSIM_ERR_CUDA;
    }
    *plan_out = B;
    return GBSSIM_OK;
}

int gbssim_batch_workspace_size(const gbssim_batch *plan, size_t *bytes) {
    if (!plan || !bytes) return GBSSIM_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return GBSSIM_OK;
}

int gbssim_batch_info(const gbssim_batch *plan, int32_t *n_images, int32_t *total_items, int32_t *grid,
                      int32_t *seg_rows) {
    if (!plan) return GBSSIM_ERR_INVALID_ARG;
    if (n_images) *n_images = plan->n_images;
    if (total_items) *total_items = plan->total_items;
    if (grid) *grid = plan->grid;
    if (seg_rows) *seg_rows = plan->seg_rows;
    return GBSSIM_OK;
}

int gbssim_batch_run(const gbssim_batch *plan, double *scores_out, double *per_scale_out, void *workspace,
                     size_t workspace_bytes, void *stream) {
    if (!plan || !scores_out) return GBSSIM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < plan->ws_bytes) return GBSSIM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = static_cast<char *>(workspace);
    if (cudaMemsetAsync(ws + plan->counter_off, 0, (size_t)plan->zero_bytes, st) != cudaSuccess)
        return GBSSIM_ERR_CUDA;
    BatchTable T;
    T.levels = plan->d_levels;
    T.items = plan->d_items;
    T.ws = ws;
    T.counter_off = plan->counter_off;
    T.done_off = plan->done_off;
    T.status_off = plan->status_off;
    T.total_items = plan->total_items;
    T.n_images = plan->n_images;
    T.scales = plan->scales;
    T.dtype = plan->dtype;
    T.tile_w = plan->tile_w;
    T.wait_limit = plan->wait_limit;
    const gbssim_params *p = &plan->params;
    Taps<11> taps;
    {
        double v[11], z = 0.0;
        for (int t = 0; t < 11; ++t) {
            v[t] = p->window == GBSSIM_WIN_BOX ? 1.0 : exp(-((t - 5.0) * (t - 5.0)) / (2.0 * p->sigma * p->sigma));
            z += v[t];
        }
        for (int t = 0; t < 11; ++t) taps.g[t] = (float)(v[t] / z);
    }
    const double c1 = (p->K1 * p->L) * (p->K1 * p->L), c2 = (p->K2 * p->L) * (p->K2 * p->L);
    const SsimConst cc = ssim_const(c1, c2);
    if (launch_batch(T, taps, cc, plan->grid, st) != cudaSuccess) return GBSSIM_ERR_CUDA;
    BatchFinalize F;
    memset(&F, 0, sizeof F);
    F.levels = plan->d_levels;
    F.ws = ws;
    F.n_images = plan->n_images;
    F.scales = plan->scales;
    F.combine = plan->combine;
    for (int j = 0; j < plan->scales; ++j) F.exps[j] = plan->exps[j];
    F.score_out = scores_out;
    F.per_scale_out = per_scale_out;
    return launch_finalize_batch(F, st) == cudaSuccess ? GBSSIM_OK : GBSSIM_ERR_CUDA;
}

int gbssim_batch_status(const gbssim_batch *plan, const void *workspace, int32_t *status_out, void *stream) {
    if (!plan || !workspace || !status_out) return GBSSIM_ERR_INVALID_ARG;
    const char *ws = static_cast<const char *>(workspace);
    return cudaMemcpyAsync(status_out, ws + plan->status_off, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream) == cudaSuccess
               ? GBSSIM_OK
               : GBSSIM_ERR_CUDA;
}

void gbssim_batch_free(gbssim_batch *plan) {
    if (!plan) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != plan->device) cudaSetDevice(plan->device);
    cudaFree(plan->d_table);
    if (cur != plan->device) cudaSetDevice(cur);
    delete plan;
}

}  // extern "C"
