// Host-side helpers of libgs: version, status text, camera tables, workspace layout.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace gs {

bool make_view_table(const gs_camera *cams, int n_views, int64_t n, ViewTable *vt) {
    if (!cams || n_views < 1 || n_views > kMaxViews || n < 0) return false;
    memset(vt, 0, sizeof(*vt));
    vt->n_views = n_views;
    vt->n = n;
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 32768 || c.height > 32768) return false;
        if (!(c.fx > 0) || !(c.fy > 0) || !isfinite(c.cx) || !isfinite(c.cy)) return false;
        for (int k = 0; k < 16; ++k)
            if (!isfinite(c.T_cw[k])) return false;
        vt->tile_off[v] = (int)tiles;
        vt->pix_off[v] = pix;
        vt->W[v] = c.width;
        vt->H[v] = c.height;
        vt->TX[v] = (c.width + kTile - 1) / kTile;
        vt->TY[v] = (c.height + kTile - 1) / kTile;
        vt->fx[v] = c.fx; vt->fy[v] = c.fy; vt->cx[v] = c.cx; vt->cy[v] = c.cy;
        for (int k = 0; k < 12; ++k) vt->T[v][k] = c.T_cw[k];
        vt->jx_lo[v] = (float)((-(double)c.cx - 0.15 * c.width) / c.fx);
        vt->jx_hi[v] = (float)(((double)c.width - c.cx + 0.15 * c.width) / c.fx);
        vt->jy_lo[v] = (float)((-(double)c.cy - 0.15 * c.height) / c.fy);
        vt->jy_hi[v] = (float)(((double)c.height - c.cy + 0.15 * c.height) / c.fy);
        tiles += (int64_t)vt->TX[v] * vt->TY[v];
        pix += (int64_t)c.width * c.height;
    }
    if (tiles >= (1 << 24)) return false;
    vt->tile_off[n_views] = (int)tiles;
    vt->pix_off[n_views] = pix;
    return true;
}

bool make_params(const gs_raster_params *p, Params *out) {
    if (!p) return false;
    if (p->tile != kTile) return false;
    if (!(p->alpha_min >= 0) || !(p->alpha_max > 0) || !(p->T_min >= 0) || !(p->radius_sigma > 0) ||
        !(p->lowpass >= 0) || !isfinite(p->z_near))
        return false;
    out->alpha_min = p->alpha_min;
    out->alpha_max = p->alpha_max;
    out->T_min = p->T_min;
    out->z_near = p->z_near;
    out->lowpass = p->lowpass;
    out->radius_sigma = p->radius_sigma;
    for (int k = 0; k < 3; ++k) out->bg[k] = p->bg_rgb[k];
    auto np_ok = [](int np) { return np == 0 || np == 1 || np == 2 || np == 4; };
    if (!np_ok(p->fwd_px_per_thread) || !np_ok(p->bwd_px_per_thread)) return false;
    out->fwd_np = p->fwd_px_per_thread;
    out->bwd_np = p->bwd_px_per_thread;
    if (p->bwd_blocks < GS_BWD_BLOCKS_DEFAULT || p->bwd_blocks > GS_BWD_BLOCKS_TILE) return false;
    out->bwd_blocks = p->bwd_blocks;
    out->bwd_warp = false;
    if (p->fwd_blocks < GS_BWD_BLOCKS_DEFAULT || p->fwd_blocks > GS_BLOCKS_RING) return false;
    out->fwd_blocks = p->fwd_blocks;
    out->fwd_group = false;
    out->fwd_ring = false;
    if (p->jacobian != GS_JACOBIAN_CLAMPED && p->jacobian != GS_JACOBIAN_EXACT) return false;
    out->exact_jacobian = p->jacobian == GS_JACOBIAN_EXACT;
    out->spin_limit = p->spin_limit == 0 ? kDefaultSpinLimit : (p->spin_limit < 0 ? -1 : p->spin_limit);
    if (p->fwd_batch != 0 && p->fwd_batch != 64 && p->fwd_batch != 128 && p->fwd_batch != 256) return false;
    out->fwd_batch = p->fwd_batch ? p->fwd_batch : 128;
    return true;
}

void apply_jacobian_mode(const Params &prm, ViewTable *vt) {
    if (!prm.exact_jacobian) return;
    for (int v = 0; v < vt->n_views; ++v) {
        vt->jx_lo[v] = vt->jy_lo[v] = -INFINITY;
        vt->jx_hi[v] = vt->jy_hi[v] = INFINITY;
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(int64_t n, int n_views, int64_t capacity, const ViewTable *vt) {
    WsLayout L;
    memset(&L, 0, sizeof(L));
    int64_t vn = n * n_views;
    L.vn = vn;
    L.capacity = capacity;
    int64_t scan_n = vn > capacity ? vn : capacity;
    int64_t nb1 = (scan_n + 255) / 256 + 1;  // block sums of the 256-item emission blocks (the largest use)
    L.lb_tiles_depth = (int)((vn + depth_sort_tile(vn) - 1) / depth_sort_tile(vn));
    L.lb_tiles_inst = (int)((capacity + kSortTileInst - 1) / kSortTileInst);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L.scan_blocks = take(sizeof(uint32_t) * (size_t)nb1);
    L.emit_sums = take(sizeof(uint32_t) * (size_t)((vn + 255) / 256 + 1));
    L.counters = take(sizeof(uint32_t) * 64);
    L.dkeys_a = take(sizeof(uint32_t) * (size_t)vn);
    L.dvals_a = take(sizeof(uint32_t) * (size_t)vn);
    L.dkeys_b = take(sizeof(uint32_t) * (size_t)vn);
    L.dvals_b = take(sizeof(uint32_t) * (size_t)vn);
    L.tkeys_a = take(sizeof(uint32_t) * (size_t)capacity);
    L.tkeys_b = take(sizeof(uint32_t) * (size_t)capacity);
    L.tvals_b = take(sizeof(uint32_t) * (size_t)capacity);
    L.hist = take(sizeof(uint32_t) * 8 * 256);
    L.lookback = take(sizeof(uint32_t) * 256 * ((size_t)4 * L.lb_tiles_depth + (size_t)3 * L.lb_tiles_inst));
    L.tile_counts = take(sizeof(uint32_t) * (vt ? (size_t)vt->tile_off[vt->n_views] : 0));
    L.bin_end = off;
    off = 0;
    L.med_hist = take(sizeof(uint32_t) * 4 * 256 * (size_t)n_views);
    L.loss_part_f = take(sizeof(float) * (size_t)kLossBlocks * (32 * 32 + 32));
    const int64_t P = vt ? vt->pix_off[vt->n_views] : 0;
    const int ssim_rows = vt ? ssim_blocks(*vt) : 0;
    L.loss_part_d = take(sizeof(double) * ((size_t)kLossBlocks + ssim_rows) * 3);
    L.dsr_part = take(sizeof(double) * 512 * 6 + 2 * sizeof(uint32_t));  // partials + two arrival counters
    L.ssim_maps = take(sizeof(float) * 9 * (size_t)P);
    L.expand_counts = take(sizeof(uint32_t) * 2 * (vt ? (size_t)vt->n_views * expand_blocks_x(*vt) : 0));
    L.misc_end = off;
    L.total = L.bin_end;
    if (L.misc_end > L.total) L.total = L.misc_end;
    return L;
}

}  // namespace gs

namespace gs {
thread_local cudaError_t g_last_cuda_error = cudaSuccess;
}  // namespace gs

extern "C" {

int gs_version(void) { return 10000; }

const char *gs_cuda_error(void) { return cudaGetErrorString(gs::g_last_cuda_error); }

const char *gs_strerror(int status) {
    switch (status) {
        case GS_OK: return "ok";
        case GS_ERR_ARG: return "invalid argument";
        case GS_ERR_CAPACITY: return "tile instance count exceeds the binning capacity";
        case GS_ERR_CUDA: return "CUDA runtime error";
        case GS_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        case GS_ERR_UNSUPPORTED: return "unsupported configuration";
        case GS_ERR_CHECK: return "a checked build found an index out of range";
        default: return "unknown status";
    }
}

size_t gs_workspace_size(int64_t n, int n_views, const gs_camera *cams, int64_t inst_capacity,
                         int feat_dim) {
    gs::ViewTable vt;
    if (!gs::make_view_table(cams, n_views, n, &vt)) return 0;
    if (inst_capacity < 0 || inst_capacity >= (int64_t)1 << 30 || !gs::feat_dim_ok(feat_dim)) return 0;
    if (n * n_views >= (int64_t)1 << 30) return 0;
    return gs::ws_layout(n, n_views, inst_capacity, &vt).total;
}

}  // extern "C"
