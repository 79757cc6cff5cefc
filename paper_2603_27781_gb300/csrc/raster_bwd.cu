// Entry point of the blend backward (kernels in raster_bwd.cuh, instantiated by
// raster_bwd_map.cu and raster_bwd_pose.cu).
#include "raster_bwd_warp.cuh"

namespace gs {
bool storage_ok(const gs_gaussians *g);
}  // namespace gs

namespace gs {
// Zeroes the sums gs_render_bwd accumulates into (vn = n_views * g->n items).
static gs_status clear_splat_grads(const gs_gaussians *g, int64_t vn, bool map, gs_splat_grads *sg, float *d_feat,
                                   cudaStream_t st) {
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(sg->uvod, 0, sizeof(float4) * vn, st)))) return s;
    if ((s = cuda_status(cudaMemsetAsync(sg->conic, 0, sizeof(float4) * vn, st)))) return s;
    if (map) {
        if ((s = cuda_status(cudaMemsetAsync(sg->rgb, 0, sizeof(float4) * g->n, st)))) return s;
        if (g->feat_dim && (s = cuda_status(cudaMemsetAsync(d_feat, 0, sizeof(float) * g->feat_dim * g->n, st))))
            return s;
    }
    return GS_OK;
}
}  // namespace gs

extern "C" gs_status gs_splat_grads_clear(const gs_gaussians *g, int n_views, int grad_mode, gs_splat_grads *sg,
                                          float *d_feat, gs_stream stream) {
    GS_NVTX_RANGE("gs_splat_grads_clear");
    using namespace gs;
    if (!g || !sg || g->n < 0 || n_views < 1 || n_views > kMaxViews) return GS_ERR_ARG;
    if ((grad_mode & ~(GS_GRAD_MAP | GS_GRAD_POSE | GS_GRAD_ACCUMULATE)) || !(grad_mode & (GS_GRAD_MAP | GS_GRAD_POSE)))
        return GS_ERR_ARG;
    if (!feat_dim_ok(g->feat_dim)) return GS_ERR_UNSUPPORTED;
    const bool map = grad_mode & GS_GRAD_MAP;
    if (g->n == 0) return GS_OK;
    if (!sg->uvod || !sg->conic || (map && (!sg->rgb || (g->feat_dim && !d_feat)))) return GS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(sg->uvod) | reinterpret_cast<uintptr_t>(sg->conic) |
         reinterpret_cast<uintptr_t>(sg->rgb) | reinterpret_cast<uintptr_t>(d_feat)) & 15)
        return GS_ERR_ARG;
    return clear_splat_grads(g, (int64_t)n_views * g->n, map, sg, d_feat, (cudaStream_t)stream);
}

extern "C" gs_status gs_render_bwd(const gs_gaussians *g, const gs_projected *proj, const gs_binning *bins,
                                   const gs_camera *cams, int n_views, const gs_raster_params *p, int grad_mode,
                                   const gs_images *fwd, const gs_image_grads *dL, gs_splat_grads *sg, float *d_feat,
                                   gs_stream stream) {
    GS_NVTX_RANGE("gs_render_bwd");
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    if (!g || !proj || !bins || !fwd || !dL || !sg || g->n < 0) return GS_ERR_ARG;
    if ((grad_mode & ~(GS_GRAD_MAP | GS_GRAD_POSE | GS_GRAD_ACCUMULATE)) || !(grad_mode & (GS_GRAD_MAP | GS_GRAD_POSE)))
        return GS_ERR_ARG;
    const bool accumulate = grad_mode & GS_GRAD_ACCUMULATE;
    ViewTable vt;
    Params prm;
    if (!make_view_table(cams, n_views, g->n, &vt) || !make_params(p, &prm)) return GS_ERR_ARG;
    if (!feat_dim_ok(g->feat_dim)) return GS_ERR_UNSUPPORTED;
    const bool map = grad_mode & GS_GRAD_MAP;
    if (g->n == 0) return GS_OK;
    if (!storage_ok(g)) return GS_ERR_UNSUPPORTED;
    if (!sg->uvod || !sg->conic || (map && (!sg->rgb || (g->feat_dim && !d_feat)))) return GS_ERR_ARG;
    const bool factored = dL->feat_basis != nullptr;
    if (!proj->uvdo || !proj->uv_lo || !proj->conic || !bins->vals || !bins->ranges || !fwd->T_final || !fwd->n_contrib ||
        !dL->rgb || !dL->depth || (g->feat_dim && !factored && !dL->feat) || (factored && !dL->feat_coef))
        return GS_ERR_ARG;
    if (factored && (dL->feat_rank < 1 || dL->feat_rank > kFactorK)) return GS_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(sg->uvod) | reinterpret_cast<uintptr_t>(sg->conic) |
         reinterpret_cast<uintptr_t>(sg->rgb) | reinterpret_cast<uintptr_t>(d_feat)) & 15)
        return GS_ERR_ARG;
    if (g->feat_dim && (reinterpret_cast<uintptr_t>(g->feat) & 15)) return GS_ERR_ARG;
    const int64_t vn = g->n * n_views;
    float4 *acc_uvod = reinterpret_cast<float4 *>(sg->uvod);
    float4 *acc_conic = reinterpret_cast<float4 *>(sg->conic);
    float4 *acc_rgb = reinterpret_cast<float4 *>(sg->rgb);
    gs_status s;
    if (!accumulate && (s = clear_splat_grads(g, vn, map, sg, d_feat, st))) return s;
    BwdArgs A;
    A.uvdo = reinterpret_cast<const float4 *>(proj->uvdo);
    A.uv_lo = reinterpret_cast<const float2 *>(proj->uv_lo);
    A.conic = reinterpret_cast<const float4 *>(proj->conic);
    A.rgb = g->rgb;
    A.feat = g->feat;
    A.vals = bins->vals;
    A.ranges = bins->ranges;
    A.P = vt.pix_off[n_views];
    A.T_final = fwd->T_final;
    A.n_contrib = fwd->n_contrib;
    A.g_rgb = dL->rgb;
    A.g_depth = dL->depth;
    A.g_sil = dL->sil;
    A.g_feat = dL->feat;
    A.feat_coef = factored ? dL->feat_coef : nullptr;
    A.feat_basis = factored ? dL->feat_basis : nullptr;
    A.feat_rank = factored ? dL->feat_rank : 0;
    A.acc_uvod = acc_uvod;
    A.acc_conic = acc_conic;
    A.acc_rgb = acc_rgb;
    A.d_feat = map ? d_feat : nullptr;
    A.bmask = fwd->blend_mask;
    A.bm_stride = bins->capacity / 32 + 1;
    A.order = bins->tile_order;
    A.status = bins->status;
    A.capacity = bins->capacity;
    // block shape: per pixel group where that form applies (D 16 or 32, the blend mask,
    // 1 or 2 pixels per thread), unless the caller asks for one
    const int D = g->feat_dim;
    const bool group_ok = (D == 16 || D == 32) && A.bmask && prm.bwd_np <= 2;
    Params pr = prm;
    pr.bwd_warp = prm.bwd_blocks == GS_BWD_BLOCKS_GROUP || (prm.bwd_blocks == GS_BWD_BLOCKS_DEFAULT && group_ok);
    if (factored && !pr.bwd_warp) return GS_ERR_UNSUPPORTED;  // the tile kernel takes the features' gradient
    // default pixels per thread: 2 for the per-group form at D = 16 (8x8 blocks), else 1
    const int np = prm.bwd_np ? prm.bwd_np : (pr.bwd_warp ? (D == 16 ? 2 : 1) : default_bwd_np(D));
    const bool half = g->rgb_dtype == GS_F16;
    return map ? dispatch_bwd_map(D, np, half, vt, pr, A, st) : dispatch_bwd_pose(D, np, half, vt, pr, A, st);
}
