// Forward blend (GS3LAM Eq. 4-7 and 10): one CTA per 16x16 tile, one thread per
// pixel.  Splats of the tile are staged 256 at a time in shared memory (one
// coalesced-per-thread record each) and read back as broadcasts; every thread
// walks them front to back and stops at the T_min threshold; the CTA leaves
// as soon as all of its pixels are done.
#include "raster.cuh"

namespace gs {
namespace {

constexpr int kBatch = 256;

template <int D, typename RT, typename FT>
__global__ void __launch_bounds__(kTilePix) raster_fwd_kernel(ViewTable vt, Params prm, const float4 *__restrict__ uvdo,
                                                              const float2 *__restrict__ uv_lo,
                                                              const float4 *__restrict__ conic,
                                                              const RT *__restrict__ rgb, const FT *__restrict__ feat,
                                                              const uint32_t *__restrict__ vals,
                                                              const uint32_t *__restrict__ ranges, int64_t P,
                                                              float *o_rgb, float *o_depth, float *o_sil, float *o_feat,
                                                              float *o_T, int32_t *o_nc, int32_t *o_nb) {
    constexpr int D4 = D / 4;
    __shared__ SplatGeo s_geo[kBatch];
    __shared__ float4 s_rgb[kBatch];
    __shared__ float4 s_feat[kBatch * (D4 > 0 ? D4 : 1)];

    const int gt = blockIdx.x;
    const int v = view_of_tile(vt, gt);
    const int t = gt - vt.tile_off[v];
    const int tx = t % vt.TX[v], ty = t / vt.TX[v];
    const int tid = threadIdx.x;
    int px, py;
    tile_pixel(tid, tx, ty, px, py);
    const bool inside = px < vt.W[v] && py < vt.H[v];
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const uint32_t start = ranges[2 * gt], end = ranges[2 * gt + 1];
    const int64_t voff = (int64_t)v * vt.n;

    float T = 1.f, acc_r = 0.f, acc_g = 0.f, acc_b = 0.f, acc_d = 0.f, acc_s = 0.f;
    float acc_f[D > 0 ? D : 1];
#pragma unroll
    for (int d = 0; d < (D > 0 ? D : 1); ++d) acc_f[d] = 0.f;
    int last = 0, blended = 0;
    bool done = !inside;

    for (uint32_t b0 = start; b0 < end; b0 += kBatch) {
        if (__syncthreads_count(!done) == 0) break;
        uint32_t j = b0 + tid;
        if (j < end) {
            uint32_t item = vals[j];
            int64_t g = (int64_t)item - voff;
            const float4 a = uvdo[item];
            s_geo[tid] = make_geo(a, uv_lo[item], conic[item]);
            s_rgb[tid] = load_rgbd(rgb, g, a.z);
#pragma unroll
            for (int q = 0; q < D4; ++q) s_feat[tid * D4 + q] = load_feat4(feat, g * D + 4 * q);
        }
        __syncthreads();
        const int nb = min((uint32_t)kBatch, end - b0);
        for (int k = 0; k < nb && !done; ++k) {
            const SplatGeo s = s_geo[k];
            PairEval e = eval_pair(s, pxc, pyc, prm.alpha_min, prm.alpha_max);
            if (e.skip) continue;
            float Tn = T * (1.f - e.alpha);
            if (Tn < prm.T_min) {
                done = true;
                break;
            }
            float w = e.alpha * T;
            float4 c = s_rgb[k];
            acc_r = fmaf(w, c.x, acc_r);
            acc_g = fmaf(w, c.y, acc_g);
            acc_b = fmaf(w, c.z, acc_b);
            acc_d = fmaf(w, c.w, acc_d);
            acc_s += w;
#pragma unroll
            for (int q = 0; q < D4; ++q) {
                float4 f = s_feat[k * D4 + q];
                acc_f[4 * q] = fmaf(w, f.x, acc_f[4 * q]);
                acc_f[4 * q + 1] = fmaf(w, f.y, acc_f[4 * q + 1]);
                acc_f[4 * q + 2] = fmaf(w, f.z, acc_f[4 * q + 2]);
                acc_f[4 * q + 3] = fmaf(w, f.w, acc_f[4 * q + 3]);
            }
            T = Tn;
            last = (int)(b0 - start) + k + 1;
            ++blended;
        }
    }
    if (!inside) return;
    const int64_t pix = vt.pix_off[v] + (int64_t)py * vt.W[v] + px;
    o_rgb[pix] = acc_r + T * prm.bg[0];
    o_rgb[P + pix] = acc_g + T * prm.bg[1];
    o_rgb[2 * P + pix] = acc_b + T * prm.bg[2];
    o_depth[pix] = acc_d;
    o_sil[pix] = acc_s;
#pragma unroll
    for (int d = 0; d < D; ++d) o_feat[d * P + pix] = acc_f[d];
    o_T[pix] = T;
    o_nc[pix] = last;
    if (o_nb) o_nb[pix] = blended;
}

template <int D, typename RT, typename FT>
gs_status launch(const ViewTable &vt, const Params &prm, const gs_gaussians *g, const gs_projected *proj,
                 const gs_binning *bins, gs_images *out, cudaStream_t st) {
    int tiles = vt.tile_off[vt.n_views];
    int64_t P = vt.pix_off[vt.n_views];
    raster_fwd_kernel<D, RT, FT><<<tiles, kTilePix, 0, st>>>(
        vt, prm, reinterpret_cast<const float4 *>(proj->uvdo), reinterpret_cast<const float2 *>(proj->uv_lo),
        reinterpret_cast<const float4 *>(proj->conic), static_cast<const RT *>(g->rgb),
        static_cast<const FT *>(g->feat), bins->vals, bins->ranges, P, out->rgb,
        out->depth, out->sil, out->feat, out->T_final, out->n_contrib, out->n_blended);
    return last_launch();
}

template <typename RT, typename FT>
gs_status dispatch_d(int D, const ViewTable &vt, const Params &prm, const gs_gaussians *g, const gs_projected *proj,
                     const gs_binning *bins, gs_images *out, cudaStream_t st) {
    switch (D) {
        case 0: return launch<0, RT, FT>(vt, prm, g, proj, bins, out, st);
        case 4: return launch<4, RT, FT>(vt, prm, g, proj, bins, out, st);
        case 8: return launch<8, RT, FT>(vt, prm, g, proj, bins, out, st);
        case 16: return launch<16, RT, FT>(vt, prm, g, proj, bins, out, st);
        case 32: return launch<32, RT, FT>(vt, prm, g, proj, bins, out, st);
        default: return GS_ERR_UNSUPPORTED;
    }
}

template <>
gs_status dispatch_d<__half, __nv_bfloat16>(int D, const ViewTable &vt, const Params &prm, const gs_gaussians *g,
                                            const gs_projected *proj, const gs_binning *bins, gs_images *out,
                                            cudaStream_t st) {
    switch (D) {
        case 16: return launch<16, __half, __nv_bfloat16>(vt, prm, g, proj, bins, out, st);
        case 32: return launch<32, __half, __nv_bfloat16>(vt, prm, g, proj, bins, out, st);
        default: return GS_ERR_UNSUPPORTED;
    }
}

}  // namespace

bool storage_ok(const gs_gaussians *g) {
    bool plain = g->rgb_dtype == GS_F32 && g->feat_dtype == GS_F32;
    bool half = g->rgb_dtype == GS_F16 && g->feat_dtype == GS_BF16 && (g->feat_dim == 16 || g->feat_dim == 32);
    return (plain || half) && feat_dim_ok(g->feat_dim) && g->rgb && (g->feat || g->feat_dim == 0);
}

}  // namespace gs

extern "C" gs_status gs_render_fwd(const gs_gaussians *g, const gs_projected *proj, const gs_binning *bins,
                                   const gs_camera *cams, int n_views, const gs_raster_params *p, gs_images *out,
                                   gs_stream stream) {
    using namespace gs;
    if (!g || !proj || !bins || !out || g->n < 0) return GS_ERR_ARG;
    ViewTable vt;
    Params prm;
    if (!make_view_table(cams, n_views, g->n, &vt) || !make_params(p, &prm)) return GS_ERR_ARG;
    if (!feat_dim_ok(g->feat_dim)) return GS_ERR_UNSUPPORTED;
    if (!out->rgb || !out->depth || !out->sil || !out->T_final || !out->n_contrib || (g->feat_dim && !out->feat) ||
        !bins->ranges)
        return GS_ERR_ARG;
    if (g->n > 0 && (!storage_ok(g) || !bins->vals || !proj->uvdo || !proj->uv_lo || !proj->conic)) {
        return storage_ok(g) ? GS_ERR_ARG : GS_ERR_UNSUPPORTED;
    }
    if (g->feat_dim && (reinterpret_cast<uintptr_t>(g->feat) & 15)) return GS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (g->rgb_dtype == GS_F16) return dispatch_d<__half, __nv_bfloat16>(g->feat_dim, vt, prm, g, proj, bins, out, st);
    return dispatch_d<float, float>(g->feat_dim, vt, prm, g, proj, bins, out, st);
}
