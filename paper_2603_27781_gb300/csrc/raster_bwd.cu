// Backward of the blend and the projection (supplementary B.1 chain rule).
//
// Same grid as the forward: one CTA per 16x16 tile, one thread per pixel.  A
// pixel walks the splats it blended back to front, starting from its stored
// final transmittance and last-contributor position; the transmittance in
// front of each splat is recovered as T / (1 - alpha) and a running value S
// of everything behind it gives d out / d alpha = T (x - S).
//
// Per splat the warp's 32 pixel contributions are summed with a transpose
// reduction (each shuffle step halves the values a lane carries, so N values
// take N - 1 shuffles and lane l ends with the sum of value l), the 8 warps
// combine through shared-memory atomics, and each (tile, splat) issues one
// 16-byte vector atomic per 4 values to the per-Gaussian accumulators.
#include <type_traits>

#include "raster.cuh"

namespace gs {

bool storage_ok(const gs_gaussians *g);

namespace {

constexpr int kBatch = 128;

constexpr int pow2_at_least(int x) { return x <= 8 ? 8 : (x <= 16 ? 16 : 32); }

// Sums v[0..N) over the warp; lane l returns the total of value (l mod N).
template <int N>
__device__ __forceinline__ float warp_transpose_reduce(float (&v)[N], int lane) {
#pragma unroll
    for (int s = N / 2; s >= 1; s >>= 1) {
        const bool up = lane & s;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            float send = up ? v[i] : v[i + s];
            float keep = up ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    float r = v[0];
#pragma unroll
    for (int s = N; s < 32; s <<= 1) r += __shfl_xor_sync(0xffffffffu, r, s);
    return r;
}

template <int D, bool MAP>
struct Layout {
    static constexpr int NV = MAP ? 10 + D : 6;                 // reduced values per splat
    static constexpr int C0 = NV > 32 ? 32 : pow2_at_least(NV);  // first chunk (power of two)
    static constexpr int R1 = NV > 32 ? NV - 32 : 0;             // values in the second chunk
    static constexpr int C1 = R1 > 0 ? pow2_at_least(R1) : 0;
    static constexpr int ROW = C0 + C1;                          // shared accumulator row
};

template <int D, bool MAP, typename RT, typename FT>
__global__ void __launch_bounds__(kTilePix) raster_bwd_kernel(
    ViewTable vt, Params prm, const float4 *__restrict__ uvdo, const float2 *__restrict__ uv_lo,
    const float4 *__restrict__ conic,
    const RT *__restrict__ rgb, const FT *__restrict__ feat, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ ranges, int64_t P, const float *__restrict__ T_final,
    const int32_t *__restrict__ n_contrib, const float *__restrict__ g_rgb, const float *__restrict__ g_depth,
    const float *__restrict__ g_sil, const float *__restrict__ g_feat, float4 *acc_uvod, float4 *acc_conic,
    float4 *acc_rgb, float *d_feat) {
    using LY = Layout<D, MAP>;
    constexpr int D4 = D / 4;
    constexpr int NCH = 5 + D;  // r, g, b, depth, sil, features
    __shared__ SplatGeo s_geo[kBatch];
    __shared__ float4 s_rgb[kBatch];
    __shared__ float4 s_feat[kBatch * (D4 > 0 ? D4 : 1)];
    __shared__ float s_acc[kBatch * LY::ROW];
    __shared__ int s_max_last;

    const int gt = blockIdx.x;
    const int v = view_of_tile(vt, gt);
    const int t = gt - vt.tile_off[v];
    const int tx = t % vt.TX[v], ty = t / vt.TX[v];
    const int tid = threadIdx.x, lane = tid & 31;
    int px, py;
    tile_pixel(tid, tx, ty, px, py);
    const bool inside = px < vt.W[v] && py < vt.H[v];
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const uint32_t start = ranges[2 * gt];
    const int64_t voff = (int64_t)v * vt.n;
    const int64_t pix = vt.pix_off[v] + (int64_t)py * vt.W[v] + px;

    // per-pixel state: upstream gradient g and running background-side value S per channel
    float gch[NCH], S[NCH];
    float T = 1.f;
    int last = 0;
    if (inside) {
        T = T_final[pix];
        last = n_contrib[pix];
        gch[0] = g_rgb[pix];
        gch[1] = g_rgb[P + pix];
        gch[2] = g_rgb[2 * P + pix];
        gch[3] = g_depth[pix];
        gch[4] = g_sil ? g_sil[pix] : 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d) gch[5 + d] = g_feat[d * P + pix];
    } else {
#pragma unroll
        for (int c = 0; c < NCH; ++c) gch[c] = 0.f;
    }
    S[0] = prm.bg[0];
    S[1] = prm.bg[1];
    S[2] = prm.bg[2];
#pragma unroll
    for (int c = 3; c < NCH; ++c) S[c] = 0.f;

    if (tid == 0) s_max_last = 0;
    __syncthreads();
    if (last > 0) atomicMax(&s_max_last, last);
    __syncthreads();
    const int max_last = s_max_last;

    for (int b_end = max_last; b_end > 0; b_end -= kBatch) {
        const int b_start = max(0, b_end - kBatch);
        const int cnt = b_end - b_start;
        __syncthreads();
        if (tid < cnt) {
            uint32_t item = vals[start + b_start + tid];
            int64_t g = (int64_t)item - voff;
            const float4 a = uvdo[item];
            s_geo[tid] = make_geo(a, uv_lo[item], conic[item]);
            s_rgb[tid] = load_rgbd(rgb, g, a.z);
#pragma unroll
            for (int q = 0; q < D4; ++q) s_feat[tid * D4 + q] = load_feat4(feat, g * D + 4 * q);
        }
        for (int i = tid; i < cnt * LY::ROW; i += kTilePix) s_acc[i] = 0.f;
        __syncthreads();

        for (int k = cnt - 1; k >= 0; --k) {
            const int pos = b_start + k;
            if (!__any_sync(0xffffffffu, pos < last)) continue;
            const SplatGeo s = s_geo[k];
            PairEval e = eval_pair(s, pxc, pyc, prm.alpha_min, prm.alpha_max);
            const bool contrib = pos < last && !e.skip;
            if (!__any_sync(0xffffffffu, contrib)) continue;

            float val[LY::C0 + LY::C1];
#pragma unroll
            for (int i = 0; i < LY::C0 + LY::C1; ++i) val[i] = 0.f;
            if (contrib) {
                const float a = e.alpha;
                const float Tb = __fdividef(T, 1.f - a);
                const float w = a * Tb;
                float4 c = s_rgb[k];
                float x[NCH];
                x[0] = c.x; x[1] = c.y; x[2] = c.z; x[3] = c.w; x[4] = 1.f;
#pragma unroll
                for (int q = 0; q < D4; ++q) {
                    float4 f = s_feat[k * D4 + q];
                    x[5 + 4 * q] = f.x; x[6 + 4 * q] = f.y; x[7 + 4 * q] = f.z; x[8 + 4 * q] = f.w;
                }
                float da = 0.f;
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    float diff = x[ch] - S[ch];
                    da = fmaf(gch[ch], diff, da);
                    S[ch] = fmaf(a, diff, S[ch]);
                }
                da *= Tb;
                T = Tb;
                float du = 0.f, dv = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dop = 0.f;
                if (e.oG < prm.alpha_max) {
                    dop = e.G * da;
                    const float dpow = e.oG * da;
                    const float dxx = e.dx * e.dx, dyy = e.dy * e.dy, dxy = e.dx * e.dy;
                    dA = -0.5f * dxx * dpow;
                    dB = -dxy * dpow;
                    dC = -0.5f * dyy * dpow;
                    // (A dx + B dy, B dx + C dy) from the log2 e-scaled conic
                    const float sc = -dpow * (1.f / kLog2e);
                    du = (2.f * s.qa * e.dx + s.qb * e.dy) * sc;
                    dv = (s.qb * e.dx + 2.f * s.qc * e.dy) * sc;
                }
                val[0] = du; val[1] = dv; val[2] = dA; val[3] = dB; val[4] = dC;
                if (MAP) {
                    val[5] = dop;
                    val[6] = w * gch[3];
                    val[7] = w * gch[0];
                    val[8] = w * gch[1];
                    val[9] = w * gch[2];
#pragma unroll
                    for (int d = 0; d < D; ++d) val[10 + d] = w * gch[5 + d];
                } else {
                    val[5] = w * gch[3];
                }
            }
            // warp reduction, then CTA combine in shared memory
            {
                float v0[LY::C0];
#pragma unroll
                for (int i = 0; i < LY::C0; ++i) v0[i] = val[i];
                float r = warp_transpose_reduce<LY::C0>(v0, lane);
                int idx = lane & (LY::C0 - 1);
                if (lane < LY::C0 && idx < LY::NV && r != 0.f) atomicAdd(&s_acc[k * LY::ROW + idx], r);
            }
            if constexpr (LY::C1 > 0) {
                float v1[LY::C1];
#pragma unroll
                for (int i = 0; i < LY::C1; ++i) v1[i] = val[LY::C0 + i];
                float r = warp_transpose_reduce<LY::C1>(v1, lane);
                int idx = lane & (LY::C1 - 1);
                if (lane < LY::C1 && idx < LY::R1 && r != 0.f) atomicAdd(&s_acc[k * LY::ROW + LY::C0 + idx], r);
            }
        }
        __syncthreads();
        // one set of vector atomics per (tile, splat)
        if (tid < cnt) {
            const float *a = s_acc + tid * LY::ROW;
            bool any = false;
#pragma unroll
            for (int i = 0; i < LY::NV; ++i) any |= a[i] != 0.f;
            if (any) {
                uint32_t item = vals[start + b_start + tid];
                int64_t g = (int64_t)item - voff;
                if (MAP) {
                    atomicAdd(&acc_uvod[item], make_float4(a[0], a[1], a[5], a[6]));
                    atomicAdd(&acc_conic[item], make_float4(a[2], a[3], a[4], 0.f));
                    atomicAdd(&acc_rgb[g], make_float4(a[7], a[8], a[9], 0.f));
#pragma unroll
                    for (int q = 0; q < D4; ++q)
                        atomicAdd(reinterpret_cast<float4 *>(d_feat + g * D) + q,
                                  make_float4(a[10 + 4 * q], a[11 + 4 * q], a[12 + 4 * q], a[13 + 4 * q]));
                } else {
                    atomicAdd(&acc_uvod[item], make_float4(a[0], a[1], 0.f, a[5]));
                    atomicAdd(&acc_conic[item], make_float4(a[2], a[3], a[4], 0.f));
                }
            }
        }
    }
}

template <int D, bool MAP, typename RT, typename FT>
gs_status launch(const ViewTable &vt, const Params &prm, const gs_gaussians *g, const gs_projected *proj,
                 const gs_binning *bins, const gs_images *fwd, const gs_image_grads *dL, float4 *acc_uvod,
                 float4 *acc_conic, float4 *acc_rgb, float *d_feat, cudaStream_t st) {
    int tiles = vt.tile_off[vt.n_views];
    int64_t P = vt.pix_off[vt.n_views];
    raster_bwd_kernel<D, MAP, RT, FT><<<tiles, kTilePix, 0, st>>>(
        vt, prm, reinterpret_cast<const float4 *>(proj->uvdo), reinterpret_cast<const float2 *>(proj->uv_lo),
        reinterpret_cast<const float4 *>(proj->conic), static_cast<const RT *>(g->rgb),
        static_cast<const FT *>(g->feat), bins->vals, bins->ranges, P, fwd->T_final,
        fwd->n_contrib, dL->rgb, dL->depth, dL->sil, dL->feat, acc_uvod, acc_conic, acc_rgb, d_feat);
    return last_launch();
}

template <bool MAP, typename RT, typename FT>
gs_status dispatch_d(int D, const ViewTable &vt, const Params &prm, const gs_gaussians *g, const gs_projected *proj,
                     const gs_binning *bins, const gs_images *fwd, const gs_image_grads *dL, float4 *acc_uvod,
                     float4 *acc_conic, float4 *acc_rgb, float *d_feat, cudaStream_t st) {
#define GS_CASE(DD) \
    case DD: return launch<DD, MAP, RT, FT>(vt, prm, g, proj, bins, fwd, dL, acc_uvod, acc_conic, acc_rgb, d_feat, st);
    if constexpr (std::is_same<RT, float>::value) {
        switch (D) {
            GS_CASE(0) GS_CASE(4) GS_CASE(8) GS_CASE(16) GS_CASE(32)
            default: return GS_ERR_UNSUPPORTED;
        }
    } else {
        switch (D) {
            GS_CASE(16) GS_CASE(32)
            default: return GS_ERR_UNSUPPORTED;
        }
    }
#undef GS_CASE
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_render_bwd(const gs_gaussians *g, const gs_projected *proj, const gs_binning *bins,
                                   const gs_camera *cams, int n_views, const gs_raster_params *p, int grad_mode,
                                   const gs_images *fwd, const gs_image_grads *dL, gs_splat_grads *sg, float *d_feat,
                                   gs_stream stream) {
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    if (!g || !proj || !bins || !fwd || !dL || !sg || g->n < 0) return GS_ERR_ARG;
    if (grad_mode <= 0 || grad_mode > (GS_GRAD_MAP | GS_GRAD_POSE)) return GS_ERR_ARG;
    ViewTable vt;
    Params prm;
    if (!make_view_table(cams, n_views, g->n, &vt) || !make_params(p, &prm)) return GS_ERR_ARG;
    if (!feat_dim_ok(g->feat_dim)) return GS_ERR_UNSUPPORTED;
    const bool map = grad_mode & GS_GRAD_MAP;
    if (g->n == 0) return GS_OK;
    if (!storage_ok(g)) return GS_ERR_UNSUPPORTED;
    if (!sg->uvod || !sg->conic || (map && (!sg->rgb || (g->feat_dim && !d_feat)))) return GS_ERR_ARG;
    if (!proj->uvdo || !proj->uv_lo || !proj->conic || !bins->vals || !bins->ranges || !fwd->T_final || !fwd->n_contrib ||
        !dL->rgb || !dL->depth || (g->feat_dim && !dL->feat))
        return GS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(sg->uvod) | reinterpret_cast<uintptr_t>(sg->conic) |
         reinterpret_cast<uintptr_t>(sg->rgb) | reinterpret_cast<uintptr_t>(d_feat)) & 15)
        return GS_ERR_ARG;
    if (g->feat_dim && (reinterpret_cast<uintptr_t>(g->feat) & 15)) return GS_ERR_ARG;
    const int64_t vn = g->n * n_views;
    float4 *acc_uvod = reinterpret_cast<float4 *>(sg->uvod);
    float4 *acc_conic = reinterpret_cast<float4 *>(sg->conic);
    float4 *acc_rgb = reinterpret_cast<float4 *>(sg->rgb);
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(acc_uvod, 0, sizeof(float4) * vn, st)))) return s;
    if ((s = cuda_status(cudaMemsetAsync(acc_conic, 0, sizeof(float4) * vn, st)))) return s;
    if (map) {
        if ((s = cuda_status(cudaMemsetAsync(acc_rgb, 0, sizeof(float4) * g->n, st)))) return s;
        if (g->feat_dim && (s = cuda_status(cudaMemsetAsync(d_feat, 0, sizeof(float) * g->feat_dim * g->n, st))))
            return s;
    }
    float *df = map ? d_feat : nullptr;
    if (g->rgb_dtype == GS_F16) {
        return map ? dispatch_d<true, __half, __nv_bfloat16>(g->feat_dim, vt, prm, g, proj, bins, fwd, dL, acc_uvod,
                                                             acc_conic, acc_rgb, df, st)
                   : dispatch_d<false, __half, __nv_bfloat16>(g->feat_dim, vt, prm, g, proj, bins, fwd, dL, acc_uvod,
                                                              acc_conic, acc_rgb, df, st);
    }
    return map ? dispatch_d<true, float, float>(g->feat_dim, vt, prm, g, proj, bins, fwd, dL, acc_uvod, acc_conic,
                                                acc_rgb, df, st)
               : dispatch_d<false, float, float>(g->feat_dim, vt, prm, g, proj, bins, fwd, dL, acc_uvod, acc_conic,
                                                 acc_rgb, df, st);
}
