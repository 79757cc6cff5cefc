// Losses and reductions around the blend:
//   - decoder + L1 colour/depth + semantic cross-entropy with image gradients
//     (Eq. 8, 15-17) and the tracking mask M_obs (Eq. 21), whose depth-error
//     median is found by a 4-pass 8-bit radix select over f32 bit patterns;
//   - depth-adaptive scale regularisation (Eq. 12);
//   - the f64 reduction of the pose-twist contributions (supplementary B.1);
//   - the Adam + SE(3) exponential pose step (Sec. 3.4, supplementary C.1).
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace gs {
namespace {

constexpr int kMaxK = 32;

// Median of view v from the per-pass digit histograms hist[p][v][256]:
// returns the f32 bit pattern of the lower median (element floor((n-1)/2)),
// selecting `passes` digits from the top; *n_out = number of valid pixels.
__device__ uint32_t select_prefix(const uint32_t *hist, int n_views, int v, int passes, uint32_t *n_out) {
    const uint32_t *h0 = hist + (size_t)v * 256;
    uint32_t n = 0;
    for (int d = 0; d < 256; ++d) n += h0[d];
    *n_out = n;
    if (n == 0) return 0;
    uint32_t k = (n - 1) / 2, prefix = 0;
    for (int p = 0; p < passes; ++p) {
        const uint32_t *h = hist + ((size_t)p * n_views + v) * 256;
        uint32_t cum = 0;
        int sel = 255;
        for (int d = 0; d < 256; ++d) {
            if (cum + h[d] > k) { sel = d; break; }
            cum += h[d];
        }
        k -= cum;
        prefix |= (uint32_t)sel << (24 - 8 * p);
    }
    return prefix;
}

__device__ __forceinline__ float depth_error(float d, float dgt) { return fabsf(__fsub_rn(d, dgt)); }

__global__ void __launch_bounds__(256) median_hist_kernel(ViewTable vt, int pass, const float *depth,
                                                          const float *tdepth, uint32_t *hist) {
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_prefix;
    const int v = blockIdx.y;
    const int64_t Pv = (int64_t)vt.W[v] * vt.H[v];
    if ((int64_t)blockIdx.x * 256 >= Pv) return;
    s_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        uint32_t n;
        s_prefix = pass > 0 ? select_prefix(hist, vt.n_views, v, pass, &n) : 0u;
    }
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    bool valid = false;
    uint32_t bits = 0;
    if (i < Pv) {
        int64_t pix = vt.pix_off[v] + i;
        float dgt = tdepth[pix];
        if (dgt > 0.f) {
            bits = __float_as_uint(depth_error(depth[pix], dgt));
            valid = pass == 0 || (bits >> (32 - 8 * pass)) == (s_prefix >> (32 - 8 * pass));
        }
    }
    uint32_t d = valid ? (bits >> (24 - 8 * pass)) & 255u : 256u + (threadIdx.x & 31);
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s_hist[d], __popc(peers));
    __syncthreads();
    uint32_t c = s_hist[threadIdx.x];
    if (c) atomicAdd(&hist[((size_t)pass * vt.n_views + v) * 256 + threadIdx.x], c);
}

struct LossP {
    float color, depth, sem, tau_obs;
    int mask_mode, K;
};

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

__device__ __forceinline__ double block_sum_f64(double x, double *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[w] = x;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_red[i];
    return t;  // valid in thread 0
}

template <int D>
__global__ void __launch_bounds__(256) loss_kernel(ViewTable vt, LossP lp, const float *rgb, const float *depth,
                                                   const float *sil, const float *feat, const float *trgb,
                                                   const float *tdepth, const uint8_t *label, const float *Wd,
                                                   const float *bd, int64_t P, const uint32_t *med_hist,
                                                   float *g_rgb, float *g_depth, float *g_sil, float *g_feat,
                                                   float *dW, float *db, double *loss_out, float *mask_out,
                                                   float *median_out) {
    constexpr int DD = D > 0 ? D : 1;
    __shared__ float s_W[kMaxK * DD], s_b[kMaxK];
    __shared__ float s_dW[kMaxK * DD + kMaxK];
    __shared__ double s_red[8];
    __shared__ float s_med;
    const int v = blockIdx.y;
    const int64_t Pv = (int64_t)vt.W[v] * vt.H[v];
    if ((int64_t)blockIdx.x * 256 >= Pv) return;
    const int K = lp.K, tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < K * D; i += 256) s_W[i] = Wd[i];
    for (int i = tid; i < K; i += 256) s_b[i] = bd[i];
    for (int i = tid; i < K * D + K; i += 256) s_dW[i] = 0.f;
    if (tid == 0) {
        float med = 0.f;
        if (lp.mask_mode == 1) {
            uint32_t n;
            med = __uint_as_float(select_prefix(med_hist, vt.n_views, v, 4, &n));
            if (median_out && blockIdx.x == 0) median_out[v] = med;
        }
        s_med = med;
    }
    __syncthreads();
    const float invP = 1.f / (float)Pv;
    const int64_t i = (int64_t)blockIdx.x * 256 + tid;
    const bool inpix = i < Pv;
    const int64_t pix = vt.pix_off[v] + (inpix ? i : 0);
    double lc = 0, ld = 0, ls = 0;
    float f[DD], dz[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) dz[k] = 0.f;
#pragma unroll
    for (int d = 0; d < DD; ++d) f[d] = 0.f;
    if (inpix) {
        const float dgt = tdepth[pix], dd = depth[pix];
        float m = 1.f;
        if (lp.mask_mode == 1)
            m = (sil[pix] > lp.tau_obs && dgt > 0.f && depth_error(dd, dgt) < 10.f * s_med) ? 1.f : 0.f;
        if (mask_out) mask_out[pix] = m;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float r = rgb[c * P + pix] - trgb[c * P + pix];
            lc += (double)(m * fabsf(r));
            g_rgb[c * P + pix] = m * lp.color * (r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f)) * invP;
        }
        float gd = 0.f;
        if (dgt > 0.f) {
            float r = dd - dgt;
            ld += (double)(m * fabsf(r));
            gd = m * lp.depth * (r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f)) * invP;
        }
        g_depth[pix] = gd;
        g_sil[pix] = 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d) f[d] = feat[d * P + pix];
        const int lab = label[pix];
        float gf[DD];
#pragma unroll
        for (int d = 0; d < DD; ++d) gf[d] = 0.f;
        if (lab != 255 && lab < K) {
            float z[kMaxK];
            float zmax = -INFINITY;
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) {
                if (k < K) {
                    float s = s_b[k];
#pragma unroll
                    for (int d = 0; d < D; ++d) s = fmaf(s_W[k * D + d], f[d], s);
                    z[k] = s;
                    zmax = fmaxf(zmax, s);
                }
            }
            float se = 0.f;
#pragma unroll
            for (int k = 0; k < kMaxK; ++k)
                if (k < K) se += expf(z[k] - zmax);
            const float lse = zmax + logf(se);
            float zl = 0.f;
#pragma unroll
            for (int k = 0; k < kMaxK; ++k)
                if (k == lab) zl = z[k];
            ls += (double)(m * (lse - zl));
            const float scale = m * lp.sem * invP;
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) {
                if (k < K) {
                    dz[k] = scale * (expf(z[k] - lse) - (k == lab ? 1.f : 0.f));
#pragma unroll
                    for (int d = 0; d < D; ++d) gf[d] = fmaf(s_W[k * D + d], dz[k], gf[d]);
                }
            }
        }
#pragma unroll
        for (int d = 0; d < D; ++d) g_feat[d * P + pix] = gf[d];
    }
    // decoder gradients dW[k][d] = sum dz_k f_d and db[k] = sum dz_k: one warp
    // transpose reduction per class row (k is unrolled so dz stays in registers)
    const int nval = K * D + K;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        if (k < K) {
            if constexpr (D > 0) {
                constexpr int DP = D < 8 ? 8 : D;
                float vals[DP];
#pragma unroll
                for (int d = 0; d < DP; ++d) vals[d] = d < D ? dz[k] * f[d] : 0.f;
                float r = warp_transpose_reduce<DP>(vals, lane);
                if (lane < D && r != 0.f) atomicAdd(&s_dW[k * D + lane], r);
            }
        }
    }
    {
        float vals[kMaxK];
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) vals[k] = dz[k];
        float r = warp_transpose_reduce<kMaxK>(vals, lane);
        if (lane < K && r != 0.f) atomicAdd(&s_dW[K * D + lane], r);
    }
    // loss sums in f64, already weighted and normalised by the view's pixel count
    double wc = block_sum_f64(lc * (double)lp.color / (double)Pv, s_red);
    double wd = block_sum_f64(ld * (double)lp.depth / (double)Pv, s_red);
    double wsm = block_sum_f64(ls * (double)lp.sem / (double)Pv, s_red);
    __syncthreads();
    for (int j = tid; j < nval; j += 256) {
        float x = s_dW[j];
        if (x != 0.f) atomicAdd(j < K * D ? &dW[j] : &db[j - K * D], x);
    }
    if (tid == 0) {
        atomicAdd(&loss_out[0], wc + wd + wsm);
        atomicAdd(&loss_out[1], wc);
        atomicAdd(&loss_out[2], wd);
        atomicAdd(&loss_out[3], wsm);
    }
}

// --------------------------------------------------------------------- DSR
__global__ void __launch_bounds__(256) dsr_stats_kernel(int64_t m, const float *ls, double *acc) {
    __shared__ double s_red[8];
    double s1 = 0, s2 = 0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < m; i += (int64_t)gridDim.x * 256) {
        double s = (double)expf(ls[i]);
        s1 += s;
        s2 += s * s;
    }
    double t1 = block_sum_f64(s1, s_red);
    double t2 = block_sum_f64(s2, s_red);
    if (threadIdx.x == 0) {
        atomicAdd(&acc[0], t1);
        atomicAdd(&acc[1], t2);
    }
}

__device__ __forceinline__ void dsr_bounds(const double *acc, int64_t m, double &hi, double &lo, double &mu,
                                           double &sd) {
    mu = acc[0] / (double)m;
    double var = acc[1] / (double)m - mu * mu;
    sd = sqrt(var > 0 ? var : 0.0);
    hi = mu + 2.0 * sd;
    lo = mu - 2.0 * sd;
}

__global__ void __launch_bounds__(256) dsr_mask_kernel(int64_t m, const float *ls, double *acc) {
    __shared__ double s_red[8];
    double hi, lo, mu, sd;
    dsr_bounds(acc, m, hi, lo, mu, sd);
    double sb = 0, nb = 0, ss = 0, ns = 0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < m; i += (int64_t)gridDim.x * 256) {
        float l = ls[i];
        double s = (double)expf(l);
        if (s > hi) { sb += s; nb += 1; }
        if (s < lo) { ss += -(double)l; ns += 1; }
    }
    double t[4] = {block_sum_f64(sb, s_red), block_sum_f64(nb, s_red), block_sum_f64(ss, s_red),
                   block_sum_f64(ns, s_red)};
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k)
            if (t[k] != 0) atomicAdd(&acc[2 + k], t[k]);
}

__global__ void __launch_bounds__(256) dsr_grad_kernel(int64_t m, const float *ls, float lam_big, float lam_small,
                                                       const double *acc, float *d_ls, double *out) {
    double hi, lo, mu, sd;
    dsr_bounds(acc, m, hi, lo, mu, sd);
    const double nb = acc[3], ns = acc[5];
    const float gb = nb > 0 ? (float)(lam_big / nb) : 0.f;
    const float gs = ns > 0 ? (float)(lam_small / ns) : 0.f;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < m; i += (int64_t)gridDim.x * 256) {
        float l = ls[i];
        float sf = expf(l);
        double s = (double)sf;
        float g = 0.f;
        if (s > hi) g += gb * sf;
        if (s < lo) g -= gs;
        if (g != 0.f) d_ls[i] += g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double Lb = nb > 0 ? acc[2] / nb : 0.0, Ls = ns > 0 ? acc[4] / ns : 0.0;
        out[0] = (double)lam_big * Lb + (double)lam_small * Ls;
        out[1] = mu; out[2] = sd; out[3] = nb; out[4] = ns; out[5] = Lb; out[6] = Ls; out[7] = 0.0;
    }
}

// ------------------------------------------------------------ pose reduction
__global__ void __launch_bounds__(256) pose_reduce_kernel(int64_t n, const float *pose_part, double *d_twist) {
    __shared__ double s_red[8];
    const int vk = blockIdx.y;  // view * 6 + component
    const float *p = pose_part + (int64_t)vk * n;
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) s += (double)p[i];
    double t = block_sum_f64(s, s_red);
    if (threadIdx.x == 0 && t != 0) atomicAdd(&d_twist[vk], t);
}

// ------------------------------------------------------------------ pose step
__global__ void pose_step_kernel(int n_views, const double *grad, double *Tst, double *adam, int step, double lr0,
                                 double lr1, double lr2, double lr3, double lr4, double lr5, double b1, double b2,
                                 double eps, float *pose_f32) {
    int v = threadIdx.x;
    if (v >= n_views) return;
    const double lr[6] = {lr0, lr1, lr2, lr3, lr4, lr5};
    double *m = adam + 12 * v, *vv = m + 6, *T = Tst + 16 * v;
    double dl[6];
    for (int k = 0; k < 6; ++k) {
        double g = grad[6 * v + k];
        m[k] = b1 * m[k] + (1 - b1) * g;
        vv[k] = b2 * vv[k] + (1 - b2) * g * g;
        double mh = m[k] / (1 - pow(b1, step)), vh = vv[k] / (1 - pow(b2, step));
        dl[k] = -lr[k] * mh / (sqrt(vh) + eps);
    }
    // SE(3) exponential of (rho, phi) = dl
    double ph[3] = {dl[3], dl[4], dl[5]};
    double th = sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
    double a, b, c;
    if (th < 1e-8) { a = 1 - th * th / 6; b = 0.5 - th * th / 24; c = 1.0 / 6 - th * th / 120; }
    else { a = sin(th) / th; b = (1 - cos(th)) / (th * th); c = (th - sin(th)) / (th * th * th); }
    double K[9] = {0, -ph[2], ph[1], ph[2], 0, -ph[0], -ph[1], ph[0], 0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
    double R[9], V[9];
    for (int k = 0; k < 9; ++k) {
        double id = (k % 4 == 0) ? 1.0 : 0.0;
        R[k] = id + a * K[k] + b * K2[k];
        V[k] = id + b * K[k] + c * K2[k];
    }
    double E[16] = {R[0], R[1], R[2], V[0] * dl[0] + V[1] * dl[1] + V[2] * dl[2],
                    R[3], R[4], R[5], V[3] * dl[0] + V[4] * dl[1] + V[5] * dl[2],
                    R[6], R[7], R[8], V[6] * dl[0] + V[7] * dl[1] + V[8] * dl[2],
                    0, 0, 0, 1};
    double out[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0;
            for (int k = 0; k < 4; ++k) s += E[4 * i + k] * T[4 * k + j];
            out[4 * i + j] = s;
        }
    for (int k = 0; k < 16; ++k) {
        T[k] = out[k];
        if (pose_f32) pose_f32[16 * v + k] = (float)out[k];
    }
}

template <int D>
gs_status launch_loss(const ViewTable &vt, const LossP &lp, const gs_images *img, const gs_targets *tgt,
                      const float *W, const float *b, int64_t P, const uint32_t *mh, gs_image_grads_out *g,
                      float *dW, float *db, double *loss_out, float *mask_out, float *median_out, cudaStream_t st) {
    int64_t maxPv = 0;
    for (int v = 0; v < vt.n_views; ++v) maxPv = std::max<int64_t>(maxPv, (int64_t)vt.W[v] * vt.H[v]);
    dim3 grid(ceil_div(maxPv, 256), vt.n_views);
    loss_kernel<D><<<grid, 256, 0, st>>>(vt, lp, img->rgb, img->depth, img->sil, img->feat, tgt->rgb, tgt->depth,
                                         tgt->label, W, b, P, mh, g->rgb, g->depth, g->sil, g->feat, dW, db,
                                         loss_out, mask_out, median_out);
    return last_launch();
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_loss_fwd_bwd(const gs_camera *cams, int n_views, int feat_dim, const gs_images *img,
                                     const gs_targets *tgt, const float *dec_W, const float *dec_b,
                                     const gs_loss_params *lp, void *ws, size_t ws_bytes, gs_image_grads_out *grad,
                                     float *d_dec_W, float *d_dec_b, double *loss_out, float *mask_out,
                                     float *median_out, gs_stream stream) {
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    ViewTable vt;
    if (!img || !tgt || !lp || !grad || !loss_out || !make_view_table(cams, n_views, 0, &vt)) return GS_ERR_ARG;
    if (!feat_dim_ok(feat_dim)) return GS_ERR_UNSUPPORTED;
    if (lp->n_classes < 0 || lp->n_classes > 32 || (lp->mask_mode != 0 && lp->mask_mode != 1)) return GS_ERR_ARG;
    if (!img->rgb || !img->depth || !img->sil || (feat_dim && !img->feat) || !tgt->rgb || !tgt->depth ||
        !tgt->label || !grad->rgb || !grad->depth || !grad->sil || (feat_dim && !grad->feat))
        return GS_ERR_ARG;
    if (lp->n_classes > 0 && (!dec_W || !dec_b || !d_dec_W || !d_dec_b)) return GS_ERR_ARG;
    WsLayout L = ws_layout(0, n_views, 0);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < L.misc_end) return GS_ERR_ARG;
    char *w = static_cast<char *>(ws);
    uint32_t *mh = reinterpret_cast<uint32_t *>(w + L.med_hist);
    int64_t P = vt.pix_off[n_views];
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(loss_out, 0, 4 * sizeof(double), st)))) return s;
    if (lp->n_classes > 0) {
        if ((s = cuda_status(cudaMemsetAsync(d_dec_W, 0, sizeof(float) * lp->n_classes * feat_dim, st)))) return s;
        if ((s = cuda_status(cudaMemsetAsync(d_dec_b, 0, sizeof(float) * lp->n_classes, st)))) return s;
    }
    int64_t maxPv = 0;
    for (int v = 0; v < n_views; ++v) maxPv = std::max<int64_t>(maxPv, (int64_t)vt.W[v] * vt.H[v]);
    if (lp->mask_mode == 1) {
        if ((s = cuda_status(cudaMemsetAsync(mh, 0, sizeof(uint32_t) * 4 * 256 * n_views, st)))) return s;
        dim3 grid(ceil_div(maxPv, 256), n_views);
        for (int pass = 0; pass < 4; ++pass)
            median_hist_kernel<<<grid, 256, 0, st>>>(vt, pass, img->depth, tgt->depth, mh);
        if ((s = last_launch())) return s;
    }
    LossP q{lp->color, lp->depth, lp->sem, lp->tau_obs, lp->mask_mode, lp->n_classes};
    switch (feat_dim) {
        case 0: return launch_loss<0>(vt, q, img, tgt, dec_W, dec_b, P, mh, grad, d_dec_W, d_dec_b, loss_out, mask_out, median_out, st);
        case 4: return launch_loss<4>(vt, q, img, tgt, dec_W, dec_b, P, mh, grad, d_dec_W, d_dec_b, loss_out, mask_out, median_out, st);
        case 8: return launch_loss<8>(vt, q, img, tgt, dec_W, dec_b, P, mh, grad, d_dec_W, d_dec_b, loss_out, mask_out, median_out, st);
        case 16: return launch_loss<16>(vt, q, img, tgt, dec_W, dec_b, P, mh, grad, d_dec_W, d_dec_b, loss_out, mask_out, median_out, st);
        case 32: return launch_loss<32>(vt, q, img, tgt, dec_W, dec_b, P, mh, grad, d_dec_W, d_dec_b, loss_out, mask_out, median_out, st);
        default: return GS_ERR_UNSUPPORTED;
    }
}

extern "C" gs_status gs_dsr(int64_t n, const float *log_scales, float lam_big, float lam_small, void *ws,
                            size_t ws_bytes, float *d_log_scales, double *out, gs_stream stream) {
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 0 || !out || !ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return GS_ERR_ARG;
    WsLayout L = ws_layout(0, 1, 0);
    if (ws_bytes < L.misc_end) return GS_ERR_ARG;
    double *acc = reinterpret_cast<double *>(static_cast<char *>(ws) + L.dsr_acc);
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(acc, 0, 8 * sizeof(double), st)))) return s;
    if ((s = cuda_status(cudaMemsetAsync(out, 0, 8 * sizeof(double), st)))) return s;
    if (n == 0) return GS_OK;
    if (!log_scales || !d_log_scales) return GS_ERR_ARG;
    int64_t m = 3 * n;
    int grid = std::min(ceil_div(m, 256), 152 * 8);
    dsr_stats_kernel<<<grid, 256, 0, st>>>(m, log_scales, acc);
    dsr_mask_kernel<<<grid, 256, 0, st>>>(m, log_scales, acc);
    dsr_grad_kernel<<<grid, 256, 0, st>>>(m, log_scales, lam_big, lam_small, acc, d_log_scales, out);
    return last_launch();
}

extern "C" gs_status gs_pose_grad(int64_t n, int n_views, const float *pose_part, double *d_twist, gs_stream stream) {
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 0 || n_views < 1 || n_views > kMaxViews || !d_twist) return GS_ERR_ARG;
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(d_twist, 0, sizeof(double) * 6 * n_views, st)))) return s;
    if (n == 0) return GS_OK;
    if (!pose_part) return GS_ERR_ARG;
    dim3 grid(std::min(ceil_div(n, 256 * 4), 152 * 2), 6 * n_views);
    pose_reduce_kernel<<<grid, 256, 0, st>>>(n, pose_part, d_twist);
    return last_launch();
}

extern "C" gs_status gs_pose_step(int n_views, const double *d_twist, double *T_state, double *adam, int step,
                                  const double *lr, double beta1, double beta2, double eps, float *pose_f32,
                                  gs_stream stream) {
    using namespace gs;
    if (n_views < 1 || n_views > kMaxViews || !d_twist || !T_state || !adam || !lr || step < 1) return GS_ERR_ARG;
    pose_step_kernel<<<1, 64, 0, (cudaStream_t)stream>>>(n_views, d_twist, T_state, adam, step, lr[0], lr[1], lr[2],
                                                         lr[3], lr[4], lr[5], beta1, beta2, eps, pose_f32);
    return last_launch();
}
