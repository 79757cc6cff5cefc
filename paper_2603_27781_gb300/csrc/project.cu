// Projection of the Gaussians (Eq. 2, 3; supp. B.1) and its backward, with the
// per-Gaussian contributions to the SE(3) pose-twist gradient.
//
// One thread per Gaussian; the forward writes one 32-byte record per (view,
// Gaussian), the backward loops over the views of its Gaussian so that the
// view-summed parameter gradients are written once, without atomics.
#include "common.cuh"

namespace gs {
namespace {

struct Cov3 {  // symmetric 3x3: xx, xy, xz, yy, yz, zz
    float m[6];
};

__device__ __forceinline__ void quat_rot(const float q[4], float R[9]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Activated shape of one Gaussian: unit quaternion, its rotation, scales, M = Rq S, Sigma = M M^T.
struct Shape {
    float qn, qh[4], Rq[9], s[3], M[9];
    Cov3 Sig;
    bool ok;
};

__device__ __forceinline__ void load_shape(const float *quats, const float *log_scales, int64_t g, Shape &sh) {
    float4 q = reinterpret_cast<const float4 *>(quats)[g];
    sh.qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    sh.ok = sh.qn > 0.f;
    float inv = sh.ok ? 1.f / sh.qn : 0.f;
    sh.qh[0] = q.x * inv; sh.qh[1] = q.y * inv; sh.qh[2] = q.z * inv; sh.qh[3] = q.w * inv;
    quat_rot(sh.qh, sh.Rq);
#pragma unroll
    for (int c = 0; c < 3; ++c) sh.s[c] = expf(log_scales[3 * g + c]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) sh.M[3 * r + c] = sh.Rq[3 * r + c] * sh.s[c];
    const float *M = sh.M;
    sh.Sig.m[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    sh.Sig.m[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    sh.Sig.m[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    sh.Sig.m[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    sh.Sig.m[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    sh.Sig.m[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

__device__ __forceinline__ float sym(const Cov3 &c, int r, int k) {
    const int idx[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    return c.m[idx[3 * r + k]];
}

// View-dependent geometry of one (view, Gaussian) pair.
struct Geo {
    float p[3];
    Cov3 Sc;                     // R_cw Sigma R_cw^T
    float j00, j02, j11, j12;    // perspective Jacobian at the clamped point
    float tx, ty;                // clamped (x/z, y/z) where J is evaluated
    bool in_x, in_y;             // whether x/z, y/z lie inside the clamp interval
    float a, b, c;               // Sigma2D + lowpass I
    float A, B, C;               // its inverse
    float u, v;                  // f32 centre (u_lo, v_lo: remainders, forward only)
    float ulo, vlo;
    bool ok;
};

// EWA projection of one Gaussian into view v.  J is evaluated at (x/z, y/z)
// clamped to the view table's interval: by default the view widened by 15% of its
// size per side (1.3 x the half field of view for a centred principal point), which
// keeps splats whose centres fall far outside the view from stretching with
// (x/z)^2; the whole line for the exact Jacobian.  The centre is not clamped.
__device__ __forceinline__ void project_geo(const float mu[3], const Shape &sh, const float R[9], const float t[3],
                                            const ViewTable &vt, int v, const Params &prm, Geo &o,
                                            bool precise_centre = false) {
    const float fx = vt.fx[v], fy = vt.fy[v], cx = vt.cx[v], cy = vt.cy[v];
    // p = R mu + t as an explicit fused chain; p.z is the sort key
#pragma unroll
    for (int r = 0; r < 3; ++r)
        o.p[r] = __fmaf_rn(R[3 * r], mu[0], __fmaf_rn(R[3 * r + 1], mu[1], __fmaf_rn(R[3 * r + 2], mu[2], t[r])));
    o.ok = sh.ok && (o.p[2] > prm.z_near);
    if (!o.ok) return;
    // Sc = R Sigma R^T
    float RS[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            RS[3 * r + k] = R[3 * r] * sym(sh.Sig, 0, k) + R[3 * r + 1] * sym(sh.Sig, 1, k) + R[3 * r + 2] * sym(sh.Sig, 2, k);
    const int pr[6] = {0, 0, 0, 1, 1, 2}, pc[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        int r = pr[e], k = pc[e];
        o.Sc.m[e] = RS[3 * r] * R[3 * k] + RS[3 * r + 1] * R[3 * k + 1] + RS[3 * r + 2] * R[3 * k + 2];
    }
    float iz = 1.f / o.p[2];
    const float xz = o.p[0] * iz, yz = o.p[1] * iz;
    o.in_x = xz >= vt.jx_lo[v] && xz <= vt.jx_hi[v];
    o.in_y = yz >= vt.jy_lo[v] && yz <= vt.jy_hi[v];
    o.tx = fminf(fmaxf(xz, vt.jx_lo[v]), vt.jx_hi[v]);
    o.ty = fminf(fmaxf(yz, vt.jy_lo[v]), vt.jy_hi[v]);
    o.j00 = fx * iz;
    o.j11 = fy * iz;
    o.j02 = -fx * o.tx * iz;
    o.j12 = -fy * o.ty * iz;
    const float *S = o.Sc.m;
    o.a = o.j00 * o.j00 * S[0] + 2.f * o.j00 * o.j02 * S[2] + o.j02 * o.j02 * S[5] + prm.lowpass;
    o.b = o.j00 * o.j11 * S[1] + o.j00 * o.j12 * S[2] + o.j02 * o.j11 * S[4] + o.j02 * o.j12 * S[5];
    o.c = o.j11 * o.j11 * S[3] + 2.f * o.j11 * o.j12 * S[4] + o.j12 * o.j12 * S[5] + prm.lowpass;
    if (precise_centre) {
        // p and the pinhole division in compensated arithmetic: u, v to ~1e-10 px
        float xh, xl, yh, yl, zh, zl;
        dot3_dd(R[0], R[1], R[2], mu[0], mu[1], mu[2], t[0], xh, xl);
        dot3_dd(R[3], R[4], R[5], mu[0], mu[1], mu[2], t[1], yh, yl);
        dot3_dd(R[6], R[7], R[8], mu[0], mu[1], mu[2], t[2], zh, zl);
        proj_dd(fx, xh, xl, zh, zl, cx, o.u, o.ulo);
        proj_dd(fy, yh, yl, zh, zl, cy, o.v, o.vlo);
    } else {
        o.u = fx * o.p[0] * iz + cx;
        o.v = fy * o.p[1] * iz + cy;
        o.ulo = o.vlo = 0.f;
    }
    // det = a c - b^2 by Kahan's FMA algorithm for 2x2 determinants (the rounding error of b^2,
    // recovered exactly by a second FMA, is added back): accurate to a few units in the last
    // place of det itself even when a c and b^2 nearly cancel (an elongated splat), so the
    // inverse needs no wider arithmetic
    const float bb = __fmul_rn(o.b, o.b);
    const float det = __fadd_rn(__fmaf_rn(o.a, o.c, -bb), __fmaf_rn(-o.b, o.b, bb));
    if (!(det > 0.f) || !isfinite(det)) { o.ok = false; return; }
    const float id = 1.f / det;
    o.A = o.c * id; o.B = -o.b * id; o.C = o.a * id;
    o.ok = isfinite(o.u) && isfinite(o.v) && isfinite(o.A) && isfinite(o.B) && isfinite(o.C);
}

__global__ void __launch_bounds__(256) project_fwd_kernel(ViewTable vt, Params prm, int64_t n,
                                                          const float *__restrict__ means,
                                                          const float *__restrict__ quats,
                                                          const float *__restrict__ log_scales,
                                                          const float *__restrict__ logits,
                                                          const float *__restrict__ pose_dev, float4 *__restrict__ uvdo,
                                                          float2 *__restrict__ uv_lo, float4 *__restrict__ conic,
                                                          int32_t *__restrict__ touched) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    if (g >= n) return;
    int64_t item = (int64_t)v * n + g;
    Shape sh;
    load_shape(quats, log_scales, g, sh);
    float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    float o = 1.f / (1.f + expf(-logits[g]));
    float R[9], t[3];
    load_pose(vt, pose_dev, v, R, t);
    Geo ge;
    project_geo(mu, sh, R, t, vt, v, prm, ge, true);
    float4 rec = make_float4(0.f, 0.f, ge.p[2], o);
    float2 lo = make_float2(0.f, 0.f);
    float4 cn = make_float4(0.f, 0.f, 0.f, 0.f);
    int tt = 0;
    if (ge.ok) {
        float mid = 0.5f * (ge.a + ge.c);
        float det = ge.a * ge.c - ge.b * ge.b;
        float lmax = mid + sqrtf(fmaxf(mid * mid - det, 0.f));
        float rr = fminf(prm.radius_sigma * sqrtf(lmax), 16777216.f);
        int r = (int)ceilf(rr);
        if (r > 0) {
            int x0, y0, x1, y1;
            tile_rect(ge.u, ge.v, r, vt.TX[v], vt.TY[v], x0, y0, x1, y1);
            tt = (x1 - x0) * (y1 - y0);
        }
        rec.x = ge.u;
        rec.y = ge.v;
        lo = make_float2(ge.ulo, ge.vlo);
        cn = make_float4(ge.A, ge.B, ge.C, (float)r);
    }
    uvdo[item] = rec;
    uv_lo[item] = lo;
    conic[item] = cn;
    touched[item] = tt;
}

// Register cap: six 128-thread blocks per SM (80 registers, 16 bytes spilled) instead of
// four at 124 registers: the kernel is latency-bound and the extra warps hide it (five
// blocks at 96 registers: -13 %; six: a further -8 %; seven spill 80 bytes).
__global__ void __launch_bounds__(128, 6) project_bwd_kernel(ViewTable vt, Params prm, int64_t n,
                                                          const float *__restrict__ means,
                                                          const float *__restrict__ quats,
                                                          const float *__restrict__ log_scales,
                                                          const float *__restrict__ logits,
                                                          const float *__restrict__ pose_dev,
                                                          const float4 *__restrict__ acc_uvod,
                                                          const float4 *__restrict__ acc_conic,
                                                          const float4 *__restrict__ acc_rgb, int grad_mode,
                                                          float *__restrict__ d_means, float *__restrict__ d_quats,
                                                          float *__restrict__ d_log_scales,
                                                          float *__restrict__ d_logits, float *__restrict__ d_rgb,
                                                          float *__restrict__ pose_part) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    Shape sh;
    load_shape(quats, log_scales, g, sh);
    float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    float gmu[3] = {0.f, 0.f, 0.f};
    float GS[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma (trace form)
    float dop = 0.f;
    for (int v = 0; v < vt.n_views; ++v) {
        int64_t item = (int64_t)v * n + g;
        float4 a0 = acc_uvod[item], a1 = acc_conic[item];
        float tw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool any = (a0.x != 0.f) | (a0.y != 0.f) | (a0.z != 0.f) | (a0.w != 0.f) | (a1.x != 0.f) | (a1.y != 0.f) |
                   (a1.z != 0.f);
        if (any) {
            float R[9], t[3];
            load_pose(vt, pose_dev, v, R, t);
            float fx = vt.fx[v], fy = vt.fy[v];
            Geo ge;
            project_geo(mu, sh, R, t, vt, v, prm, ge);
            if (ge.ok) {
                dop += a0.z;
                // conic -> Sigma2D: G2 = -conic Ghat conic, Ghat = [[dA, dB/2], [dB/2, dC]]
                float hA = a1.x, hB = 0.5f * a1.y, hC = a1.z;
                float X00 = ge.A * hA + ge.B * hB, X01 = ge.A * hB + ge.B * hC;
                float X10 = ge.B * hA + ge.C * hB, X11 = ge.B * hB + ge.C * hC;
                float g00 = -(X00 * ge.A + X01 * ge.B);
                float g01 = -(X00 * ge.B + X01 * ge.C);
                float g11 = -(X10 * ge.B + X11 * ge.C);
                // Sigma2D = J Sc J^T: Gc = J^T G2 J, dJ = 2 G2 J Sc
                Cov3 Gc;
                Gc.m[0] = ge.j00 * ge.j00 * g00;
                Gc.m[1] = ge.j00 * ge.j11 * g01;
                Gc.m[2] = ge.j00 * (ge.j02 * g00 + ge.j12 * g01);
                Gc.m[3] = ge.j11 * ge.j11 * g11;
                Gc.m[4] = ge.j11 * (ge.j02 * g01 + ge.j12 * g11);
                Gc.m[5] = ge.j02 * ge.j02 * g00 + 2.f * ge.j02 * ge.j12 * g01 + ge.j12 * ge.j12 * g11;
                const float *S = ge.Sc.m;
                float JS0[3] = {ge.j00 * S[0] + ge.j02 * S[2], ge.j00 * S[1] + ge.j02 * S[4], ge.j00 * S[2] + ge.j02 * S[5]};
                float JS1[3] = {ge.j11 * S[1] + ge.j12 * S[2], ge.j11 * S[3] + ge.j12 * S[4], ge.j11 * S[4] + ge.j12 * S[5]};
                float dJ00 = 2.f * (g00 * JS0[0] + g01 * JS1[0]);
                float dJ02 = 2.f * (g00 * JS0[2] + g01 * JS1[2]);
                float dJ11 = 2.f * (g01 * JS0[1] + g11 * JS1[1]);
                float dJ12 = 2.f * (g01 * JS0[2] + g11 * JS1[2]);
                // camera-frame centre
                float x = ge.p[0], y = ge.p[1], z = ge.p[2];
                float iz = 1.f / z, iz2 = iz * iz;
                // J02 = -fx t_x / z with t_x = clamp(x / z): dt_x/dx = 1/z, dt_x/dz = -x/z^2 inside, 0 outside
                const float dtx_dx = ge.in_x ? iz : 0.f, dtx_dz = ge.in_x ? -x * iz2 : 0.f;
                const float dty_dy = ge.in_y ? iz : 0.f, dty_dz = ge.in_y ? -y * iz2 : 0.f;
                float gp0 = a0.x * fx * iz + dJ02 * (-fx * iz) * dtx_dx;
                float gp1 = a0.y * fy * iz + dJ12 * (-fy * iz) * dty_dy;
                float gp2 = -a0.x * fx * x * iz2 - a0.y * fy * y * iz2 + a0.w + dJ00 * (-fx * iz2) +
                            dJ02 * (-fx * dtx_dz * iz + fx * ge.tx * iz2) + dJ11 * (-fy * iz2) +
                            dJ12 * (-fy * dty_dz * iz + fy * ge.ty * iz2);
#pragma unroll
                for (int k = 0; k < 3; ++k) gmu[k] += R[k] * gp0 + R[3 + k] * gp1 + R[6 + k] * gp2;
                // Sigma gradient: R^T Gc R
                float GR[9];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        GR[3 * r + k] = sym(Gc, r, 0) * R[k] + sym(Gc, r, 1) * R[3 + k] + sym(Gc, r, 2) * R[6 + k];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int k = 0; k < 3; ++k) GS[3 * r + k] += R[r] * GR[k] + R[3 + r] * GR[3 + k] + R[6 + r] * GR[6 + k];
                if (grad_mode & GS_GRAD_POSE) {
                    // A = Sc Gc - Gc Sc (antisymmetric); twist phi gets p x g_p + 2 (A12, A20, A01)
                    auto prod = [&](int r, int k) {
                        return sym(ge.Sc, r, 0) * sym(Gc, 0, k) + sym(ge.Sc, r, 1) * sym(Gc, 1, k) +
                               sym(ge.Sc, r, 2) * sym(Gc, 2, k);
                    };
                    float A12 = prod(1, 2) - prod(2, 1);
                    float A20 = prod(2, 0) - prod(0, 2);
                    float A01 = prod(0, 1) - prod(1, 0);
                    tw[0] = gp0; tw[1] = gp1; tw[2] = gp2;
                    tw[3] = y * gp2 - z * gp1 + 2.f * A12;
                    tw[4] = z * gp0 - x * gp2 + 2.f * A20;
                    tw[5] = x * gp1 - y * gp0 + 2.f * A01;
                }
            }
        }
        if (grad_mode & GS_GRAD_POSE) {
#pragma unroll
            for (int k = 0; k < 6; ++k) pose_part[((int64_t)v * 6 + k) * n + g] = tw[k];
        }
    }
    if (!(grad_mode & GS_GRAD_MAP)) return;
    // Sigma = M M^T -> M -> (s, Rq) -> q
    float dM[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dM[3 * r + k] = 2.f * (GS[3 * r] * sh.M[k] + GS[3 * r + 1] * sh.M[3 + k] + GS[3 * r + 2] * sh.M[6 + k]);
    float dR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ds = dM[k] * sh.Rq[k] + dM[3 + k] * sh.Rq[3 + k] + dM[6 + k] * sh.Rq[6 + k];
        d_log_scales[3 * g + k] = ds * sh.s[k];
#pragma unroll
        for (int r = 0; r < 3; ++r) dR[3 * r + k] = dM[3 * r + k] * sh.s[k];
    }
    float w = sh.qh[0], x = sh.qh[1], y = sh.qh[2], z = sh.qh[3];
    float gq[4];
    gq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    gq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2.f * x * dR[8]);
    gq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
    gq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
    float dot = gq[0] * sh.qh[0] + gq[1] * sh.qh[1] + gq[2] * sh.qh[2] + gq[3] * sh.qh[3];
    float iq = sh.ok ? 1.f / sh.qn : 0.f;
    float4 dq = make_float4((gq[0] - sh.qh[0] * dot) * iq, (gq[1] - sh.qh[1] * dot) * iq,
                            (gq[2] - sh.qh[2] * dot) * iq, (gq[3] - sh.qh[3] * dot) * iq);
    reinterpret_cast<float4 *>(d_quats)[g] = dq;
#pragma unroll
    for (int k = 0; k < 3; ++k) d_means[3 * g + k] = gmu[k];
    float o = 1.f / (1.f + expf(-logits[g]));
    d_logits[g] = o * (1.f - o) * dop;
    float4 cr = acc_rgb[g];
    d_rgb[3 * g] = cr.x;
    d_rgb[3 * g + 1] = cr.y;
    d_rgb[3 * g + 2] = cr.z;
}

}  // namespace

}  // namespace gs

extern "C" gs_status gs_project(const gs_gaussians *g, const gs_camera *cams, int n_views, const float *pose_dev,
                                const gs_raster_params *p, gs_projected *out, gs_stream stream) {
    GS_NVTX_RANGE("gs_project");
    using namespace gs;
    if (!g || !out || g->n < 0) return GS_ERR_ARG;
    ViewTable vt;
    Params prm;
    if (!make_view_table(cams, n_views, g->n, &vt) || !make_params(p, &prm)) return GS_ERR_ARG;
    apply_jacobian_mode(prm, &vt);
    if (g->n * n_views >= ((int64_t)1 << 30)) return GS_ERR_ARG;
    if (g->n == 0) return GS_OK;
    if (!g->means || !g->quats || !g->log_scales || !g->opacity_logits || !out->uvdo || !out->uv_lo ||
        !out->conic || !out->tiles_touched)
        return GS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(g->quats) | reinterpret_cast<uintptr_t>(out->uvdo) |
         reinterpret_cast<uintptr_t>(out->conic)) & 15 || (reinterpret_cast<uintptr_t>(out->uv_lo) & 7))
        return GS_ERR_ARG;
    dim3 grid(ceil_div(g->n, 256), n_views);
    return launch_pdl(project_fwd_kernel, grid, 256, 0, (cudaStream_t)stream, vt, prm, g->n, g->means, g->quats,
                      g->log_scales, g->opacity_logits, pose_dev, reinterpret_cast<float4 *>(out->uvdo),
                      reinterpret_cast<float2 *>(out->uv_lo), reinterpret_cast<float4 *>(out->conic),
                      out->tiles_touched);
}

extern "C" gs_status gs_project_bwd(const gs_gaussians *g, const gs_camera *cams, int n_views, const float *pose_dev,
                                    const gs_raster_params *p, int grad_mode, const gs_splat_grads *sg,
                                    gs_gaussian_grads *out, float *pose_part, gs_stream stream) {
    GS_NVTX_RANGE("gs_project_bwd");
    using namespace gs;
    if (!g || !sg || g->n < 0) return GS_ERR_ARG;
    if (grad_mode <= 0 || grad_mode > (GS_GRAD_MAP | GS_GRAD_POSE)) return GS_ERR_ARG;
    ViewTable vt;
    Params prm;
    if (!make_view_table(cams, n_views, g->n, &vt) || !make_params(p, &prm)) return GS_ERR_ARG;
    apply_jacobian_mode(prm, &vt);
    const bool map = grad_mode & GS_GRAD_MAP, pose = grad_mode & GS_GRAD_POSE;
    if (map && (!out || !out->means || !out->quats || !out->log_scales || !out->opacity_logits || !out->rgb))
        return GS_ERR_ARG;
    if (pose && !pose_part) return GS_ERR_ARG;
    if (g->n == 0) return GS_OK;
    if (!g->means || !g->quats || !g->log_scales || !g->opacity_logits || !sg->uvod || !sg->conic ||
        (map && !sg->rgb))
        return GS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(g->quats) | reinterpret_cast<uintptr_t>(sg->uvod) |
         reinterpret_cast<uintptr_t>(sg->conic) | reinterpret_cast<uintptr_t>(sg->rgb) |
         reinterpret_cast<uintptr_t>(map ? out->quats : nullptr)) & 15)
        return GS_ERR_ARG;
    dim3 grid(ceil_div(g->n, 128));
    return launch_pdl(project_bwd_kernel, grid, 128, 0, (cudaStream_t)stream, vt, prm, g->n, g->means, g->quats,
                      g->log_scales, g->opacity_logits, pose_dev, reinterpret_cast<const float4 *>(sg->uvod),
                      reinterpret_cast<const float4 *>(sg->conic), reinterpret_cast<const float4 *>(sg->rgb),
                      grad_mode, map ? out->means : nullptr, map ? out->quats : nullptr,
                      map ? out->log_scales : nullptr, map ? out->opacity_logits : nullptr,
                      map ? out->rgb : nullptr, pose ? pose_part : nullptr);
}
