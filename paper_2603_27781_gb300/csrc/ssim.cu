// SSIM term of the mapping colour loss (Eq. 15, read as lambda_c lambda (1 - SSIM)):
// per view, channel and pixel the window moments over an 11x11 Gaussian window
// (sigma 1.5, zero outside the image), S = (2 mx my + C1)(2 sxy + C2) /
// ((mx^2 + my^2 + C1)(sx + sy + C2)), averaged over the view's 3 P_v positions.
//
// Two passes over 32x16-pixel tiles of one channel (one CTA each, 256 threads):
//   forward: the tile and a 5-pixel halo of the rendered and observed colour in
//     shared memory, the separable window (rows, then columns) applied to x, y,
//     x^2, y^2, x y; per pixel S and the partials A = dS/dmx - 2 mx dS/dsx -
//     my dS/dsxy, B = dS/dsx, C = dS/dsxy (stored, f32), and the tile's sum of S
//     (f64 partial, fixed order);
//   backward: dS/dx(q) = sum_p w(q - p) (A(p) + 2 B(p) x(q) + C(p) y(q)), the
//     same separable window over A, B and C, added to the colour gradient.
#include "common.cuh"

namespace gs {
namespace {

constexpr int kSW = 32, kSH = 16, kR = 5;                 // tile and window radius
constexpr int kIW = kSW + 2 * kR, kIH = kSH + 2 * kR;     // tile with halo: 42 x 26
constexpr int kSThreads = 256;

struct SsimTable {
    int off[kMaxViews + 1];  // first CTA of each view (3 channels x tiles)
    int tx[kMaxViews];       // tiles per row
    float g[11];             // normalised 1D window
    float coef;              // lambda_c * lambda
};

__device__ __forceinline__ void locate(const ViewTable &vt, const SsimTable &t, int &v, int &ch, int &x0, int &y0) {
    const int b = blockIdx.x;
    v = 0;
    while (v + 1 < vt.n_views && b >= t.off[v + 1]) ++v;
    const int tiles = (t.off[v + 1] - t.off[v]) / 3;
    const int r = b - t.off[v];
    ch = r / tiles;
    const int k = r - ch * tiles;
    x0 = (k % t.tx[v]) * kSW;
    y0 = (k / t.tx[v]) * kSH;
}

// Block sum in f64 (fixed order); thread 0 gets the total.
__device__ double block_sum_d(double x, double *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[w] = x;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kSThreads / 32; ++i) t += s_red[i];
    return t;
}

// Loads a channel tile with halo (zero outside the image) into dst[kIH][kIW].
__device__ __forceinline__ void load_halo(const float *src, int W, int H, int x0, int y0, float (*dst)[kIW]) {
    for (int i = threadIdx.x; i < kIW * kIH; i += kSThreads) {
        const int r = i / kIW, c = i - r * kIW;
        const int gy = y0 + r - kR, gx = x0 + c - kR;
        dst[r][c] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? src[(int64_t)gy * W + gx] : 0.f;
    }
}

__global__ void __launch_bounds__(kSThreads) ssim_fwd_kernel(ViewTable vt, SsimTable t, const float *rgb,
                                                             const float *trgb, int64_t P, float *maps,
                                                             double *part) {
    __shared__ float s_x[kIH][kIW], s_y[kIH][kIW];
    __shared__ float s_h[5][kIH][kSW];
    __shared__ double s_red[kSThreads / 32];
    int v, ch, x0, y0;
    locate(vt, t, v, ch, x0, y0);
    const int W = vt.W[v], H = vt.H[v];
    const int64_t base = ch * P + vt.pix_off[v];
    load_halo(rgb + base, W, H, x0, y0, s_x);
    load_halo(trgb + base, W, H, x0, y0, s_y);
    __syncthreads();
    for (int i = threadIdx.x; i < kIH * kSW; i += kSThreads) {
        const int r = i / kSW, c = i - r * kSW;
        float mx = 0.f, my = 0.f, mxx = 0.f, myy = 0.f, mxy = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = t.g[k], a = s_x[r][c + k], b = s_y[r][c + k];
            mx = fmaf(w, a, mx);
            my = fmaf(w, b, my);
            mxx = fmaf(w * a, a, mxx);
            myy = fmaf(w * b, b, myy);
            mxy = fmaf(w * a, b, mxy);
        }
        s_h[0][r][c] = mx; s_h[1][r][c] = my; s_h[2][r][c] = mxx; s_h[3][r][c] = myy; s_h[4][r][c] = mxy;
    }
    __syncthreads();
    constexpr float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    const int64_t Pv = (int64_t)W * H;
    double ssum = 0.0;
    for (int i = threadIdx.x; i < kSW * kSH; i += kSThreads) {
        const int r = i / kSW, c = i - r * kSW;
        const int py = y0 + r, px = x0 + c;
        if (py >= H || px >= W) continue;
        float m[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) s = fmaf(t.g[k], s_h[q][r + k][c], s);
            m[q] = s;
        }
        const float mx = m[0], my = m[1];
        const float sx = m[2] - mx * mx, sy = m[3] - my * my, sxy = m[4] - mx * my;
        const float N1 = 2.f * mx * my + C1, N2 = 2.f * sxy + C2;
        const float D1 = mx * mx + my * my + C1, D2 = sx + sy + C2;
        const float inv = 1.f / (D1 * D2);
        const float S = N1 * N2 * inv;
        const float dS_dmx = 2.f * my * N2 * inv - S * 2.f * mx / D1;
        const float dS_dsx = -S / D2;
        const float dS_dsxy = 2.f * N1 * inv;
        const int64_t o = (int64_t)py * W + px;
        // maps of (channel, view): 3 planes of P_v floats at 3 (ch P + pix_off(v))
        const int64_t mb = (int64_t)3 * (ch * P + vt.pix_off[v]);
        maps[mb + o] = dS_dmx - 2.f * mx * dS_dsx - my * dS_dsxy;
        maps[mb + Pv + o] = dS_dsx;
        maps[mb + 2 * Pv + o] = dS_dsxy;
        ssum += (double)S;
    }
    const double tot = block_sum_d(ssum, s_red);
    if (threadIdx.x == 0) {
        // colour-term share of this tile: coef (1 - S_sum / (3 P_v)) summed over the view's tiles
        double val = -(double)t.coef * tot / (3.0 * (double)Pv);
        if (blockIdx.x == t.off[v]) val += (double)t.coef;
        part[3 * blockIdx.x] = val;
        part[3 * blockIdx.x + 1] = 0.0;
        part[3 * blockIdx.x + 2] = 0.0;
    }
}

__global__ void __launch_bounds__(kSThreads) ssim_bwd_kernel(ViewTable vt, SsimTable t, const float *rgb,
                                                             const float *trgb, int64_t P, const float *maps,
                                                             float *g_rgb) {
    __shared__ float s_m[3][kIH][kIW];
    __shared__ float s_h[3][kIH][kSW];
    int v, ch, x0, y0;
    locate(vt, t, v, ch, x0, y0);
    const int W = vt.W[v], H = vt.H[v];
    const int64_t Pv = (int64_t)W * H;
    const int64_t mb = (int64_t)3 * (ch * P + vt.pix_off[v]);
#pragma unroll
    for (int q = 0; q < 3; ++q) load_halo(maps + mb + q * Pv, W, H, x0, y0, s_m[q]);
    __syncthreads();
    for (int i = threadIdx.x; i < kIH * kSW; i += kSThreads) {
        const int r = i / kSW, c = i - r * kSW;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) s = fmaf(t.g[k], s_m[q][r][c + k], s);
            s_h[q][r][c] = s;
        }
    }
    __syncthreads();
    const float scale = -t.coef / (3.f * (float)Pv);
    const int64_t base = ch * P + vt.pix_off[v];
    for (int i = threadIdx.x; i < kSW * kSH; i += kSThreads) {
        const int r = i / kSW, c = i - r * kSW;
        const int py = y0 + r, px = x0 + c;
        if (py >= H || px >= W) continue;
        float f[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) s = fmaf(t.g[k], s_h[q][r + k][c], s);
            f[q] = s;
        }
        const int64_t pix = base + (int64_t)py * W + px;
        const float grad = f[0] + 2.f * rgb[pix] * f[1] + trgb[pix] * f[2];
        g_rgb[pix] = fmaf(scale, grad, g_rgb[pix]);
    }
}

}  // namespace

int ssim_blocks(const ViewTable &vt) {
    int b = 0;
    for (int v = 0; v < vt.n_views; ++v) b += 3 * ((vt.W[v] + kSW - 1) / kSW) * ((vt.H[v] + kSH - 1) / kSH);
    return b;
}

// Adds the SSIM term to the loss partials (rows part[0 .. ssim_blocks) of f64 [.][3], colour
// column) and its gradient to g_rgb.  maps: f32 scratch [9 P].
gs_status launch_ssim(const ViewTable &vt, float coef, const float *rgb, const float *trgb, float *maps,
                      double *part, float *g_rgb, cudaStream_t st) {
    SsimTable t;
    t.off[0] = 0;
    for (int v = 0; v < vt.n_views; ++v) {
        t.tx[v] = (vt.W[v] + kSW - 1) / kSW;
        t.off[v + 1] = t.off[v] + 3 * t.tx[v] * ((vt.H[v] + kSH - 1) / kSH);
    }
    double g[11], gs = 0.0;
    for (int k = 0; k < 11; ++k) {
        g[k] = exp(-(double)((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5));
        gs += g[k];
    }
    for (int k = 0; k < 11; ++k) t.g[k] = (float)(g[k] / gs);
    t.coef = coef;
    const int blocks = t.off[vt.n_views];
    if (blocks == 0) return GS_OK;
    const int64_t P = vt.pix_off[vt.n_views];
    ssim_fwd_kernel<<<blocks, kSThreads, 0, st>>>(vt, t, rgb, trgb, P, maps, part);
    ssim_bwd_kernel<<<blocks, kSThreads, 0, st>>>(vt, t, rgb, trgb, P, maps, g_rgb);
    return last_launch();
}

}  // namespace gs
