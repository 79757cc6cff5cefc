// Losses and reductions around the blend:
//   - decoder + L1 colour/depth + semantic cross-entropy with image gradients
//     (Eq. 8, 15-17) and the tracking mask M_obs (Eq. 21), whose depth-error
//     median is found by a 4-pass 8-bit radix select over f32 bit patterns;
//   - depth-adaptive scale regularisation (Eq. 12);
//   - the reduction of the pose-twist contributions (supplementary B.1);
//   - the Adam + SE(3) exponential pose step (Sec. 3.4, supplementary C.1).
//
// Reductions are two-level and deterministic: a bounded grid of blocks writes
// per-block partials (f32 sums inside a thread, f64 across threads and
// blocks), and a finishing step sums the partials in a fixed order.  GB300's
// f64 rate is a small fraction of its f32 rate, so f64 is kept to the
// cross-thread sums.
#include <math.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace gs {
namespace {

constexpr int kMaxK = 32;

// Block-wide (256 threads) exclusive scan of one u32 per thread.
__device__ __forceinline__ uint32_t scan256(uint32_t x, uint32_t *total, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane < 8 ? s_warp[lane] : 0;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < 8) s_warp[lane] = ti - t;
        if (lane == 7) s_warp[8] = ti;
    }
    __syncthreads();
    const uint32_t r = s_warp[w] + inc - x;
    *total = s_warp[8];
    __syncthreads();
    return r;
}

// Lower median (element floor((n-1)/2) in sorted order) of view v, as the f32
// bit pattern selected digit by digit from the per-pass histograms
// hist[p][v][256] (p < passes); the whole 256-thread block cooperates.
__device__ uint32_t block_select(const uint32_t *hist, int n_views, int v, int passes) {
    __shared__ uint32_t s_warp[9];
    __shared__ uint32_t s_k, s_prefix, s_sel, s_below;
    const int d = threadIdx.x;
    uint32_t n;
    scan256(hist[(size_t)v * 256 + d], &n, s_warp);
    if (d == 0) {
        s_k = n > 0 ? (n - 1) / 2 : 0;
        s_prefix = 0;
    }
    __syncthreads();
    if (n == 0) return 0;
    for (int p = 0; p < passes; ++p) {
        const uint32_t h = hist[((size_t)p * n_views + v) * 256 + d];
        uint32_t tot;
        const uint32_t ex = scan256(h, &tot, s_warp);
        const uint32_t k = s_k;
        if (k >= ex && k < ex + h) {
            s_sel = d;
            s_below = ex;
        }
        __syncthreads();
        if (d == 0) {
            s_prefix |= s_sel << (24 - 8 * p);
            s_k = k - s_below;
        }
        __syncthreads();
    }
    return s_prefix;
}

__device__ __forceinline__ float depth_error(float d, float dgt) { return fabsf(__fsub_rn(d, dgt)); }

__global__ void __launch_bounds__(256) median_hist_kernel(ViewTable vt, int pass, const float *depth,
                                                          const float *tdepth, uint32_t *hist) {
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_prefix;
    const int v = blockIdx.y;
    const int64_t Pv = (int64_t)vt.W[v] * vt.H[v];
    s_hist[threadIdx.x] = 0;
    const uint32_t pre = pass > 0 ? block_select(hist, vt.n_views, v, pass) : 0u;
    if (threadIdx.x == 0) s_prefix = pre;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * 256; base < Pv; base += (int64_t)gridDim.x * 256) {
        const int64_t i = base + threadIdx.x;
        bool valid = false;
        uint32_t bits = 0;
        if (i < Pv) {
            const int64_t pix = vt.pix_off[v] + i;
            const float dgt = tdepth[pix];
            if (dgt > 0.f) {
                bits = __float_as_uint(depth_error(depth[pix], dgt));
                valid = pass == 0 || (bits >> (32 - 8 * pass)) == (s_prefix >> (32 - 8 * pass));
            }
        }
        const uint32_t dg = valid ? (bits >> (24 - 8 * pass)) & 255u : 256u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_hist[dg], __popc(peers));
    }
    __syncthreads();
    const uint32_t c = s_hist[threadIdx.x];
    if (c) atomicAdd(&hist[((size_t)pass * vt.n_views + v) * 256 + threadIdx.x], c);
}

struct LossP {
    float color, depth, sem, tau_obs;  // color: weight of the L1 part
    int mask_mode, K;
    float ssim_coef;                   // lambda_c lambda of Eq. 15 (0: no SSIM term)
    float *ssim_maps;
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

// Sum over the block (any multiple of 32 threads, up to 1024) in f64; valid in thread 0.
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
    return t;
}

// Per-pixel losses and image gradients; per-block partials of the decoder
// gradient (f32 [nblk][K*D + K]) and of the three loss sums (f64 [nblk][3]).
//
// KC is a compile-time bound on the class count (K <= KC).  The decoder
// gradient dW[k][d] = sum_px dz_k f_d, db[k] = sum_px dz_k is a contraction over
// pixels: each warp stages dz and f of its 32 pixels in shared memory, and every
// lane keeps EPL consecutive entries of one row of dW (lanes < KC also one
// entry of db) in registers for the whole grid-stride loop; they reach the
// block's shared sums once, at the end.
template <int D, int KC>
struct LossShape {
    static constexpr int NT = (KC <= 8 && D <= 16) ? 256 : 128;  // keeps the static shared memory < 48 KB
    static constexpr int WARPS = NT / 32;
    static constexpr int DD = D > 0 ? D : 1;
    static constexpr int EPL = D > 0 ? KC * D / 32 : 1;          // dW entries per lane
    static constexpr int FROW = D > 0 ? D + 4 : 4;              // staged feature row (16-byte aligned, padded)
    static_assert(D == 0 || ((KC * D) % 32 == 0 && D % EPL == 0), "lane blocks of dW");
};

template <int D, int KC>
__global__ void __launch_bounds__(LossShape<D, KC>::NT) loss_kernel(
    ViewTable vt, LossP lp, const float *__restrict__ rgb, const float *__restrict__ depth,
    const float *__restrict__ sil, const float *__restrict__ feat, const float *__restrict__ trgb,
    const float *__restrict__ tdepth, const uint8_t *__restrict__ label, const float *__restrict__ Wd,
    const float *__restrict__ bd, int64_t P, const uint32_t *__restrict__ med_hist, float *__restrict__ g_rgb,
    float *__restrict__ g_depth, float *__restrict__ g_sil, float *__restrict__ g_feat, float *__restrict__ g_coef,
    float *__restrict__ part_f, double *__restrict__ part_d, float *__restrict__ mask_out,
    float *__restrict__ median_out) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    using SH = LossShape<D, KC>;
    constexpr int NT = SH::NT, DD = SH::DD, EPL = SH::EPL;
    __shared__ __align__(16) float s_W[KC * DD];
    __shared__ float s_b[KC];
    __shared__ float s_dW[KC * DD + KC];
    __shared__ float s_dz[SH::WARPS][32][KC + 1];
    __shared__ __align__(16) float s_f[SH::WARPS][32][SH::FROW];
    __shared__ double s_red[8];
    __shared__ float s_med;
    const int v = blockIdx.y;
    const int blk = v * gridDim.x + blockIdx.x;
    const int64_t Pv = (int64_t)vt.W[v] * vt.H[v];
    const int K = lp.K, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nval = K * D + K;
    for (int i = tid; i < K * D; i += NT) s_W[i] = Wd[i];
    for (int i = tid; i < K; i += NT) s_b[i] = bd[i];
    for (int i = tid; i < nval; i += NT) s_dW[i] = 0.f;
    float med = 0.f;
    if (lp.mask_mode == 1) med = __uint_as_float(block_select(med_hist, vt.n_views, v, 4));
    if (tid == 0) {
        s_med = med;
        if (median_out && blockIdx.x == 0) median_out[v] = med;
    }
    __syncthreads();
    const float invP = 1.f / (float)Pv;
    float lc = 0.f, ld = 0.f, ls = 0.f;  // per-thread partial sums (a thread sees few pixels)
    // this lane's decoder-gradient entries: dW[kr][d0, d0 + EPL) and db[lane]
    const int kr = D > 0 ? (lane * EPL) / D : 0, d0 = D > 0 ? (lane * EPL) % D : 0;
    float accW[EPL], accb = 0.f;
#pragma unroll
    for (int e = 0; e < EPL; ++e) accW[e] = 0.f;

    // two pixels of the grid-stride loop in flight: the next one's loads issue beside this one's work
#pragma unroll 2
    for (int64_t base = (int64_t)blockIdx.x * NT; base < Pv; base += (int64_t)gridDim.x * NT) {
        const int64_t i = base + tid;
        float f[DD], dz[KC];
#pragma unroll
        for (int k = 0; k < KC; ++k) dz[k] = 0.f;
#pragma unroll
        for (int d = 0; d < DD; ++d) f[d] = 0.f;
        if (i < Pv) {
            const int64_t pix = vt.pix_off[v] + i;
            const float dgt = tdepth[pix], dd = depth[pix];
            float m = 1.f;
            if (lp.mask_mode == 1)
                m = (sil[pix] > lp.tau_obs && dgt > 0.f && depth_error(dd, dgt) < 10.f * s_med) ? 1.f : 0.f;
            if (mask_out) mask_out[pix] = m;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float r = rgb[c * P + pix] - trgb[c * P + pix];
                lc += m * fabsf(r);
                g_rgb[c * P + pix] = m * lp.color * (r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f)) * invP;
            }
            float gd = 0.f;
            if (dgt > 0.f) {
                const float r = dd - dgt;
                ld += m * fabsf(r);
                gd = m * lp.depth * (r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f)) * invP;
            }
            g_depth[pix] = gd;
            g_sil[pix] = 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) f[d] = feat[d * P + pix];
            const int lab = label[pix];
            if (lab != 255 && lab < K) {
                // z = W f + b, each row read as float4 and summed in four partial sums
                float z[KC];
                float zmax = -INFINITY;
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    z[k] = 0.f;
                    if (k < K) {
                        float a[4] = {0.f, 0.f, 0.f, 0.f};
                        if constexpr (D % 4 == 0) {
                            const float4 *wr = reinterpret_cast<const float4 *>(s_W + k * D);
#pragma unroll
                            for (int q = 0; q < D / 4; ++q) {
                                const float4 w4 = wr[q];
                                a[0] = fmaf(w4.x, f[4 * q], a[0]);
                                a[1] = fmaf(w4.y, f[4 * q + 1], a[1]);
                                a[2] = fmaf(w4.z, f[4 * q + 2], a[2]);
                                a[3] = fmaf(w4.w, f[4 * q + 3], a[3]);
                            }
                        } else {
#pragma unroll
                            for (int d = 0; d < D; ++d) a[d & 3] = fmaf(s_W[k * D + d], f[d], a[d & 3]);
                        }
                        const float s = s_b[k] + ((a[0] + a[1]) + (a[2] + a[3]));
                        z[k] = s;
                        zmax = fmaxf(zmax, s);
                    }
                }
                // softmax from one exponential per class: p_k = e_k / sum_j e_j, e_k = exp(z_k - zmax)
                float e[KC], se = 0.f, zl = 0.f;
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    e[k] = 0.f;
                    if (k < K) {
                        e[k] = expf(z[k] - zmax);
                        se += e[k];
                        if (k == lab) zl = z[k];
                    }
                }
                const float lse = zmax + logf(se);
                ls += m * (lse - zl);
                const float scale = m * lp.sem * invP;
                const float inv_se = 1.f / se;
#pragma unroll
                for (int k = 0; k < KC; ++k)
                    if (k < K) dz[k] = scale * (e[k] * inv_se - (k == lab ? 1.f : 0.f));
            }
            if (g_coef) {
                // the factored feature gradient: dL/dz itself (g_feat = W^T dz is left to the backward)
#pragma unroll
                for (int k = 0; k < KC; ++k)
                    if (k < K) g_coef[k * P + pix] = dz[k];
            } else {
                float gf[DD];
#pragma unroll
                for (int d = 0; d < DD; ++d) gf[d] = 0.f;
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    if (k < K) {
                        if constexpr (D % 4 == 0) {
                            const float4 *wr = reinterpret_cast<const float4 *>(s_W + k * D);
#pragma unroll
                            for (int q = 0; q < D / 4; ++q) {
                                const float4 w4 = wr[q];
                                gf[4 * q] = fmaf(w4.x, dz[k], gf[4 * q]);
                                gf[4 * q + 1] = fmaf(w4.y, dz[k], gf[4 * q + 1]);
                                gf[4 * q + 2] = fmaf(w4.z, dz[k], gf[4 * q + 2]);
                                gf[4 * q + 3] = fmaf(w4.w, dz[k], gf[4 * q + 3]);
                            }
                        } else {
#pragma unroll
                            for (int d = 0; d < D; ++d) gf[d] = fmaf(s_W[k * D + d], dz[k], gf[d]);
                        }
                    }
                }
#pragma unroll
                for (int d = 0; d < D; ++d) g_feat[d * P + pix] = gf[d];
            }
        }
        if (K > 0) {
            // stage the warp's dz and f, then accumulate this lane's dW / db entries over its 32 pixels
#pragma unroll
            for (int k = 0; k < KC; ++k) s_dz[wid][lane][k] = dz[k];
            if constexpr (D > 0) {
                float4 *fr = reinterpret_cast<float4 *>(&s_f[wid][lane][0]);
#pragma unroll
                for (int q = 0; q < D / 4; ++q) fr[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
            }
            __syncwarp();
#pragma unroll 4
            for (int px = 0; px < 32; ++px) {
                if constexpr (D > 0) {
                    const float zk = s_dz[wid][px][kr];
                    if constexpr (EPL % 4 == 0) {
                        const float4 *fr = reinterpret_cast<const float4 *>(&s_f[wid][px][d0]);
#pragma unroll
                        for (int q = 0; q < EPL / 4; ++q) {
                            const float4 fv = fr[q];
                            accW[4 * q] = fmaf(zk, fv.x, accW[4 * q]);
                            accW[4 * q + 1] = fmaf(zk, fv.y, accW[4 * q + 1]);
                            accW[4 * q + 2] = fmaf(zk, fv.z, accW[4 * q + 2]);
                            accW[4 * q + 3] = fmaf(zk, fv.w, accW[4 * q + 3]);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) accW[e] = fmaf(zk, s_f[wid][px][d0 + e], accW[e]);
                    }
                }
                if (lane < KC) accb += s_dz[wid][px][lane];
            }
            __syncwarp();
        }
    }
    // the warps' sums enter the block's in warp order (one warp at a time), so the decoder
    // gradient is the same bits on every run and through every entry point
    for (int w = 0; w < SH::WARPS; ++w) {
        if (K > 0 && wid == w) {
            if constexpr (D > 0) {
                if (kr < K) {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) s_dW[kr * D + d0 + e] += accW[e];
                }
            }
            if (lane < K) s_dW[K * D + lane] += accb;
        }
        __syncthreads();
    }
    // per-block partials, weighted and normalised by the view's pixel count
    const double wc = block_sum_f64((double)lc * lp.color / (double)Pv, s_red);
    const double wd = block_sum_f64((double)ld * lp.depth / (double)Pv, s_red);
    const double wsm = block_sum_f64((double)ls * lp.sem / (double)Pv, s_red);
    __syncthreads();
    for (int j = tid; j < nval; j += NT) part_f[(size_t)blk * nval + j] = s_dW[j];
    if (tid == 0) {
        part_d[3 * blk] = wc;
        part_d[3 * blk + 1] = wd;
        part_d[3 * blk + 2] = wsm;
    }
}

// Sums the per-block partials in a fixed order (nblk rows of decoder partials, nrows_d rows
// of loss-term partials: the loss blocks, then any SSIM tiles).  Block j < K*D+K reduces decoder
// gradient column j; blocks nval+t (t < 3) loss term t; block nval+3 the total
// (recomputing the three terms in the same order, so the total is their exact sum).
__global__ void __launch_bounds__(256) loss_finish_kernel(int nblk, int nrows_d, int K, int D, const float *part_f,
                                                          const double *part_d, float *dW, float *db,
                                                          double *loss_out) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ double s_red[8];
    const int nval = K * D + K, j = blockIdx.x;
    if (j < nval) {
        double x = 0;
        for (int b = threadIdx.x; b < nblk; b += 256) x += (double)part_f[(size_t)b * nval + j];
        const double t = block_sum_f64(x, s_red);
        if (threadIdx.x == 0) {
            if (j < K * D) dW[j] = (float)t;
            else db[j - K * D] = (float)t;
        }
        return;
    }
    const int term = j - nval;
    double tot[3];
    for (int c = 0; c < 3; ++c) {
        double x = 0;
        for (int b = threadIdx.x; b < nrows_d; b += 256) x += part_d[3 * b + c];
        tot[c] = block_sum_f64(x, s_red);
    }
    if (threadIdx.x == 0) loss_out[term < 3 ? 1 + term : 0] = term < 3 ? tot[term] : tot[0] + tot[1] + tot[2];
}

// --------------------------------------------------------------------- DSR
// Compensated (Kahan) f32 accumulation inside a thread.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

constexpr int kRedBlocks = 512;

// Calls f(i, x[i]) for the elements of x this thread owns: block b owns a contiguous range
// (a multiple of 4 long), which its threads read as float4 with four loads in flight per
// iteration (scalar loads if x is not 16-byte aligned); a fixed assignment, so per-thread
// sums are reproducible.
template <typename F>
__device__ __forceinline__ void for_my_elements(int64_t m, const float *x, F f) {
    const int64_t per = ((m + gridDim.x - 1) / gridDim.x + 3) / 4 * 4;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(m, b0 + per);
    if (b0 >= b1) return;
    if (reinterpret_cast<uintptr_t>(x) & 15) {
        for (int64_t e = b0 + threadIdx.x; e < b1; e += blockDim.x) f(e, x[e]);
        return;
    }
    const int64_t n4 = (b1 - b0) / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(x + b0);
    for (int64_t i = threadIdx.x; i < n4; i += 4 * (int64_t)blockDim.x) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t j = i + u * (int64_t)blockDim.x;
            v[u] = j < n4 ? x4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t j = i + u * (int64_t)blockDim.x;
            if (j < n4) {
                const int64_t e = b0 + 4 * j;
                f(e, v[u].x);
                f(e + 1, v[u].y);
                f(e + 2, v[u].z);
                f(e + 3, v[u].w);
            }
        }
    }
    for (int64_t e = b0 + 4 * n4 + threadIdx.x; e < b1; e += blockDim.x) f(e, x[e]);
}


// True in the block that finishes last (its partial and every other block's are written
// and visible); that block then resets *ctr for the next call.
__device__ bool last_block(uint32_t *ctr) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    __syncthreads();
    return s_last;
}

// Sum of a strided f64 partial column written by other blocks of this grid (read past L1).
__device__ double sum_partials_cg(const double *part, int stride, int col, int nb, double *s_red) {
    double x = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) x += __ldcg(part + (size_t)b * stride + col);
    return block_sum_f64(x, s_red);
}

// Pass 1 of Eq. 12: per-block sums of s and s^2 over the 3N scales; the last block turns
// them into the population mean and deviation, out[1], out[2] (detached constants).
__global__ void __launch_bounds__(256) dsr_stats_kernel(int64_t m, const float *ls, double *part, double *out,
                                                        uint32_t *ctr) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ double s_red[8];
    Kahan s1, s2;
    for_my_elements(m, ls, [&](int64_t, float l) {
        const float s = expf(l);
        s1.add(s);
        s2.add(s * s);
    });
    const double t1 = block_sum_f64((double)s1.s - s1.c, s_red);
    const double t2 = block_sum_f64((double)s2.s - s2.c, s_red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = t1;
        part[2 * blockIdx.x + 1] = t2;
    }
    if (!last_block(ctr)) return;
    const double u1 = sum_partials_cg(part, 2, 0, gridDim.x, s_red);
    const double u2 = sum_partials_cg(part, 2, 1, gridDim.x, s_red);
    if (threadIdx.x == 0) {
        const double mu = u1 / (double)m, var = u2 / (double)m - mu * mu;
        out[1] = mu;
        out[2] = sqrt(var > 0 ? var : 0.0);
        *ctr = 0u;
    }
}

// Thresholds mu +- 2 sigma in f32, formed the same way by both passes that compare against them.
__device__ __forceinline__ float2 dsr_bounds(const double *out) {
    return make_float2((float)(out[1] + 2.0 * out[2]), (float)(out[1] - 2.0 * out[2]));
}

// Pass 2: per-block sizes and sums of the two sets; the last block forms their means and
// the regulariser's value, out = (lam_big L_big + lam_small L_small, mu, sigma, n_big,
// n_small, L_big, L_small, 0).
__global__ void __launch_bounds__(256) dsr_mask_kernel(int64_t m, const float *ls, double *out, double *mask_part,
                                                       float lam_big, float lam_small, uint32_t *ctr) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ double s_red[8];
    const float2 bd = dsr_bounds(out);
    Kahan sb, ss;
    int nb = 0, ns = 0;
    for_my_elements(m, ls, [&](int64_t, float l) {
        const float s = expf(l);
        if (s > bd.x) { sb.add(s); ++nb; }
        if (s < bd.y) { ss.add(-l); ++ns; }
    });
    const double t[4] = {block_sum_f64((double)sb.s - sb.c, s_red), block_sum_f64((double)nb, s_red),
                         block_sum_f64((double)ss.s - ss.c, s_red), block_sum_f64((double)ns, s_red)};
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) mask_part[4 * blockIdx.x + k] = t[k];
    if (!last_block(ctr)) return;
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = sum_partials_cg(mask_part, 4, k, gridDim.x, s_red);
    if (threadIdx.x == 0) {
        const double Lb = u[1] > 0 ? u[0] / u[1] : 0.0, Ls = u[3] > 0 ? u[2] / u[3] : 0.0;
        out[0] = (double)lam_big * Lb + (double)lam_small * Ls;
        out[3] = u[1];
        out[4] = u[3];
        out[5] = Lb;
        out[6] = Ls;
        out[7] = 0.0;
        *ctr = 0u;
    }
}

__global__ void __launch_bounds__(256) dsr_grad_kernel(int64_t m, const float *ls, float lam_big, float lam_small,
                                                       const double *out, float *d_ls) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    const float2 bd = dsr_bounds(out);
    const double nb = out[3], ns = out[4];
    const float gb = nb > 0 ? (float)(lam_big / nb) : 0.f;
    const float gsm = ns > 0 ? (float)(lam_small / ns) : 0.f;
    for_my_elements(m, ls, [&](int64_t i, float l) {
        const float s = expf(l);
        float g = 0.f;
        if (s > bd.x) g += gb * s;
        if (s < bd.y) g -= gsm;
        if (g != 0.f) d_ls[i] += g;
    });
}

// ------------------------------------------------------------ pose reduction
// Block (x, vk) sums a contiguous slice of component vk in compensated f32 and
// adds its f64 total into d_twist[vk] (at most kPoseBlocks adds per value).
constexpr int kPoseBlocks = 128;

__global__ void __launch_bounds__(256) pose_reduce_kernel(int64_t n, const float *pose_part, double *d_twist) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ double s_red[8];
    const int vk = blockIdx.y;  // view * 6 + component
    const float *p = pose_part + (int64_t)vk * n;
    Kahan s;
    for_my_elements(n, p, [&](int64_t, float x) { s.add(x); });
    const double t = block_sum_f64((double)s.s - s.c, s_red);
    if (threadIdx.x == 0 && t != 0) atomicAdd(&d_twist[vk], t);
}

// ------------------------------------------------------------------ pose step
// bc1 < 0 selects the device step counter: adam[12 * n_views] holds the number
// of steps taken so far (as a double); this step is that number + 1 and the
// bias corrections 1 - beta^step are formed here.
// One block, 16 threads per view: the six Adam components, then the SE(3) exponential
// (one thread for theta and its sin/cos, nine for the 3x3 products, sixteen for T <- E T).
constexpr int kPoseLanes = 16;

__global__ void pose_step_kernel(int n_views, const double *grad, double *Tst, double *adam, double bc1, double bc2,
                                 double lr0, double lr1, double lr2, double lr3, double lr4, double lr5, double b1,
                                 double b2, double lb1, double lb2, double eps, float *pose_f32) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ double s_bc[2];
    __shared__ double s_dl[kMaxViews][6], s_abc[kMaxViews][3], s_R[kMaxViews][9], s_V[kMaxViews][9];
    __shared__ double s_t[kMaxViews][3];
    const int v = threadIdx.x / kPoseLanes, j = threadIdx.x % kPoseLanes;
    const bool active = v < n_views;
    if (threadIdx.x == 0) {
        double c1 = bc1, c2 = bc2;
        if (bc1 < 0.0) {  // device step count: this step is the stored count + 1
            const double step = adam[12 * n_views] + 1.0;
            // beta^step as exp(step ln beta), ln beta from the host (one exp instead of a pow)
            c1 = 1.0 - exp(step * lb1);
            c2 = 1.0 - exp(step * lb2);
            adam[12 * n_views] = step;
        }
        s_bc[0] = c1;
        s_bc[1] = c2;
    }
    __syncthreads();
    if (active && j < 6) {
        const double lr[6] = {lr0, lr1, lr2, lr3, lr4, lr5};
        double *m = adam + 12 * v, *vv = m + 6;
        const double g = grad[6 * v + j];
        m[j] = b1 * m[j] + (1 - b1) * g;
        vv[j] = b2 * vv[j] + (1 - b2) * g * g;
        const double mh = m[j] / s_bc[0], vh = vv[j] / s_bc[1];
        s_dl[v][j] = -lr[j] * mh / (sqrt(vh) + eps);
    }
    __syncthreads();
    // SE(3) exponential of (rho, phi) = dl
    if (active && j == 0) {
        const double *ph = s_dl[v] + 3;
        const double th = sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
        double a, b, c;
        if (th < 0.05) {
            // a = sin(th)/th, b = (1 - cos th)/th^2, c = (th - sin th)/th^3 by their Taylor series in
            // t = th^2 up to t^4: the next terms are below 1e-20 here, and the series avoids the
            // cancellation of 1 - cos th (the rotation increments of a tracking step are ~1e-3)
            const double t = th * th;
            a = 1.0 + t * (-1.0 / 6 + t * (1.0 / 120 + t * (-1.0 / 5040 + t * (1.0 / 362880))));
            b = 0.5 + t * (-1.0 / 24 + t * (1.0 / 720 + t * (-1.0 / 40320 + t * (1.0 / 3628800))));
            c = 1.0 / 6 + t * (-1.0 / 120 + t * (1.0 / 5040 + t * (-1.0 / 362880 + t * (1.0 / 39916800))));
        } else {
            const double sn = sin(th), cs = cos(th);
            a = sn / th;
            b = (1 - cs) / (th * th);
            c = (th - sn) / (th * th * th);
        }
        s_abc[v][0] = a;
        s_abc[v][1] = b;
        s_abc[v][2] = c;
    }
    __syncthreads();
    if (active && j < 9) {
        const double *ph = s_dl[v] + 3;
        const double K[9] = {0, -ph[2], ph[1], ph[2], 0, -ph[0], -ph[1], ph[0], 0};
        const int i = j / 3, jj = j % 3;
        const double K2 = K[3 * i] * K[jj] + K[3 * i + 1] * K[3 + jj] + K[3 * i + 2] * K[6 + jj];
        const double id = (j % 4 == 0) ? 1.0 : 0.0;
        s_R[v][j] = id + s_abc[v][0] * K[j] + s_abc[v][1] * K2;
        s_V[v][j] = id + s_abc[v][1] * K[j] + s_abc[v][2] * K2;
    }
    __syncthreads();
    if (active && j < 3) {
        const double *V = s_V[v], *dl = s_dl[v];
        s_t[v][j] = V[3 * j] * dl[0] + V[3 * j + 1] * dl[1] + V[3 * j + 2] * dl[2];
    }
    __syncthreads();
    double out = 0.0;
    double *T = Tst + 16 * v;
    if (active) {
        const int i = j / 4, c = j % 4;
        const double E[4] = {i < 3 ? s_R[v][3 * i] : 0.0, i < 3 ? s_R[v][3 * i + 1] : 0.0,
                             i < 3 ? s_R[v][3 * i + 2] : 0.0, i < 3 ? s_t[v][i] : 1.0};
        for (int k = 0; k < 4; ++k) out += E[k] * T[4 * k + c];
    }
    __syncthreads();  // every thread has read T before any writes it
    if (active) {
        T[j] = out;
        if (pose_f32) pose_f32[16 * v + j] = (float)out;
    }
}

// Blocks per view: at most one resident wave of the loss kernel over all views (resident
// = blocks per SM x SMs of the current device; 0 = unknown), and at most kLossBlocks in all.
int loss_blocks_x(const ViewTable &vt, int resident = 0) {
    int64_t maxPv = 0;
    for (int v = 0; v < vt.n_views; ++v) maxPv = std::max<int64_t>(maxPv, (int64_t)vt.W[v] * vt.H[v]);
    const int total = resident > 0 ? std::min(resident, kLossBlocks) : kLossBlocks;
    const int per_view = std::max(1, total / vt.n_views);
    return (int)std::max<int64_t>(1, std::min<int64_t>((maxPv + 255) / 256, per_view));
}

template <typename K>
int resident_blocks(K kernel, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) return 0;
    return per_sm * sms;
}

template <int D>
gs_status launch_loss(const ViewTable &vt, const LossP &lp, const gs_images *img, const gs_targets *tgt,
                      const float *W, const float *b, int64_t P, const uint32_t *mh, gs_image_grads_out *g,
                      float *part_f, double *part_d, float *dW, float *db, double *loss_out, float *mask_out,
                      float *median_out, cudaStream_t st) {
    const int bx = loss_blocks_x(vt, lp.K <= 8 ? resident_blocks(loss_kernel<D, 8>, LossShape<D, 8>::NT)
                                              : resident_blocks(loss_kernel<D, kMaxK>, LossShape<D, kMaxK>::NT));
    dim3 grid(bx, vt.n_views);
    const gs_status ls =
        lp.K <= 8 ? launch_pdl(loss_kernel<D, 8>, grid, LossShape<D, 8>::NT, 0, st, vt, lp, img->rgb, img->depth,
                               img->sil, img->feat, tgt->rgb, tgt->depth, tgt->label, W, b, P, mh, g->rgb, g->depth,
                               g->sil, g->feat, g->feat_coef, part_f, part_d, mask_out, median_out)
                  : launch_pdl(loss_kernel<D, kMaxK>, grid, LossShape<D, kMaxK>::NT, 0, st, vt, lp, img->rgb,
                               img->depth, img->sil, img->feat, tgt->rgb, tgt->depth, tgt->label, W, b, P, mh,
                               g->rgb, g->depth, g->sil, g->feat, g->feat_coef, part_f, part_d, mask_out,
                               median_out);
    if (ls) return ls;
    int rows = bx * vt.n_views;
    if (lp.ssim_coef != 0.f) {
        // the SSIM tiles add their colour-term shares as further partial rows
        const gs_status s = launch_ssim(vt, lp.ssim_coef, img->rgb, tgt->rgb, lp.ssim_maps, part_d + 3 * (size_t)rows,
                                        g->rgb, st);
        if (s) return s;
        rows += ssim_blocks(vt);
    }
    return launch_pdl(loss_finish_kernel, lp.K * D + lp.K + 4, 256, 0, st, bx * vt.n_views, rows, lp.K, D, part_f,
                      part_d, dW, db, loss_out);
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_loss_fwd_bwd(const gs_camera *cams, int n_views, int feat_dim, const gs_images *img,
                                     const gs_targets *tgt, const float *dec_W, const float *dec_b,
                                     const gs_loss_params *lp, void *ws, size_t ws_bytes, gs_image_grads_out *grad,
                                     float *d_dec_W, float *d_dec_b, double *loss_out, float *mask_out,
                                     float *median_out, gs_stream stream) {
    GS_NVTX_RANGE("gs_loss_fwd_bwd");
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    ViewTable vt;
    if (!img || !tgt || !lp || !grad || !loss_out || !make_view_table(cams, n_views, 0, &vt)) return GS_ERR_ARG;
    if (!feat_dim_ok(feat_dim)) return GS_ERR_UNSUPPORTED;
    if (lp->n_classes < 0 || lp->n_classes > kMaxK || (lp->mask_mode != 0 && lp->mask_mode != 1)) return GS_ERR_ARG;
    if (!img->rgb || !img->depth || !img->sil || (feat_dim && !img->feat) || !tgt->rgb || !tgt->depth ||
        !tgt->label || !grad->rgb || !grad->depth || !grad->sil || (feat_dim && !grad->feat && !grad->feat_coef))
        return GS_ERR_ARG;
    if (lp->n_classes > 0 && (!dec_W || !dec_b || !d_dec_W || !d_dec_b)) return GS_ERR_ARG;
    if (!(lp->ssim >= 0.f && lp->ssim <= 1.f) || (lp->ssim > 0.f && lp->mask_mode != 0)) return GS_ERR_ARG;
    WsLayout L = ws_layout(0, n_views, 0, &vt);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < L.misc_end) return GS_ERR_ARG;
    char *w = static_cast<char *>(ws);
    uint32_t *mh = reinterpret_cast<uint32_t *>(w + L.med_hist);
    float *part_f = reinterpret_cast<float *>(w + L.loss_part_f);
    double *part_d = reinterpret_cast<double *>(w + L.loss_part_d);
    const int64_t P = vt.pix_off[n_views];
    gs_status s;
    if (lp->mask_mode == 1) {
        if ((s = cuda_status(cudaMemsetAsync(mh, 0, sizeof(uint32_t) * 4 * 256 * n_views, st)))) return s;
        dim3 grid(loss_blocks_x(vt), n_views);
        for (int pass = 0; pass < 4; ++pass)
            median_hist_kernel<<<grid, 256, 0, st>>>(vt, pass, img->depth, tgt->depth, mh);
        if ((s = last_launch())) return s;
    }
    // Eq. 15: the L1 part weighted lambda_c (1 - lambda), the SSIM part lambda_c lambda
    LossP q{lp->color * (1.f - lp->ssim), lp->depth, lp->sem, lp->tau_obs, lp->mask_mode, lp->n_classes,
            lp->color * lp->ssim, reinterpret_cast<float *>(w + L.ssim_maps)};
#define GS_LOSS(DD)                                                                                              \
    case DD:                                                                                                     \
        return launch_loss<DD>(vt, q, img, tgt, dec_W, dec_b, P, mh, grad, part_f, part_d, d_dec_W, d_dec_b,     \
                               loss_out, mask_out, median_out, st);
    switch (feat_dim) {
        GS_LOSS(0) GS_LOSS(4) GS_LOSS(8) GS_LOSS(16) GS_LOSS(32)
        default: return GS_ERR_UNSUPPORTED;
    }
#undef GS_LOSS
}

namespace gs {
namespace {
static_assert(6 * kRedBlocks * sizeof(double) + 2 * sizeof(uint32_t) <= GS_DSR_SCRATCH_BYTES,
              "the DSR partials and their arrival counters fit the scratch");

// The value of Eq. 12 into out, with its partials (and two arrival counters after them) in part.
gs_status dsr_value(int64_t n, const float *log_scales, float lam_big, float lam_small, double *part, double *out,
                    cudaStream_t st) {
    if (n == 0) return cuda_status(cudaMemsetAsync(out, 0, 8 * sizeof(double), st));
    const int64_t m = 3 * n;
    const int grid = std::min(ceil_div(m, 256), kRedBlocks);
    // the arrival counters are zeroed here; each finishing block resets its own
    uint32_t *ctr = reinterpret_cast<uint32_t *>(part + 6 * kRedBlocks);
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(ctr, 0, 2 * sizeof(uint32_t), st)))) return s;
    if ((s = launch_pdl(dsr_stats_kernel, grid, 256, 0, st, m, log_scales, part, out, ctr))) return s;
    return launch_pdl(dsr_mask_kernel, grid, 256, 0, st, m, log_scales, out, part + 2 * kRedBlocks, lam_big, lam_small,
                      ctr + 1);
}

gs_status dsr_grad(int64_t n, const float *log_scales, float lam_big, float lam_small, const double *out,
                   float *d_log_scales, cudaStream_t st) {
    if (n == 0) return GS_OK;
    const int64_t m = 3 * n;
    return launch_pdl(dsr_grad_kernel, std::min(ceil_div(m, 256), kRedBlocks), 256, 0, st, m, log_scales, lam_big,
                      lam_small, out, d_log_scales);
}
}  // namespace
}  // namespace gs

extern "C" gs_status gs_dsr(int64_t n, const float *log_scales, float lam_big, float lam_small, void *ws,
                            size_t ws_bytes, float *d_log_scales, double *out, gs_stream stream) {
    GS_NVTX_RANGE("gs_dsr");
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 0 || !out || !ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return GS_ERR_ARG;
    WsLayout L = ws_layout(0, 1, 0);
    if (ws_bytes < L.misc_end) return GS_ERR_ARG;
    if (n > 0 && (!log_scales || !d_log_scales)) return GS_ERR_ARG;
    double *part = reinterpret_cast<double *>(static_cast<char *>(ws) + L.dsr_part);
    gs_status s;
    if ((s = dsr_value(n, log_scales, lam_big, lam_small, part, out, st))) return s;
    return dsr_grad(n, log_scales, lam_big, lam_small, out, d_log_scales, st);
}

extern "C" gs_status gs_dsr_value(int64_t n, const float *log_scales, float lam_big, float lam_small, void *scratch,
                                  double *out, gs_stream stream) {
    GS_NVTX_RANGE("gs_dsr_value");
    using namespace gs;
    if (n < 0 || !out || !scratch || (reinterpret_cast<uintptr_t>(scratch) & 255) || (n > 0 && !log_scales))
        return GS_ERR_ARG;
    return dsr_value(n, log_scales, lam_big, lam_small, static_cast<double *>(scratch), out, (cudaStream_t)stream);
}

extern "C" gs_status gs_dsr_grad(int64_t n, const float *log_scales, float lam_big, float lam_small, const double *out,
                                 float *d_log_scales, gs_stream stream) {
    GS_NVTX_RANGE("gs_dsr_grad");
    using namespace gs;
    if (n < 0 || !out || (n > 0 && (!log_scales || !d_log_scales))) return GS_ERR_ARG;
    return dsr_grad(n, log_scales, lam_big, lam_small, out, d_log_scales, (cudaStream_t)stream);
}

extern "C" gs_status gs_pose_grad(int64_t n, int n_views, const float *pose_part, double *d_twist, gs_stream stream) {
    GS_NVTX_RANGE("gs_pose_grad");
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 0 || n_views < 1 || n_views > kMaxViews || !d_twist) return GS_ERR_ARG;
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(d_twist, 0, sizeof(double) * 6 * n_views, st)))) return s;
    if (n == 0) return GS_OK;
    if (!pose_part) return GS_ERR_ARG;
    dim3 grid(std::min(ceil_div(n, 256 * 8), kPoseBlocks), 6 * n_views);
    return launch_pdl(pose_reduce_kernel, grid, 256, 0, st, n, pose_part, d_twist);
}

extern "C" gs_status gs_pose_step(int n_views, const double *d_twist, double *T_state, double *adam, int step,
                                  const double *lr, double beta1, double beta2, double eps, float *pose_f32,
                                  gs_stream stream) {
    GS_NVTX_RANGE("gs_pose_step");
    using namespace gs;
    if (n_views < 1 || n_views > kMaxViews || !d_twist || !T_state || !adam || !lr || step < 0) return GS_ERR_ARG;
    // Adam bias corrections 1 - beta^step: on the host for a given step, on the
    // device (from the counter after the moments) for step 0
    const double bc1 = step ? 1.0 - pow(beta1, step) : -1.0, bc2 = step ? 1.0 - pow(beta2, step) : -1.0;
    return launch_pdl(pose_step_kernel, 1, kPoseLanes * n_views, 0, (cudaStream_t)stream, n_views, d_twist, T_state,
                      adam, bc1, bc2, lr[0], lr[1], lr[2], lr[3], lr[4], lr[5], beta1, beta2, log(beta1),
                      log(beta2), eps, pose_f32);
}

// ------------------------------------------------- allocation-free loss entry
// Same computation as gs_loss_fwd_bwd for callers that cannot allocate device
// memory: the scratch (median histograms of up to kNoAllocMaxViews views and the
// per-block partials) lives in one file-scope device array that every GPU which
// loads the library holds until the process exits.
namespace gs {
namespace {

constexpr int kNoAllocMaxViews = 16;
constexpr size_t kNoAllocHistBytes = sizeof(uint32_t) * 4 * 256 * kNoAllocMaxViews;          //    65,536
constexpr size_t kNoAllocPartFBytes = sizeof(float) * (size_t)kLossBlocks * (kMaxK * 32 + kMaxK);  // 4,325,376
constexpr size_t kNoAllocPartDBytes = sizeof(double) * (size_t)kLossBlocks * 3;                //    24,576
constexpr size_t kNoAllocBytes = kNoAllocHistBytes + kNoAllocPartFBytes + kNoAllocPartDBytes;   // 4,415,488

static __device__ __align__(256) unsigned char g_noalloc_loss_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 256;
std::atomic<void *> g_noalloc_scratch_addr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device (host code only sees a
// host-side stand-in for the symbol).  Outside a stream capture it is looked up on every
// call (cheap once the module is loaded), so a context torn down and created again gets
// its own address; during a capture, where the lookup is not attempted, the address of the
// last call outside a capture on this device is used.
gs_status noalloc_scratch(cudaStream_t st, char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GS_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
    (void)cudaGetLastError();  // a refused query must not linger as the sticky last error
    void *p = nullptr;
    if (!capturing) {
        if (cudaGetSymbolAddress(&p, g_noalloc_loss_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
        g_noalloc_scratch_addr[dev].store(p, std::memory_order_release);
    } else {
        p = g_noalloc_scratch_addr[dev].load(std::memory_order_acquire);
        if (!p) return GS_ERR_UNSUPPORTED;  // first call on this device inside a capture
    }
    *out = static_cast<char *>(p);
    return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_loss_fwd_bwd_noalloc(const gs_camera *cams, int n_views, int feat_dim, const gs_images *img,
                                             const gs_targets *tgt, const float *dec_W, const float *dec_b,
                                             const gs_loss_params *lp, gs_image_grads_out *grad, float *d_dec_W,
                                             float *d_dec_b, double *loss_out, float *mask_out, float *median_out,
                                             gs_stream stream) {
    GS_NVTX_RANGE("gs_loss_fwd_bwd_noalloc");
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    ViewTable vt;
    if (!img || !tgt || !lp || !grad || !loss_out || !make_view_table(cams, n_views, 0, &vt)) return GS_ERR_ARG;
    if (n_views > kNoAllocMaxViews) return GS_ERR_UNSUPPORTED;
    if (!feat_dim_ok(feat_dim)) return GS_ERR_UNSUPPORTED;
    if (lp->n_classes < 0 || lp->n_classes > kMaxK || (lp->mask_mode != 0 && lp->mask_mode != 1)) return GS_ERR_ARG;
    if (!img->rgb || !img->depth || !img->sil || (feat_dim && !img->feat) || !tgt->rgb || !tgt->depth ||
        !tgt->label || !grad->rgb || !grad->depth || !grad->sil || (feat_dim && !grad->feat && !grad->feat_coef))
        return GS_ERR_ARG;
    if (lp->n_classes > 0 && (!dec_W || !dec_b || !d_dec_W || !d_dec_b)) return GS_ERR_ARG;
    if (!(lp->ssim >= 0.f && lp->ssim <= 1.f) || (lp->ssim > 0.f && lp->mask_mode != 0)) return GS_ERR_ARG;
    if (lp->ssim != 0.f) return GS_ERR_UNSUPPORTED;  // the SSIM maps need per-pixel scratch
    // every argument is checked: only now is the shared array touched
    char *w = nullptr;
    gs_status s;
    if ((s = noalloc_scratch(st, &w))) return s;
    uint32_t *mh = reinterpret_cast<uint32_t *>(w);
    float *part_f = reinterpret_cast<float *>(w + kNoAllocHistBytes);
    double *part_d = reinterpret_cast<double *>(w + kNoAllocHistBytes + kNoAllocPartFBytes);
    const int64_t P = vt.pix_off[n_views];
    if (lp->mask_mode == 1) {
        // the histograms keep the previous call's counts: clear them first
        if ((s = cuda_status(cudaMemsetAsync(mh, 0, sizeof(uint32_t) * 4 * 256 * n_views, st)))) return s;
        dim3 grid(loss_blocks_x(vt), n_views);
        for (int pass = 0; pass < 4; ++pass)
            median_hist_kernel<<<grid, 256, 0, st>>>(vt, pass, img->depth, tgt->depth, mh);
        if ((s = last_launch())) return s;
    }
    LossP q{lp->color, lp->depth, lp->sem, lp->tau_obs, lp->mask_mode, lp->n_classes};
#define GS_LOSS(DD)                                                                                              \
    case DD:                                                                                                     \
        return launch_loss<DD>(vt, q, img, tgt, dec_W, dec_b, P, mh, grad, part_f, part_d, d_dec_W, d_dec_b,     \
                               loss_out, mask_out, median_out, st);
    switch (feat_dim) {
        GS_LOSS(0) GS_LOSS(4) GS_LOSS(8) GS_LOSS(16) GS_LOSS(32)
        default: return GS_ERR_UNSUPPORTED;
    }
#undef GS_LOSS
}

// ---------------------------------------------------- adaptive Gaussian expansion
// Eq. 11: M_unobs = (o_hat < tau) or (d_hat > d_gt and |d_gt - d_hat| > 50 median) on pixels with
// d_gt > 0, the median being the view's lower median of |d - d_gt| over d_gt > 0 (the same radix
// selection as the tracking mask).  One new Gaussian per masked pixel, in pixel order per view,
// views in order: a count per 256-pixel block, an ordered scan of the counts, then an emit pass
// that ranks the block's masked pixels by warp ballots.
namespace gs {
namespace {

__device__ __forceinline__ bool unobserved(float sil, float d, float dgt, float med, float tau) {
    if (!(dgt > 0.f)) return false;
    return sil < tau || (d > dgt && depth_error(d, dgt) > 50.f * med);
}

__global__ void __launch_bounds__(256) expand_count_kernel(ViewTable vt, const float *sil, const float *depth,
                                                           const float *tdepth, const uint32_t *hist, float tau,
                                                           uint32_t *counts) {
    __shared__ uint32_t s_cnt;
    const int v = blockIdx.y;
    // every thread of the block takes part in the selection (it synchronises the block)
    const float med = __uint_as_float(block_select(hist, vt.n_views, v, 4));
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int64_t Pv = (int64_t)vt.W[v] * vt.H[v];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    bool m = false;
    if (i < Pv) {
        const int64_t pix = vt.pix_off[v] + i;
        m = unobserved(sil[pix], depth[pix], tdepth[pix], med, tau);
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&s_cnt, __popc(bal));
    __syncthreads();
    if (threadIdx.x == 0) counts[(int64_t)v * gridDim.x + blockIdx.x] = s_cnt;
}

// One block: exclusive scan of the counts in order (views, then blocks); the total to *n_new.
__global__ void __launch_bounds__(1024) expand_scan_kernel(const uint32_t *counts, int64_t n, uint32_t *offsets,
                                                           int64_t *n_new) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint64_t s_carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint32_t c = i < n ? counts[i] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t t = s_warp[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, d);
                if (lane >= d) t += y;
            }
            s_warp[lane] = t;
        }
        __syncthreads();
        const uint64_t before = s_carry + (w > 0 ? s_warp[w - 1] : 0u) + x - c;
        if (i < n) offsets[i] = (uint32_t)before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_new = (int64_t)s_carry;
}

struct ExpandOut {
    float *means, *quats, *log_scales, *logits, *rgb, *feat;
    int64_t *src_pix;
};

__global__ void __launch_bounds__(256) expand_emit_kernel(ViewTable vt, const float *sil, const float *depth,
                                                          const float *trgb, const float *tdepth,
                                                          const uint32_t *hist, float tau, const uint32_t *offsets,
                                                          int64_t room, int64_t P, int D, const float *feat_init,
                                                          ExpandOut o, int32_t *status) {
    __shared__ uint32_t s_warp[8];
    const int v = blockIdx.y, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // every thread of the block takes part in the selection (it synchronises the block)
    const float med = __uint_as_float(block_select(hist, vt.n_views, v, 4));
    const int64_t Pv = (int64_t)vt.W[v] * vt.H[v];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t pix = vt.pix_off[v] + i;
    float d = 0.f;
    bool m = false;
    if (i < Pv) {
        d = tdepth[pix];
        m = unobserved(sil[pix], depth[pix], d, med, tau);
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) s_warp[w] = __popc(bal);
    __syncthreads();
    uint32_t before = 0;
    for (int k = 0; k < w; ++k) before += s_warp[k];
    if (!m) return;
    const int64_t rank = (int64_t)offsets[(int64_t)v * gridDim.x + blockIdx.x] + before +
                         __popc(bal & ((1u << lane) - 1u));
    if (rank >= room) {
        set_status(status, GS_ERR_CAPACITY);
        return;
    }
    const int x = (int)(i % vt.W[v]), y = (int)(i / vt.W[v]);
    // the pixel centre unprojected at d_gt: camera point, then world = R^T (p_c - t)
    const float pc[3] = {((float)x + 0.5f - vt.cx[v]) / vt.fx[v] * d, ((float)y + 0.5f - vt.cy[v]) / vt.fy[v] * d, d};
    const float *T = vt.T[v];
    const float q[3] = {pc[0] - T[3], pc[1] - T[7], pc[2] - T[11]};
#pragma unroll
    for (int j = 0; j < 3; ++j) o.means[3 * rank + j] = T[j] * q[0] + T[4 + j] * q[1] + T[8 + j] * q[2];
    o.quats[4 * rank] = 1.f;
    o.quats[4 * rank + 1] = o.quats[4 * rank + 2] = o.quats[4 * rank + 3] = 0.f;
    const float ls = logf(d / vt.fx[v]);
#pragma unroll
    for (int j = 0; j < 3; ++j) o.log_scales[3 * rank + j] = ls;
    o.logits[rank] = 0.f;                       // opacity 0.5
#pragma unroll
    for (int c = 0; c < 3; ++c) o.rgb[3 * rank + c] = trgb[c * P + pix];
    for (int k = 0; k < D; ++k) o.feat[rank * D + k] = feat_init[rank * D + k];
    if (o.src_pix) o.src_pix[rank] = pix;
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_expand(const gs_camera *cams, int n_views, const gs_images *img, const gs_targets *tgt,
                               float tau_unobs, const float *feat_init, int64_t n_existing, gs_field_mut *field,
                               int64_t *n_new, int64_t *src_pix, int32_t *status, void *ws, size_t ws_bytes,
                               gs_stream stream) {
    GS_NVTX_RANGE("gs_expand");
    using namespace gs;
    ViewTable vt;
    if (!img || !tgt || !field || !n_new || !status || !make_view_table(cams, n_views, 0, &vt)) return GS_ERR_ARG;
    if (!feat_dim_ok(field->feat_dim)) return GS_ERR_UNSUPPORTED;
    const int64_t capacity = field->n;  // rows of the field's arrays
    if (n_existing < 0 || capacity < n_existing || !img->sil || !img->depth || !tgt->rgb || !tgt->depth ||
        !field->means || !field->quats || !field->log_scales || !field->opacity_logits || !field->rgb ||
        (field->feat_dim && (!field->feat || !feat_init)) || !(tau_unobs >= 0.f))
        return GS_ERR_ARG;
    WsLayout L = ws_layout(0, n_views, 0, &vt);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < L.misc_end) return GS_ERR_ARG;
    char *w = static_cast<char *>(ws);
    uint32_t *mh = reinterpret_cast<uint32_t *>(w + L.med_hist);
    const int bx = expand_blocks_x(vt);
    uint32_t *counts = reinterpret_cast<uint32_t *>(w + L.expand_counts);
    uint32_t *offsets = counts + (size_t)n_views * bx;
    cudaStream_t st = (cudaStream_t)stream;
    gs_status s;
    if ((s = cuda_status(cudaMemsetAsync(status, 0, sizeof(int32_t), st)))) return s;
    if ((s = cuda_status(cudaMemsetAsync(mh, 0, sizeof(uint32_t) * 4 * 256 * n_views, st)))) return s;
    const dim3 hgrid(loss_blocks_x(vt), n_views);
    for (int pass = 0; pass < 4; ++pass)
        median_hist_kernel<<<hgrid, 256, 0, st>>>(vt, pass, img->depth, tgt->depth, mh);
    const dim3 grid(bx, n_views);
    expand_count_kernel<<<grid, 256, 0, st>>>(vt, img->sil, img->depth, tgt->depth, mh, tau_unobs, counts);
    expand_scan_kernel<<<1, 1024, 0, st>>>(counts, (int64_t)n_views * bx, offsets, n_new);
    const int64_t D = field->feat_dim;
    ExpandOut o{field->means + 3 * n_existing, field->quats + 4 * n_existing, field->log_scales + 3 * n_existing,
                field->opacity_logits + n_existing, field->rgb + 3 * n_existing,
                D ? field->feat + D * n_existing : nullptr, src_pix};
    expand_emit_kernel<<<grid, 256, 0, st>>>(vt, img->sil, img->depth, tgt->rgb, tgt->depth, mh, tau_unobs, offsets,
                                             capacity - n_existing, vt.pix_off[n_views], (int)D, feat_init, o,
                                             status);
    return last_launch();
}
