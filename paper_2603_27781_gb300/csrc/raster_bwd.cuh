// Backward of the blend (Eq. 4-7, 10): kernel template shared by the map-mode
// and pose-mode translation units.
//
// Same grid as the forward: one CTA per 16x16 tile, NP pixels per thread.  A
// pixel walks the splats it blended back to front, starting from its stored
// final transmittance and last-contributor position; the transmittance in
// front of each splat is recovered as T / (1 - alpha).  With S the blended
// value behind a splat, d out / d alpha = T (x - S) per channel; the loss needs
// only sum_ch g_ch (x_ch - S_ch) = g.x - g.S, and g.S obeys the same recurrence
// as S, so one scalar per pixel replaces the per-channel S.
//
// Per splat a thread first sums its pixels' contributions, the warp sums its
// lanes with a transpose reduction (each shuffle step halves the values a lane
// carries, so N values take N - 1 shuffles and lane l ends with the sum of
// value l), the warps combine through shared-memory atomics, and each
// (tile, splat) issues one 16-byte vector atomic per 4 values to the
// per-Gaussian accumulators.  A warp skips splats whose alpha >= alpha_min
// region misses its pixel box, exactly as the forward did.
#pragma once

#include "raster.cuh"

namespace gs {

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

constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

// Per splat, lanes 0-4 of a warp hold the reduced moments S = sum over its pixels of
// (dx, dy, dx^2, dx dy, dy^2) x dpow, dpow = o G dL/dalpha.  The centre gradient is
// -(1/log2 e) (2 qa S_x + qb S_y, qb S_x + 2 qc S_y) and the conic's is -(S_xx/2, S_xy,
// S_yy/2) with (qa, qb, qc) the splat's log2-scaled conic; lane i returns gradient value i
// (lanes >= 5 return r unchanged).  All lanes must call it (a shuffle pairs lanes 0 and 1).
// Branch-free: a lane-dependent branch here would serialise five paths per splat.
__device__ __forceinline__ float geo_grads(float r, int i, const SplatGeo &s) {
    const float o = __shfl_xor_sync(0xffffffffu, r, 1);
    const float a = i == 0 ? 2.f * s.qa : 2.f * s.qc;
    const float centre = (-1.f / kLog2e) * fmaf(a, r, s.qb * o);
    const float scale = (i == 2 || i == 4) ? -0.5f : (i == 3 ? -1.f : 1.f);
    return i < 2 ? centre : scale * r;
}

// Per splat the kernel accumulates: centre (2), conic (3), opacity, then the
// alpha-T weighted terms depth, r, g, b and the D features.
//
// With D >= 16 in map mode the weighted terms are not reduced by shuffles: a
// warp records the weight w of each of its pixels for up to SLOTS splats and
// then contracts them with its pixels' upstream gradients in one pass, a lane
// owning one splat and half of the terms (sum over the warp's pixels of
// w * g, exact FP32 FMAs).  The shuffle reduction then carries 6 values, not 26.
template <int D, int NP, bool MAP>
struct BwdLayout {
    static constexpr int NV = MAP ? 10 + D : 6;                  // values accumulated per splat
    static constexpr bool DEFER = MAP && D >= 16;
    static constexpr int NW = 4 + D;                             // deferred weighted terms
    static constexpr int HW = NW / 2;                            // terms per half-warp
    static constexpr int HWP = (HW + 3) / 4 * 4;                 // padded to 16-byte loads
    static constexpr int GROW = 2 * HWP;                         // gradient row of one pixel
    static constexpr int NR = DEFER ? 6 : NV;                    // values reduced by shuffles
    static constexpr int C0 = NR > 32 ? 32 : pow2_at_least(NR);  // first chunk (power of two)
    static constexpr int R1 = NR > 32 ? NR - 32 : 0;             // values in the second chunk
    static constexpr int C1 = R1 > 0 ? pow2_at_least(R1) : 0;
    static constexpr int ROW = DEFER ? NV : C0 + C1;             // shared accumulator row
    static constexpr int BATCH = kBatch;                         // splats staged per round
    static constexpr int SLOTS = 16;                             // splats per deferred pass
    static constexpr int WARPS = Shape<NP>::WARPS;
    static constexpr int PXW = 32 * NP;                          // pixels of one warp
    static constexpr int WROW = PXW + 4;                         // 16-byte rows; 8 lanes' float4 reads span 32 banks
    static constexpr int D4 = D / 4 > 0 ? D / 4 : 1;
    // dynamic shared memory, in bytes
    static constexpr size_t OFF_EXT = sizeof(SplatGeo) * BATCH;
    static constexpr size_t OFF_RGBD = OFF_EXT + sizeof(float2) * BATCH;
    static constexpr size_t OFF_FEAT = OFF_RGBD + sizeof(float4) * BATCH;
    static constexpr size_t OFF_ACC = OFF_FEAT + sizeof(float4) * BATCH * D4;
    static constexpr size_t OFF_W = OFF_ACC + align16(sizeof(float) * BATCH * ROW);
    static constexpr size_t OFF_G = OFF_W + (DEFER ? align16(sizeof(float) * WARPS * SLOTS * WROW) : 0);
    static constexpr size_t OFF_SLOT = OFF_G + (DEFER ? align16(sizeof(float) * WARPS * PXW * GROW) : 0);
    static constexpr size_t BYTES = OFF_SLOT + (DEFER ? sizeof(int) * WARPS * SLOTS : 0);
    static_assert(PXW % 4 == 0, "weights are read four pixels at a time");
};

struct BwdArgs {
    const float4 *uvdo;
    const float2 *uv_lo;
    const float4 *conic;
    const void *rgb;
    const void *feat;
    const uint32_t *vals;
    const uint32_t *ranges;
    int64_t P;
    const float *T_final;
    const int32_t *n_contrib;
    const float *g_rgb, *g_depth, *g_sil, *g_feat;
    // factored feature gradient g_feat = feat_basis^T feat_coef (NULL basis: g_feat as given)
    const float *feat_coef;   // [feat_rank, P]
    const float *feat_basis;  // [feat_rank, D]
    int feat_rank;
    float4 *acc_uvod, *acc_conic, *acc_rgb;
    float *d_feat;
    const uint32_t *bmask;  // blend-mask planes from the forward (NULL: scan every splat)
    int64_t bm_stride;
    const uint32_t *order;  // tile launch order (NULL: tile = block index)
    int32_t *status;        // the binning's status word: set means render nothing
    int64_t capacity;       // the binning's instance capacity
};

template <int D, int NP, bool MAP, typename RT, typename FT>
__global__ void __launch_bounds__(Shape<NP>::THREADS) raster_bwd_kernel(ViewTable vt, Params prm, BwdArgs A) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    using LY = BwdLayout<D, NP, MAP>;
    using SH = Shape<NP>;
    constexpr int NT = SH::THREADS;
    constexpr int D4 = D / 4;
    constexpr int NCH = 5 + D;  // r, g, b, depth, sil, features
    extern __shared__ __align__(16) unsigned char smem[];
    SplatGeo *s_geo = reinterpret_cast<SplatGeo *>(smem);
    float2 *s_ext = reinterpret_cast<float2 *>(smem + LY::OFF_EXT);
    float4 *s_rgbd = reinterpret_cast<float4 *>(smem + LY::OFF_RGBD);
    float4 *s_feat = reinterpret_cast<float4 *>(smem + LY::OFF_FEAT);
    float *s_acc = reinterpret_cast<float *>(smem + LY::OFF_ACC);
    float *s_w = reinterpret_cast<float *>(smem + LY::OFF_W);        // [warp][slot][pixel] weights
    float *s_g = reinterpret_cast<float *>(smem + LY::OFF_G);        // [warp][pixel][term] gradients
    int *s_slot = reinterpret_cast<int *>(smem + LY::OFF_SLOT);      // [warp][slot] batch index
    __shared__ int s_max_last;
    const RT *rgb = static_cast<const RT *>(A.rgb);
    const FT *feat = static_cast<const FT *>(A.feat);

    if (binning_failed(A.status)) return;  // the binning overflowed or gave up
    const int gt = A.order ? (int)A.order[blockIdx.x] : (int)blockIdx.x;
    if (gt < 0 || gt >= vt.tile_off[vt.n_views]) return;  // not a permutation of the tiles: leave the tile
    const int v = view_of_tile(vt, gt);
    const int t = gt - vt.tile_off[v];
    const int tx = t % vt.TX[v], ty = t / vt.TX[v];
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t start = A.ranges[2 * gt];
    const int64_t voff = (int64_t)v * vt.n;
    const int64_t P = A.P;
    int bx0, by0;
    SH::warp_origin(tid >> 5, bx0, by0);
    const float bcx = (float)(tx * kTile + bx0) + 0.5f * SH::BW, bcy = (float)(ty * kTile + by0) + 0.5f * SH::BH;
    const float hx = 0.5f * (SH::BW - 1), hy = 0.5f * (SH::BH - 1);

    // per-pixel state: upstream gradient g, transmittance, g.S behind the current splat
    float gch[NP][NCH], T[NP], gS[NP], pxc[NP], pyc[NP];
    int last[NP];
    int my_max = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        int lx, ly;
        SH::pixel(tid, p, lx, ly);
        const int px = tx * kTile + lx, py = ty * kTile + ly;
        pxc[p] = (float)px + 0.5f;
        pyc[p] = (float)py + 0.5f;
        T[p] = 1.f;
        last[p] = 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) gch[p][c] = 0.f;
        if (px < vt.W[v] && py < vt.H[v]) {
            const int64_t pix = vt.pix_off[v] + (int64_t)py * vt.W[v] + px;
            T[p] = A.T_final[pix];
            last[p] = A.n_contrib[pix];
            gch[p][0] = A.g_rgb[pix];
            gch[p][1] = A.g_rgb[P + pix];
            gch[p][2] = A.g_rgb[2 * P + pix];
            gch[p][3] = A.g_depth[pix];
            gch[p][4] = A.g_sil ? A.g_sil[pix] : 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) gch[p][5 + d] = A.g_feat[d * P + pix];
        }
        gS[p] = gch[p][0] * prm.bg[0] + gch[p][1] * prm.bg[1] + gch[p][2] * prm.bg[2];
        my_max = max(my_max, last[p]);
    }
    const int warp = tid >> 5;
    if constexpr (LY::DEFER) {
        // the warp's pixel p * 32 + lane: gradients of depth, r, g, b, features
        // (terms [0, HW) at row[0..], terms [HW, NW) at row[HWP..]; padding is zero)
        float *gw = s_g + (size_t)warp * LY::PXW * LY::GROW;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float term[LY::NW];
            term[0] = gch[p][3];
            term[1] = gch[p][0];
            term[2] = gch[p][1];
            term[3] = gch[p][2];
#pragma unroll
            for (int d = 0; d < D; ++d) term[4 + d] = gch[p][5 + d];
            float *row = gw + (p * 32 + lane) * LY::GROW;
#pragma unroll
            for (int c = 0; c < LY::GROW; ++c) {
                const int h = c / LY::HWP, i = c % LY::HWP;
                row[c] = i < LY::HW ? term[h * LY::HW + i] : 0.f;
            }
        }
    }
    int n_slot = 0;  // splats recorded in the warp's weight slots (warp-uniform)
    // Deferred weighted terms: lane (j, h) sums w * g over the warp's pixels for
    // slot j and terms [h * HW, (h + 1) * HW), then adds them to the splat's row.
    auto flush = [&]() {
        __syncwarp();
        const int j = lane & (LY::SLOTS - 1), h = lane >> 4;
        const float4 *wr = reinterpret_cast<const float4 *>(s_w + ((size_t)warp * LY::SLOTS + j) * LY::WROW);
        const float4 *gr =
            reinterpret_cast<const float4 *>(s_g + (size_t)warp * LY::PXW * LY::GROW + h * LY::HWP);
        float acc[LY::HWP];
#pragma unroll
        for (int c = 0; c < LY::HWP; ++c) acc[c] = 0.f;
#pragma unroll 2
        for (int q = 0; q < LY::PXW / 4; ++q) {
            const float4 w4 = wr[q];
            const float wq[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 *g4 = gr + (4 * q + i) * (LY::GROW / 4);
#pragma unroll
                for (int c = 0; c < LY::HWP / 4; ++c) {
                    const float4 gv = g4[c];
                    acc[4 * c] = fmaf(wq[i], gv.x, acc[4 * c]);
                    if (4 * c + 1 < LY::HW) acc[4 * c + 1] = fmaf(wq[i], gv.y, acc[4 * c + 1]);
                    if (4 * c + 2 < LY::HW) acc[4 * c + 2] = fmaf(wq[i], gv.z, acc[4 * c + 2]);
                    if (4 * c + 3 < LY::HW) acc[4 * c + 3] = fmaf(wq[i], gv.w, acc[4 * c + 3]);
                }
            }
        }
        if (j < n_slot) {
            float *a = s_acc + s_slot[warp * LY::SLOTS + j] * LY::ROW + 6 + h * LY::HW;
#pragma unroll
            for (int c = 0; c < LY::HW; ++c)
                if (acc[c] != 0.f) atomicAdd(a + c, acc[c]);
        }
        __syncwarp();
        n_slot = 0;
    };

    if (tid == 0) s_max_last = 0;
    __syncthreads();
    if (my_max > 0) atomicMax(&s_max_last, my_max);
    __syncthreads();
    const int max_last = checked_last(start, A.ranges, gt, s_max_last, A.capacity, A.status);

    for (int b_end = max_last; b_end > 0; b_end -= LY::BATCH) {
        const int b_start = max(0, b_end - LY::BATCH);
        const int cnt = b_end - b_start;
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            const uint32_t item = checked_item(A.vals[start + b_start + i], voff, vt.n, A.status);
            const int64_t g = (int64_t)item - voff;
            const float4 a = A.uvdo[item];
            const float4 c = A.conic[item];
            s_geo[i] = make_geo(a, A.uv_lo[item], c);
            s_ext[i] = splat_extent(c, a.w, prm.alpha_min);
            s_rgbd[i] = load_rgbd(rgb, g, a.z);
#pragma unroll
            for (int q = 0; q < D4; ++q) s_feat[i * D4 + q] = load_feat4(feat, g * D + 4 * q);
        }
        for (int i = tid; i < cnt * LY::ROW; i += NT) s_acc[i] = 0.f;
        __syncthreads();

        auto process = [&](const int k) {
            const int pos = b_start + k;
            if (!__any_sync(0xffffffffu, pos < my_max)) return;
            const SplatGeo s = s_geo[k];
            if (!reaches_box(s.u, s.v, s_ext[k], bcx, bcy, hx, hy)) return;
            PairEval e[NP];
            bool contrib[NP], any = false;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                e[p] = eval_pair(s, pxc[p], pyc[p], prm.alpha_min, prm.alpha_max);
                contrib[p] = pos < last[p] && !e[p].skip;
                any |= contrib[p];
            }
            if (!__any_sync(0xffffffffu, any)) return;

            float val[LY::C0 + LY::C1], wv[NP];
#pragma unroll
            for (int i = 0; i < LY::C0 + LY::C1; ++i) val[i] = 0.f;
#pragma unroll
            for (int p = 0; p < NP; ++p) wv[p] = 0.f;
            {
                const float4 c = s_rgbd[k];
                float x[NCH];
                x[0] = c.x; x[1] = c.y; x[2] = c.z; x[3] = c.w; x[4] = 1.f;
#pragma unroll
                for (int q = 0; q < D4; ++q) {
                    const float4 f = s_feat[k * D4 + q];
                    x[5 + 4 * q] = f.x; x[6 + 4 * q] = f.y; x[7 + 4 * q] = f.z; x[8 + 4 * q] = f.w;
                }
                // Branch-free over the lanes: a pixel that did not blend the splat runs the same
                // instructions with alpha 0 and keeps its state, and every sum it adds to is 0.
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float a = contrib[p] ? e[p].alpha : 0.f;
                    const float Tb = __fdividef(T[p], 1.f - a);
                    const float w = a * Tb;
                    // g.x as three interleaved partial sums (shorter dependent chain)
                    float gx3[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int ch = 0; ch < NCH; ++ch) gx3[ch % 3] = fmaf(gch[p][ch], x[ch], gx3[ch % 3]);
                    const float gx = gx3[0] + gx3[1] + gx3[2];
                    const float da = Tb * (gx - gS[p]);
                    gS[p] = fmaf(a, gx - gS[p], gS[p]);
                    T[p] = contrib[p] ? Tb : T[p];
                    // moments of dpow over the pixels where alpha is not clamped; the splat's
                    // constants scale them once, after the warp reduction (geo_grads)
                    const bool free_alpha = contrib[p] && e[p].oG < prm.alpha_max;
                    const float dpow = free_alpha ? e[p].oG * da : 0.f;
                    const float dx = e[p].dx, dy = e[p].dy;
                    const float ax = dx * dpow, ay = dy * dpow;
                    val[0] += ax;
                    val[1] += ay;
                    val[2] = fmaf(ax, dx, val[2]);
                    val[3] = fmaf(ax, dy, val[3]);
                    val[4] = fmaf(ay, dy, val[4]);
                    if (MAP) val[5] += e[p].G * (free_alpha ? da : 0.f);
                    if constexpr (LY::DEFER) {
                        wv[p] = w;
                    } else if (MAP) {
                        val[6] = fmaf(w, gch[p][3], val[6]);
                        val[7] = fmaf(w, gch[p][0], val[7]);
                        val[8] = fmaf(w, gch[p][1], val[8]);
                        val[9] = fmaf(w, gch[p][2], val[9]);
#pragma unroll
                        for (int d = 0; d < D; ++d) val[10 + d] = fmaf(w, gch[p][5 + d], val[10 + d]);
                    } else {
                        val[5] = fmaf(w, gch[p][3], val[5]);
                    }
                }
            }
            if constexpr (LY::DEFER) {
                float *wr = s_w + ((size_t)warp * LY::SLOTS + n_slot) * LY::WROW;
#pragma unroll
                for (int p = 0; p < NP; ++p) wr[p * 32 + lane] = wv[p];
                if (lane == 0) s_slot[warp * LY::SLOTS + n_slot] = k;
                ++n_slot;
            }
            // warp reduction, then CTA combine in shared memory
            {
                float v0[LY::C0];
#pragma unroll
                for (int i = 0; i < LY::C0; ++i) v0[i] = val[i];
                const int idx = lane & (LY::C0 - 1);
                const float r = geo_grads(warp_transpose_reduce<LY::C0>(v0, lane), idx, s);
                if (lane < LY::C0 && idx < LY::NR && r != 0.f) atomicAdd(&s_acc[k * LY::ROW + idx], r);
            }
            if constexpr (LY::C1 > 0) {
                float v1[LY::C1];
#pragma unroll
                for (int i = 0; i < LY::C1; ++i) v1[i] = val[LY::C0 + i];
                const float r = warp_transpose_reduce<LY::C1>(v1, lane);
                const int idx = lane & (LY::C1 - 1);
                if (lane < LY::C1 && idx < LY::R1 && r != 0.f) atomicAdd(&s_acc[k * LY::ROW + LY::C0 + idx], r);
            }
            if constexpr (LY::DEFER) {
                if (n_slot == LY::SLOTS) flush();
            }
        };
        if (A.bmask) {
            // only the instances some pixel of the warp's groups blended, back to front
            const int64_t lo_i = (int64_t)start + b_start, hi_i = (int64_t)start + b_end;
            for (int64_t wi = (hi_i - 1) >> 5; wi >= (lo_i >> 5); --wi) {
                uint32_t m = 0u;
#pragma unroll
                for (int j = 0; j < NP; ++j) m |= A.bmask[(int64_t)SH::group(warp, j) * A.bm_stride + wi];
                const int64_t base = wi << 5;
                if (base < lo_i) m &= ~0u << (int)(lo_i - base);
                if (hi_i - base < 32) m &= (1u << (int)(hi_i - base)) - 1u;
                while (m) {
                    const int bit = 31 - __clz(m);
                    m &= ~(1u << bit);
                    process((int)(base + bit - lo_i));
                }
            }
        } else {
            for (int k = cnt - 1; k >= 0; --k) process(k);
        }
        if constexpr (LY::DEFER) {
            if (n_slot > 0) flush();
        }
        __syncthreads();
        // one set of vector atomics per (tile, splat)
        for (int i = tid; i < cnt; i += NT) {
            const float *a = s_acc + i * LY::ROW;
            bool nz = false;
#pragma unroll
            for (int j = 0; j < LY::NV; ++j) nz |= a[j] != 0.f;
            if (!nz) continue;
            const uint32_t item = checked_item(A.vals[start + b_start + i], voff, vt.n, A.status);
            const int64_t g = (int64_t)item - voff;
            if (MAP) {
                atomicAdd(&A.acc_uvod[item], make_float4(a[0], a[1], a[5], a[6]));
                atomicAdd(&A.acc_conic[item], make_float4(a[2], a[3], a[4], 0.f));
                atomicAdd(&A.acc_rgb[g], make_float4(a[7], a[8], a[9], 0.f));
#pragma unroll
                for (int q = 0; q < D4; ++q)
                    atomicAdd(reinterpret_cast<float4 *>(A.d_feat + g * D) + q,
                              make_float4(a[10 + 4 * q], a[11 + 4 * q], a[12 + 4 * q], a[13 + 4 * q]));
            } else {
                atomicAdd(&A.acc_uvod[item], make_float4(a[0], a[1], 0.f, a[5]));
                atomicAdd(&A.acc_conic[item], make_float4(a[2], a[3], a[4], 0.f));
            }
        }
    }
}

template <int D, int NP, bool MAP, typename RT, typename FT>
gs_status launch_bwd(const ViewTable &vt, const Params &prm, const BwdArgs &A, cudaStream_t st) {
    constexpr size_t bytes = BwdLayout<D, NP, MAP>::BYTES;
    auto kern = raster_bwd_kernel<D, NP, MAP, RT, FT>;
    if (bytes > 48 * 1024) {
        const gs_status s = cuda_status(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        if (s) return s;
    }
    return launch_pdl(kern, vt.tile_off[vt.n_views], Shape<NP>::THREADS, bytes, st, vt, prm, A);
}

// Dispatch over feature dim, pixels per thread and storage for one mode.
template <bool MAP>
gs_status dispatch_bwd(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                       cudaStream_t st) {
    if (half) {
        if (D == 16) {
            if (np == 1) return launch_bwd<16, 1, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
            if (np == 2) return launch_bwd<16, 2, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
            if (np == 4) return launch_bwd<16, 4, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
        } else if (D == 32) {
            if (np == 1) return launch_bwd<32, 1, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
            if (np == 2) return launch_bwd<32, 2, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
        }
        return GS_ERR_UNSUPPORTED;
    }
    switch (D) {
        case 0: if (np == 1) return launch_bwd<0, 1, MAP, float, float>(vt, prm, A, st); break;
        case 4: if (np == 1) return launch_bwd<4, 1, MAP, float, float>(vt, prm, A, st); break;
        case 8: if (np == 1) return launch_bwd<8, 1, MAP, float, float>(vt, prm, A, st); break;
        case 16:
            if (np == 1) return launch_bwd<16, 1, MAP, float, float>(vt, prm, A, st);
            if (np == 2) return launch_bwd<16, 2, MAP, float, float>(vt, prm, A, st);
            if (np == 4) return launch_bwd<16, 4, MAP, float, float>(vt, prm, A, st);
            break;
        case 32:
            if (np == 1) return launch_bwd<32, 1, MAP, float, float>(vt, prm, A, st);
            if (np == 2) return launch_bwd<32, 2, MAP, float, float>(vt, prm, A, st);
            break;
        default: break;
    }
    return GS_ERR_UNSUPPORTED;
}

// The per-group form with half storage (f16 colour, bf16 features), one translation unit per mode.
gs_status dispatch_bwd_warp_map_half(int D, int np, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                                     cudaStream_t st);
gs_status dispatch_bwd_warp_pose_half(int D, int np, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                                      cudaStream_t st);
gs_status dispatch_bwd_map(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                           cudaStream_t st);
gs_status dispatch_bwd_pose(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                            cudaStream_t st);

}  // namespace gs
