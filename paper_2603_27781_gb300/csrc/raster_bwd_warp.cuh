// Blend backward (Eq. 4-7 differentiated) with one single-warp block per pixel
// group, D 16 or 32, with the forward's blend mask: map mode (every parameter's
// sums, the weighted terms deferred) and pose-only mode (the six sums the
// projection backward needs for the twist).
//
// The tile kernel's eight warps share one staged splat batch and meet at a CTA
// barrier per batch, so a tile's warps all wait for whichever of them has the
// longest masked list, and the CTA holds its registers and shared memory until
// its slowest warp ends.  Here each pixel group (the same 8x4 groups, NP of them
// per warp) is its own 32-thread block: it builds its own list of the instances
// its pixels blended (back to front, from the mask words), stages 16 splat
// records at a time in its own shared memory, runs the same per-pixel recurrence
// and the same deferred contraction of the alpha-T weighted terms, and adds its
// sums to the per-Gaussian accumulators with L2 reductions (one warp-wide scalar
// instruction for the six geometric sums, float4/float2 ones for the deferred
// terms).  Nothing waits on another warp, and a finished group frees its
// resources at once.
#pragma once

#include "raster_bwd.cuh"

namespace gs {

// Adds terms [T0, T0 + HW) of a deferred row (depth, r, g, b, then the D
// features) to the accumulators: depth to acc_uvod[item].w, colour as one float4,
// features as float4 / float2 runs on their natural alignment.
template <int D, int HW, int T0>
__device__ __forceinline__ void add_deferred(const float (&a)[HW], int64_t item, int64_t g, float4 *acc_uvod,
                                             float4 *acc_rgb, float *d_feat) {
    if constexpr (T0 == 0) {
        if (a[0] != 0.f) atomicAdd(reinterpret_cast<float *>(acc_uvod + item) + 3, a[0]);
        if (a[1] != 0.f || a[2] != 0.f || a[3] != 0.f) atomicAdd(acc_rgb + g, make_float4(a[1], a[2], a[3], 0.f));
    }
    constexpr int fa = (T0 > 4 ? T0 : 4) - 4;  // first feature of these terms
    constexpr int fb = T0 + HW - 4;            // one past the last
    float *f = d_feat + g * D;
#pragma unroll
    for (int q = 0; q < D / 4; ++q) {
        const int lo = 4 * q > fa ? 4 * q : fa, hi = 4 * q + 4 < fb ? 4 * q + 4 : fb;
        if (lo >= hi) continue;
        const int c0 = lo + 4 - T0;  // index of feature lo in a[]
        if (hi - lo == 4) {
            const float4 v = make_float4(a[c0], a[c0 + 1], a[c0 + 2], a[c0 + 3]);
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                atomicAdd(reinterpret_cast<float4 *>(f + lo), v);
        } else if (hi - lo == 2 && (lo & 1) == 0) {
            const float2 v = make_float2(a[c0], a[c0 + 1]);
            if (v.x != 0.f || v.y != 0.f) atomicAdd(reinterpret_cast<float2 *>(f + lo), v);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < hi - lo && a[c0 + k] != 0.f) atomicAdd(f + lo + k, a[c0 + k]);
        }
    }
}

// Register cap: with one pixel per thread 24 blocks per SM (80 registers at D = 16; shared
// memory would allow 26); with two, shared memory bounds the blocks at 16, which 127
// registers still allow.
template <int D, int NP> constexpr int warp_bwd_min_blocks() { return NP == 1 ? 24 : 16; }

template <int D, int NP, bool MAP, typename RT, typename FT>
__global__ void __launch_bounds__(32, warp_bwd_min_blocks<D, NP>())
    raster_bwd_warp_kernel(ViewTable vt, Params prm, BwdArgs A) {
    using LY = BwdLayout<D, NP, MAP>;
    using SH = Shape<NP>;
    static_assert(!MAP || LY::DEFER, "the map-mode warp-block backward is the deferred form");
    constexpr int D4 = D / 4;
    constexpr int NCH = 5 + D;
    constexpr int GW = SH::WARPS;  // pixel-group blocks per tile
    constexpr int STAGE = 16;      // splat records staged at a time
    __shared__ SplatGeo s_geo[STAGE];
    __shared__ float4 s_rgbd[STAGE];
    __shared__ float4 s_feat[STAGE * D4];
    __shared__ uint32_t s_item[STAGE];
    __shared__ int s_pos[STAGE];
    __shared__ uint32_t s_list[64];
    __shared__ __align__(16) float s_w[MAP ? LY::SLOTS * LY::WROW : 4];
    __shared__ __align__(16) float s_g[MAP ? LY::PXW * LY::GROW : 4];
    __shared__ uint32_t s_slot_item[MAP ? LY::SLOTS : 1];
    const RT *rgb = static_cast<const RT *>(A.rgb);
    const FT *feat = static_cast<const FT *>(A.feat);

    if (binning_failed(A.status)) return;  // the binning overflowed or gave up
    const int rank = blockIdx.x / GW, grp = blockIdx.x % GW;
    const int gt = A.order ? (int)A.order[rank] : rank;
    if (gt < 0 || gt >= vt.tile_off[vt.n_views]) return;  // not a permutation of the tiles: leave the tile
    const int v = view_of_tile(vt, gt);
    const int t = gt - vt.tile_off[v];
    const int tx = t % vt.TX[v], ty = t / vt.TX[v];
    const int lane = threadIdx.x;
    const int tid = grp * 32 + lane;  // the thread's index in the tile kernel's numbering
    const uint32_t start = A.ranges[2 * gt];
    const int64_t voff = (int64_t)v * vt.n;
    const int64_t P = A.P;

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
    const int wmax = checked_last(start, A.ranges, gt, __reduce_max_sync(0xffffffffu, my_max), A.capacity, A.status);
    if (wmax == 0) return;  // no pixel of the group blended anything (warp-uniform)
    // the group's pixel p * 32 + lane: gradients of depth, r, g, b, features
#pragma unroll
    for (int p = 0; p < (MAP ? NP : 0); ++p) {
        float term[LY::NW];
        term[0] = gch[p][3];
        term[1] = gch[p][0];
        term[2] = gch[p][1];
        term[3] = gch[p][2];
#pragma unroll
        for (int d = 0; d < D; ++d) term[4 + d] = gch[p][5 + d];
        float *row = s_g + (p * 32 + lane) * LY::GROW;
#pragma unroll
        for (int c = 0; c < LY::GROW; ++c) {
            const int h = c / LY::HWP, i = c % LY::HWP;
            row[c] = i < LY::HW ? term[h * LY::HW + i] : 0.f;
        }
    }
    int n_slot = 0;
    // lane (j, h) contracts slot j's weights with terms [h HW, (h + 1) HW) of the
    // group's gradients and adds the sums to splat j's accumulators
    auto flush = [&]() {
        if constexpr (!MAP) return;
        __syncwarp();
        const int j = lane & (LY::SLOTS - 1), h = lane >> 4;
        const float4 *wr = reinterpret_cast<const float4 *>(s_w + j * LY::WROW);
        const float4 *gr = reinterpret_cast<const float4 *>(s_g + h * LY::HWP);
        float acc[LY::HW];
        float accp[LY::HWP];
#pragma unroll
        for (int c = 0; c < LY::HWP; ++c) accp[c] = 0.f;
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
                    accp[4 * c] = fmaf(wq[i], gv.x, accp[4 * c]);
                    if (4 * c + 1 < LY::HW) accp[4 * c + 1] = fmaf(wq[i], gv.y, accp[4 * c + 1]);
                    if (4 * c + 2 < LY::HW) accp[4 * c + 2] = fmaf(wq[i], gv.z, accp[4 * c + 2]);
                    if (4 * c + 3 < LY::HW) accp[4 * c + 3] = fmaf(wq[i], gv.w, accp[4 * c + 3]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < LY::HW; ++c) acc[c] = accp[c];
        if (j < n_slot) {
            const int64_t item = s_slot_item[j];
            const int64_t g = item - voff;
            if (h == 0)
                add_deferred<D, LY::HW, 0>(acc, item, g, A.acc_uvod, A.acc_rgb, A.d_feat);
            else
                add_deferred<D, LY::HW, LY::HW>(acc, item, g, A.acc_uvod, A.acc_rgb, A.d_feat);
        }
        __syncwarp();
        n_slot = 0;
    };

    // Every listed splat was blended by a pixel of the group, so no box culling is needed.
    auto process = [&](const int k) {
        const int pos = s_pos[k];
        const SplatGeo s = s_geo[k];
        // the mask listed this splat because a pixel of the group blended it, so some lane
        // contributes: no vote is needed before the work
        PairEval e[NP];
        bool contrib[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            e[p] = eval_pair(s, pxc[p], pyc[p], prm.alpha_min, prm.alpha_max);
            contrib[p] = pos < last[p] && !e[p].skip;
        }
        float val[8], wv[NP];
#pragma unroll
        for (int i = 0; i < 8; ++i) val[i] = 0.f;
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
                if (MAP) wv[p] = a * Tb;
                else val[5] = fmaf(a * Tb, gch[p][3], val[5]);  // pose mode: the depth term
            }
        }
        const uint32_t item = s_item[k];
        if constexpr (MAP) {
            float *wr = s_w + n_slot * LY::WROW;
#pragma unroll
            for (int p = 0; p < NP; ++p) wr[p * 32 + lane] = wv[p];
            if (lane == 0) s_slot_item[n_slot] = item;
            ++n_slot;
        }
        // lane i ends with the warp's gradient value (i mod 8): centre (0, 1), conic (2-4), and
        // opacity (map mode) or depth (pose mode) (5); lanes 0-5 add them in one warp-wide
        // reduction instruction (two 16-byte targets: acc_uvod (u, v, opacity, depth) and
        // acc_conic (A, B, C))
        const float r = geo_grads(warp_transpose_reduce<8>(val, lane), lane & 7, s);
        if (lane < 6 && r != 0.f) {
            float *dst = lane == 5 ? reinterpret_cast<float *>(A.acc_uvod + item) + (MAP ? 2 : 3)
                         : lane < 2 ? reinterpret_cast<float *>(A.acc_uvod + item) + lane
                                    : reinterpret_cast<float *>(A.acc_conic + item) + (lane - 2);
            atomicAdd(dst, r);
        }
        if constexpr (MAP) {
            if (n_slot == LY::SLOTS) flush();
        }
    };

    // stages list entries [off, off + cnt) (instance indices, back to front; cnt <= STAGE)
    // and walks them
    auto stage_and_process = [&](const int off, const int cnt) {
        if (lane < cnt) {
            const uint32_t ii = s_list[off + lane];
            const uint32_t item = checked_item(A.vals[ii], voff, vt.n, A.status);
            const int64_t g = (int64_t)item - voff;
            const float4 a = A.uvdo[item];
            const float4 c = A.conic[item];
            s_geo[lane] = make_geo(a, A.uv_lo[item], c);
            s_rgbd[lane] = load_rgbd(rgb, g, a.z);
#pragma unroll
            for (int q = 0; q < D4; ++q) s_feat[lane * D4 + q] = load_feat4(feat, g * D + 4 * q);
            s_item[lane] = item;
            s_pos[lane] = (int)(ii - start);
        }
        __syncwarp();
        for (int k = 0; k < cnt; ++k) process(k);
        __syncwarp();
    };

    // the group's blended instances, back to front: each mask word appends its set bits
    // (highest first) to the list; every 32 entries are staged and processed
    const int64_t lo_i = start, hi_i = (int64_t)start + wmax;
    int n = 0;  // entries in the list (warp-uniform, < 32 between words)
    for (int64_t wi = (hi_i - 1) >> 5; wi >= (lo_i >> 5); --wi) {
        uint32_t m = 0u;
#pragma unroll
        for (int j = 0; j < NP; ++j) m |= A.bmask[(int64_t)SH::group(grp, j) * A.bm_stride + wi];
        const int64_t base = wi << 5;
        if (base < lo_i) m &= ~0u << (int)(lo_i - base);
        if (hi_i - base < 32) m &= (1u << (int)(hi_i - base)) - 1u;
        if (m == 0u) continue;
        const int b = 31 - lane;
        const int above = lane == 0 ? 0 : __popc(m >> (32 - lane));  // set bits above bit b
        if ((m >> b) & 1u) s_list[n + above] = (uint32_t)(base + b);
        n += __popc(m);
        __syncwarp();
        if (n >= 32) {
#pragma unroll
            for (int off = 0; off < 32; off += STAGE) stage_and_process(off, STAGE);
            if (lane < n - 32) s_list[lane] = s_list[32 + lane];
            __syncwarp();
            n -= 32;
        }
    }
    for (int off = 0; off < n; off += STAGE) stage_and_process(off, min(STAGE, n - off));
    if constexpr (MAP) {
        if (n_slot > 0) flush();
    }
}

template <int D, int NP, bool MAP, typename RT, typename FT>
gs_status launch_bwd_warp(const ViewTable &vt, const Params &prm, const BwdArgs &A, cudaStream_t st) {
    const int n_tiles = vt.tile_off[vt.n_views];
    raster_bwd_warp_kernel<D, NP, MAP, RT, FT><<<n_tiles * Shape<NP>::WARPS, 32, 0, st>>>(vt, prm, A);
    return last_launch();
}

// The warp-block form: D 16 or 32, 1 or 2 pixels per thread, blend mask present.
template <bool MAP>
gs_status dispatch_bwd_warp(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                            cudaStream_t st) {
    if (!A.bmask) return GS_ERR_UNSUPPORTED;
    if (half) {
        if (D == 16 && np == 1) return launch_bwd_warp<16, 1, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
        if (D == 16 && np == 2) return launch_bwd_warp<16, 2, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
        if (D == 32 && np == 1) return launch_bwd_warp<32, 1, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
        if (D == 32 && np == 2) return launch_bwd_warp<32, 2, MAP, __half, __nv_bfloat16>(vt, prm, A, st);
        return GS_ERR_UNSUPPORTED;
    }
    if (D == 16 && np == 1) return launch_bwd_warp<16, 1, MAP, float, float>(vt, prm, A, st);
    if (D == 16 && np == 2) return launch_bwd_warp<16, 2, MAP, float, float>(vt, prm, A, st);
    if (D == 32 && np == 1) return launch_bwd_warp<32, 1, MAP, float, float>(vt, prm, A, st);
    if (D == 32 && np == 2) return launch_bwd_warp<32, 2, MAP, float, float>(vt, prm, A, st);
    return GS_ERR_UNSUPPORTED;
}

}  // namespace gs
