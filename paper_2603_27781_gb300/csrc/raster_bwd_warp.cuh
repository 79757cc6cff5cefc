// Blend backward (Eq. 4-7 differentiated) with one single-warp block per pixel
// group, D 16 or 32, with the forward's blend mask: map mode (every parameter's
// sums) and pose-only mode (the six sums the projection backward needs for the
// twist).
//
// The tile kernel's eight warps share one staged splat batch and meet at a CTA
// barrier per batch, so a tile's warps all wait for whichever of them has the
// longest masked list, and the CTA holds its registers and shared memory until
// its slowest warp ends.  Here each pixel group (an 8x4 group, or an 8x8 block of
// two with two pixels per thread) is its own 32-thread block: it builds its own
// list of the instances its pixels blended (back to front, from the mask words),
// stages a few splat records at a time in its own shared memory and runs the
// per-pixel recurrence on them.  Nothing waits on another warp, and a finished
// group frees its resources at once.
//
// Map mode defers every per-splat sum.  While it walks a stage of splats, each
// pixel only records, per splat, its weight w = alpha T (the factor of the depth,
// colour and feature gradients) and dpow = o G dL/dalpha (zero where alpha is
// clamped), the factor of every geometric gradient: with (lx, ly) the pixel centre
// relative to the block centre and (cx, cy) the splat centre, dx = lx - cx, so the
// centre and conic gradients need only the moments of dpow
//   S1, Sx, Sy, Sxx, Sxy, Syy = sum over pixels of dpow (1, lx, ly, lx^2, lx ly, ly^2),
// expanded about the splat centre afterwards (sum dpow dx = Sx - cx S1, and so on),
// and the opacity gradient is S1 / o.  After the stage, lanes (pixel column, slot
// pair) contract the slots with the block's per-pixel terms (weights against the
// gradients of depth, colour and features; dpow against the row coordinates) down
// their column in FP32 FMAs, the eight columns are combined by one transpose
// reduction per stage, and each slot's sums go out as 16-byte L2 reductions.  No
// warp reduction runs per splat.
//
// Factored feature gradients.  When the image gradient of the features comes from
// a linear decoder (Eq. 8 read as a 1x1 convolution), g_feat = W^T e with e the
// gradient of the K logits.  Then g_feat . f = e . (W f) and sum_p w_p g_feat,p =
// W^T sum_p w_p e_p, so the kernel stages z = W f (K values) per splat, evaluates
// the K-term dot product per pixel and contracts K terms, and multiplies by W^T once
// per splat: the same sums, in fewer operations when K < D.
#pragma once

#include "raster_bwd.cuh"

namespace gs {

// Feature-like gradient channels per pixel in the factored form: the K <= kFactorK logit
// gradients (zero beyond K).
constexpr int kFactorK = 8;

// Map-mode layout: SL slots (splats staged and contracted together); in the contraction lane
// (column c, slot group j) sums the NWT weighted terms and the dpow column sums of SPL slots over
// the ROWS pixels of column c, and the eight columns are then added by shuffles.  In the epilogue
// LPS = 32 / SL lanes serve each slot.
template <int D, int NP, int KF, int SL>
struct WarpMapLayout {
    static constexpr int F = KF ? KF : D;
    static constexpr int PXW = 32 * NP;         // pixels of the block, 8 wide
    static constexpr int ROWS = PXW / 8;
    static constexpr int LPS = 32 / SL;
    static constexpr int SPL = SL / 4;          // slots per lane in the contraction
    static constexpr int NWT = 4 + F;           // weighted terms: depth, r, g, b, F
    static constexpr int GROW = NWT;            // a pixel's row of weighted terms
    static constexpr int NSV = NWT + 6;         // a slot's sums: the terms and six moments
    // The contraction runs in up to four chunks of terms so that a lane's running sums fit in
    // its registers (at most 2 CAPS values): the first chunk [0, T1) carries the moments,
    // then [T1, T2), [T2, T3) and [T3, NWT).
    static constexpr int CAPS = NP == 1 ? 12 : 28;
    static constexpr int TC = CAPS / 4 * 4;
    static constexpr int T1 = NWT < (CAPS - 6) / 4 * 4 ? NWT : (CAPS - 6) / 4 * 4;
    static constexpr int T2 = NWT < T1 + TC ? NWT : T1 + TC;
    static constexpr int T3 = NWT < T2 + TC ? NWT : T2 + TC;
    static_assert(NWT <= T3 + TC, "four chunks cover the terms");
    static constexpr int WROW = PXW + 4;        // a slot's row of per-pixel values (padded against bank conflicts)
    static_assert(NWT % 4 == 0 && SL == 8 && D % (4 * LPS) == 0, "16-byte rows; lanes divide the work");
};

template <int V> struct IntC { static constexpr int value = V; };

// Slots per stage in map mode: 8 (four lanes per slot) keeps the per-slot arrays small
// enough for more resident blocks; pose mode stages 16.
constexpr int kMapSlots = 8;
constexpr int kPoseStage = 16;

// Resident blocks per SM the register allocation must allow: 24 with one pixel per thread
// (80 registers), 16 with two (128), except where 16 would spill at D = 32: the map mode with
// the features themselves (whose 19.5 KB of shared memory allows 11 blocks anyway) and the
// pose mode with the factored form.
template <int D, int NP, bool MAP, int KF> constexpr int warp_bwd_min_blocks() {
    return NP == 1 ? 24 : (D == 32 && (MAP ? KF == 0 : KF > 0)) ? (MAP ? 11 : 12) : 16;
}

template <int D, int NP, bool MAP, int KF, typename RT, typename FT>
__global__ void __launch_bounds__(32, warp_bwd_min_blocks<D, NP, MAP, KF>())
    raster_bwd_warp_kernel(ViewTable vt, Params prm, BwdArgs A) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    using SH = Shape<NP>;
    using WL = WarpMapLayout<D, NP, KF, kMapSlots>;
    constexpr int F = WL::F;
    constexpr int F4 = F / 4;
    constexpr int NCH = 5 + F;            // r, g, b, depth, sil, then F
    constexpr int GW = SH::WARPS;         // pixel-group blocks per tile
    constexpr int STAGE = MAP ? kMapSlots : kPoseStage;
    constexpr int PARTS = 32 / STAGE;     // lanes per staged splat
    static_assert(F % 4 == 0 && (KF == 0 || KF % PARTS == 0), "staged values in float4 / lane parts");
    __shared__ SplatGeo s_geo[STAGE];
    __shared__ float4 s_rgbd[STAGE];
    __shared__ __align__(16) float s_feat[STAGE * F];  // features, or z = W f in the factored form
    __shared__ uint32_t s_item[STAGE];
    __shared__ int s_pos[STAGE];
    __shared__ uint32_t s_list[64];
    __shared__ __align__(16) float s_w[MAP ? STAGE * WL::WROW : 4];   // [slot][pixel] alpha T
    __shared__ __align__(16) float s_p[MAP ? STAGE * WL::WROW : 4];   // [slot][pixel] dpow
    __shared__ __align__(16) float s_g[MAP ? WL::PXW * WL::GROW : 4]; // [pixel][term] gradients
    __shared__ float s_t[MAP ? STAGE * WL::NSV : 4];                  // [slot][sum] sums
    // W, K x D (rows >= K zero), rows padded by 4 so that the four lane parts, which read rows
    // k = part (K / 4) + kk, fall in different banks
    constexpr int BROW = D + 4;
    __shared__ __align__(16) float s_basis[KF ? KF * BROW : 4];
    // raw records of two stages (the next one is copied while the current one is processed):
    // centre / depth / opacity, conic / radius, centre low parts, colour (f32 storage), features
    constexpr bool RGB32 = sizeof(RT) == 4;
    constexpr int FB = D * (int)sizeof(FT);   // feature bytes per Gaussian
    constexpr int FCH = FB / 16;              // their 16-byte chunks
    // a staged slot's feature row, padded to an odd number of 16-byte chunks so that the eight
    // slots' rows start in different banks (the copies and the reads of one chunk index are
    // then conflict-free)
    constexpr int FBP = FCH % 2 == 0 ? FB + 16 : FB;
    constexpr int NCOPY = 3 + (RGB32 ? 3 : 0) + FCH;
    static_assert(FB % 16 == 0, "features in 16-byte chunks");
    __shared__ float4 r_a[2][STAGE], r_c[2][STAGE];
    __shared__ float2 r_lo[2][STAGE];
    __shared__ float r_rgb[2][STAGE][4];
    __shared__ __align__(16) unsigned char r_f[2][STAGE * FBP];
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
    int bx0, by0;
    SH::warp_origin(grp, bx0, by0);
    // block centre: pixel (lx, ly) of the block sits at (lx - 3.5, ly + 0.5 - ROWS / 2) from it
    const float bcx = (float)(tx * kTile + bx0) + 4.f, bcy = (float)(ty * kTile + by0) + 0.5f * WL::ROWS;

    if constexpr (KF > 0) {
        for (int i = lane; i < KF * D; i += 32)
            s_basis[(i / D) * BROW + i % D] = i < A.feat_rank * D ? A.feat_basis[i] : 0.f;
    }

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
            if constexpr (KF > 0) {
#pragma unroll
                for (int k = 0; k < KF; ++k) gch[p][5 + k] = k < A.feat_rank ? A.feat_coef[k * P + pix] : 0.f;
            } else {
#pragma unroll
                for (int d = 0; d < D; ++d) gch[p][5 + d] = A.g_feat[d * P + pix];
            }
        }
        gS[p] = gch[p][0] * prm.bg[0] + gch[p][1] * prm.bg[1] + gch[p][2] * prm.bg[2];
        my_max = max(my_max, last[p]);
    }
    const int wmax = checked_last(start, A.ranges, gt, __reduce_max_sync(0xffffffffu, my_max), A.capacity, A.status);
    if (wmax == 0) return;  // no pixel of the group blended anything (warp-uniform)
    if constexpr (MAP) {
        // pixel q = p * 32 + lane of the block: its weighted terms (depth, r, g, b, F), part by part
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float term[WL::NWT];
            term[0] = gch[p][3];
            term[1] = gch[p][0];
            term[2] = gch[p][1];
            term[3] = gch[p][2];
#pragma unroll
            for (int f = 0; f < F; ++f) term[4 + f] = gch[p][5 + f];
            float4 *row = reinterpret_cast<float4 *>(s_g + (p * 32 + lane) * WL::GROW);
#pragma unroll
            for (int c = 0; c < WL::NWT / 4; ++c)
                row[c] = make_float4(term[4 * c], term[4 * c + 1], term[4 * c + 2], term[4 * c + 3]);
        }
    }

    // Map mode, after a stage of cnt splats: lane (column col, slot group jg) sums, for slots
    // jg SPL + sj, w times the weighted terms [T0, T1) and (with MOM) dpow times (1, ly, ly^2) over
    // the pixels of its column (eight distinct 16-byte rows per quarter-warp read), scales the
    // column sums by the column's coordinate into the six moments, and the eight columns are
    // added by a transpose reduction, lane col keeping block col of the chunk's sums.
    auto contract_chunk = [&](auto t0c, auto t1c, auto momc) {
        constexpr int T0 = decltype(t0c)::value, T1 = decltype(t1c)::value;
        constexpr bool MOM = decltype(momc)::value != 0;
        constexpr int NT = T1 - T0, CV = NT + (MOM ? 6 : 0);
        constexpr int CVP = (WL::SPL * CV + 7) / 8 * 8;
        const int col = lane & 7, jg = lane >> 3;
        float acc[CVP];
#pragma unroll
        for (int c = 0; c < CVP; ++c) acc[c] = 0.f;
#pragma unroll
        for (int ly = 0; ly < WL::ROWS; ++ly) {
            const int q = ly * 8 + col;
            const float lyc = (float)ly + 0.5f - 0.5f * WL::ROWS;
            float w[WL::SPL];
#pragma unroll
            for (int sj = 0; sj < WL::SPL; ++sj) {
                const int j = jg * WL::SPL + sj;
                w[sj] = s_w[j * WL::WROW + q];
                if constexpr (MOM) {
                    const float dp = s_p[j * WL::WROW + q];
                    float *a = acc + sj * CV + NT;
                    a[0] += dp;
                    a[1] = fmaf(lyc, dp, a[1]);
                    a[2] = fmaf(lyc * lyc, dp, a[2]);
                }
            }
            const float4 *g4 = reinterpret_cast<const float4 *>(s_g + q * WL::GROW + T0);
#pragma unroll
            for (int c = 0; c < NT / 4; ++c) {
                const float4 gv = g4[c];
#pragma unroll
                for (int sj = 0; sj < WL::SPL; ++sj) {
                    float *a = acc + sj * CV + 4 * c;
                    a[0] = fmaf(w[sj], gv.x, a[0]);
                    a[1] = fmaf(w[sj], gv.y, a[1]);
                    a[2] = fmaf(w[sj], gv.z, a[2]);
                    a[3] = fmaf(w[sj], gv.w, a[3]);
                }
            }
        }
        if constexpr (MOM) {
            // column sums of dpow (1, ly, ly^2) -> moments (1, lx, ly, lx^2, lx ly, ly^2)
            const float lxc = (float)col - 3.5f;
#pragma unroll
            for (int sj = 0; sj < WL::SPL; ++sj) {
                float *a = acc + sj * CV + NT;
                const float c0 = a[0], c1 = a[1], c2 = a[2];
                a[1] = lxc * c0;
                a[2] = c1;
                a[3] = lxc * lxc * c0;
                a[4] = lxc * c1;
                a[5] = c2;
            }
        }
        // transpose reduction over the eight columns (lanes xor 4, 2, 1)
#pragma unroll
        for (int sft = 4, len = CVP; sft >= 1; sft >>= 1, len >>= 1) {
            const bool up = col & sft;
#pragma unroll
            for (int i = 0; i < len / 2; ++i) {
                const float send = up ? acc[i] : acc[i + len / 2];
                const float keep = up ? acc[i + len / 2] : acc[i];
                acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
            }
        }
#pragma unroll
        for (int i = 0; i < CVP / 8; ++i) {
            const int v = col * (CVP / 8) + i, sj = v / CV, t = v % CV;
            if (v < WL::SPL * CV) s_t[(jg * WL::SPL + sj) * WL::NSV + (t < NT ? T0 + t : WL::NWT + t - NT)] = acc[i];
        }
    };
    // Then lanes (slot j, part) send slot j's sums to the splat's accumulators.
    auto contract = [&](const int cnt) {
        __syncwarp();
        contract_chunk(IntC<0>(), IntC<WL::T1>(), IntC<1>());
        if constexpr (WL::T2 > WL::T1) contract_chunk(IntC<WL::T1>(), IntC<WL::T2>(), IntC<0>());
        if constexpr (WL::T3 > WL::T2) contract_chunk(IntC<WL::T2>(), IntC<WL::T3>(), IntC<0>());
        if constexpr (WL::NWT > WL::T3) contract_chunk(IntC<WL::T3>(), IntC<WL::NWT>(), IntC<0>());
        __syncwarp();
        const int j = lane % STAGE, part = lane / STAGE;
        if (j < cnt) {
            const int64_t item = s_item[j];
            const int64_t g = item - voff;
            // slot j's sums: the terms (depth, r, g, b, F) then the moments (S1, Sx, Sy, Sxx, Sxy, Syy)
            const float *tj = s_t + j * WL::NSV;
            const float m1 = tj[WL::NWT], mx = tj[WL::NWT + 1], my = tj[WL::NWT + 2];
            const float mxx = tj[WL::NWT + 3], mxy = tj[WL::NWT + 4], myy = tj[WL::NWT + 5];
            if (part == 0) {
                // centre and opacity from the moments expanded about the splat centre; depth
                const SplatGeo sg = s_geo[j];
                const float cx = __fadd_rn(__fsub_rn(sg.u, bcx), sg.ulo), cy = __fadd_rn(__fsub_rn(sg.v, bcy), sg.vlo);
                const float Mx = fmaf(-cx, m1, mx), My = fmaf(-cy, m1, my);
                const float du = (-1.f / kLog2e) * fmaf(2.f * sg.qa, Mx, sg.qb * My);
                const float dv = (-1.f / kLog2e) * fmaf(2.f * sg.qc, My, sg.qb * Mx);
                const float4 val = make_float4(du, dv, m1 / sg.o, tj[0]);
                if (val.x != 0.f || val.y != 0.f || val.z != 0.f || val.w != 0.f) atomicAdd(A.acc_uvod + item, val);
            } else if (part == 1) {
                const SplatGeo sg = s_geo[j];
                const float cx = __fadd_rn(__fsub_rn(sg.u, bcx), sg.ulo), cy = __fadd_rn(__fsub_rn(sg.v, bcy), sg.vlo);
                // sum dpow dx^2 = Sxx - 2 cx Sx + cx^2 S1, and likewise
                const float Mxx = fmaf(-cx, fmaf(-cx, m1, 2.f * mx), mxx);
                const float Mxy = fmaf(cx * cy, m1, fmaf(-cx, my, fmaf(-cy, mx, mxy)));
                const float Myy = fmaf(-cy, fmaf(-cy, m1, 2.f * my), myy);
                const float4 val = make_float4(-0.5f * Mxx, -Mxy, -0.5f * Myy, 0.f);
                if (val.x != 0.f || val.y != 0.f || val.z != 0.f) atomicAdd(A.acc_conic + item, val);
            }
            if (part == (WL::LPS > 2 ? 2 : 0)) {
                const float4 val = make_float4(tj[1], tj[2], tj[3], 0.f);
                if (val.x != 0.f || val.y != 0.f || val.z != 0.f) atomicAdd(A.acc_rgb + g, val);
            }
            // features [part D / LPS, (part + 1) D / LPS): the summed feature terms, or W^T times the
            // summed logit terms
            constexpr int DP = D / WL::LPS;
            float *fo = A.d_feat + g * D + part * DP;
#pragma unroll
            for (int c4 = 0; c4 < DP / 4; ++c4) {
                float o4[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = part * DP + 4 * c4 + i;
                    if constexpr (KF > 0) {
                        float sacc = 0.f;
#pragma unroll
                        for (int k = 0; k < KF; ++k) sacc = fmaf(s_basis[k * BROW + c], tj[4 + k], sacc);
                        o4[i] = sacc;
                    } else {
                        o4[i] = tj[4 + c];
                    }
                }
                const float4 val = make_float4(o4[0], o4[1], o4[2], o4[3]);
                if (val.x != 0.f || val.y != 0.f || val.z != 0.f || val.w != 0.f)
                    atomicAdd(reinterpret_cast<float4 *>(fo) + c4, val);
            }
        }
        __syncwarp();
    };

    // Every listed splat was blended by a pixel of the group, so no box culling is needed.
    auto process = [&](const int k, const float *sfeat, const int fstride) {
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
        float val[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) val[i] = 0.f;
        float x[NCH];
        {
            const float4 c = s_rgbd[k];
            x[0] = c.x; x[1] = c.y; x[2] = c.z; x[3] = c.w; x[4] = 1.f;
            const float4 *sf = reinterpret_cast<const float4 *>(sfeat + k * fstride);
#pragma unroll
            for (int q = 0; q < F4; ++q) {
                const float4 f = sf[q];
                x[5 + 4 * q] = f.x; x[6 + 4 * q] = f.y; x[7 + 4 * q] = f.z; x[8 + 4 * q] = f.w;
            }
        }
        // Branch-free over the lanes: a pixel that did not blend the splat runs the same
        // instructions with alpha 0 and keeps its state, and every value it records is 0.
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
            const bool free_alpha = contrib[p] && e[p].oG < prm.alpha_max;
            const float dpow = free_alpha ? e[p].oG * da : 0.f;
            if constexpr (MAP) {
                s_w[k * WL::WROW + p * 32 + lane] = a * Tb;
                s_p[k * WL::WROW + p * 32 + lane] = dpow;
            } else {
                // moments of dpow over the pixels; the splat's constants scale them once, after
                // the warp reduction (geo_grads); the depth term as the sixth value
                const float dx = e[p].dx, dy = e[p].dy;
                const float ax = dx * dpow, ay = dy * dpow;
                val[0] += ax;
                val[1] += ay;
                val[2] = fmaf(ax, dx, val[2]);
                val[3] = fmaf(ax, dy, val[3]);
                val[4] = fmaf(ay, dy, val[4]);
                val[5] = fmaf(a * Tb, gch[p][3], val[5]);
            }
        }
        if constexpr (!MAP) {
            // lane i ends with the warp's value (i mod 8): centre (0, 1), conic (2-4), depth (5); lanes
            // 0-5 add them in one warp-wide reduction instruction
            const uint32_t item = s_item[k];
            const float r = geo_grads(warp_transpose_reduce<8>(val, lane), lane & 7, s);
            if (lane < 6 && r != 0.f) {
                float *dst = lane == 5 ? reinterpret_cast<float *>(A.acc_uvod + item) + 3
                             : lane < 2 ? reinterpret_cast<float *>(A.acc_uvod + item) + lane
                                        : reinterpret_cast<float *>(A.acc_conic + item) + (lane - 2);
                atomicAdd(dst, r);
            }
        }
    };

    // Stages and walks list entries [0, cnt) (instance indices, back to front; cnt <= 32), STAGE at
    // a time: the batch's items are loaded once (one per lane), each stage's records are copied
    // into shared memory asynchronously, the next stage's while the current one is processed,
    // and in map mode each stage's slots are contracted after it.
    auto run_batch = [&](const int cnt) {
        const int si = lane % STAGE, part = lane / STAGE;
        const uint32_t my_ii = lane < cnt ? s_list[lane] : 0u;
        const uint32_t my_item = lane < cnt ? checked_item(A.vals[my_ii], voff, vt.n, A.status) : (uint32_t)voff;
        const int n_st = (cnt + STAGE - 1) / STAGE;
        auto issue = [&](const int st) {
            const int e = st * STAGE + si, b = st & 1;
            const uint32_t item = __shfl_sync(0xffffffffu, my_item, e & 31);
            if (e < cnt) {
                const int64_t g = (int64_t)item - voff;
#pragma unroll
                for (int c = part; c < NCOPY; c += PARTS) {
                    if (c == 0) cp_async16(&r_a[b][si], A.uvdo + item);
                    else if (c == 1) cp_async16(&r_c[b][si], A.conic + item);
                    else if (c == 2) cp_async8(&r_lo[b][si], A.uv_lo + item);
                    else if (RGB32 && c < 6) cp_async4(&r_rgb[b][si][c - 3], rgb + 3 * g + (c - 3));
                    else {
                        const int q = c - (RGB32 ? 6 : 3);
                        cp_async16(&r_f[b][si * FBP + 16 * q], reinterpret_cast<const unsigned char *>(feat + g * D) + 16 * q);
                    }
                }
            }
            cp_async_commit();
        };
        issue(0);
        for (int st = 0; st < n_st; ++st) {
            const int b = st & 1, c_cnt = min(STAGE, cnt - st * STAGE);
            if (st + 1 < n_st) {
                issue(st + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            // the stage's working records from the raw ones
            const int e = st * STAGE + si;
            const uint32_t ii = __shfl_sync(0xffffffffu, my_ii, e & 31);
            const uint32_t item = __shfl_sync(0xffffffffu, my_item, e & 31);
            if (si < c_cnt) {
                const int64_t g = (int64_t)item - voff;
                if (part == 0) {
                    const float4 a = r_a[b][si];
                    s_geo[si] = make_geo(a, r_lo[b][si], r_c[b][si]);
                    s_rgbd[si] = RGB32 ? make_float4(r_rgb[b][si][0], r_rgb[b][si][1], r_rgb[b][si][2], a.z)
                                       : load_rgbd(rgb, g, a.z);
                    s_item[si] = item;
                    s_pos[si] = (int)(ii - start);
                }
                const FT *fr = reinterpret_cast<const FT *>(&r_f[b][si * FBP]);
                if constexpr (KF > 0) {
                    // z = W f for this part's K / PARTS logits
#pragma unroll
                    for (int kk = 0; kk < KF / PARTS; ++kk) {
                        const int k = part * (KF / PARTS) + kk;
                        float z = 0.f;
#pragma unroll
                        for (int q = 0; q < D / 4; ++q) {
                            const float4 f4 = load_feat4(fr, 4 * q);
                            const float4 w4 = reinterpret_cast<const float4 *>(s_basis + k * BROW)[q];
                            z = fmaf(w4.x, f4.x, z);
                            z = fmaf(w4.y, f4.y, z);
                            z = fmaf(w4.z, f4.z, z);
                            z = fmaf(w4.w, f4.w, z);
                        }
                        s_feat[si * F + k] = z;
                    }
                } else if (!RGB32 || sizeof(FT) != 4) {
                    // half storage: the features widened to f32
                    for (int q = part; q < D / 4; q += PARTS)
                        reinterpret_cast<float4 *>(s_feat + si * F)[q] = load_feat4(fr, 4 * q);
                }
            }
            __syncwarp();
            // f32 features are read where they landed; the others from the widened copy
            constexpr bool IN_PLACE = KF == 0 && sizeof(FT) == 4;
            const float *sfeat = IN_PLACE ? reinterpret_cast<const float *>(r_f[b]) : s_feat;
            for (int k = 0; k < c_cnt; ++k) process(k, sfeat, IN_PLACE ? FBP / 4 : F);
            if constexpr (MAP) contract(c_cnt);
            __syncwarp();
        }
    };

    // the group's blended instances, back to front: the mask words are read 32 at a time (lane
    // l holds word wc - l), each word appends its set bits (highest first) to the list, and every
    // 32 entries are staged and processed
    const int64_t lo_i = start, hi_i = (int64_t)start + wmax;
    const int64_t w_lo = lo_i >> 5;
    int n = 0;  // entries in the list (warp-uniform, < 32 between words)
    for (int64_t wc = (hi_i - 1) >> 5; wc >= w_lo; wc -= 32) {
        const int64_t wl = wc - lane;
        uint32_t mw = 0u;
        if (wl >= w_lo) {
#pragma unroll
            for (int j = 0; j < NP; ++j) mw |= A.bmask[(int64_t)SH::group(grp, j) * A.bm_stride + wl];
            const int64_t base = wl << 5;
            if (base < lo_i) mw &= ~0u << (int)(lo_i - base);
            if (hi_i - base < 32) mw &= (1u << (int)(hi_i - base)) - 1u;
        }
        const int nw = wc - w_lo + 1 < 32 ? (int)(wc - w_lo + 1) : 32;
        for (int t = 0; t < nw; ++t) {
            const uint32_t m = __shfl_sync(0xffffffffu, mw, t);
            if (m == 0u) continue;
            const int64_t base = (wc - t) << 5;
            const int b = 31 - lane;
            const int above = lane == 0 ? 0 : __popc(m >> (32 - lane));  // set bits above bit b
            if ((m >> b) & 1u) s_list[n + above] = (uint32_t)(base + b);
            n += __popc(m);
            __syncwarp();
            if (n >= 32) {
                run_batch(32);
                if (lane < n - 32) s_list[lane] = s_list[32 + lane];
                __syncwarp();
                n -= 32;
            }
        }
    }
    if (n > 0) run_batch(n);
}

template <int D, int NP, bool MAP, int KF, typename RT, typename FT>
gs_status launch_bwd_warp(const ViewTable &vt, const Params &prm, const BwdArgs &A, cudaStream_t st) {
    const int n_tiles = vt.tile_off[vt.n_views];
    return launch_pdl(raster_bwd_warp_kernel<D, NP, MAP, KF, RT, FT>, n_tiles * Shape<NP>::WARPS, 32, 0, st, vt, prm,
                      A);
}

// The warp-block form: D 16 or 32, 1 or 2 pixels per thread, blend mask present; factored
// feature gradients (A.feat_basis) with at most kFactorK logits.
template <bool MAP, typename RT, typename FT>
gs_status dispatch_bwd_warp_typed(int D, int np, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                                  cudaStream_t st) {
    if (!A.bmask) return GS_ERR_UNSUPPORTED;
    const bool fact = A.feat_basis != nullptr;
    if (fact && (A.feat_rank < 1 || A.feat_rank > kFactorK || !A.feat_coef)) return GS_ERR_UNSUPPORTED;
#define GS_BWD_WARP(DD, NN)                                                                              \
    if (D == DD && np == NN)                                                                             \
        return fact ? launch_bwd_warp<DD, NN, MAP, kFactorK, RT, FT>(vt, prm, A, st)                     \
                    : launch_bwd_warp<DD, NN, MAP, 0, RT, FT>(vt, prm, A, st);
    GS_BWD_WARP(16, 1) GS_BWD_WARP(16, 2) GS_BWD_WARP(32, 1) GS_BWD_WARP(32, 2)
#undef GS_BWD_WARP
    return GS_ERR_UNSUPPORTED;
}

}  // namespace gs
