// Forward blend (GS3LAM Eq. 4-7 and 10): one CTA per 16x16 tile, NP pixels per
// thread.  Splats of the tile are staged 128 at a time in shared memory (one
// record per thread load) and read back as broadcasts; a warp tests 32 splats at
// a time (one per lane, one ballot) for whether their alpha >= alpha_min region
// reaches its pixel box, and walks only those that do; every pixel walks the
// rest front to back and stops at the T_min threshold; the CTA leaves as soon
// as all of its pixels are done.  With a blend mask, each warp also records, per
// 8x4 pixel group and 32-instance word, which splats any pixel of it blended.
#include <type_traits>

#include "raster.cuh"

namespace gs {
namespace {

// Resident CTAs per SM the register allocation must allow, per feature width and
// pixels per thread: the blend loop is issue-bound, so warps resident matter
// more than the few values ptxas would otherwise keep live across the mask flush.
constexpr int fwd_min_blocks(int D, int NP) {
    return NP == 1 ? (D == 0 ? 8 : D <= 4 ? 6 : D <= 16 ? 5 : 3) : NP == 2 ? (D <= 16 ? 6 : 4) : 6;
}

// One 16x16 tile gt of the blend, by the whole CTA (every exit is uniform over the CTA), staging
// BATCH splats per round; with CNT it also counts each pixel's blended splats (o_nb).
template <int D, int NP, typename RT, typename FT, int BATCH, bool CNT>
__device__ __forceinline__ void fwd_tile(
    const ViewTable &vt, const Params &prm, const float4 *__restrict__ uvdo, const float2 *__restrict__ uv_lo,
    const float4 *__restrict__ conic, const RT *__restrict__ rgb, const FT *__restrict__ feat,
    const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges, int64_t P, float *o_rgb, float *o_depth,
    float *o_sil, float *o_feat, float *o_T, int32_t *o_nc, int32_t *o_nb, uint32_t *bmask, int64_t bm_stride,
    const int gt, int32_t *status, int64_t capacity) {
    using SH = Shape<NP, true>;  // horizontal pixel pairs
    constexpr int NT = SH::THREADS;
    constexpr int NL = SH::PIX_GROUPS ? NP : 1;  // mask bit registers per thread
    constexpr int D4 = D / 4, DD = D > 0 ? D : 1;
    // the batch's records: geometry, culling extents, colour and depth, features
    constexpr int batch = BATCH;
    __shared__ SplatGeo s_geo[BATCH];
    __shared__ float2 s_ext[BATCH];
    __shared__ float4 s_cull[BATCH];
    __shared__ float4 s_rgbd[BATCH];
    __shared__ float4 s_feat[BATCH * (D4 > 0 ? D4 : 1)];

    if (gt < 0 || gt >= vt.tile_off[vt.n_views]) return;  // not a permutation of the tiles: leave the tile
    const int v = view_of_tile(vt, gt);
    const int t = gt - vt.tile_off[v];
    const int tx = t % vt.TX[v], ty = t / vt.TX[v];
    const int tid = threadIdx.x;
    uint32_t start = ranges[2 * gt], end = ranges[2 * gt + 1];
    checked_range(start, end, capacity, status);
    const int64_t voff = (int64_t)v * vt.n;
    int bx0, by0;
    SH::warp_origin(tid >> 5, bx0, by0);
    const float bcx = (float)(tx * kTile + bx0) + 0.5f * SH::BW, bcy = (float)(ty * kTile + by0) + 0.5f * SH::BH;
    const float hx = 0.5f * (SH::BW - 1), hy = 0.5f * (SH::BH - 1);

    float pxc[NP], pyc[NP], T[NP], ar[NP], ag[NP], ab[NP], ad[NP], as[NP], af[NP][DD];
    int last[NP], blended[NP];
    bool inside[NP], done[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        int lx, ly;
        SH::pixel(tid, p, lx, ly);
        const int px = tx * kTile + lx, py = ty * kTile + ly;
        inside[p] = px < vt.W[v] && py < vt.H[v];
        done[p] = !inside[p];
        pxc[p] = (float)px + 0.5f;
        pyc[p] = (float)py + 0.5f;
        T[p] = 1.f;
        ar[p] = ag[p] = ab[p] = ad[p] = as[p] = 0.f;
#pragma unroll
        for (int d = 0; d < DD; ++d) af[p][d] = 0.f;
        last[p] = blended[p] = 0;
    }
    auto all_done = [&]() {
        bool a = true;
#pragma unroll
        for (int p = 0; p < NP; ++p) a = a && done[p];
        return a;
    };
    // blend-mask bits: batches start on 32-instance boundaries, so each 32-splat
    // chunk of a batch is one word of the mask; a lane ORs "my pixel(s) of group j
    // blended splat k" into a register (one per group its pixels lie in) and the
    // warp combines the lanes of each of its NP groups at the end of the chunk
    const int warp = tid >> 5, lane = tid & 31;
    auto flush = [&](const uint32_t (&lbits)[NL], uint32_t word_idx) {
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const uint32_t mine =
                SH::PIX_GROUPS ? lbits[j % NL] : ((SH::lanes_of_group(j) >> lane) & 1u ? lbits[0] : 0u);
            const uint32_t word = __reduce_or_sync(0xffffffffu, mine);
            if (lane == 0 && word) atomicOr(&bmask[(int64_t)SH::group(warp, j) * bm_stride + word_idx], word);
        }
    };

    bool finished = false;
    // every warp stays in the batch loop (it stages splats and meets the CTA
    // barriers); a warp whose pixels are all done only skips the splat loop
    for (uint32_t b0 = start & ~31u; b0 < end; b0 += batch) {
        if (__syncthreads_count(!all_done()) == 0) break;
        for (int i = tid; i < batch; i += NT) {
            const uint32_t j = b0 + i;
            if (j >= start && j < end) {
                const uint32_t item = checked_item(vals[j], voff, vt.n, status);
                const int64_t g = (int64_t)item - voff;
                const float4 a = uvdo[item];
                const float4 c = conic[item];
                s_geo[i] = make_geo(a, uv_lo[item], c);
                s_ext[i] = splat_extent(c, a.w, prm.alpha_min);
                s_cull[i] = ellipse_cull(s_geo[i], prm.alpha_min);
                s_rgbd[i] = load_rgbd(rgb, g, a.z);
#pragma unroll
                for (int q = 0; q < D4; ++q) s_feat[i * D4 + q] = load_feat4(feat, g * D + 4 * q);
            }
        }
        __syncthreads();
        const int k_lo = b0 < start ? (int)(start - b0) : 0;
        const int nb = min((uint32_t)batch, end - b0);
        for (int c0 = k_lo & ~31; c0 < nb && !finished; c0 += 32) {
            uint32_t lbits[NL];
#pragma unroll
            for (int j = 0; j < NL; ++j) lbits[j] = 0u;
            // the chunk's splats in [k_lo, nb) that can reach the warp's box, lane k - c0
            // testing splat k
            const int kl = c0 + lane;
            bool reach = false;
            if (kl >= k_lo && kl < nb) {
                const SplatGeo sg = s_geo[kl];
                reach = reaches_box(sg.u, sg.v, s_ext[kl], bcx, bcy, hx, hy) &&
                        reaches_box_exact(sg, s_cull[kl], bcx, bcy, hx, hy);
            }
            uint32_t todo = __ballot_sync(0xffffffffu, reach);
            for (int n_run = 0; todo; ++n_run) {
                const int k = c0 + __ffs(todo) - 1;
                todo &= todo - 1;
                // every 4th splat walked: are all of the warp's pixels done? (a later exit only
                // runs splats whose pairs blend nothing)
                if ((n_run & 3) == 0 && __all_sync(0xffffffffu, all_done())) { finished = true; break; }
                const SplatGeo s = s_geo[k];
                float al[NP];
                bool ok[NP];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const PairEval e = eval_pair(s, pxc[p], pyc[p], prm.alpha_min, prm.alpha_max);
                    al[p] = e.alpha;
                    ok[p] = !done[p] && !e.skip;
                }
                float wgt[NP];
                bool any = false;
                const int pos = (int)(b0 - start) + k + 1;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float Tn = T[p] * (1.f - al[p]);
                    const bool stop = ok[p] && Tn < prm.T_min;
                    const bool b = ok[p] && !stop;
                    done[p] = done[p] || stop;
                    wgt[p] = b ? al[p] * T[p] : 0.f;
                    T[p] = b ? Tn : T[p];
                    last[p] = b ? pos : last[p];
                    if constexpr (CNT) blended[p] += b ? 1 : 0;
                    any = any || b;
                    if (SH::PIX_GROUPS) lbits[p % NL] |= (b ? 1u : 0u) << (k & 31);
                }
                if (!SH::PIX_GROUPS) lbits[0] |= (any ? 1u : 0u) << (k & 31);
                if (!any) continue;
                const float4 c = s_rgbd[k];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float w = wgt[p];
                    ar[p] = fmaf(w, c.x, ar[p]);
                    ag[p] = fmaf(w, c.y, ag[p]);
                    ab[p] = fmaf(w, c.z, ab[p]);
                    ad[p] = fmaf(w, c.w, ad[p]);
                    as[p] += w;
                }
#pragma unroll
                for (int q = 0; q < D4; ++q) {
                    const float4 f = s_feat[k * D4 + q];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        af[p][4 * q] = fmaf(wgt[p], f.x, af[p][4 * q]);
                        af[p][4 * q + 1] = fmaf(wgt[p], f.y, af[p][4 * q + 1]);
                        af[p][4 * q + 2] = fmaf(wgt[p], f.z, af[p][4 * q + 2]);
                        af[p][4 * q + 3] = fmaf(wgt[p], f.w, af[p][4 * q + 3]);
                    }
                }
            }
            if (bmask) flush(lbits, (b0 + c0) >> 5);
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (!inside[p]) continue;
        const int64_t pix = vt.pix_off[v] + (int64_t)((int)pyc[p]) * vt.W[v] + (int)pxc[p];
        o_rgb[pix] = ar[p] + T[p] * prm.bg[0];
        o_rgb[P + pix] = ag[p] + T[p] * prm.bg[1];
        o_rgb[2 * P + pix] = ab[p] + T[p] * prm.bg[2];
        o_depth[pix] = ad[p];
        o_sil[pix] = as[p];
#pragma unroll
        for (int d = 0; d < D; ++d) o_feat[d * P + pix] = af[p][d];
        o_T[pix] = T[p];
        o_nc[pix] = last[p];
        if (CNT && o_nb) o_nb[pix] = blended[p];
    }
}

// With QUEUE, the grid is as many CTAs as fit on the GPU at once and each takes tiles, in the
// tile order, from the work counter queue[0] until none is left; the last CTA to finish
// (counted in queue[1]) sets both counters back to 0 for the next launch.  Nothing waits.
template <int D, int NP, typename RT, typename FT, bool QUEUE, int BATCH, bool CNT>
__global__ void __launch_bounds__(Shape<NP>::THREADS, fwd_min_blocks(D, NP)) raster_fwd_kernel(
    ViewTable vt, Params prm, const float4 *__restrict__ uvdo, const float2 *__restrict__ uv_lo,
    const float4 *__restrict__ conic, const RT *__restrict__ rgb, const FT *__restrict__ feat,
    const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges, int64_t P, float *o_rgb, float *o_depth,
    float *o_sil, float *o_feat, float *o_T, int32_t *o_nc, int32_t *o_nb, uint32_t *bmask, int64_t bm_stride,
    const uint32_t *__restrict__ order, int32_t *status, int64_t capacity, uint32_t *queue) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    const int n_tiles = vt.tile_off[vt.n_views];
    const bool failed = binning_failed(status);  // the binning overflowed or gave up: render nothing
    if constexpr (QUEUE) {
        __shared__ int s_idx;
        for (;;) {
            __syncthreads();  // the previous tile's reads of shared memory and s_idx are done
            if (threadIdx.x == 0) s_idx = failed ? n_tiles : (int)atomicAdd(queue, 1u);
            __syncthreads();
            const int idx = s_idx;
            if (idx >= n_tiles) break;
            fwd_tile<D, NP, RT, FT, BATCH, CNT>(vt, prm, uvdo, uv_lo, conic, rgb, feat, vals, ranges, P, o_rgb, o_depth, o_sil,
                                    o_feat, o_T, o_nc, o_nb, bmask, bm_stride, order ? (int)order[idx] : idx,
                                    status, capacity);
        }
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {  // every CTA has taken its last item
                queue[0] = 0u;
                queue[1] = 0u;
            }
        }
    } else {
        if (failed) return;
        fwd_tile<D, NP, RT, FT, BATCH, CNT>(vt, prm, uvdo, uv_lo, conic, rgb, feat, vals, ranges, P, o_rgb, o_depth, o_sil,
                                o_feat, o_T, o_nc, o_nb, bmask, bm_stride,
                                order ? (int)order[blockIdx.x] : (int)blockIdx.x, status, capacity);
    }
}

// The same blend with one 32-thread block per pixel group (an 8x4 group with one pixel
// per thread, an 8x8 block with two): the group stages the tile's splats 32 at a time in
// its own shared memory, so it never waits at a barrier for the tile's other groups, and
// it leaves as soon as its own pixels are done, freeing its registers and shared memory.
// Arithmetic, order and outputs are those of raster_fwd_kernel.
// Register caps that keep the blocks spill-free: 80 registers up to D = 16, 128 at D = 32 with two
// pixels per thread.
constexpr int fwd_group_min_blocks(int D, int NP) { return NP == 1 ? 24 : (D <= 16 ? 22 : 16); }

template <int D, int NP, typename RT, typename FT>
__global__ void __launch_bounds__(32, fwd_group_min_blocks(D, NP)) raster_fwd_group_kernel(
    ViewTable vt, Params prm, const float4 *__restrict__ uvdo, const float2 *__restrict__ uv_lo,
    const float4 *__restrict__ conic, const RT *__restrict__ rgb, const FT *__restrict__ feat,
    const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges, int64_t P, float *o_rgb, float *o_depth,
    float *o_sil, float *o_feat, float *o_T, int32_t *o_nc, int32_t *o_nb, uint32_t *bmask, int64_t bm_stride,
    const uint32_t *__restrict__ order, int32_t *status, int64_t capacity, uint32_t * /*queue*/) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    using SH = Shape<NP, true>;  // horizontal pixel pairs
    constexpr int D4 = D / 4, DD = D > 0 ? D : 1;
    constexpr int NL = SH::PIX_GROUPS ? NP : 1;  // mask bit registers per thread
    constexpr int GW = SH::WARPS;  // pixel-group blocks per tile
    __shared__ SplatGeo s_geo[32];
    __shared__ float4 s_rgbd[32];
    __shared__ float4 s_feat[32 * (D4 > 0 ? D4 : 1)];

    if (binning_failed(status)) return;  // the binning overflowed or gave up: render nothing
    const int rank = blockIdx.x / GW, grp = blockIdx.x % GW;
    const int gt = order ? (int)order[rank] : rank;
    if (gt < 0 || gt >= vt.tile_off[vt.n_views]) return;  // not a permutation of the tiles: leave the tile
    const int v = view_of_tile(vt, gt);
    const int t = gt - vt.tile_off[v];
    const int tx = t % vt.TX[v], ty = t / vt.TX[v];
    const int lane = threadIdx.x;
    const int tid = grp * 32 + lane;  // the thread's index in the tile kernel's numbering
    uint32_t start = ranges[2 * gt], end = ranges[2 * gt + 1];
    checked_range(start, end, capacity, status);
    const int64_t voff = (int64_t)v * vt.n;
    int bx0, by0;
    SH::warp_origin(grp, bx0, by0);
    const float bcx = (float)(tx * kTile + bx0) + 0.5f * SH::BW, bcy = (float)(ty * kTile + by0) + 0.5f * SH::BH;
    const float hx = 0.5f * (SH::BW - 1), hy = 0.5f * (SH::BH - 1);

    float pxc[NP], pyc[NP], T[NP], ar[NP], ag[NP], ab[NP], ad[NP], as[NP], af[NP][DD];
    int last[NP], blended[NP];
    bool inside[NP], done[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        int lx, ly;
        SH::pixel(tid, p, lx, ly);
        const int px = tx * kTile + lx, py = ty * kTile + ly;
        inside[p] = px < vt.W[v] && py < vt.H[v];
        done[p] = !inside[p];
        pxc[p] = (float)px + 0.5f;
        pyc[p] = (float)py + 0.5f;
        T[p] = 1.f;
        ar[p] = ag[p] = ab[p] = ad[p] = as[p] = 0.f;
#pragma unroll
        for (int d = 0; d < DD; ++d) af[p][d] = 0.f;
        last[p] = blended[p] = 0;
    }
    auto all_done = [&]() {
        bool a = true;
#pragma unroll
        for (int p = 0; p < NP; ++p) a = a && done[p];
        return a;
    };
    for (uint32_t b0 = start & ~31u; b0 < end; b0 += 32) {
        if (__all_sync(0xffffffffu, all_done())) break;
        // lane k stages splat b0 + k and tests whether it can reach the group's box
        bool reach = false;
        {
            const uint32_t j = b0 + lane;
            if (j >= start && j < end) {
                const uint32_t item = checked_item(vals[j], voff, vt.n, status);
                const int64_t g = (int64_t)item - voff;
                const float4 a = uvdo[item];
                const float4 c = conic[item];
                const SplatGeo sg = make_geo(a, uv_lo[item], c);
                s_geo[lane] = sg;
                reach = reaches_box(a.x, a.y, splat_extent(c, a.w, prm.alpha_min), bcx, bcy, hx, hy) &&
                        reaches_box_exact(sg, ellipse_cull(sg, prm.alpha_min), bcx, bcy, hx, hy);
                s_rgbd[lane] = load_rgbd(rgb, g, a.z);
#pragma unroll
                for (int q = 0; q < D4; ++q) s_feat[lane * D4 + q] = load_feat4(feat, g * D + 4 * q);
            }
        }
        uint32_t todo = __ballot_sync(0xffffffffu, reach);
        __syncwarp();
        uint32_t lbits[NL];
#pragma unroll
        for (int j = 0; j < NL; ++j) lbits[j] = 0u;
        for (int n_run = 0; todo; ++n_run) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1;
            if ((n_run & 3) == 0 && __all_sync(0xffffffffu, all_done())) break;
            const SplatGeo sg = s_geo[k];
            float al[NP];
            bool ok[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const PairEval e = eval_pair(sg, pxc[p], pyc[p], prm.alpha_min, prm.alpha_max);
                al[p] = e.alpha;
                ok[p] = !done[p] && !e.skip;
            }
            float wgt[NP];
            bool any = false;
            const int pos = (int)(b0 - start) + k + 1;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float Tn = T[p] * (1.f - al[p]);
                const bool stop = ok[p] && Tn < prm.T_min;
                const bool b = ok[p] && !stop;
                done[p] = done[p] || stop;
                wgt[p] = b ? al[p] * T[p] : 0.f;
                T[p] = b ? Tn : T[p];
                last[p] = b ? pos : last[p];
                blended[p] += b ? 1 : 0;
                any = any || b;
                if (SH::PIX_GROUPS) lbits[p % NL] |= (b ? 1u : 0u) << k;
            }
            if (!SH::PIX_GROUPS) lbits[0] |= (any ? 1u : 0u) << k;
            if (!any) continue;
            const float4 c = s_rgbd[k];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float w = wgt[p];
                ar[p] = fmaf(w, c.x, ar[p]);
                ag[p] = fmaf(w, c.y, ag[p]);
                ab[p] = fmaf(w, c.z, ab[p]);
                ad[p] = fmaf(w, c.w, ad[p]);
                as[p] += w;
            }
#pragma unroll
            for (int q = 0; q < D4; ++q) {
                const float4 f = s_feat[k * D4 + q];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    af[p][4 * q] = fmaf(wgt[p], f.x, af[p][4 * q]);
                    af[p][4 * q + 1] = fmaf(wgt[p], f.y, af[p][4 * q + 1]);
                    af[p][4 * q + 2] = fmaf(wgt[p], f.z, af[p][4 * q + 2]);
                    af[p][4 * q + 3] = fmaf(wgt[p], f.w, af[p][4 * q + 3]);
                }
            }
        }
        if (bmask) {
            // the chunk is one mask word; words at a tile's ends are shared with the
            // neighbouring tile's blocks, hence the atomic OR
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const uint32_t mine =
                    SH::PIX_GROUPS ? lbits[j % NL] : ((SH::lanes_of_group(j) >> lane) & 1u ? lbits[0] : 0u);
                const uint32_t word = __reduce_or_sync(0xffffffffu, mine);
                if (lane == 0 && word) atomicOr(&bmask[(int64_t)SH::group(grp, j) * bm_stride + (b0 >> 5)], word);
            }
        }
        __syncwarp();  // every lane is done with the staged chunk before the next one
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (!inside[p]) continue;
        const int64_t pix = vt.pix_off[v] + (int64_t)((int)pyc[p]) * vt.W[v] + (int)pxc[p];
        o_rgb[pix] = ar[p] + T[p] * prm.bg[0];
        o_rgb[P + pix] = ag[p] + T[p] * prm.bg[1];
        o_rgb[2 * P + pix] = ab[p] + T[p] * prm.bg[2];
        o_depth[pix] = ad[p];
        o_sil[pix] = as[p];
#pragma unroll
        for (int d = 0; d < D; ++d) o_feat[d * P + pix] = af[p][d];
        o_T[pix] = T[p];
        o_nc[pix] = last[p];
        if (o_nb) o_nb[pix] = blended[p];
    }
}

// One batch slot of the ring forward: B staged splat records.
template <int D, int B>
struct RingSlot {
    SplatGeo geo[B];
    float2 ext[B];
    float4 cull[B];
    float4 rgbd[B];
    float4 feat[B * (D / 4 > 0 ? D / 4 : 1)];
};

// The per-tile forward with its splats staged into a ring of NBUF batch slots of B records:
// the four warps stage each batch together (a quarter each) and walk the staged batches at
// their own pace, synchronised per slot by mbarriers instead of CTA barriers: slot full (every
// warp has staged its quarter) and slot empty (every warp has walked it), so a warp can run up
// to NBUF - 1 batches ahead of the slowest.  A warp whose pixels are all done still stages
// its quarters; once every warp's pixels are done, the next batch staged carries a stop flag
// and every warp leaves at that same batch.  Arithmetic, order and outputs are those of
// raster_fwd_kernel.  Every wait is bounded (prm.spin_limit polls); one that gives up sets
// GS_ERR_TIMEOUT in the status word and its warp leaves without writing its pixels.
template <int D, typename RT, typename FT, int B, int NBUF>
__global__ void __launch_bounds__(Shape<2, true>::THREADS, fwd_min_blocks(D, 2)) raster_fwd_ring_kernel(
    ViewTable vt, Params prm, const float4 *__restrict__ uvdo, const float2 *__restrict__ uv_lo,
    const float4 *__restrict__ conic, const RT *__restrict__ rgb, const FT *__restrict__ feat,
    const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges, int64_t P, float *o_rgb, float *o_depth,
    float *o_sil, float *o_feat, float *o_T, int32_t *o_nc, int32_t *o_nb, uint32_t *bmask, int64_t bm_stride,
    const uint32_t *__restrict__ order, int32_t *status, int64_t capacity, uint32_t * /*queue*/) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    constexpr int NP = 2;
    using SH = Shape<NP, true>;  // horizontal pixel pairs
    constexpr int NT = SH::THREADS, NW = SH::WARPS;
    constexpr int NL = SH::PIX_GROUPS ? NP : 1;
    constexpr int D4 = D / 4, DD = D > 0 ? D : 1;
    constexpr int QB = B / NW;  // records a warp stages per batch
    static_assert(B % 32 == 0 && QB <= 32 && NBUF >= 2, "ring shape");
    __shared__ RingSlot<D, B> s_slot[NBUF];
    __shared__ __align__(8) uint64_t s_full[NBUF], s_empty[NBUF];
    __shared__ int s_stop[NBUF][NW];
    __shared__ int s_done;

    if (binning_failed(status)) return;  // the binning overflowed or gave up: render nothing
    const int gt = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    if (gt < 0 || gt >= vt.tile_off[vt.n_views]) return;  // not a permutation of the tiles: leave the tile
    const int v = view_of_tile(vt, gt);
    const int t = gt - vt.tile_off[v];
    const int tx = t % vt.TX[v], ty = t / vt.TX[v];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t start = ranges[2 * gt], end = ranges[2 * gt + 1];
    checked_range(start, end, capacity, status);
    const int64_t voff = (int64_t)v * vt.n;
    if (tid < NBUF) {
        mbar_init(&s_full[tid], NT);
        mbar_init(&s_empty[tid], NT);
    }
    if (tid == 0) s_done = 0;
    __syncthreads();  // the barriers are initialised before any thread uses them

    const uint32_t first = start & ~31u;
    const int n_batch = end > first ? (int)((end - first + B - 1) / B) : 0;
    // warp `warp` stages records [warp QB, (warp + 1) QB) of batch j into its slot, with its
    // stop flag (every warp's pixels done when it staged), then arrives on the slot's full barrier
    auto stage = [&](int j) {
        RingSlot<D, B> &S = s_slot[j % NBUF];
        const uint32_t b0 = first + (uint32_t)j * B;
        if (lane < QB) {
            const int k = warp * QB + lane;
            const uint32_t jj = b0 + k;
            if (jj >= start && jj < end) {
                const uint32_t item = checked_item(vals[jj], voff, vt.n, status);
                const int64_t g = (int64_t)item - voff;
                const float4 a = uvdo[item];
                const float4 c = conic[item];
                const SplatGeo sg = make_geo(a, uv_lo[item], c);
                S.geo[k] = sg;
                S.ext[k] = splat_extent(c, a.w, prm.alpha_min);
                S.cull[k] = ellipse_cull(sg, prm.alpha_min);
                S.rgbd[k] = load_rgbd(rgb, g, a.z);
#pragma unroll
                for (int q = 0; q < D4; ++q) S.feat[k * D4 + q] = load_feat4(feat, g * D + 4 * q);
            }
        }
        if (lane == 0) s_stop[j % NBUF][warp] = *(volatile int *)&s_done == NW;
        mbar_arrive(&s_full[j % NBUF]);
    };

    int bx0, by0;
    SH::warp_origin(warp, bx0, by0);
    const float bcx = (float)(tx * kTile + bx0) + 0.5f * SH::BW, bcy = (float)(ty * kTile + by0) + 0.5f * SH::BH;
    const float hx = 0.5f * (SH::BW - 1), hy = 0.5f * (SH::BH - 1);
    float pxc[NP], pyc[NP], T[NP], ar[NP], ag[NP], ab[NP], ad[NP], as[NP], af[NP][DD];
    int last[NP], blended[NP];
    bool inside[NP], done[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        int lx, ly;
        SH::pixel(tid, p, lx, ly);
        const int px = tx * kTile + lx, py = ty * kTile + ly;
        inside[p] = px < vt.W[v] && py < vt.H[v];
        done[p] = !inside[p];
        pxc[p] = (float)px + 0.5f;
        pyc[p] = (float)py + 0.5f;
        T[p] = 1.f;
        ar[p] = ag[p] = ab[p] = ad[p] = as[p] = 0.f;
#pragma unroll
        for (int d = 0; d < DD; ++d) af[p][d] = 0.f;
        last[p] = blended[p] = 0;
    }
    auto all_done = [&]() {
        bool a = true;
#pragma unroll
        for (int p = 0; p < NP; ++p) a = a && done[p];
        return a;
    };
    auto flush = [&](const uint32_t (&lbits)[NL], uint32_t word_idx) {
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const uint32_t mine =
                SH::PIX_GROUPS ? lbits[j % NL] : ((SH::lanes_of_group(j) >> lane) & 1u ? lbits[0] : 0u);
            const uint32_t word = __reduce_or_sync(0xffffffffu, mine);
            if (lane == 0 && word) atomicOr(&bmask[(int64_t)SH::group(warp, j) * bm_stride + word_idx], word);
        }
    };

    // a wait the whole warp takes together (every lane sees the phase complete), bounded
    auto wait_warp = [&](uint64_t *bar, uint32_t parity) {
        for (int it = 0;; ++it) {
            if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
            if (prm.spin_limit < 0 || it >= prm.spin_limit) return false;
        }
    };
    for (int j = 0; j < NBUF - 1 && j < n_batch; ++j) stage(j);
    bool counted = false;  // this warp's pixels are all done and s_done counts it
    bool ok = true;
    for (int i = 0; i < n_batch; ++i) {
        const int slot = i % NBUF;
        if (!wait_warp(&s_full[slot], (uint32_t)(i / NBUF) & 1u)) {
            ok = false;
            break;
        }
        bool stop = false;
#pragma unroll
        for (int w = 0; w < NW; ++w) stop = stop || s_stop[slot][w];
        if (stop) break;  // the same batch for every warp: every pixel of the tile is done
        const RingSlot<D, B> &S = s_slot[slot];
        const uint32_t b0 = first + (uint32_t)i * B;
        if (!__all_sync(0xffffffffu, all_done())) {
            const int k_lo = b0 < start ? (int)(start - b0) : 0;
            const int nb = min((uint32_t)B, end - b0);
            bool finished = false;
            for (int c0 = k_lo & ~31; c0 < nb && !finished; c0 += 32) {
                uint32_t lbits[NL];
#pragma unroll
                for (int jj = 0; jj < NL; ++jj) lbits[jj] = 0u;
                const int kl = c0 + lane;
                bool reach = false;
                if (kl >= k_lo && kl < nb) {
                    const SplatGeo sg = S.geo[kl];
                    reach = reaches_box(sg.u, sg.v, S.ext[kl], bcx, bcy, hx, hy) &&
                            reaches_box_exact(sg, S.cull[kl], bcx, bcy, hx, hy);
                }
                uint32_t todo = __ballot_sync(0xffffffffu, reach);
                for (int n_run = 0; todo; ++n_run) {
                    const int k = c0 + __ffs(todo) - 1;
                    todo &= todo - 1;
                    if ((n_run & 3) == 0 && __all_sync(0xffffffffu, all_done())) { finished = true; break; }
                    const SplatGeo s = S.geo[k];
                    float al[NP];
                    bool okp[NP];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const PairEval e = eval_pair(s, pxc[p], pyc[p], prm.alpha_min, prm.alpha_max);
                        al[p] = e.alpha;
                        okp[p] = !done[p] && !e.skip;
                    }
                    float wgt[NP];
                    bool any = false;
                    const int pos = (int)(b0 - start) + k + 1;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const float Tn = T[p] * (1.f - al[p]);
                        const bool stp = okp[p] && Tn < prm.T_min;
                        const bool b = okp[p] && !stp;
                        done[p] = done[p] || stp;
                        wgt[p] = b ? al[p] * T[p] : 0.f;
                        T[p] = b ? Tn : T[p];
                        last[p] = b ? pos : last[p];
                        blended[p] += b ? 1 : 0;
                        any = any || b;
                        if (SH::PIX_GROUPS) lbits[p % NL] |= (b ? 1u : 0u) << (k & 31);
                    }
                    if (!SH::PIX_GROUPS) lbits[0] |= (any ? 1u : 0u) << (k & 31);
                    if (!any) continue;
                    const float4 c = S.rgbd[k];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const float w = wgt[p];
                        ar[p] = fmaf(w, c.x, ar[p]);
                        ag[p] = fmaf(w, c.y, ag[p]);
                        ab[p] = fmaf(w, c.z, ab[p]);
                        ad[p] = fmaf(w, c.w, ad[p]);
                        as[p] += w;
                    }
#pragma unroll
                    for (int q = 0; q < D4; ++q) {
                        const float4 f = S.feat[k * D4 + q];
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            af[p][4 * q] = fmaf(wgt[p], f.x, af[p][4 * q]);
                            af[p][4 * q + 1] = fmaf(wgt[p], f.y, af[p][4 * q + 1]);
                            af[p][4 * q + 2] = fmaf(wgt[p], f.z, af[p][4 * q + 2]);
                            af[p][4 * q + 3] = fmaf(wgt[p], f.w, af[p][4 * q + 3]);
                        }
                    }
                }
                if (bmask) flush(lbits, (b0 + c0) >> 5);
            }
        }
        if (!counted && __all_sync(0xffffffffu, all_done())) {
            counted = true;
            if (lane == 0) atomicAdd(&s_done, 1);
        }
        __syncwarp();
        mbar_arrive(&s_empty[slot]);
        // batch i + NBUF - 1 goes into the slot batch i - 1 used, once every warp has walked it
        const int jn = i + NBUF - 1;
        if (jn < n_batch) {
            if (i >= 1 && !wait_warp(&s_empty[jn % NBUF], (uint32_t)((i - 1) / NBUF) & 1u)) {
                ok = false;
                break;
            }
            stage(jn);
        }
    }
    if (!ok) {
        set_status(status, GS_ERR_TIMEOUT);
        return;  // this warp's pixels stay unwritten; the status word says so
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (!inside[p]) continue;
        const int64_t pix = vt.pix_off[v] + (int64_t)((int)pyc[p]) * vt.W[v] + (int)pxc[p];
        o_rgb[pix] = ar[p] + T[p] * prm.bg[0];
        o_rgb[P + pix] = ag[p] + T[p] * prm.bg[1];
        o_rgb[2 * P + pix] = ab[p] + T[p] * prm.bg[2];
        o_depth[pix] = ad[p];
        o_sil[pix] = as[p];
#pragma unroll
        for (int d = 0; d < D; ++d) o_feat[d * P + pix] = af[p][d];
        o_T[pix] = T[p];
        o_nc[pix] = last[p];
        if (o_nb) o_nb[pix] = blended[p];
    }
}

template <int D, int NP, typename RT, typename FT>
gs_status launch(const ViewTable &vt, const Params &prm, const gs_gaussians *g, const gs_projected *proj,
                 const gs_binning *bins, gs_images *out, cudaStream_t st) {
    const int tiles = vt.tile_off[vt.n_views];
    const int64_t P = vt.pix_off[vt.n_views];
    auto args = [&](auto kern, int blocks, int threads, size_t smem) -> gs_status {
        return launch_pdl(
            kern, blocks, threads, smem, st, vt, prm, reinterpret_cast<const float4 *>(proj->uvdo),
            reinterpret_cast<const float2 *>(proj->uv_lo), reinterpret_cast<const float4 *>(proj->conic),
            static_cast<const RT *>(g->rgb), static_cast<const FT *>(g->feat), bins->vals, bins->ranges, P, out->rgb,
            out->depth, out->sil, out->feat, out->T_final, out->n_contrib, out->n_blended, out->blend_mask,
            bins->capacity / 32 + 1, bins->tile_order, bins->status, bins->capacity, bins->queue);
    };
    if constexpr (NP <= 2) {
        if (prm.fwd_group) {
            return args(raster_fwd_group_kernel<D, NP, RT, FT>, tiles * Shape<NP>::WARPS, 32, 0);
        }
    }
    if (prm.fwd_ring) {
        // batch slots within the 48 KB of static shared memory: two of 128 or four of 64 records
        // at D = 16, three of 64 at D = 32
        if constexpr (NP == 2 && D == 16) {
            if (prm.fwd_batch == 128)
                return args(raster_fwd_ring_kernel<D, RT, FT, 128, 2>, tiles, Shape<2, true>::THREADS, 0);
            if (prm.fwd_batch == 64)
                return args(raster_fwd_ring_kernel<D, RT, FT, 64, 4>, tiles, Shape<2, true>::THREADS, 0);
        }
        if constexpr (NP == 2 && D == 32)
            if (prm.fwd_batch == 64)
                return args(raster_fwd_ring_kernel<D, RT, FT, 64, 3>, tiles, Shape<2, true>::THREADS, 0);
        return GS_ERR_UNSUPPORTED;
    }
    // the per-tile forward with BATCH splats staged per round; batches other than 128 are built
    // for the two-pixel shape: 64 at feature widths 16 and 32, 256 at 16
    // (the blended-splat count is compiled in only for a caller that asks for it)
    auto per_tile_cnt = [&](auto batch_c, auto cnt_c) -> gs_status {
        constexpr int B = decltype(batch_c)::value;
        constexpr bool C = decltype(cnt_c)::value;
        if (prm.fwd_queue) {
            // one wave: as many CTAs as are resident at once
            static int res = 0;  // this kernel instance: SMs x resident CTAs per SM
            if (res == 0) {
                int dev = 0, sms = 0, per_sm = 0;
                if (cudaGetDevice(&dev) != cudaSuccess ||
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_fwd_kernel<D, NP, RT, FT, true, B, C>,
                                                                  Shape<NP>::THREADS, 0) != cudaSuccess)
                    return GS_ERR_CUDA;
                res = sms * (per_sm > 0 ? per_sm : 1);
            }
            return args(raster_fwd_kernel<D, NP, RT, FT, true, B, C>, tiles < res ? tiles : res, Shape<NP>::THREADS,
                        0);
        }
        return args(raster_fwd_kernel<D, NP, RT, FT, false, B, C>, tiles, Shape<NP>::THREADS, 0);
    };
    auto per_tile = [&](auto batch_c) -> gs_status {
        return out->n_blended ? per_tile_cnt(batch_c, std::true_type()) : per_tile_cnt(batch_c, std::false_type());
    };
    if (prm.fwd_batch == 128) return per_tile(std::integral_constant<int, 128>());
    if constexpr (NP == 2 && D >= 16)
        if (prm.fwd_batch == 64) return per_tile(std::integral_constant<int, 64>());
    if constexpr (NP == 2 && D == 16)  // 256 records of D = 32 would not fit the 48 KB of static shared memory
        if (prm.fwd_batch == 256) return per_tile(std::integral_constant<int, 256>());
    return GS_ERR_UNSUPPORTED;
}

template <int D, typename RT, typename FT>
gs_status by_np(int np, const ViewTable &vt, const Params &prm, const gs_gaussians *g, const gs_projected *proj,
                const gs_binning *bins, gs_images *out, cudaStream_t st) {
    if (np == 1) return launch<D, 1, RT, FT>(vt, prm, g, proj, bins, out, st);
    if constexpr (D >= 16) {
        if (np == 2) return launch<D, 2, RT, FT>(vt, prm, g, proj, bins, out, st);
        if constexpr (D <= 16)
            if (np == 4) return launch<D, 4, RT, FT>(vt, prm, g, proj, bins, out, st);
    }
    return GS_ERR_UNSUPPORTED;
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
    GS_NVTX_RANGE("gs_render_fwd");
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
    if (out->blend_mask) {
        const gs_status s = cuda_status(cudaMemsetAsync(
            out->blend_mask, 0, sizeof(uint32_t) * kGroups * (size_t)(bins->capacity / 32 + 1), st));
        if (s) return s;
    }
    const int np = prm.fwd_np ? prm.fwd_np : default_fwd_np(g->feat_dim);
    prm.fwd_group = prm.fwd_blocks == GS_BWD_BLOCKS_GROUP;
    prm.fwd_queue = prm.fwd_blocks == GS_BLOCKS_QUEUE;
    prm.fwd_ring = prm.fwd_blocks == GS_BLOCKS_RING;
    if (prm.fwd_ring && np != 2) return GS_ERR_UNSUPPORTED;
    if (prm.fwd_group && np > 2) return GS_ERR_UNSUPPORTED;
    if (prm.fwd_queue && !bins->queue) return GS_ERR_ARG;
    if (g->rgb_dtype == GS_F16) {
        if (g->feat_dim == 16) return by_np<16, __half, __nv_bfloat16>(np, vt, prm, g, proj, bins, out, st);
        return by_np<32, __half, __nv_bfloat16>(np, vt, prm, g, proj, bins, out, st);
    }
    switch (g->feat_dim) {
        case 0: return by_np<0, float, float>(np, vt, prm, g, proj, bins, out, st);
        case 4: return by_np<4, float, float>(np, vt, prm, g, proj, bins, out, st);
        case 8: return by_np<8, float, float>(np, vt, prm, g, proj, bins, out, st);
        case 16: return by_np<16, float, float>(np, vt, prm, g, proj, bins, out, st);
        case 32: return by_np<32, float, float>(np, vt, prm, g, proj, bins, out, st);
        default: return GS_ERR_UNSUPPORTED;
    }
}
