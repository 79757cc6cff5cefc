// Shared pieces of the blend kernels: launch shapes, splat staging and culling,
// storage conversions.
#pragma once

#include "common.cuh"

namespace gs {

constexpr int kBatch = 128;  // splats staged in shared memory per round

// Launch shape with NP pixels per thread (1, 2 or 4) for one 16x16 tile.
//   NP = 1: 8 warps, each an 8x4 block of pixels;
//   NP = 2: 4 warps, each an 8x8 block, a thread owning 2 pixels 4 rows apart
//           (pixel p in the block's p-th 8x4 half), or with HPAIR 2 horizontal
//           neighbours;
//   NP = 4: 2 warps, each a 16x8 band, a thread owning a 2x2 block.
// A thread's pixels share every shared-memory read of a splat and are
// evaluated together, so their arithmetic chains interleave.  Square 8x8 blocks
// have a shorter edge than 16x4 bands, so fewer splats reach a block without
// reaching most of its pixels (6 % fewer walked by the per-group backward).  On the
// 1M-Gaussian 1200x680 frame the forward ran fastest with horizontal pairs and the
// backward with vertical ones.
template <int NP, bool HPAIR = false> struct Shape {
    static constexpr int THREADS = kTilePix / NP;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int BW = NP == 4 ? 16 : 8;  // warp box width
    static constexpr int BH = NP == 1 ? 4 : 8;
    // pixel p of every thread lies in the warp's p-th blend-mask group (vertical pairs);
    // otherwise all pixels of a thread lie in one group
    static constexpr bool PIX_GROUPS = NP == 2 && !HPAIR;
    __device__ static void warp_origin(int w, int &x0, int &y0) {
        x0 = NP == 4 ? 0 : (w & 1) * 8;
        y0 = NP == 1 ? (w >> 1) * 4 : (NP == 2 ? (w >> 1) * 8 : w * BH);
    }
    __device__ static void pixel(int tid, int p, int &lx, int &ly) {
        const int lane = tid & 31, w = tid >> 5;
        int x0, y0;
        warp_origin(w, x0, y0);
        if (NP == 1) { lx = x0 + (lane & 7); ly = y0 + (lane >> 3); }
        else if (NP == 2 && HPAIR) { lx = x0 + (lane & 3) * 2 + p; ly = y0 + (lane >> 2); }
        else if (NP == 2) { lx = x0 + (lane & 7); ly = y0 + (lane >> 3) + 4 * p; }
        else { lx = (lane & 7) * 2 + (p & 1); ly = y0 + (lane >> 3) * 2 + (p >> 1); }
    }
    // blend-mask group of the j-th (j < NP) of warp w's groups
    __host__ __device__ static constexpr int group(int w, int j) {
        return NP == 1 ? w : (NP == 2 ? ((w >> 1) * 2 + j) * 2 + (w & 1) : w * 4 + j);
    }
    // where a thread's pixels share one group: which lanes own pixels of warp group j
    __device__ static uint32_t lanes_of_group(int j) {
        if (NP == 1 || PIX_GROUPS) return 0xffffffffu;
        if (NP == 2) return j == 0 ? 0x0000ffffu : 0xffff0000u;
        const uint32_t m[4] = {0x00000f0fu, 0x0000f0f0u, 0x0f0f0000u, 0xf0f00000u};
        return m[j];
    }
};

// Blend-mask groups: fixed 8x4 pixel groups g = (ly / 4) * 2 + lx / 8 of a tile, whatever
// the launch shape.  Warp w of a Shape covers groups Shape::group(w, j), j < NP.
constexpr int kGroups = 8;

// Colour of Gaussian g with the splat depth in the fourth lane (both are blended values).
template <typename T>
__device__ __forceinline__ float4 load_rgbd(const T *rgb, int64_t g, float depth) {
    return make_float4(to_f32(rgb[3 * g]), to_f32(rgb[3 * g + 1]), to_f32(rgb[3 * g + 2]), depth);
}

// Loads 4 consecutive feature values (16-byte aligned for f32, 8 for bf16).
template <typename T> __device__ __forceinline__ float4 load_feat4(const T *f, int64_t idx);
template <> __device__ __forceinline__ float4 load_feat4<float>(const float *f, int64_t idx) {
    return *reinterpret_cast<const float4 *>(f + idx);
}
template <> __device__ __forceinline__ float4 load_feat4<__nv_bfloat16>(const __nv_bfloat16 *f, int64_t idx) {
    uint2 raw = *reinterpret_cast<const uint2 *>(f + idx);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&raw.x), b = *reinterpret_cast<__nv_bfloat162 *>(&raw.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

__device__ __forceinline__ SplatGeo make_geo(float4 a, float2 lo, float4 c) {
    SplatGeo s;
    s.u = a.x;
    s.v = a.y;
    s.ulo = lo.x;
    s.vlo = lo.y;
    s.o = a.w;
    s.qa = -0.5f * kLog2e * c.x;
    s.qb = -kLog2e * c.y;
    s.qc = -0.5f * kLog2e * c.z;
    return s;
}

// Half extents (x, y) of the region where the splat can reach alpha >= alpha_min:
// o exp(-q/2) >= alpha_min  <=>  q <= 2 ln(o / alpha_min), and the ellipse
// x^T Sigma^-1 x <= qmax spans +-sqrt(qmax Sigma_xx) in x.  Widened by 0.1% and
// 0.01 px so that f32 rounding never culls a pixel the evaluation would blend;
// infinite (no culling) when alpha_min is 0.
__device__ __forceinline__ float2 splat_extent(float4 c, float o, float alpha_min) {
    if (!(alpha_min > 0.f)) return make_float2(INFINITY, INFINITY);
    if (!(o > alpha_min)) return make_float2(-1.f, -1.f);
    const float qmax = 2.f * logf(o / alpha_min);
    const float det = c.x * c.z - c.y * c.y;
    if (!(det > 0.f)) return make_float2(INFINITY, INFINITY);
    const float sxx = c.z / det, syy = c.x / det;
    return make_float2(sqrtf(qmax * sxx) * 1.001f + 0.01f, sqrtf(qmax * syy) * 1.001f + 0.01f);
}

// Checked build (compiled with GS_CHECKS=1): the indices a blend kernel takes from the
// binning and the forward images are verified before use.  A tile's instance range must lie
// within the binning's capacity and a staged item must be one of its view's Gaussians; a
// violation sets GS_ERR_CHECK in the binning's status word and the access is replaced by an
// in-bounds one (an empty range, the view's first Gaussian).  Without GS_CHECKS these are
// no-ops.
#ifndef GS_CHECKS
#define GS_CHECKS 0
#endif

__device__ __forceinline__ void checked_range(uint32_t &start, uint32_t &end, int64_t capacity, int32_t *status) {
    if (GS_CHECKS && !(start <= end && (int64_t)end <= capacity)) {
        set_status(status, GS_ERR_CHECK);
        end = start = 0;
    }
}

__device__ __forceinline__ uint32_t checked_item(uint32_t item, int64_t voff, int64_t n, int32_t *status) {
    if (GS_CHECKS && !((int64_t)item >= voff && (int64_t)item < voff + n)) {
        set_status(status, GS_ERR_CHECK);
        return (uint32_t)voff;
    }
    return item;
}

// The number of a tile's instances the backward walks (the largest last-contributor position
// of its pixels): within the tile's range, which lies within the capacity; else 0.
__device__ __forceinline__ int checked_last(uint32_t start, const uint32_t *ranges, int gt, int last,
                                            int64_t capacity, int32_t *status) {
    if (GS_CHECKS) {
        const uint32_t end = ranges[2 * gt + 1];
        if (!(start <= end && (int64_t)end <= capacity && last >= 0 && (uint32_t)last <= end - start)) {
            set_status(status, GS_ERR_CHECK);
            return 0;
        }
    }
    return last;
}

// Whether a splat centred at (u, v) with extent e can reach the warp's pixel box
// (pixel centres from (bx0 + 0.5, by0 + 0.5), bw x bh of them).
__device__ __forceinline__ bool reaches_box(float u, float v, float2 e, float bcx, float bcy, float hx, float hy) {
    return fabsf(u - bcx) <= e.x + hx && fabsf(v - bcy) <= e.y + hy;
}

// The splat's constants for reaches_box_exact: the edge optima rx = -qb / (2 qc), ry = -qb /
// (2 qa) and the exponent threshold log2(alpha_min / o) (-inf when alpha_min is 0).
__device__ __forceinline__ float4 ellipse_cull(const SplatGeo &s, float alpha_min) {
    return make_float4(-s.qb / (2.f * s.qc), -s.qb / (2.f * s.qa), __log2f(alpha_min) - __log2f(s.o), 0.f);
}

// Whether any point of the box of pixel centres [bcx - hx, bcx + hx] x [bcy - hy, bcy + hy]
// can have alpha >= alpha_min, i.e. exponent p(x, y) = qa x^2 + qb x y + qc y^2 >= log2(alpha_min
// / o) with (x, y) relative to the centre: the exact ellipse against the box, where the
// extent test bounds the ellipse by its rectangle.  p is concave with its maximum 0 at the
// centre; with the centre outside the box its maximum over the box lies on an edge, on the
// vertical edge x = xe at y = clamp(rx xe) and on the horizontal edge y = ye at
// x = clamp(ry ye).  Conservative: the box is widened by 0.01 px (the centre's low part and the
// rounding of pixel - centre) and the threshold lowered by 1e-5 of the largest term magnitude
// over the box plus 1e-4 (rounding of p and of the exponential), so no pair that the evaluation
// would blend is culled.
__device__ __forceinline__ bool reaches_box_exact(const SplatGeo &s, float4 k, float bcx, float bcy, float hx,
                                                  float hy) {
    const float x0 = (bcx - hx - 0.01f) - s.u, x1 = (bcx + hx + 0.01f) - s.u;
    const float y0 = (bcy - hy - 0.01f) - s.v, y1 = (bcy + hy + 0.01f) - s.v;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
    auto p = [&](float x, float y) { return fmaf(fmaf(s.qa, x, s.qb * y), x, s.qc * y * y); };
    const float ya = fminf(fmaxf(k.x * x0, y0), y1), yb = fminf(fmaxf(k.x * x1, y0), y1);
    const float xa = fminf(fmaxf(k.y * y0, x0), x1), xb = fminf(fmaxf(k.y * y1, x0), x1);
    const float best = fmaxf(fmaxf(p(x0, ya), p(x1, yb)), fmaxf(p(xa, y0), p(xb, y1)));
    const float X = fmaxf(fabsf(x0), fabsf(x1)), Y = fmaxf(fabsf(y0), fabsf(y1));
    const float mag = fmaf(-s.qa, X * X, fmaf(fabsf(s.qb), X * Y, -s.qc * Y * Y));
    return best >= k.z - fmaf(1e-5f, mag, 1e-4f);
}

}  // namespace gs
