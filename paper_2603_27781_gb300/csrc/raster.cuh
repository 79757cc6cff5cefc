// Shared pieces of the blend kernels: splat staging and storage conversions.
#pragma once

#include "common.cuh"

namespace gs {

// Storage forms of colour and feature (F32 plain, F16 colour + BF16 feature).
template <typename T> struct Store;
template <> struct Store<float> { static constexpr int code = GS_F32; };
template <> struct Store<__half> { static constexpr int code = GS_F16; };
template <> struct Store<__nv_bfloat16> { static constexpr int code = GS_BF16; };

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

// Pixel of thread `tid` in a 16x16 tile: each warp covers an 8x4 block.
__device__ __forceinline__ void tile_pixel(int tid, int tx, int ty, int &px, int &py) {
    int lane = tid & 31, w = tid >> 5;
    px = tx * kTile + (w & 1) * 8 + (lane & 7);
    py = ty * kTile + (w >> 1) * 4 + (lane >> 3);
}

}  // namespace gs
