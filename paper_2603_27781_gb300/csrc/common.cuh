// Shared device/host helpers of libgs (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <algorithm>

#include "gs.h"

namespace gs {

constexpr int kMaxViews = 64;
constexpr int kTile = 16;
constexpr int kTilePix = kTile * kTile;  // one thread per pixel, 8 warps per tile
constexpr float kLog2e = 1.4426950408889634f;

// Per-call camera table, passed by value as a kernel argument.
struct ViewTable {
    int n_views;
    int64_t n;                       // Gaussians per view
    int tile_off[kMaxViews + 1];     // first global tile of each view
    int64_t pix_off[kMaxViews + 1];  // first pixel of each view
    int W[kMaxViews], H[kMaxViews], TX[kMaxViews], TY[kMaxViews];
    float fx[kMaxViews], fy[kMaxViews], cx[kMaxViews], cy[kMaxViews];
    float T[kMaxViews][12];          // rows 0..2 of world->camera
    // clamp interval of (x/z, y/z) for the EWA Jacobian: the view widened by 15% per side
    float jx_lo[kMaxViews], jx_hi[kMaxViews], jy_lo[kMaxViews], jy_hi[kMaxViews];
};

struct Params {
    float alpha_min, alpha_max, T_min, z_near, lowpass, radius_sigma;
    float bg[3];
    int fwd_np, bwd_np;  // pixels per thread of the blend kernels (0 = default for the feature dim)
    int bwd_blocks;      // map-mode backward block shape (GS_BWD_BLOCKS_*)
    bool bwd_warp;       // resolved: map-mode backward as one 32-thread block per pixel group
    int fwd_blocks;      // forward block shape (GS_BWD_BLOCKS_*)
    bool fwd_group;      // resolved: forward as one 32-thread block per pixel group
    bool fwd_queue;      // resolved: forward as resident CTAs taking tiles from a work counter
    bool fwd_ring;       // resolved: forward with the tile's splats staged into a ring of batch slots
    bool exact_jacobian; // GS_JACOBIAN_EXACT: J of Eq. 3 at the unclamped (x/z, y/z)
    int spin_limit;      // polls of a bounded wait before it gives up (< 0: at once)
    int fwd_batch;       // splats staged per round by the per-tile forward (64, 128 or 256)
};

constexpr int kDefaultSpinLimit = 1 << 22;

// Whether a binning's status word is set (capacity overflow or a wait that gave up): every
// kernel after the failure skips its work.  The word was written by an earlier kernel of the
// stream or by a block of the running one; either way a set word is never cleared before the
// next binning.
__device__ __forceinline__ bool binning_failed(const int32_t *status) {
    return status && __ldcg(status) != 0;
}

// Default pixels per thread of the blend kernels for a feature dimension.
inline int default_fwd_np(int D) { return D >= 16 ? 2 : 1; }
inline int default_bwd_np(int D) { return D >= 32 ? 2 : (D >= 16 ? 4 : 1); }

// Builds the table from host cameras; returns false on invalid input.
bool make_view_table(const gs_camera *cams, int n_views, int64_t n, ViewTable *vt);
bool make_params(const gs_raster_params *p, Params *out);
// With GS_JACOBIAN_EXACT, opens the Jacobian's clamp interval of every view to the whole line.
void apply_jacobian_mode(const Params &prm, ViewTable *vt);

__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int gt) {
    int v = 0;
    while (v + 1 < vt.n_views && gt >= vt.tile_off[v + 1]) ++v;
    return v;
}

__device__ __forceinline__ int view_of_pixel(const ViewTable &vt, int64_t pix) {
    int v = 0;
    while (v + 1 < vt.n_views && pix >= vt.pix_off[v + 1]) ++v;
    return v;
}

// Loads row-major world->camera rows 0..2, from device poses when given.
__device__ __forceinline__ void load_pose(const ViewTable &vt, const float *pose_dev, int v,
                                          float R[9], float t[3]) {
    if (pose_dev) {
        const float *P = pose_dev + 16 * v;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R[3 * r] = P[4 * r]; R[3 * r + 1] = P[4 * r + 1]; R[3 * r + 2] = P[4 * r + 2];
            t[r] = P[4 * r + 3];
        }
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R[3 * r] = vt.T[v][4 * r]; R[3 * r + 1] = vt.T[v][4 * r + 1];
            R[3 * r + 2] = vt.T[v][4 * r + 2]; t[r] = vt.T[v][4 * r + 3];
        }
    }
}

// 2^x on the special-function unit (PTX ex2.approx.ftz.f32; relative error
// about 2^-22).  e^p is evaluated as 2^(p log2 e) with the log2 e factor
// folded into the stored conic.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Error-free transformations (Dekker, Knuth; Ogita-Rump-Oishi compensated dot):
// a*b = p + e and a+b = s + e exactly, with explicitly rounded operations so
// the compiler cannot contract or reassociate them.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// r0 x0 + r1 x1 + r2 x2 + t as an unevaluated sum hi + lo (compensated dot
// product: as accurate as a twice-precision evaluation rounded at the end).
__device__ __forceinline__ void dot3_dd(float r0, float r1, float r2, float x0, float x1, float x2, float t,
                                        float &hi, float &lo) {
    float p, s, h, e, q;
    two_prod(r0, x0, p, s);
    two_prod(r1, x1, h, e);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, e));
    two_prod(r2, x2, h, e);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, e));
    two_sum(p, t, p, q);
    s = __fadd_rn(s, q);
    two_sum(p, s, hi, lo);
}

// f (xh + xl) / (zh + zl) + c as an unevaluated sum hi + lo.
__device__ __forceinline__ void proj_dd(float f, float xh, float xl, float zh, float zl, float c, float &hi,
                                        float &lo) {
    float q1 = __fdiv_rn(xh, zh);
    float ph, pe;
    two_prod(q1, zh, ph, pe);
    float r = __fadd_rn(__fsub_rn(__fsub_rn(xh, ph), pe), __fsub_rn(xl, __fmul_rn(q1, zl)));
    float q2 = __fdiv_rn(r, zh);
    float h, e, s, e2;
    two_prod(f, q1, h, e);
    e = __fmaf_rn(f, q2, e);
    two_sum(h, c, s, e2);
    two_sum(s, __fadd_rn(e, e2), hi, lo);
}

// Splat record staged in shared memory for the blend loops.  The centre is the
// unevaluated sum (u + ulo, v + vlo); the conic is kept pre-scaled:
// (qa, qb, qc) = (-A/2, -B, -C/2) * log2 e, so that
// power2 = qa dx^2 + qb dx dy + qc dy^2 = power * log2 e and G = 2^power2.
struct SplatGeo {
    float u, v, ulo, vlo;
    float qa, qb, qc, o;
};

// Evaluates one (pixel, splat) pair.  Both blend kernels call this one
// function, written with explicitly rounded operations so that forward and
// backward take bit-identical skip / clamp decisions.
struct PairEval {
    float dx, dy, G, oG, alpha;
    bool skip;
};

__device__ __forceinline__ PairEval eval_pair(const SplatGeo &s, float pxc, float pyc,
                                              float alpha_min, float alpha_max) {
    PairEval e;
    e.dx = __fsub_rn(__fsub_rn(pxc, s.u), s.ulo);
    e.dy = __fsub_rn(__fsub_rn(pyc, s.v), s.vlo);
    float t = __fmaf_rn(s.qa, e.dx, __fmul_rn(s.qb, e.dy));
    float p2 = __fmaf_rn(t, e.dx, __fmul_rn(__fmul_rn(s.qc, e.dy), e.dy));
    e.G = ex2_approx(p2);
    e.oG = __fmul_rn(s.o, e.G);
    e.alpha = fminf(alpha_max, e.oG);
    e.skip = (p2 > 0.f) || (e.alpha < alpha_min);
    return e;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Asynchronous global -> shared copies (cp.async; 4, 8 or 16 bytes, both addresses aligned to
// the size).  A thread's copies are grouped by cp_async_commit(); cp_async_wait<N>() waits
// until at most N of its groups are still in flight (its own copies only: a warp then needs a
// __syncwarp before its lanes read each other's).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Relaxed device-scope load / store (flags of the chained scans).
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

template <typename T> __device__ __forceinline__ float to_f32(T x);
template <> __device__ __forceinline__ float to_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f32<__half>(__half x) { return __half2float(x); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 x) {
    return __bfloat162float(x);
}

// Exact tile rectangle of a splat (half-open, in tiles): floor((u - r)/16) is
// floordiv(floor(u) - r, 16) because r is an integer.
__device__ __forceinline__ void tile_rect(float u, float v, int r, int TX, int TY, int &x0, int &y0,
                                          int &x1, int &y1) {
    const float lim = 1099511627776.0f;  // 2^40
    float fu = fminf(fmaxf(floorf(u), -lim), lim), fv = fminf(fmaxf(floorf(v), -lim), lim);
    long long iu = (long long)fu, iv = (long long)fv;
    auto fdiv = [](long long a) -> long long { return a >= 0 ? a / kTile : -((-a + kTile - 1) / kTile); };
    auto cl = [](long long a, long long hi) -> int { return (int)(a < 0 ? 0 : (a > hi ? hi : a)); };
    x0 = cl(fdiv(iu - r), TX);
    y0 = cl(fdiv(iv - r), TY);
    x1 = cl(fdiv(iu + r) + 1, TX);
    y1 = cl(fdiv(iv + r) + 1, TY);
}

// Programmatic dependent launch: a kernel launched with launch_pdl may start (be scheduled,
// run its prologue) while the kernel before it on the stream finishes; pdl_wait() blocks until
// that kernel has completed and its writes are visible, so every read of its results comes
// after it.  pdl_trigger() lets the next kernel be launched once every block of this one has
// called it (or exited).  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Shared-memory mbarriers (CTA scope): init with the number of arrivals a phase takes, arrive
// (release), and a test whether the phase of the given parity has completed (acquire); the
// caller bounds its polls.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Host helpers.
// A named NVTX range for the duration of an entry point: a profiler's timeline shows each
// call around its launches (nvtx3 is header-only; without a tool attached the calls cost a
// few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define GS_NVTX_RANGE(name) ::gs::NvtxRange gs_nvtx_range_(name)

// The CUDA error behind this host thread's last GS_ERR_CUDA from cuda_status (gs_cuda_error).
extern thread_local cudaError_t g_last_cuda_error;
inline gs_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GS_OK;
    g_last_cuda_error = e;
    return GS_ERR_CUDA;
}

// Launches kernel<<<grid, block, smem, st>>>(args...) with programmatic stream serialization
// (the kernel must call pdl_wait() before it reads what earlier work on the stream wrote).
template <typename... KArgs, typename... Args>
gs_status launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cuda_status(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}
inline gs_status last_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline bool feat_dim_ok(int d) { return d == 0 || d == 4 || d == 8 || d == 16 || d == 32; }

// Workspace layout shared by the entry points (offsets in bytes, 256-aligned).
struct WsLayout {
    // bin_sort
    size_t scan_blocks;   // u32 [scan block sums], two levels
    size_t emit_sums;     // u32 [emission blocks + 1]: instances per 256 depth-sorted items, then their offsets
    size_t counters;      // u32 [16]: n_vis, M (clamped), tile counters ...
    size_t dkeys_a, dvals_a, dkeys_b, dvals_b;  // u32 [VN]
    size_t tkeys_a, tkeys_b, tvals_b;           // u32 [capacity]
    size_t hist;          // u32 [8 passes][256]
    size_t lookback;      // u32 [8 passes][max tiles][256]
    size_t tile_counts;   // u32 [total image tiles]: instances per image tile
    size_t bin_end;
    // loss / dsr
    size_t med_hist;      // u32 [4][V][256]
    size_t loss_part_f;   // f32 [kLossBlocks][32 * 32 + 32] decoder-gradient partials
    size_t loss_part_d;   // f64 [kLossBlocks + SSIM tiles][3] loss-term partials
    size_t ssim_maps;     // f32 [9 P] SSIM window partials (3 planes per channel)
    size_t expand_counts; // u32 [2][views x 256-pixel blocks] expansion counts and offsets
    size_t dsr_part;      // f64 [512][6] DSR partials, then two u32 arrival counters
    size_t misc_end;
    size_t total;
    int64_t vn, capacity;
    int lb_tiles_depth, lb_tiles_inst;
};

constexpr int kLossBlocks = 1024;
// Depth-sort passes run blocks of 256 threads with 4 keys each up to kSortSmallItems (view,
// Gaussian) items, so that the visible items of a frame or two still spread over every SM (one
// 1M-Gaussian frame: 184k visible items, 180 blocks instead of 90: binning 0.159 -> 0.150 ms), and 8
// keys each above, where the larger blocks are faster (8 frames: 0.662 against 0.692 ms).
constexpr int kSortThreads = 256;       // threads of a depth-sort pass block
constexpr int64_t kSortSmallItems = (int64_t)1 << 21;
constexpr int kSortIPTSmall = 4, kSortIPTLarge = 8;  // keys per thread of a depth-sort pass
inline int depth_sort_tile(int64_t vn) { return kSortThreads * (vn <= kSortSmallItems ? kSortIPTSmall : kSortIPTLarge); }
constexpr int kSortThreadsInst = 1024;  // threads of a tile-sort pass block
constexpr int kSortIPTInst = 8;         // keys per thread of a tile-sort pass
constexpr int kSortTileInst = kSortThreadsInst * kSortIPTInst;
constexpr int kScanIPT = 8;
constexpr int kScanBlock = 256 * kScanIPT;

// Workspace layout; vt (may be NULL) adds the per-pixel space of the SSIM term.
WsLayout ws_layout(int64_t n, int n_views, int64_t capacity, const ViewTable *vt = nullptr);

// 256-pixel blocks per view row of the expansion grid (the largest view's count).
inline int expand_blocks_x(const ViewTable &vt) {
    int64_t m = 0;
    for (int v = 0; v < vt.n_views; ++v) m = std::max<int64_t>(m, (int64_t)vt.W[v] * vt.H[v]);
    return (int)std::max<int64_t>(1, (m + 255) / 256);
}

// SSIM term of the mapping colour loss (ssim.cu).
int ssim_blocks(const ViewTable &vt);
gs_status launch_ssim(const ViewTable &vt, float coef, const float *rgb, const float *trgb, float *maps,
                      double *part, float *g_rgb, cudaStream_t st);

}  // namespace gs
