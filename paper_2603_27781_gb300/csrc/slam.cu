// RSKM keyframe draw (Eq. 13) and the gather of the drawn frame's observation.
//
// The keyframes' observations stay resident in HBM (a 1200x680 frame is 13.9 MB:
// rgb 3P + depth P floats, label P bytes), so a mapping iteration needs no host
// transfer: a one-thread kernel takes the draw from the device iteration counter
// and the caller's random words, and a grid copies the drawn slot into the
// buffers the loss reads, with its pose for the projection.  Both read the
// counter and the slot from device memory, so a captured graph replays the draw.
#include "common.cuh"

namespace gs {
namespace {

struct DrawArgs {
    const double *T_cw;
    int32_t n_cand, cur_slot, t_opt;
    const uint32_t *draws;
    int64_t n_draws;
    int32_t *state;
    int32_t *picked;
    float *pose_f32;
};

// Eq. 13: on every t_opt-th mapping iteration (k = 0, t_opt, 2 t_opt, ...) the current
// frame; otherwise a frame drawn uniformly from the candidates.
__global__ void rskm_select_kernel(DrawArgs a) {
    const int32_t k = a.state[0];
    int32_t slot;
    if (k % a.t_opt == 0) {
        slot = a.cur_slot;
    } else {
        const uint32_t r = a.draws[(int64_t)k % a.n_draws];
        slot = (int32_t)(r % (uint32_t)a.n_cand);
    }
    a.state[1] = slot;
    if (a.picked && k < a.n_draws) a.picked[k] = slot;
    a.state[0] = k + 1;
    if (a.pose_f32)
        for (int i = 0; i < 16; ++i) a.pose_f32[i] = (float)a.T_cw[(int64_t)slot * 16 + i];
}

struct GatherArgs {
    const float *rgb, *depth;
    const uint8_t *label;
    int64_t P;
    const int32_t *state;
    float *out_rgb, *out_depth;
    uint8_t *out_label;
    bool vec;  // every plane starts on a 16-byte boundary and P % 16 == 0
};

__global__ void __launch_bounds__(256) rskm_gather_kernel(GatherArgs a) {
    const int64_t slot = a.state[1];
    const int64_t P = a.P;
    const float *src_rgb = a.rgb + slot * 3 * P, *src_d = a.depth + slot * P;
    const uint8_t *src_l = a.label + slot * P;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a.vec) {
        // 4 floats of rgb and depth per thread step, 16 label bytes per thread step
        const float4 *sr = reinterpret_cast<const float4 *>(src_rgb);
        const float4 *sd = reinterpret_cast<const float4 *>(src_d);
        float4 *dr = reinterpret_cast<float4 *>(a.out_rgb);
        float4 *dd = reinterpret_cast<float4 *>(a.out_depth);
        const int64_t n_rgb = 3 * P / 4, n_d = P / 4;
        for (int64_t i = t0; i < n_rgb; i += stride) dr[i] = sr[i];
        for (int64_t i = t0; i < n_d; i += stride) dd[i] = sd[i];
        const uint4 *sl = reinterpret_cast<const uint4 *>(src_l);
        uint4 *dl = reinterpret_cast<uint4 *>(a.out_label);
        for (int64_t i = t0; i < P / 16; i += stride) dl[i] = sl[i];
    } else {
        for (int64_t i = t0; i < 3 * P; i += stride) a.out_rgb[i] = src_rgb[i];
        for (int64_t i = t0; i < P; i += stride) {
            a.out_depth[i] = src_d[i];
            a.out_label[i] = src_l[i];
        }
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_rskm_draw(const gs_keyframes *kf, int32_t n_kf, int32_t cur_slot, int32_t t_opt,
                                  const uint32_t *draws, int64_t n_draws, int32_t *state, int32_t *picked,
                                  float *out_rgb, float *out_depth, uint8_t *out_label, float *pose_f32,
                                  gs_stream stream) {
    GS_NVTX_RANGE("gs_rskm_draw");
    if (!kf || !kf->rgb || !kf->depth || !kf->label || !kf->T_cw || kf->P <= 0 || kf->capacity <= 0)
        return GS_ERR_ARG;
    if (n_kf < 0 || n_kf > kf->capacity || cur_slot < 0 || cur_slot > n_kf || cur_slot >= kf->capacity)
        return GS_ERR_ARG;
    if (t_opt < 1 || !draws || n_draws < 1 || !state || !out_rgb || !out_depth || !out_label) return GS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    DrawArgs d;
    d.T_cw = kf->T_cw;
    d.n_cand = std::max(n_kf, cur_slot + 1);
    d.cur_slot = cur_slot;
    d.t_opt = t_opt;
    d.draws = draws;
    d.n_draws = n_draws;
    d.state = state;
    d.picked = picked;
    d.pose_f32 = pose_f32;
    rskm_select_kernel<<<1, 1, 0, st>>>(d);
    const gs_status s = last_launch();
    if (s) return s;
    GatherArgs g;
    g.rgb = kf->rgb;
    g.depth = kf->depth;
    g.label = kf->label;
    g.P = kf->P;
    g.state = state;
    g.out_rgb = out_rgb;
    g.out_depth = out_depth;
    g.out_label = out_label;
    g.vec = kf->P % 16 == 0 && aligned16(kf->rgb) && aligned16(kf->depth) && aligned16(kf->label) &&
            aligned16(out_rgb) && aligned16(out_depth) && aligned16(out_label);
    const int64_t work = g.vec ? 3 * kf->P / 4 : 3 * kf->P;
    const int grid = (int)std::min<int64_t>((work + 255) / 256, 152 * 8);
    rskm_gather_kernel<<<grid, 256, 0, st>>>(g);
    return last_launch();
}
