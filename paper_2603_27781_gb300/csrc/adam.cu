// Mapping update: one bias-corrected Adam step of every parameter group of the field
// with the per-group learning rates of supplementary C.1.  One launch walks all six
// groups as 4-element chunks (float4 loads and stores where the arrays allow);
// 28 bytes per parameter (read p, g, m, v; write p, m, v), an HBM-bound pass.
#include "common.cuh"

namespace gs {
namespace {

constexpr int kGroups = 6;

struct AdamGroups {
    float *p[kGroups];
    const float *g[kGroups];
    float *m[kGroups], *v[kGroups];
    int64_t count[kGroups];
    int64_t chunk_off[kGroups + 1];  // first 4-element chunk of each group
    float lr[kGroups];
};

// Decay factors in f32 and their complements formed in double: 1 - 0.999f in f32 is
// off by 1.3e-5 relative, so c1 = 1 - b1, c2 = 1 - b2 come from the double betas.
struct AdamCoef {
    float b1, b2, c1, c2, eps;
    double b1d, b2d;        // for the bias corrections of a device-counted step
    double bc1, bc2;        // bias corrections of a host-numbered step
};

__global__ void adam_count_kernel(double *ctr) { *ctr += 1.0; }

__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float lr, const AdamCoef &k,
                                         float bc1, float bc2) {
    m = fmaf(k.b1, m, k.c1 * g);
    v = fmaf(k.b2, v, k.c2 * g * g);
    p -= lr * (m / bc1) / (sqrtf(v / bc2) + k.eps);
}

__global__ void __launch_bounds__(256) adam_kernel(AdamGroups G, AdamCoef K, const double *ctr) {
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) {
        double bc1 = K.bc1, bc2 = K.bc2;
        if (ctr) {  // device step count, already incremented for this step
            const double step = *ctr;
            bc1 = 1.0 - pow(K.b1d, step);
            bc2 = 1.0 - pow(K.b2d, step);
        }
        s_bc[0] = (float)bc1;
        s_bc[1] = (float)bc2;
    }
    __syncthreads();
    const float bc1 = s_bc[0], bc2 = s_bc[1];
    const int64_t total = G.chunk_off[kGroups];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < kGroups && c >= G.chunk_off[k + 1]) ++k;
        const int64_t e0 = 4 * (c - G.chunk_off[k]);
        const int n = (int)min((int64_t)4, G.count[k] - e0);
        float *p = G.p[k] + e0, *m = G.m[k] + e0, *v = G.v[k] + e0;
        const float *g = G.g[k] + e0;
        const float lr = G.lr[k];
        const bool vec = n == 4 && ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                                     reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
        if (vec) {
            float4 P = *reinterpret_cast<float4 *>(p), M = *reinterpret_cast<float4 *>(m);
            float4 V = *reinterpret_cast<float4 *>(v);
            const float4 Gr = *reinterpret_cast<const float4 *>(g);
            adam_one(P.x, Gr.x, M.x, V.x, lr, K, bc1, bc2);
            adam_one(P.y, Gr.y, M.y, V.y, lr, K, bc1, bc2);
            adam_one(P.z, Gr.z, M.z, V.z, lr, K, bc1, bc2);
            adam_one(P.w, Gr.w, M.w, V.w, lr, K, bc1, bc2);
            *reinterpret_cast<float4 *>(p) = P;
            *reinterpret_cast<float4 *>(m) = M;
            *reinterpret_cast<float4 *>(v) = V;
        } else {
            for (int j = 0; j < n; ++j) adam_one(p[j], g[j], m[j], v[j], lr, K, bc1, bc2);
        }
    }
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_adam_step(const gs_field_mut *f, const gs_gaussian_grads *grads, float *moments, int step,
                                  double *step_ctr, const float *lr, double beta1, double beta2, double eps,
                                  gs_stream stream) {
    GS_NVTX_RANGE("gs_adam_step");
    using namespace gs;
    if (!f || !grads || !lr || f->n < 0 || step < 0 || (step == 0 && !step_ctr)) return GS_ERR_ARG;
    if (!(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps >= 0.0)) return GS_ERR_ARG;
    if (!feat_dim_ok(f->feat_dim)) return GS_ERR_UNSUPPORTED;
    if (f->n == 0) return GS_OK;
    if (!moments || !f->means || !f->quats || !f->log_scales || !f->opacity_logits || !f->rgb ||
        (f->feat_dim && !f->feat) || !grads->means || !grads->quats || !grads->log_scales ||
        !grads->opacity_logits || !grads->rgb || (f->feat_dim && !grads->feat))
        return GS_ERR_ARG;
    const int64_t n = f->n;
    const int width[kGroups] = {3, 4, 3, 1, 3, f->feat_dim};
    float *ps[kGroups] = {f->means, f->quats, f->log_scales, f->opacity_logits, f->rgb, f->feat};
    const float *gr[kGroups] = {grads->means, grads->quats, grads->log_scales, grads->opacity_logits, grads->rgb,
                                grads->feat};
    const int64_t M = n * (14 + f->feat_dim);
    AdamGroups G;
    int64_t off = 0;
    G.chunk_off[0] = 0;
    for (int k = 0; k < kGroups; ++k) {
        G.p[k] = ps[k];
        G.g[k] = gr[k];
        G.m[k] = moments + off;
        G.v[k] = moments + M + off;
        G.count[k] = n * width[k];
        G.lr[k] = lr[k];
        G.chunk_off[k + 1] = G.chunk_off[k] + (G.count[k] + 3) / 4;
        off += G.count[k];
    }
    AdamCoef K;
    K.b1 = (float)beta1;
    K.b2 = (float)beta2;
    K.c1 = (float)(1.0 - beta1);
    K.c2 = (float)(1.0 - beta2);
    K.eps = (float)eps;
    K.b1d = beta1;
    K.b2d = beta2;
    K.bc1 = step ? 1.0 - pow(beta1, step) : 0.0;
    K.bc2 = step ? 1.0 - pow(beta2, step) : 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    if (step == 0) adam_count_kernel<<<1, 1, 0, st>>>(step_ctr);
    const int64_t chunks = G.chunk_off[kGroups];
    const int grid = (int)std::min<int64_t>((chunks + 255) / 256, 152 * 16);
    adam_kernel<<<grid, 256, 0, st>>>(G, K, step ? nullptr : step_ctr);
    return last_launch();
}
