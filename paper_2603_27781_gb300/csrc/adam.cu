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

// One 4-element chunk of a group: where it is, how many elements, and whether its four
// arrays allow float4 access.
struct Chunk {
    float *p, *m, *v;
    const float *g;
    float lr;
    int n;
    bool vec;
};

__device__ __forceinline__ Chunk locate(const AdamGroups &G, int64_t c) {
    int k = 0;
    while (k + 1 < kGroups && c >= G.chunk_off[k + 1]) ++k;
    const int64_t e0 = 4 * (c - G.chunk_off[k]);
    Chunk r;
    r.n = (int)min((int64_t)4, G.count[k] - e0);
    r.p = G.p[k] + e0;
    r.m = G.m[k] + e0;
    r.v = G.v[k] + e0;
    r.g = G.g[k] + e0;
    r.lr = G.lr[k];
    r.vec = r.n == 4 && ((reinterpret_cast<uintptr_t>(r.p) | reinterpret_cast<uintptr_t>(r.g) |
                          reinterpret_cast<uintptr_t>(r.m) | reinterpret_cast<uintptr_t>(r.v)) & 15) == 0;
    return r;
}

__device__ __forceinline__ void load4(const Chunk &a, float4 &P, float4 &M, float4 &V, float4 &Gr) {
    P = *reinterpret_cast<const float4 *>(a.p);
    M = *reinterpret_cast<const float4 *>(a.m);
    V = *reinterpret_cast<const float4 *>(a.v);
    Gr = *reinterpret_cast<const float4 *>(a.g);
}

// The update of a chunk: from the loaded float4s, or element by element when not vec.
__device__ __forceinline__ void update(const Chunk &a, float4 &P, float4 &M, float4 &V, const float4 &Gr,
                                       const AdamCoef &K, float bc1, float bc2) {
    if (a.vec) {
        adam_one(P.x, Gr.x, M.x, V.x, a.lr, K, bc1, bc2);
        adam_one(P.y, Gr.y, M.y, V.y, a.lr, K, bc1, bc2);
        adam_one(P.z, Gr.z, M.z, V.z, a.lr, K, bc1, bc2);
        adam_one(P.w, Gr.w, M.w, V.w, a.lr, K, bc1, bc2);
        *reinterpret_cast<float4 *>(a.p) = P;
        *reinterpret_cast<float4 *>(a.m) = M;
        *reinterpret_cast<float4 *>(a.v) = V;
    } else {
        for (int j = 0; j < a.n; ++j) adam_one(a.p[j], a.g[j], a.m[j], a.v[j], a.lr, K, bc1, bc2);
    }
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
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // two chunks per iteration, c and c + stride, with their loads issued before either update
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += 2 * stride) {
        Chunk a = locate(G, c), b = locate(G, c + stride < total ? c + stride : c);
        const bool two = c + stride < total;
        float4 Pa, Ma, Va, Ga, Pb, Mb, Vb, Gb;
        if (a.vec) load4(a, Pa, Ma, Va, Ga);
        if (two && b.vec) load4(b, Pb, Mb, Vb, Gb);
        update(a, Pa, Ma, Va, Ga, K, bc1, bc2);
        if (two) update(b, Pb, Mb, Vb, Gb, K, bc1, bc2);
    }
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_adam_step(const gs_field_mut *f, const gs_gaussian_grads *grads, float *moments, int step,
                                  double *step_ctr, const float *lr, double beta1, double beta2, double eps,
                                  gs_stream stream) {
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
