// Blend backward kernels for gradients of the Gaussian parameters (map mode), f32 storage;
// the half-storage per-group kernels are in raster_bwd_map_half.cu.
#include "raster_bwd_warp.cuh"

namespace gs {
gs_status dispatch_bwd_map(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                           cudaStream_t st) {
    if (prm.bwd_warp)
        return half ? dispatch_bwd_warp_map_half(D, np, vt, prm, A, st)
                    : dispatch_bwd_warp_typed<true, float, float>(D, np, vt, prm, A, st);
    return dispatch_bwd<true>(D, np, half, vt, prm, A, st);
}
}  // namespace gs
