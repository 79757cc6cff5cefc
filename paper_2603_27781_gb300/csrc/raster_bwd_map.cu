// Blend backward kernels for gradients of the Gaussian parameters (map mode).
#include "raster_bwd_warp.cuh"

namespace gs {
gs_status dispatch_bwd_map(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                           cudaStream_t st) {
    if (prm.bwd_warp) return dispatch_bwd_warp<true>(D, np, half, vt, prm, A, st);
    return dispatch_bwd<true>(D, np, half, vt, prm, A, st);
}
}  // namespace gs
