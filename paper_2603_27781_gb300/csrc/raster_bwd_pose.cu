// Blend backward kernels for the pose gradient only (tracking mode: no colour or
// feature gradients are reduced).
#include "raster_bwd_warp.cuh"

namespace gs {
gs_status dispatch_bwd_pose(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                            cudaStream_t st) {
    if (prm.bwd_warp) return dispatch_bwd_warp<false>(D, np, half, vt, prm, A, st);
    return dispatch_bwd<false>(D, np, half, vt, prm, A, st);
}
}  // namespace gs
