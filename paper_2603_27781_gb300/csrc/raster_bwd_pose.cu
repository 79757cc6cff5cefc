// Blend backward kernels for the pose gradient only (tracking mode: no colour or
// feature gradients are reduced), f32 storage; the half-storage per-group kernels are in
// raster_bwd_pose_half.cu.
#include "raster_bwd_warp.cuh"

namespace gs {
gs_status dispatch_bwd_pose(int D, int np, bool half, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                            cudaStream_t st) {
    if (prm.bwd_warp)
        return half ? dispatch_bwd_warp_pose_half(D, np, vt, prm, A, st)
                    : dispatch_bwd_warp_typed<false, float, float>(D, np, vt, prm, A, st);
    return dispatch_bwd<false>(D, np, half, vt, prm, A, st);
}
}  // namespace gs
