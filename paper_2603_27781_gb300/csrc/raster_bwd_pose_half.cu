// Per-group blend backward kernels, pose-only mode, f16 colour and bf16 feature storage.
#include "raster_bwd_warp.cuh"

namespace gs {
gs_status dispatch_bwd_warp_pose_half(int D, int np, const ViewTable &vt, const Params &prm, const BwdArgs &A,
                                      cudaStream_t st) {
    return dispatch_bwd_warp_typed<false, __half, __nv_bfloat16>(D, np, vt, prm, A, st);
}
}  // namespace gs
