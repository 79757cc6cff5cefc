/*
 * libgs — C ABI of the GB300 (sm_103a) semantic-splatting rasterizer.
 *
 * The library computes the differentiable splatting renderer of a Semantic
 * Gaussian Field (GS3LAM, Sec. 3.2): projection of 3D Gaussians through a
 * pinhole camera with EWA 2D covariances, binning into 16x16 tiles with a
 * (tile | depth) sort, front-to-back alpha blending of colour, depth,
 * D-dimensional semantic feature and silhouette, the tracking and mapping
 * losses, and the backward pass to every Gaussian parameter and to the camera
 * pose as an SE(3) twist (supplementary B.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every data pointer is DEVICE memory owned by the caller unless the
 *    argument says "host".  The library never allocates device memory; the
 *    scratch it needs is a caller-provided workspace sized by
 *    gs_workspace_size().
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) and never synchronise the device, so they can be
 *    captured in a CUDA graph.  Host-side argument errors return before any
 *    launch; launch failures return GS_ERR_CUDA.  Conditions only the device
 *    can see (instance overflow, a bounded wait that gave up) set a device
 *    status word (gs_binning.status) that the caller reads after the stream
 *    completes.  Nothing crosses the ABI as an exception, and the library
 *    never exits, aborts or traps.
 *  - Cameras and parameters are host structs copied into kernel arguments at
 *    call time.
 *  - Items: with V views and N Gaussians the projected records are indexed by
 *    item = view * N + gaussian.  Tiles of view v are numbered after all tiles
 *    of views 0..v-1; images of view v occupy pixels [pix_off(v), pix_off(v) +
 *    W_v H_v) of every planar channel, pix_off(v) = sum of earlier W H.
 *  - Gradient outputs are overwritten by each call unless documented "+=".
 *    With several views, per-Gaussian gradients are summed over the views.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *gs_stream; /* cudaStream_t */

typedef enum {
    GS_OK = 0,
    GS_ERR_ARG = -1,         /* invalid argument (null pointer, bad size, bad enum) */
    GS_ERR_CAPACITY = -2,    /* more tile instances than gs_binning.capacity */
    GS_ERR_CUDA = -3,        /* a CUDA runtime call or launch failed */
    GS_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    GS_ERR_UNSUPPORTED = -5, /* valid but not built (feature dim, tile size, dtype) */
    GS_ERR_CHECK = -6        /* a library built with GS_CHECKS=1 found an index out of range */
} gs_status;

typedef enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype;

/* gs_render_bwd modes (bit set).  GS3LAM optimises poses and the field
 * separately (Sec. 3.2.3): tracking needs only the pose twist, mapping only
 * the Gaussian parameters.  GS_GRAD_ACCUMULATE (with either): gs_render_bwd
 * adds to sg and d_feat as they are instead of first setting them to zero, for
 * a caller that cleared them beforehand with gs_splat_grads_clear (on another
 * stream, say, beside the forward blend). */
enum { GS_GRAD_MAP = 1, GS_GRAD_POSE = 2, GS_GRAD_ACCUMULATE = 4 };

/* Pinhole camera.  T_cw is the row-major 4x4 world-to-camera transform
 * (Sec. 3.2.1), OpenCV axes: x right, y down, z forward.  Pixel (x, y) samples
 * the point (x + 0.5, y + 0.5). */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float T_cw[16];
} gs_camera;

/* Raster parameters the paper leaves open (defaults in parentheses).
 * tile: tile edge in pixels (16; the only size built).  A splat is skipped at a
 * pixel where alpha < alpha_min (1/255), alpha is clamped to alpha_max (0.99),
 * and a pixel stops blending before the splat that would take its
 * transmittance below T_min (1e-4).  Gaussians with camera z <= z_near (0.2)
 * are culled; lowpass (0.3 px^2) is added to the diagonal of Sigma2D; the
 * splat radius is ceil(radius_sigma (3) * sqrt(lambda_max(Sigma2D))).
 * bg_rgb is the colour behind the last splat (0,0,0). */
typedef struct {
    int32_t tile;
    float alpha_min, alpha_max, T_min, z_near, lowpass, radius_sigma;
    float bg_rgb[3];
    /* Launch shape of the blend kernels (results do not depend on it): pixels
     * per thread of gs_render_fwd / gs_render_bwd, 1, 2 or 4 (2 and 4 only for
     * feature dims 16 and 32; 4 only up to 16); 0 = the library's default. */
    int32_t fwd_px_per_thread, bwd_px_per_thread;
    /* Block shape of gs_render_bwd (results do not depend on it beyond the
     * order of float atomics): GS_BWD_BLOCKS_GROUP = one 32-thread block per
     * 8x4 pixel group (bwd_px_per_thread 1, or 2 for 16x4 bands; 0 means 2 at
     * feature dim 16, else 1),
     * each adding its own sums with atomics, for feature dims 16 and 32 with
     * the forward's blend mask (else GS_ERR_UNSUPPORTED); GS_BWD_BLOCKS_TILE =
     * one block per 16x16 tile whose warps combine each splat's sums in shared
     * memory; GS_BWD_BLOCKS_DEFAULT (0) = per pixel group where that form
     * applies, else per tile. */
    int32_t bwd_blocks;
    /* Block shape of gs_render_fwd (images identical either way; the blend mask
     * too): GS_BWD_BLOCKS_GROUP = one 32-thread block per pixel group
     * (fwd_px_per_thread 1 or 2), which leaves as soon as its pixels are done;
     * GS_BWD_BLOCKS_TILE = one block per tile; GS_BLOCKS_QUEUE = one block per
     * tile's worth of threads, but only as many blocks as are resident on the
     * GPU at once, each taking tiles (in the tile order) from the work counters
     * gs_binning.queue, which must then not be NULL (else GS_ERR_ARG), until
     * none is left; GS_BLOCKS_RING = one block per tile whose warps stage the
     * tile's splats into a ring of batch slots and walk them each at its own
     * pace (two pixels per thread, feature dims 16 and 32, else
     * GS_ERR_UNSUPPORTED; fwd_batch 128 gives two slots of 128 splats, 64 four
     * slots of 64 at dim 16 and three at dim 32); GS_BWD_BLOCKS_DEFAULT (0) = the
     * library's choice for the launch shape. */
    int32_t fwd_blocks;
    /* Where the EWA Jacobian J of Eq. 3 is evaluated (gs_project, gs_project_bwd):
     * GS_JACOBIAN_CLAMPED (0, the default) at (x/z, y/z) clamped to the view
     * widened by 15% of its size per side (the 3DGS rasterizer convention: a
     * Gaussian far outside the view keeps the footprint it would have at that
     * boundary; the clamped coordinate has zero derivative), GS_JACOBIAN_EXACT
     * (1) at (x/z, y/z) itself, the literal perspective Jacobian.  Other values
     * return GS_ERR_ARG. */
    int32_t jacobian;
    /* Bounded device-side waits (the look-back of gs_bin_sort's radix passes): a
     * wait gives up after this many polls of a flag another block has not yet
     * published, sets GS_ERR_TIMEOUT in the status word and lets the call finish
     * without reading what it waited for.  0 = the library default (2^22 polls,
     * about 0.3 s); negative = a block gives up at the first earlier block it
     * looks at (a test hook: gs_bin_sort then reports GS_ERR_TIMEOUT whenever a
     * radix pass has more than one block of keys: 1,024 visible items per depth
     * pass block up to 2^21 (view, Gaussian) items and 2,048 above, 8,192
     * instances per tile pass block; and a GS_BLOCKS_RING
     * forward whenever one of its warps has to wait for another). */
    int32_t spin_limit;
    /* Splats the per-tile forward (fwd_blocks GS_BWD_BLOCKS_TILE or
     * GS_BLOCKS_QUEUE) stages in shared memory per round: 64, 128 or 256
     * (0 = 128); other values return GS_ERR_ARG.  64 is built for two pixels
     * per thread at feature dims 16 and 32, 256 for two pixels per thread at
     * feature dim 16 (else GS_ERR_UNSUPPORTED).
     * Results do not depend on it. */
    int32_t fwd_batch;
} gs_raster_params;

enum { GS_BWD_BLOCKS_DEFAULT = 0, GS_BWD_BLOCKS_GROUP = 1, GS_BWD_BLOCKS_TILE = 2, GS_BLOCKS_QUEUE = 3, GS_BLOCKS_RING = 4 };
enum { GS_JACOBIAN_CLAMPED = 0, GS_JACOBIAN_EXACT = 1 };

/* The Semantic Gaussian Field of Eq. 1, structure of arrays.
 *   means [n,3], quats [n,4] (w,x,y,z; normalised inside), log_scales [n,3]
 *   (Eq. 2: S = diag(exp(log_s))), opacity_logits [n] (o = sigmoid), all f32;
 *   rgb [n,3] in rgb_dtype (F32 or F16), feat [n,feat_dim] in feat_dtype (F32
 *   or BF16).  feat_dim is one of 0, 4, 8, 16, 32; feat may be NULL when 0. */
typedef struct {
    int64_t n;
    int32_t feat_dim;
    const float *means;
    const float *quats;
    const float *log_scales;
    const float *opacity_logits;
    const void *rgb;
    int32_t rgb_dtype;
    const void *feat;
    int32_t feat_dtype;
} gs_gaussians;

/* Projected splats, one record per item (16-byte aligned arrays):
 *   uvdo[4*item]  = (u, v, depth, opacity): centre g_i (supp. B.1), camera-frame
 *                   depth d_i (Eq. 6) and the activated opacity o_i (Eq. 5);
 *   uv_lo[2*item] = (u - u_f32, v - v_f32): the centre is carried as an
 *                   unevaluated f32 sum (hi in uvdo, lo here) because a pixel
 *                   coordinate near 1000 has an f32 spacing of 6e-5 px;
 *   conic[4*item] = (A, B, C, radius): Sigma2D^-1 = [[A, B], [B, C]] (Eq. 3, 5)
 *                   and the integer pixel radius stored as a float;
 *   tiles_touched[item] = tiles covered (0 = culled).  Binning uses the f32
 *   centre uvdo.xy. */
typedef struct {
    float *uvdo;
    float *uv_lo;
    float *conic;
    int32_t *tiles_touched;
} gs_projected;

/* Tile binning.  keys[j] = (tile << 32) | bits(depth as float32) of sorted
 * instance j (may be NULL if not wanted), vals[j] = its item; ranges[2t],
 * ranges[2t+1] = [start, end) of tile t; n_inst = instance count (device
 * int64); status = device word, 0 or a negative gs_status.  capacity bounds
 * keys/vals.  tile_order (optional, device u32 [total tiles]): a permutation
 * of the tiles by decreasing instance count (order within equal counts
 * unspecified), in which gs_render_fwd / gs_render_bwd launch their tiles
 * when it is not NULL; gs_bin_sort writes it whenever it is not NULL.
 * queue (optional, device u32 [2]): the work counters of the GS_BLOCKS_QUEUE
 * forward; gs_bin_sort sets them to 0 whenever queue is not NULL, and every
 * such launch leaves them 0 when it completes, so launches may repeat.  Two
 * launches that share a queue must not overlap on the GPU. */
typedef struct {
    int64_t capacity;
    uint64_t *keys;
    uint32_t *vals;
    uint32_t *ranges;
    int64_t *n_inst;
    int32_t *status;
    uint32_t *tile_order;
    uint32_t *queue;
} gs_binning;

/* Rendered images, planar f32 over all views' pixels (P = sum W H):
 * rgb [3,P], depth [P], sil [P] (cumulative opacity, Eq. 10), feat [D,P],
 * T_final [P] (transmittance after the last blended splat), n_contrib [P]
 * (1-based position in the tile list of the last blended splat) and, if not
 * NULL, n_blended [P] (number of splats blended into the pixel) and
 * blend_mask: u32 [8][capacity / 32 + 1] bit planes, one per 8x4 pixel group
 * g = (y % 16 / 4) * 2 + (x % 16 / 8) of a tile, bit i of plane g set when a
 * pixel of that group of instance i's tile blended instance i.  gs_render_bwd
 * uses the mask, when given, to skip instances no pixel of a group blended. */
typedef struct {
    float *rgb;
    float *depth;
    float *sil;
    float *feat;
    float *T_final;
    int32_t *n_contrib;
    int32_t *n_blended;
    uint32_t *blend_mask;
} gs_images;

/* Gradients of the loss w.r.t. the rendered images, same layout as gs_images.
 * sil may be NULL (treated as zero).
 * Factored feature gradient (optional): with feat_basis not NULL, the gradient of
 * the features is feat_basis^T feat_coef, feat_basis being device f32
 * [feat_rank, D] (the weights of a linear decoder, Eq. 8) and feat_coef device f32
 * [feat_rank, P] planes (the gradient w.r.t. the decoder's logits, as
 * gs_loss_fwd_bwd writes it), and feat is ignored.  gs_render_bwd then evaluates
 * the K-term products and multiplies by feat_basis^T once per splat: the same
 * gradient in fewer operations when feat_rank < D.  Supported by the per-group
 * backward (feature dims 16 and 32 with the blend mask) for feat_rank <= 8, else
 * GS_ERR_UNSUPPORTED.  feat_basis NULL: the fields after feat are not read. */
typedef struct {
    const float *rgb;
    const float *depth;
    const float *sil;
    const float *feat;
    const float *feat_coef;
    const float *feat_basis;
    int32_t feat_rank;
} gs_image_grads;

/* Writable image gradients produced by gs_loss_fwd_bwd.  feat_coef (optional,
 * device f32 [K, P]): if not NULL, the loss writes the gradient w.r.t. the
 * decoder's logits there (the factored form of gs_image_grads, with the decoder
 * weights as the basis) and does not write feat, which may then be NULL. */
typedef struct {
    float *rgb;
    float *depth;
    float *sil;
    float *feat;
    float *feat_coef;
} gs_image_grads_out;

/* Gradients w.r.t. the gs_gaussians parameters, all f32, same shapes. */
typedef struct {
    float *means;
    float *quats;
    float *log_scales;
    float *opacity_logits;
    float *rgb;
    float *feat;
} gs_gaussian_grads;

/* Writable view of the field's FP32 parameter arrays (same shapes as
 * gs_gaussians), for the mapping update. */
typedef struct {
    int64_t n;
    int32_t feat_dim;
    float *means;
    float *quats;
    float *log_scales;
    float *opacity_logits;
    float *rgb;
    float *feat;
} gs_field_mut;

/* Targets of the losses, planar over all views' pixels: rgb [3,P] f32,
 * depth [P] f32 (<= 0: no measurement), label [P] u8 (255: unlabelled). */
typedef struct {
    const float *rgb;
    const float *depth;
    const uint8_t *label;
} gs_targets;

/* Loss weights and mode.  mask_mode 0 = mapping (Eq. 18 without the DSR
 * terms), 1 = tracking (Eq. 21 with the M_obs mask, tau_obs threshold on the
 * silhouette).  n_classes = K of the linear decoder (<= 32).  ssim = lambda
 * of Eq. 15 in [0, 1] (mapping only; the paper uses 0.2): the colour term
 * becomes color ((1 - lambda) L1 + lambda (1 - SSIM)), SSIM over an 11x11
 * Gaussian window (sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2)
 * averaged over the view's 3 P_v channel-pixels; 0 leaves the L1 term alone. */
typedef struct {
    float color, depth, sem;
    int32_t mask_mode;
    float tau_obs;
    int32_t n_classes;
    float ssim;
} gs_loss_params;

/* Library version (major * 10000 + minor * 100 + patch). */
int gs_version(void);

/* Human-readable text of a status code (static storage). */
const char *gs_strerror(int status);

/* Text of the CUDA runtime error behind the calling host thread's last
 * GS_ERR_CUDA from a failed CUDA call ("no error" if there was none; static
 * storage). */
const char *gs_cuda_error(void);

/* Bytes of workspace needed by gs_bin_sort, gs_loss_fwd_bwd and gs_dsr for n
 * Gaussians, n_views host cameras, an instance capacity and a
 * feature dimension.  One buffer of this size serves all of them in stream
 * order.  Must be 256-byte aligned.  Returns 0 on invalid arguments. */
size_t gs_workspace_size(int64_t n, int n_views, const gs_camera *cams, int64_t inst_capacity,
                         int feat_dim);

/* Projection (Eq. 2, 3; supp. B.1).  For every view and Gaussian: quaternion
 * and scale to Sigma, camera-frame centre p = R_cw mu + t_cw, pinhole centre
 * (u, v) = (fx x/z + cx, fy y/z + cy), Sigma2D = J R_cw Sigma R_cw^T J^T +
 * lowpass I, its inverse (in f64 when near singular), the radius and the number
 * of tiles it covers.  The depth is computed as the f32 fused chain
 * fma(r20, x, fma(r21, y, fma(r22, z, t_z))); the centre (u, v) is computed
 * with compensated (double-f32) arithmetic.  pose_dev, if not NULL, is a
 * device f32 [n_views,16] array of world-to-camera transforms that replaces
 * cams[v].T_cw (for device-resident poses); intrinsics always come from cams.
 * out arrays hold n_views * n items. */
gs_status gs_project(const gs_gaussians *g, const gs_camera *cams, int n_views,
                     const float *pose_dev, const gs_raster_params *p, gs_projected *out,
                     gs_stream stream);

/* Binning and depth sort (Sec. 3.2.1: "sorting the Gaussians in depth order";
 * tile-based rasterisation).  Emits one instance per (item, covered tile) and
 * orders instances by (tile, f32 depth bits, item), i.e. a stable sort by the
 * 64-bit key (tile << 32 | depth bits) of items listed in index order.  Writes
 * ranges for every tile (empty tiles get [0,0)), n_inst, and keys if non-NULL.
 * If the count exceeds out->capacity, *out->status = GS_ERR_CAPACITY and the
 * binning is incomplete (its required size is still written to n_inst).  If a
 * bounded wait gives up, *out->status = GS_ERR_TIMEOUT.  Once the status word is
 * set, the remaining binning kernels skip their work (ranges stay empty), and
 * gs_render_fwd / gs_render_bwd given that binning render nothing: images,
 * blend mask contents beyond their clearing, and gradients beyond their zeroing
 * are left as they were.
 * ws: workspace of ws_bytes >= gs_workspace_size(...). */
gs_status gs_bin_sort(int64_t n, const gs_projected *proj, const gs_camera *cams, int n_views,
                      const gs_raster_params *p, void *ws, size_t ws_bytes, gs_binning *out,
                      gs_stream stream);

/* Forward blend (Eq. 4-7, 10).  One thread per pixel walks its tile's
 * instances front to back: alpha = min(alpha_max, o exp(-1/2 s^T Sigma2D^-1 s))
 * (Eq. 5), skip below alpha_min, stop before T drops below T_min, accumulate
 * w = alpha T times colour, depth, feature and 1.  rgb gets + T_final * bg. */
gs_status gs_render_fwd(const gs_gaussians *g, const gs_projected *proj, const gs_binning *bins,
                        const gs_camera *cams, int n_views, const gs_raster_params *p,
                        gs_images *out, gs_stream stream);

/* Per-splat gradients of the blend, written by gs_render_bwd and consumed by
 * gs_project_bwd (device f32, 16-byte aligned):
 *   uvod[4*item]  = dL/du, dL/dv, dL/do (activated opacity), dL/ddepth;
 *   conic[4*item] = dL/dA, dL/dB, dL/dC, 0;
 *   rgb[4*g]      = dL/dc of Gaussian g summed over views, 0 (GS_GRAD_MAP only). */
typedef struct {
    float *uvod;
    float *conic;
    float *rgb;
} gs_splat_grads;

/* Backward of the blend (Eq. 4-7, 10).  Per pixel the blend is walked back to
 * front from n_contrib, recomputing each alpha exactly as the forward did and
 * the transmittance in front of it as T / (1 - alpha) from T_final; with S the
 * blended value behind a splat, d out / d alpha = T (x - S).  Per-splat
 * gradients are reduced across the warp and the CTA before one atomic add per
 * (tile, splat).  Overwrites sg (rgb only with GS_GRAD_MAP) and, with
 * GS_GRAD_MAP, d_feat (f32 [n, feat_dim], summed over views); adds to them
 * with GS_GRAD_ACCUMULATE.  fwd must be the
 * gs_render_fwd output of the same inputs (T_final, n_contrib are read). */
gs_status gs_render_bwd(const gs_gaussians *g, const gs_projected *proj, const gs_binning *bins,
                        const gs_camera *cams, int n_views, const gs_raster_params *p, int grad_mode,
                        const gs_images *fwd, const gs_image_grads *dL, gs_splat_grads *sg, float *d_feat,
                        gs_stream stream);

/* Sets to zero what gs_render_bwd with the same g, n_views and grad_mode
 * (GS_GRAD_MAP and/or GS_GRAD_POSE) accumulates into: sg->uvod and sg->conic
 * (n_views * g->n float4 each) and, with GS_GRAD_MAP, sg->rgb (g->n float4)
 * and d_feat (g->n * feat_dim f32; may be NULL when feat_dim is 0).  Device
 * buffers, 16-byte aligned, owned by the caller; asynchronous on stream.
 * Returns GS_ERR_ARG for a bad mode, a NULL or misaligned buffer. */
gs_status gs_splat_grads_clear(const gs_gaussians *g, int n_views, int grad_mode, gs_splat_grads *sg,
                               float *d_feat, gs_stream stream);

/* Backward of the projection (chain rule of supp. B.1, per factor): from the
 * per-splat gradients to the 3D parameters, summed over views.  GS_GRAD_MAP
 * writes out->means, quats, log_scales, opacity_logits and rgb (out->feat is
 * not touched: gs_render_bwd wrote it).  GS_GRAD_POSE writes pose_part, a
 * device f32 [n_views, 6, n] array of per-Gaussian contributions to the
 * gradient of the left twist (rho, phi): rho gets g_p, phi gets
 * p x g_p + 2 (A12, A20, A01) with A = Sc Gc - Gc Sc, g_p and Gc being the
 * gradients w.r.t. the camera-frame centre and covariance Sc.  pose_dev as for
 * gs_project. */
gs_status gs_project_bwd(const gs_gaussians *g, const gs_camera *cams, int n_views, const float *pose_dev,
                         const gs_raster_params *p, int grad_mode, const gs_splat_grads *sg,
                         gs_gaussian_grads *out, float *pose_part, gs_stream stream);

/* Pose twist gradient (supp. B.1), reduced in double precision:
 * d_twist[6 v + k] = sum over Gaussians of pose_part[v, k, :], k = rho_x,
 * rho_y, rho_z, phi_x, phi_y, phi_z, for the left perturbation
 * T(xi) = Exp(xi) T_cw at xi = 0.  d_twist: device f64 [6 n_views]. */
gs_status gs_pose_grad(int64_t n, int n_views, const float *pose_part, double *d_twist,
                       gs_stream stream);

/* Decoder and losses (Eq. 8, 15-17, 21) with their gradients.  Per view v
 * with P_v pixels: logits z = W f + b (W: dec_W [K,D] f32, b: dec_b [K]);
 * L_v = (color sum |c - c_gt|_1 + depth sum_{d_gt>0} |d - d_gt| +
 * sem sum_{label != 255} (logsumexp z - z_label)) / P_v (with the SSIM term of
 * gs_loss_params.ssim in the colour part), times M_obs in
 * tracking mode (sil > tau_obs, d_gt > 0, |d - d_gt| < 10 x the lower median
 * of |d - d_gt| over the view's pixels with d_gt > 0).  Writes grad (all four
 * images; sil gradient is zero), d_dec_W, d_dec_b (overwritten), loss_out
 * (device f64 [4]: total, colour, depth, semantic summed over views),
 * mask_out (optional device f32 [P]) and median_out (optional device f32
 * [n_views]). */
gs_status gs_loss_fwd_bwd(const gs_camera *cams, int n_views, int feat_dim, const gs_images *img,
                          const gs_targets *tgt, const float *dec_W, const float *dec_b,
                          const gs_loss_params *lp, void *ws, size_t ws_bytes,
                          gs_image_grads_out *grad, float *d_dec_W, float *d_dec_b,
                          double *loss_out, float *mask_out, float *median_out, gs_stream stream);

/* Allocation-free variant of gs_loss_fwd_bwd, for callers that cannot call
 * cudaMalloc: code that must not allocate while a CUDA graph is being captured
 * or inside a per-frame real-time budget, plugins whose host application owns
 * every device allocation, and bindings from environments without a device
 * allocator.  The paper has no counterpart; it is a deployment convenience.
 * Arguments and results are those of gs_loss_fwd_bwd without the workspace,
 * with two limits: at most 16 views, and no SSIM term (lp->ssim must be 0; a
 * nonzero value in [0, 1] returns GS_ERR_UNSUPPORTED, a value outside it or a
 * nonzero one in tracking mode GS_ERR_ARG).  Every argument is checked before
 * anything is launched.  Its scratch is one static device array of 4,415,488
 * bytes (4.2 MiB) that every GPU which loads the library holds until the
 * process exits.  The array's device address is looked up (cudaGetSymbolAddress,
 * with the device current) on each call made outside a stream capture; a call
 * inside a capture reuses the address of the device's last call outside one, so
 * make a first call on each device before any stream capture, and again after
 * the device's context has been reset (cudaDeviceReset) before capturing.  All
 * calls share the one array: calls that overlap on the GPU (concurrent streams,
 * or host threads using the same device) race and must be serialised by the
 * caller.  The call allocates nothing and frees nothing. */
gs_status gs_loss_fwd_bwd_noalloc(const gs_camera *cams, int n_views, int feat_dim, const gs_images *img,
                                  const gs_targets *tgt, const float *dec_W, const float *dec_b,
                                  const gs_loss_params *lp, gs_image_grads_out *grad, float *d_dec_W,
                                  float *d_dec_b, double *loss_out, float *mask_out, float *median_out,
                                  gs_stream stream);

/* Depth-adaptive scale regularisation (Eq. 12) over the 3n axis scales
 * s = exp(log_scales): mu, sigma = population mean and deviation (constants
 * for differentiation), L_big = mean of s > mu + 2 sigma, L_small = mean of
 * -log s < mu - 2 sigma.  Adds lam_big * dL_big + lam_small * dL_small to
 * d_log_scales (+=).  out: device f64 [8] = (lam_big L_big + lam_small
 * L_small, mu, sigma, n_big, n_small, L_big, L_small, 0). */
gs_status gs_dsr(int64_t n, const float *log_scales, float lam_big, float lam_small, void *ws,
                 size_t ws_bytes, float *d_log_scales, double *out, gs_stream stream);

/* The two halves of gs_dsr, so that the value (two reductions over the scales,
 * which need only log_scales) can run on another stream beside the rest of a
 * step and only the gradient waits for the projection backward.
 * gs_dsr_value writes out exactly as gs_dsr does, with its partial sums in
 * scratch: device memory of GS_DSR_SCRATCH_BYTES bytes, 256-byte aligned, used
 * by one call at a time (it need not be the workspace, so the call may overlap
 * gs_bin_sort and gs_loss_fwd_bwd).  gs_dsr_grad then adds lam_big * dL_big +
 * lam_small * dL_small to d_log_scales (+=) from that out, after gs_dsr_value
 * has completed (stream order or an event).  n = 0: gs_dsr_value writes zeros,
 * gs_dsr_grad does nothing.  GS_ERR_ARG for a missing buffer or n < 0. */
#define GS_DSR_SCRATCH_BYTES 24832
gs_status gs_dsr_value(int64_t n, const float *log_scales, float lam_big, float lam_small, void *scratch,
                       double *out, gs_stream stream);
gs_status gs_dsr_grad(int64_t n, const float *log_scales, float lam_big, float lam_small, const double *out,
                      float *d_log_scales, gs_stream stream);

/* Pose step for tracking (Sec. 3.4; learning rates of supp. C.1): Adam on
 * the left twist of each view, then T <- Exp(delta) T.  T_state: device f64
 * [n_views,16] (updated); adam: device f64 [n_views,12] (m, v; zero before
 * step 1); lr: host [6] (rho, phi); step: 1-based.  step = 0 keeps the count
 * on the device instead: adam then holds n_views*12 + 1 doubles, the last one
 * the number of steps taken (zero before the first), which the call reads and
 * increments, so that a captured CUDA graph can replay the step.  If pose_f32
 * is not NULL it receives the f32 copy of the new poses (for gs_project's
 * pose_dev).  GS_ERR_ARG for step < 0 or a missing buffer. */
gs_status gs_pose_step(int n_views, const double *d_twist, double *T_state, double *adam,
                       int step, const double *lr, double beta1, double beta2, double eps,
                       float *pose_f32, gs_stream stream);

/* Mapping update (Sec. 3.3; learning rates of supp. C.1, which names no
 * optimiser: read as Adam with bias correction, as for the pose): for every
 * parameter p of the groups means, quats, log_scales, opacity_logits, rgb,
 * feat (in this order), m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr_group (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), in f32 with
 * 1 - b1, 1 - b2 and the bias corrections formed in double.  f: the field,
 * updated in place (f32 storage only); grads: the gradients of the step
 * (gs_render_bwd / gs_project_bwd / gs_dsr); moments: device f32
 * [2][n (14 + feat_dim)], m then v, each the six groups back to back (zero
 * before the first step); lr: host [6] in group order (C.1: 1e-4, 1e-3, 1e-3,
 * 0.05, 2.5e-3, 2.5e-3).  step >= 1 is the 1-based step t; step 0 keeps t on
 * the device in *step_ctr (f64, zero before the first step), which the call
 * increments, so that a captured CUDA graph can replay the update.
 * GS_ERR_ARG for a missing buffer, step < 0 or betas outside [0, 1). */
gs_status gs_adam_step(const gs_field_mut *f, const gs_gaussian_grads *grads, float *moments, int step,
                       double *step_ctr, const float *lr, double beta1, double beta2, double eps,
                       gs_stream stream);

/* Adaptive Gaussian expansion (Eq. 11 and the initialisation that follows it
 * in Sec. 3.3).  Per view, M_unobs = (sil < tau_unobs) or (depth > d_gt and
 * |d_gt - depth| > 50 x median) on pixels with d_gt > 0, where median is the
 * lower median of |depth - d_gt| over the view's pixels with d_gt > 0 and
 * sil, depth are the rendered images (img->sil, img->depth).  One Gaussian is
 * appended per masked pixel, pixels in raster order and views in order: mean =
 * the pixel centre unprojected at d_gt into the world frame, rotation identity,
 * log-scale log(d_gt / fx) on every axis, opacity 0.5 (logit 0), colour =
 * tgt->rgb at the pixel, features = row k of feat_init (device f32
 * [field->n - n_existing, feat_dim], values the caller draws) for the k-th new
 * Gaussian.  field: arrays of field->n rows; rows [0, n_existing) are kept and
 * the new ones written from row n_existing.  n_new (device int64) receives the
 * number of masked pixels; if it exceeds field->n - n_existing only that many
 * are written and *status (device) becomes GS_ERR_CAPACITY (else 0).  src_pix
 * (optional device int64 [field->n - n_existing]) receives each new Gaussian's
 * pixel index (pix_off(v) + y W + x).  ws: the workspace of gs_workspace_size
 * for these cameras.  GS_ERR_ARG for missing buffers or n_existing outside
 * [0, field->n]. */
gs_status gs_expand(const gs_camera *cams, int n_views, const gs_images *img, const gs_targets *tgt,
                    float tau_unobs, const float *feat_init, int64_t n_existing, gs_field_mut *field,
                    int64_t *n_new, int64_t *src_pix, int32_t *status, void *ws, size_t ws_bytes,
                    gs_stream stream);

/* Keyframe store of one camera's frames (device memory, caller-owned), slot
 * s holding: rgb[s] [3,P] f32, depth[s] [P] f32, label[s] [P] u8 (planar, the
 * layout of gs_targets) and T_cw[s] [16] f64 (the frame's estimated
 * world-to-camera pose, row-major). */
typedef struct {
    int32_t capacity;
    int64_t P;
    const float *rgb;
    const float *depth;
    const uint8_t *label;
    const double *T_cw;
} gs_keyframes;

/* RSKM keyframe draw (Eq. 13, Sec. 3.3) for one mapping iteration.  The
 * candidates are the keyframe set K = slots [0, n_kf) together with the
 * current frame f_cur = cur_slot (0 <= cur_slot <= n_kf: either a stored
 * keyframe or the slot after them), |K u {f_cur}| = max(n_kf, cur_slot + 1)
 * candidates in slot order.  With k the mapping iteration counter state[0]
 * (device int32, set to 0 before a frame's first iteration): if k mod t_opt
 * is 0 the draw is f_cur (Eq. 13 gives it probability 1 there), otherwise
 * candidate draws[k mod n_draws] mod |K u {f_cur}| (a uniform draw; draws:
 * device u32 random words the caller supplies, n_draws >= 1).  The call writes
 * the slot to state[1] and to picked[k] (optional, device int32 [n_draws],
 * for k < n_draws), increments state[0], copies the slot's observation into
 * out_rgb [3,P], out_depth [P], out_label [P] (device) and its pose, rounded
 * to f32, into pose_f32 [16] (optional; gs_project's pose_dev).  The counter
 * and slot live on the device, so a captured CUDA graph replays the draw.
 * GS_ERR_ARG for a missing buffer, t_opt < 1 or slots outside the store. */
gs_status gs_rskm_draw(const gs_keyframes *kf, int32_t n_kf, int32_t cur_slot, int32_t t_opt,
                       const uint32_t *draws, int64_t n_draws, int32_t *state, int32_t *picked,
                       float *out_rgb, float *out_depth, uint8_t *out_label, float *pose_f32,
                       gs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
