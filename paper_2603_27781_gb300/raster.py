"""Torch-side driver of libgs: device buffers, one fwd+bwd iteration, autograd.

PyTorch provides device memory and the stream; every step of the rasterizer
runs in the CUDA library through the C ABI (`_lib`).  Nothing here computes
any part of the method.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L


@dataclasses.dataclass
class RasterParams:
    """Raster parameters the paper leaves open (see include/gs.h)."""
    tile: int = 16
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    z_near: float = 0.2
    lowpass: float = 0.3
    radius_sigma: float = 3.0
    bg: tuple = (0.0, 0.0, 0.0)
    fwd_px_per_thread: int = 0     # launch shape only (0 = library default)
    bwd_px_per_thread: int = 0
    bwd_blocks: int = 0            # backward block shape (0 default, 1 per pixel group, 2 per tile)
    fwd_blocks: int = 0            # forward block shape (same values, and 3 resident blocks on a tile queue)
    exact_jacobian: bool = False   # J of Eq. 3 at the unclamped (x/z, y/z) (GS_JACOBIAN_EXACT)
    spin_limit: int = 0            # polls of a bounded wait (0 library default; < 0 give up at once)
    fwd_batch: int = 0             # splats staged per round by the per-tile forward (64, 128, 256; 0 = 128)

    def c(self) -> L.gs_raster_params:
        return L.gs_raster_params(self.tile, self.alpha_min, self.alpha_max, self.T_min, self.z_near, self.lowpass,
                                  self.radius_sigma, (ctypes.c_float * 3)(*self.bg), self.fwd_px_per_thread,
                                  self.bwd_px_per_thread, self.bwd_blocks, self.fwd_blocks,
                                  L.GS_JACOBIAN_EXACT if self.exact_jacobian else L.GS_JACOBIAN_CLAMPED,
                                  self.spin_limit, self.fwd_batch)


@dataclasses.dataclass
class LossWeights:
    """Loss weights of supplementary C.1 (mapping defaults) and the tracking mask switch."""
    color: float = 0.5
    depth: float = 1.0
    sem: float = 0.01
    big: float = 0.01
    small: float = 0.001
    mask_mode: int = 0
    tau_obs: float = 0.99
    ssim: float = 0.0      # lambda of Eq. 15 (mapping colour: (1 - lambda) L1 + lambda (1 - SSIM))


MAPPING = LossWeights()
MAPPING_SSIM = LossWeights(ssim=0.2)      # Eq. 15 with the paper's lambda = 0.2
TRACKING = LossWeights(color=0.5, depth=1.0, sem=0.001, big=0.0, small=0.0, mask_mode=1)
# supplementary C.1: pose learning rates, translation (rho) then rotation (phi)
TRACKING_LR = (2e-3, 2e-3, 2e-3, 4e-4, 4e-4, 4e-4)


def camera_c(cam) -> L.gs_camera:
    T = [float(x) for x in torch.as_tensor(cam.T_cw, dtype=torch.float64).reshape(16).tolist()]
    return L.gs_camera(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                       (ctypes.c_float * 16)(*T))


def cameras_c(cams) -> ctypes.Array:
    arr = (L.gs_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_c(c)
    return arr


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_DTYPE = {torch.float32: L.GS_F32, torch.float16: L.GS_F16, torch.bfloat16: L.GS_BF16}

# largest decoder class count of the factored feature gradient (gs_image_grads.feat_rank)
FACTOR_K = 8


@dataclasses.dataclass
class Field:
    """Semantic Gaussian field on the device (Eq. 1), structure of arrays."""
    means: torch.Tensor
    quats: torch.Tensor
    log_scales: torch.Tensor
    opacity_logits: torch.Tensor
    rgb: torch.Tensor
    feat: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def feat_dim(self) -> int:
        return int(self.feat.shape[1])

    @staticmethod
    def from_numpy(gs, device="cuda", rgb_dtype=torch.float32, feat_dtype=torch.float32) -> "Field":
        t = lambda a, dt=torch.float32: torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
        return Field(t(gs.means), t(gs.quats), t(gs.log_scales), t(gs.opacity_logits), t(gs.rgb, rgb_dtype),
                     t(gs.feat, feat_dtype))

    def c(self) -> L.gs_gaussians:
        return L.gs_gaussians(self.n, self.feat_dim, _p(self.means), _p(self.quats), _p(self.log_scales),
                              _p(self.opacity_logits), _p(self.rgb), _DTYPE[self.rgb.dtype],
                              _p(self.feat) if self.feat_dim else None, _DTYPE[self.feat.dtype])


class Renderer:
    """Device buffers for rendering a field of n Gaussians into a fixed set of views.

    One instance serves repeated iterations (and CUDA-graph capture): every
    buffer is allocated here, once.  `capacity` bounds the (tile, splat)
    instances; `status()` reports an overflow after the stream has run.
    """

    def __init__(self, n: int, cams: Sequence, feat_dim: int, capacity: int, device="cuda",
                 params: RasterParams = RasterParams(), n_classes: int = 0):
        self.n, self.feat_dim, self.capacity = int(n), int(feat_dim), int(capacity)
        self.n_cap = self.n            # Gaussians the per-Gaussian buffers hold (set_n picks n <= n_cap)
        self.params = params
        self.device = torch.device(device)
        self.set_cameras(cams)
        V, dev = self.n_views, self.device
        f32, i32 = torch.float32, torch.int32
        self.uvdo = torch.zeros(V * n, 4, dtype=f32, device=dev)
        self.uv_lo = torch.zeros(V * n, 2, dtype=f32, device=dev)
        self.conic = torch.zeros(V * n, 4, dtype=f32, device=dev)
        self.touched = torch.zeros(V * n, dtype=i32, device=dev)
        self.keys = torch.zeros(max(capacity, 1), dtype=torch.int64, device=dev)
        self.vals = torch.zeros(max(capacity, 1), dtype=i32, device=dev)
        self.ranges = torch.zeros(2 * self.n_tiles, dtype=i32, device=dev)
        self.tile_order = torch.zeros(max(self.n_tiles, 1), dtype=i32, device=dev)
        self.use_tile_order = True      # blend tiles launched longest first
        self.queue = torch.zeros(2, dtype=i32, device=dev)  # work counters of the queued forward
        self.n_inst = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status_word = torch.zeros(1, dtype=i32, device=dev)
        ws_bytes = L.library().gs_workspace_size(n, V, self.cams_c, capacity, feat_dim)
        if ws_bytes == 0:
            raise ValueError("invalid renderer configuration (workspace size 0)")
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        P, D = self.P, feat_dim
        self.img_rgb = torch.zeros(3, P, dtype=f32, device=dev)
        self.img_depth = torch.zeros(P, dtype=f32, device=dev)
        self.img_sil = torch.zeros(P, dtype=f32, device=dev)
        self.img_feat = torch.zeros(max(D, 1), P, dtype=f32, device=dev)
        self.img_T = torch.zeros(P, dtype=f32, device=dev)
        self.img_nc = torch.zeros(P, dtype=i32, device=dev)
        self.img_nb = torch.zeros(P, dtype=i32, device=dev)
        self.count_blended = False
        self.blend_mask = torch.zeros(8 * (max(capacity, 1) // 32 + 1), dtype=i32, device=dev)
        self.use_blend_mask = True
        self.sg_uvod = torch.zeros(V * n, 4, dtype=f32, device=dev)
        self.sg_conic = torch.zeros(V * n, 4, dtype=f32, device=dev)
        self.sg_rgb = torch.zeros(n, 4, dtype=f32, device=dev)
        self.g_rgb = torch.zeros(3, P, dtype=f32, device=dev)
        self.g_depth = torch.zeros(P, dtype=f32, device=dev)
        self.g_sil = torch.zeros(P, dtype=f32, device=dev)
        self.g_feat = torch.zeros(max(D, 1), P, dtype=f32, device=dev)
        self.d_means = torch.zeros(n, 3, dtype=f32, device=dev)
        self.d_quats = torch.zeros(n, 4, dtype=f32, device=dev)
        self.d_log_scales = torch.zeros(n, 3, dtype=f32, device=dev)
        self.d_logits = torch.zeros(n, dtype=f32, device=dev)
        self.d_rgb = torch.zeros(n, 3, dtype=f32, device=dev)
        self.d_feat = torch.zeros(n, max(D, 1), dtype=f32, device=dev)
        self.pose_part = torch.zeros(V, 6, n, dtype=f32, device=dev)
        self.d_twist = torch.zeros(V, 6, dtype=torch.float64, device=dev)
        self.loss_out = torch.zeros(4, dtype=torch.float64, device=dev)
        self.dsr_out = torch.zeros(8, dtype=torch.float64, device=dev)
        self.dsr_scratch = torch.empty(L.GS_DSR_SCRATCH_BYTES, dtype=torch.uint8, device=dev)
        self.mask = torch.zeros(P, dtype=f32, device=dev)
        self.median = torch.zeros(V, dtype=f32, device=dev)
        K = max(int(n_classes), 1)
        self.d_dec_W = torch.zeros(K, max(D, 1), dtype=f32, device=dev)
        self.d_dec_b = torch.zeros(K, dtype=f32, device=dev)
        # factored feature gradient (gs_image_grads.feat_basis): the loss writes dL/dz of the decoder's
        # K <= 8 logits and the per-group backward contracts those, for feature widths 16 and 32
        self.factored = D in (16, 32) and 1 <= int(n_classes) <= FACTOR_K
        self.g_coef = torch.zeros(FACTOR_K, P, dtype=f32, device=dev) if self.factored else None
        self._basis = None             # decoder weights of the last factored loss
        self.prm_c = params.c()

    OUTPUTS = ("d_means", "d_quats", "d_log_scales", "d_logits", "d_rgb", "d_feat", "d_dec_W", "d_dec_b",
               "d_twist", "loss_out", "dsr_out")

    def output_set(self) -> dict:
        """A new set of the step's result tensors (gradients, losses) shaped like the bound one."""
        return {k: torch.zeros_like(getattr(self, k)) for k in self.OUTPUTS}

    def bind_outputs(self, outs: dict):
        """Makes the following calls write their results into `outs` (an output_set())."""
        for k, t in outs.items():
            setattr(self, k, t)

    def set_n(self, n: int):
        """Serves a field of n <= n_cap Gaussians with the buffers already allocated (every
        per-Gaussian buffer keeps its n_cap rows; the calls use the first n)."""
        if not 0 <= n <= self.n_cap:
            raise ValueError(f"field of {n} Gaussians exceeds the renderer's {self.n_cap}")
        self.n = int(n)

    def ensure_capacity(self, need: int, growth: float = 1.5):
        """Grows the instance capacity (keys, values, blend mask, workspace) to hold `need`
        (tile, splat) instances; a no-op when it already does."""
        if need <= self.capacity:
            return
        cap = int(max(need, self.capacity * growth))
        dev = self.device
        self.capacity = cap
        self.keys = torch.zeros(cap, dtype=torch.int64, device=dev)
        self.vals = torch.zeros(cap, dtype=torch.int32, device=dev)
        self.blend_mask = torch.zeros(8 * (cap // 32 + 1), dtype=torch.int32, device=dev)
        ws_bytes = L.library().gs_workspace_size(self.n_cap, self.n_views, self.cams_c, cap, self.feat_dim)
        if ws_bytes == 0:
            raise ValueError("invalid renderer configuration (workspace size 0)")
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)

    def instances_needed(self, field: Field, pose_dev: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Projects the field and returns the (tile, splat) instance count on the device."""
        self.project(field, pose_dev)
        return self.touched[: self.n_views * field.n].sum(dtype=torch.int64)

    # ------------------------------------------------------------ geometry
    def set_cameras(self, cams):
        self.cams = list(cams)
        self.n_views = len(self.cams)
        self.cams_c = cameras_c(self.cams)
        self.sizes = [(int(c.height), int(c.width)) for c in self.cams]
        self.P = sum(h * w for h, w in self.sizes)
        self.pix_off = [0]
        for h, w in self.sizes:
            self.pix_off.append(self.pix_off[-1] + h * w)
        t = 16
        self.n_tiles = sum(((h + t - 1) // t) * ((w + t - 1) // t) for h, w in self.sizes)

    # -------------------------------------------------------------- C ABI
    def projected_c(self):
        return L.gs_projected(_p(self.uvdo), _p(self.uv_lo), _p(self.conic), _p(self.touched))

    def binning_c(self, want_keys=False):
        return L.gs_binning(self.capacity, _p(self.keys) if want_keys else None, _p(self.vals), _p(self.ranges),
                            _p(self.n_inst), _p(self.status_word),
                            _p(self.tile_order) if self.use_tile_order else None, _p(self.queue))

    def images_c(self):
        return L.gs_images(_p(self.img_rgb), _p(self.img_depth), _p(self.img_sil),
                           _p(self.img_feat) if self.feat_dim else None, _p(self.img_T), _p(self.img_nc),
                           _p(self.img_nb) if self.count_blended else None,
                           _p(self.blend_mask) if self.use_blend_mask else None)

    def splat_grads_c(self):
        return L.gs_splat_grads(_p(self.sg_uvod), _p(self.sg_conic), _p(self.sg_rgb))

    def image_grads_c(self, factored=False):
        """The image gradients for gs_render_bwd; factored: the decoder-logit form the last
        factored loss() wrote (g_feat = W^T g_coef)."""
        if factored:
            W = self._basis
            if W is None:
                raise ValueError("no factored loss has been computed with this renderer")
            return L.gs_image_grads(_p(self.g_rgb), _p(self.g_depth), _p(self.g_sil), None, _p(self.g_coef), _p(W),
                                    int(W.shape[0]))
        return L.gs_image_grads(_p(self.g_rgb), _p(self.g_depth), _p(self.g_sil),
                                _p(self.g_feat) if self.feat_dim else None, None, None, 0)

    def image_grads_out_c(self, factored=False):
        """The image-gradient outputs of gs_loss_fwd_bwd (factored: the logit gradient)."""
        return L.gs_image_grads_out(_p(self.g_rgb), _p(self.g_depth), _p(self.g_sil),
                                    _p(self.g_feat) if self.feat_dim and not factored else None,
                                    _p(self.g_coef) if factored else None)

    def gaussian_grads_c(self):
        return L.gs_gaussian_grads(_p(self.d_means), _p(self.d_quats), _p(self.d_log_scales), _p(self.d_logits),
                                   _p(self.d_rgb), _p(self.d_feat) if self.feat_dim else None)

    def project(self, field: Field, pose_dev: Optional[torch.Tensor] = None, stream=None):
        pc = self.projected_c()
        L.check("gs_project", L.gs_project(ctypes.byref(field.c()), self.cams_c, self.n_views, _p(pose_dev),
                                           ctypes.byref(self.prm_c), ctypes.byref(pc), _stream(stream)))

    def bin_sort(self, want_keys=False, stream=None):
        pc, bc = self.projected_c(), self.binning_c(want_keys)
        L.check("gs_bin_sort", L.gs_bin_sort(self.n, ctypes.byref(pc), self.cams_c, self.n_views,
                                             ctypes.byref(self.prm_c), _p(self.ws), self.ws.numel(),
                                             ctypes.byref(bc), _stream(stream)))

    def render_fwd(self, field: Field, stream=None):
        pc, bc, ic = self.projected_c(), self.binning_c(), self.images_c()
        L.check("gs_render_fwd", L.gs_render_fwd(ctypes.byref(field.c()), ctypes.byref(pc), ctypes.byref(bc),
                                                 self.cams_c, self.n_views, ctypes.byref(self.prm_c),
                                                 ctypes.byref(ic), _stream(stream)))

    def loss(self, targets, decoder_W: torch.Tensor, decoder_b: torch.Tensor, w: LossWeights, stream=None,
             factored=False):
        """Decoder and losses (gs_loss_fwd_bwd).  factored: write the gradient of the decoder's
        logits (g_coef) instead of the features' (needs self.factored), for a following
        render_bwd(factored=True)."""
        K = int(decoder_W.shape[0]) if decoder_W is not None else 0
        if factored:
            if not self.factored or not 1 <= K <= FACTOR_K:
                raise ValueError("the factored feature gradient needs feature width 16 or 32 and 1-8 classes")
            self._basis = decoder_W
        lp = L.gs_loss_params(w.color, w.depth, w.sem, w.mask_mode, w.tau_obs, K, w.ssim)
        tc = L.gs_targets(_p(targets["rgb"]), _p(targets["depth"]), _p(targets["label"]))
        ic, gc = self.images_c(), self.image_grads_out_c(factored)
        L.check("gs_loss_fwd_bwd", L.gs_loss_fwd_bwd(self.cams_c, self.n_views, self.feat_dim, ctypes.byref(ic),
                                                     ctypes.byref(tc), _p(decoder_W), _p(decoder_b),
                                                     ctypes.byref(lp), _p(self.ws), self.ws.numel(),
                                                     ctypes.byref(gc), _p(self.d_dec_W), _p(self.d_dec_b),
                                                     _p(self.loss_out), _p(self.mask), _p(self.median),
                                                     _stream(stream)))

    def render_bwd(self, field: Field, grad_mode: int = L.GS_GRAD_MAP, stream=None, factored=False,
                   accumulate=False):
        """gs_render_bwd; with accumulate, into the splat sums as they are (cleared before by
        clear_grads, possibly on another stream that this one has waited for)."""
        pc, bc, ic, gc, sg = (self.projected_c(), self.binning_c(), self.images_c(), self.image_grads_c(factored),
                              self.splat_grads_c())
        mode = grad_mode | (L.GS_GRAD_ACCUMULATE if accumulate else 0)
        L.check("gs_render_bwd", L.gs_render_bwd(ctypes.byref(field.c()), ctypes.byref(pc), ctypes.byref(bc),
                                                 self.cams_c, self.n_views, ctypes.byref(self.prm_c), mode,
                                                 ctypes.byref(ic), ctypes.byref(gc), ctypes.byref(sg),
                                                 _p(self.d_feat) if self.feat_dim else None, _stream(stream)))

    def clear_grads(self, field: Field, grad_mode: int = L.GS_GRAD_MAP, stream=None):
        """gs_splat_grads_clear: zeroes the splat sums a render_bwd with this mode adds to."""
        sg = self.splat_grads_c()
        L.check("gs_splat_grads_clear", L.gs_splat_grads_clear(ctypes.byref(field.c()), self.n_views, grad_mode,
                                                               ctypes.byref(sg),
                                                               _p(self.d_feat) if self.feat_dim else None,
                                                               _stream(stream)))

    def project_bwd(self, field: Field, grad_mode: int = L.GS_GRAD_MAP, pose_dev=None, stream=None):
        sg, oc = self.splat_grads_c(), self.gaussian_grads_c()
        L.check("gs_project_bwd", L.gs_project_bwd(ctypes.byref(field.c()), self.cams_c, self.n_views,
                                                   _p(pose_dev), ctypes.byref(self.prm_c), grad_mode,
                                                   ctypes.byref(sg), ctypes.byref(oc), _p(self.pose_part),
                                                   _stream(stream)))

    def backward(self, field: Field, grad_mode: int = L.GS_GRAD_MAP, pose_dev=None, stream=None, factored=False):
        """Blend backward then projection backward (and the twist reduction in pose mode)."""
        self.render_bwd(field, grad_mode, stream, factored)
        self.project_bwd(field, grad_mode, pose_dev, stream)
        if grad_mode & L.GS_GRAD_POSE:
            self.pose_grad(stream)

    def pose_grad(self, stream=None):
        L.check("gs_pose_grad", L.gs_pose_grad(self.n, self.n_views, _p(self.pose_part), _p(self.d_twist),
                                               _stream(stream)))

    def dsr(self, field: Field, lam_big: float, lam_small: float, stream=None):
        L.check("gs_dsr", L.gs_dsr(self.n, _p(field.log_scales), lam_big, lam_small, _p(self.ws), self.ws.numel(),
                                   _p(self.d_log_scales), _p(self.dsr_out), _stream(stream)))

    def dsr_value(self, field: Field, lam_big: float, lam_small: float, stream=None):
        """The value of Eq. 12 into dsr_out (gs_dsr_value; its own scratch, so it may run beside
        the binning and the loss on another stream)."""
        L.check("gs_dsr_value", L.gs_dsr_value(self.n, _p(field.log_scales), lam_big, lam_small,
                                               _p(self.dsr_scratch), _p(self.dsr_out), _stream(stream)))

    def dsr_grad(self, field: Field, lam_big: float, lam_small: float, stream=None):
        """Adds the gradient of Eq. 12 from dsr_out to d_log_scales (gs_dsr_grad)."""
        L.check("gs_dsr_grad", L.gs_dsr_grad(self.n, _p(field.log_scales), lam_big, lam_small, _p(self.dsr_out),
                                             _p(self.d_log_scales), _stream(stream)))

    def pose_step(self, T_state, adam, step, lr=TRACKING_LR, b1=0.9, b2=0.999, eps=1e-15, pose_f32=None,
                  stream=None):
        """Adam step on the view twists.  step >= 1 is the 1-based step number; step 0
        keeps the count on the device (adam then holds 12 * n_views + 1 doubles, the
        last one the steps taken so far), which a captured CUDA graph can replay."""
        need = 12 * self.n_views + (1 if step == 0 else 0)
        if adam.numel() < need or adam.dtype != torch.float64:
            raise ValueError(f"adam state needs {need} float64 values")
        lr_c = (ctypes.c_double * 6)(*lr)
        L.check("gs_pose_step", L.gs_pose_step(self.n_views, _p(self.d_twist), _p(T_state), _p(adam), step, lr_c,
                                               b1, b2, eps, _p(pose_f32), _stream(stream)))

    # --------------------------------------------------------- iteration
    def forward(self, field: Field, pose_dev=None, stream=None, want_keys=False):
        self.project(field, pose_dev, stream)
        self.bin_sort(want_keys, stream)
        self.render_fwd(field, stream)

    def iteration(self, field: Field, targets, decoder_W, decoder_b, w: LossWeights, grad_mode=L.GS_GRAD_MAP,
                  pose_dev=None, stream=None):
        """One fwd+bwd pass of the whole path: project, bin/sort, blend, loss, blend and
        projection backward, pose-twist reduction, DSR.  Asynchronous.  On a side stream beside
        the forward half: the clearing of the blend backward's sums and the DSR's value (which
        needs only the log-scales); the blend backward waits for them.  The DSR's gradient runs
        there beside the twist reduction once the projection backward has written the
        log-scale gradient, and the side stream rejoins `stream` before the call returns (also
        inside a CUDA-graph capture)."""
        dsr = (grad_mode & L.GS_GRAD_MAP) and (w.big or w.small)

        def side(s):
            self.clear_grads(field, grad_mode, s)
            if dsr:
                self.dsr_value(field, w.big, w.small, s)
        self.side_start(side, stream)
        self.forward(field, pose_dev, stream)
        fac = self.use_factored(decoder_W)
        self.loss(targets, decoder_W, decoder_b, w, stream, factored=fac)
        self.side_join(stream)
        self.render_bwd(field, grad_mode, stream, factored=fac, accumulate=True)
        self.project_bwd(field, grad_mode, pose_dev, stream)
        if not dsr:
            if grad_mode & L.GS_GRAD_POSE:
                self.pose_grad(stream)
            return
        main = (lambda: self.pose_grad(stream)) if grad_mode & L.GS_GRAD_POSE else (lambda: None)
        self.side_by_side(lambda s: self.dsr_grad(field, w.big, w.small, s), main, stream)

    def use_factored(self, decoder_W) -> bool:
        """Whether a step with this decoder takes the factored feature gradient: the renderer
        supports it, the decoder has 1-8 classes and the per-group backward will run (the
        blend mask is on and the backward block shape is not forced to whole tiles)."""
        K = int(decoder_W.shape[0]) if decoder_W is not None else 0
        return (self.factored and 1 <= K <= FACTOR_K and self.use_blend_mask
                and self.params.bwd_blocks != L.GS_BWD_BLOCKS_TILE and self.params.bwd_px_per_thread <= 2)

    def side_start(self, side_work, stream=None):
        """Runs side_work(side_stream) on the renderer's side stream after everything issued so
        far on `stream`, without waiting for it; a later side_by_side joins it."""
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(self.device)
        self._side.wait_stream(main)
        with torch.cuda.stream(self._side):
            side_work(self._side)

    def side_join(self, stream=None):
        """Makes `stream` wait for everything issued so far on the side stream."""
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        if getattr(self, "_side", None) is not None:
            main.wait_stream(self._side)

    def side_by_side(self, side_work, main_work, stream=None):
        """Runs side_work(side_stream) on the renderer's side stream after everything issued
        so far on `stream`, main_work() on `stream`, and makes `stream` wait for both."""
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(self.device)
        self._side.wait_stream(main)
        with torch.cuda.stream(self._side):
            side_work(self._side)
        main_work()
        main.wait_stream(self._side)

    def status(self) -> int:
        """Device status word of the last binning (0 = ok); synchronises."""
        return int(self.status_word.item())

    def instances(self) -> int:
        return int(self.n_inst.item())

    def images(self, view: int = 0):
        """Views of the rendered images of one view as [C,H,W] tensors (renderer-owned)."""
        h, w = self.sizes[view]
        a, b = self.pix_off[view], self.pix_off[view + 1]
        return dict(rgb=self.img_rgb[:, a:b].view(3, h, w), depth=self.img_depth[a:b].view(h, w),
                    sil=self.img_sil[a:b].view(h, w), feat=self.img_feat[: self.feat_dim, a:b].view(-1, h, w),
                    T=self.img_T[a:b].view(h, w), n_contrib=self.img_nc[a:b].view(h, w))


def fit_capacity(field: Field, cams, feat_dim: int, margin: float = 1.25, params: RasterParams = RasterParams(),
                 n_classes: int = 0, device="cuda") -> Renderer:
    """Builds a Renderer whose instance capacity fits this field and these views (the
    instances of one projection, times the margin)."""
    r = Renderer(field.n, cams, feat_dim, 0, device, params, n_classes)
    need = int(r.instances_needed(field).item())
    r.ensure_capacity(max(1024, int(need * margin)))
    return r


# supplementary C.1 mapping learning rates, in the update's group order:
# position, rotation, scaling, opacity, colour, feature
MAPPING_LR = (1e-4, 1e-3, 1e-3, 0.05, 2.5e-3, 2.5e-3)


class MappingAdam:
    """Adam state of the field's parameters (gs_adam_step): moments m, v of every group and a
    device step counter, so the update can be part of a captured mapping iteration."""

    def __init__(self, field: Field, lr=MAPPING_LR, betas=(0.9, 0.999), eps=1e-15,
                 moments: Optional[torch.Tensor] = None):
        if field.rgb.dtype != torch.float32 or field.feat.dtype != torch.float32:
            raise ValueError("the mapping update works on f32 parameter storage")
        self.field, self.lr, self.betas, self.eps = field, tuple(lr), betas, eps
        n, D = field.n, field.feat_dim
        size = 2 * n * (14 + D)
        if moments is None:
            self.moments = torch.zeros(size, dtype=torch.float32, device=field.means.device)
        else:                          # a caller's f32 buffer of at least that many values, zeroed here
            if moments.dtype != torch.float32 or moments.numel() < size:
                raise ValueError(f"the moments need {size} float32 values")
            self.moments = moments[:size]
            self.moments.zero_()
        self.step_ctr = torch.zeros(1, dtype=torch.float64, device=field.means.device)

    def step(self, r: "Renderer", step: int = 0, stream=None):
        """One update from the renderer's gradients; step 0 counts on the device."""
        f = self.field
        fm = L.gs_field_mut(f.n, f.feat_dim, _p(f.means), _p(f.quats), _p(f.log_scales), _p(f.opacity_logits),
                            _p(f.rgb), _p(f.feat) if f.feat_dim else None)
        lr = (ctypes.c_float * 6)(*self.lr)
        L.check("gs_adam_step", L.gs_adam_step(ctypes.byref(fm), ctypes.byref(r.gaussian_grads_c()),
                                               _p(self.moments), step, _p(self.step_ctr), lr, self.betas[0],
                                               self.betas[1], self.eps, _stream(stream)))


def expand(r: "Renderer", field: Field, targets, feat_init: torch.Tensor, tau_unobs: float = 0.5, stream=None):
    """Adaptive Gaussian expansion (Eq. 11) after the renderer's last forward over its views:
    returns (the field with one Gaussian appended per unobserved pixel, the new Gaussians'
    source pixels, the number of unobserved pixels, the status word: GS_ERR_CAPACITY when that
    number exceeds n_max and only the first n_max were added).  feat_init [n_max, D] holds the
    new Gaussians' features (the caller draws them).  Reads the count back to the host (the
    field's size sets every later launch)."""
    if field.rgb.dtype != torch.float32 or field.feat.dtype != torch.float32:
        raise ValueError("expansion appends to f32 parameter storage")
    n, D = field.n, field.feat_dim
    n_max = int(feat_init.shape[0])
    grow = lambda t: torch.cat([t, t.new_zeros((n_max,) + tuple(t.shape[1:]))]).contiguous()
    out = Field(*(grow(t) for t in (field.means, field.quats, field.log_scales, field.opacity_logits, field.rgb,
                                    field.feat)))
    fm = L.gs_field_mut(n + n_max, D, _p(out.means), _p(out.quats), _p(out.log_scales), _p(out.opacity_logits),
                        _p(out.rgb), _p(out.feat) if D else None)
    dev = field.means.device
    n_new = torch.zeros(1, dtype=torch.int64, device=dev)
    src = torch.zeros(max(n_max, 1), dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    tc = L.gs_targets(_p(targets["rgb"]), _p(targets["depth"]), _p(targets["label"]))
    fi = feat_init.contiguous().to(torch.float32)
    L.check("gs_expand", L.gs_expand(r.cams_c, r.n_views, ctypes.byref(r.images_c()), ctypes.byref(tc), tau_unobs,
                                     _p(fi) if D else None, n, ctypes.byref(fm), _p(n_new), _p(src), _p(status),
                                     _p(r.ws), r.ws.numel(), _stream(stream)))
    total = int(n_new.item())
    k = min(total, n_max)
    keep = lambda t: t[: n + k].contiguous()
    return Field(*(keep(t) for t in (out.means, out.quats, out.log_scales, out.opacity_logits, out.rgb,
                                     out.feat))), src[:k], total, int(status.item())


class Tracker:
    """Frame-to-model tracking (Sec. 3.4) against a fixed map on the GPU.  A frame's n_it
    pose-only iterations (tracking loss of Eq. 20-21 with the M_obs mask; Adam on the twist with
    the C.1 rates, moments reset per frame) are n_it replays of one captured iteration, whose
    pose step writes the pose the next projection reads and counts Adam's steps on the device;
    per frame the observation is copied into the graph's input buffers and the start pose is
    set before the replays."""

    def __init__(self, field: Field, cam, dec_W: torch.Tensor, dec_b: torch.Tensor, n_it: int = 40,
                 params: RasterParams = RasterParams(), margin: float = 1.6, lr=TRACKING_LR, use_graph: bool = True,
                 renderer: Optional[Renderer] = None):
        dev = field.means.device
        self.field, self.W, self.b, self.n_it, self.lr = field, dec_W, dec_b, n_it, lr
        self.use_graph = use_graph
        # a caller's renderer (one view of cam's size, sized for this field) or a fitted one
        self.r = renderer if renderer is not None else fit_capacity(
            field, [cam], field.feat_dim, margin=margin, params=params, n_classes=int(dec_W.shape[0]), device=dev)
        P = cam.width * cam.height
        self.tg = dict(rgb=torch.zeros(3, P, device=dev), depth=torch.zeros(P, device=dev),
                       label=torch.zeros(P, dtype=torch.uint8, device=dev))
        self.T = torch.zeros(1, 16, dtype=torch.float64, device=dev)
        self.adam = torch.zeros(13, dtype=torch.float64, device=dev)
        self.pose = torch.zeros(1, 16, dtype=torch.float32, device=dev)
        self.graph = None

    def _iteration(self):
        self.r.iteration(self.field, self.tg, self.W, self.b, TRACKING, L.GS_GRAD_POSE, pose_dev=self.pose)
        self.r.pose_step(self.T, self.adam, 0, lr=self.lr, pose_f32=self.pose)

    def _start(self, T_init):
        self.T.copy_(torch.as_tensor(np.asarray(T_init, np.float64).reshape(1, 16)))
        self.adam.zero_()
        self.pose.copy_(self.T.float())

    def track(self, frame, T_init) -> np.ndarray:
        """Pose (4x4 world-to-camera, f64) of one observed frame (host arrays rgb [3,H,W],
        depth [H,W], label [H,W], or a dict of device targets rgb [3,P], depth [P], label [P])
        from the start pose T_init."""
        if isinstance(frame, dict):
            for k in ("rgb", "depth", "label"):
                self.tg[k].copy_(frame[k].reshape(self.tg[k].shape))
        else:
            self.tg["rgb"].copy_(torch.as_tensor(np.ascontiguousarray(frame.rgb, np.float32).reshape(3, -1)))
            self.tg["depth"].copy_(torch.as_tensor(np.ascontiguousarray(frame.depth, np.float32).ravel()))
            self.tg["label"].copy_(torch.as_tensor(np.ascontiguousarray(frame.label, np.uint8).ravel()))
        if self.use_graph and self.graph is None:
            self._start(T_init)
            cur = torch.cuda.current_stream()
            side = torch.cuda.Stream()
            side.wait_stream(cur)
            with torch.cuda.stream(side):
                self._iteration()                    # module loads before the capture
            cur.wait_stream(side)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._iteration()
        self._start(T_init)
        for _ in range(self.n_it):
            if self.use_graph:
                self.graph.replay()
            else:
                self._iteration()
        T = self.T.cpu().numpy().reshape(4, 4)
        if self.r.status() != 0:
            raise L.GsError("tracking binning", self.r.status())
        return T


def constant_velocity(T_prev, T_prev2):
    """Eq. 19: T_t = T_{t-1} T_{t-2}^-1 T_{t-1} (world-to-camera, f64)."""
    return np.asarray(T_prev, np.float64) @ np.linalg.inv(np.asarray(T_prev2, np.float64)) @ T_prev


def track_sequence(tracker: Tracker, frames, T_known):
    """Poses of a frame sequence: the first len(T_known) frames keep the given poses; each later
    frame is tracked from the constant-velocity prediction (Eq. 19)."""
    est = [np.asarray(T, np.float64) for T in T_known]
    for t in range(len(est), len(frames)):
        est.append(tracker.track(frames[t], constant_velocity(est[-1], est[-2] if len(est) >= 2 else est[-1])))
    return est


class RasterizeSG(torch.autograd.Function):
    """Differentiable render of a Semantic Gaussian Field through libgs.

    forward(renderer, means, quats, log_scales, opacity_logits, rgb, feat) returns
    (rgb [3,P], depth [P], sil [P], feat [D,P]) over the renderer's views;
    backward runs gs_render_bwd and returns the parameter gradients.
    """

    @staticmethod
    def forward(ctx, renderer: Renderer, means, quats, log_scales, opacity_logits, rgb, feat):
        field = Field(means.detach().contiguous(), quats.detach().contiguous(), log_scales.detach().contiguous(),
                      opacity_logits.detach().contiguous(), rgb.detach().contiguous(), feat.detach().contiguous())
        renderer.forward(field)
        ctx.renderer, ctx.field = renderer, field
        D = renderer.feat_dim
        return (renderer.img_rgb.clone(), renderer.img_depth.clone(), renderer.img_sil.clone(),
                renderer.img_feat[:D].clone())

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_sil, g_feat):
        r = ctx.renderer
        z = lambda g, like: like.zero_() if g is None else like.copy_(g)
        z(g_rgb, r.g_rgb)
        z(g_depth, r.g_depth)
        z(g_sil, r.g_sil)
        if r.feat_dim:
            z(g_feat, r.g_feat[: r.feat_dim])
        r.backward(ctx.field, L.GS_GRAD_MAP)
        D = r.feat_dim
        return (None, r.d_means.clone(), r.d_quats.clone(), r.d_log_scales.clone(), r.d_logits.clone(),
                r.d_rgb.clone(), r.d_feat[:, :D].clone() if D else torch.zeros_like(ctx.field.feat))


def rasterize(renderer: Renderer, means, quats, log_scales, opacity_logits, rgb, feat):
    return RasterizeSG.apply(renderer, means, quats, log_scales, opacity_logits, rgb, feat)


_FIELD_ARRAYS = ("means", "quats", "log_scales", "opacity_logits", "rgb", "feat")


class HostStepper:
    """Steps whose inputs (field parameters and targets) come from pinned host memory and
    whose results (device tensors the step writes) go back to pinned host memory, with each
    step's transfers overlapped with its neighbours' compute: step i's upload runs on a copy
    stream into one of two device input sets while step i-1 computes, and step i's results
    are downloaded on a second copy stream while step i+1 computes.  `step(field, targets)`
    issues one step on the current stream; `outputs` are the tensors it writes.  With
    `bind`, bind(k) makes the next step write output set k (k = 0, 1) and returns that set's
    tensors, and the results are downloaded from there (the set of the last step stays bound
    when run returns); without it they are first copied on the device into one of two
    staging sets.  With `graphs`, the first step on each input set runs as called and is
    captured in a CUDA graph, and every later step on that set replays it: the step must then
    launch the same work on the same buffers each time, with any state that changes from step
    to step kept on the device (the capture synchronises the device once per set)."""

    def __init__(self, like_field: Field, like_targets: dict, outputs: Sequence[torch.Tensor], bind=None,
                 graphs: bool = False):
        dev = like_field.means.device
        clone = lambda t: torch.empty_like(t)
        self.fields = [Field(*(clone(getattr(like_field, k)) for k in _FIELD_ARRAYS)) for _ in range(2)]
        self.targets = [{k: clone(v) for k, v in like_targets.items()} for _ in range(2)]
        self.outputs = list(outputs)
        self.bind = bind
        self.graphs = [None, None] if graphs else None
        self.staging = None if bind is not None else [[clone(o) for o in self.outputs] for _ in range(2)]
        self.host_out = [[torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in self.outputs]
                         for _ in range(2)]
        self.h2d, self.d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev = lambda: [torch.cuda.Event() for _ in range(2)]
        self.uploaded, self.computed, self.downloaded = ev(), ev(), ev()
        self.bytes_in = sum(getattr(like_field, k).numel() * getattr(like_field, k).element_size()
                            for k in _FIELD_ARRAYS) + sum(v.numel() * v.element_size() for v in like_targets.values())
        self.bytes_out = sum(o.numel() * o.element_size() for o in self.outputs)

    def _step(self, step, buf, f, tg):
        if self.graphs is None:
            step(f, tg)
        elif self.graphs[buf] is None:
            # first step on set buf: run it (these are its results), then capture it for the
            # later steps on the set
            step(f, tg)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step(f, tg)
            self.graphs[buf] = g
        else:
            self.graphs[buf].replay()

    def run(self, step, host_inputs, on_result=None):
        """Runs one step per (host_field, host_targets) pair of `host_inputs` (dicts of pinned
        host tensors keyed like Field's arrays and like the targets).  on_result(i, tensors)
        receives step i's results in pinned host memory once they have arrived (valid until
        the callback returns).  Returns the number of steps."""
        compute = torch.cuda.current_stream()
        pending = [None, None]          # step whose download occupies host_out[buf]
        n = 0
        for i, (hf, ht) in enumerate(host_inputs):
            buf = i & 1
            # upload into input set buf once step i-2 has finished computing on it
            if i >= 2:
                self.h2d.wait_event(self.computed[buf])
            with torch.cuda.stream(self.h2d):
                f, tg = self.fields[buf], self.targets[buf]
                for k in _FIELD_ARRAYS:
                    getattr(f, k).copy_(hf[k], non_blocking=True)
                for k, v in ht.items():
                    tg[k].copy_(v, non_blocking=True)
                self.uploaded[buf].record(self.h2d)
            compute.wait_event(self.uploaded[buf])
            if self.bind is not None:
                # the step writes output set buf once step i-2's download from it is done
                if i >= 2:
                    compute.wait_event(self.downloaded[buf])
                results = self.bind(buf)
                self._step(step, buf, f, tg)
            else:
                self._step(step, buf, f, tg)
                # results to staging set buf once step i-2's download from it is done
                if i >= 2:
                    compute.wait_event(self.downloaded[buf])
                for s, o in zip(self.staging[buf], self.outputs):
                    s.copy_(o, non_blocking=True)
                results = self.staging[buf]
            self.computed[buf].record(compute)
            # host buffer buf is free once step i-2's results were handed over
            if pending[buf] is not None:
                self.downloaded[buf].synchronize()
                if on_result is not None:
                    on_result(pending[buf], self.host_out[buf])
            self.d2h.wait_event(self.computed[buf])
            with torch.cuda.stream(self.d2h):
                for h, s in zip(self.host_out[buf], results):
                    h.copy_(s, non_blocking=True)
                self.downloaded[buf].record(self.d2h)
            pending[buf] = i
            n += 1
        for buf in sorted((b for b in range(2) if pending[b] is not None), key=lambda b: pending[b]):
            self.downloaded[buf].synchronize()
            if on_result is not None:
                on_result(pending[buf], self.host_out[buf])
        return n
