"""The GS3LAM loop on the GPU: tracking, adaptive expansion and RSKM keyframe mapping.

Per frame (Sec. 3.3-3.4): the pose is tracked from the constant-velocity
prediction (Eq. 19) against the map so far, the map rendered at that pose is
expanded where it does not explain the observation (Eq. 11), and the field is
optimised for a number of mapping iterations, each on a frame drawn by RSKM
(Eq. 13) from the keyframes and the current frame.  The keyframes' observations
and estimated poses stay on the device (gs_keyframes), the field lives in
preallocated device arrays that expansion appends to, and each mapping
iteration is: the draw and gather (gs_rskm_draw), one fwd+bwd pass of the
mapping loss with D-SSIM (Eq. 14-18) and the fused Adam update.  The host only
sequences the calls and reads back the pose and the expansion count per frame.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time
from typing import Optional

import numpy as np
import torch

from . import _lib as L
from .raster import MAPPING_SSIM, Field, MappingAdam, RasterParams, Renderer, Tracker, _p, _stream, constant_velocity


_GROUPS = ("means", "quats", "log_scales", "opacity_logits", "rgb", "feat")


@dataclasses.dataclass
class SlamConfig:
    """Iterations per frame (C.1, Replica: 40 tracking, 60 mapping) and the values the paper
    leaves open: the first frame's mapping iterations, the RSKM interval t_opt, the keyframe
    interval and the expansion threshold on the silhouette."""
    n_track: int = 40
    n_map: int = 60
    n_init: int = 60
    t_opt: int = 2
    kf_every: int = 5
    tau_unobs: float = 0.5


class KeyframeStore:
    """Observations (planar rgb [3,P], depth [P], label [P]) and estimated poses (f64 [16]) of
    up to `capacity` frames of one camera, resident on the device."""

    def __init__(self, capacity: int, width: int, height: int, device="cuda"):
        self.capacity, self.P = int(capacity), int(width) * int(height)
        P, dev = self.P, torch.device(device)
        self.rgb = torch.zeros(capacity, 3, P, dtype=torch.float32, device=dev)
        self.depth = torch.zeros(capacity, P, dtype=torch.float32, device=dev)
        self.label = torch.zeros(capacity, P, dtype=torch.uint8, device=dev)
        self.T = torch.zeros(capacity, 16, dtype=torch.float64, device=dev)

    def put_frame(self, slot: int, frame):
        """Uploads a host frame (rgb [3,H,W], depth [H,W], label [H,W]) into a slot."""
        self.rgb[slot].copy_(torch.as_tensor(np.ascontiguousarray(frame.rgb, np.float32).reshape(3, -1)))
        self.depth[slot].copy_(torch.as_tensor(np.ascontiguousarray(frame.depth, np.float32).ravel()))
        self.label[slot].copy_(torch.as_tensor(np.ascontiguousarray(frame.label, np.uint8).ravel()))

    def put_pose(self, slot: int, T):
        self.T[slot].copy_(torch.as_tensor(np.asarray(T, np.float64).reshape(16)))

    def targets(self, slot: int):
        return dict(rgb=self.rgb[slot], depth=self.depth[slot], label=self.label[slot])

    def c(self) -> L.gs_keyframes:
        return L.gs_keyframes(self.capacity, self.P, _p(self.rgb), _p(self.depth), _p(self.label), _p(self.T))


class RskmSampler:
    """Device state of the RSKM draws: the random words (u32), the per-frame iteration
    counter and drawn slot, the log of drawn slots, and the buffers the drawn frame's
    observation and pose are gathered into (the loss targets and gs_project's pose_dev)."""

    def __init__(self, store: KeyframeStore, draws: np.ndarray, device="cuda"):
        dev = torch.device(device)
        self.store = store
        words = np.ascontiguousarray(np.asarray(draws, np.uint32)).view(np.int32)
        self.draws = torch.as_tensor(words).to(dev)
        self.state = torch.zeros(2, dtype=torch.int32, device=dev)
        self.picked = torch.full((len(words),), -1, dtype=torch.int32, device=dev)
        P = store.P
        self.targets = dict(rgb=torch.zeros(3, P, device=dev), depth=torch.zeros(P, device=dev),
                            label=torch.zeros(P, dtype=torch.uint8, device=dev))
        self.pose = torch.zeros(1, 16, dtype=torch.float32, device=dev)
        self.kf_c = store.c()

    def begin(self, offset: int, count: int, n_kf: int, cur_slot: int, t_opt: int):
        """Starts a frame's mapping: its iterations use draws[offset, offset + count)."""
        if offset < 0 or count < 1 or offset + count > self.draws.numel():
            raise ValueError("not enough random words for the mapping iterations")
        self.offset, self.count, self.n_kf, self.cur_slot, self.t_opt = offset, count, n_kf, cur_slot, t_opt
        self.state.zero_()

    def draw(self, stream=None):
        """One draw and gather; asynchronous."""
        off = self.offset
        L.check("gs_rskm_draw", L.gs_rskm_draw(
            ctypes.byref(self.kf_c), self.n_kf, self.cur_slot, self.t_opt, _p(self.draws[off:]), self.count,
            _p(self.state), _p(self.picked[off:]), _p(self.targets["rgb"]), _p(self.targets["depth"]),
            _p(self.targets["label"]), _p(self.pose), _stream(stream)))


class Slam:
    """The loop over a sequence of frames of one camera (intrinsics of `cam`).  The first
    frame keeps the pose T0; the field starts empty and grows by expansion (new features
    taken from feat_bank in order: Gaussian i gets row i); the decoder stays fixed.
    draws: one u32 random word per mapping iteration of the whole sequence."""

    def __init__(self, cam, dec_W: torch.Tensor, dec_b: torch.Tensor, n_frames: int, draws: np.ndarray,
                 feat_bank: torch.Tensor, cfg: SlamConfig = SlamConfig(), params: RasterParams = RasterParams(),
                 gaussian_capacity: Optional[int] = None, graphs: bool = True, device="cuda"):
        dev = torch.device(device)
        self.cam, self.W, self.b, self.cfg, self.params = cam, dec_W, dec_b, cfg, params
        self.graphs = graphs
        self.D, self.K = int(dec_W.shape[1]), int(dec_W.shape[0])
        P = cam.width * cam.height
        cap = int(gaussian_capacity or P * n_frames)
        if feat_bank.shape[0] < cap or feat_bank.shape[1] != self.D:
            raise ValueError("feat_bank needs [gaussian_capacity, feat_dim] rows")
        self.cap = cap
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=dev)
        self._store = Field(z(cap, 3), z(cap, 4), z(cap, 3), z(cap), z(cap, 3), z(cap, self.D))
        self.feat_bank = feat_bank.to(device=dev, dtype=torch.float32).contiguous()
        self.n = 0
        self.kf = KeyframeStore(n_frames // cfg.kf_every + 2, cam.width, cam.height, dev)
        self.sampler = RskmSampler(self.kf, draws, dev)
        # one renderer serves tracking, expansion and mapping of every frame: its per-Gaussian
        # buffers hold the field's capacity, its instance capacity grows when a probe asks
        self.r = Renderer(cap, [cam], self.D, 4 * P, dev, params, self.K)
        self.moments = torch.zeros(2 * cap * (14 + self.D), dtype=torch.float32, device=dev)
        self.n_kf = 0
        self.n_drawn = 0
        self.est = []
        self.sizes = []
        self.kf_frames = []
        self.timings = []      # per frame: wall ms of tracking, expansion, mapping (each ends in a sync)

    def field(self) -> Field:
        return Field(*(getattr(self._store, k)[: self.n] for k in _GROUPS))

    def _at(self, T):
        return dataclasses.replace(self.cam, T_cw=np.asarray(T, np.float64))

    def _fit(self, field: Field, poses=(None,), margin: float = 1.25):
        """Sets the renderer to the field and grows its instance capacity to the most any of
        the poses (device f32 [1,16]; None = the renderer's camera) needs, with a margin."""
        r = self.r
        r.set_n(field.n)
        need = None
        for pose in poses:
            k = r.instances_needed(field, pose)
            need = k if need is None else torch.maximum(need, k)
        r.ensure_capacity(int(int(need.item()) * margin) + 1024)

    def _expand(self, T, slot: int):
        """Eq. 11 at pose T: render the field, append one Gaussian per unobserved pixel."""
        field = self.field()
        r = self.r
        r.set_cameras([self._at(T)])
        self._fit(field)
        r.forward(field)
        s = self._store
        fm = L.gs_field_mut(self.cap, self.D, _p(s.means), _p(s.quats), _p(s.log_scales), _p(s.opacity_logits),
                            _p(s.rgb), _p(s.feat))
        dev = s.means.device
        n_new = torch.zeros(1, dtype=torch.int64, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        tg = self.kf.targets(slot)
        tc = L.gs_targets(_p(tg["rgb"]), _p(tg["depth"]), _p(tg["label"]))
        L.check("gs_expand", L.gs_expand(r.cams_c, 1, ctypes.byref(r.images_c()), ctypes.byref(tc),
                                         self.cfg.tau_unobs, _p(self.feat_bank[self.n:]), self.n, ctypes.byref(fm),
                                         _p(n_new), None, _p(status), _p(r.ws), r.ws.numel(), _stream()))
        if int(status.item()) != 0:
            raise L.GsError("expansion (Gaussian capacity)", int(status.item()))
        self.n += int(n_new.item())
        if r.status() != 0:
            raise L.GsError("expansion binning", r.status())

    def process(self, frame, T0=None) -> np.ndarray:
        """One frame (host rgb [3,H,W], depth [H,W], label [H,W]); returns its estimated pose.
        T0: the first frame's pose."""
        cfg = self.cfg
        t = len(self.est)
        slot = self.n_kf                      # the current frame's slot (kept if it is a keyframe)
        t0 = time.perf_counter()
        self.kf.put_frame(slot, frame)
        if t == 0:
            if T0 is None:
                raise ValueError("the first frame needs its pose")
            T = np.asarray(T0, np.float64)
        else:
            T_pred = constant_velocity(self.est[-1], self.est[-2] if t >= 2 else self.est[-1])
            self.r.set_cameras([self._at(T_pred)])
            self._fit(self.field(), margin=1.6)
            tracker = Tracker(self.field(), self._at(T_pred), self.W, self.b, n_it=cfg.n_track, params=self.params,
                              use_graph=self.graphs, renderer=self.r)
            T = tracker.track(self.kf.targets(slot), T_pred) if cfg.n_track > 0 else T_pred
        self.est.append(T)
        t1 = time.perf_counter()
        self.kf.put_pose(slot, T)
        self._expand(T, slot)
        t2 = time.perf_counter()
        if t % cfg.kf_every == 0:
            self.kf_frames.append(t)
            self.n_kf += 1
        n_it = cfg.n_init if t == 0 else cfg.n_map
        if n_it > 0:
            field = self.field()
            r = self.r
            self._fit(field, [self.kf.T[c: c + 1].float() for c in range(max(self.n_kf, slot + 1))])
            opt = MappingAdam(field, moments=self.moments)
            self.sampler.begin(self.n_drawn, n_it, self.n_kf, slot, cfg.t_opt)

            def iteration():
                self.sampler.draw()
                r.iteration(field, self.sampler.targets, self.W, self.b, MAPPING_SSIM, L.GS_GRAD_MAP,
                            pose_dev=self.sampler.pose)
                opt.step(r, 0)
            if self.graphs and t > 0:
                # every iteration is the same launches (the draw counter and Adam's step count
                # live on the device): capture one, replay it; the first frame ran eagerly, so
                # every kernel is loaded before any capture
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    iteration()
                for _ in range(n_it):
                    g.replay()
            else:
                for _ in range(n_it):
                    iteration()
            self.n_drawn += n_it
            if r.status() != 0:
                raise L.GsError("mapping binning", r.status())
        self.sizes.append(self.n)
        t3 = time.perf_counter()
        self.timings.append(dict(track_ms=1e3 * (t1 - t0), expand_ms=1e3 * (t2 - t1), map_ms=1e3 * (t3 - t2)))
        return T

    def picks(self):
        """Frame index of every mapping iteration's draw so far."""
        slots = self.sampler.picked[: self.n_drawn].cpu().numpy()
        out = []
        # slot -> frame: keyframe slots hold their frames; the slot after them held the frame
        # being mapped when it was drawn
        it = 0
        for t in range(len(self.est)):
            n_it = self.cfg.n_init if t == 0 else self.cfg.n_map
            kf_upto = sum(1 for f in self.kf_frames if f <= t)
            for s in slots[it: it + n_it]:
                out.append(self.kf_frames[s] if s < kf_upto else t)
            it += n_it
        return out
