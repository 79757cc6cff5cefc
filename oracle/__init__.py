"""FP64 CPU oracle of the GS3LAM semantic-splatting rasterizer (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The product path (the CUDA library and its binding) never calls
it; there is no CPU fallback.  The C source `gs_oracle.c` is compiled with gcc
into `oracle/_build/libgs_oracle.so` on first use (or by `build()`).

Every function takes float64 numpy arrays (float32 inputs are widened exactly)
and returns float64 results.  Images are planar [C, H, W].

Parity status per function (pins live in tests/test_oracle_pins.py):
  project       pinned: closed forms, Monte-Carlo EWA, rotation invariance
  rects         pinned: brute-force tile/square intersection
  bin_sort      pinned: brute-force per-tile lists
  render_fwd    pinned: closed forms, brute force without tiles, Eq. 4 literal sum
  render_bwd    pinned: central finite differences
  project_bwd   pinned: central finite differences, translation invariance
  loss          pinned: textbook softmax-CE, hand-computed L1, median by sorting
  dsr           pinned: hand-sized arrays
  pose_step     pinned: matrix exponential, first Adam step
  ssim          pinned: identical and constant images (closed form), central differences
  adam_step     pinned: sign steps from zero moments, written-out moment series
  expand        pinned: empty render (reprojection), explained frame, 50 x median rule
  constant_velocity, track_sequence, ate_rmse
                pinned: constant screw motion, shifted trajectory, wiring without steps
  rskm_select   pinned: Eq. 13 cases, full cycles of words, long-run share (fractions)
  slam          pinned: first frame expands every pixel, mapping lowers the loss,
                draws and poses with constant words and no tracking steps
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgs_oracle.so")
_lib = None

# Raster parameter order of the C source.
PARAM_NAMES = ("tile", "alpha_min", "alpha_max", "T_min", "z_near", "lowpass", "radius_sigma",
               "bg_r", "bg_g", "bg_b", "exact_jacobian")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC,
               "-lm"]
        try:      # per-row / per-Gaussian loops in parallel where gcc has OpenMP
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_count_instances.restype = ctypes.c_int64
        _lib.or_bin_sort.restype = ctypes.c_int64
        _lib.or_loss.restype = ctypes.c_double
        _lib.or_dsr.restype = ctypes.c_double
        _lib.or_ssim.restype = ctypes.c_double
        _lib.or_lower_median.restype = ctypes.c_double
        _lib.or_get_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (0: every core); returns the count in use."""
    _L().or_set_threads(ctypes.c_int(n))
    return int(_L().or_get_threads())


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


I64 = ctypes.c_int64


@dataclasses.dataclass
class Params:
    tile: int = 16
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    z_near: float = 0.2
    lowpass: float = 0.3
    radius_sigma: float = 3.0
    bg: tuple = (0.0, 0.0, 0.0)
    # False: the EWA Jacobian is evaluated at (x/z, y/z) clamped to the view widened by 15 %
    # per side (the 3DGS rasterizer convention); True: unclamped, the literal Eq. 3
    exact_jacobian: bool = False

    def array(self):
        return np.array([self.tile, self.alpha_min, self.alpha_max, self.T_min, self.z_near,
                         self.lowpass, self.radius_sigma, *self.bg, float(self.exact_jacobian)],
                        dtype=np.float64)


def _cam(cam):
    return (np.array([cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy], np.float64),
            _d(np.asarray(cam.T_cw, np.float64).reshape(16)))


def _tiles(cam, tile):
    tx = (cam.width + tile - 1) // tile
    ty = (cam.height + tile - 1) // tile
    return tx, ty


# ------------------------------------------------------------------ projection
def project(gs, cam, prm: Params):
    n = gs.n
    c, T = _cam(cam)
    out = dict(uv=np.zeros((n, 2)), depth=np.zeros(n), depth_key=np.zeros(n, np.float32),
               conic=np.zeros((n, 3)), opacity=np.zeros(n), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), touched=np.zeros(n, np.int32),
               radius_real=np.zeros(n), cov2d=np.zeros((n, 3)))
    a = [_d(gs.means), _d(gs.quats), _d(gs.log_scales), _d(gs.opacity_logits)]
    _L().or_project(I64(n), *map(_p, a), _p(c), _p(T), _p(prm.array()),
                    *(_p(out[k]) for k in ("uv", "depth", "depth_key", "conic", "opacity", "radius",
                                           "rect", "touched", "radius_real", "cov2d")))
    return out


def rects(uv, radius, width, height, tile=16):
    uv = _d(uv)
    radius = np.ascontiguousarray(radius, np.int32)
    n = radius.shape[0]
    rect = np.zeros((n, 4), np.int32)
    touched = np.zeros(n, np.int32)
    _L().or_rects(I64(n), _p(uv), _p(radius), ctypes.c_int(width), ctypes.c_int(height),
                  ctypes.c_int(tile), _p(rect), _p(touched))
    return rect, touched


def bin_sort(rect, depth_key, cams, tile=16, n_per_view=None):
    """Keys, values and per-tile ranges of the (tile | depth) order over all views."""
    rect = np.ascontiguousarray(rect, np.int32)
    depth_key = np.ascontiguousarray(depth_key, np.float32)
    nv = len(cams)
    n_per_view = rect.shape[0] // nv if n_per_view is None else n_per_view
    txs = np.array([_tiles(c, tile)[0] for c in cams], np.int32)
    tpv = np.array([np.prod(_tiles(c, tile)) for c in cams], np.int32)
    m = int(((rect[:, 2] - rect[:, 0]).astype(np.int64) * (rect[:, 3] - rect[:, 1])).sum())
    keys = np.zeros(max(m, 1), np.uint64)
    vals = np.zeros(max(m, 1), np.uint32)
    ranges = np.zeros((int(tpv.sum()), 2), np.uint32)
    got = _L().or_bin_sort(ctypes.c_int(nv), I64(n_per_view), _p(rect), _p(depth_key), _p(txs),
                           _p(tpv), _p(keys), _p(vals), _p(ranges))
    assert got == m
    return keys[:m], vals[:m], ranges


# ---------------------------------------------------------------------- render
def render_fwd(cam, proj, rgb, feat, vals, ranges, prm: Params, view_offset=0, tile_offset=0,
               conditioning=True):
    """Front-to-back blend of one view; with conditioning, also the per-pixel rounding figures
    margin, sens and sens_depth (see gs_oracle.c)."""
    W, H = cam.width, cam.height
    D = feat.shape[1]
    P = W * H
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), sil=np.zeros((H, W)),
               feat=np.zeros((D, H, W)), T=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32))
    if conditioning:
        out.update(margin=np.zeros((H, W)), sens=np.zeros((H, W)), sens_depth=np.zeros((H, W)))
    args = [_d(proj["uv"]), _d(proj["conic"]), _d(proj["opacity"]), _d(proj["depth"]), _d(rgb), _d(feat)]
    cond = [_p(out[k]) if conditioning else None for k in ("margin", "sens", "sens_depth")]
    _L().or_render_fwd(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(prm.tile), ctypes.c_int(D),
                       I64(view_offset), I64(tile_offset), *map(_p, args),
                       _p(np.ascontiguousarray(vals, np.uint32)), _p(np.ascontiguousarray(ranges, np.uint32)),
                       _p(prm.array()), *(_p(out[k]) for k in ("rgb", "depth", "sil", "feat", "T", "n_contrib")),
                       *cond)
    return out


def render_bwd(cam, proj, rgb, feat, vals, ranges, prm: Params, g_rgb, g_depth, g_sil, g_feat,
               view_offset=0, tile_offset=0):
    W, H = cam.width, cam.height
    n = proj["uv"].shape[0]
    D = feat.shape[1]
    out = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), depth=np.zeros(n),
               rgb=np.zeros((n, 3)), feat=np.zeros((n, D)))
    args = [_d(proj["uv"]), _d(proj["conic"]), _d(proj["opacity"]), _d(proj["depth"]), _d(rgb), _d(feat)]
    g = [_d(g_rgb), _d(g_depth), _d(g_sil), _d(g_feat)]
    _L().or_render_bwd(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(prm.tile), ctypes.c_int(D),
                       I64(view_offset), I64(tile_offset), *map(_p, args),
                       _p(np.ascontiguousarray(vals, np.uint32)), _p(np.ascontiguousarray(ranges, np.uint32)),
                       _p(prm.array()), *map(_p, g),
                       *(_p(out[k]) for k in ("uv", "conic", "opacity", "depth", "rgb", "feat")))
    return out


def project_bwd(gs, cam, prm: Params, d_uv, d_conic, d_opacity, d_depth):
    n = gs.n
    c, T = _cam(cam)
    out = dict(means=np.zeros((n, 3)), quats=np.zeros((n, 4)), log_scales=np.zeros((n, 3)),
               opacity_logits=np.zeros(n), twist=np.zeros(6))
    a = [_d(gs.means), _d(gs.quats), _d(gs.log_scales), _d(gs.opacity_logits)]
    g = [_d(d_uv), _d(d_conic), _d(d_opacity), _d(d_depth)]
    _L().or_project_bwd(I64(n), *map(_p, a), _p(c), _p(T), _p(prm.array()), *map(_p, g),
                        *(_p(out[k]) for k in ("means", "quats", "log_scales", "opacity_logits", "twist")))
    return out


# ------------------------------------------------------------------------ loss
@dataclasses.dataclass
class LossWeights:
    color: float = 0.5
    depth: float = 1.0
    sem: float = 0.01
    big: float = 0.01
    small: float = 0.001
    mask_mode: int = 0      # 0 mapping (no mask), 1 tracking (Eq. 21 mask)
    tau_obs: float = 0.99
    ssim: float = 0.0       # lambda of Eq. 15: colour = (1 - lambda) L1 + lambda (1 - SSIM); mapping only


MAPPING = LossWeights()
MAPPING_SSIM = LossWeights(ssim=0.2)          # Eq. 15 with the paper's lambda = 0.2
TRACKING = LossWeights(color=0.5, depth=1.0, sem=0.001, big=0.0, small=0.0, mask_mode=1)


def loss(images, target, dec, w: LossWeights):
    rgb, depth, sil, feat = images["rgb"], images["depth"], images["sil"], images["feat"]
    D = feat.shape[0]
    H, W = depth.shape
    P = H * W
    K = dec.W.shape[0]
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), sil=np.zeros((H, W)),
               feat=np.zeros((D, H, W)), W=np.zeros((K, D)), b=np.zeros(K), mask=np.zeros((H, W)),
               terms=np.zeros(3), median=np.zeros(1))
    if w.ssim and w.mask_mode != 0:
        raise ValueError("the SSIM term belongs to the mapping loss (tracking colour is L1 only)")
    med = ctypes.c_double(0)
    a = [_d(rgb), _d(depth), _d(sil), _d(feat), _d(target.rgb), _d(target.depth)]
    total = _L().or_loss(I64(P), ctypes.c_int(D), ctypes.c_int(K), *map(_p, a),
                         _p(np.ascontiguousarray(target.label, np.uint8)), _p(_d(dec.W)), _p(_d(dec.b)),
                         ctypes.c_double(w.color * (1.0 - w.ssim)), ctypes.c_double(w.depth),
                         ctypes.c_double(w.sem), ctypes.c_int(w.mask_mode), ctypes.c_double(w.tau_obs),
                         *(_p(out[k]) for k in ("rgb", "depth", "sil", "feat", "W", "b", "mask", "terms")),
                         ctypes.byref(med))
    if w.ssim:
        # Eq. 15: colour = lambda_c ((1 - lambda) L1 + lambda (1 - SSIM))
        s, g = ssim(rgb, target.rgb)
        term = w.color * w.ssim * (1.0 - s)
        out["terms"][0] += term
        total += term
        out["rgb"] -= w.color * w.ssim * g
        out["ssim"] = s
    out["median"] = med.value
    out["total"] = total
    return out


def ssim(x, y):
    """Mean SSIM of two [3, H, W] images (11x11 Gaussian window, sigma 1.5, zero padding,
    C1 = 0.01^2, C2 = 0.03^2) and its gradient with respect to x."""
    x, y = _d(x), _d(y)
    H, W = x.shape[1], x.shape[2]
    grad = np.zeros_like(x)
    val = _L().or_ssim(I64(H), I64(W), _p(x), _p(y), _p(grad))
    return val, grad


def lower_median(values):
    v = _d(values).ravel()
    return _L().or_lower_median(I64(v.shape[0]), _p(v))


def dsr(log_scales, lam_big, lam_small):
    ls = _d(log_scales)
    grad = np.zeros_like(ls)
    stats = np.zeros(6)
    n = ls.size // 3
    val = _L().or_dsr(I64(n), _p(ls), ctypes.c_double(lam_big), ctypes.c_double(lam_small), _p(grad),
                      _p(stats))
    return val, grad, dict(mu=stats[0], sigma=stats[1], n_big=int(stats[2]), n_small=int(stats[3]),
                           L_big=stats[4], L_small=stats[5])


def pose_step(T, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-15):
    T = _d(np.asarray(T).reshape(16)).copy()
    m = _d(m).copy()
    v = _d(v).copy()
    _L().or_pose_step(_p(T), _p(_d(grad)), _p(m), _p(v), ctypes.c_int(step), _p(_d(lr)),
                      ctypes.c_double(b1), ctypes.c_double(b2), ctypes.c_double(eps))
    return T.reshape(4, 4), m, v


# ------------------------------------------------------------- full pipelines
def forward(gs, cam, prm: Params, conditioning=True):
    """Projection, binning, sort and blend of one view; returns (proj, bins, images)."""
    proj = project(gs, cam, prm)
    keys, vals, ranges = bin_sort(proj["rect"], proj["depth_key"], [cam], prm.tile)
    img = render_fwd(cam, proj, gs.rgb, gs.feat, vals, ranges, prm, conditioning=conditioning)
    return proj, (keys, vals, ranges), img


def backward_from_image_grads(gs, cam, prm: Params, proj, bins, g):
    """All parameter gradients and the pose twist from image gradients g."""
    _, vals, ranges = bins
    r = render_bwd(cam, proj, gs.rgb, gs.feat, vals, ranges, prm, g["rgb"], g["depth"], g["sil"], g["feat"])
    p = project_bwd(gs, cam, prm, r["uv"], r["conic"], r["opacity"], r["depth"])
    return dict(means=p["means"], quats=p["quats"], log_scales=p["log_scales"],
                opacity_logits=p["opacity_logits"], rgb=r["rgb"], feat=r["feat"], twist=p["twist"],
                d2=r)


def step(gs, cam, prm: Params, target, dec, w: LossWeights, with_dsr=True, conditioning=True):
    """One fwd+bwd iteration: render, loss (+ DSR), all gradients, pose twist (with
    conditioning, the images carry the rounding figures of render_fwd)."""
    proj, bins, img = forward(gs, cam, prm, conditioning)
    L = loss(img, target, dec, w)
    grads = backward_from_image_grads(gs, cam, prm, proj, bins, L)
    total = L["total"]
    if with_dsr and (w.big or w.small):
        v, gls, stats = dsr(gs.log_scales, w.big, w.small)
        total += v
        grads["log_scales"] = grads["log_scales"] + gls
        grads["dsr"] = stats
    grads["W"], grads["b"] = L["W"], L["b"]
    return dict(total=total, proj=proj, bins=bins, img=img, loss=L, grads=grads)


# parameter groups of the field in the order the Adam update walks them, with the mapping
# learning rates of supplementary C.1 (position, rotation, scaling, opacity, colour, feature)
ADAM_GROUPS = ("means", "quats", "log_scales", "opacity_logits", "rgb", "feat")
MAPPING_LR = dict(means=1e-4, quats=1e-3, log_scales=1e-3, opacity_logits=0.05, rgb=2.5e-3, feat=2.5e-3)


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step (Kingma and Ba, bias-corrected) of every parameter group, in FP64.
    params/grads/m/v: dicts of arrays by group name; step: 1-based; lr: dict by group.
    Returns new (params, m, v) dicts; the inputs are left unchanged."""
    out_p, out_m, out_v = {}, {}, {}
    for k in ADAM_GROUPS:
        g = np.asarray(grads[k], np.float64)
        mk = b1 * np.asarray(m[k], np.float64) + (1 - b1) * g
        vk = b2 * np.asarray(v[k], np.float64) + (1 - b2) * g * g
        mhat = mk / (1 - b1 ** step)
        vhat = vk / (1 - b2 ** step)
        out_p[k] = np.asarray(params[k], np.float64) - lr[k] * mhat / (np.sqrt(vhat) + eps)
        out_m[k], out_v[k] = mk, vk
    return out_p, out_m, out_v


TAU_UNOBS = 0.5     # Eq. 11 threshold on the cumulative opacity (silent in the paper; reading)


def expand(images, target, cam, feat_init, tau_unobs=TAU_UNOBS):
    """Adaptive Gaussian expansion (Eq. 11 and the initialisation after it), one view.

    M_unobs = (o_hat < tau_unobs) or (d_hat > d_gt and |d_gt - d_hat| > 50 median), the median
    being the lower median of |d_gt - d_hat| over pixels with d_gt > 0; only pixels with
    d_gt > 0 can be unprojected.  The decisions are taken in f32 on the f32 inputs (they decide
    integers).  One Gaussian per masked pixel in raster order: mean = the pixel centre
    unprojected at d_gt (world frame, FP64), identity rotation, log-scale log(d_gt / fx) on
    every axis, opacity 0.5 (logit 0), the observed colour, features feat_init[k] for the
    k-th new Gaussian.  Returns a dict of the new parameters and their source pixels."""
    sil = np.asarray(images["sil"], np.float32)
    d_hat = np.asarray(images["depth"], np.float32)
    d_gt = np.asarray(target.depth, np.float32)
    H, W = d_gt.shape
    valid = d_gt > np.float32(0)
    err = np.abs(d_gt - d_hat).astype(np.float32)
    med = np.float32(lower_median(err[valid].astype(np.float64))) if valid.any() else np.float32(0)
    mask = (sil < np.float32(tau_unobs)) | ((d_hat > d_gt) & (err > np.float32(50) * med))
    mask &= valid
    pix = np.nonzero(mask.ravel())[0]
    py, px = pix // W, pix % W
    d = d_gt.ravel()[pix].astype(np.float64)
    pc = np.stack([(px + 0.5 - cam.cx) / cam.fx * d, (py + 0.5 - cam.cy) / cam.fy * d, d], 1)
    T = np.asarray(cam.T_cw, np.float64)
    means = (pc - T[:3, 3]) @ T[:3, :3]          # R^T (p_c - t), row-wise
    n = len(pix)
    return dict(src_pix=pix.astype(np.int64), means=means,
                quats=np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (n, 1)),
                log_scales=np.repeat(np.log(d / cam.fx)[:, None], 3, 1), opacity_logits=np.zeros(n),
                rgb=np.asarray(target.rgb, np.float64).reshape(3, -1)[:, pix].T,
                feat=np.asarray(feat_init, np.float64)[:n], median=float(med), mask=mask)


def constant_velocity(T_prev, T_prev2):
    """Eq. 19: the pose of a new frame from the two before it, T_t = T_{t-1} T_{t-2}^-1 T_{t-1}
    (world-to-camera, FP64)."""
    T_prev, T_prev2 = np.asarray(T_prev, np.float64), np.asarray(T_prev2, np.float64)
    return T_prev @ np.linalg.inv(T_prev2) @ T_prev


def track_sequence(gs, cam, prm: Params, frames, dec, T_known, n_it=40, lr=None):
    """Frame-to-model tracking (Sec. 3.4) over a sequence with a fixed map: the first
    len(T_known) frames keep the given poses; each later frame starts from the constant-velocity
    prediction of Eq. 19 (from one known pose only: that pose) and takes n_it pose-only steps of
    the tracking loss (Eq. 20-21) with Adam (moments reset per frame).  cam gives the
    intrinsics.  Returns the list of poses."""
    if lr is None:
        lr = np.array([2e-3, 2e-3, 2e-3, 4e-4, 4e-4, 4e-4])
    est = [np.asarray(T, np.float64) for T in T_known]
    for t in range(len(est), len(frames)):
        T = constant_velocity(est[-1], est[-2] if t >= 2 else est[-1])
        m, v = np.zeros(6), np.zeros(6)
        for it in range(1, n_it + 1):
            c = type(cam)(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, T)
            out = step(gs, c, prm, frames[t], dec, TRACKING)
            T, m, v = pose_step(T, out["grads"]["twist"], m, v, it, lr)
        est.append(T)
    return est


def ate_rmse(est, gt):
    """Absolute trajectory error: RMS distance between estimated and true camera centres."""
    centre = lambda T: -np.asarray(T)[:3, :3].T @ np.asarray(T)[:3, 3]
    return float(np.sqrt(np.mean([np.sum((centre(a) - centre(b)) ** 2) for a, b in zip(est, gt)])))


# --------------------------------------------------------------- SLAM loop
def rskm_select(k_m, t_opt, cur, keyframes, draw):
    """RSKM keyframe draw of Eq. 13 for mapping iteration k_m (0-based) of the current frame
    cur.  Where k_m mod t_opt = 0 the formula gives the current frame probability 1: it is
    taken.  Elsewhere every frame of the candidate set (the keyframe set K, in insertion
    order, together with the current frame when it is not a keyframe) has probability
    1/|K|: the candidate with index draw mod |candidates| is taken, draw a uniform 32-bit
    integer supplied by the caller."""
    if k_m % t_opt == 0:
        return cur
    cands = list(keyframes) + ([] if cur in keyframes else [cur])
    return cands[int(draw) % len(cands)]


@dataclasses.dataclass
class SlamConfig:
    """Iteration counts and intervals of the SLAM loop.  C.1 gives 40 tracking and 60
    mapping iterations per frame (Replica); the paper gives no value for t_opt, the first
    frame's k_init, or the keyframe interval (readings: 2, the mapping count, every 5th)."""
    n_track: int = 40
    n_map: int = 60
    n_init: int = 60
    t_opt: int = 2
    kf_every: int = 5
    tau_unobs: float = TAU_UNOBS


@dataclasses.dataclass
class Field:
    """A Gaussian field as FP64 arrays (the attributes the functions above read)."""
    means: np.ndarray
    quats: np.ndarray
    log_scales: np.ndarray
    opacity_logits: np.ndarray
    rgb: np.ndarray
    feat: np.ndarray

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


def _append(gs, new):
    cat = lambda a, b: np.concatenate([np.asarray(a, np.float64), np.asarray(b, np.float64).reshape(
        (-1,) + np.asarray(a).shape[1:])])
    return Field(*(cat(getattr(gs, k), new[k]) for k in ADAM_GROUPS))


def slam(frames, cam, prm: Params, dec, T0, draws, feat_bank, cfg: SlamConfig = SlamConfig()):
    """The GS3LAM loop over a sequence (Sec. 3.3-3.4), FP64.  For frame t: the pose (T0 for
    the first frame; later frames tracked for n_track steps from the constant-velocity
    prediction of Eq. 19 against the map so far); adaptive expansion (Eq. 11) of the map
    rendered at that pose, new features taken in order from feat_bank; every kf_every-th
    frame joins the keyframe set; then n_map mapping iterations (n_init for the first
    frame), each on the frame drawn by RSKM (Eq. 13, one word of draws per iteration,
    consumed in order) at its estimated pose, with the mapping loss (Eq. 14-18 with the
    D-SSIM term of Eq. 15) and an Adam step of every parameter group (C.1 rates; moments
    reset per frame, like the pose's).  The decoder stays fixed.  cam gives the
    intrinsics.  Returns the estimated poses, the final field, the frames drawn and the
    field size after each frame."""
    D = dec.W.shape[1]
    z = lambda *s: np.zeros(s, np.float64)
    gs = Field(z(0, 3), z(0, 4), z(0, 3), z(0), z(0, 3), z(0, D))
    at = lambda T: type(cam)(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, np.asarray(T, np.float64))
    lr_pose = np.array([2e-3, 2e-3, 2e-3, 4e-4, 4e-4, 4e-4])
    est, keyframes, picks, sizes = [], [], [], []
    n_drawn = n_feat = 0
    for t, frame in enumerate(frames):
        if t == 0:
            T = np.asarray(T0, np.float64)
        else:
            T = constant_velocity(est[-1], est[-2] if t >= 2 else est[-1])
            m, v = np.zeros(6), np.zeros(6)
            for it in range(1, cfg.n_track + 1):
                out = step(gs, at(T), prm, frame, dec, TRACKING)
                T, m, v = pose_step(T, out["grads"]["twist"], m, v, it, lr_pose)
        est.append(T)
        img = forward(gs, at(T), prm)[2]
        new = expand(img, frame, at(T), feat_bank[n_feat:], cfg.tau_unobs)
        n_feat += len(new["src_pix"])
        gs = _append(gs, new)
        if t % cfg.kf_every == 0:
            keyframes.append(t)
        p = {k: getattr(gs, k) for k in ADAM_GROUPS}
        m = {k: np.zeros_like(p[k]) for k in ADAM_GROUPS}
        v = {k: np.zeros_like(p[k]) for k in ADAM_GROUPS}
        for k_m in range(cfg.n_init if t == 0 else cfg.n_map):
            f = rskm_select(k_m, cfg.t_opt, t, keyframes, draws[n_drawn])
            n_drawn += 1
            picks.append(f)
            out = step(gs, at(est[f]), prm, frames[f], dec, MAPPING_SSIM)
            p, m, v = adam_step(p, out["grads"], m, v, k_m + 1, MAPPING_LR)
            gs = Field(*(p[k] for k in ADAM_GROUPS))
        sizes.append(gs.n)
    return dict(poses=est, gs=gs, picks=picks, sizes=sizes)
