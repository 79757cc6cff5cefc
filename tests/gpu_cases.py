"""Shared helpers of the GPU parity tests: seeded cases, the CUDA path, the oracle, comparison rules."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

import oracle
from paper_2603_27781_gb300 import raster, synth
from paper_2603_27781_gb300 import _lib as L

# Forward tolerances (FP32 vs FP64): rgb/sil/feat max abs, depth max relative (per pixel).
TOL_ABS = 1e-5
TOL_DEPTH_REL = 1e-5
# Gradient tolerance: per group, max |g - r| <= 1e-3 max |r| and ||g - r|| <= 1e-3 ||r||.
TOL_GRAD = 1e-3
# The oracle states, per pixel, how well single-precision inputs determine it (render_fwd's
# margin, sens, sens_depth: first-order bounds in units of a 1e-7 relative rounding of each
# splat's 2D covariance and alpha).  A pixel is excluded from the element-wise comparison (and
# counted) when a threshold decision is within MARGIN_MIN of its rounding bound, or when its
# rounding bound exceeds the gradient tolerance (SENS_CUT x 1e-7 = 1e-3).  Where the bound
# exceeds the forward tolerance (SENS_MAX x 1e-7 = 1e-5), that pixel's forward tolerance is
# widened to WIDEN times its bound (absolute for colour, silhouette and features, relative
# for the depth) and the pixel is still compared.
MARGIN_MIN = 10.0
SENS_MAX = 100.0
SENS_CUT = 1e4
WIDEN = 2.0
# Largest excluded share of the compared pixels.
EXCL_MAX = 5e-3


def params_pair(**kw):
    return raster.RasterParams(**kw), oracle.Params(**kw)


def box_case(n=2000, d=16, w=64, h=48, fx=60.0, seed=0, T=None):
    gs = synth.box_field(n, d, seed=seed)
    cam = synth.camera(w, h, fx, cx=w / 2, cy=h / 2, T_cw=T)
    return gs, cam


def offview_case(seed=7):
    """Box scene with 300 of its 2,000 Gaussians moved beside the view, their centres at
    |x/z| in [0.72, 1.0] (the Jacobian clamp starts at 0.69 for this camera), scales e times
    larger, so their tails reach into the image: the clamped and the exact Jacobian of Eq. 3
    give them different footprints."""
    gs = synth.box_field(2000, 8, seed=seed)
    cam = synth.camera(64, 48, 60.0, cx=32, cy=24)
    g = synth.rng(seed + 1)
    k = 300
    z = gs.means[:k, 2]
    side = np.where(g.random(k) < 0.5, -1.0, 1.0)
    gs.means[:k, 0] = (side * g.uniform(0.72, 1.0, k) * z).astype(np.float32)
    gs.log_scales[:k] += np.float32(1.0)
    return gs, cam


def room_case(n, d=16, w=1200, h=680, fx=600.0, seed=0):
    room = synth.make_room(seed)
    gs = synth.room_field(n, d, seed=seed, room=room)
    cam = synth.room_camera(w, h, fx, room=room)
    return gs, cam, room


def gpu_forward(gs, cams, prm, capacity=None, want_keys=True, rgb_dtype=torch.float32, feat_dtype=torch.float32,
                n_classes=0):
    field = raster.Field.from_numpy(gs, "cuda", rgb_dtype, feat_dtype)
    cams = cams if isinstance(cams, (list, tuple)) else [cams]
    if capacity is None:
        r = raster.fit_capacity(field, cams, gs.feat_dim, params=prm, n_classes=n_classes)
    else:
        r = raster.Renderer(gs.n, cams, gs.feat_dim, capacity, params=prm, n_classes=n_classes)
    r.forward(field, want_keys=want_keys)
    torch.cuda.synchronize()
    return field, r


def gpu_projection(r):
    """uv: the f32 centre the binning uses; uv_full: f32 centre plus its low part."""
    uvdo = r.uvdo.cpu().numpy()
    conic = r.conic.cpu().numpy()
    lo = r.uv_lo.cpu().numpy().astype(np.float64)
    return dict(uv=uvdo[:, :2].astype(np.float64), uv_full=uvdo[:, :2].astype(np.float64) + lo, depth=uvdo[:, 2],
                opacity=uvdo[:, 3], conic=conic[:, :3], radius=conic[:, 3].astype(np.int32),
                touched=r.touched.cpu().numpy())


def gpu_binning(r):
    m = r.instances()
    return (r.keys[:m].cpu().numpy().view(np.uint64), r.vals[:m].cpu().numpy().view(np.uint32),
            r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2))


@dataclasses.dataclass
class Exclusion:
    """Pixels where FP32 and FP64 may legitimately differ, by reason: rect (a splat whose tile
    rectangle differs between the two projections can be blended there), margin (a threshold
    decision within MARGIN_MIN of its rounding bound) and cond (rounding bound above the
    gradient tolerance).  shifted: the tiles where such a splat is in one list only, whose
    later list positions (n_contrib) differ by one while the images agree.  widened: pixels
    compared with a forward tolerance widened to their rounding bound."""
    rect: np.ndarray
    margin: np.ndarray
    cond: np.ndarray
    shifted: np.ndarray
    widened: np.ndarray
    n_rect_splats: int

    @property
    def mask(self):
        return self.rect | self.margin | self.cond

    def report(self, region=None):
        r = np.ones_like(self.mask) if region is None else region
        n = int(r.sum())
        parts = {k: int((getattr(self, k) & r).sum()) for k in ("rect", "margin", "cond", "widened", "shifted")}
        tot = int((self.mask & r).sum())
        return (f"excluded {tot} of {n} pixels ({tot / max(n, 1):.3%}): rect {parts['rect']} "
                f"({self.n_rect_splats} splats), margin {parts['margin']}, cond {parts['cond']}; "
                f"tolerance widened at {parts['widened']}, list positions shifted at {parts['shifted']}")

    def check(self, where, region=None, limit=EXCL_MAX):
        r = np.ones_like(self.mask) if region is None else region
        frac = (self.mask & r).sum() / max(int(r.sum()), 1)
        print(f"{where}: {self.report(region)}")
        assert frac <= limit, (where, self.report(region))
        return self


def exclusion(cam, orc_proj, gpu_proj, orc_img, alpha_min=1.0 / 255.0, tile=16):
    """The Exclusion of one view: orc_proj / orc_img from the oracle, gpu_proj the GPU's
    projection of the same Gaussians (same order).  A splat whose rectangle differs changes a
    pixel's list only in the tiles one rectangle has and the other lacks, and only where it
    can be blended (its oracle alpha reaches half of alpha_min; every pixel of those tiles
    when alpha_min is 0)."""
    W, H = cam.width, cam.height
    g_rect, _ = oracle.rects(gpu_proj["uv"], gpu_proj["radius"], W, H, tile)
    o_rect = orc_proj["rect"]
    diff = np.nonzero(np.any(g_rect != o_rect, axis=1))[0]
    rect = np.zeros((H, W), bool)
    shifted = np.zeros((H, W), bool)
    for i in diff:
        cover = np.zeros(((H + tile - 1) // tile, (W + tile - 1) // tile), np.int8)
        for rc in (g_rect[i], o_rect[i]):
            cover[rc[1]:rc[3], rc[0]:rc[2]] += 1
        sym = np.repeat(np.repeat(cover == 1, tile, 0), tile, 1)[:H, :W]
        if not sym.any():
            continue
        shifted |= sym
        ys, xs = np.nonzero(sym)
        if alpha_min > 0 and orc_proj["radius"][i] > 0:
            A, B, C = orc_proj["conic"][i]
            dx, dy = xs + 0.5 - orc_proj["uv"][i, 0], ys + 0.5 - orc_proj["uv"][i, 1]
            a = orc_proj["opacity"][i] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
            keep = a >= 0.5 * alpha_min
            ys, xs = ys[keep], xs[keep]
        rect[ys, xs] = True
    margin = orc_img["margin"] < MARGIN_MIN
    cond = (orc_img["sens"] > SENS_CUT) | (orc_img["sens_depth"] > SENS_CUT)
    widened = ~cond & ((orc_img["sens"] > SENS_MAX) | (orc_img["sens_depth"] > SENS_MAX))
    return Exclusion(rect, margin, cond, shifted, widened, len(diff))


def excluded_pixels(cam, orc_proj, gpu_proj, orc_img, tile=16, alpha_min=1.0 / 255.0):
    ex = exclusion(cam, orc_proj, gpu_proj, orc_img, alpha_min, tile)
    return ex.mask, ex.n_rect_splats


def assert_forward_close(gimg, oimg, excl, D, shifted=None):
    """Element-wise forward parity on the pixels not in excl: colour, silhouette and features
    within TOL_ABS, depth within TOL_DEPTH_REL of the oracle's depth (0 where nothing is
    blended), each widened to WIDEN times the pixel's first-order rounding bound where that is
    larger; the last contributor equal outside the shifted tiles."""
    keep = ~excl
    tol = np.maximum(TOL_ABS, WIDEN * 1e-7 * oimg["sens"])[keep]
    for k in ("rgb", "feat"):
        a, b = gimg[k], oimg[k]
        err = np.abs(a - b)[:, keep] if a.ndim == 3 else np.abs(a - b)[keep]
        if err.size:
            assert (err <= tol).all(), (k, float(err.max()), float((err / tol).max()))
    err = np.abs(gimg["sil"] - oimg["sil"])[keep]
    assert err.size == 0 or (err <= tol).all(), ("sil", float(err.max()), float((err / tol).max()))
    d_o, d_g = oimg["depth"][keep], gimg["depth"][keep]
    if d_o.size:
        rel = np.maximum(TOL_DEPTH_REL, WIDEN * 1e-7 * oimg["sens_depth"][keep])
        err = np.abs(d_g - d_o)
        bad = err > rel * np.abs(d_o)
        assert not bad.any(), ("depth", int(bad.sum()), float((err / np.maximum(rel * np.abs(d_o), 1e-300)).max()))
    same = keep if shifted is None else keep & ~shifted
    np.testing.assert_array_equal(gimg["n_contrib"][same], oimg["n_contrib"][same])


def rounding_report(gimg, oimg, excl):
    """Observed FP32 error over the oracle's first-order rounding bound plus an allowance of
    1e-6 (a tenth of the tolerance) for the rounding of the sums themselves, which the figure
    does not model: |err| / (1e-7 sens + 1e-6) for colour, silhouette and features,
    |err| / ((1e-7 sens_depth + 1e-6) |depth|) for the depth, on the kept pixels (max, 99.9 %
    quantile per output)."""
    keep = ~excl
    out = {}
    for k in ("rgb", "sil", "feat", "depth"):
        e = np.abs(gimg[k] - oimg[k])
        if k == "depth":
            b = (1e-7 * oimg["sens_depth"] + 1e-6) * np.abs(oimg["depth"])
        else:
            b = 1e-7 * oimg["sens"] + 1e-6
        ratio = np.where(e > 0, e / np.maximum(b, 1e-300), 0.0)
        ratio = ratio[:, keep] if ratio.ndim == 3 else ratio[keep]
        out[k] = (float(ratio.max()), float(np.quantile(ratio, 0.999))) if ratio.size else (0.0, 0.0)
    return out


def assert_grad_close(name, g, r, tol=TOL_GRAD):
    g = np.asarray(g, np.float64).ravel()
    r = np.asarray(r, np.float64).ravel()
    rmax = np.abs(r).max()
    if rmax == 0:
        assert np.abs(g).max() == 0, name
        return
    emax = np.abs(g - r).max()
    assert emax <= tol * rmax, (name, float(emax), float(rmax))
    assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r), (name, float(np.linalg.norm(g - r)),
                                                             float(np.linalg.norm(r)))


def np_images(r, view=0):
    im = r.images(view)
    return {k: v.cpu().numpy().astype(np.float64) if v.dtype != torch.int32 else v.cpu().numpy()
            for k, v in im.items()}


def random_image_grads(P, D, seed, scale=1.0):
    g = synth.rng(seed)
    return dict(rgb=scale * g.standard_normal((3, P)), depth=scale * g.standard_normal(P),
                sil=scale * g.standard_normal(P), feat=scale * g.standard_normal((D, P)))


def oracle_multiview(gs, cams, prm):
    """Oracle projection of every view, one joint binning over all views, per-view blends."""
    projs = [oracle.project(gs, c, prm) for c in cams]
    rect = np.concatenate([p["rect"] for p in projs])
    dk = np.concatenate([p["depth_key"] for p in projs])
    keys, vals, ranges = oracle.bin_sort(rect, dk, cams, prm.tile, n_per_view=gs.n)
    imgs, toff = [], 0
    for v, c in enumerate(cams):
        imgs.append(oracle.render_fwd(c, projs[v], gs.rgb, gs.feat, vals, ranges, prm, view_offset=v * gs.n,
                                      tile_offset=toff))
        toff += ((c.width + 15) // 16) * ((c.height + 15) // 16)
    return projs, (keys, vals, ranges), imgs


def oracle_multiview_backward(gs, cams, prm, projs, bins, grads_per_view):
    _, vals, ranges = bins
    out = dict(means=0, quats=0, log_scales=0, opacity_logits=0, rgb=0, feat=0)
    twists, toff = [], 0
    for v, c in enumerate(cams):
        g = grads_per_view[v]
        r = oracle.render_bwd(c, projs[v], gs.rgb, gs.feat, vals, ranges, prm, g["rgb"], g["depth"], g["sil"],
                              g["feat"], view_offset=v * gs.n, tile_offset=toff)
        p = oracle.project_bwd(gs, c, prm, r["uv"], r["conic"], r["opacity"], r["depth"])
        for k in ("means", "quats", "log_scales", "opacity_logits"):
            out[k] = out[k] + p[k]
        out["rgb"] = out["rgb"] + r["rgb"]
        out["feat"] = out["feat"] + r["feat"]
        twists.append(p["twist"])
        toff += ((c.width + 15) // 16) * ((c.height + 15) // 16)
    out["twist"] = np.stack(twists)
    return out


def bwd_compare(gs, cams, prm_g, prm_o, seed=7, rgb_dtype=torch.float32, feat_dtype=torch.float32,
                gs_oracle=None):
    """Forward images and every gradient of the CUDA path against the oracle, over several views,
    for random upstream image gradients that are zero at pixels excluded by the comparison rules."""
    field, r = gpu_forward(gs, cams, prm_g, rgb_dtype=rgb_dtype, feat_dtype=feat_dtype)
    gso = gs if gs_oracle is None else gs_oracle
    projs, bins, oimgs = oracle_multiview(gso, cams, prm_o)
    gp = gpu_projection(r)
    grads_v, P_off, excls = [], 0, []
    for v, cam in enumerate(cams):
        sl = slice(v * gs.n, (v + 1) * gs.n)
        gpv = {k: a[sl] for k, a in gp.items()}
        ex = exclusion(cam, projs[v], gpv, oimgs[v], prm_o.alpha_min).check(f"view {v} ({cam.width}x{cam.height})")
        excls.append(ex)
        excl = ex.mask
        assert_forward_close(np_images(r, v), oimgs[v], excl, gs.feat_dim, ex.shifted)
        P = cam.width * cam.height
        g = random_image_grads(P, gs.feat_dim, seed + v)
        keep = ~excl.ravel()
        for k in g:
            g[k] = g[k] * keep
        grads_v.append({k: a.reshape((-1, cam.height, cam.width) if a.ndim == 2 else (cam.height, cam.width))
                        for k, a in g.items()})
        # upload into the renderer's image-gradient buffers
        a, b = r.pix_off[v], r.pix_off[v + 1]
        r.g_rgb[:, a:b] = torch.as_tensor(g["rgb"], dtype=torch.float32)
        r.g_depth[a:b] = torch.as_tensor(g["depth"], dtype=torch.float32)
        r.g_sil[a:b] = torch.as_tensor(g["sil"], dtype=torch.float32)
        if gs.feat_dim:
            r.g_feat[:, a:b] = torch.as_tensor(g["feat"], dtype=torch.float32)
    r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
    torch.cuda.synchronize()
    ob = oracle_multiview_backward(gso, cams, prm_o, projs, bins, grads_v)
    ob["images"], ob["exclusions"] = oimgs, excls
    D = gs.feat_dim
    got = dict(means=r.d_means, quats=r.d_quats, log_scales=r.d_log_scales, opacity_logits=r.d_logits, rgb=r.d_rgb,
               feat=r.d_feat[:, :D], twist=r.d_twist)
    for k, t in got.items():
        if k == "feat" and D == 0:
            continue
        assert_grad_close(k, t.cpu().numpy(), ob[k])
    return r, ob
