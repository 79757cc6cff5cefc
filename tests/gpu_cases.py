"""Shared helpers of the GPU parity tests: seeded cases, the CUDA path, the oracle, comparison rules."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2603_27781_gb300 import raster, synth
from paper_2603_27781_gb300 import _lib as L

# Forward tolerances (FP32 vs FP64): rgb/sil/feat max abs, depth max relative.
TOL_ABS = 1e-5
TOL_DEPTH_REL = 1e-5
# Gradient tolerance: per group, max |g - r| <= 1e-3 max |r| and ||g - r|| <= 1e-3 ||r||.
TOL_GRAD = 1e-3
# A pixel whose nearest threshold decision (alpha_min, alpha_max, T_min) is within this
# relative distance in the oracle is excluded (FP32 rounding may decide it differently).
MARGIN = 1e-4
# A pixel whose blend amplifies relative rounding of the 2D covariances by more than this
# (oracle "sens": blend-weighted |A|dx^2 + 2|B dx dy| + |C|dy^2, halved) is excluded: at
# f32's ~1e-7 relative rounding of Sigma2D its value is not determined to 1e-5.
SENS_MAX = 100.0


def params_pair(**kw):
    return raster.RasterParams(**kw), oracle.Params(**kw)


def box_case(n=2000, d=16, w=64, h=48, fx=60.0, seed=0, T=None):
    gs = synth.box_field(n, d, seed=seed)
    cam = synth.camera(w, h, fx, cx=w / 2, cy=h / 2, T_cw=T)
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


def excluded_pixels(cam, orc_proj, gpu_proj, orc_img, tile=16):
    """Pixels where FP32 and FP64 may legitimately differ: tiles covered by a splat whose
    rectangle differs between the two projections, pixels whose nearest threshold decision
    lies within MARGIN (relative) in the oracle, and ill-conditioned pixels (SENS_MAX)."""
    W, H = cam.width, cam.height
    g_rect, _ = oracle.rects(gpu_proj["uv"], gpu_proj["radius"], W, H, tile)
    diff = np.nonzero(np.any(g_rect != orc_proj["rect"], axis=1))[0]
    tx = (W + tile - 1) // tile
    ty = (H + tile - 1) // tile
    bad_tiles = np.zeros((ty, tx), bool)
    for i in diff:
        for rc in (g_rect[i], orc_proj["rect"][i]):
            bad_tiles[rc[1]:rc[3], rc[0]:rc[2]] = True
    mask = np.repeat(np.repeat(bad_tiles, tile, 0), tile, 1)[:H, :W]
    mask |= orc_img["margin"] < MARGIN
    mask |= orc_img["sens"] > SENS_MAX
    return mask, len(diff)


def assert_forward_close(gimg, oimg, excl, D):
    keep = ~excl
    for k in ("rgb", "feat"):
        a, b = gimg[k], oimg[k]
        err = np.abs(a - b)[:, keep] if a.ndim == 3 else np.abs(a - b)[keep]
        if err.size:
            assert err.max() <= TOL_ABS, (k, float(err.max()))
    err = np.abs(gimg["sil"] - oimg["sil"])[keep]
    assert err.size == 0 or err.max() <= TOL_ABS, ("sil", float(err.max()))
    # depth: relative 1e-5 image-wise (max error over max depth, as for the gradient groups) and
    # per pixel wherever the pixel is covered (sil >= 0.5); a faint pixel's depth is a small sum
    # of weights whose f32 rounding is bounded by the silhouette tolerance instead
    d_o, d_g = oimg["depth"][keep], gimg["depth"][keep]
    if d_o.size:
        assert np.abs(d_g - d_o).max() <= TOL_DEPTH_REL * np.abs(oimg["depth"]).max(), ("depth", "image")
        cov = oimg["sil"][keep] >= 0.5
        if cov.any():
            err = np.abs(d_g[cov] - d_o[cov]) / np.abs(d_o[cov])
            assert err.max() <= TOL_DEPTH_REL, ("depth", float(err.max()))
    np.testing.assert_array_equal(gimg["n_contrib"][keep], oimg["n_contrib"][keep])


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
    grads_v, P_off = [], 0
    for v, cam in enumerate(cams):
        sl = slice(v * gs.n, (v + 1) * gs.n)
        gpv = {k: a[sl] for k, a in gp.items()}
        excl, _ = excluded_pixels(cam, projs[v], gpv, oimgs[v])
        assert_forward_close(np_images(r, v), oimgs[v], excl, gs.feat_dim)
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
    D = gs.feat_dim
    got = dict(means=r.d_means, quats=r.d_quats, log_scales=r.d_log_scales, opacity_logits=r.d_logits, rgb=r.d_rgb,
               feat=r.d_feat[:, :D], twist=r.d_twist)
    for k, t in got.items():
        if k == "feat" and D == 0:
            continue
        assert_grad_close(k, t.cpu().numpy(), ob[k])
    return r, ob
