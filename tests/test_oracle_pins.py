"""Pins of the FP64 oracle to what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed
form, an invariant, a textbook or library routine, brute force on tiny inputs,
or central finite differences.  Between them a dropped term, a wrong sign or
index, or a transposed operand anywhere in the oracle fails at least one.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg
import scipy.special
from scipy.spatial.transform import Rotation

import oracle
from oracle import Params
from paper_2603_27781_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))

# Literal Eq. 4-7: no thresholds, no early stop, radius wide enough to cover the image.
EXACT = Params(alpha_min=0.0, alpha_max=1.0, T_min=0.0, lowpass=0.0, radius_sigma=40.0)


def field(means, quats, log_scales, logits, rgb, feat):
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64))
    return synth.Gaussians(f(means), f(quats), f(log_scales), f(logits), f(rgb), f(feat))


def camera(*args, **kw):
    """Cameras of the pins keep their exact float64 values (finite differences perturb them)."""
    return synth.camera(*args, round_f32=False, **kw)


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


# ----------------------------------------------------------------- closed forms
@pytest.mark.parametrize("rot90", [False, True])
def test_single_gaussian_closed_form(rot90):
    """Eq. 2-7 for one Gaussian on the optical axis: Sigma2D = diag((f s_x / z)^2, (f s_y / z)^2)."""
    cam = camera(33, 33, 40.0, cx=16.5, cy=16.5)
    q = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)] if rot90 else [1, 0, 0, 0]
    s = np.array([0.1, 0.05, 0.2])
    logit = 0.3
    c = np.array([0.2, 0.5, 0.9])
    f = np.array([1.0, -2.0, 3.0, 0.5])
    gs = field([[0, 0, 2.0]], [q], [np.log(s)], [logit], [c], [f])
    proj, bins, img = oracle.forward(gs, cam, EXACT)
    sx, sy = 40 * 0.1 / 2, 40 * 0.05 / 2           # 2 px and 1 px
    if rot90:                                        # 90 deg about the optical axis swaps them
        sx, sy = sy, sx
    o = sigmoid(logit)
    py, px = np.mgrid[0:33, 0:33]
    dx, dy = px + 0.5 - 16.5, py + 0.5 - 16.5
    alpha = o * np.exp(-0.5 * (dx ** 2 / sx ** 2 + dy ** 2 / sy ** 2))
    np.testing.assert_allclose(proj["uv"][0], [16.5, 16.5], rtol=0, atol=1e-12)
    np.testing.assert_allclose(proj["cov2d"][0], [sx ** 2, 0, sy ** 2], rtol=1e-12, atol=1e-12)
    for ch in range(3):
        np.testing.assert_allclose(img["rgb"][ch], alpha * c[ch], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(img["depth"], alpha * 2.0, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(img["sil"], alpha, rtol=1e-12, atol=1e-15)
    for d in range(4):
        np.testing.assert_allclose(img["feat"][d], alpha * f[d], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(img["T"], 1 - alpha, rtol=1e-12, atol=1e-15)
    assert (img["n_contrib"] == 1).all()
    # centre pixel: rgb = o c, depth = o z, sil = o, feat = o f
    assert img["sil"][16, 16] == pytest.approx(o, abs=1e-15)
    # radius = ceil(3 sqrt(lambda_max)) = ceil(3 * 2) with lowpass 0
    p3 = Params(lowpass=0.0)
    assert oracle.project(gs, cam, p3)["radius"][0] == 6


def test_pinhole_centre_and_depth():
    """The projected centre is K [R|t] mu (homogeneous pinhole, supp. B.1) and d = camera z."""
    g = synth.rng(11)
    T = synth.look_pose((0.3, -0.2, 0.1), (0.2, 1.0, 0.3))
    cam = camera(200, 150, 180.0, 170.0, 97.0, 71.0, T_cw=T)
    n = 50
    mu = T[:3, :3].T @ (np.stack([g.uniform(-1, 1, n), g.uniform(-1, 1, n), g.uniform(1, 4, n)]) - T[:3, 3:4])
    gs = field(mu.T, np.tile([1.0, 0, 0, 0], (n, 1)), np.full((n, 3), -3.0), np.zeros(n),
               np.zeros((n, 3)), np.zeros((n, 1)))
    proj = oracle.project(gs, cam, Params())
    K = np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1]])
    h = K @ cam.T_cw[:3, :] @ np.vstack([mu, np.ones(n)])
    np.testing.assert_allclose(proj["uv"], (h[:2] / h[2]).T, rtol=1e-12)
    np.testing.assert_allclose(proj["depth"], h[2], rtol=1e-12)
    np.testing.assert_allclose(proj["depth_key"], h[2].astype(np.float32), rtol=2e-7)


def test_ewa_covariance_matches_monte_carlo():
    """Eq. 3 is the linearisation of the pinhole map: compare with sampled projections."""
    g = synth.rng(12)
    T = synth.look_pose((0.0, 0.0, 0.0), (0.3, 1.0, -0.2))
    cam = camera(640, 480, 500.0, 520.0, 320.0, 240.0, T_cw=T)
    q_wxyz = g.standard_normal(4)
    q_wxyz /= np.linalg.norm(q_wxyz)
    s = np.array([0.02, 0.008, 0.014])
    p_cam = np.array([0.5, -0.35, 2.5])
    mu = T[:3, :3].T @ (p_cam - T[:3, 3])
    gs = field([mu], [q_wxyz], [np.log(s)], [0.0], [[0, 0, 0]], [[0.0]])
    proj = oracle.project(gs, cam, Params(lowpass=0.0))
    R = Rotation.from_quat([q_wxyz[1], q_wxyz[2], q_wxyz[3], q_wxyz[0]]).as_matrix()
    Sigma = R @ np.diag(s ** 2) @ R.T
    x = g.multivariate_normal(mu, Sigma, 400_000)
    pc = x @ T[:3, :3].T + T[:3, 3]
    uv = np.stack([500.0 * pc[:, 0] / pc[:, 2] + 320.0, 520.0 * pc[:, 1] / pc[:, 2] + 240.0], 1)
    C = np.cov(uv.T)
    a, b, c = proj["cov2d"][0]
    scale = math.sqrt(a * c)
    np.testing.assert_allclose([a, b, c], [C[0, 0], C[0, 1], C[1, 1]], rtol=0, atol=1.5e-2 * scale)
    # the conic is the inverse of Sigma2D
    A, B, Cc = proj["conic"][0]
    np.testing.assert_allclose(np.array([[A, B], [B, Cc]]) @ np.array([[a, b], [b, c]]), np.eye(2),
                               atol=1e-12)


def test_joint_rigid_motion_leaves_image_unchanged():
    """Moving the world and the camera by the same rigid motion gives the same render."""
    gs = synth.box_field(60, 4, seed=21)
    cam = camera(48, 40, 50.0, cx=24, cy=20)
    base = oracle.forward(gs, cam, EXACT)[2]
    Q = Rotation.from_rotvec([0.3, -0.5, 0.8]).as_matrix()
    shift = np.array([0.4, -1.0, 2.0])
    moved = gs.copy()
    moved.means = (gs.means.astype(np.float64) @ Q.T + shift)
    rq = Rotation.from_matrix(Q)
    qs = gs.quats.astype(np.float64)
    prod = (rq * Rotation.from_quat(np.c_[qs[:, 1:], qs[:, :1]])).as_quat()
    moved.quats = np.c_[prod[:, 3:], prod[:, :3]]
    M = np.eye(4)
    M[:3, :3], M[:3, 3] = Q, shift
    cam2 = camera(48, 40, 50.0, cx=24, cy=20, T_cw=np.linalg.inv(M))
    img2 = oracle.forward(moved, cam2, EXACT)[2]
    for k in ("rgb", "depth", "sil", "feat"):
        np.testing.assert_allclose(img2[k], base[k], atol=1e-9)


def test_two_gaussians_front_to_back():
    """Eq. 4: c = a1 c1 + a2 (1 - a1) c2 with the nearer splat first, whatever the input order."""
    cam = camera(17, 17, 30.0, cx=8.5, cy=8.5)
    c1, c2 = [0.9, 0.1, 0.2], [0.1, 0.8, 0.3]
    l1, l2 = 0.7, -0.2
    a1, a2 = sigmoid(l1), sigmoid(l2)

    def render(order, z1, z2):
        rows = [([0, 0, z1], c1, l1), ([0, 0, z2], c2, l2)]
        rows = [rows[i] for i in order]
        gs = field([r[0] for r in rows], [[1, 0, 0, 0]] * 2, [[-2.5] * 3] * 2, [r[2] for r in rows],
                   [r[1] for r in rows], [[0.0]] * 2)
        return oracle.forward(gs, cam, EXACT)[2]

    for order in ([0, 1], [1, 0]):
        img = render(order, 2.0, 3.0)
        want = a1 * np.array(c1) + a2 * (1 - a1) * np.array(c2)
        np.testing.assert_allclose(img["rgb"][:, 8, 8], want, rtol=1e-12)
        assert img["depth"][8, 8] == pytest.approx(a1 * 2.0 + a2 * (1 - a1) * 3.0, rel=1e-12)
        assert img["T"][8, 8] == pytest.approx((1 - a1) * (1 - a2), rel=1e-12)
    img = render([0, 1], 3.0, 2.0)
    want = a2 * np.array(c2) + a1 * (1 - a2) * np.array(c1)
    np.testing.assert_allclose(img["rgb"][:, 8, 8], want, rtol=1e-12)


def test_early_stop_at_min_transmittance():
    """A splat that would take T below T_min ends the pixel's blend: later splats are not
    blended even when their own alpha would keep T above T_min."""
    cam = camera(9, 9, 20.0, cx=4.5, cy=4.5)
    alphas = [0.95, 0.95, 0.95, 0.95, 0.1]
    logits = [math.log(a / (1 - a)) for a in alphas]
    cols = synth.rng(70).random((5, 3))
    gs = field([[0, 0, 2.0 + 0.1 * k] for k in range(5)], [[1, 0, 0, 0]] * 5, [[-2.0] * 3] * 5, logits,
               cols, [[0.0]] * 5)
    prm = Params(alpha_max=0.99, T_min=1e-4, lowpass=0.0)
    img = oracle.forward(gs, cam, prm)[2]
    o = [sigmoid(l) for l in logits]
    T, want = 1.0, np.zeros(3)
    for k in range(3):                   # T: 0.05, 0.0025, 1.25e-4; the 4th would give 6.25e-6
        want += o[k] * T * cols[k]
        T *= 1 - o[k]
    assert img["n_contrib"][4, 4] == 3
    assert img["T"][4, 4] == pytest.approx(T, rel=1e-12)
    np.testing.assert_allclose(img["rgb"][:, 4, 4], want, rtol=1e-12)


def test_empty_and_fully_culled_maps_render_background():
    cam = camera(40, 24, 30.0)
    prm = Params(bg=(0.1, 0.2, 0.3))
    for gs in (field(np.zeros((0, 3)), np.zeros((0, 4)), np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3)),
                     np.zeros((0, 8))),
               synth.box_field(30, 8, seed=3)):
        if gs.n:
            gs.means[:, 2] = -gs.means[:, 2]          # everything behind the camera
        proj, bins, img = oracle.forward(gs, cam, prm)
        assert len(bins[0]) == 0
        for ch in range(3):
            assert (img["rgb"][ch] == prm.bg[ch]).all()
        assert (img["depth"] == 0).all() and (img["sil"] == 0).all() and (img["feat"] == 0).all()
        assert (img["T"] == 1).all() and (img["n_contrib"] == 0).all()
        g = dict(rgb=np.ones((3, 24, 40)), depth=np.ones((24, 40)), sil=np.ones((24, 40)),
                 feat=np.ones((8, 24, 40)))
        gr = oracle.backward_from_image_grads(gs, cam, prm, proj, bins, g)
        for k in ("means", "quats", "log_scales", "opacity_logits", "rgb", "feat", "twist"):
            assert not np.any(gr[k])


def test_silhouette_plus_transmittance_is_one():
    gs = synth.box_field(500, 8, seed=5)
    cam = camera(64, 48, 60.0, cx=32, cy=24)
    img = oracle.forward(gs, cam, Params())[2]
    np.testing.assert_allclose(img["sil"] + img["T"], 1.0, atol=1e-12)
    assert img["sil"].max() > 0.9


def test_input_order_invariance():
    gs = synth.box_field(300, 8, seed=6)
    cam = camera(64, 48, 60.0, cx=32, cy=24)
    base = oracle.forward(gs, cam, Params())[2]
    perm = synth.rng(9).permutation(gs.n)
    img = oracle.forward(gs.subset(perm), cam, Params())[2]
    for k in ("rgb", "depth", "sil", "feat", "T", "n_contrib"):
        assert np.array_equal(img[k], base[k]), k


# ------------------------------------------------------------- brute force
def brute_force_render(gs, cam, prm, use_tiles=True):
    """Per-pixel loop over every Gaussian (no tile lists): the blend rule of Eq. 4-7 plus
    the thresholds, with the tile-membership rule applied pixel by pixel."""
    proj = oracle.project(gs, cam, prm)
    W, H, D = cam.width, cam.height, gs.feat.shape[1]
    order = sorted(range(gs.n), key=lambda i: (float(proj["depth_key"][i]), i))
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), sil=np.zeros((H, W)),
               feat=np.zeros((D, H, W)), T=np.zeros((H, W)), prodT=np.zeros((H, W)))
    for py in range(H):
        for px in range(W):
            T, prod = 1.0, 1.0
            acc = np.zeros(5 + D)
            tx, ty = px // prm.tile, py // prm.tile
            for i in order:
                if use_tiles:
                    x0, y0, x1, y1 = proj["rect"][i]
                    if proj["radius"][i] <= 0 or not (x0 <= tx < x1 and y0 <= ty < y1):
                        continue
                elif not proj["depth"][i] > prm.z_near:
                    continue
                u, v = proj["uv"][i]
                A, B, C = proj["conic"][i]
                dx, dy = px + 0.5 - u, py + 0.5 - v
                power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
                if power > 0:
                    continue
                alpha = min(prm.alpha_max, proj["opacity"][i] * math.exp(power))
                if alpha < prm.alpha_min:
                    continue
                if T * (1 - alpha) < prm.T_min:
                    break
                w = alpha * T
                acc[:3] += w * gs.rgb[i]
                acc[3] += w * proj["depth"][i]
                acc[4] += w
                acc[5:] += w * gs.feat[i]
                T *= 1 - alpha
                prod *= 1 - alpha
            out["rgb"][:, py, px] = acc[:3] + T * np.array(prm.bg)
            out["depth"][py, px] = acc[3]
            out["sil"][py, px] = acc[4]
            out["feat"][:, py, px] = acc[5:]
            out["T"][py, px] = T
            out["prodT"][py, px] = prod
    return out


@pytest.mark.parametrize("dense", [False, True])
def test_tiled_equals_brute_force(dense):
    gs = synth.box_field(200 if dense else 40, 3, seed=7)
    gs.log_scales[:] += 0.8 if dense else -0.5
    if dense:
        gs.opacity_logits[:] += 2.0
    cam = camera(32, 32, 60.0 if dense else 30.0, cx=16, cy=16)
    prm = Params()
    img = oracle.forward(gs, cam, prm)[2]
    bf = brute_force_render(gs, cam, prm)
    if dense:   # the T_min stop and the alpha_max clamp are exercised
        assert (img["T"] < 1e-3).sum() > 50
    for k in ("rgb", "depth", "sil", "feat", "T"):
        np.testing.assert_allclose(img[k], bf[k], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(img["T"], bf["prodT"], rtol=1e-12)   # T_final = prod(1 - alpha)


def test_exact_mode_equals_literal_eq4_sum():
    """With no thresholds and a covering radius the tiled blend is the literal sum of Eq. 4."""
    gs = synth.box_field(30, 2, seed=8)
    cam = camera(32, 24, 30.0, cx=16, cy=12)
    img = oracle.forward(gs, cam, EXACT)[2]
    bf = brute_force_render(gs, cam, EXACT, use_tiles=False)
    for k in ("rgb", "depth", "sil", "feat"):
        np.testing.assert_allclose(img[k], bf[k], rtol=1e-11, atol=1e-14)


# ------------------------------------------------------------ binning and sort
def test_tile_rect_matches_interval_intersection():
    g = synth.rng(13)
    u = np.concatenate([g.uniform(-40, 140, 300), np.arange(-20, 120, 1.0), np.arange(-20, 120, 16.0) - 1e-9])
    v = g.uniform(-40, 100, u.shape[0])
    r = g.integers(1, 40, u.shape[0]).astype(np.int32)
    W, H, tile = 100, 60, 16
    rect, touched = oracle.rects(np.c_[u, v], r, W, H, tile)
    tx, ty = (W + 15) // 16, (H + 15) // 16
    for i in range(u.shape[0]):
        def span(c, n):
            lo, hi = Fraction(c) - int(r[i]), Fraction(c) + int(r[i])
            inside = [t for t in range(n) if tile * t <= hi and tile * (t + 1) > lo]
            return (inside[0], inside[-1] + 1) if inside else None
        sx, sy = span(u[i], tx), span(v[i], ty)
        if sx is None or sy is None:
            assert touched[i] == 0
        else:
            assert tuple(rect[i]) == (sx[0], sy[0], sx[1], sy[1])
            assert touched[i] == (sx[1] - sx[0]) * (sy[1] - sy[0])


def test_bin_sort_matches_per_tile_brute_force():
    gs = synth.box_field(120, 2, seed=14)
    cams = [camera(64, 48, 60.0, cx=32, cy=24),
            camera(40, 40, 50.0, T_cw=synth.look_pose((0.2, 0, 0), (0.05, 0.0, 1.0), up=(0, -1, 0)))]
    projs = [oracle.project(gs, c, Params()) for c in cams]
    rect = np.concatenate([p["rect"] for p in projs])
    dk = np.concatenate([p["depth_key"] for p in projs])
    dk[5] = dk[6]                        # force an equal-depth tie
    keys, vals, ranges = oracle.bin_sort(rect, dk, cams)
    tile_base = 0
    for v, cam in enumerate(cams):
        tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
        for t in range(tx * ty):
            x, y = t % tx, t // tx
            members = [v * gs.n + i for i in range(gs.n)
                       if projs[v]["rect"][i][0] <= x < projs[v]["rect"][i][2]
                       and projs[v]["rect"][i][1] <= y < projs[v]["rect"][i][3]]
            members.sort(key=lambda j: (float(dk[j]), j))
            s, e = ranges[tile_base + t]
            assert list(vals[s:e]) == members
            for j, m in zip(range(s, e), members):
                assert int(keys[j]) == ((tile_base + t) << 32) | int(dk[m:m + 1].view(np.uint32)[0])
        tile_base += tx * ty


# ------------------------------------------------------------ finite differences
def _render_functional(gs, cam, prm, g):
    img = oracle.forward(gs, cam, prm)[2]
    return sum(float((img[k] * g[k]).sum()) for k in ("rgb", "depth", "sil", "feat"))


def _fd_setup(seed, prm):
    gs = synth.box_field(14, 4, seed=seed)
    gs = synth.Gaussians(*(a.astype(np.float64) for a in gs.arrays()))
    gs.log_scales += 0.6
    T = synth.look_pose((0.1, -0.05, -0.2), (0.05, 0.03, 1.0), up=(0, -1, 0))
    cam = camera(24, 20, 22.0, cx=11.7, cy=10.2, T_cw=T)
    g = synth.rng(seed + 100)
    H, W = cam.height, cam.width
    gimg = dict(rgb=g.standard_normal((3, H, W)), depth=g.standard_normal((H, W)),
                sil=g.standard_normal((H, W)), feat=g.standard_normal((4, H, W)))
    return gs, cam, gimg


def _se3_exp(xi):
    M = np.zeros((4, 4))
    rho, phi = xi[:3], xi[3:]
    M[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    M[:3, 3] = rho
    return scipy.linalg.expm(M)


def _check_fd(gs, cam, prm, gimg, h, rtol):
    proj, bins, _ = oracle.forward(gs, cam, prm)
    an = oracle.backward_from_image_grads(gs, cam, prm, proj, bins, gimg)
    g = synth.rng(3)
    for name in ("means", "quats", "log_scales", "opacity_logits", "rgb", "feat"):
        arr = getattr(gs, name)
        for flat in g.choice(arr.size, 6, replace=False):
            idx = np.unravel_index(flat, arr.shape)
            keep = arr[idx]
            arr[idx] = keep + h
            fp = _render_functional(gs, cam, prm, gimg)
            arr[idx] = keep - h
            fm = _render_functional(gs, cam, prm, gimg)
            arr[idx] = keep
            fd = (fp - fm) / (2 * h)
            assert an[name][idx] == pytest.approx(fd, rel=rtol, abs=rtol * 1e-2), (name, idx)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        vals = []
        for sgn in (1, -1):
            c2 = camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                              T_cw=_se3_exp(sgn * e) @ cam.T_cw)
            vals.append(_render_functional(gs, c2, prm, gimg))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert an["twist"][k] == pytest.approx(fd, rel=rtol, abs=rtol * 1e-2), ("twist", k)
    return an


def test_backward_matches_finite_differences_exact_mode():
    prm = Params(alpha_min=0.0, alpha_max=1.0, T_min=0.0, lowpass=0.3, radius_sigma=40.0)
    gs, cam, gimg = _fd_setup(31, prm)
    _check_fd(gs, cam, prm, gimg, 1e-6, 1e-6)


def test_backward_matches_finite_differences_with_thresholds():
    """Default thresholds, on a scene whose threshold decisions are far from flipping."""
    prm = Params(radius_sigma=40.0, alpha_max=0.99)
    gs, cam, gimg = _fd_setup(32, prm)
    gs.opacity_logits[:2] = 6.0                   # alpha_max clamp is active at their centres
    img = oracle.forward(gs, cam, prm)[2]
    # every decision's relative gap is over 1e-4 (margin is in units of 1e-7 r_j, r_j >= 4)
    assert img["margin"].min() > 250
    _check_fd(gs, cam, prm, gimg, 1e-7, 1e-5)


def test_backward_matches_finite_differences_with_clamped_jacobian():
    """Gaussians whose centres lie beyond the Jacobian clamp (off to the side of the view)
    still reach it with their tails: their gradients follow the clamped J."""
    prm = Params(alpha_min=0.0, alpha_max=1.0, T_min=0.0, lowpass=0.3, radius_sigma=40.0)
    gs, cam, gimg = _fd_setup(34, prm)
    gs.means[:4, 0] = gs.means[:4, 2] * np.array([1.1, -1.2, 1.05, -1.3])   # x/z far outside 0.65 W/fx
    gs.log_scales[:4] += 1.0
    proj = oracle.project(gs, cam, prm)
    tx = (gs.means[:4] @ cam.T_cw[:3, :3].T + cam.T_cw[:3, 3])
    assert (np.abs(tx[:, 0] / tx[:, 2]) > 0.65 * cam.width / cam.fx + 0.1).all()
    assert (proj["radius"][:4] > 0).all()
    _check_fd(gs, cam, prm, gimg, 1e-6, 1e-6)


def test_jacobian_clamp_bounds_off_view_footprints():
    """Eq. 3 with J at the clamped point: a Gaussian far to the side keeps a footprint like
    one at the clamp boundary instead of stretching with (x/z)^2."""
    cam = camera(64, 48, 40.0, cx=32, cy=24)
    s = np.log(np.array([0.05, 0.05, 0.05]))
    at_edge = field([[0.65 * 64 / 40 * 1.0, 0, 1.0]], [[1, 0, 0, 0]], [s], [0.0], [[0, 0, 0]], [[0.0]])
    far = field([[8.0, 0, 1.0]], [[1, 0, 0, 0]], [s], [0.0], [[0, 0, 0]], [[0.0]])
    ce = oracle.project(at_edge, cam, Params(lowpass=0.0))["cov2d"][0]
    cf = oracle.project(far, cam, Params(lowpass=0.0))["cov2d"][0]
    np.testing.assert_allclose(cf, ce, rtol=1e-12)


def _pinhole(cam, p):
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


def test_exact_jacobian_is_the_linearised_pinhole_map():
    """exact_jacobian: Sigma2D = J Sc J^T with J the derivative of the pinhole map at the
    camera-frame centre (central differences of the map itself), also far outside the view,
    where the clamped mode keeps the boundary's footprint instead."""
    cam = camera(64, 48, 40.0, cx=32, cy=24)
    q = np.array([0.9, 0.2, -0.3, 0.25])
    q /= np.linalg.norm(q)
    s = np.array([0.05, 0.02, 0.08])
    for p in ([0.1, -0.05, 1.5], [8.0, 0.3, 1.0], [-3.0, 5.0, 2.0]):
        p = np.array(p)
        gs = field([p], [q], [np.log(s)], [0.0], [[0, 0, 0]], [[0.0]])
        got = oracle.project(gs, cam, Params(lowpass=0.0, exact_jacobian=True))["cov2d"][0]
        h = 1e-6
        J = np.stack([(_pinhole(cam, p + h * e) - _pinhole(cam, p - h * e)) / (2 * h) for e in np.eye(3)], 1)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S2 = J @ (R @ np.diag(s ** 2) @ R.T) @ J.T
        np.testing.assert_allclose(got, [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7, atol=1e-9 * S2.max())
        clamped = oracle.project(gs, cam, Params(lowpass=0.0))["cov2d"][0]
        inside = abs(p[0] / p[2]) <= 0.65 * 64 / 40 and abs(p[1] / p[2]) <= 0.65 * 48 / 40
        assert np.array_equal(clamped, got) == inside


def test_backward_matches_finite_differences_with_exact_jacobian():
    """The clamped-Jacobian scene of the test above with the literal Eq. 3 Jacobian."""
    prm = Params(alpha_min=0.0, alpha_max=1.0, T_min=0.0, lowpass=0.3, radius_sigma=40.0, exact_jacobian=True)
    gs, cam, gimg = _fd_setup(34, prm)
    gs.means[:4, 0] = gs.means[:4, 2] * np.array([1.1, -1.2, 1.05, -1.3])
    gs.log_scales[:4] += 1.0
    assert (oracle.project(gs, cam, prm)["radius"][:4] > 0).all()
    _check_fd(gs, cam, prm, gimg, 1e-6, 1e-6)


# -------------------------------------------------------------- rounding figures
def _perturbed_images(gs, cam, prm, proj, bins, corner, eps):
    """Renders with every splat's Sigma2D entries (a, b, c) moved by eps * lambda_max * corner
    (corner: [n, 3] in [-1, 1]), the same bins (the perturbation is far too small to move a
    rectangle)."""
    a, b, c = proj["cov2d"].T
    m = 0.5 * (a + c)
    lam = m + np.sqrt(np.maximum(m * m - (a * c - b * b), 0))
    cov = proj["cov2d"] + eps * lam[:, None] * corner
    det = cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2
    live = proj["radius"] > 0
    conic = proj["conic"].copy()
    conic[live] = np.stack([cov[:, 2], -cov[:, 1], cov[:, 0]], 1)[live] / det[live, None]
    p2 = dict(proj, conic=conic)
    return oracle.render_fwd(cam, p2, gs.rgb, gs.feat, bins[1], bins[2], prm)


def test_rounding_figures_bound_first_order_perturbations():
    """sens and sens_depth, times eps, bound the change of every output under any perturbation
    of the 2D covariances by eps * lambda_max per entry, at every pixel whose decisions cannot
    flip."""
    gs = synth.box_field(300, 4, seed=41)
    gs = synth.Gaussians(*(x.astype(np.float64) for x in gs.arrays()))
    cam = camera(40, 30, 36.0, cx=20, cy=15)
    prm = Params()
    proj, bins, img = oracle.forward(gs, cam, prm)
    eps = 1e-10
    ok = img["margin"] > 1
    assert ok.mean() > 0.99
    g = synth.rng(42)
    for trial in range(4):
        corner = g.uniform(-1, 1, (gs.n, 3)) if trial < 2 else np.sign(g.standard_normal((gs.n, 3)))
        img2 = _perturbed_images(gs, cam, prm, proj, bins, corner, eps)
        assert np.array_equal(img2["n_contrib"][ok], img["n_contrib"][ok])
        bound = eps * img["sens"] * (1 + 1e-6) + 1e-18
        for k in ("rgb", "feat"):
            assert (np.abs(img2[k] - img[k])[:, ok] <= bound[ok]).all(), k
        assert (np.abs(img2["sil"] - img["sil"])[ok] <= bound[ok]).all()
        dbound = eps * img["sens_depth"] * np.abs(img["depth"]) * (1 + 1e-6) + 1e-18
        assert (np.abs(img2["depth"] - img["depth"])[ok] <= dbound[ok]).all()


def _needle(alpha_min=1.0 / 255.0, stacked=False):
    """One splat, 4 px along the image diagonal and 0.1 px (plus the low-pass) across it; with
    stacked, a second one 10 % farther and 10 % larger behind it (the same footprint)."""
    cam = camera(32, 24, 60.0, cx=16, cy=12)
    q = [math.cos(math.pi / 8), 0, 0, math.sin(math.pi / 8)]       # 45 deg about the optical axis
    ls = np.log([0.2, 0.005, 0.005])
    if not stacked:
        gs = field([[0, 0, 3.0]], [q], [ls], [2.2], [[0.3, 0.6, 0.9]], [[1.0, -1.0]])
    else:
        gs = field([[0, 0, 3.0], [0, 0, 3.3]], [q, q], [ls, ls + np.log(1.1)], [0.0, 0.5],
                   [[0.3, 0.6, 0.9], [0.8, 0.1, 0.5]], [[0.5, -0.3], [0.2, -0.1]])
    return gs, cam, Params(alpha_min=alpha_min)


@pytest.mark.parametrize("stacked", [False, True])
def test_rounding_figures_are_attained_across_a_needle(stacked):
    """At a pixel across the needle's short axis the worst corner of the perturbation reaches
    the bound to within the alpha rounding term that a covariance perturbation does not
    exercise (more than 90 % of it); with two needles the front one's term counts what is
    blended behind it (the silhouette, whose bound is the largest here)."""
    gs, cam, prm = _needle(stacked=stacked)
    proj, bins, img = oracle.forward(gs, cam, prm)
    assert img["n_contrib"][12, 15] == (2 if stacked else 1)
    y, x = 12, 15                                   # centre offset (-0.5, +0.5): across the needle
    assert 0.1 < img["sil"][y, x] < 0.9
    eps = 1e-10
    best_s, best_d = 0.0, 0.0
    for corner in np.array(np.meshgrid([-1, 1], [-1, 1], [-1, 1])).reshape(3, -1).T:
        img2 = _perturbed_images(gs, cam, prm, proj, bins, corner[None, :].astype(float), eps)
        best_s = max(best_s, abs(img2["sil"][y, x] - img["sil"][y, x]))
        best_d = max(best_d, abs(img2["depth"][y, x] - img["depth"][y, x]) / img["depth"][y, x])
    assert 0.9 <= best_s / (eps * img["sens"][y, x]) <= 1.0 + 1e-6
    assert 0.9 <= best_d / (eps * img["sens_depth"][y, x]) <= 1.0 + 1e-6


@pytest.mark.parametrize("which", ["alpha_min", "T_min"])
def test_margin_is_the_distance_to_a_flipped_decision(which):
    """With alpha_min just under the needle's alpha at one pixel (or T_min just over the
    transmittance it leaves), a worst-corner perturbation of 0.9 margin units keeps the
    decision and one of 1.2 units flips it."""
    gs, cam, _ = _needle()
    y, x = 12, 15
    a0 = oracle.forward(gs, cam, Params())[2]["sil"][y, x]
    prm = Params(alpha_min=a0 * (1 - 1e-6)) if which == "alpha_min" else Params(T_min=(1 - a0) * (1 + 1e-6))
    proj, bins, img = oracle.forward(gs, cam, prm)
    m = img["margin"][y, x]
    assert 0.01 < m < 1
    blended = img["n_contrib"][y, x]
    corners = np.array(np.meshgrid([-1, 1], [-1, 1], [-1, 1])).reshape(3, -1).T.astype(float)
    for scale, flips in ((0.9, False), (1.2, True)):
        got = [_perturbed_images(gs, cam, prm, proj, bins, c[None, :], scale * m * 1e-7)["n_contrib"][y, x] != blended
               for c in corners]
        assert any(got) == flips, scale


def test_pose_translation_gradient_is_rotated_mean_gradient_sum():
    """Translating the camera by delta equals moving every mean by -R^T delta: g_rho = R sum g_mu."""
    gs, cam, gimg = _fd_setup(33, Params())
    proj, bins, _ = oracle.forward(gs, cam, Params())
    an = oracle.backward_from_image_grads(gs, cam, Params(), proj, bins, gimg)
    np.testing.assert_allclose(an["twist"][:3], cam.T_cw[:3, :3] @ an["means"].sum(0), rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------- losses
def _images(seed, H=12, W=10, D=5):
    g = synth.rng(seed)
    return dict(rgb=g.random((3, H, W)), depth=g.uniform(1, 4, (H, W)), sil=g.random((H, W)),
                feat=g.standard_normal((D, H, W)))


def test_cross_entropy_gradient_is_softmax_minus_onehot():
    img = _images(40)
    D, H, W = img["feat"].shape
    K = 6
    dec = synth.decoder(K, D, seed=41)
    g = synth.rng(42)
    tgt = synth.Frame(img["rgb"].copy(), img["depth"].copy(), g.integers(0, K, (H, W)).astype(np.uint8))
    tgt.label[0, :3] = 255
    w = oracle.LossWeights(color=0.0, depth=0.0, sem=1.0)
    out = oracle.loss(img, tgt, dec, w)
    f = img["feat"].reshape(D, -1).T
    z = f @ dec.W.T.astype(np.float64) + dec.b
    lab = tgt.label.ravel()
    valid = lab != 255
    logp = scipy.special.log_softmax(z, axis=1)
    P = H * W
    assert out["terms"][2] == pytest.approx(-logp[valid, lab[valid]].sum() / P, rel=1e-12)
    dz = scipy.special.softmax(z, axis=1)
    dz[np.arange(P), np.where(valid, lab, 0)] -= 1
    dz[~valid] = 0
    dz /= P
    np.testing.assert_allclose(out["feat"].reshape(D, -1).T, dz @ dec.W.astype(np.float64), atol=1e-14)
    np.testing.assert_allclose(out["W"], dz.T @ f, atol=1e-14)
    np.testing.assert_allclose(out["b"], dz.sum(0), atol=1e-14)


def test_l1_terms_and_tracking_mask():
    img = _images(50)
    D, H, W = img["feat"].shape
    P = H * W
    dec = synth.decoder(3, D, seed=51)
    g = synth.rng(52)
    tgt = synth.Frame(g.random((3, H, W)), img["depth"] + g.normal(0, 0.05, (H, W)),
                      np.full((H, W), 255, np.uint8))
    tgt.depth[0, 0] = 0.0                 # no measurement
    tgt.depth[1, 1] = img["depth"][1, 1] + 5.0   # gross depth outlier
    img["sil"][2, 2] = 0.5                # not observed
    img["sil"][3:] = 0.995
    img["sil"][:3] = 0.995
    img["sil"][2, 2] = 0.5
    # mapping: L1 over all pixels / P, depth only where d_gt > 0
    w = oracle.LossWeights(color=0.5, depth=1.0, sem=0.0)
    out = oracle.loss(img, tgt, dec, w)
    assert out["terms"][0] == pytest.approx(0.5 * np.abs(img["rgb"] - tgt.rgb).sum() / P, rel=1e-12)
    valid = tgt.depth > 0
    assert out["terms"][1] == pytest.approx(np.abs(img["depth"] - tgt.depth)[valid].sum() / P, rel=1e-12)
    np.testing.assert_allclose(out["rgb"], 0.5 * np.sign(img["rgb"] - tgt.rgb) / P)
    assert out["depth"][0, 0] == 0
    # tracking: mask = sil > 0.99, d_gt > 0, |err| < 10 * lower median of |err| over d_gt > 0
    wt = oracle.LossWeights(color=0.5, depth=1.0, sem=0.0, mask_mode=1, tau_obs=0.99)
    out = oracle.loss(img, tgt, dec, wt)
    err = np.abs(img["depth"] - tgt.depth)[valid]
    med = np.sort(err)[(err.size - 1) // 2]
    assert out["median"] == med
    mask = (img["sil"] > 0.99) & valid & (np.abs(img["depth"] - tgt.depth) < 10 * med)
    assert mask[0, 0] == 0 and mask[1, 1] == 0 and mask[2, 2] == 0
    np.testing.assert_array_equal(out["mask"], mask.astype(float))
    np.testing.assert_allclose(out["rgb"], 0.5 * mask * np.sign(img["rgb"] - tgt.rgb) / P)


def test_lower_median():
    g = synth.rng(60)
    for n in (1, 2, 7, 10, 1001):
        v = g.random(n)
        assert oracle.lower_median(v) == np.sort(v)[(n - 1) // 2]
    assert oracle.lower_median([3.0, 1.0, 2.0, 4.0]) == 2.0


def test_dsr_hand_sized():
    """Eq. 12 on 9 scales: one outlier at sqrt(8) population-sigma is the only 'big' (or 'small') one."""
    ls = np.log(np.array([[1.0, 1.0, 1.0], [1.0, 10.0, 1.0], [1.0, 1.0, 1.0]]))
    val, grad, st = oracle.dsr(ls, 0.01, 0.001)
    assert st["mu"] == pytest.approx(2.0) and st["sigma"] == pytest.approx(math.sqrt(8.0))
    assert st["n_big"] == 1 and st["n_small"] == 0
    assert val == pytest.approx(0.01 * 10.0)
    want = np.zeros((3, 3))
    want[1, 1] = 0.01 * 10.0
    np.testing.assert_allclose(grad, want, rtol=1e-12)
    ls = np.log(np.array([[1.0, 1.0, 1.0], [1.0, 1e-3, 1.0], [1.0, 1.0, 1.0]]))
    val, grad, st = oracle.dsr(ls, 0.01, 0.001)
    assert st["n_big"] == 0 and st["n_small"] == 1
    assert val == pytest.approx(0.001 * -math.log(1e-3))
    want = np.zeros((3, 3))
    want[1, 1] = -0.001
    np.testing.assert_allclose(grad, want, rtol=1e-12)
    assert oracle.dsr(np.zeros((4, 3)), 1.0, 1.0)[0] == 0.0     # no spread: both sets empty


def test_pose_step_exponential_and_first_adam_step():
    T = synth.look_pose((0.5, 1.0, 1.5), (1.0, 0.2, 0.1))
    grad = np.array([0.3, -2.0, 0.01, -0.5, 0.2, 4.0])
    lr = np.array([2e-3, 2e-3, 2e-3, 4e-4, 4e-4, 4e-4])
    Tn, m, v = oracle.pose_step(T, grad, np.zeros(6), np.zeros(6), 1, lr)
    np.testing.assert_allclose(Tn, _se3_exp(-lr * np.sign(grad)) @ T, atol=1e-12)
    np.testing.assert_allclose(m, 0.1 * grad)
    np.testing.assert_allclose(v, 0.001 * grad ** 2)
    xi = np.array([0.2, -0.1, 0.3, 0.4, -0.9, 0.25])
    big = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    T2, _, _ = oracle.pose_step(np.eye(4), -np.sign(xi), np.zeros(6), np.zeros(6), 1, np.abs(xi) * big)
    np.testing.assert_allclose(T2, _se3_exp(xi), atol=1e-12)


def test_paper_hyperparameters_fixture():
    with open(os.path.join(HERE, "golden", "paper_hyperparameters.json")) as fh:
        hp = json.load(fh)
    m, t = oracle.MAPPING, oracle.TRACKING
    assert (m.color, m.depth, m.sem, m.big, m.small) == (
        hp["mapping"]["lambda_color"], hp["mapping"]["lambda_depth"], hp["mapping"]["lambda_sem"],
        hp["mapping"]["lambda_big"], hp["mapping"]["lambda_small"])
    assert (t.color, t.depth, t.sem) == (hp["tracking"]["lambda_color"], hp["tracking"]["lambda_depth"],
                                         hp["tracking"]["lambda_sem"])
    assert oracle.MAPPING_SSIM.ssim == hp["ssim_lambda"]


# ---------------------------------------------------------------- SSIM (Eq. 15)
def _gauss11():
    k = np.arange(11) - 5
    g = np.exp(-k ** 2 / (2 * 1.5 ** 2))
    return g / g.sum()


def test_ssim_of_identical_images_is_one_with_zero_gradient():
    x = synth.rng(60).random((3, 14, 19))
    s, g = oracle.ssim(x, x)
    assert s == pytest.approx(1.0, abs=1e-15)
    assert np.abs(g).max() < 1e-13


def test_ssim_of_constant_images_closed_form():
    """Constant images a and b: with zero padding a pixel whose window keeps mass m of the
    weights sees mx = a m, sx = a^2 m (1 - m), sxy = a b m (1 - m), so every term of the
    formula (C1, C2, the window, the padding) shows at the borders."""
    H, W, a, b = 12, 23, 0.7, 0.25
    g = _gauss11()
    mass1 = lambda n: np.array([g[max(0, 5 - i):min(11, n + 5 - i)].sum() for i in range(n)])
    m = np.outer(mass1(H), mass1(W))
    C1, C2 = 1e-4, 9e-4
    S = ((2 * a * b * m ** 2 + C1) * (2 * a * b * m * (1 - m) + C2)
         / (((a * a + b * b) * m ** 2 + C1) * ((a * a + b * b) * m * (1 - m) + C2)))
    s, _ = oracle.ssim(np.full((3, H, W), a), np.full((3, H, W), b))
    assert s == pytest.approx(S.mean(), rel=1e-12)
    assert (m < 0.999).any() and (m > 0.999).any()      # both borders and interior present


def test_ssim_gradient_matches_central_differences():
    r = synth.rng(61)
    x, y = r.random((3, 13, 17)), r.random((3, 13, 17))
    _, g = oracle.ssim(x, y)
    h = 1e-6
    for c, i, j in [(0, 0, 0), (1, 6, 8), (2, 12, 16), (0, 3, 15), (2, 10, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (oracle.ssim(xp, y)[0] - oracle.ssim(xm, y)[0]) / (2 * h)
        assert g[c, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_ssim_is_symmetric():
    r = synth.rng(62)
    x, y = r.random((3, 11, 12)), r.random((3, 11, 12))
    assert oracle.ssim(x, y)[0] == pytest.approx(oracle.ssim(y, x)[0], rel=1e-14)


def test_mapping_loss_with_ssim_is_eq15_and_its_gradient():
    """lambda_c ((1 - lambda) L1 + lambda (1 - SSIM)) with lambda = 0.2, and the colour image
    gradient of the whole mapping loss against central differences."""
    r = synth.rng(63)
    H, W, D, K = 12, 14, 4, 3
    img = dict(rgb=r.random((3, H, W)), depth=r.uniform(2, 4, (H, W)), sil=r.random((H, W)),
               feat=r.standard_normal((D, H, W)))
    tgt = synth.Frame(r.random((3, H, W)), r.uniform(2, 4, (H, W)), r.integers(0, K, (H, W)).astype(np.uint8))
    dec = synth.Decoder(r.standard_normal((K, D)), r.standard_normal(K))
    w = oracle.MAPPING_SSIM
    assert w.ssim == 0.2
    out = oracle.loss(img, tgt, dec, w)
    l1 = np.abs(img["rgb"] - tgt.rgb).sum() / (H * W)
    s, _ = oracle.ssim(img["rgb"], tgt.rgb)
    assert out["terms"][0] == pytest.approx(w.color * (0.8 * l1 + 0.2 * (1 - s)), rel=1e-12)
    h = 1e-7
    for c, i, j in [(0, 0, 0), (1, 5, 7), (2, 11, 13)]:
        p, m_ = {k: v.copy() for k, v in img.items()}, {k: v.copy() for k, v in img.items()}
        p["rgb"][c, i, j] += h
        m_["rgb"][c, i, j] -= h
        fd = (oracle.loss(p, tgt, dec, w)["total"] - oracle.loss(m_, tgt, dec, w)["total"]) / (2 * h)
        assert out["rgb"][c, i, j] == pytest.approx(fd, rel=1e-5)
    with pytest.raises(ValueError):
        oracle.loss(img, tgt, dec, oracle.LossWeights(mask_mode=1, ssim=0.2))


# ------------------------------------------------------- Adam (mapping update)
def test_adam_first_steps_are_sign_steps_and_zero_gradients_stay():
    """With zero moments, the first step moves every parameter by lr against the sign of its
    gradient; a constant gradient keeps that step size; a zero gradient moves nothing."""
    r = synth.rng(64)
    shapes = dict(means=(5, 3), quats=(5, 4), log_scales=(5, 3), opacity_logits=(5,), rgb=(5, 3), feat=(5, 4))
    p = {k: r.standard_normal(s) for k, s in shapes.items()}
    g = {k: r.standard_normal(s) for k, s in shapes.items()}
    g["feat"][0] = 0.0
    z = {k: np.zeros(s) for k, s in shapes.items()}
    lr = oracle.MAPPING_LR
    p1, m1, v1 = oracle.adam_step(p, g, z, z, 1, lr)
    p2, _, _ = oracle.adam_step(p1, g, m1, v1, 2, lr)
    for k in shapes:
        np.testing.assert_allclose(p1[k], p[k] - lr[k] * np.sign(g[k]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(p2[k], p[k] - 2 * lr[k] * np.sign(g[k]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(m1[k], 0.1 * g[k], rtol=1e-14)
        np.testing.assert_allclose(v1[k], 0.001 * g[k] ** 2, rtol=1e-14)
    assert (p1["feat"][0] == p["feat"][0]).all()


def test_adam_learning_rates_are_the_papers():
    with open(os.path.join(HERE, "golden", "paper_hyperparameters.json")) as fh:
        hp = json.load(fh)["mapping"]
    lr = oracle.MAPPING_LR
    assert (lr["means"], lr["rgb"], lr["quats"], lr["opacity_logits"], lr["log_scales"], lr["feat"]) == (
        hp["lr_position"], hp["lr_color"], hp["lr_rotation"], hp["lr_opacity"], hp["lr_scaling"], hp["lr_feature"])


def test_adam_steps_follow_the_bias_corrected_recursion_on_a_scalar():
    """A gradient sequence g_t on one scalar: after T steps the update of step T equals
    lr m_T / (1 - b1^T) / (sqrt(v_T / (1 - b2^T)) + eps) with m, v the exponential sums written
    out as series."""
    gs_ = [0.3, -1.2, 0.7, 2.0]
    b1, b2, lr = 0.9, 0.999, 0.01
    keys = oracle.ADAM_GROUPS
    p = {k: np.zeros(1) for k in keys}
    m = {k: np.zeros(1) for k in keys}
    v = {k: np.zeros(1) for k in keys}
    for t, gt in enumerate(gs_, start=1):
        prev = p["rgb"].copy()
        p, m, v = oracle.adam_step(p, {k: np.array([gt]) for k in keys}, m, v, t, {k: lr for k in keys})
    T = len(gs_)
    mT = sum((1 - b1) * b1 ** (T - 1 - i) * g for i, g in enumerate(gs_))
    vT = sum((1 - b2) * b2 ** (T - 1 - i) * g * g for i, g in enumerate(gs_))
    want = lr * (mT / (1 - b1 ** T)) / (math.sqrt(vT / (1 - b2 ** T)) + 1e-15)
    assert prev[0] - p["rgb"][0] == pytest.approx(want, rel=1e-12)


# -------------------------------------------------- adaptive expansion (Eq. 11)
def _expand_frame(H=9, W=13, seed=65):
    r = synth.rng(seed)
    depth = r.uniform(1.5, 4.0, (H, W)).astype(np.float32)
    depth[0, :4] = 0.0                                   # invalid depth: never unprojected
    return synth.Frame(r.random((3, H, W)).astype(np.float32), depth, np.zeros((H, W), np.uint8))


def test_expand_adds_nothing_where_the_map_explains_the_frame():
    tgt = _expand_frame()
    cam = camera(13, 9, 7.0, T_cw=synth.look_pose((0.3, -0.2, 0.1), (0.2, 0.1, 1.0), up=(0, -1, 0)))
    out = oracle.expand(dict(sil=np.ones((9, 13)), depth=tgt.depth), tgt, cam, np.zeros((200, 4)))
    assert len(out["src_pix"]) == 0


def test_expand_of_an_empty_render_unprojects_every_valid_pixel():
    """Every pixel with depth: the new mean reprojects to its pixel centre at d_gt, scale d/fx,
    opacity 1/2, the observed colour, features in order."""
    tgt = _expand_frame()
    cam = camera(13, 9, 7.0, T_cw=synth.look_pose((0.3, -0.2, 0.1), (0.2, 0.1, 1.0), up=(0, -1, 0)))
    feat = synth.rng(66).standard_normal((200, 4))
    out = oracle.expand(dict(sil=np.zeros((9, 13)), depth=np.zeros((9, 13))), tgt, cam, feat)
    want = np.nonzero(tgt.depth.ravel() > 0)[0]
    np.testing.assert_array_equal(out["src_pix"], want)
    T = np.asarray(cam.T_cw)
    pc = out["means"] @ T[:3, :3].T + T[:3, 3]
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    np.testing.assert_allclose(u, want % 13 + 0.5, atol=1e-12)
    np.testing.assert_allclose(v, want // 13 + 0.5, atol=1e-12)
    np.testing.assert_allclose(pc[:, 2], tgt.depth.ravel()[want], rtol=1e-12)
    d = tgt.depth.ravel()[want].astype(np.float64)
    np.testing.assert_allclose(out["log_scales"], np.log(d / 7.0)[:, None] * np.ones(3), rtol=1e-12)
    assert (out["opacity_logits"] == 0).all() and sigmoid(0.0) == 0.5
    np.testing.assert_array_equal(out["rgb"], tgt.rgb.reshape(3, -1)[:, want].T)
    np.testing.assert_array_equal(out["feat"], feat[:len(want)])
    np.testing.assert_array_equal(out["quats"], np.tile([1.0, 0, 0, 0], (len(want), 1)))


def test_expand_depth_rule_is_fifty_times_the_lower_median():
    """Covered pixels (sil = 1): a pixel expands only if rendered behind the observation by more
    than 50 x the lower median of |d_gt - d_hat| (errors exact in f32)."""
    H, W = 4, 8
    tgt = synth.Frame(np.zeros((3, H, W), np.float32), np.full((H, W), 2.0, np.float32), np.zeros((H, W), np.uint8))
    e = np.full(H * W, 2.0 ** -12, np.float32)             # the median error: 2^-12
    e[3] = 50 * 2.0 ** -12 + 2.0 ** -10                     # behind, just over 50 x median: expands
    e[4] = 50 * 2.0 ** -12 - 2.0 ** -10                     # behind, just under: no
    e[5] = -(50 * 2.0 ** -12 + 2.0 ** -10)                  # in front by as much: no (d_hat < d_gt)
    e[6] = 50 * 2.0 ** -12                                  # exactly 50 x median: no (strict)
    d_hat = (tgt.depth.ravel() + e).reshape(H, W)
    out = oracle.expand(dict(sil=np.ones((H, W)), depth=d_hat), tgt, camera(W, H, 5.0), np.zeros((50, 2)))
    assert out["median"] == 2.0 ** -12
    np.testing.assert_array_equal(out["src_pix"], [3])
    out2 = oracle.expand(dict(sil=np.full((H, W), 0.49), depth=d_hat), tgt, camera(W, H, 5.0), np.zeros((50, 2)),
                         tau_unobs=0.5)
    assert len(out2["src_pix"]) == H * W                    # low opacity alone expands


# --------------------------------------------- tracking over a sequence (Eq. 19)
def test_constant_velocity_is_exact_for_a_constant_screw_motion():
    """T_k = Exp(k xi) T_0: the prediction from frames t-1, t-2 is frame t."""
    xi = np.array([0.03, -0.01, 0.02, 0.01, -0.02, 0.015])
    T0 = synth.look_pose((1.0, 2.0, 1.5), (0.3, 1.0, -0.1))
    T = [_se3_exp(k * xi) @ T0 for k in range(5)]
    for t in range(2, 5):
        np.testing.assert_allclose(oracle.constant_velocity(T[t - 1], T[t - 2]), T[t], atol=1e-12)


def test_ate_of_a_shifted_trajectory_is_the_shift():
    T0 = synth.look_pose((1.0, 2.0, 1.5), (0.3, 1.0, -0.1))
    gt = [_se3_exp(k * np.array([0.02, 0, 0, 0, 0.01, 0])) @ T0 for k in range(4)]
    shift = np.array([0.03, -0.04, 0.0])                       # camera centres moved by 5 cm
    est = []
    for T in gt:
        R, t = T[:3, :3], T[:3, 3]
        S = T.copy()
        S[:3, 3] = t - R @ shift                               # centre -R^T t moves by +shift
        est.append(S)
    assert oracle.ate_rmse(gt, gt) == 0.0
    assert oracle.ate_rmse(est, gt) == pytest.approx(0.05, rel=1e-12)


def test_sequence_without_tracking_steps_follows_the_constant_velocity_predictions():
    """The sequence wiring: frames after the given poses start from Eq. 19's prediction, which
    is exact under a constant screw motion, so with no tracking step every estimate is the true
    pose (tracking steps themselves are pinned by the single-frame loop's tests)."""
    gs = synth.box_field(400, 4, seed=9)
    xi = np.array([0.01, -0.005, 0.0, 0.002, -0.004, 0.003])
    gt = [_se3_exp(k * xi) for k in range(5)]
    prm = Params()
    frames = [synth.Frame(np.zeros((3, 36, 48)), np.ones((36, 48)), np.full((36, 48), 255, np.uint8))] * 5
    dec = synth.Decoder(np.zeros((2, 4)), np.zeros(2))
    est = oracle.track_sequence(gs, camera(48, 36, 45.0), prm, frames, dec, gt[:2], n_it=0)
    assert len(est) == 5
    for a, b in zip(est, gt):
        np.testing.assert_allclose(a, b, atol=1e-9)


# ------------------------------------------------- RSKM keyframe draw (Eq. 13)
def test_rskm_takes_the_current_frame_every_t_opt_iterations():
    """Eq. 13 with mod(k_m, t_opt) = 0: p(f_cur) = 1/|K| + (1 - 1/|K|) = 1, whatever the draw."""
    for draw in (0, 1, 7, 2 ** 32 - 1):
        for k_m in (0, 3, 6, 9):
            assert oracle.rskm_select(k_m, 3, 4, [0, 2, 4], draw) == 4
    assert all(oracle.rskm_select(k, 1, 9, [0, 5], d) == 9 for k in range(5) for d in range(5))


def test_rskm_draws_uniformly_between_the_current_frame_iterations():
    """mod(k_m, t_opt) != 0: p(f) = 1/|K| for every keyframe; a full cycle of draws hits each
    candidate once, and a current frame that is not a keyframe is a candidate too."""
    K = [0, 5, 10]
    got = [oracle.rskm_select(1, 2, 10, K, d) for d in range(3)]
    assert sorted(got) == K
    got = [oracle.rskm_select(1, 2, 12, K, d) for d in range(4)]
    assert sorted(got) == [0, 5, 10, 12]
    assert oracle.rskm_select(5, 2, 12, K, 0) == 0          # word 0: the oldest keyframe


def test_rskm_long_run_share_of_the_current_frame():
    """Over t_opt |K| m iterations with every draw residue equally often, the current frame's
    share is 1/t_opt + (1 - 1/t_opt) / |K| (the two cases of Eq. 13 mixed)."""
    K, t_opt, m = [0, 3, 6, 9], 3, 5
    n = t_opt * len(K) * m
    draws = np.arange(n)                                     # residues mod |K| equally often
    picks = [oracle.rskm_select(k, t_opt, 9, K, draws[k]) for k in range(n)]
    share = Fraction(sum(p == 9 for p in picks), n)
    assert share >= Fraction(1, t_opt)
    # every non-multiple iteration draws one of |K| frames; with k running over whole cycles
    # of lcm(t_opt, |K|) the residues are equally frequent among them
    assert share == Fraction(1, t_opt) + (1 - Fraction(1, t_opt)) * Fraction(1, len(K))


# ------------------------------------------------------ the SLAM loop (Sec. 3.3-3.4)
def _slam_case(n_frames=3, W=32, H=24):
    room = synth.make_room()
    path = synth.smooth_path(n_frames, step_deg=0.8, room=room)
    frames = [synth.raycast_room(room, synth.camera(W, H, 30.0, T_cw=T)) for T in path]
    return path, frames, synth.camera(W, H, 30.0, T_cw=path[0]), synth.decoder(4, 4)


def test_slam_first_frame_unprojects_every_pixel_and_draws_only_it():
    """An empty map renders nothing (silhouette 0), so the first frame's expansion adds one
    Gaussian per pixel with depth; its mapping iterations can only draw the first frame."""
    path, frames, cam, dec = _slam_case(1)
    cfg = oracle.SlamConfig(n_track=0, n_map=0, n_init=3)
    out = oracle.slam(frames, cam, Params(), dec, path[0], synth.rskm_draws(10), synth.feature_bank(2000, 4), cfg)
    assert out["sizes"] == [int((frames[0].depth > 0).sum())] == [32 * 24]
    assert out["picks"] == [0, 0, 0]


def test_slam_mapping_lowers_the_mapping_loss():
    """The loop's mapping iterations descend the mapping loss of the frame they map (a sign or
    wiring error in the update would raise it)."""
    path, frames, cam, dec = _slam_case(1)
    bank = synth.feature_bank(2000, 4)
    loss_after = []
    for n_init in (0, 8):
        cfg = oracle.SlamConfig(n_track=0, n_map=0, n_init=n_init)
        out = oracle.slam(frames, cam, Params(), dec, path[0], synth.rskm_draws(10), bank, cfg)
        loss_after.append(oracle.step(out["gs"], cam, Params(), frames[0], dec, oracle.MAPPING_SSIM)["total"])
    assert loss_after[1] < 0.9 * loss_after[0]


def test_slam_keyframes_and_draws_with_one_word():
    """Every draw word 0 (the first candidate) and t_opt = 2: even iterations take the current
    frame, odd ones the first keyframe, frame 0; with every frame a keyframe that holds for
    each frame of the sequence; frames without tracking steps keep Eq. 19's prediction."""
    path, frames, cam, dec = _slam_case(3)
    cfg = oracle.SlamConfig(n_track=0, n_map=4, n_init=2, t_opt=2, kf_every=1)
    out = oracle.slam(frames, cam, Params(), dec, path[0], np.zeros(20, np.uint32), synth.feature_bank(3000, 4), cfg)
    assert out["picks"] == [0, 0] + [1, 0, 1, 0] + [2, 0, 2, 0]
    np.testing.assert_allclose(out["poses"][1], path[0], atol=1e-12)   # from one pose: that pose
    np.testing.assert_allclose(out["poses"][2], path[0], atol=1e-12)
    assert out["sizes"][0] == 32 * 24 and out["sizes"][2] >= out["sizes"][1] >= out["sizes"][0]
