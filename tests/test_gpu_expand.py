"""Adaptive Gaussian expansion (Eq. 11) through the C ABI against the oracle.

The mask and the order of the new Gaussians are integer decisions taken in f32 on
the same inputs on both sides (the GPU's rendered silhouette and depth, the
observed frame), so the source pixels are compared bit for bit; the unprojected
means within f32 rounding; colours, features, rotations and opacities exactly.
A sparse field leaves holes (low silhouette) and surfaces rendered behind the
observation, so both branches of the mask occur.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_27781_gb300 import raster, synth
from paper_2603_27781_gb300 import _lib as L

import gpu_cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    from paper_2603_27781_gb300 import build
    build.build()
    L.library()


def _scene(sizes, n=6000, seed=0):
    gs, _, room = C.room_case(n, 8, 160, 96, 80.0, seed=seed)
    poses = synth.keyframe_loop(8, room=room)
    cams = [synth.camera(w, h, 0.5 * w, T_cw=poses[2 * i + 1]) for i, (w, h) in enumerate(sizes)]
    frames = [synth.raycast_room(room, c) for c in cams]
    return gs, cams, frames


def _run(gs, cams, frames, n_max, seed=3):
    field, r = C.gpu_forward(gs, cams, C.params_pair()[0])
    cat = lambda xs: torch.as_tensor(np.ascontiguousarray(np.concatenate(xs, axis=-1))).cuda()
    tg = dict(rgb=cat([f.rgb.reshape(3, -1) for f in frames]), depth=cat([f.depth.ravel() for f in frames]),
              label=cat([f.label.ravel() for f in frames]))
    feat = torch.as_tensor(synth.rng(seed).standard_normal((n_max, gs.feat_dim)), dtype=torch.float32).cuda()
    out, src, total, status = raster.expand(r, field, tg, feat)
    torch.cuda.synchronize()
    # the oracle, view by view on the same rendered images; feature rows continue across views
    ref, used = [], 0
    for v, (cam, fr) in enumerate(zip(cams, frames)):
        im = r.images(v)
        o = oracle.expand(dict(sil=im["sil"].cpu().numpy(), depth=im["depth"].cpu().numpy()), fr, cam,
                          feat.cpu().numpy().astype(np.float64)[used:])
        o["src_pix"] = o["src_pix"] + r.pix_off[v]
        used += len(o["src_pix"])
        ref.append(o)
    want = {k: np.concatenate([o[k] for o in ref]) for k in ("src_pix", "means", "quats", "log_scales",
                                                             "opacity_logits", "rgb", "feat")}
    return gs.n, out, src, total, status, want


def _check(n0, out, src, k, want):
    np.testing.assert_array_equal(src.cpu().numpy(), want["src_pix"][:k])
    new = lambda t: t[n0:].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(new(out.means), want["means"][:k], rtol=0, atol=2e-6 * np.abs(want["means"]).max())
    np.testing.assert_allclose(new(out.log_scales), want["log_scales"][:k], rtol=0, atol=1e-6)
    np.testing.assert_array_equal(new(out.quats), want["quats"][:k])
    np.testing.assert_array_equal(new(out.opacity_logits), want["opacity_logits"][:k])
    np.testing.assert_array_equal(new(out.rgb), want["rgb"][:k].astype(np.float32))
    np.testing.assert_array_equal(new(out.feat), want["feat"][:k].astype(np.float32))


@pytest.mark.parametrize("sizes", [[(330, 190)], [(160, 96), (97, 61)]])
def test_expansion_matches_oracle(sizes):
    gs, cams, frames = _scene(sizes)
    n0, out, src, total, status, want = _run(gs, cams, frames, n_max=sum(w * h for w, h in sizes))
    assert status == 0 and total == len(want["src_pix"]) > 0
    assert out.n == n0 + total
    np.testing.assert_array_equal(out.means[:n0].cpu().numpy(), gs.means)    # existing rows kept
    _check(n0, out, src, total, want)
    # both branches of Eq. 11 occur: holes and surfaces rendered behind the observation
    assert want["src_pix"].size < sum(w * h for w, h in sizes)


def test_expansion_beyond_capacity_writes_the_first_rows_and_reports():
    gs, cams, frames = _scene([(330, 190)])
    n0, out, src, total, status, want = _run(gs, cams, frames, n_max=500)
    assert total == len(want["src_pix"]) > 500
    assert status == L.GS_ERR_CAPACITY and out.n == n0 + 500
    _check(n0, out, src, 500, want)
