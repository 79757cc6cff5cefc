"""The C-ABI library builds, loads and exports every symbol include/gs.h declares (no GPU needed).

Only host-side argument checks are exercised here: they return before any CUDA call.
"""
import ctypes
import os
import re

import pytest

from paper_2603_27781_gb300 import _lib as L
from paper_2603_27781_gb300 import build, raster, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
        assert name in L.exported_symbols(), name


def test_version_and_status_text(lib):
    assert lib.gs_version() >= 10000
    assert lib.gs_strerror(L.GS_ERR_CAPACITY).decode().startswith("tile instance")
    assert isinstance(lib.gs_cuda_error().decode(), str) and lib.gs_cuda_error()  # a text, never NULL
    assert lib.gs_strerror(12345).decode() == "unknown status"


def test_workspace_size(lib):
    cams = raster.cameras_c([synth.camera(1200, 680, 600.0)])
    small = lib.gs_workspace_size(1000, 1, cams, 10000, 16)
    big = lib.gs_workspace_size(1_000_000, 1, cams, 4_000_000, 16)
    assert 0 < small < big
    assert lib.gs_workspace_size(1000, 1, cams, 10000, 5) == 0          # unsupported feature dim
    assert lib.gs_workspace_size(1000, 1, cams, 1 << 30, 16) == 0       # capacity too large
    assert lib.gs_workspace_size(1000, 0, cams, 100, 16) == 0           # no views


def test_argument_errors_before_any_launch(lib):
    cam = raster.cameras_c([synth.camera(64, 48, 60.0)])
    prm = raster.RasterParams().c()
    g = L.gs_gaussians(10, 16, None, None, None, None, None, 0, None, 0)
    pj = L.gs_projected(None, None, None)
    assert lib.gs_project(ctypes.byref(g), cam, 0, None, ctypes.byref(prm), ctypes.byref(pj), None) == L.GS_ERR_ARG
    bad = raster.RasterParams(tile=8).c()
    assert lib.gs_project(ctypes.byref(g), cam, 1, None, ctypes.byref(bad), ctypes.byref(pj), None) == L.GS_ERR_ARG
    assert lib.gs_project(ctypes.byref(g), cam, 1, None, ctypes.byref(prm), ctypes.byref(pj), None) == L.GS_ERR_ARG
    b = L.gs_binning(-1, None, None, None, None, None)
    assert lib.gs_bin_sort(10, ctypes.byref(pj), cam, 1, ctypes.byref(prm), None, 0, ctypes.byref(b),
                           None) == L.GS_ERR_ARG
    assert lib.gs_pose_grad(10, 0, None, None, None) == L.GS_ERR_ARG
    assert lib.gs_dsr(-1, None, 0.0, 0.0, None, 0, None, None, None) == L.GS_ERR_ARG
    lr = (ctypes.c_double * 6)(*([1e-3] * 6))
    assert lib.gs_pose_step(1, None, None, None, 1, lr, 0.9, 0.999, 1e-15, None, None) == L.GS_ERR_ARG
    zero_w = synth.camera(64, 48, 60.0)
    zero_w.width = 0
    assert lib.gs_workspace_size(10, 1, raster.cameras_c([zero_w]), 10, 16) == 0
    # the SSIM weight of Eq. 15: in [0, 1] and for the mapping loss only (checked before any
    # launch; the non-null pointers below are never dereferenced on the host)
    fake = ctypes.c_void_p(1 << 20)
    img = L.gs_images(fake, fake, fake, fake, fake, fake, None, None)
    tgt = L.gs_targets(fake, fake, fake)
    grads = L.gs_image_grads_out(fake, fake, fake, fake, None)
    for weights in ((0.5, 1.0, 0.01, 1, 0.99, 8, 0.2), (0.5, 1.0, 0.01, 0, 0.99, 8, 1.5),
                    (0.5, 1.0, 0.01, 0, 0.99, 8, -0.1)):
        lp = L.gs_loss_params(*weights)
        assert lib.gs_loss_fwd_bwd(cam, 1, 16, ctypes.byref(img), ctypes.byref(tgt), fake, fake, ctypes.byref(lp),
                                   fake, 1 << 30, ctypes.byref(grads), fake, fake, fake, None, None,
                                   None) == L.GS_ERR_ARG

    # the RSKM draw: slots inside the store, the current slot at most one past the keyframes,
    # t_opt >= 1, random words present
    kf = L.gs_keyframes(4, 64 * 48, fake, fake, fake, fake)
    args = lambda n_kf, cur, t_opt, draws, n: (ctypes.byref(kf), n_kf, cur, t_opt, draws, n, fake, None, fake, fake,
                                               fake, None, None)
    for bad_args in (args(2, 3, 2, fake, 8), args(5, 4, 2, fake, 8), args(2, 2, 0, fake, 8), args(2, 2, 2, None, 8),
                     args(2, 2, 2, fake, 0), args(4, 4, 2, fake, 8), args(-1, 0, 2, fake, 8)):
        assert lib.gs_rskm_draw(*bad_args) == L.GS_ERR_ARG
    # the halves of the DSR: missing buffers, a negative count, an unaligned scratch
    assert lib.gs_dsr_value(10, None, 1.0, 1.0, None, None, None) == L.GS_ERR_ARG
    assert lib.gs_dsr_value(-1, None, 1.0, 1.0, None, None, None) == L.GS_ERR_ARG
    assert lib.gs_dsr_value(10, 4096, 1.0, 1.0, 257, 4096, None) == L.GS_ERR_ARG
    assert lib.gs_dsr_grad(10, None, 1.0, 1.0, None, None, None) == L.GS_ERR_ARG
    assert lib.gs_dsr_grad(-1, 4096, 1.0, 1.0, 4096, 4096, None) == L.GS_ERR_ARG
    # clearing the splat sums: a mode without MAP or POSE, an unknown bit, missing or unaligned
    # buffers, no views
    sg = L.gs_splat_grads(fake, fake, fake)
    for mode in (0, L.GS_GRAD_ACCUMULATE, 8 | L.GS_GRAD_MAP):
        assert lib.gs_splat_grads_clear(ctypes.byref(g), 1, mode, ctypes.byref(sg), fake, None) == L.GS_ERR_ARG
    assert lib.gs_splat_grads_clear(ctypes.byref(g), 0, L.GS_GRAD_MAP, ctypes.byref(sg), fake, None) == L.GS_ERR_ARG
    assert lib.gs_splat_grads_clear(ctypes.byref(g), 1, L.GS_GRAD_MAP, ctypes.byref(sg), None, None) == L.GS_ERR_ARG
    odd = L.gs_splat_grads(ctypes.c_void_p((1 << 20) + 4), fake, fake)
    assert lib.gs_splat_grads_clear(ctypes.byref(g), 1, L.GS_GRAD_POSE, ctypes.byref(odd), None, None) == L.GS_ERR_ARG
    assert lib.gs_splat_grads_clear(None, 1, L.GS_GRAD_MAP, ctypes.byref(sg), fake, None) == L.GS_ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        L.library()
