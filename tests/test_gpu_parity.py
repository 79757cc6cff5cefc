"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Sizes run from the tiny box scene to room scenes spanning hundreds of tiles with
ragged image edges, multi-view batches and the reduced-precision storage form.
Binning and sort are compared bit for bit; floating-point outputs within the
stated tolerances, excluding (and counting) pixels where a threshold decision is
within rounding distance in the oracle.
"""
import ctypes
import dataclasses

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


def _cases():
    T = synth.look_pose((0.15, -0.1, -0.3), (0.05, 0.04, 1.0), up=(0, -1, 0))
    return {
        "box_64x48": lambda: C.box_case(2000, 16, 64, 48, 60.0),
        "box_ragged_pose_70x50": lambda: C.box_case(3000, 8, 70, 50, 55.0, seed=3, T=T),
        "room_20k_330x190": lambda: C.room_case(20000, 16, 330, 190, 165.0)[:2],
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_projection_matches_oracle(name):
    gs, cam = CASES[name]()
    prm_g, prm_o = C.params_pair()
    _, r = C.gpu_forward(gs, cam, prm_g)
    gp = C.gpu_projection(r)
    op = oracle.project(gs, cam, prm_o)
    # the sort key is the same f32 fused chain on both sides: bit-exact
    np.testing.assert_array_equal(gp["depth"].view(np.uint32), op["depth_key"].view(np.uint32))
    np.testing.assert_allclose(gp["opacity"], op["opacity"], rtol=0, atol=1e-6)
    vis = (gp["radius"] > 0) & (op["radius"] > 0)
    # culling agrees except within rounding of z_near
    assert ((gp["radius"] > 0) != (op["radius"] > 0)).sum() == 0
    # the centre is carried in compensated precision: f32 hi + lo matches the f64 centre
    np.testing.assert_allclose(gp["uv_full"][vis], op["uv"][vis], rtol=0, atol=2e-6)
    np.testing.assert_allclose(gp["uv"][vis], op["uv"][vis], rtol=1e-7, atol=0)
    scale = np.maximum(np.abs(op["conic"][vis, 0]), np.abs(op["conic"][vis, 2]))[:, None]
    assert (np.abs(gp["conic"][vis] - op["conic"][vis]) <= 2e-4 * scale).all()
    near_int = np.abs(op["radius_real"] - np.round(op["radius_real"])) < 1e-4
    rad_diff = (gp["radius"] != op["radius"]) & ~near_int
    assert rad_diff.sum() == 0
    # tiles touched follow the exact integer rectangle rule from the GPU's own centre and radius
    _, touched = oracle.rects(gp["uv"], gp["radius"], cam.width, cam.height)
    np.testing.assert_array_equal(gp["touched"], touched)


@pytest.mark.parametrize("exact", [False, True])
def test_jacobian_modes_match_oracle(exact):
    """Gaussians beside the view: projection, forward and every gradient against the oracle
    with the clamped Jacobian and with the exact one of Eq. 3, whose footprints differ."""
    gs, cam = C.offview_case()
    prm_g, prm_o = C.params_pair(exact_jacobian=exact)
    _, r = C.gpu_forward(gs, cam, prm_g)
    gp = C.gpu_projection(r)
    op = oracle.project(gs, cam, prm_o)
    vis = (gp["radius"] > 0) & (op["radius"] > 0)
    scale = np.maximum(np.abs(op["conic"][vis, 0]), np.abs(op["conic"][vis, 2]))[:, None]
    assert (np.abs(gp["conic"][vis] - op["conic"][vis]) <= 2e-4 * scale).all()
    other = oracle.project(gs, cam, C.params_pair(exact_jacobian=not exact)[1])
    moved = np.abs(other["conic"][:300] - op["conic"][:300]).max(1) > 1e-2 * np.abs(op["conic"][:300]).max(1)
    assert moved.sum() > 100          # the two modes differ for the Gaussians beside the view
    C.bwd_compare(gs, [cam], prm_g, prm_o, seed=21)


def _check_sort(gs, cams, prm_g):
    _, r = C.gpu_forward(gs, cams, prm_g)
    assert r.status() == 0
    gp = C.gpu_projection(r)
    n = gs.n
    rects = []
    for v, cam in enumerate(cams):
        sl = slice(v * n, (v + 1) * n)
        rects.append(oracle.rects(gp["uv"][sl], gp["radius"][sl], cam.width, cam.height)[0])
    keys, vals, ranges = oracle.bin_sort(np.concatenate(rects), gp["depth"].astype(np.float32), cams,
                                         n_per_view=n)
    gk, gv, gr = C.gpu_binning(r)
    assert r.instances() == len(keys)
    np.testing.assert_array_equal(gk, keys)
    np.testing.assert_array_equal(gv, vals)
    np.testing.assert_array_equal(gr, ranges)


@pytest.mark.parametrize("name", list(CASES))
def test_bin_sort_bit_exact(name):
    gs, cam = CASES[name]()
    _check_sort(gs, [cam], C.params_pair()[0])


def test_bin_sort_bit_exact_multiview_and_ties():
    gs, cam, room = C.room_case(30000, 8, 200, 120, 100.0)
    poses = synth.keyframe_loop(12, room=room)
    cams = [synth.camera(200, 120, 100.0, T_cw=poses[0]), synth.camera(97, 61, 50.0, T_cw=poses[5]),
            synth.camera(160, 90, 80.0, T_cw=poses[9])]
    gs.means[1::2] = gs.means[0::2][: gs.means[1::2].shape[0]]  # duplicated centres: equal depth keys
    _check_sort(gs, cams, C.params_pair()[0])


def test_bin_sort_bit_exact_with_the_larger_depth_blocks():
    """The depth passes take 1,024-key blocks up to 2^21 (view, Gaussian) items and 2,048-key
    blocks above; the other sort cases are below the switch, this one (300,000 Gaussians in 8
    views, 2.4M items) is above it."""
    gs, _, room = C.room_case(300_000, 8, 160, 96, 80.0)
    poses = synth.keyframe_loop(16, room=room)
    cams = [synth.camera(160, 96, 80.0, T_cw=poses[2 * i]) for i in range(8)]
    assert gs.n * len(cams) > 1 << 21
    _check_sort(gs, cams, C.params_pair()[0])


@pytest.mark.parametrize("width", [16, 48])
def test_bin_sort_bit_exact_long_tiles(width):
    """Tiles of more than 4096 instances: 9,000 Gaussians in front of a 16x16 (one tile) or
    48x16 image, half of them on the centres of the others (equal depth keys, ordered by
    item)."""
    gs, cam = C.box_case(9000, 8, width, 16, 12.0)
    gs.means[1::2] = gs.means[0::2][: gs.means[1::2].shape[0]]
    _check_sort(gs, [cam], C.params_pair()[0])
    _, r = C.gpu_forward(gs, [cam], C.params_pair()[0])
    rg = r.ranges.cpu().numpy().astype(np.int64).reshape(-1, 2)
    assert (rg[:, 1] - rg[:, 0]).max() > 4096


@pytest.mark.parametrize("name", list(CASES))
def test_render_fwd_matches_oracle(name):
    gs, cam = CASES[name]()
    prm_g, prm_o = C.params_pair()
    _, r = C.gpu_forward(gs, cam, prm_g)
    gimg = C.np_images(r)
    op, _, oimg = oracle.forward(gs, cam, prm_o)
    ex = C.exclusion(cam, op, C.gpu_projection(r), oimg).check(name)
    C.assert_forward_close(gimg, oimg, ex.mask, gs.feat_dim, ex.shifted)
    np.testing.assert_allclose(gimg["sil"] + gimg["T"], 1.0, atol=1e-5)


@pytest.mark.parametrize("name", list(CASES))
def test_render_bwd_matches_oracle(name):
    gs, cam = CASES[name]()
    prm_g, prm_o = C.params_pair()
    C.bwd_compare(gs, [cam], prm_g, prm_o)


@pytest.mark.parametrize("np_,fwd_blocks", [(1, 2), (2, 2), (4, 2), (1, 1), (2, 1)])
def test_launch_shapes_agree(np_, fwd_blocks):
    """Every launch shape (pixels per thread; forward blocks per tile or per pixel group)
    renders bit-identical images and blend masks and the same gradients."""
    gs, cam, _ = C.room_case(20000, 16, 330, 190, 165.0)
    prm0, prm_o = C.params_pair()
    field, r0 = C.gpu_forward(gs, cam, prm0)
    ref = {k: v.clone() for k, v in r0.images().items()}
    g = C.random_image_grads(r0.P, 16, 5)
    for rr in (r0,):
        rr.g_rgb.copy_(torch.as_tensor(g["rgb"])); rr.g_depth.copy_(torch.as_tensor(g["depth"]))
        rr.g_sil.copy_(torch.as_tensor(g["sil"])); rr.g_feat.copy_(torch.as_tensor(g["feat"]))
    r0.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
    want = [t.clone() for t in (r0.d_means, r0.d_quats, r0.d_log_scales, r0.d_logits, r0.d_rgb, r0.d_feat,
                                r0.d_twist)]
    mask_ref = r0.blend_mask.clone()
    prm = raster.RasterParams(fwd_px_per_thread=np_, bwd_px_per_thread=np_, fwd_blocks=fwd_blocks)
    r0.params, r0.prm_c = prm, prm.c()
    r0.forward(field)
    for k, t in r0.images().items():
        assert torch.equal(t, ref[k]), k
    assert torch.equal(r0.blend_mask, mask_ref)
    r0.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
    for name, a, b in zip(("means", "quats", "log_scales", "logits", "rgb", "feat", "twist"), want,
                          (r0.d_means, r0.d_quats, r0.d_log_scales, r0.d_logits, r0.d_rgb, r0.d_feat, r0.d_twist)):
        C.assert_grad_close(name, b.cpu().numpy(), a.cpu().numpy(), 1e-5)


@pytest.mark.parametrize("D,np_", [(16, 1), (16, 2), (32, 1), (32, 2)])
def test_warp_block_backward_matches_oracle(D, np_):
    """The map-mode backward as one 32-thread block per pixel group, over a frame and a
    ragged second view, against the oracle."""
    gs, cam, room = C.room_case(6000, D, 96, 64, 48.0)
    cams = [cam, synth.camera(70, 45, 40.0, T_cw=synth.keyframe_loop(8, room=room)[2])]
    prm_g = raster.RasterParams(bwd_blocks=L.GS_BWD_BLOCKS_GROUP, bwd_px_per_thread=np_)
    C.bwd_compare(gs, cams, prm_g, C.params_pair()[1])


@pytest.mark.parametrize("np_", [1, 2])
def test_warp_block_backward_agrees_with_the_tile_kernel(np_):
    """Same frame, same upstream gradients: the per-group blocks give the tile kernel's
    gradients (f32 and half storage); unsupported shapes are refused."""
    gs, cam, _ = C.room_case(20000, 16, 330, 190, 165.0)
    for rgb_dt, feat_dt in ((torch.float32, torch.float32), (torch.float16, torch.bfloat16)):
        field, r = C.gpu_forward(gs, cam, C.params_pair()[0], rgb_dtype=rgb_dt, feat_dtype=feat_dt)
        g = C.random_image_grads(r.P, 16, 11)
        r.g_rgb.copy_(torch.as_tensor(g["rgb"])); r.g_depth.copy_(torch.as_tensor(g["depth"]))
        r.g_sil.copy_(torch.as_tensor(g["sil"])); r.g_feat.copy_(torch.as_tensor(g["feat"]))
        outs = []
        for blocks in (L.GS_BWD_BLOCKS_TILE, L.GS_BWD_BLOCKS_GROUP, L.GS_BWD_BLOCKS_DEFAULT):
            prm = raster.RasterParams(bwd_px_per_thread=np_, bwd_blocks=blocks)
            r.params, r.prm_c = prm, prm.c()
            r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
            outs.append([t.clone() for t in (r.d_means, r.d_quats, r.d_log_scales, r.d_logits, r.d_rgb,
                                             r.d_feat, r.d_twist)])
        for other in outs[1:]:
            for name, a, b in zip(("means", "quats", "log_scales", "logits", "rgb", "feat", "twist"), outs[0],
                                  other):
                C.assert_grad_close(name, b.cpu().numpy(), a.cpu().numpy(), 1e-5)
        # pose-only mode (tracking): the twist and the splat sums it is reduced from
        twists = []
        for blocks in (L.GS_BWD_BLOCKS_TILE, L.GS_BWD_BLOCKS_GROUP):
            prm = raster.RasterParams(bwd_px_per_thread=np_, bwd_blocks=blocks)
            r.params, r.prm_c = prm, prm.c()
            r.backward(field, L.GS_GRAD_POSE)
            twists.append((r.d_twist.clone(), r.sg_uvod.clone(), r.sg_conic.clone()))
        for name, a, b in zip(("twist", "uvod", "conic"), *twists):
            C.assert_grad_close("pose " + name, b.cpu().numpy(), a.cpu().numpy(), 1e-5)
    for bad in (raster.RasterParams(bwd_px_per_thread=4, bwd_blocks=L.GS_BWD_BLOCKS_GROUP),):
        r.params, r.prm_c = bad, bad.c()
        with pytest.raises(L.GsError):
            r.backward(field, L.GS_GRAD_MAP)
    r.use_blend_mask = False
    r.params = raster.RasterParams(bwd_blocks=L.GS_BWD_BLOCKS_GROUP)
    r.prm_c = r.params.c()
    r.forward(field)
    with pytest.raises(L.GsError):
        r.backward(field, L.GS_GRAD_MAP)


@pytest.mark.parametrize("D,np_", [(16, 1), (16, 2), (32, 1), (32, 2)])
def test_factored_feature_gradient_matches_the_feature_form(D, np_):
    """The loss's decoder-logit gradient e satisfies W^T e = its feature gradient, and the
    per-group backward given (e, W) returns the gradients it returns given W^T e, in map mode
    (every group) and pose mode (the twist), over a frame and a ragged second view."""
    gs, cam, room = C.room_case(20000, D, 200, 120, 100.0)
    cams = [cam, synth.camera(90, 61, 45.0, T_cw=synth.keyframe_loop(8, room=room)[3])]
    prm = raster.RasterParams(bwd_blocks=L.GS_BWD_BLOCKS_GROUP, bwd_px_per_thread=np_)
    field, r = C.gpu_forward(gs, cams, prm, n_classes=8)
    assert r.factored
    dec = synth.decoder(8, D, seed=3)
    Wd, bd = torch.as_tensor(dec.W).cuda(), torch.as_tensor(dec.b).cuda()
    rast = [synth.raycast_room(room, c) for c in cams]
    tg = dict(rgb=torch.as_tensor(np.concatenate([t.rgb.reshape(3, -1) for t in rast], 1)).cuda(),
              depth=torch.as_tensor(np.concatenate([t.depth.ravel() for t in rast])).cuda(),
              label=torch.as_tensor(np.concatenate([t.label.ravel() for t in rast])).cuda())
    r.loss(tg, Wd, bd, raster.MAPPING)
    g_feat = r.g_feat[:D].clone()
    r.loss(tg, Wd, bd, raster.MAPPING, factored=True)
    C.assert_grad_close("W^T e", (Wd.t() @ r.g_coef).cpu().numpy(), g_feat.cpu().numpy(), 1e-6)
    outs = []
    for fac in (False, True):
        r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE, factored=fac)
        outs.append([t.clone() for t in (r.d_means, r.d_quats, r.d_log_scales, r.d_logits, r.d_rgb, r.d_feat[:, :D],
                                         r.d_twist)])
    for name, a, b in zip(("means", "quats", "log_scales", "logits", "rgb", "feat", "twist"), *outs):
        C.assert_grad_close(name, b.cpu().numpy(), a.cpu().numpy(), 1e-5)
    twists = []
    for fac in (False, True):
        r.backward(field, L.GS_GRAD_POSE, factored=fac)
        twists.append(r.d_twist.clone())
    C.assert_grad_close("pose twist", twists[1].cpu().numpy(), twists[0].cpu().numpy(), 1e-5)


def test_blend_mask_skips_only_non_contributing_splats():
    """The backward with the forward's blend mask equals the full scan."""
    gs, cam, _ = C.room_case(20000, 16, 330, 190, 165.0)
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0])
    g = C.random_image_grads(r.P, 16, 8)
    r.g_rgb.copy_(torch.as_tensor(g["rgb"])); r.g_depth.copy_(torch.as_tensor(g["depth"]))
    r.g_sil.copy_(torch.as_tensor(g["sil"])); r.g_feat.copy_(torch.as_tensor(g["feat"]))
    outs = []
    for use_mask in (True, False):
        r.use_blend_mask = use_mask
        r.forward(field)
        r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
        outs.append([t.clone() for t in (r.d_means, r.d_quats, r.d_log_scales, r.d_logits, r.d_rgb, r.d_feat,
                                         r.d_twist)])
    for a, b in zip(*outs):
        C.assert_grad_close("masked", a.cpu().numpy(), b.cpu().numpy(), 1e-5)


def test_tile_order_is_a_longest_first_permutation_and_changes_nothing():
    """Two views: the launch order lists every tile once, by non-increasing instance count
    (in the order's count buckets), and rendering in it or in index order gives the same
    images and gradients."""
    gs, cam, room = C.room_case(20000, 16, 330, 190, 165.0)
    cams = [cam, synth.camera(100, 70, 60.0, T_cw=synth.keyframe_loop(8, room=room)[3])]
    field, r = C.gpu_forward(gs, cams, C.params_pair()[0])
    order = r.tile_order.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(r.n_tiles))
    rng_ = r.ranges.cpu().numpy().astype(np.int64).reshape(-1, 2)
    count = rng_[:, 1] - rng_[:, 0]
    bucket = np.where(count < 1024, count >> 2, np.minimum(256 + ((count - 1024) >> 6), 1023))
    assert np.all(np.diff(bucket[order]) <= 0)
    g = C.random_image_grads(r.P, 16, 9)
    r.g_rgb.copy_(torch.as_tensor(g["rgb"])); r.g_depth.copy_(torch.as_tensor(g["depth"]))
    r.g_sil.copy_(torch.as_tensor(g["sil"])); r.g_feat.copy_(torch.as_tensor(g["feat"]))
    imgs, grads = [], []
    for use_order in (True, False):
        r.use_tile_order = use_order
        r.forward(field)
        r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
        imgs.append([t.clone() for t in (r.img_rgb, r.img_depth, r.img_sil, r.img_feat, r.img_T, r.img_nc)])
        grads.append([t.clone() for t in (r.d_means, r.d_quats, r.d_log_scales, r.d_logits, r.d_rgb, r.d_feat,
                                          r.d_twist)])
    for a, b in zip(*imgs):
        assert torch.equal(a, b)
    for a, b in zip(*grads):
        C.assert_grad_close("ordered", a.cpu().numpy(), b.cpu().numpy(), 1e-5)


def test_blended_count_only_when_asked_leaves_the_images_alike():
    """The per-tile forward compiled with and without the blended-splat count (n_blended is
    asked for or not) renders the same images; the count is at most the 1-based position of the
    last blended splat, positive exactly where a splat was blended, and its sum over the frame
    is the number of blended (pixel, splat) pairs the blend mask's pairs bound."""
    gs, cam, _ = C.room_case(20000, 16, 330, 190, 165.0)
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0])
    names = ("img_rgb", "img_depth", "img_sil", "img_feat", "img_T", "img_nc", "blend_mask")
    r.count_blended = False
    r.render_fwd(field)
    torch.cuda.synchronize()
    plain = [getattr(r, n).clone() for n in names]
    r.count_blended = True
    r.img_nb.fill_(-1)
    r.render_fwd(field)
    torch.cuda.synchronize()
    for n, a in zip(names, plain):
        assert torch.equal(getattr(r, n), a), n
    nb, nc = r.img_nb.cpu().numpy(), r.img_nc.cpu().numpy()
    assert (nb >= 0).all() and (nb <= nc).all() and ((nb > 0) == (nc > 0)).all()
    assert nb.sum() > 0


def test_ring_forward_matches_one_block_per_tile():
    """The forward whose warps walk a ring of staged batch slots at their own pace renders the
    same images and blend mask, bit for bit, as one block per tile with CTA barriers: two views
    in the tile order and in index order, two slots of 128 or four of 64 splats; one 16x16 tile
    of 9,000 Gaussians (more than 4,096 instances, the tile's pixels saturate, so every warp
    leaves at the same batch before the end); D = 32 with three slots of 64.  Other pixels per
    thread and batch sizes are refused."""
    names = ("img_rgb", "img_depth", "img_sil", "img_feat", "img_T", "img_nc", "blend_mask")

    def render(r, field, base, blocks, batch):
        r.params = dataclasses.replace(base, fwd_px_per_thread=2, fwd_blocks=blocks, fwd_batch=batch)
        r.prm_c = r.params.c()
        r.project(field)
        r.bin_sort()
        r.render_fwd(field)
        torch.cuda.synchronize()
        assert r.status() == 0
        return [getattr(r, n).clone() for n in names]

    base = C.params_pair()[0]
    gs, cam, room = C.room_case(20000, 16, 330, 190, 165.0)
    cams = [cam, synth.camera(100, 70, 60.0, T_cw=synth.keyframe_loop(8, room=room)[3])]
    long_gs, long_cam = C.box_case(9000, 16, 16, 16, 12.0)
    d32_gs, d32_cam, _ = C.room_case(20000, 32, 200, 120, 100.0)
    for g, c, batches in ((gs, cams, (128, 64)), (long_gs, [long_cam], (128, 64)), (d32_gs, [d32_cam], (64,))):
        field, r = C.gpu_forward(g, c, base)
        for use_order in (True, False):
            r.use_tile_order = use_order
            ref = render(r, field, base, L.GS_BWD_BLOCKS_TILE, 0)
            for batch in batches:
                out = render(r, field, base, L.GS_BLOCKS_RING, batch)
                for n, a, b in zip(names, ref, out):
                    assert torch.equal(a, b), (g.n, use_order, batch, n)
        if g is long_gs:
            nc = r.img_nc.cpu().numpy()
            rg = r.ranges.cpu().numpy().astype(np.int64).reshape(-1, 2)
            assert (rg[:, 1] - rg[:, 0]).max() > 4096 and nc.max() < (rg[:, 1] - rg[:, 0]).max() - 256
    for np_, batch in ((1, 128), (4, 128), (2, 256)):
        r.params = dataclasses.replace(base, fwd_px_per_thread=np_, fwd_blocks=L.GS_BLOCKS_RING, fwd_batch=batch)
        r.prm_c = r.params.c()
        with pytest.raises(L.GsError) as e:
            r.render_fwd(field)
        assert e.value.status == L.GS_ERR_UNSUPPORTED


def test_queued_forward_matches_one_block_per_tile_and_resets_its_counters():
    """Two views: resident blocks taking tiles from the work counter render the same images
    and blend mask as one block per tile, for every pixels-per-thread shape and staged batch
    of 64, 128 or 256 splats, in the tile order and in index order; the counters are back at
    0 after each launch, so repeated launches after one binning agree; a NULL counter pointer
    and a batch of another size are refused."""
    gs, cam, room = C.room_case(20000, 16, 330, 190, 165.0)
    cams = [cam, synth.camera(100, 70, 60.0, T_cw=synth.keyframe_loop(8, room=room)[3])]
    base = C.params_pair()[0]
    field, r = C.gpu_forward(gs, cams, base)
    names = ("img_rgb", "img_depth", "img_sil", "img_feat", "img_T", "img_nc", "blend_mask")
    for use_order in (True, False):
        r.use_tile_order = use_order
        for np_ in (1, 2, 4):
            outs = []
            for blocks, batch in ((L.GS_BWD_BLOCKS_TILE, 0), (L.GS_BLOCKS_QUEUE, 0), (L.GS_BLOCKS_QUEUE, 128),
                                  (L.GS_BWD_BLOCKS_TILE, 64), (L.GS_BWD_BLOCKS_TILE, 256),
                                  (L.GS_BLOCKS_QUEUE, 64), (L.GS_BLOCKS_QUEUE, 256)):
                r.params = dataclasses.replace(base, fwd_px_per_thread=np_, fwd_blocks=blocks, fwd_batch=batch)
                r.prm_c = r.params.c()
                r.project(field)
                r.bin_sort()
                if batch in (64, 256) and np_ != 2:  # built for two pixels per thread (and D = 16, 32) only
                    with pytest.raises(L.GsError) as e:
                        r.render_fwd(field)
                    assert e.value.status == L.GS_ERR_UNSUPPORTED
                    continue
                for _ in range(2 if blocks == L.GS_BLOCKS_QUEUE else 1):
                    r.render_fwd(field)
                    torch.cuda.synchronize()
                    assert r.queue.cpu().tolist() == [0, 0]
                outs.append([getattr(r, n).clone() for n in names])
            for other in outs[1:]:
                for n, a, b in zip(names, outs[0], other):
                    assert torch.equal(a, b), (use_order, np_, n)
    r.params = dataclasses.replace(base, fwd_blocks=L.GS_BLOCKS_QUEUE)
    r.prm_c = r.params.c()
    b = r.binning_c()
    b.queue = None
    status = L.gs_render_fwd(ctypes.byref(field.c()), ctypes.byref(r.projected_c()), ctypes.byref(b), r.cams_c,
                             r.n_views, ctypes.byref(r.prm_c), ctypes.byref(r.images_c()), None)
    assert status == L.GS_ERR_ARG
    r.params = dataclasses.replace(base, fwd_batch=100)
    with pytest.raises(L.GsError) as e:
        r.prm_c = r.params.c()
        r.render_fwd(field)
    assert e.value.status == L.GS_ERR_ARG


def test_autotuner_picks_a_supported_shape():
    from paper_2603_27781_gb300 import autotune
    gs, cam, _ = C.room_case(20000, 16, 330, 190, 165.0)
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0])
    g = C.random_image_grads(r.P, 16, 6)
    r.g_rgb.copy_(torch.as_tensor(g["rgb"])); r.g_feat.copy_(torch.as_tensor(g["feat"]))
    tuned, t = autotune.tune_blend(r, field, L.GS_GRAD_MAP)
    assert set(t["fwd"]) == {1, 2, 4, "w1", "w2", "q1", "q2", "q4", "r2", "r2@64"}
    assert set(t["bwd"]) == {1, 2, 4, "w1", "w2"}
    kf, kb = autotune.shape_keys(tuned)
    assert kf in t["fwd"] and kb in t["bwd"]
    assert autotune.parse_shapes(f"{kf},{kb}") == {k: getattr(tuned, k) for k in (
        "fwd_px_per_thread", "fwd_blocks", "bwd_px_per_thread", "bwd_blocks")}


def test_render_bwd_multiview_sums_views():
    gs, cam, room = C.room_case(20000, 16, 160, 96, 80.0)
    poses = synth.keyframe_loop(8, room=room)
    cams = [synth.camera(160, 96, 80.0, T_cw=poses[1]), synth.camera(100, 70, 60.0, T_cw=poses[4])]
    prm_g, prm_o = C.params_pair()
    C.bwd_compare(gs, cams, prm_g, prm_o)


def test_half_storage_matches_oracle_on_rounded_values():
    """F16 colour and BF16 features, blended in f32: against the oracle fed the same rounded values."""
    gs, cam = C.box_case(2000, 16, 64, 48, 60.0)
    rounded = gs.copy()
    rounded.rgb = torch.as_tensor(gs.rgb).to(torch.float16).float().numpy()
    rounded.feat = torch.as_tensor(gs.feat).to(torch.bfloat16).float().numpy()
    prm_g, prm_o = C.params_pair()
    C.bwd_compare(gs, [cam], prm_g, prm_o, rgb_dtype=torch.float16, feat_dtype=torch.bfloat16, gs_oracle=rounded)


def test_pose_translation_gradient_invariant_on_gpu():
    """g_rho = R_cw sum_i g_mu,i, checked between two outputs of the CUDA path."""
    gs, cam, _ = C.room_case(20000, 8, 160, 96, 80.0)
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0])
    g = C.random_image_grads(r.P, 8, 3)
    r.g_rgb.copy_(torch.as_tensor(g["rgb"])); r.g_depth.copy_(torch.as_tensor(g["depth"]))
    r.g_sil.copy_(torch.as_tensor(g["sil"])); r.g_feat.copy_(torch.as_tensor(g["feat"]))
    r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
    R = torch.as_tensor(cam.T_cw[:3, :3])
    want = R @ r.d_means.double().sum(0).cpu()
    np.testing.assert_allclose(r.d_twist[0, :3].cpu().numpy(), want.numpy(), rtol=1e-4,
                               atol=1e-4 * float(want.abs().max()))


# --------------------------------------------------------------------- losses
def _loss_case(P_shape=(48, 64), D=16, K=8, seed=20, views=1):
    g = synth.rng(seed)
    H, W = P_shape
    cams = [synth.camera(W, H, 60.0) for _ in range(views)]
    imgs = [dict(rgb=g.random((3, H, W)), depth=g.uniform(2, 5, (H, W)), sil=g.uniform(0.9, 1.0, (H, W)),
                 feat=g.standard_normal((D, H, W))) for _ in range(views)]
    tgts = [synth.Frame(g.random((3, H, W)).astype(np.float32), (im["depth"] + g.normal(0, 0.05, (H, W))).astype(np.float32),
                        g.integers(0, K, (H, W)).astype(np.uint8)) for im in imgs]
    for t in tgts:
        t.depth[0, :5] = 0.0
        t.label[1, :7] = 255
    dec = synth.decoder(K, D, seed=seed + 1)
    imgs = [{k: v.astype(np.float32).astype(np.float64) for k, v in im.items()} for im in imgs]
    return cams, imgs, tgts, dec


@pytest.mark.parametrize("mode", ["mapping", "tracking"])
@pytest.mark.parametrize("views", [1, 2])
def test_loss_matches_oracle(mode, views):
    _check_loss(mode, views, 16, 8)


@pytest.mark.parametrize("D,K", [(32, 13), (8, 32), (4, 3), (32, 8)])
def test_loss_feature_and_class_widths(D, K):
    """The compile-time class bounds (8 and 32) and every staged feature width."""
    _check_loss("mapping", 1, D, K)


@pytest.mark.parametrize("views,shape", [(1, (48, 64)), (2, (45, 70))])
def test_loss_with_ssim_matches_oracle(views, shape):
    """Eq. 15 with lambda = 0.2: the SSIM tiles (32x16 with a 5-pixel halo) over whole and
    ragged frames, one and two views."""
    _check_loss("mapping_ssim", views, 16, 8, shape)


def _check_loss(mode, views, D, K, shape=(48, 64)):
    cams, imgs, tgts, dec = _loss_case(P_shape=shape, views=views, D=D, K=K)
    w = dict(mapping=raster.MAPPING, mapping_ssim=raster.MAPPING_SSIM, tracking=raster.TRACKING)[mode]
    wo = dict(mapping=oracle.MAPPING, mapping_ssim=oracle.MAPPING_SSIM, tracking=oracle.TRACKING)[mode]
    r = raster.Renderer(0, cams, D, 0, n_classes=K)
    cat = lambda key, f=lambda a: a: torch.as_tensor(np.concatenate([f(im[key]).reshape(im[key].shape[0], -1)
                                                                     if im[key].ndim == 3 else f(im[key]).reshape(1, -1)
                                                                     for im in imgs], 1), dtype=torch.float32).cuda()
    r.img_rgb.copy_(cat("rgb")); r.img_depth.copy_(cat("depth")[0]); r.img_sil.copy_(cat("sil")[0])
    r.img_feat.copy_(cat("feat"))
    tg = dict(rgb=torch.as_tensor(np.concatenate([t.rgb.reshape(3, -1) for t in tgts], 1)).cuda(),
              depth=torch.as_tensor(np.concatenate([t.depth.ravel() for t in tgts])).cuda(),
              label=torch.as_tensor(np.concatenate([t.label.ravel() for t in tgts])).cuda())
    Wd, bd = torch.as_tensor(dec.W).cuda(), torch.as_tensor(dec.b).cuda()
    r.loss(tg, Wd, bd, w)
    torch.cuda.synchronize()
    total, dW, db = 0.0, 0.0, 0.0
    for v, (im, t) in enumerate(zip(imgs, tgts)):
        o = oracle.loss(im, t, dec, wo)
        a, b = r.pix_off[v], r.pix_off[v + 1]
        H, W = r.sizes[v]
        if mode == "tracking":
            # the median is an integer decision taken on the f32 depth errors
            e = np.abs(im["depth"].astype(np.float32) - t.depth)[t.depth > 0]
            assert r.median[v].item() == np.float32(oracle.lower_median(e.astype(np.float64)))
            gmask = r.mask[a:b].cpu().numpy().reshape(H, W)
            near = np.abs(np.abs(im["depth"] - t.depth) - 10 * o["median"]) < 1e-5 * o["median"]
            assert (gmask != o["mask"])[~near].sum() == 0
        # the SSIM gradient is a sum of 121 window terms over f32 moments: 1e-4 of the largest
        atol = 1e-9 if not w.ssim else 1e-4 * np.abs(o["rgb"]).max()
        np.testing.assert_allclose(r.g_rgb[:, a:b].cpu().numpy().reshape(3, H, W), o["rgb"], atol=atol)
        np.testing.assert_allclose(r.g_depth[a:b].cpu().numpy().reshape(H, W), o["depth"], atol=1e-9)
        np.testing.assert_allclose(r.g_feat[:, a:b].cpu().numpy().reshape(D, H, W), o["feat"], atol=1e-9,
                                   rtol=1e-5)
        total += o["total"]
        dW = dW + o["W"]
        db = db + o["b"]
    assert r.loss_out[0].item() == pytest.approx(total, rel=1e-5)
    C.assert_grad_close("dW", r.d_dec_W.cpu().numpy(), dW, 1e-5)
    C.assert_grad_close("db", r.d_dec_b.cpu().numpy(), db, 1e-5)


def test_median_is_bit_exact_on_large_views():
    g = synth.rng(33)
    cams = [synth.camera(1200, 680, 600.0), synth.camera(640, 480, 525.0)]
    r = raster.Renderer(0, cams, 0, 0, n_classes=1)
    depth = g.uniform(0.5, 6.0, r.P).astype(np.float32)
    tdepth = (depth + g.standard_normal(r.P).astype(np.float32) * 0.02).astype(np.float32)
    tdepth[g.random(r.P) < 0.1] = 0.0
    r.img_depth.copy_(torch.as_tensor(depth))
    r.img_sil.fill_(1.0)
    tg = dict(rgb=torch.zeros(3, r.P, device="cuda"), depth=torch.as_tensor(tdepth).cuda(),
              label=torch.full((r.P,), 255, dtype=torch.uint8, device="cuda"))
    r.loss(tg, None, None, raster.TRACKING)
    for v in range(2):
        a, b = r.pix_off[v], r.pix_off[v + 1]
        e = np.abs(depth[a:b] - tdepth[a:b])[tdepth[a:b] > 0]
        assert r.median[v].item() == np.float32(oracle.lower_median(e.astype(np.float64)))


def test_cleared_sums_accumulate_like_the_clearing_backward():
    """gs_splat_grads_clear on the side stream beside the forward, then gs_render_bwd with
    GS_GRAD_ACCUMULATE, gives the sums of gs_render_bwd's own clearing (the atomic sums agree
    to their rounding), whatever the buffers held before; a second accumulating call adds the
    same sums again."""
    gs, cam = C.box_case(2000, 16, 64, 48, 60.0)
    prm = C.params_pair()[0]
    mode = L.GS_GRAD_MAP | L.GS_GRAD_POSE
    field, r = C.gpu_forward(gs, cam, prm)
    g = torch.Generator(device="cuda").manual_seed(5)
    for t in (r.g_rgb, r.g_depth, r.g_feat):
        t.copy_(torch.randn(t.shape, generator=g, device="cuda"))
    sums = lambda: [t.clone() for t in (r.sg_uvod, r.sg_conic, r.sg_rgb, r.d_feat)]
    r.render_bwd(field, mode)
    torch.cuda.synchronize()
    ref = sums()
    for t in (r.sg_uvod, r.sg_conic, r.sg_rgb, r.d_feat):
        t.fill_(3.0)
    r.side_start(lambda s: r.clear_grads(field, mode, s))
    r.render_fwd(field)
    r.side_join()
    r.render_bwd(field, mode, accumulate=True)
    torch.cuda.synchronize()
    once = sums()
    r.render_bwd(field, mode, accumulate=True)
    torch.cuda.synchronize()
    twice = sums()
    for a, b, c in zip(ref, once, twice):
        tol = 1e-5 * float(a.abs().max()) + 1e-30
        assert float((a - b).abs().max()) <= tol
        assert float((2 * a - c).abs().max()) <= 2 * tol
    assert float(ref[0].abs().max()) > 0 and float(ref[3].abs().max()) > 0


def test_dsr_in_two_halves_equals_one_call():
    """gs_dsr_value on a side stream (its own scratch) followed by gs_dsr_grad gives the
    value and the gradient of gs_dsr bit for bit."""
    gs, _, _ = C.room_case(200000, 0, 64, 48, 60.0)
    ls = torch.as_tensor(gs.log_scales).cuda()
    r = raster.Renderer(gs.n, [synth.camera(64, 48, 60.0)], 0, 0)
    field = raster.Field(torch.zeros(gs.n, 3).cuda(), torch.zeros(gs.n, 4).cuda(), ls, torch.zeros(gs.n).cuda(),
                         torch.zeros(gs.n, 3).cuda(), torch.zeros(gs.n, 0).cuda())
    base = torch.randn(gs.n, 3, generator=torch.Generator().manual_seed(3)).cuda()
    r.d_log_scales.copy_(base)
    r.dsr(field, 0.01, 0.001)
    torch.cuda.synchronize()
    one = (r.dsr_out.clone(), r.d_log_scales.clone())
    r.d_log_scales.copy_(base)
    r.dsr_out.zero_()
    r.side_start(lambda s: r.dsr_value(field, 0.01, 0.001, s))
    r.side_by_side(lambda s: r.dsr_grad(field, 0.01, 0.001, s), lambda: None)
    torch.cuda.synchronize()
    assert torch.equal(r.dsr_out, one[0]) and torch.equal(r.d_log_scales, one[1])
    assert float(one[0][3]) > 0                                  # the large-scale set is not empty


def test_dsr_matches_oracle():
    gs, _, _ = C.room_case(200000, 0, 64, 48, 60.0)
    ls = torch.as_tensor(gs.log_scales).cuda()
    r = raster.Renderer(gs.n, [synth.camera(64, 48, 60.0)], 0, 0)
    r.d_log_scales.zero_()
    field = raster.Field(torch.zeros(gs.n, 3).cuda(), torch.zeros(gs.n, 4).cuda(), ls, torch.zeros(gs.n).cuda(),
                         torch.zeros(gs.n, 3).cuda(), torch.zeros(gs.n, 0).cuda())
    r.dsr(field, 0.01, 0.001)
    torch.cuda.synchronize()
    val, grad, st = oracle.dsr(gs.log_scales, 0.01, 0.001)
    s = np.exp(gs.log_scales.astype(np.float64))
    # membership of a scale within f32 rounding of mu +- 2 sigma may be decided either way
    near = (np.abs(s - (st["mu"] + 2 * st["sigma"])) < 1e-6 * s) | (np.abs(s - (st["mu"] - 2 * st["sigma"])) < 1e-6 * s)
    assert near.sum() <= 10
    out = r.dsr_out.cpu().numpy()
    nb = near.sum()
    assert abs(out[3] - st["n_big"]) + abs(out[4] - st["n_small"]) <= nb
    assert out[0] == pytest.approx(val, rel=1e-5 + nb / max(min(st["n_big"], st["n_small"]), 1))
    g = r.d_log_scales.cpu().numpy()
    if nb == 0:
        np.testing.assert_allclose(g, grad, rtol=1e-5, atol=1e-12)
    else:   # the per-member gradient is lam / n: compare where both sides agree on membership
        agree = (g != 0) == (grad != 0)
        assert (~agree).sum() <= nb
        np.testing.assert_allclose(g[agree & ~near], grad[agree & ~near], rtol=nb / 1000 + 1e-5, atol=1e-12)


def test_pose_step_matches_oracle():
    T = synth.look_pose((1.0, 2.0, 1.5), (0.3, 1.0, -0.1))
    g = synth.rng(40)
    r = raster.Renderer(0, [synth.camera(64, 48, 60.0)], 0, 0)
    Ts = torch.as_tensor(T.reshape(1, 16)).cuda()
    adam = torch.zeros(1, 12, dtype=torch.float64, device="cuda")
    Tf = torch.zeros(1, 16, device="cuda")
    Tref, m, v = T.copy(), np.zeros(6), np.zeros(6)
    for step in range(1, 4):
        grad = g.standard_normal(6)
        r.d_twist.copy_(torch.as_tensor(grad.reshape(1, 6)))
        r.pose_step(Ts, adam, step, pose_f32=Tf)
        Tref, m, v = oracle.pose_step(Tref, grad, m, v, step, np.array(raster.TRACKING_LR))
    np.testing.assert_allclose(Ts.cpu().numpy().reshape(4, 4), Tref, atol=1e-12)
    np.testing.assert_allclose(Tf.cpu().numpy().reshape(4, 4), Tref, atol=1e-6)


def test_pose_step_large_and_small_rotations_match_oracle():
    """Adam steps whose rotation increments lie above 0.05 rad (the exponential's coefficients
    from sin and cos) and below it (their Taylor series), on both sides of the switch, against
    the oracle's closed form."""
    T = synth.look_pose((1.0, 2.0, 1.5), (0.3, 1.0, -0.1))
    g = synth.rng(43)
    r = raster.Renderer(0, [synth.camera(64, 48, 60.0)], 0, 0)
    for rot_lr in (0.06, 0.02):  # first-step |phi| = rot_lr * sqrt(3): 0.104 and 0.035 rad
        lr = np.array([0.01, 0.01, 0.01, rot_lr, rot_lr, rot_lr])
        Ts = torch.as_tensor(T.reshape(1, 16)).cuda()
        adam = torch.zeros(1, 12, dtype=torch.float64, device="cuda")
        Tref, m, v = T.copy(), np.zeros(6), np.zeros(6)
        for step in range(1, 4):
            grad = g.standard_normal(6)
            r.d_twist.copy_(torch.as_tensor(grad.reshape(1, 6)))
            r.pose_step(Ts, adam, step, lr=tuple(lr))
            Tref, m, v = oracle.pose_step(Tref, grad, m, v, step, lr)
        np.testing.assert_allclose(Ts.cpu().numpy().reshape(4, 4), Tref, atol=1e-12)
        assert abs(np.arccos(np.clip((np.trace(Tref[:3, :3] @ T[:3, :3].T) - 1) / 2, -1, 1))) > 0.02


# ---------------------------------------------------------------- whole step
@pytest.mark.parametrize("exact,ssim", [(True, False), (False, False), (False, True)])
def test_full_iteration_tiny_scene(exact, ssim):
    """Box scene, 64x48, mapping loss + DSR + pose twist vs oracle.step.  In exact mode (no
    thresholds) every pixel is comparable; the default-threshold scene (seed 11) has no pixel
    within rounding distance of a decision, so the whole iteration is compared."""
    # exact mode has no T_min stop: keep the field thin enough that T stays far above f32 underflow
    gs, cam = C.box_case(300 if exact else 2000, 16, 64, 48, 60.0, seed=0 if exact else 11)
    kw = dict(alpha_min=0.0, alpha_max=1.0, T_min=0.0, radius_sigma=8.0) if exact else {}
    prm_g, prm_o = C.params_pair(**kw)
    dec = synth.decoder(8, 16)
    tgt_img = oracle.forward(synth.jitter_means(gs), cam, prm_o)[2]
    f = tgt_img["feat"].reshape(16, -1).T
    label = np.argmax(f @ dec.W.T.astype(np.float64) + dec.b, 1).astype(np.uint8).reshape(48, 64)
    tgt = synth.Frame(tgt_img["rgb"].astype(np.float32), tgt_img["depth"].astype(np.float32), label)
    wo, wg = (oracle.MAPPING_SSIM, raster.MAPPING_SSIM) if ssim else (oracle.MAPPING, raster.MAPPING)
    ref = oracle.step(gs, cam, prm_o, tgt, dec, wo)
    field, r = C.gpu_forward(gs, cam, prm_g, n_classes=8)
    ex = C.exclusion(cam, ref["proj"], C.gpu_projection(r), ref["img"], prm_o.alpha_min)
    assert ex.check("whole iteration").mask.sum() == 0
    tg = dict(rgb=torch.as_tensor(tgt.rgb.reshape(3, -1)).cuda(), depth=torch.as_tensor(tgt.depth.ravel()).cuda(),
              label=torch.as_tensor(tgt.label.ravel()).cuda())
    r.iteration(field, tg, torch.as_tensor(dec.W).cuda(), torch.as_tensor(dec.b).cuda(), wg,
                L.GS_GRAD_MAP | L.GS_GRAD_POSE)
    torch.cuda.synchronize()
    total = r.loss_out[0].item() + r.dsr_out[0].item()
    assert total == pytest.approx(ref["total"], rel=1e-5)
    gr = ref["grads"]
    for k, t in dict(means=r.d_means, quats=r.d_quats, log_scales=r.d_log_scales, opacity_logits=r.d_logits,
                     rgb=r.d_rgb, feat=r.d_feat, twist=r.d_twist[0], W=r.d_dec_W, b=r.d_dec_b).items():
        C.assert_grad_close(k, t.cpu().numpy(), gr[k])


def test_autograd_function_matches_direct_backward():
    gs, cam = C.box_case(2000, 8, 64, 48, 60.0)
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0])
    params = [torch.as_tensor(a).cuda().requires_grad_(True) for a in gs.arrays()]
    rgb, depth, sil, feat = raster.rasterize(r, *params)
    g = C.random_image_grads(r.P, 8, 11)
    gl = [torch.as_tensor(g[k], dtype=torch.float32).cuda() for k in ("rgb", "depth", "sil", "feat")]
    loss = (rgb * gl[0]).sum() + (depth * gl[1]).sum() + (sil * gl[2]).sum() + (feat * gl[3]).sum()
    loss.backward()
    r.g_rgb.copy_(gl[0]); r.g_depth.copy_(gl[1]); r.g_sil.copy_(gl[2]); r.g_feat.copy_(gl[3])
    r.backward(field, L.GS_GRAD_MAP)
    # same kernels, same inputs: equal up to the order of the float atomics
    for name, p, d in zip(("means", "quats", "log_scales", "logits", "rgb", "feat"), params,
                          (r.d_means, r.d_quats, r.d_log_scales, r.d_logits, r.d_rgb, r.d_feat)):
        C.assert_grad_close(name, p.grad.cpu().numpy(), d.cpu().numpy(), 1e-5)


def _autograd_grads(r, gs, gl):
    """Parameter gradients of sum_k <image_k, gl_k> through RasterizeSG."""
    params = [torch.as_tensor(a).cuda().requires_grad_(True) for a in gs.arrays()]
    rgb, depth, sil, feat = raster.rasterize(r, *params)
    loss = (rgb * gl[0]).sum() + (depth * gl[1]).sum() + (sil * gl[2]).sum() + (feat * gl[3]).sum()
    loss.backward()
    return dict(zip(("means", "quats", "log_scales", "opacity_logits", "rgb", "feat"),
                    (p.grad.double().cpu().numpy() for p in params)))


@pytest.mark.parametrize("name", ["box_64x48", "room_20k_330x190"])
def test_autograd_function_matches_oracle(name):
    """Gradients of a linear functional of the rendered images through the torch.autograd
    wrapper against the oracle's analytic backward of the same functional (upstream gradients
    zero at the excluded pixels)."""
    gs, cam = CASES[name]()
    prm_g, prm_o = C.params_pair()
    field, r = C.gpu_forward(gs, cam, prm_g)
    proj, bins, oimg = oracle.forward(gs, cam, prm_o)
    ex = C.exclusion(cam, proj, C.gpu_projection(r), oimg).check(f"autograd {name}")
    g = C.random_image_grads(r.P, gs.feat_dim, 12)
    keep = ~ex.mask.ravel()
    gl = [torch.as_tensor(g[k] * keep, dtype=torch.float32).cuda() for k in ("rgb", "depth", "sil", "feat")]
    got = _autograd_grads(r, gs, gl)
    H, W = cam.height, cam.width
    gimg = {k: (g[k] * keep).reshape((-1, H, W) if g[k].ndim == 2 else (H, W)) for k in g}
    want = oracle.backward_from_image_grads(gs, cam, prm_o, proj, bins, gimg)
    for k, v in got.items():
        C.assert_grad_close(k, v, want[k])


def test_autograd_function_matches_central_differences():
    """The wrapper's gradients against FP64 central differences (step 1e-6) of the oracle's
    render of the same functional, in exact mode (Eq. 4-7 without thresholds), on 24
    parameters drawn over every group."""
    gs, cam = C.box_case(300, 4, 48, 40, 45.0, seed=5)
    kw = dict(alpha_min=0.0, alpha_max=1.0, T_min=0.0, radius_sigma=8.0)
    prm_g, prm_o = C.params_pair(**kw)
    field, r = C.gpu_forward(gs, cam, prm_g)
    g = C.random_image_grads(r.P, 4, 13)
    gl = [torch.as_tensor(g[k], dtype=torch.float32).cuda() for k in ("rgb", "depth", "sil", "feat")]
    got = _autograd_grads(r, gs, gl)
    H, W = cam.height, cam.width
    gimg = {k: v.reshape((-1, H, W) if v.ndim == 2 else (H, W)) for k, v in g.items()}
    base = synth.Gaussians(*(a.astype(np.float64) for a in gs.arrays()))

    def functional(x):
        img = oracle.forward(x, cam, prm_o)[2]
        return sum(float((img[k] * gimg[k]).sum()) for k in gimg)

    rng_ = synth.rng(14)
    h = 1e-6
    for k in range(24):
        name = ("means", "quats", "log_scales", "opacity_logits", "rgb", "feat")[k % 6]
        arr = getattr(base, name)
        idx = np.unravel_index(int(rng_.integers(arr.size)), arr.shape)
        keep = arr[idx]
        arr[idx] = keep + h
        fp = functional(base)
        arr[idx] = keep - h
        fm = functional(base)
        arr[idx] = keep
        fd = (fp - fm) / (2 * h)
        scale = np.abs(got[name]).max()
        assert abs(got[name][idx] - fd) <= 1e-3 * max(abs(fd), 1e-2 * scale), (name, idx, got[name][idx], fd)


# ----------------------------------------------------------------- edge cases
def test_empty_field_renders_background():
    cam = synth.camera(50, 37, 40.0)
    prm = raster.RasterParams(bg=(0.2, 0.4, 0.6))
    gs = synth.box_field(0, 8)
    field, r = C.gpu_forward(gs, cam, prm, capacity=16)
    img = C.np_images(r)
    for c in range(3):
        np.testing.assert_array_equal(img["rgb"][c], np.float32(prm.bg[c]))
    assert (img["depth"] == 0).all() and (img["sil"] == 0).all() and (img["T"] == 1).all()
    assert (img["n_contrib"] == 0).all() and r.instances() == 0 and r.status() == 0


def test_all_culled_field():
    gs, cam = C.box_case(500, 8, 40, 30, 40.0)
    gs.means[:, 2] *= -1
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0], capacity=64)
    assert r.instances() == 0 and r.status() == 0
    r.g_rgb.fill_(1.0); r.g_depth.fill_(1.0); r.g_feat.fill_(1.0)
    r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
    for t in (r.d_means, r.d_quats, r.d_log_scales, r.d_logits, r.d_rgb, r.d_feat, r.d_twist):
        assert not bool(t.abs().max() > 0)


def test_capacity_overflow_is_reported():
    gs, cam = C.box_case(2000, 8, 64, 48, 60.0)
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0], capacity=100)
    assert r.status() == L.GS_ERR_CAPACITY
    op = oracle.project(gs, cam, oracle.Params())
    assert r.instances() == int(op["touched"].sum())


def test_bounded_wait_that_gives_up_reports_timeout_and_renders_nothing():
    """With the spin limit's test hook every radix-sort block after the first gives up its
    look-back at once (8,000 visible Gaussians and about 31,600 instances: several blocks in
    every pass): the binning reports GS_ERR_TIMEOUT, the ranges stay empty, and the blend
    kernels leave the images and the gradients as they were (the images keep a sentinel, the
    zeroed gradients stay zero).  The same renderer then renders normally again."""
    gs, cam = C.box_case(8000, 16, 160, 120, 150.0)
    field, r = C.gpu_forward(gs, cam, C.params_pair()[0])
    assert r.instances() > 2 * 8192                   # the tile sort has several 8192-key blocks
    good = {k: v.clone() for k, v in r.images().items()}
    for t in (r.img_rgb, r.img_depth, r.img_sil, r.img_feat, r.img_T):
        t.fill_(-7.0)
    r.params = raster.RasterParams(spin_limit=-1)
    r.prm_c = r.params.c()
    r.forward(field)
    r.g_rgb.fill_(1.0); r.g_depth.fill_(1.0); r.g_feat.fill_(1.0)
    r.backward(field, L.GS_GRAD_MAP | L.GS_GRAD_POSE)
    torch.cuda.synchronize()
    assert r.status() == L.GS_ERR_TIMEOUT
    assert int(r.ranges.view(torch.int32).abs().max()) == 0
    for t in (r.img_rgb, r.img_depth, r.img_sil, r.img_feat, r.img_T):
        assert bool((t == -7.0).all())
    for t in (r.d_means, r.d_quats, r.d_log_scales, r.d_logits, r.d_rgb, r.d_feat, r.d_twist):
        assert not bool(t.abs().max() > 0)
    r.params = raster.RasterParams()
    r.prm_c = r.params.c()
    r.forward(field)
    torch.cuda.synchronize()
    assert r.status() == 0
    for k, v in r.images().items():
        assert torch.equal(v, good[k]), k


def test_argument_errors_return_status():
    gs, cam = C.box_case(10, 8, 32, 32, 30.0)
    field = raster.Field.from_numpy(gs)
    r = raster.Renderer(gs.n, [cam], 8, 64)
    bad = raster.RasterParams(tile=8)
    with pytest.raises(L.GsError) as e:
        r.prm_c = bad.c()
        r.project(field)
    assert e.value.status == L.GS_ERR_ARG
