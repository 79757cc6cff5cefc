"""The mapping update (gs_adam_step) and whole mapping iterations.

Adam against the oracle's FP64 restatement over three steps (host-numbered and
device-counted, aligned and ragged array lengths); one mapping iteration of the
tiny scene (forward, the Eq. 15 loss with SSIM, backward, DSR, update) against
oracle.step + oracle.adam_step; and the whole iteration replayed from one CUDA
graph.  Adam normalises every gradient, so a parameter whose gradient is within
rounding of zero may step either way: the iteration's update is compared where
the gradient is well determined and checked to stay within the learning rate
elsewhere.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_27781_gb300 import raster, synth
from paper_2603_27781_gb300 import _lib as L

import gpu_cases as C

pytestmark = pytest.mark.gpu

GROUPS = oracle.ADAM_GROUPS
GRAD_NAME = dict(means="d_means", quats="d_quats", log_scales="d_log_scales", opacity_logits="d_logits",
                 rgb="d_rgb", feat="d_feat")


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    from paper_2603_27781_gb300 import build
    build.build()
    L.library()


@pytest.mark.parametrize("n,D", [(1000, 16), (1001, 8), (37, 0)])
def test_adam_step_matches_oracle(n, D):
    gs = synth.box_field(n, D, seed=n)
    field = raster.Field.from_numpy(gs, "cuda")
    r = raster.Renderer(n, [synth.camera(16, 16, 10.0)], D, 0)
    opt = raster.MappingAdam(field)
    assert dict(zip(GROUPS, opt.lr)) == oracle.MAPPING_LR
    g = synth.rng(n + 1)
    p_ref = {k: getattr(gs, k).astype(np.float64) for k in GROUPS}
    z = {k: np.zeros_like(p_ref[k]) for k in GROUPS}
    m_ref, v_ref = dict(z), dict(z)
    for step in (1, 2, 0):      # two host-numbered steps, then the device counter
        grads = {k: g.standard_normal(p_ref[k].shape).astype(np.float32) for k in GROUPS}
        grads["feat"][: n // 5] = 0.0
        for k in GROUPS:
            t = getattr(r, GRAD_NAME[k])
            t.zero_()
            if grads[k].size:
                t.view(-1)[: grads[k].size] = torch.as_tensor(grads[k].ravel()).cuda()
        if step == 0:
            opt.step_ctr.fill_(2.0)      # continue at t = 3 on the device
        opt.step(r, step)
        p_ref, m_ref, v_ref = oracle.adam_step(p_ref, grads, m_ref, v_ref, step if step else 3,
                                               oracle.MAPPING_LR)
    torch.cuda.synchronize()
    assert opt.step_ctr.item() == 3.0
    M = n * (14 + D)
    mom = opt.moments.cpu().numpy().astype(np.float64)
    off = 0
    for k in GROUPS:
        if k == "feat" and D == 0:
            continue
        got = getattr(field, k).cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, p_ref[k], rtol=3e-7, atol=1e-4 * oracle.MAPPING_LR[k], err_msg=k)
        size = p_ref[k].size
        # m is a sum of terms 0.1 g ~ 0.1 that may cancel: f32 rounding of ~1e-8 absolute
        np.testing.assert_allclose(mom[off:off + size], m_ref[k].ravel(), rtol=1e-5, atol=1e-7, err_msg=k)
        np.testing.assert_allclose(mom[M + off:M + off + size], v_ref[k].ravel(), rtol=1e-5, atol=1e-12,
                                   err_msg=k)
        off += size


def _tiny_mapping_case():
    gs, cam = C.box_case(2000, 16, 64, 48, 60.0, seed=11)
    prm_g, prm_o = C.params_pair()
    dec = synth.decoder(8, 16)
    tgt_img = oracle.forward(synth.jitter_means(gs), cam, prm_o)[2]
    f = tgt_img["feat"].reshape(16, -1).T
    label = np.argmax(f @ dec.W.T.astype(np.float64) + dec.b, 1).astype(np.uint8).reshape(48, 64)
    tgt = synth.Frame(tgt_img["rgb"].astype(np.float32), tgt_img["depth"].astype(np.float32), label)
    return gs, cam, prm_g, prm_o, dec, tgt


def _targets(tgt):
    return dict(rgb=torch.as_tensor(tgt.rgb.reshape(3, -1)).cuda(), depth=torch.as_tensor(tgt.depth.ravel()).cuda(),
                label=torch.as_tensor(tgt.label.ravel()).cuda())


def test_mapping_iteration_with_update_matches_oracle():
    """Forward, mapping loss with SSIM (Eq. 15, lambda 0.2), backward, DSR and the Adam update
    against the oracle's iteration followed by its Adam step."""
    gs, cam, prm_g, prm_o, dec, tgt = _tiny_mapping_case()
    ref = oracle.step(gs, cam, prm_o, tgt, dec, oracle.MAPPING_SSIM)
    z = {k: np.zeros_like(getattr(gs, k), dtype=np.float64) for k in GROUPS}
    p_ref, _, _ = oracle.adam_step({k: getattr(gs, k) for k in GROUPS}, ref["grads"], z, z, 1, oracle.MAPPING_LR)
    field, r = C.gpu_forward(gs, cam, prm_g, n_classes=8)
    # every pixel of this scene is determined to the tolerances by its f32 inputs
    ex = C.exclusion(cam, ref["proj"], C.gpu_projection(r), ref["img"], prm_o.alpha_min)
    assert ex.check("mapping iteration").mask.sum() == 0
    opt = raster.MappingAdam(field)
    r.iteration(field, _targets(tgt), torch.as_tensor(dec.W).cuda(), torch.as_tensor(dec.b).cuda(),
                raster.MAPPING_SSIM, L.GS_GRAD_MAP)
    opt.step(r, 1)
    torch.cuda.synchronize()
    assert r.loss_out[0].item() + r.dsr_out[0].item() == pytest.approx(ref["total"], rel=1e-5)
    for k in GROUPS:
        g = np.asarray(ref["grads"][k], np.float64)
        p0 = getattr(gs, k).astype(np.float64)
        got = getattr(field, k).cpu().numpy().astype(np.float64)
        step_gpu, step_ref = got - p0, p_ref[k] - p0
        lr = oracle.MAPPING_LR[k]
        sure = np.abs(g) > 1e-2 * np.abs(g).max()       # gradient well above the parity tolerance
        assert sure.sum() > 0.05 * g.size, k
        ulp = 4e-7 * np.abs(p0).max()                    # f32 rounding of the stored parameter
        np.testing.assert_allclose(step_gpu[sure], step_ref[sure], rtol=0, atol=1e-3 * lr + ulp, err_msg=k)
        assert np.abs(step_gpu).max() <= lr * (1 + 1e-3) + ulp, k


def test_mapping_iterations_replay_from_one_graph():
    """Three mapping iterations (forward, loss with SSIM, backward, DSR, update with the device
    step counter) as one captured graph: the first iteration's loss equals the eager one bit for
    bit (same parameters, deterministic forward), the counter reaches 3 and the loss falls."""
    gs, cam, prm_g, _, dec, tgt = _tiny_mapping_case()
    field, r = C.gpu_forward(gs, cam, prm_g, n_classes=8)
    tg = _targets(tgt)
    W, b = torch.as_tensor(dec.W).cuda(), torch.as_tensor(dec.b).cuda()
    r.iteration(field, tg, W, b, raster.MAPPING_SSIM, L.GS_GRAD_MAP)
    torch.cuda.synchronize()
    eager_loss = r.loss_out[0].item()
    start = {k: getattr(field, k).clone() for k in GROUPS}
    opt = raster.MappingAdam(field)
    losses = torch.zeros(3, dtype=torch.float64, device="cuda")

    def iterations():
        for i in range(3):
            r.iteration(field, tg, W, b, raster.MAPPING_SSIM, L.GS_GRAD_MAP)
            losses[i:i + 1].copy_(r.loss_out[:1])
            opt.step(r, 0)

    cur = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        iterations()
    cur.wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        iterations()
    for k in GROUPS:
        getattr(field, k).copy_(start[k])
    opt.moments.zero_()
    opt.step_ctr.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert r.status() == 0
    assert opt.step_ctr.item() == 3.0
    ls = losses.cpu().numpy()
    assert ls[0] == eager_loss
    assert ls[2] < ls[0]
