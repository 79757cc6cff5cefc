"""The RSKM keyframe draw (Eq. 13) and the whole SLAM loop on the GPU.

gs_rskm_draw against the oracle's rule (slots, the gather of the drawn frame and its pose,
the device counter, graph replay); the loop of tracking (Eq. 19-21), expansion (Eq. 11) and
RSKM mapping (Eq. 13-18) over a short sequence against the oracle's loop: the same draws,
the same first-frame field, field sizes and poses that follow the oracle's, and a final map
that renders like the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_27781_gb300 import raster, slam, synth
from paper_2603_27781_gb300 import _lib as L

import gpu_cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    from paper_2603_27781_gb300 import build
    build.build()
    L.library()


def _store(cap, W, H, seed=80):
    g = synth.rng(seed)
    P = W * H
    st = slam.KeyframeStore(cap, W, H)
    st.rgb.copy_(torch.as_tensor(g.random((cap, 3, P)).astype(np.float32)))
    st.depth.copy_(torch.as_tensor(g.uniform(0.5, 5.0, (cap, P)).astype(np.float32)))
    st.label.copy_(torch.as_tensor(g.integers(0, 256, (cap, P)).astype(np.uint8)))
    st.T.copy_(torch.as_tensor(g.standard_normal((cap, 16))))
    return st


@pytest.mark.parametrize("W,H", [(64, 48), (37, 23)])      # vector and scalar gather
def test_rskm_draw_and_gather_follow_the_oracle_rule(W, H):
    cap = 5
    st = _store(cap, W, H)
    draws = synth.rskm_draws(64, seed=81)
    smp = slam.RskmSampler(st, draws)
    # (n_kf, current slot, t_opt, first word, iterations)
    for n_kf, cur, t_opt, off, cnt in [(3, 3, 2, 0, 10), (4, 2, 3, 10, 9), (0, 0, 1, 19, 4), (4, 4, 2, 23, 12)]:
        smp.begin(off, cnt, n_kf, cur, t_opt)
        for k in range(cnt + 2):                           # two past the window: words wrap around
            smp.draw()
            torch.cuda.synchronize()
            want = oracle.rskm_select(k, t_opt, cur, list(range(n_kf)), draws[off + k % cnt])
            slot = int(smp.state[1].item())
            assert slot == want, (n_kf, cur, t_opt, k)
            assert torch.equal(smp.targets["rgb"], st.rgb[slot])
            assert torch.equal(smp.targets["depth"], st.depth[slot])
            assert torch.equal(smp.targets["label"], st.label[slot])
            assert torch.equal(smp.pose[0], st.T[slot].float())
        assert int(smp.state[0].item()) == cnt + 2
        log = smp.picked[off:off + cnt].cpu().numpy()
        want = [oracle.rskm_select(k, t_opt, cur, list(range(n_kf)), draws[off + k]) for k in range(cnt)]
        np.testing.assert_array_equal(log, want)
    assert int(smp.picked[35].item()) == -1                # nothing logged past the last window
    with pytest.raises(L.GsError):
        smp.begin(0, 4, 2, 3, 2)                           # current slot beyond the keyframes + 1
        smp.draw()
    with pytest.raises(L.GsError):
        smp.begin(0, 4, 2, 1, 0)                           # t_opt = 0
        smp.draw()


def test_rskm_draws_replay_from_a_graph():
    st = _store(4, 64, 48, seed=82)
    draws = synth.rskm_draws(16, seed=83)
    smp = slam.RskmSampler(st, draws)
    smp.begin(0, 8, 3, 3, 2)
    for _ in range(8):
        smp.draw()
    eager = smp.picked[:8].clone()
    smp.picked.fill_(-1)
    smp.begin(0, 8, 3, 3, 2)
    cur = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        smp.draw()
    cur.wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(8):
            smp.draw()
    smp.picked.fill_(-1)
    smp.state.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(smp.picked[:8], eager)
    assert int(smp.state[0].item()) == 8


def _rot_deg(A, B):
    R = A[:3, :3] @ B[:3, :3].T
    return np.degrees(np.linalg.norm([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]]) / 2)


def _centre(T):
    return -T[:3, :3].T @ T[:3, 3]


def test_slam_loop_follows_the_oracle():
    """Four frames of a room sequence at 64x48: tracking 20 steps, expansion, 6 mapping
    iterations (10 for the first frame), t_opt 2, every other frame a keyframe."""
    n_frames, W, H, f = 4, 64, 48, 60.0
    P = W * H
    room = synth.make_room()
    path = synth.smooth_path(n_frames, step_deg=0.8, room=room)
    frames = [synth.raycast_room(room, synth.camera(W, H, f, T_cw=T)) for T in path]
    cam = synth.camera(W, H, f, T_cw=path[0])
    dec = synth.decoder(8, 16)
    prm_g, prm_o = C.params_pair()
    draws = synth.rskm_draws(64)
    bank = synth.feature_bank(n_frames * P, 16)
    kw = dict(n_track=20, n_map=6, n_init=10, t_opt=2, kf_every=2)
    ref = oracle.slam(frames, cam, prm_o, dec, path[0], draws, bank, oracle.SlamConfig(**kw))

    s = slam.Slam(cam, torch.as_tensor(dec.W).cuda(), torch.as_tensor(dec.b).cuda(), n_frames, draws,
                  torch.as_tensor(bank), slam.SlamConfig(**kw), params=prm_g)
    for t, fr in enumerate(frames):
        s.process(fr, T0=path[0] if t == 0 else None)
    torch.cuda.synchronize()

    assert s.picks() == ref["picks"]
    assert s.kf_frames == [0, 2]
    assert s.sizes[0] == ref["sizes"][0] == P
    print("sizes gpu", s.sizes, "oracle", ref["sizes"])
    for a, b in zip(s.sizes, ref["sizes"]):
        assert abs(a - b) <= 0.01 * P
    for t in range(1, n_frames):
        dr, dc = _rot_deg(s.est[t], ref["poses"][t]), np.linalg.norm(_centre(s.est[t]) - _centre(ref["poses"][t]))
        print(f"frame {t}: gpu vs oracle {dr:.4f} deg {dc * 1e3:.3f} mm; gpu vs truth "
              f"{_rot_deg(s.est[t], path[t]):.3f} deg {np.linalg.norm(_centre(s.est[t]) - _centre(path[t])) * 1e3:.2f} mm")
        assert dr < 0.05 and dc < 5e-3, t
    # the final maps render alike at the last true pose
    fg = s.field()
    gs_gpu = oracle.Field(*(getattr(fg, k).cpu().numpy().astype(np.float64) for k in oracle.ADAM_GROUPS))
    last = synth.camera(W, H, f, T_cw=path[-1], round_f32=False)
    img_g = oracle.forward(gs_gpu, last, prm_o)[2]
    img_o = oracle.forward(ref["gs"], last, prm_o)[2]
    rms = lambda a, b: float(np.sqrt(np.mean((a - b) ** 2)))
    print("map renders: rgb rms", rms(img_g["rgb"], img_o["rgb"]), "depth rms", rms(img_g["depth"], img_o["depth"]))
    assert rms(img_g["rgb"], img_o["rgb"]) < 0.01
    assert rms(img_g["depth"], img_o["depth"]) < 0.01
