"""Host logic of the surrogate pipeline (paper_2405_02914_gb300/surrogate.py)
on the CPU: the keyframe trajectory it reads poses from, the per-frame
loading scalars fed to the network, and the fallback rule whose served-rate
summary the benchmark reports.  Expected values are worked by hand from the
definitions in the docstrings."""
import numpy as np
import pytest

from paper_2405_02914_gb300 import inputs as I
from paper_2405_02914_gb300 import surrogate as G


def _kf():
    # press 0.4 mm in 100 substeps, slip 0.5 mm along +x in 200, turn 0.3 rad in 100
    return I.press_slip_rotate((1e-3, 2e-3, 5e-3), 0.4e-3, 0.5e-3, 0.3, 100, 200, 100)


@pytest.mark.parametrize("k,tip,yaw", [
    (-5, (1e-3, 2e-3, 5e-3), 0.0),              # before the first keyframe: the first pose
    (0, (1e-3, 2e-3, 5e-3), 0.0),
    (50, (1e-3, 2e-3, 4.8e-3), 0.0),            # half way down
    (100, (1e-3, 2e-3, 4.6e-3), 0.0),
    (200, (1.25e-3, 2e-3, 4.6e-3), 0.0),        # half way along the slip
    (300, (1.5e-3, 2e-3, 4.6e-3), 0.0),
    (350, (1.5e-3, 2e-3, 4.6e-3), 0.15),        # half way through the turn
    (400, (1.5e-3, 2e-3, 4.6e-3), 0.3),
    (10**6, (1.5e-3, 2e-3, 4.6e-3), 0.3),       # after the last keyframe: the last pose
])
def test_trajectory_state_is_piecewise_linear(k, tip, yaw):
    t, y = G.trajectory_state(_kf(), k)
    # keyframes are stored as float32 values (the kernels read float32 poses)
    np.testing.assert_allclose(t, tip, rtol=0, atol=1e-9)
    assert y == pytest.approx(yaw, abs=1e-7)


def test_frame_scalars_by_phase():
    sc = I.scene_small(cx=16, cy=16, cz=4, press=0.3e-3, slip=0.4e-3, rotate=0.2, n_press=100, n_slip=200,
                       n_rot=100, mu=1.0, E=2.4e5, nu=0.46)
    H, dx = sc.gel.height, sc.gel.dx
    descent = 0.3e-3 + 0.37 * dx                # the tip starts 0.37 cells above the gel
    mm_per_ks = 1e-3 * 1e-3                      # rates are in mm per 1000 substeps
    # mid-press: depth below the gel top, descent rate, no tangential motion
    s = G.frame_scalars(sc, 60)
    tip_z = H + 0.37 * dx - 0.6 * descent
    assert s[0] == pytest.approx(max(0.0, H - tip_z) / 1e-3, rel=1e-5)
    assert s[7] == pytest.approx(descent / 100 / mm_per_ks, rel=1e-5)
    assert s[1] == 0 and s[2] == 0 and s[3] == 0 and s[8] == 0
    # material constants centred on their ranges
    assert s[4] == pytest.approx((2.4e5 - 1.9e5) / 1e5, rel=1e-6)
    assert s[5] == pytest.approx((0.46 - 0.44) / 0.04, rel=1e-5)
    assert s[6] == pytest.approx((1.0 - 0.6) / 0.4, rel=1e-6)
    # mid-slip: full press depth, slip so far along +x, slip speed as the tangential rate
    s = G.frame_scalars(sc, 200)
    assert s[0] == pytest.approx(0.3, rel=1e-4)
    assert s[1] == pytest.approx(0.2, rel=1e-4) and abs(s[2]) < 1e-6 and s[3] == 0
    assert s[7] == pytest.approx(0.0, abs=1e-6)
    assert s[8] == pytest.approx(0.4e-3 / 200 / mm_per_ks, rel=1e-4)
    # mid-turn: the rotation so far, and its speed at 3 mm from the axis
    s = G.frame_scalars(sc, 350)
    assert s[1] == pytest.approx(0.4, rel=1e-4) and s[3] == pytest.approx(0.1, rel=1e-5)
    assert s[8] == pytest.approx(0.2 / 100 * 3e-3 / mm_per_ks, rel=1e-4)


def test_serve_summary_hand_worked():
    err = np.array([0.01, 0.03, 0.05, 0.015])
    ind = np.array([0.01, 0.05, 0.01, 0.03])
    s = G.serve_summary(err, ind, threshold=0.02)
    # frames 1 and 3 exceed the indicator threshold and go to the simulator
    assert s["n"] == 4 and s["fallback_frac"] == 0.5
    # served errors [0.01, 0, 0.05, 0]: three of four within 2 %
    assert s["served_within"] == 0.75 and s["max_served_err"] == 0.05
    # the network alone: 0.01 and 0.015 within 2 %
    assert s["surrogate_within"] == 0.5
    assert s["median_err"] == pytest.approx(0.0225) and s["p90_err"] == pytest.approx(0.044)


def test_served_time_charges_the_trajectory_prefix():
    """Hand-worked: 6 frames of two trajectories (frames at substeps 100, 200,
    300), network 100 frames/s, IMPM 10 frames/s.  Trajectory 0 falls back at
    its frames 1 and 2 (pays 2 IMPM frames: the run to frame 2 also gives
    frame 1), trajectory 1 at its frame 3 (pays 3): 6/100 + 2/10 + 3/10."""
    fb = np.array([True, True, False, False, False, True])
    traj = np.array([0, 0, 0, 1, 1, 1])
    sub = np.array([100, 200, 300, 100, 200, 300])
    t = G.served_seconds(fb, traj, sub, 100, 100.0, 10.0)
    assert t == pytest.approx(0.06 + 0.2 + 0.3)
    assert G.served_seconds(np.zeros(6, bool), traj, sub, 100, 100.0, 10.0) == pytest.approx(0.06)


def test_forward_flops_counts_real_channels():
    """Hand-worked for an 8 x 8 frame: pixels per layer 64, 16, 4, 1, 1, 4,
    16, 64, 64; real channels 12 -> 32 -> ... -> 32 -> 4; 2 x 9 FLOPs per
    multiply-add of a 3 x 3 tap.  Sum of pixels x cin x cout = 589,824 on the
    real channels and 622,592 with the 16-wide stored input and output."""
    assert G.forward_flops(8) == 18 * 589824
    assert G.forward_flops(8, stored=True) == 18 * 622592


def test_chunked_generation_resumes_and_keeps_trajectory_indices(tmp_path, monkeypatch):
    """generate_chunks writes one file per batch of trajectories, keeps the
    chunks already on disk (an interrupted run resumes), numbers the
    trajectories globally (also the ones left out after a latched error),
    and load_chunks returns the frames in order.  The IMPM of a batch is
    replaced here by a stub that encodes the trajectory in its frames."""
    import numpy as np
    from paper_2405_02914_gb300 import inputs as I
    from paper_2405_02914_gb300 import surrogate as G
    from paper_2405_02914_gb300 import tsim as T
    torch = pytest.importorskip("torch")
    scenes = I.surrogate_scenes(5, seed=0)
    every = scenes[0].n_substeps // 4
    px = scenes[0].readout_px
    calls = []

    def stub(chunk, every_, px_, pitch, x_ref):
        ids = [scenes.index(s) for s in chunk]
        calls.append(ids)
        if 3 in ids and len(ids) == 2:             # the first try of trajectory 3's batch latches an error
            raise T.TsimError(4, "non-finite state (instance %d)" % ids.index(3))
        nf = chunk[0].n_substeps // every_
        H = torch.stack([torch.full((nf, px_, px_), float(j)) for j in ids])
        U = torch.stack([torch.full((nf, px_, px_, 3), float(j) + 0.5) for j in ids])
        return H, U, 0.25 * len(ids), 1.0

    monkeypatch.setattr(G, "_run_chunk", stub)
    monkeypatch.setattr(G, "_torch", lambda: torch)     # host logic only: no device needed here
    paths = G.generate_chunks(scenes, str(tmp_path), every=every, batch=2, device="cpu")
    assert [p.split("/")[-1] for p in paths] == ["chunk_00000.npz", "chunk_00001.npz", "chunk_00002.npz"]
    assert calls == [[0, 1], [2, 3], [2], [4]]
    calls.clear()
    G.generate_chunks(scenes, str(tmp_path), every=every, batch=2, device="cpu")
    assert calls == []                                   # everything on disk is kept
    (tmp_path / "chunk_00002.npz").unlink()
    G.generate_chunks(scenes, str(tmp_path), every=every, batch=2, device="cpu")
    assert calls == [[4]]                                # only the missing chunk is simulated again
    fr = G.load_chunks(str(tmp_path), device="cpu")
    assert fr.dropped == [3]
    assert list(fr.traj) == [0] * 4 + [1] * 4 + [2] * 4 + [4] * 4
    assert np.array_equal(fr.height[:, 0, 0].numpy() * G.MM, fr.traj.astype(np.float32))
    assert fr.mpm_seconds == pytest.approx(0.25 * 4) and fr.mpm_frames == 16
    assert list(fr.substep[:4]) == [every, 2 * every, 3 * every, 4 * every]
