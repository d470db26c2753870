"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

from oracle import gn, imu, maps
from oracle.so3 import State, boxminus, boxplus
from paper_2207_10940_gb300 import dri, synth
from parity import (POSE_M, POSE_RAD, REL, compare_linearisation, configs, new_stream, pose_error, to_dri,
                    to_oracle)

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair_setup(seq, levels, iters, **kw):
    """Library stream and oracle tracker after the initialising first frame, with
    the second frame uploaded."""
    _torch()
    ocfg, dcfg = configs(seq, levels, iters, **kw)
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    r = dri.dri_track(st.handle)
    assert r.status == 0 and r.initialised == 1
    dri.dri_upload_frame(st.handle, seq.frame_times[1], seq.depth[1], seq.intensity[1])
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(seq.imu)
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    return st, tr, ocfg, dcfg


def _oracle_system(tr, seq, ocfg, level, x0, x1):
    levels = maps.frame_levels(seq.depth[1], seq.intensity[1], ocfg)
    t0, t1 = seq.frame_times[0], seq.frame_times[1]
    W, _ = imu.weight(x0, tr.imu, t0, t1, ocfg)
    H, b, parts = tr.linearise_all(levels, level, x0, x1, t0, t1, W)
    d = boxminus(x0, tr.xbar)
    prior_cost = float(d @ tr.Hs @ d)
    return H, b, parts, prior_cost, levels


def _compare_linearisation(st, tr, seq, ocfg, level, x0, x1, rel=None):
    """dri_linearise at (x0, x1) against the oracle tracker `tr` (its state
    before the frame): per-pixel validity and association outside margins,
    counts, every system (parity.compare_linearisation) and the IMU term."""
    lvl_shape = (ocfg.height >> level, ocfg.width >> level)
    out, flags = dri.dri_linearise(st.handle, level, to_dri(x0), to_dri(x1), want_flags=True,
                                   shape=lvl_shape)
    H, b, parts, prior_cost, levels = _oracle_system(tr, seq, ocfg, level, x0, x1)
    lin = parts["lin"]
    np.testing.assert_allclose(out.e_imu, parts["e_imu"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(out.cost_imu, parts["cost_imu"], rtol=1e-8, atol=1e-9)
    cost = lin["cost_icp"] + lin["cost_rgb"] + parts["cost_imu"] + prior_cost
    compare_linearisation(out, flags, lin, H, b, cost, levels[level], tr.ref[level], x0, x1, ocfg,
                          rel=REL if rel is None else rel, what=f"level {level}")
    return out, lin


@pytest.mark.parametrize("cam,seed", [(synth.scaled_camera(100, 75), 3), (synth.CAM_320, 1)])
def test_linearisation_matches_oracle(cam, seed):
    seq = synth.frame_pair(seed=seed, cam=cam)
    st, tr, ocfg, dcfg = _pair_setup(seq, 2, (10, 5))
    rng = np.random.default_rng(seed)
    gt0, gt1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    cases = [(gt0, gt1),
             (boxplus(gt0, rng.normal(size=17) * 1e-3), boxplus(gt1, rng.normal(size=17) * 5e-3))]
    for x0, x1 in cases:
        for level in range(2):
            out, lin = _compare_linearisation(st, tr, seq, ocfg, level, x0, x1)
            assert lin["n_icp"] > 50 and lin["n_rgb"] > 50
    st.close()


def test_track_pair_matches_oracle():
    """The 320x240 frame pair, 2 levels, 10/5 iterations: final pose within
    1e-6 rad / 1e-6 m of the oracle, prior H* within the system tolerance."""
    seq = synth.frame_pair(seed=1)
    st, tr, ocfg, dcfg = _pair_setup(seq, 2, (10, 5))
    res = dri.dri_track(st.handle)
    ores = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    assert da < POSE_RAD and dr < POSE_M, (da, dr)
    x1 = to_oracle(res.x1)
    np.testing.assert_allclose(x1.v, ores["x1"].v, atol=1e-5)
    np.testing.assert_allclose(x1.bg, ores["x1"].bg, atol=1e-6)
    np.testing.assert_allclose(x1.ba, ores["x1"].ba, atol=1e-5)
    for l in range(2):
        n_icp, n_rgb = ores["counts"][l]
        assert abs(res.n_icp[l] - n_icp) <= max(3, 1e-3 * n_icp)
        assert abs(res.n_rgb[l] - n_rgb) <= max(3, 1e-3 * n_rgb)
    _, Hs, bs = dri.dri_get_state(st.handle, with_prior=True)
    # H* = H_11 - H_10 H_00^-1 H_01 (Eq. 8) is gated on the scale of the system it
    # is computed from, the x1 block of the last joint system: the Schur
    # complement removes the information x0 carried, so H*'s own diagonal can be
    # far below the scale at which the system's entries are rounded
    d1 = np.sqrt(np.diag(ores["H"])[17:])
    ds = np.sqrt(np.diag(ores["H_prior"]))
    err = np.abs(Hs - ores["H_prior"])
    r_sys = np.max(err / np.outer(d1, d1))
    r_own = np.max(err / np.outer(ds, ds))
    assert r_sys <= 1e-5, f"H*: err / system scale {r_sys:.3g}, err / own diagonal {r_own:.3g}"
    st.close()


def test_sequence_matches_oracle():
    """Five chained frames of a sinusoidal sequence (3 levels): prior, reference
    swap and IMU chaining agree with the oracle frame by frame."""
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=5)
    _torch()
    ocfg, dcfg = configs(seq, 3, (6, 4, 3))
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(seq.imu)
    for i in range(5):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        assert res.status == 0
        if i:
            da, dr = pose_error(res.x1, ores["x1"])
            assert da < 5 * POSE_RAD and dr < 5 * POSE_M, (i, da, dr)
    st.close()


def test_missing_imu_coverage_is_not_ready():
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    _torch()
    ocfg, dcfg = configs(seq, 2, (2, 2))
    st = new_stream(dcfg, synth.initial_state(seq))
    dri.dri_push_imu(st.handle, seq.imu[:3])      # ends before the second frame
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    assert dri.dri_track(st.handle).initialised == 1
    dri.dri_upload_frame(st.handle, seq.frame_times[1], seq.depth[1], seq.intensity[1])
    with pytest.raises(dri.DriError) as e:
        dri.dri_track(st.handle)
    assert e.value.code == dri.DRI_ENOTREADY
    dri.dri_push_imu(st.handle, seq.imu[3:])
    assert dri.dri_track(st.handle).status == 0
    st.close()


def test_no_valid_depth_reports_lost_and_keeps_state():
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    _torch()
    ocfg, dcfg = configs(seq, 2, (2, 2))
    st = new_stream(dcfg, synth.initial_state(seq))
    dri.dri_push_imu(st.handle, seq.imu)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    dri.dri_track(st.handle)
    before = dri.dri_get_state(st.handle)
    dri.dri_upload_frame(st.handle, seq.frame_times[1], np.zeros_like(seq.depth[1]), seq.intensity[1])
    res = dri.dri_track(st.handle)
    assert res.status == dri.DRI_ELOST
    after = dri.dri_get_state(st.handle)
    assert list(after.r_WC) == list(before.r_WC) and list(after.q_WC) == list(before.q_WC)
    st.close()


def test_invalid_arguments_are_rejected():
    _torch()
    cfg = dri.dri_config_default(64, 48)
    x = dri.dri_state()
    x.q_WC[0] = 1.0
    x.q_IW[0] = 1.0
    cfg.sigma_I = -1.0
    with pytest.raises(dri.DriError) as e:
        dri.dri_create_stream(cfg, x)
    assert e.value.code == dri.DRI_EINVAL
    cfg = dri.dri_config_default(64, 48)
    h = dri.dri_create_stream(cfg, x)
    bad = np.array([[0.0] + [0.0] * 6, [0.0] + [0.0] * 6])        # non-increasing times
    with pytest.raises(dri.DriError):
        dri.dri_push_imu(h, bad)
    with pytest.raises(dri.DriError):
        dri.dri_track(h)                                          # no frame uploaded
    dri.dri_destroy_stream(h)


def test_pipelined_frames_match_synchronous_tracking():
    """Frames queued back to back (device uploads, no waits, many frames in
    flight) give bit-identical states to tracking them one at a time."""
    torch = _torch()
    seq = synth.sinusoid_sequence(seed=5, cam=synth.scaled_camera(160, 120), n_frames=12)
    _, dcfg = configs(seq, 3, (4, 3, 2))
    x_init = synth.initial_state(seq)
    dev = torch.device("cuda")
    D = torch.stack([torch.from_numpy(d) for d in seq.depth]).to(dev)
    I = torch.stack([torch.from_numpy(i) for i in seq.intensity]).to(dev)
    torch.cuda.synchronize()
    states = []
    for pipelined in (False, True):
        st = new_stream(dcfg, x_init)
        dri.dri_push_imu(st.handle, seq.imu)
        for i in range(12):
            dri.dri_upload_frame(st.handle, seq.frame_times[i], D[i], I[i])
            r = dri.dri_track(st.handle, wait=not pipelined)
            if not pipelined:
                assert r.status == 0
        x, Hs, bs = dri.dri_get_state(st.handle, with_prior=True)
        ok, failed = dri.dri_frame_counts(st.handle)
        assert (ok, failed) == (12, 0)
        states.append((dri.state_to_dict(x), Hs, bs))
        st.close()
    (a, Ha, ba), (b, Hb, bb) = states
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(Ha, Hb)


def test_pinned_host_upload_matches_device_upload():
    """Pinned host frames (read by the GPU directly), pageable host frames (copied)
    and device frames give bit-identical tracking."""
    torch = _torch()
    seq = synth.sinusoid_sequence(seed=7, cam=synth.scaled_camera(160, 120), n_frames=4)
    _, dcfg = configs(seq, 3, (4, 3, 2))
    x_init = synth.initial_state(seq)
    kinds = {
        "device": [(torch.from_numpy(d).cuda(), torch.from_numpy(i).cuda()) for d, i in
                   zip(seq.depth, seq.intensity)],
        "pinned": [(torch.from_numpy(d).pin_memory(), torch.from_numpy(i).pin_memory()) for d, i in
                   zip(seq.depth, seq.intensity)],
        "pageable": list(zip(seq.depth, seq.intensity)),
    }
    torch.cuda.synchronize()
    out = {}
    for name, frames in kinds.items():
        st = new_stream(dcfg, x_init)
        dri.dri_push_imu(st.handle, seq.imu)
        for k, (d, i) in enumerate(frames):
            mk = dri.DRI_DEVICE if name == "device" else dri.DRI_HOST
            dri.dri_upload_frame(st.handle, seq.frame_times[k], d, i, mem_kind=mk)
            assert dri.dri_track(st.handle).status == 0
        out[name] = dri.state_to_dict(dri.dri_get_state(st.handle))
        h2d, _ = dri.dri_io_bytes(st.handle)
        if name != "device":
            assert h2d >= 2 * 4 * seq.cam.width * seq.cam.height
        st.close()
    for name in ("pinned", "pageable"):
        for key in out["device"]:
            np.testing.assert_array_equal(out[name][key], out["device"][key], err_msg=f"{name} {key}")
