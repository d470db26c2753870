"""DRI_TRACK_GYRO_ONLY (the paper's gyroscope-only setup, the accelerometer-
related residuals ignored: Sec. VII, Fig. 5, Table VI) against the oracle's
track_mode 2: the joint system at given states, a tracked pair with its prior,
a chained sequence, the accelerometer readings' irrelevance, and a batch that
mixes the three tracking modes."""
import numpy as np
import pytest

from oracle import gn, imu, maps
from oracle.so3 import State, boxminus, boxplus
from paper_2207_10940_gb300 import dri, synth
from parity import (POSE_M, POSE_RAD, check_system, configs, margin_allowance, new_stream, pose_error, to_dri,
                    to_oracle)

pytestmark = pytest.mark.gpu

GYRO = dri.DRI_TRACK_GYRO_ONLY
HELD = np.r_[gn.HELD_GYRO_ONLY, 17 + gn.HELD_GYRO_ONLY]


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair_setup(seq, levels, iters, imu_samples=None):
    _torch()
    ocfg, dcfg = configs(seq, levels, iters, track_mode=GYRO)
    x_init = synth.initial_state(seq)
    samples = seq.imu if imu_samples is None else imu_samples
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, samples)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    assert dri.dri_track(st.handle).status == 0
    dri.dri_upload_frame(st.handle, seq.frame_times[1], seq.depth[1], seq.intensity[1])
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(samples)
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    return st, tr, ocfg


def test_joint_system_matches_oracle():
    seq = synth.frame_pair(seed=3, cam=synth.scaled_camera(100, 75))
    st, tr, ocfg = _pair_setup(seq, 2, (6, 4))
    rng = np.random.default_rng(5)
    gt0, gt1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    t0, t1 = seq.frame_times[0], seq.frame_times[1]
    levels = maps.frame_levels(seq.depth[1], seq.intensity[1], ocfg)
    for x0, x1 in [(gt0, gt1),
                   (boxplus(gt0, rng.normal(size=17) * 1e-3), boxplus(gt1, rng.normal(size=17) * 5e-3))]:
        _, S = imu.weight(x0, tr.imu, t0, t1, ocfg)
        Wg = imu.weight_gyro_only(S)
        for level in range(2):
            shape = (ocfg.height >> level, ocfg.width >> level)
            out, flags = dri.dri_linearise(st.handle, level, to_dri(x0), to_dri(x1), want_flags=True,
                                           shape=shape)
            H, b, parts = tr.linearise_all(levels, level, x0, x1, t0, t1, Wg)
            d = boxminus(x0, tr.xbar)
            lin = parts["lin"]
            cost = lin["cost_icp"] + lin["cost_rgb"] + parts["cost_imu"] + float(d @ tr.Hs @ d)
            Hg = np.array(out.H).reshape(34, 34)
            al = margin_allowance(lin, flags, levels[level], tr.ref[level], x0, x1, ocfg)
            check_system(Hg, out.b, H, b, cost, what=f"gyro-only joint, level {level}", allow=al["joint"])
            # held components: exactly the identity's rows, zero right-hand side
            assert np.array_equal(Hg[HELD], np.eye(34)[HELD])
            assert not np.asarray(out.b)[HELD].any()
            np.testing.assert_allclose(out.cost_imu, parts["cost_imu"], rtol=1e-8, atol=1e-9)
    st.close()


def test_track_pair_matches_oracle_with_prior():
    seq = synth.frame_pair(seed=1)
    st, tr, _ = _pair_setup(seq, 2, (10, 5))
    res = dri.dri_track(st.handle)
    ores = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    assert da < POSE_RAD and dr < POSE_M, (da, dr)
    x1, x_init = to_oracle(res.x1), State.from_dict(synth.initial_state(seq))
    np.testing.assert_allclose(x1.bg, ores["x1"].bg, atol=1e-6)
    assert np.array_equal(x1.v, x_init.v) and np.array_equal(x1.ba, x_init.ba)
    _, Hs, bs = dri.dri_get_state(st.handle, with_prior=True)
    held = gn.HELD_GYRO_ONLY
    assert not Hs[held].any() and not Hs[:, held].any() and not bs[held].any()
    d = np.sqrt(np.maximum(np.diag(ores["H_prior"]), 0.0))
    assert np.all(np.abs(Hs - ores["H_prior"]) <= 1e-4 * np.outer(d, d))
    st.close()


def test_sequence_matches_oracle():
    _torch()
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=6)
    ocfg, dcfg = configs(seq, 3, (6, 4, 3), track_mode=GYRO)
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(seq.imu)
    for i in range(6):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        assert res.status == 0
        if i:
            da, dr = pose_error(res.x1, ores["x1"])
            assert da < (i + 1) * POSE_RAD and dr < (i + 1) * POSE_M, (i, da, dr)
            np.testing.assert_allclose(list(res.x1.bg), ores["x1"].bg, atol=(i + 1) * 1e-6)
    st.close()


def test_accelerometer_readings_change_no_bit():
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(96, 72))
    bad = seq.imu.copy()
    bad[:, 4:7] = np.random.default_rng(9).normal(scale=5.0, size=(len(bad), 3))
    out = []
    for samples in (seq.imu, bad):
        st, _, _ = _pair_setup(seq, 2, (5, 3), imu_samples=samples)
        assert dri.dri_track(st.handle).status == 0
        out.append(dri.dri_get_state(st.handle, with_prior=True))
        st.close()
    (xa, Ha, ba), (xb, Hb, bb) = out
    for f in ("r_WC", "q_WC", "v_I", "bg", "ba", "q_IW"):
        assert list(getattr(xa, f)) == list(getattr(xb, f)), f
    assert np.array_equal(Ha, Hb) and np.array_equal(ba, bb)


def test_mixed_batch_equals_each_stream_alone():
    torch = _torch()
    seq = synth.sinusoid_sequence(seed=7, cam=synth.scaled_camera(96, 72), n_frames=3)
    cfgs = [configs(seq, 2, (4, 3), track_mode=m)[1]
            for m in (dri.DRI_TRACK_INERTIAL, GYRO, dri.DRI_TRACK_RGBD_ONLY)]
    x_init = synth.initial_state(seq)

    def run(cs, batched):
        ts = torch.cuda.Stream()
        sts = [dri.Stream(c, dri.state_from_dict(x_init, 0.0), ts) for c in cs]
        for st in sts:
            dri.dri_push_imu(st.handle, seq.imu)
        for i in range(3):
            for st in sts:
                dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
            if batched:
                dri.dri_track_batch(sts, wait=True)
            else:
                for st in sts:
                    dri.dri_track(st.handle)
        res = [dri.dri_get_state(st.handle, with_prior=True) for st in sts]
        for st in sts:
            st.close()
        return res

    alone = [run([c], False)[0] for c in cfgs]
    mixed = run(cfgs, True)
    # the batched pixel kernel sums in another order than the single-stream one
    for (xa, _, _), (xb, _, _) in zip(alone, mixed):
        da, dr = pose_error(xa, xb)
        assert da < POSE_RAD and dr < POSE_M, (da, dr)
    assert list(mixed[1][0].v_I) == list(alone[1][0].v_I) == list(x_init["v_I"])
    # the three modes really differ
    for i in range(3):
        for j in range(i):
            da, dr = pose_error(mixed[i][0], mixed[j][0])
            assert da + dr > 1e-6, (i, j)
