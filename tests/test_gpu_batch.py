"""Batched tracking (dri_track_batch) against the same streams tracked alone and
against the FP64 oracle.

Streams of uneven sizes share one launch per step; each stream's result must be
what it gets alone (dri_track), within the parity tolerance: the batch plan
chooses its own rows per thread, so the per-block summation order, and with it
the last bits, may differ.
"""
import numpy as np
import pytest

from oracle import gn
from paper_2207_10940_gb300 import dri, synth
from parity import POSE_M, POSE_RAD, configs, new_stream, pose_error

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


SIZES = [(160, 120), (200, 150), (96, 72), (320, 240)]   # 200 x 150 and 96 x 72: ragged tiles


def _sequences(n_frames):
    return [synth.sinusoid_sequence(seed=30 + i, cam=synth.scaled_camera(w, h), n_frames=n_frames)
            for i, (w, h) in enumerate(SIZES)]


def _streams(seqs, torch_stream):
    out = []
    for seq in seqs:
        _, dcfg = configs(seq, 3, (4, 3, 2))
        x_init = synth.initial_state(seq)
        st = dri.Stream(dcfg, dri.state_from_dict(x_init, x_init.get("t", 0.0)), torch_stream)
        dri.dri_push_imu(st.handle, seq.imu)
        out.append(st)
    return out


def test_batch_matches_streams_tracked_alone():
    torch = _torch()
    n_frames = 4
    seqs = _sequences(n_frames)
    alone = []
    for seq in seqs:
        st = _streams([seq], torch.cuda.Stream())[0]
        for i in range(n_frames):
            dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
            assert dri.dri_track(st.handle).status == 0
        alone.append(dri.dri_get_state(st.handle, with_prior=True))
        st.close()
    ts = torch.cuda.Stream()
    batch = _streams(seqs, ts)
    for i in range(n_frames):
        for st, seq in zip(batch, seqs):
            dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track_batch(batch)
        assert [r.status for r in res] == [0] * len(batch)
        assert [r.initialised for r in res] == [int(i == 0)] * len(batch)
    opts = dri.dri_batch_get_options(batch)
    assert all(p in (2, 4, 8, 16, 32) for p in opts.rows_per_thread[:3])
    assert opts.groups == 1 and opts.autotune == 0
    for st, (xa, Ha, ba) in zip(batch, alone):
        xb, Hb, bb = dri.dri_get_state(st.handle, with_prior=True)
        da, dr = pose_error(xa, xb)
        assert da < POSE_RAD and dr < POSE_M, (da, dr)
        d = np.sqrt(np.diag(Ha))
        assert np.all(np.abs(Hb - Ha) <= 1e-5 * np.outer(d, d))
        assert xb.t == xa.t
    ok = [dri.dri_frame_counts(st.handle) for st in batch]
    assert ok == [(n_frames, 0)] * len(batch)
    for st in batch:
        st.close()


def test_batch_pair_matches_oracle():
    """The 320 x 240 frame pair tracked as one slot of a batch with two other
    streams: final pose within 1e-6 rad / 1e-6 m of the oracle."""
    torch = _torch()
    pair = synth.frame_pair(seed=1)
    ocfg, dcfg = configs(pair, 2, (10, 5))
    x_init = synth.initial_state(pair)
    ts = torch.cuda.Stream()
    others = []
    for k, (w, h) in enumerate([(160, 120), (96, 72)]):
        seq = synth.frame_pair(seed=7 + k, cam=synth.scaled_camera(w, h))
        _, c = configs(seq, 2, (10, 5))
        xi = synth.initial_state(seq)
        st = dri.Stream(c, dri.state_from_dict(xi, xi.get("t", 0.0)), ts)
        dri.dri_push_imu(st.handle, seq.imu)
        others.append((st, seq))
    st = dri.Stream(dcfg, dri.state_from_dict(x_init, x_init.get("t", 0.0)), ts)
    dri.dri_push_imu(st.handle, pair.imu)
    streams = [others[0][0], st, others[1][0]]
    seqs = [others[0][1], pair, others[1][1]]
    for i in range(2):
        for s, q in zip(streams, seqs):
            dri.dri_upload_frame(s.handle, q.frame_times[i], q.depth[i], q.intensity[i])
        res = dri.dri_track_batch(streams)
        assert [r.status for r in res] == [0, 0, 0]
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(pair.imu)
    tr.track(pair.depth[0], pair.intensity[0], pair.frame_times[0])
    ores = tr.track(pair.depth[1], pair.intensity[1], pair.frame_times[1])
    da, dr = pose_error(res[1].x1, ores["x1"])
    assert da < POSE_RAD and dr < POSE_M, (da, dr)
    for s in streams:
        s.close()


def test_idle_slot_sits_out_and_keeps_its_frame():
    torch = _torch()
    seqs = _sequences(3)[:3]
    ts = torch.cuda.Stream()
    batch = _streams(seqs, ts)
    for i in range(2):
        for st, seq in zip(batch, seqs):
            dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        assert [r.status for r in dri.dri_track_batch(batch)] == [0, 0, 0]
    before = dri.dri_get_state(batch[1].handle)
    for k in (0, 2):                                   # stream 1 has no new frame
        dri.dri_upload_frame(batch[k].handle, seqs[k].frame_times[2], seqs[k].depth[2],
                             seqs[k].intensity[2])
    res = dri.dri_track_batch(batch)
    assert [r.status for r in res] == [0, dri.DRI_ENOTREADY, 0]
    after = dri.dri_get_state(batch[1].handle)
    assert list(after.r_WC) == list(before.r_WC) and after.t == before.t
    with pytest.raises(dri.DriError) as e:              # nobody has work
        dri.dri_track_batch(batch)
    assert e.value.code == dri.DRI_ENOTREADY
    dri.dri_upload_frame(batch[1].handle, seqs[1].frame_times[2], seqs[1].depth[2],
                         seqs[1].intensity[2])
    res = dri.dri_track_batch(batch)
    assert [r.status for r in res] == [dri.DRI_ENOTREADY, 0, dri.DRI_ENOTREADY]
    for st in batch:
        st.close()


def test_batch_rejects_mismatched_streams():
    torch = _torch()
    seqs = _sequences(2)[:2]
    ts = torch.cuda.Stream()
    a, b = _streams(seqs, ts)
    with pytest.raises(dri.DriError) as e:
        dri.dri_track_batch([a, a])
    assert e.value.code == dri.DRI_EINVAL
    _, c2 = configs(seqs[1], 2, (4, 3))
    x_init = synth.initial_state(seqs[1])
    c = dri.Stream(c2, dri.state_from_dict(x_init, 0.0), ts)
    with pytest.raises(dri.DriError) as e:
        dri.dri_track_batch([a, c])                    # other level count
    assert e.value.code == dri.DRI_EINVAL
    d = _streams([seqs[1]], torch.cuda.Stream())[0]
    with pytest.raises(dri.DriError) as e:
        dri.dri_track_batch([a, d])                    # other CUDA stream
    assert e.value.code == dri.DRI_EINVAL
    for s in (a, b, c, d):
        s.close()


def test_fixed_tiles_give_identical_bits_for_any_group_count():
    """With the rows per thread fixed, the result does not depend on how many
    slot groups (CUDA streams) run the Gauss-Newton loop: every slot sums the
    same pixels in the same order, so the states are bit-identical."""
    torch = _torch()
    seqs = _sequences(3)
    results = []
    for groups in (1, 2, 3):
        batch = _streams(seqs, torch.cuda.Stream())
        dri.dri_batch_set_options(batch, rows_per_thread=[2, 2, 1], groups=groups)
        opts = dri.dri_batch_get_options(batch)
        assert opts.groups == groups and opts.autotune == 0
        assert list(opts.rows_per_thread) == [2, 2, 1, 0]
        for i in range(3):
            for st, seq in zip(batch, seqs):
                dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
            assert [r.status for r in dri.dri_track_batch(batch)] == [0] * len(batch)
        results.append([dri.dri_get_state(st.handle, with_prior=True) for st in batch])
        for st in batch:
            st.close()
    for other in results[1:]:
        for (xa, Ha, ba), (xb, Hb, bb) in zip(results[0], other):
            a, b = dri.state_to_dict(xa), dri.state_to_dict(xb)
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
            np.testing.assert_array_equal(Ha, Hb)
            np.testing.assert_array_equal(ba, bb)


def test_batch_options_are_checked():
    torch = _torch()
    seqs = _sequences(2)[:2]
    batch = _streams(seqs, torch.cuda.Stream())
    for kw in ({"groups": -1}, {"groups": 3}, {"rows_per_thread": [0, 1, 1]},
               {"rows_per_thread": [65, 1, 1]}):
        with pytest.raises(dri.DriError) as e:
            dri.dri_batch_set_options(batch, **kw)
        assert e.value.code == dri.DRI_EINVAL
    # groups 0 keeps the plan's groups
    dri.dri_batch_set_options(batch, rows_per_thread=[4, 4, 2], groups=2)
    dri.dri_batch_set_options(batch, rows_per_thread=[8, 4, 2], groups=0)
    opts = dri.dri_batch_get_options(batch)
    assert opts.groups == 2 and list(opts.rows_per_thread[:3]) == [8, 4, 2]
    own = dri.dri_batch_get_options([batch[0]])        # a stream's own plan
    assert own.groups == 1 and own.autotune == 0
    for st in batch:
        st.close()


def test_default_slot_groups():
    """A new batch plan runs its Gauss-Newton loop as one slot group per 16
    slots (at most 4); results match the one-group plan."""
    torch = _torch()
    seq = synth.frame_pair(seed=5, cam=synth.scaled_camera(64, 48))
    _, dcfg = configs(seq, 2, (3, 2))
    x_init = synth.initial_state(seq)
    for n, groups in ((16, 1), (32, 2)):
        states = []
        for forced in (None, 1):
            ts = torch.cuda.Stream()
            batch = [dri.Stream(dcfg, dri.state_from_dict(x_init, 0.0), ts) for _ in range(n)]
            for st in batch:
                dri.dri_push_imu(st.handle, seq.imu)
            if forced is not None:
                dri.dri_batch_set_options(batch, rows_per_thread=[4, 2], groups=forced)
            else:
                dri.dri_batch_set_options(batch, rows_per_thread=[4, 2])
            for i in range(2):
                for st in batch:
                    dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
                res = dri.dri_track_batch(batch)
                assert [r.status for r in res] == [0] * n
            assert dri.dri_batch_get_options(batch).groups == (groups if forced is None else 1)
            states.append([dri.dri_get_state(st.handle) for st in batch])
            for st in batch:
                st.close()
        # the same fixed tiles: every slot sums its pixels in the same order
        for a, b in zip(*states):
            for f in ("r_WC", "q_WC", "v_I", "bg", "ba", "q_IW"):
                assert list(getattr(a, f)) == list(getattr(b, f)), f
