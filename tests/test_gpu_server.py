"""Serving loop (dri_server_*): results in the mix equal results alone, admission
by HBM budget, IMU coverage errors per request, concurrent clients."""
import threading

import numpy as np
import pytest

from paper_2207_10940_gb300 import dri, synth
from parity import POSE_M, POSE_RAD, configs, pose_error

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


SIZES = [(160, 120), (200, 150), (96, 72)]
N_FRAMES = 4


def _sequences():
    return [synth.sinusoid_sequence(seed=40 + i, cam=synth.scaled_camera(w, h), n_frames=N_FRAMES)
            for i, (w, h) in enumerate(SIZES)]


def _cfg(seq):
    return configs(seq, 3, (4, 3, 2))[1]


def _x0(seq):
    x = synth.initial_state(seq)
    return dri.state_from_dict(x, x.get("t", 0.0))


def _imu_between(seq, t_lo, t_hi):
    """Samples with t_lo < t <= t_hi (all up to t_hi when t_lo is None)."""
    ts = np.array([m[0] for m in seq.imu])
    keep = (ts <= t_hi) if t_lo is None else ((ts > t_lo) & (ts <= t_hi))
    return [seq.imu[k] for k in np.nonzero(keep)[0]]


def _imu_for_frame(seq, i):
    # everything up to the first sample at or after the frame (the covering sample)
    ts = np.array([m[0] for m in seq.imu])
    hi = ts[np.searchsorted(ts, seq.frame_times[i])]
    lo = None if i == 0 else ts[np.searchsorted(ts, seq.frame_times[i - 1])]
    return _imu_between(seq, lo, hi)


def test_results_in_the_mix_equal_results_alone():
    torch = _torch()
    seqs = _sequences()
    alone = []
    for seq in seqs:
        st = dri.Stream(_cfg(seq), _x0(seq), torch.cuda.Stream())
        for i in range(N_FRAMES):
            dri.dri_push_imu(st.handle, _imu_for_frame(seq, i))
            dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
            assert dri.dri_track(st.handle).status == 0
        alone.append(dri.dri_get_state(st.handle, with_prior=True))
        st.close()

    srv = dri.dri_server_create(8 << 30, 8, torch.cuda.Stream())
    handles = [dri.dri_server_open_stream(srv, _cfg(seq), _x0(seq)) for seq in seqs]
    tickets = {k: [] for k in range(len(seqs))}

    def client(ks):                    # two client threads submit interleaved frames
        for i in range(N_FRAMES):
            for k in ks:
                seq = seqs[k]
                tickets[k].append(dri.dri_server_submit(srv, handles[k], seq.frame_times[i], seq.depth[i],
                                                        seq.intensity[i], _imu_for_frame(seq, i)))
    threads = [threading.Thread(target=client, args=(ks,)) for ks in ((0, 1), (2,))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for k in range(len(seqs)):
        for i, tk in enumerate(tickets[k]):
            status, res = dri.dri_server_poll(srv, tk, timeout_ms=60000)
            assert status == 0, (k, i, status)
            assert res.initialised == int(i == 0)
    stats = dri.dri_server_stats_read(srv)
    assert stats.completed == len(seqs) * N_FRAMES and stats.failed == 0
    assert stats.ticks >= N_FRAMES and stats.p99_ms >= stats.p50_ms > 0
    for h, (xa, Ha, _) in zip(handles, alone):
        xb, Hb, _ = dri.dri_get_state(h, with_prior=True)
        da, dr = pose_error(xa, xb)
        assert da < POSE_RAD and dr < POSE_M, (da, dr)
        d = np.sqrt(np.diag(Ha))
        assert np.all(np.abs(Hb - Ha) <= 1e-5 * np.outer(d, d))
    dri.dri_server_destroy(srv)


def test_admission_by_hbm_budget():
    torch = _torch()
    seq = _sequences()[0]
    cfg = _cfg(seq)
    one = dri.dri_stream_workspace_bytes(cfg) + 65536
    srv = dri.dri_server_create(one + one // 2, 4, torch.cuda.Stream())
    a = dri.dri_server_open_stream(srv, cfg, _x0(seq))
    with pytest.raises(dri.DriError) as e:
        dri.dri_server_open_stream(srv, cfg, _x0(seq))
    assert e.value.code == dri.DRI_EADMIT
    assert dri.dri_server_stats_read(srv).hbm_used == one
    other = _cfg(seq)
    other.levels = 2
    dri.dri_server_close_stream(srv, a)
    assert dri.dri_server_stats_read(srv).hbm_used == 0
    b = dri.dri_server_open_stream(srv, cfg, _x0(seq))
    with pytest.raises(dri.DriError) as e:                  # other level count than the server's
        dri.dri_server_open_stream(srv, other, _x0(seq))
    assert e.value.code == dri.DRI_EINVAL
    dri.dri_server_close_stream(srv, b)
    dri.dri_server_destroy(srv)


def test_request_without_imu_coverage_fails_alone():
    torch = _torch()
    seqs = _sequences()[:2]
    srv = dri.dri_server_create(8 << 30, 8, torch.cuda.Stream())
    hs = [dri.dri_server_open_stream(srv, _cfg(s), _x0(s)) for s in seqs]
    for h, s in zip(hs, seqs):
        tk = dri.dri_server_submit(srv, h, s.frame_times[0], s.depth[0], s.intensity[0], _imu_for_frame(s, 0))
        assert dri.dri_server_poll(srv, tk)[0] == 0
    s0, s1 = seqs
    short = dri.dri_server_submit(srv, hs[0], s0.frame_times[1], s0.depth[1], s0.intensity[1])   # no IMU
    good = dri.dri_server_submit(srv, hs[1], s1.frame_times[1], s1.depth[1], s1.intensity[1],
                                 _imu_for_frame(s1, 1))
    assert dri.dri_server_poll(srv, short)[0] == dri.DRI_ENOTREADY
    assert dri.dri_server_poll(srv, good)[0] == 0
    again = dri.dri_server_submit(srv, hs[0], s0.frame_times[1], s0.depth[1], s0.intensity[1],
                                  _imu_for_frame(s0, 1))
    status, res = dri.dri_server_poll(srv, again)
    assert status == 0 and res.initialised == 0
    with pytest.raises(dri.DriError):                        # a polled ticket is released
        dri.dri_server_poll(srv, again, timeout_ms=0)
    dri.dri_server_destroy(srv)
