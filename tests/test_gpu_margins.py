"""Margin decisions of the pixel kernel in a tracked frame
(dri_track_result.n_margin, counted for streams with count_margins = 1): the
count of a level's last iteration, checked against a linearisation of the same
live frame and reference at the frame's converged state (dri_linearise's flag
bits and counts, which the parity helpers compare pixel by pixel with the
oracle's margins of the same decisions; the per-pixel tests of Sec. IV-B
evaluated in FP32)."""
import numpy as np
import pytest

from paper_2207_10940_gb300 import dri, synth
from parity import configs, new_stream

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _stream(seq, dcfg, rows):
    st = new_stream(dcfg, synth.initial_state(seq))
    dri.dri_batch_set_options([st.handle], rows_per_thread=rows)
    dri.dri_push_imu(st.handle, seq.imu)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    assert dri.dri_track(st.handle).initialised == 1
    dri.dri_upload_frame(st.handle, seq.frame_times[1], seq.depth[1], seq.intensity[1])
    return st


@pytest.mark.parametrize("dropout", [0.0, 0.01])
def test_tracked_margin_count_matches_a_linearisation_at_the_converged_state(dropout):
    """One level, 30 Gauss-Newton iterations: the last iteration linearises at
    the converged state (the last step is below what moves any FP32 transform),
    so a second stream holding the same reference and live frame, linearised
    at the tracked frame's final (x0, x1), decides every pixel as the last
    iteration did: the same valid counts and the same margin count."""
    _torch()
    seq = synth.frame_pair(seed=6, cam=synth.CAM_320, dropout=dropout)
    _, dcfg = configs(seq, 1, (30,))
    dcfg.count_margins = 1
    a = _stream(seq, dcfg, (8,))
    res = dri.dri_track(a.handle)
    assert res.status == 0
    b = _stream(seq, dcfg, (8,))
    out, flags = dri.dri_linearise(b.handle, 0, res.x0, res.x1, want_flags=True,
                                   shape=(seq.cam.height, seq.cam.width))
    n_flags = int(((flags & 64) != 0).sum() + ((flags & 128) != 0).sum())
    assert out.n_margin_icp + out.n_margin_rgb == n_flags
    assert abs(res.n_icp[0] - out.n_icp) <= 1 and abs(res.n_rgb[0] - out.n_rgb) <= 1, \
        (res.n_icp[0], out.n_icp, res.n_rgb[0], out.n_rgb)
    assert abs(res.n_margin[0] - n_flags) <= 2, (res.n_margin[0], n_flags)
    assert res.n_margin[0] > 0                       # 76,800 pixels: some decisions are marginal
    assert list(res.n_margin)[1:] == [0, 0, 0]       # levels the stream does not have
    a.close()
    b.close()


def test_every_level_reports_its_last_iteration():
    """Three levels, three frames: the initialising frame counts nothing,
    tracked frames count on their levels and never on the unused fourth one;
    a stream without count_margins reports zeros and tracks exactly as the
    counting one (the same valid counts on every level)."""
    _torch()
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=3)
    counts = {}
    for on in (1, 0):
        _, dcfg = configs(seq, 3, (6, 4, 3))
        dcfg.count_margins = on
        st = new_stream(dcfg, synth.initial_state(seq))
        dri.dri_push_imu(st.handle, seq.imu)
        counts[on] = []
        for i in range(3):
            dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
            r = dri.dri_track(st.handle)
            assert r.status == 0
            counts[on].append((list(r.n_margin), list(r.n_icp), list(r.n_rgb)))
        st.close()
    assert counts[1][0][0] == [0, 0, 0, 0]           # the initialising frame tracks nothing
    for c, _, _ in counts[1][1:]:
        assert c[3] == 0 and all(v >= 0 for v in c)
    assert sum(counts[1][1][0][:3]) + sum(counts[1][2][0][:3]) > 0
    # not asked for: zeros, and the tracking itself unchanged
    for (m0, i0, r0), (_, i1, r1) in zip(counts[0], counts[1]):
        assert m0 == [0, 0, 0, 0] and i0 == i1 and r0 == r1
