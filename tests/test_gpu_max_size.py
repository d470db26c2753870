"""The largest image the C ABI accepts, 8192 x 8192 (67 M pixels per level-0
image): indexing, pyramid, maps and the pixel kernel at that size.

A frame pair rendered at 1024 x 1024 and enlarged 8x by pixel replication has,
at pyramid level 3, exactly the 1024 x 1024 images (every 2 x 2 mean is of
equal values, Sec. IV-D's pyramid), and with fx = 8 f, cx = 8 (c + 0.5) - 0.5
level 3's intrinsics are exactly those of the 1024 x 1024 camera.  So level 3
of the 8192 x 8192 stream is linearised like level 0 of a 1024 x 1024 stream:
identical per-pixel flags and counts, and systems within the parity bar (they
differ only in the order of the FP32 sums).  At level 0 the per-pixel
decisions do not depend on the tiling: two rows-per-thread settings give
identical flags and counts.  Then the frame is tracked on all four levels."""
import numpy as np
import pytest

from paper_2207_10940_gb300 import dri, synth
from parity import check_system, configs, new_stream, to_dri

pytestmark = pytest.mark.gpu

N = 8192
K = 8                                   # replication factor: level 3 of N is N / K


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _open(dcfg, seq, big):
    up = (lambda a: np.ascontiguousarray(np.repeat(np.repeat(a, K, axis=0), K, axis=1))) if big \
        else (lambda a: a)
    st = new_stream(dcfg, synth.initial_state(seq))
    dri.dri_push_imu(st.handle, seq.imu)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], up(seq.depth[0]), up(seq.intensity[0]))
    assert dri.dri_track(st.handle).initialised == 1
    dri.dri_upload_frame(st.handle, seq.frame_times[1], up(seq.depth[1]), up(seq.intensity[1]))
    return st


def test_maximum_image_size():
    _torch()
    small = synth.scaled_camera(N // K, N // K)
    seq = synth.frame_pair(seed=3, cam=small)
    _, dcfg_s = configs(seq, 1, (1,))
    _, dcfg_b = configs(seq, 4, (2, 2, 2, 2))
    dcfg_b.width = dcfg_b.height = N
    dcfg_b.fx, dcfg_b.fy = K * small.fx, K * small.fy
    dcfg_b.cx, dcfg_b.cy = K * (small.cx + 0.5) - 0.5, K * (small.cy + 0.5) - 0.5
    st_s = _open(dcfg_s, seq, False)
    st_b = _open(dcfg_b, seq, True)
    x0, x1 = to_dri(seq.gt[0]), to_dri(seq.gt[1])

    out_s, f_s = dri.dri_linearise(st_s.handle, 0, x0, x1, want_flags=True, shape=(N // K, N // K))
    out_b, f_b = dri.dri_linearise(st_b.handle, 3, x0, x1, want_flags=True, shape=(N // K, N // K))
    assert np.array_equal(f_s, f_b)
    assert (out_s.n_icp, out_s.n_rgb, out_s.n_margin_icp, out_s.n_margin_rgb) == \
        (out_b.n_icp, out_b.n_rgb, out_b.n_margin_icp, out_b.n_margin_rgb)
    assert out_s.n_icp > 10000 and out_s.n_rgb > 100000
    for H, b, Hr, br, cost, what in (
            (out_b.H_icp, out_b.b_icp, out_s.H_icp, out_s.b_icp, out_s.cost_icp, "ICP"),
            (out_b.H_rgb, out_b.b_rgb, out_s.H_rgb, out_s.b_rgb, out_s.cost_rgb, "RGB")):
        check_system(np.array(H).reshape(6, 6), b, np.array(Hr).reshape(6, 6), br, cost, what=what)
    st_s.close()

    # level 0, 67 M pixels: two tilings decide every pixel alike
    res = []
    for rows in ((8, 8, 8, 8), (32, 32, 8, 8)):
        dri.dri_batch_set_options([st_b.handle], rows_per_thread=rows)
        res.append(dri.dri_linearise(st_b.handle, 0, x0, x1, want_flags=True, shape=(N, N)))
    (o1, g1), (o2, g2) = res
    assert np.array_equal(g1, g2)
    assert (o1.n_icp, o1.n_rgb) == (o2.n_icp, o2.n_rgb)
    assert o1.n_icp > 10 ** 6 and o1.n_rgb > 10 ** 7
    check_system(np.array(o1.H_icp).reshape(6, 6), o1.b_icp, np.array(o2.H_icp).reshape(6, 6), o2.b_icp,
                 o2.cost_icp, what="ICP level 0")
    check_system(np.array(o1.H_rgb).reshape(6, 6), o1.b_rgb, np.array(o2.H_rgb).reshape(6, 6), o2.b_rgb,
                 o2.cost_rgb, what="RGB level 0")
    del res, g1, g2

    r = dri.dri_track(st_b.handle)
    assert r.status == 0 and min(r.n_icp[l] for l in range(4)) > 0
    st_b.close()
