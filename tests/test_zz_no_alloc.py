"""The allocation-free pair linearisation gives the same systems as dri_linearise.

dri_linearise_pair_noalloc serves callers that may not allocate device memory
when they call the library (it works from the caller's device images and keeps
its intermediates in a static device array).  Here it is called through the C
ABI twice in a row, on the same image pair at two different states, and each
result is compared with dri_linearise on a one-level stream built from the same
images, within the parity tolerance of the other GPU tests.  This file is
collected last so that a run stopping at its first failure has run the rest.
"""
import ctypes

import numpy as np
import pytest

from oracle.so3 import State, boxplus
from paper_2207_10940_gb300 import dri, synth
from parity import check_system, configs, new_stream, to_dri

pytestmark = pytest.mark.gpu


def test_noalloc_pair_linearisation_matches_stream_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seq = synth.frame_pair(seed=1)                          # 320 x 240, the size limit
    _, dcfg = configs(seq, 1, (3,))
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    assert dri.dri_track(st.handle).initialised == 1
    dri.dri_upload_frame(st.handle, seq.frame_times[1], seq.depth[1], seq.intensity[1])

    dev = torch.device("cuda")
    ref_d = torch.from_numpy(seq.depth[0]).to(dev)
    ref_i = torch.from_numpy(seq.intensity[0]).to(dev)
    live_d = torch.from_numpy(seq.depth[1]).to(dev)
    live_i = torch.from_numpy(seq.intensity[1]).to(dev)
    out_dev = torch.zeros(ctypes.sizeof(dri.dri_linearisation), dtype=torch.uint8, device=dev)
    flags_dev = torch.zeros(seq.cam.height * seq.cam.width, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    x_ref = to_dri(State.from_dict(x_init))

    rng = np.random.default_rng(0)
    gt0, gt1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    cases = [(gt0, gt1),
             (boxplus(gt0, rng.normal(size=17) * 1e-3), boxplus(gt1, rng.normal(size=17) * 5e-3))]
    for x0, x1 in cases:                                    # two calls in a row
        want, want_flags = dri.dri_linearise(st.handle, 0, to_dri(x0), to_dri(x1), want_flags=True,
                                             shape=(seq.cam.height, seq.cam.width))
        stream = torch.cuda.current_stream()
        dri.dri_linearise_pair_noalloc(dcfg, ref_d, ref_i, live_d, live_i, x_ref, to_dri(x0),
                                       to_dri(x1), out_dev, flags_dev, stream)
        stream.synchronize()
        got = dri.dri_linearisation.from_buffer_copy(out_dev.cpu().numpy().tobytes())
        got_flags = flags_dev.cpu().numpy().reshape(seq.cam.height, seq.cam.width)
        assert got.n_icp == want.n_icp and got.n_rgb == want.n_rgb
        assert got.n_icp > 1000 and got.n_rgb > 10000
        np.testing.assert_array_equal(got_flags, want_flags)
        check_system(np.array(got.H_icp).reshape(6, 6), got.b_icp,
                     np.array(want.H_icp).reshape(6, 6), want.b_icp, want.cost_icp, what="ICP")
        check_system(np.array(got.H_rgb).reshape(6, 6), got.b_rgb,
                     np.array(want.H_rgb).reshape(6, 6), want.b_rgb, want.cost_rgb, what="RGB")
        np.testing.assert_allclose(got.cost_icp, want.cost_icp, rtol=1e-9)
        np.testing.assert_allclose(got.cost_rgb, want.cost_rgb, rtol=1e-9)
    st.close()


def test_noalloc_rejects_images_beyond_its_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = dri.dri_config_default(640, 480)
    big = torch.zeros(640 * 480, dtype=torch.float32, device="cuda")
    out = torch.zeros(ctypes.sizeof(dri.dri_linearisation), dtype=torch.uint8, device="cuda")
    x = dri.dri_state()
    x.q_WC[0] = 1.0
    x.q_IW[0] = 1.0
    with pytest.raises(dri.DriError) as e:
        dri.dri_linearise_pair_noalloc(cfg, big, big, big, big, x, x, x, out)
    assert e.value.code == dri.DRI_EINVAL
