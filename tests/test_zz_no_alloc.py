"""The allocation-free pair linearisation gives the same systems as dri_linearise.

dri_linearise_pair_noalloc serves callers that may not allocate device memory
when they call the library (it works from the caller's device images and keeps
its intermediates in a static device array).  Here it is called through the C
ABI twice in a row, on the same image pair at two different states, and each
result is compared with dri_linearise on a one-level stream built from the same
images, within the parity tolerance of the other GPU tests (validity bit-exact
outside the oracle's margin pixels, systems within the normalised bar), with
the default options, with the occlusion test and depth-dependent ICP weight,
and with FP16 maps and FP32 partials.  This file is
collected last so that a run stopping at its first failure has run the rest.
"""
import ctypes

import numpy as np
import pytest

from oracle import gn, maps
from oracle.photogeo import linearise
from oracle.so3 import State, boxplus
from paper_2207_10940_gb300 import dri, synth
from parity import REL, REL_FP16, check_system, configs, new_stream, to_dri

pytestmark = pytest.mark.gpu


OPTION_CASES = [
    {},
    {"occlusion_thr": 0.05, "icp_depth_weight": 1},
    {"precision_flags": 3},                 # FP16 maps and FP32 partials
]


@pytest.mark.parametrize("opts", OPTION_CASES, ids=["default", "occlusion+depth-weight", "fp16+fp32-partials"])
def test_noalloc_pair_linearisation_matches_stream_entry_point(opts):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seq = synth.frame_pair(seed=1)                          # 320 x 240, the size limit
    ocfg, dcfg = configs(seq, 1, (3,), **opts)
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    assert dri.dri_track(st.handle).initialised == 1
    dri.dri_upload_frame(st.handle, seq.frame_times[1], seq.depth[1], seq.intensity[1])
    # the oracle's margin pixels: the two entries run different instantiations of
    # the per-pixel code, which may decide a pixel within a margin differently
    tr = gn.Tracker(ocfg, x_init)
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    lv = maps.frame_levels(seq.depth[1], seq.intensity[1], ocfg)

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
        lin = linearise(lv[0], tr.ref[0], tr.T_ref[0], tr.T_ref[1], x0, x1, ocfg)
        margin = lin["icp_margin"] | lin["rgb_margin"]
        np.testing.assert_array_equal(got_flags[~margin], want_flags[~margin])
        differ = (got_flags != want_flags) & margin
        assert abs(got.n_icp - want.n_icp) <= differ.sum() and abs(got.n_rgb - want.n_rgb) <= differ.sum()
        assert got.n_icp == ((got_flags & 1) != 0).sum() and got.n_rgb == ((got_flags & 2) != 0).sum()
        assert got.n_icp > 1000 and got.n_rgb > 10000
        rel = REL_FP16 if opts.get("precision_flags", 0) & dri.DRI_FP16_MAPS else REL
        check_system(np.array(got.H_icp).reshape(6, 6), got.b_icp,
                     np.array(want.H_icp).reshape(6, 6), want.b_icp, want.cost_icp, rel=rel, what="ICP")
        check_system(np.array(got.H_rgb).reshape(6, 6), got.b_rgb,
                     np.array(want.H_rgb).reshape(6, 6), want.b_rgb, want.cost_rgb, rel=rel, what="RGB")
        # e^2 sums: FP32 per thread over different tiles, folded in FP64
        np.testing.assert_allclose(got.cost_icp, want.cost_icp, rtol=rel)
        np.testing.assert_allclose(got.cost_rgb, want.cost_rgb, rtol=rel)
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
