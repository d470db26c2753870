"""Checkpoint and resume through dri_get_state / dri_set_state.

A stream is checkpointed after a tracked frame (its state x and the prior H*,
b* that the next frame uses, Eq. 8-9) and destroyed.  A new stream created at
the checkpointed state initialises on that same frame (which becomes its
reference at the checkpointed pose, as it was for the old stream), takes the
prior back with dri_set_state and tracks the following frames: its states and
priors equal those of a stream that was never interrupted."""
import numpy as np
import pytest

from paper_2207_10940_gb300 import dri, synth
from parity import configs, new_stream

pytestmark = pytest.mark.gpu


def _track(st, seq, frames):
    out = []
    for i in frames:
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        r = dri.dri_track(st.handle)
        assert r.status == 0
        x, H, b = dri.dri_get_state(st.handle, with_prior=True)
        out.append((dri.state_to_dict(x), H, b))
    return out


def test_resumed_stream_tracks_like_the_uninterrupted_one():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seq = synth.sinusoid_sequence(seed=6, cam=synth.scaled_camera(160, 120), n_frames=7)
    _, dcfg = configs(seq, 3, (6, 4, 3))
    x_init = synth.initial_state(seq)

    ref = new_stream(dcfg, x_init)
    dri.dri_push_imu(ref.handle, seq.imu)
    want = _track(ref, seq, range(7))
    ref.close()

    a = new_stream(dcfg, x_init)
    dri.dri_push_imu(a.handle, seq.imu)
    _track(a, seq, range(4))
    x, H, b = dri.dri_get_state(a.handle, with_prior=True)           # checkpoint after frame 3
    a.close()

    bst = new_stream(dcfg, dri.state_to_dict(x))
    dri.dri_push_imu(bst.handle, seq.imu)
    dri.dri_upload_frame(bst.handle, seq.frame_times[3], seq.depth[3], seq.intensity[3])
    assert dri.dri_track(bst.handle).initialised == 1                # frame 3 becomes the reference
    dri.dri_set_state(bst.handle, x, H, b)                            # and the prior comes back
    got = _track(bst, seq, range(4, 7))
    bst.close()

    for (gx, gH, gb), (wx, wH, wb) in zip(got, want[4:]):
        for k in ("r_WC", "q_WC", "v_I", "bg", "ba", "q_IW"):
            np.testing.assert_allclose(gx[k], wx[k], rtol=0, atol=1e-10, err_msg=k)
        np.testing.assert_allclose(gH, wH, rtol=1e-8, atol=1e-8 * np.abs(wH).max())
        # b* on the scale of the information it carries: the offset it implies
        # for each component, in standard deviations of that component
        sd = np.sqrt(np.maximum(np.diag(wH), 1e-300))
        assert np.all(np.abs(gb - wb) <= 1e-8 * sd), np.max(np.abs(gb - wb) / sd)


def test_set_state_rejects_a_non_finite_state():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    _, dcfg = configs(seq, 2, (2, 2))
    st = new_stream(dcfg, synth.initial_state(seq))
    x = dri.dri_get_state(st.handle)
    x.r_WC[0] = float("nan")
    with pytest.raises(dri.DriError) as e:
        dri.dri_set_state(st.handle, x)
    assert e.value.code == dri.DRI_EINVAL
    st.close()
