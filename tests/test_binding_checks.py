"""Argument checks made before any pointer reaches a kernel (no GPU needed).

The Python binding checks tensors and arrays against the stream's image size,
dtype, memory side and contiguity; dri_linearise_pair_noalloc checks its
options and states on the host before its first CUDA call.  Each case here is
rejected with DRI_EINVAL without touching a device."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def dri():
    from paper_2207_10940_gb300 import build
    try:
        build.build()
    except RuntimeError as exc:         # no toolkit: nothing to check here
        pytest.skip(str(exc))
    from paper_2207_10940_gb300 import dri as d
    d.load_library()
    return d


def _einval(dri, fn, *a, **kw):
    with pytest.raises(dri.DriError) as e:
        fn(*a, **kw)
    assert e.value.code == dri.DRI_EINVAL
    return e.value


def test_buffer_checks(dri):
    ok = np.zeros(12, np.float32)
    assert dri._buffer(ok, "x", "float32", 12, False) == ok.ctypes.data
    assert dri._buffer(1234, "x", "float32", 12, True) == 1234          # raw pointer: passed on
    _einval(dri, dri._buffer, ok, "x", "float32", 13, False)            # too small
    _einval(dri, dri._buffer, ok, "x", "float32", 12, True)             # host array as device memory
    _einval(dri, dri._buffer, ok.astype(np.float64), "x", "float32", 12, False)
    _einval(dri, dri._buffer, np.zeros((4, 6), np.float32)[:, ::2], "x", "float32", 12, False)
    torch = pytest.importorskip("torch")
    t = torch.zeros(12)
    assert dri._buffer(t, "x", "float32", 12, False) == t.data_ptr()
    _einval(dri, dri._buffer, t, "x", "float32", 12, True)              # CPU tensor as device memory
    _einval(dri, dri._buffer, t.to(torch.uint8), "x", "float32", 12, False)
    _einval(dri, dri._buffer, torch.zeros(4, 6)[:, ::2], "x", "float32", 12, False)


def test_image_size_follows_the_stream(dri):
    dri._shapes[777] = (64, 48)
    try:
        assert dri._image_elems(777, 0) == 64 * 48
        assert dri._image_elems(777, 4 * 80) == 47 * 80 + 64
        assert dri._image_elems(778, 0) == 0                             # unknown handle: no bound
    finally:
        dri._shapes.pop(777)


def _state(dri):
    x = dri.dri_state()
    x.q_WC[0] = 1.0
    x.q_IW[0] = 1.0
    return x


def _noalloc(dri, cfg, x0=None):
    """Calls the entry with fake (never dereferenced) device pointers."""
    lib = dri.load_library()
    x = _state(dri)
    out = dri.dri_linearisation()
    p = ctypes.c_void_p(0x10000)
    return lib.dri_linearise_pair_noalloc(ctypes.byref(cfg), p, p, p, p, ctypes.byref(x),
                                          ctypes.byref(x0 or x), ctypes.byref(x), p, None, None)


def test_noalloc_rejects_options_and_states_before_any_cuda_call(dri):
    for field, value in (("precision_flags", 4), ("occlusion_thr", -0.1), ("occlusion_thr", float("nan")),
                         ("icp_depth_weight", 2), ("width", 640)):
        cfg = dri.dri_config_default(320, 240)
        setattr(cfg, field, value)
        assert _noalloc(dri, cfg) == dri.DRI_EINVAL, field
    cfg = dri.dri_config_default(320, 240)
    zero_q = _state(dri)
    zero_q.q_WC[0] = 0.0
    assert _noalloc(dri, cfg, zero_q) == dri.DRI_EINVAL
    nan_r = _state(dri)
    nan_r.r_WC[1] = float("nan")
    assert _noalloc(dri, cfg, nan_r) == dri.DRI_EINVAL


def test_gravity_form_is_validated_on_the_host(dri):
    cfg = dri.dri_config_default(320, 240)
    assert dri.dri_stream_workspace_bytes(cfg) > 0
    cfg.gravity_dof = dri.DRI_GRAVITY_3D
    assert dri.dri_stream_workspace_bytes(cfg) > 0
    cfg.track_mode = 1                       # the 3-D form serves the inertial tracker only
    _einval(dri, dri.dri_stream_workspace_bytes, cfg)
    cfg = dri.dri_config_default(320, 240)
    cfg.gravity_dof = 5
    _einval(dri, dri.dri_stream_workspace_bytes, cfg)
    cfg = dri.dri_config_default(320, 240)
    cfg.icp_angle_thr_deg = 90.0             # the angle test must reject zero normals
    _einval(dri, dri.dri_stream_workspace_bytes, cfg)
    cfg = dri.dri_config_default(320, 240)
    cfg.count_margins = 2                    # an option, 0 or 1
    _einval(dri, dri.dri_stream_workspace_bytes, cfg)


def test_empty_and_null_batches_are_rejected(dri):
    """dri_track_batch takes at least one stream: an empty, negative or NULL
    list is DRI_EINVAL before any CUDA call."""
    lib = dri.load_library()
    out = (dri.dri_track_result * 1)()
    arr = (ctypes.c_void_p * 1)()
    assert lib.dri_track_batch(None, 1, out) == dri.DRI_EINVAL
    assert lib.dri_track_batch(arr, 0, out) == dri.DRI_EINVAL
    assert lib.dri_track_batch(arr, -1, out) == dri.DRI_EINVAL
