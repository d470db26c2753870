"""Python binding of the C ABI in include/dri.h (argument marshalling only).

Every function keeps the C name and argument order; a negative status raises
DriError (dri_track returns the frame status in its result instead).  Device
memory for a stream's workspace and the CUDA stream come from PyTorch: pass a
torch.cuda.Stream and let dri_create_stream allocate the workspace as a torch
uint8 tensor, or pass your own device pointer.  The compute path is libdri.so
only: if the library is missing this module raises on import of the library,
it never falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DRI_OK = 0
DRI_EINVAL = -1
DRI_ENOMEM = -2
DRI_EADMIT = -3
DRI_ENOTREADY = -4
DRI_ELOST = -5
DRI_ETIMEDOUT = -6
DRI_ECUDA = -7
DRI_HOST = 0
DRI_DEVICE = 1
DRI_FP16_MAPS = 1
DRI_FP32_PARTIALS = 2
DRI_IMU_REINTEGRATE = 0
DRI_IMU_FIRST_ORDER = 1
DRI_TRACK_INERTIAL = 0
DRI_TRACK_RGBD_ONLY = 1
DRI_TRACK_GYRO_ONLY = 2
DRI_MAX_LEVELS = 4

c_double_p = ctypes.POINTER(ctypes.c_double)


class dri_stream_config(ctypes.Structure):
    _fields_ = [
        ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
        ("cy", ctypes.c_double),
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("iters", ctypes.c_int32 * DRI_MAX_LEVELS),
        ("T_CS", ctypes.c_double * 7),
        ("sigma_I", ctypes.c_double), ("sigma_d", ctypes.c_double),
        ("gyr_nd", ctypes.c_double), ("acc_nd", ctypes.c_double),
        ("gyr_rw", ctypes.c_double), ("acc_rw", ctypes.c_double),
        ("g", ctypes.c_double), ("sigma_grav_rw", ctypes.c_double),
        ("prior_sigma", ctypes.c_double * 5),
        ("icp_dist_thr", ctypes.c_double), ("icp_angle_thr_deg", ctypes.c_double),
        ("depth_min", ctypes.c_double), ("depth_max", ctypes.c_double),
        ("min_valid", ctypes.c_int32), ("precision_flags", ctypes.c_int32),
        ("max_imu", ctypes.c_int32), ("imu_mode", ctypes.c_int32),
        ("bias_relin_g", ctypes.c_double), ("bias_relin_a", ctypes.c_double),
        ("track_mode", ctypes.c_int32), ("count_margins", ctypes.c_int32),
        ("rgbd_lambda", ctypes.c_double), ("occlusion_thr", ctypes.c_double),
        ("icp_depth_weight", ctypes.c_int32), ("gravity_dof", ctypes.c_int32),
    ]


class dri_imu_sample(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("gyr", ctypes.c_double * 3), ("acc", ctypes.c_double * 3)]


class dri_state(ctypes.Structure):
    _fields_ = [
        ("r_WC", ctypes.c_double * 3), ("q_WC", ctypes.c_double * 4), ("v_I", ctypes.c_double * 3),
        ("bg", ctypes.c_double * 3), ("ba", ctypes.c_double * 3), ("q_IW", ctypes.c_double * 4),
        ("t", ctypes.c_double),
    ]


class dri_track_result(ctypes.Structure):
    _fields_ = [
        ("x1", dri_state), ("x0", dri_state),
        ("n_icp", ctypes.c_int32 * DRI_MAX_LEVELS), ("n_rgb", ctypes.c_int32 * DRI_MAX_LEVELS),
        ("n_margin", ctypes.c_int32 * DRI_MAX_LEVELS),
        ("cost", ctypes.c_double), ("status", ctypes.c_int32), ("initialised", ctypes.c_int32),
    ]


class dri_linearisation(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_double * (34 * 34)), ("b", ctypes.c_double * 34),
        ("H_icp", ctypes.c_double * 36), ("b_icp", ctypes.c_double * 6),
        ("H_rgb", ctypes.c_double * 36), ("b_rgb", ctypes.c_double * 6),
        ("cost_icp", ctypes.c_double), ("cost_rgb", ctypes.c_double), ("cost_imu", ctypes.c_double),
        ("e_imu", ctypes.c_double * 18),
        ("n_icp", ctypes.c_int64), ("n_rgb", ctypes.c_int64),
        ("n_margin_icp", ctypes.c_int64), ("n_margin_rgb", ctypes.c_int64),
    ]


DRI_KC_MAPS, DRI_KC_TRACK, DRI_KC_SOLVE, DRI_KC_FRAME, DRI_KC_GRAD = 0, 1, 2, 3, 4
DRI_KC_COUNT = 8


class dri_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * DRI_KC_COUNT), ("ms", ctypes.c_double * DRI_KC_COUNT),
                ("pixels", ctypes.c_double * DRI_KC_COUNT)]


class dri_batch_options(ctypes.Structure):
    _fields_ = [("rows_per_thread", ctypes.c_int32 * DRI_MAX_LEVELS), ("groups", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


class dri_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("ticks", ctypes.c_int64), ("mean_batch", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("frames_per_s", ctypes.c_double), ("hbm_used", ctypes.c_size_t),
                ("hbm_budget", ctypes.c_size_t), ("streams", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class dri_server_tick(ctypes.Structure):
    _fields_ = [("tick", ctypes.c_int64), ("requests", ctypes.c_int32), ("status", ctypes.c_int32),
                ("dequeue_ms", ctypes.c_double), ("staged_ms", ctypes.c_double),
                ("launched_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("device_ms", ctypes.c_double)]


class DriError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lib = None


def library_path():
    return _build.LIB


def load_library():
    """Loads libdri.so (built in-tree by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2207_10940_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    sig = {
        "dri_config_default": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, P(dri_stream_config)]),
        "dri_stream_workspace_bytes": (ctypes.c_int, [P(dri_stream_config), P(ctypes.c_size_t)]),
        "dri_create_stream": (ctypes.c_int, [P(dri_stream_config), P(dri_state), ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_size_t, P(ctypes.c_void_p)]),
        "dri_destroy_stream": (ctypes.c_int, [ctypes.c_void_p]),
        "dri_upload_frame": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32]),
        "dri_push_imu": (ctypes.c_int, [ctypes.c_void_p, P(dri_imu_sample), ctypes.c_size_t]),
        "dri_upload_reference": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, c_double_p, ctypes.c_size_t,
                                                ctypes.c_int32]),
        "dri_track": (ctypes.c_int, [ctypes.c_void_p, P(dri_track_result)]),
        "dri_track_batch": (ctypes.c_int, [P(ctypes.c_void_p), ctypes.c_int32, P(dri_track_result)]),
        "dri_batch_get_options": (ctypes.c_int, [P(ctypes.c_void_p), ctypes.c_int32,
                                                 P(dri_batch_options)]),
        "dri_batch_set_options": (ctypes.c_int, [P(ctypes.c_void_p), ctypes.c_int32,
                                                 P(dri_batch_options)]),
        "dri_get_state": (ctypes.c_int, [ctypes.c_void_p, P(dri_state), c_double_p, c_double_p]),
        "dri_set_state": (ctypes.c_int, [ctypes.c_void_p, P(dri_state), c_double_p, c_double_p]),
        "dri_linearise": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, P(dri_state), P(dri_state),
                                         P(dri_linearisation), ctypes.c_void_p]),
        "dri_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "dri_launch_count": (ctypes.c_int, [ctypes.c_void_p, P(ctypes.c_int64)]),
        "dri_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
        "dri_io_bytes": (ctypes.c_int, [ctypes.c_void_p, P(ctypes.c_int64), P(ctypes.c_int64)]),
        "dri_frame_counts": (ctypes.c_int, [ctypes.c_void_p, P(ctypes.c_int64), P(ctypes.c_int64)]),
        "dri_linearise_pair_noalloc": (ctypes.c_int, [P(dri_stream_config), ctypes.c_void_p,
                                                      ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_void_p, P(dri_state), P(dri_state),
                                                      P(dri_state), ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_void_p]),
        "dri_profile_read": (ctypes.c_int, [ctypes.c_void_p, P(dri_profile)]),
        "dri_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p,
                                             P(ctypes.c_void_p)]),
        "dri_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
        "dri_server_open_stream": (ctypes.c_int, [ctypes.c_void_p, P(dri_stream_config), P(dri_state),
                                                  P(ctypes.c_void_p)]),
        "dri_server_close_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
        "dri_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.c_int32, P(dri_imu_sample), ctypes.c_size_t,
                                             P(ctypes.c_uint64)]),
        "dri_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, P(dri_track_result),
                                           ctypes.c_int32]),
        "dri_server_stats_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, P(dri_server_stats)]),
        "dri_server_trace_read": (ctypes.c_int, [ctypes.c_void_p, P(dri_server_tick), ctypes.c_int32,
                                                 P(ctypes.c_int32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(code):
    return load_library().dri_status_string(int(code)).decode()


def _check(code, where):
    if code < 0:
        raise DriError(code, where)
    return code


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------

def dri_config_default(width, height):
    cfg = dri_stream_config()
    _check(load_library().dri_config_default(int(width), int(height), ctypes.byref(cfg)),
           "dri_config_default")
    return cfg


def dri_stream_workspace_bytes(cfg):
    n = ctypes.c_size_t()
    _check(load_library().dri_stream_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)),
           "dri_stream_workspace_bytes")
    return n.value


def dri_create_stream(cfg, x_init, cuda_stream=None, workspace=None, workspace_bytes=0):
    """cuda_stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (legacy default).
    workspace: a device pointer (int) or a torch tensor; None lets the library allocate."""
    h = ctypes.c_void_p()
    cs = getattr(cuda_stream, "cuda_stream", cuda_stream)
    ws = workspace
    if ws is not None and hasattr(ws, "data_ptr"):
        workspace_bytes = ws.numel() * ws.element_size()
        ws = ws.data_ptr()
    _check(load_library().dri_create_stream(ctypes.byref(cfg), ctypes.byref(x_init),
                                            ctypes.c_void_p(cs or 0), ctypes.c_void_p(ws or 0),
                                            ctypes.c_size_t(workspace_bytes), ctypes.byref(h)),
           "dri_create_stream")
    _shapes[h.value] = (int(cfg.width), int(cfg.height))
    _prior_dims[h.value] = 18 if cfg.gravity_dof == DRI_GRAVITY_3D else 17
    return h


def dri_destroy_stream(s):
    _shapes.pop(_hval(s), None)
    _prior_dims.pop(_hval(s), None)
    return _check(load_library().dri_destroy_stream(s), "dri_destroy_stream")


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


# (width, height) of each open stream handle, for the argument checks below,
# and the size of its prior (17, or 18 with the 3-D gravity form)
_shapes = {}
_prior_dims = {}
DRI_GRAVITY_2DOF = 2
DRI_GRAVITY_3D = 3


def _hval(s):
    s = getattr(s, "handle", s)
    return s.value if isinstance(s, ctypes.c_void_p) else s


def _buffer(a, name, dtype, n_min, device):
    """Pointer of an image or output argument after checking it: a torch tensor
    must be on the GPU exactly when `device` is set, contiguous, of `dtype`
    ("float32" or "uint8") and hold at least n_min elements; a numpy array must
    be host memory (device unset), C-contiguous, of `dtype`, large enough.  A
    raw integer pointer is passed as it is (the caller vouches for it)."""
    if isinstance(a, (int, ctypes.c_void_p)):
        return a.value if isinstance(a, ctypes.c_void_p) else a
    if hasattr(a, "data_ptr"):
        if bool(a.is_cuda) != bool(device):
            raise DriError(DRI_EINVAL, f"{name}: a {'device' if device else 'host'} tensor is required")
        if not a.is_contiguous():
            raise DriError(DRI_EINVAL, f"{name}: tensor must be contiguous")
        if str(a.dtype) != "torch." + dtype:
            raise DriError(DRI_EINVAL, f"{name}: dtype must be {dtype}")
        if a.numel() < n_min:
            raise DriError(DRI_EINVAL, f"{name}: {a.numel()} elements, at least {n_min} needed")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if device:
            raise DriError(DRI_EINVAL, f"{name}: device memory is required")
        if not a.flags.c_contiguous:
            raise DriError(DRI_EINVAL, f"{name}: host arrays must be C-contiguous")
        if a.dtype != np.dtype(dtype):
            raise DriError(DRI_EINVAL, f"{name}: dtype must be {dtype}")
        if a.size < n_min:
            raise DriError(DRI_EINVAL, f"{name}: {a.size} elements, at least {n_min} needed")
        return a.ctypes.data
    raise TypeError(f"{name}: expected a torch tensor, a numpy array or a pointer")


def _image_elems(s, pitch_bytes):
    """Floats an image of stream s spans (rows pitch_bytes apart), or 0 if the
    stream's size is unknown here."""
    wh = _shapes.get(_hval(s))
    if wh is None:
        return 0
    w, h = wh
    pitch = pitch_bytes // 4 if pitch_bytes else w
    return (h - 1) * pitch + w


def dri_upload_frame(s, t, depth, intensity, pitch_bytes=0, mem_kind=None):
    """depth / intensity: float32 numpy arrays (host) or torch tensors (host or
    device) of at least the stream's image size; checked before the call."""
    if mem_kind is None:
        mem_kind = DRI_DEVICE if (hasattr(depth, "is_cuda") and depth.is_cuda) else DRI_HOST
    n = _image_elems(s, pitch_bytes)
    dev = mem_kind == DRI_DEVICE
    pd = _buffer(depth, "depth", "float32", n, dev)
    pi = _buffer(intensity, "intensity", "float32", n, dev)
    return _check(load_library().dri_upload_frame(s, float(t), ctypes.c_void_p(pd), ctypes.c_void_p(pi),
                                                  pitch_bytes, mem_kind), "dri_upload_frame")


def dri_upload_reference(s, vertex_W, normal_W, intensity, T_WC_ref, pitch_px=0, mem_kind=None):
    """vertex_W, normal_W: (H, W, 3) float32; intensity (H, W) float32; numpy (host)
    or CUDA tensors (device); T_WC_ref: r (3) + q (w, x, y, z)."""
    if mem_kind is None:
        mem_kind = DRI_DEVICE if (hasattr(vertex_W, "is_cuda") and vertex_W.is_cuda) else DRI_HOST
    n = _image_elems(s, 4 * pitch_px)
    dev = mem_kind == DRI_DEVICE
    pv = _buffer(vertex_W, "vertex_W", "float32", 3 * n, dev)
    pn = _buffer(normal_W, "normal_W", "float32", 3 * n, dev)
    pi = _buffer(intensity, "intensity", "float32", n, dev)
    T = np.ascontiguousarray(T_WC_ref, dtype=np.float64)
    if T.size != 7:
        raise DriError(DRI_EINVAL, "T_WC_ref: 7 values (r, q) are required")
    return _check(load_library().dri_upload_reference(
        s, ctypes.c_void_p(pv), ctypes.c_void_p(pn), ctypes.c_void_p(pi), T.ctypes.data_as(c_double_p),
        pitch_px, mem_kind), "dri_upload_reference")


def imu_array(samples):
    """(N, 7) array [t, gyr(3), acc(3)] -> ctypes array of dri_imu_sample."""
    samples = np.ascontiguousarray(samples, dtype=np.float64).reshape(-1, 7)
    arr = (dri_imu_sample * len(samples))()
    ctypes.memmove(arr, samples.ctypes.data, samples.nbytes)
    return arr


def dri_push_imu(s, samples):
    arr = samples if isinstance(samples, ctypes.Array) else imu_array(samples)
    return _check(load_library().dri_push_imu(s, arr, len(arr)), "dri_push_imu")


def dri_track(s, wait=True):
    """Returns the dri_track_result (wait=True; its status is DRI_OK or DRI_ELOST) or
    None (asynchronous).  Other errors raise DriError."""
    if not wait:
        _check(load_library().dri_track(s, None), "dri_track")
        return None
    res = dri_track_result()
    code = load_library().dri_track(s, ctypes.byref(res))
    if code < 0 and code != DRI_ELOST:
        raise DriError(code, "dri_track")
    return res


def _handles(streams):
    arr = (ctypes.c_void_p * len(streams))()
    for i, h in enumerate(streams):
        arr[i] = getattr(h, "handle", h)
    return arr


def dri_track_batch(streams, wait=True):
    """Tracks the uploaded frame of every stream (handles or Stream objects) in
    one batched launch sequence.  wait=True: returns the list of
    dri_track_result (status DRI_OK, DRI_ELOST or DRI_ENOTREADY for a stream
    that sat the call out); wait=False: None.  Call errors raise DriError."""
    arr = _handles(streams)
    if not wait:
        _check(load_library().dri_track_batch(arr, len(streams), None), "dri_track_batch")
        return None
    res = (dri_track_result * len(streams))()
    _check(load_library().dri_track_batch(arr, len(streams), res), "dri_track_batch")
    return list(res)


def dri_batch_get_options(streams):
    out = dri_batch_options()
    _check(load_library().dri_batch_get_options(_handles(streams), len(streams), ctypes.byref(out)),
           "dri_batch_get_options")
    return out


def dri_batch_set_options(streams, rows_per_thread=None, groups=None, autotune=None):
    """Updates the given fields of this stream list's plan options."""
    try:
        opt = dri_batch_get_options(streams)
    except DriError:                       # no plan yet: it is made with its defaults
        opt = dri_batch_options()
        opt.groups = 0                     # keep the plan's own (default) groups
        opt.autotune = 0 if len(streams) == 1 else 1
    if rows_per_thread is not None:
        rows = list(rows_per_thread) + [1] * (DRI_MAX_LEVELS - len(rows_per_thread))
        opt.rows_per_thread[:] = rows
        opt.autotune = 0
    if groups is not None:
        opt.groups = int(groups)
    if autotune is not None:
        opt.autotune = int(autotune)
    _check(load_library().dri_batch_set_options(_handles(streams), len(streams), ctypes.byref(opt)),
           "dri_batch_set_options")


def prior_dim(s):
    """Size of the stream's prior (17, or 18 for the 3-D gravity form)."""
    return _prior_dims.get(_hval(s), 17)


def dri_get_state(s, with_prior=False):
    x = dri_state()
    if with_prior:
        n = prior_dim(s)
        H = np.zeros((n, n))
        b = np.zeros(n)
        _check(load_library().dri_get_state(s, ctypes.byref(x), H.ctypes.data_as(c_double_p),
                                            b.ctypes.data_as(c_double_p)), "dri_get_state")
        return x, H, b
    _check(load_library().dri_get_state(s, ctypes.byref(x), None, None), "dri_get_state")
    return x


def dri_set_state(s, x1, H_prior=None, b_prior=None):
    n = prior_dim(s)
    Hp = None if H_prior is None else np.ascontiguousarray(H_prior, dtype=np.float64)
    bp = None if b_prior is None else np.ascontiguousarray(b_prior, dtype=np.float64)
    if (Hp is not None and Hp.size != n * n) or (bp is not None and bp.size != n):
        raise DriError(DRI_EINVAL, f"dri_set_state: the prior is {n} x {n} for this stream")
    return _check(load_library().dri_set_state(
        s, ctypes.byref(x1), None if Hp is None else Hp.ctypes.data_as(c_double_p),
        None if bp is None else bp.ctypes.data_as(c_double_p)), "dri_set_state")


def dri_linearise(s, level, x0, x1, want_flags=False, shape=None):
    out = dri_linearisation()
    flags = None
    fptr = None
    if want_flags:
        flags = np.zeros(shape, dtype=np.uint8)
        fptr = ctypes.c_void_p(flags.ctypes.data)
    code = load_library().dri_linearise(s, int(level), ctypes.byref(x0), ctypes.byref(x1),
                                        ctypes.byref(out), fptr)
    _check(code, "dri_linearise")
    return out, flags


def dri_launch_count(s):
    n = ctypes.c_int64()
    _check(load_library().dri_launch_count(s, ctypes.byref(n)), "dri_launch_count")
    return n.value


def dri_linearise_pair_noalloc(cfg, ref_depth, ref_intensity, live_depth, live_intensity, x_ref,
                               x0, x1, out_ptr, flags_ptr=None, cuda_stream=None):
    """All image and output arguments are device pointers (ints) or CUDA tensors.
    Tensors are checked before the call: images float32 with cfg.width *
    cfg.height elements, out_ptr uint8 with sizeof(dri_linearisation) bytes,
    flags_ptr uint8 with cfg.width * cfg.height bytes."""
    cs = getattr(cuda_stream, "cuda_stream", cuda_stream)
    n = int(cfg.width) * int(cfg.height)
    imgs = [_buffer(a, k, "float32", n, True) for a, k in
            ((ref_depth, "ref_depth"), (ref_intensity, "ref_intensity"), (live_depth, "live_depth"),
             (live_intensity, "live_intensity"))]
    out = _buffer(out_ptr, "out", "uint8", ctypes.sizeof(dri_linearisation), True)
    flags = 0 if flags_ptr is None else _buffer(flags_ptr, "flags", "uint8", n, True)
    return _check(load_library().dri_linearise_pair_noalloc(
        ctypes.byref(cfg), *[ctypes.c_void_p(p) for p in imgs], ctypes.byref(x_ref), ctypes.byref(x0),
        ctypes.byref(x1), ctypes.c_void_p(out), ctypes.c_void_p(flags), ctypes.c_void_p(cs or 0)),
        "dri_linearise_pair_noalloc")


def dri_frame_counts(s):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().dri_frame_counts(s, ctypes.byref(a), ctypes.byref(b)), "dri_frame_counts")
    return a.value, b.value


def dri_io_bytes(s):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().dri_io_bytes(s, ctypes.byref(a), ctypes.byref(b)), "dri_io_bytes")
    return a.value, b.value


def dri_profile_enable(s, enable=True):
    return _check(load_library().dri_profile_enable(s, 1 if enable else 0), "dri_profile_enable")


def dri_profile_read(s):
    out = dri_profile()
    _check(load_library().dri_profile_read(s, ctypes.byref(out)), "dri_profile_read")
    return out


# ---------------------------------------------------------------------------
# conversions (marshalling only)
# ---------------------------------------------------------------------------

def state_from_dict(d, t=0.0):
    x = dri_state()
    x.r_WC[:] = [float(v) for v in d["r_WC"]]
    x.q_WC[:] = [float(v) for v in d["q_WC"]]
    x.v_I[:] = [float(v) for v in d["v_I"]]
    x.bg[:] = [float(v) for v in d["bg"]]
    x.ba[:] = [float(v) for v in d["ba"]]
    x.q_IW[:] = [float(v) for v in d["q_IW"]]
    x.t = float(d.get("t", t))
    return x


def state_to_dict(x):
    return dict(r_WC=np.array(x.r_WC[:]), q_WC=np.array(x.q_WC[:]), v_I=np.array(x.v_I[:]),
                bg=np.array(x.bg[:]), ba=np.array(x.ba[:]), q_IW=np.array(x.q_IW[:]), t=x.t)


def config_for(width, height, fx, fy, cx, cy, levels, iters, q_CS=None, r_CS=None, **overrides):
    """Stream configuration from intrinsics, schedule and extrinsic T_CS; other
    fields keep dri_config_default's values."""
    cfg = dri_config_default(width, height)
    cfg.fx, cfg.fy, cfg.cx, cfg.cy = float(fx), float(fy), float(cx), float(cy)
    cfg.levels = int(levels)
    for i in range(DRI_MAX_LEVELS):
        cfg.iters[i] = int(iters[i]) if i < len(iters) else 0
    if q_CS is not None:
        cfg.T_CS[3:7] = [float(v) for v in q_CS]
    if r_CS is not None:
        cfg.T_CS[0:3] = [float(v) for v in r_CS]
    for k, v in overrides.items():
        if k == "prior_sigma":
            cfg.prior_sigma[:] = list(v)
        else:
            setattr(cfg, k, v)
    return cfg


class Stream:
    """A tracking stream whose workspace is a torch uint8 device tensor and whose
    work is ordered on a torch CUDA stream."""

    def __init__(self, cfg, x_init, torch_stream=None, device="cuda"):
        import torch
        self.cfg = cfg
        self.torch_stream = torch_stream if torch_stream is not None else torch.cuda.Stream(device)
        nbytes = dri_stream_workspace_bytes(cfg)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        ptr = self.workspace.data_ptr()
        aligned = (ptr + 255) // 256 * 256
        self.handle = dri_create_stream(cfg, x_init, self.torch_stream, aligned, nbytes)

    def close(self):
        if self.handle is not None:
            dri_destroy_stream(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# serving loop
# ---------------------------------------------------------------------------

def dri_server_create(hbm_budget_bytes, max_batch, cuda_stream=None):
    cs = getattr(cuda_stream, "cuda_stream", cuda_stream)
    h = ctypes.c_void_p()
    _check(load_library().dri_server_create(int(hbm_budget_bytes), int(max_batch),
                                            ctypes.c_void_p(cs or 0), ctypes.byref(h)),
           "dri_server_create")
    return h


def dri_server_destroy(srv):
    return _check(load_library().dri_server_destroy(srv), "dri_server_destroy")


def dri_server_open_stream(srv, cfg, x_init):
    h = ctypes.c_void_p()
    _check(load_library().dri_server_open_stream(srv, ctypes.byref(cfg), ctypes.byref(x_init),
                                                 ctypes.byref(h)), "dri_server_open_stream")
    _shapes[h.value] = (int(cfg.width), int(cfg.height))
    _prior_dims[h.value] = 18 if cfg.gravity_dof == DRI_GRAVITY_3D else 17
    return h


def dri_server_close_stream(srv, s):
    _shapes.pop(_hval(s), None)
    _prior_dims.pop(_hval(s), None)
    return _check(load_library().dri_server_close_stream(srv, s), "dri_server_close_stream")


def dri_server_submit(srv, s, t, depth, intensity, imu=(), pitch_bytes=0, mem_kind=None):
    """Queues a frame; the images (checked as in dri_upload_frame) must stay
    alive until the ticket is done."""
    if mem_kind is None:
        mem_kind = DRI_DEVICE if (hasattr(depth, "is_cuda") and depth.is_cuda) else DRI_HOST
    n_px = _image_elems(s, pitch_bytes)
    dev = mem_kind == DRI_DEVICE
    pd = _buffer(depth, "depth", "float32", n_px, dev)
    pi = _buffer(intensity, "intensity", "float32", n_px, dev)
    arr = imu if isinstance(imu, ctypes.Array) else (imu_array(imu) if len(imu) else None)
    n = 0 if arr is None else len(arr)
    ticket = ctypes.c_uint64()
    _check(load_library().dri_server_submit(srv, s, float(t), ctypes.c_void_p(pd), ctypes.c_void_p(pi),
                                            pitch_bytes, mem_kind, arr, n, ctypes.byref(ticket)),
           "dri_server_submit")
    return ticket.value


def dri_server_poll(srv, ticket, timeout_ms=-1):
    """(status, dri_track_result) of a done request, or (DRI_ETIMEDOUT, None)."""
    res = dri_track_result()
    code = load_library().dri_server_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(res),
                                          int(timeout_ms))
    if code == DRI_ETIMEDOUT:
        return code, None
    if code == DRI_EINVAL:
        raise DriError(code, "dri_server_poll")
    return code, res


def dri_server_stats_read(srv, reset=False):
    out = dri_server_stats()
    _check(load_library().dri_server_stats_read(srv, int(bool(reset)), ctypes.byref(out)),
           "dri_server_stats_read")
    return out


def dri_server_trace_read(srv, cap=65536):
    """The most recent ticks' host timestamps (list of dri_server_tick, oldest first)."""
    out = (dri_server_tick * cap)()
    n = ctypes.c_int32()
    _check(load_library().dri_server_trace_read(srv, out, int(cap), ctypes.byref(n)),
           "dri_server_trace_read")
    return list(out[: n.value])
