#!/usr/bin/env python3
"""Benchmark of the tracking hot path: tracked frames/s at 640x480, batched
and plain.

A tracked frame is one pass of every step of the hot path: pyramid, normal and
gradient maps, 19 Gauss-Newton iterations of the fused photometric + ICP kernel
with the FP64 IMU / solver step, marginalisation and the reference swap, on the
seeded synthetic 640x480 RGB-D + 400 Hz IMU sequence (sinusoidal path, peak
1.5 m/s and 90 deg/s, 100-frame period rendered once and looped), 3 pyramid
levels with 10/5/4 iterations.

* batched (the headline, one step = one frame of each of 64 independent
  streams in one dri_track_batch call): stream i starts at frame 37 i mod 100
  of the loop, so a step reads 64 different frames;
* plain (one step = one frame of a single stream, dri_track);
* served: 256 streams of mixed resolution (320x240, 640x480, 1280x720 by
  stream id mod 3) submit frames at 30 Hz each with exponential arrival jitter
  to the library's serving loop (dri_server_*); p50 / p99 submit-to-result
  latency and completed frames/s are reported beside the batched number.

Frames live on the device before timing starts; the 100 distinct frames
(245 MB) exceed the 129 MB L2.  Output: one JSON line (rank 0).
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import ctypes
import gc
import hashlib
import json
import multiprocessing as mp
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, H = 640, 480
LEVELS, ITERS = 3, (10, 5, 4)
FPS = 30.0
N_UNIQUE = 100
SEQ_SEED = 2
# Algorithmic bytes per pixel-iteration (the method's unique reads, FP32 maps):
# live depth 4, intensity 4 and normal 12; reference vertex 12, normal 12,
# intensity 4 and gradient 8.  FP16 normal and gradient maps: 40 B.  The
# kernel itself reads 48 B (32 B with FP16 maps): it keeps the reference as
# depth + normal in its own camera and rebuilds the vertex from the depth.
BYTES_PER_PIXEL_ITER = 56
BYTES_PER_PIXEL_ITER_FP16 = 40
KERNEL_BYTES_PER_PIXEL_ITER = 48
KERNEL_BYTES_PER_PIXEL_ITER_FP16 = 32
PIXEL_ITERS_PER_FRAME = sum((W >> l) * (H >> l) * ITERS[l] for l in range(LEVELS))
BATCH = 64
BATCH_OFFSET = 37             # stream i starts at frame (37 i) mod 100 of the loop


def _render_one(args):
    from paper_2207_10940_gb300 import synth
    seed, i = args
    seq = synth.sinusoid_sequence(seed=seed, cam=synth.CAM_640, n_frames=N_UNIQUE, rate=400.0,
                                  render_frames=False)
    return synth.render_frame(seq, i, seed=seed)


def make_inputs(n_frames_total, workers):
    """Sequence metadata, the N_UNIQUE rendered frames and IMU samples up to the
    last timed frame (the path is periodic, so frame k shows frame k % 100)."""
    from paper_2207_10940_gb300 import synth
    seq = synth.sinusoid_sequence(seed=SEQ_SEED, cam=synth.CAM_640, n_frames=N_UNIQUE, rate=400.0,
                                  render_frames=False)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        frames = pool.map(_render_one, [(SEQ_SEED, i) for i in range(N_UNIQUE)])
    imu = synth.sequence_imu(seq, (n_frames_total + 1) / FPS, seed=SEQ_SEED)
    return seq, frames, imu


def dri_config(seq, flags=0, imu_mode=0, track_mode=0, occlusion_thr=0.0):
    from paper_2207_10940_gb300 import dri, synth
    cam = seq.cam
    return dri.config_for(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, LEVELS, ITERS,
                          q_CS=synth.matrix_to_quat(seq.R_CS), r_CS=seq.r_CS, precision_flags=flags,
                          imu_mode=imu_mode, track_mode=track_mode, occlusion_thr=occlusion_thr)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def track_traffic():
    """DRAM bytes per pixel-iteration of the track kernel from the committed ncu
    summary, or None if the kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "track_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2207_10940_gb300", "csrc", "track.cu")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    h = hashlib.sha1(open(src, "rb").read()).hexdigest()
    if d.get("track_cu_sha1") != h:
        return None
    return float(d["dram_bytes_per_pixel_iter"])


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the samples' file: DRI_CLOCKS_DIR, else the system's temporary directory
        out_dir = os.environ.get("DRI_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        # the sampler's start-up (its NVML initialisation) stays out of the timed
        # region: wait for its first sample, at most 1.5 s (by then the start-up
        # is over even if the samples are still in its output buffer)
        t = time.perf_counter()
        while time.perf_counter() - t < 1.5 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v == "Active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


class ServeMonitor:
    """Samples during a served pass, to place its slow ticks: SM clock and
    throttle reasons every 100 ms (with the sample's wall time), and the GPU's
    compute processes every 500 ms (another process on the GPU would share it)."""
    CLK = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        out_dir = os.environ.get("DRI_CLOCKS_DIR") or tempfile.gettempdir()
        self.paths = [os.path.join(out_dir, f"serve_{n}_{os.getpid()}.csv") for n in ("clk", "apps")]
        self.procs = []

    def __enter__(self):
        cmds = [["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.CLK}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                ["nvidia-smi", f"--id={self.index}", "--query-compute-apps=pid,used_memory",
                 "--format=csv,noheader,nounits", "-lms", "500"]]
        self.files = []
        for path, cmd in zip(self.paths, cmds):
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                f = open(path, "w")
                self.files.append(f)
                self.procs.append(subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL))
            except (OSError, FileNotFoundError):
                pass
        return self

    def __exit__(self, *a):
        for pr in self.procs:
            pr.terminate()
            pr.wait()
        for f in self.files:
            f.close()

    def _clock_rows(self):
        import datetime
        rows = []
        try:
            lines = open(self.paths[0]).read().splitlines()
        except OSError:
            return rows
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                t = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((t, float(parts[1]), float(parts[2]), parts[3:7]))
            except ValueError:
                pass
        return rows

    def summary(self, t0_wall, t1_wall, stalls):
        """Clock and process samples between the wall times t0 and t1, and the
        clock sample nearest to each stalled tick (wall time, tick ms)."""
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [r for r in self._clock_rows() if t0_wall <= r[0] <= t1_wall]
        out = {"clock_samples": len(rows)}
        if rows:
            mhz = np.array([r[1] for r in rows])
            out.update(sm_mhz_median=float(np.median(mhz)), sm_mhz_min=float(mhz.min()),
                       sm_max_mhz=max(r[2] for r in rows),
                       reasons=sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v == "Active"}),
                       samples_below_95pct=int(np.sum(mhz < 0.95 * max(r[2] for r in rows))))
        pids = set()
        try:
            for line in open(self.paths[1]):
                parts = [x.strip() for x in line.split(",")]
                if parts and parts[0].isdigit():
                    pids.add(int(parts[0]))
        except OSError:
            pass
        # process ids as the driver reports them (a container may number its
        # processes differently): more than one id means another process
        out["compute_pids"] = sorted(pids)
        out["own_pid"] = os.getpid()
        near = []
        for tw, tick_ms in stalls[:10]:
            if not rows:
                break
            r = min(rows, key=lambda r: abs(r[0] - tw))
            near.append({"at_s": tw - t0_wall, "tick_ms": tick_ms, "sample_dt_s": r[0] - tw,
                         "sm_mhz": r[1], "reasons": [names[i] for i, v in enumerate(r[3]) if v == "Active"]})
        out["stalled_ticks"] = near
        return out


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded samples)
# ---------------------------------------------------------------------------

_BAND = {}


def _band_setup(frames01, imu):
    """Worker state of the all-cores oracle timing: the oracle tracker after the
    first frame and the second frame's levels (pool initializer)."""
    from oracle import gn, imu as imu_mod, maps
    from oracle.params import TrackerConfig
    from paper_2207_10940_gb300 import synth
    seq = synth.sinusoid_sequence(seed=SEQ_SEED, cam=synth.CAM_640, n_frames=N_UNIQUE, rate=400.0,
                                  render_frames=False)
    cam = seq.cam
    cfg = TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=LEVELS,
                        iters=ITERS, R_CS=seq.R_CS, r_CS=seq.r_CS)
    tr = gn.Tracker(cfg, synth.initial_state(seq))
    tr.push_imu(imu)
    tr.track(frames01[0][0], frames01[0][1], 0.0)
    lv = maps.frame_levels(frames01[1][0], frames01[1][1], cfg)
    Wimu, _ = imu_mod.weight(tr.x, tr.imu, 0.0, 1.0 / FPS, cfg)
    _BAND.update(tr=tr, lv=lv, Wimu=Wimu)


def _band_work(job):
    """One worker's share: oracle linearisations (all terms) of its own band of
    level-0 rows, repeated until `seconds` have passed; returns pixel-iterations."""
    import copy
    r0, rows, seconds = job
    tr, lv, Wimu = _BAND["tr"], _BAND["lv"], _BAND["Wimu"]
    b = copy.copy(lv[0])
    sl = slice(r0, r0 + rows)
    b.depth, b.V, b.V_valid, b.N, b.N_valid, b.I = (b.depth[sl], b.V[sl], b.V_valid[sl],
                                                     b.N[sl], b.N_valid[sl], b.I[sl])
    levels = [b] + lv[1:]
    x = tr.x.copy()
    px, t = 0, time.perf_counter()
    while time.perf_counter() - t < seconds:
        tr.linearise_all(levels, 0, x, x, 0.0, 1.0 / FPS, Wimu)
        px += rows * W                     # W: pixels per level-0 row
    return px


def oracle_all_cores(frames, imu, seconds, workers):
    """The oracle's per-pixel loop spread over the host's cores (timing only):
    each worker process linearises its own band of level-0 rows with the
    unchanged FP64 oracle for `seconds`; frames/s = all workers' pixel-
    iterations / wall time / pixel-iterations per frame."""
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"                        # one thread per worker process
    try:
        ctx = mp.get_context("spawn")
        rows = max(1, H // workers)
        with ctx.Pool(workers, initializer=_band_setup, initargs=(frames[:2], imu)) as pool:
            pool.map(_band_work, [(0, 1, 0.0)] * workers)      # every worker set up
            t = time.perf_counter()
            px = sum(pool.map(_band_work, [(min(i * rows, H - rows), rows, seconds)
                                           for i in range(workers)]))
            el = time.perf_counter() - t
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return px / PIXEL_ITERS_PER_FRAME / el, el, rows


def oracle_frames_per_s(seq, frames, imu, budget_s):
    """Whole frames tracked by the FP64 oracle until the time budget is spent."""
    from oracle import gn
    from oracle.params import TrackerConfig
    from paper_2207_10940_gb300 import synth
    cam = seq.cam
    cfg = TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=LEVELS,
                        iters=ITERS, R_CS=seq.R_CS, r_CS=seq.r_CS)
    tr = gn.Tracker(cfg, synth.initial_state(seq))
    tr.push_imu(imu)
    states = [tr.track(frames[0][0], frames[0][1], 0.0)["x1"].to_dict()]
    n, t_total = 0, 0.0
    while t_total < budget_s or n == 0:
        i = n + 1
        t = time.perf_counter()
        r = tr.track(frames[i % N_UNIQUE][0], frames[i % N_UNIQUE][1], i / FPS)
        t_total += time.perf_counter() - t
        states.append(r["x1"].to_dict())
        n += 1
    return n / t_total, n, t_total, states


def odometry_pass(seq, imu, d_dev, i_dev, d_pin, i_pin, dev, n_frames, flags, imu_mode, track_mode=0,
                  occlusion_thr=0.0):
    """One stream tracked over n_frames frames of the periodic sequence with every
    result read back: its states, for the odometry errors against ground truth."""
    run = Runner(seq, imu, d_dev, i_dev, d_pin, i_pin, [0], dev, None, None, flags, imu_mode, track_mode,
                 occlusion_thr)
    states = []
    for _ in range(n_frames):
        res = run.step(wait=True)
        states.append(run.dri.state_to_dict(res.x1))
    run.close()
    return states


ODOMETRY_OCCLUSION_THR = 0.03    # m, the occlusion test's threshold in the odometry comparison


def rgbd_only_report(seq, states):
    """Trajectory errors against ground truth over the same frames as the
    odometry pass (for the RGB-D-only baseline, the gyro-only setup and the
    occlusion variant)."""
    from paper_2207_10940_gb300 import odometry
    gt = [seq.gt[k % N_UNIQUE] for k in range(len(states))]
    ev = odometry.evaluate(states, gt)
    return {k: ev[k] for k in ("frames", "ate_rmse_m", "ate_rmse_unaligned_m", "final_position_error_m",
                               "rotation_rmse_rad")}


def odometry_report(seq, states, oracle_states):
    """Errors against ground truth (frame k shows loop frame k mod 100) and the
    largest pose difference to the oracle over the frames it tracked."""
    from oracle.so3 import State
    from paper_2207_10940_gb300 import odometry
    gt = [seq.gt[k % N_UNIQUE] for k in range(len(states))]
    ev = odometry.evaluate(states, gt)
    m = min(len(states), len(oracle_states))
    da = dr = 0.0
    for a, b in zip(states[:m], oracle_states[:m]):
        xa, xb = State.from_dict(a), State.from_dict(b)
        da = max(da, odometry.rotation_angle(xa.R.T @ xb.R))
        dr = max(dr, float(np.linalg.norm(xa.r - xb.r)))
    ev["vs_oracle"] = {"frames": m, "max_rotation_diff_rad": da, "max_position_diff_m": dr}
    ev["sequence"] = "640x480 sinusoid (peak 1.5 m/s, 90 deg/s yaw), 400 Hz IMU, biases 1e-3 rad/s, 0.05 m/s^2"
    return ev


def oracle_band_steps(seq, frames, imu, steps, warmup, budget_s):
    """Reference arm: each step is one oracle Gauss-Newton iteration (linearise
    all terms, assemble, solve) on a band of level-0 rows of the second frame;
    frames/s = processed pixel-iterations / time / pixel-iterations per frame."""
    from oracle import gn, imu as imu_mod, maps
    from oracle.gn import cholesky_solve
    from oracle.params import TrackerConfig
    from paper_2207_10940_gb300 import synth
    cam = seq.cam
    cfg = TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=LEVELS,
                        iters=ITERS, R_CS=seq.R_CS, r_CS=seq.r_CS)
    tr = gn.Tracker(cfg, synth.initial_state(seq))
    tr.push_imu(imu)
    tr.track(frames[0][0], frames[0][1], 0.0)
    lv = maps.frame_levels(frames[1][0], frames[1][1], cfg)
    x0 = tr.x.copy()
    x1 = tr.x.copy()
    t0, t1 = 0.0, 1.0 / FPS
    Wimu, _ = imu_mod.weight(x0, tr.imu, t0, t1, cfg)

    def band(rows, r0):
        import copy
        b = copy.copy(lv[0])
        sl = slice(r0, r0 + rows)
        b.depth, b.V, b.V_valid, b.N, b.N_valid, b.I = (b.depth[sl], b.V[sl], b.V_valid[sl],
                                                         b.N[sl], b.N_valid[sl], b.I[sl])
        return [b] + lv[1:]

    def one(rows, r0):
        Hs, bs, _ = tr.linearise_all(band(rows, r0), 0, x0, x1, t0, t1, Wimu)
        cholesky_solve(Hs, bs)

    t = time.perf_counter()
    one(8, 0)
    per_row = (time.perf_counter() - t) / 8
    rows = int(max(1, min(H, budget_s / max(1, steps + warmup) / per_row)))
    r0 = 0
    for _ in range(warmup):
        one(rows, r0)
        r0 = (r0 + rows) % max(1, H - rows + 1)
    px = 0
    t = time.perf_counter()
    for _ in range(steps):
        one(rows, r0)
        px += rows * W
        r0 = (r0 + rows) % max(1, H - rows + 1)
    el = time.perf_counter() - t
    return px / PIXEL_ITERS_PER_FRAME / el, rows, el


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    seq, frames, imu = make_inputs(4, min(16, os.cpu_count() or 4))
    value, rows, el = oracle_band_steps(seq, frames, imu, args.steps, args.warmup, budget_s=120.0)
    line = {
        "impl": "reference", "metric": "tracked frames/s at 640x480 (batched vs plain)",
        "value": value, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * el / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_json(args),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "impl": "FP64 numpy oracle (vectorised over pixels; not a C++ program)",
                         "sample": f"per step one oracle Gauss-Newton iteration on {rows} level-0 rows "
                                   f"of a 640x480 frame; frames/s = pixel-iterations/s / "
                                   f"{PIXEL_ITERS_PER_FRAME}"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def dtype_of(flags):
    maps = "f16 normal/gradient maps, " if flags & 1 else ""
    red = "f32" if flags & 2 else "f64"
    return f"{maps}f32 per-pixel, {red} reduction, f64 solve"


def config_json(args):
    """The workload of the line, the same for both arms."""
    batch = args.batch
    return {"workload": f"{batch} independent streams of 640x480 RGB-D + 400 Hz IMU per step "
                        f"(one dri_track_batch call), 3 levels 10/5/4 GN iterations; plain: one "
                        f"stream, one frame per step",
            "model": "dense RGB-D-inertial tracking (photometric + ICP + IMU, 34-D joint GN)",
            "global_batch": batch, "seq_len": 1, "parallelism": "replicas (independent streams per GPU)",
            "width": W, "height": H, "levels": LEVELS, "iters": list(ITERS),
            "l2": "inputs larger than L2 (100 distinct frames, 245 MB, cycled; a batched step "
                  f"reads {min(batch, N_UNIQUE)} of them)",
            "imu_mode": args.imu_mode, "occlusion_thr": args.occlusion_thr,
            "precision_flags": args.precision_flags}


def initial_state_at(seq, i):
    """State at loop frame i for a stream whose world frame is that camera frame."""
    from paper_2207_10940_gb300 import synth
    g = seq.gt[i % N_UNIQUE]
    return dict(t=i / FPS, r_WC=np.zeros(3), q_WC=np.array([1.0, 0, 0, 0]), v_I=g["v_I"].copy(),
                bg=np.zeros(3), ba=np.zeros(3), q_IW=synth.matrix_to_quat(g["R_IW"]))


def kernel_classes(prof, dri):
    return {name: {"launches": int(prof.launches[c]), "ms": round(prof.ms[c], 4)}
            for name, c in (("maps", dri.DRI_KC_MAPS), ("track", dri.DRI_KC_TRACK),
                            ("solve", dri.DRI_KC_SOLVE), ("frame", dri.DRI_KC_FRAME),
                            ("grad", dri.DRI_KC_GRAD))}


def bytes_per_pixel_iter(flags):
    """(algorithmic, kernel) bytes per pixel-iteration for the precision flags."""
    if flags & 1:
        return BYTES_PER_PIXEL_ITER_FP16, KERNEL_BYTES_PER_PIXEL_ITER_FP16
    return BYTES_PER_PIXEL_ITER, KERNEL_BYTES_PER_PIXEL_ITER


def roofline(prof, dri, traffic_bpp, n_streams, ms_per_step, flags=0):
    """The pixel kernel against HBM: `frac` from its launches timed one by one
    with CUDA events (the profiled pass: slot groups one after the other), and
    `step_frac` from the timed region (every pixel kernel's bytes of a step over
    the step's time, in which the groups' pixel kernels overlap one another and
    the FP64 steps; a lower bound of the kernel's bandwidth in the timed run)."""
    t_ms = prof.ms[dri.DRI_KC_TRACK]
    px = prof.pixels[dri.DRI_KC_TRACK]
    n = max(1, prof.launches[dri.DRI_KC_TRACK])
    bpp, kbpp = bytes_per_pixel_iter(flags)
    achieved = bpp * px / (t_ms / 1000.0) / 1e9
    step_px = PIXEL_ITERS_PER_FRAME * n_streams
    step_achieved = bpp * step_px / (ms_per_step / 1000.0) / 1e9
    peak, peak_kind = measured_peaks()
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind,
            "kernel": "k_track_batch (fused photometric + ICP linearisation)",
            "bytes_per_pixel_iter": bpp, "avg_launch_us": 1000.0 * t_ms / n,
            "pixel_iters_per_launch": px / n,
            "step_achieved": step_achieved, "step_frac": step_achieved / peak,
            "step_pixel_iters": step_px, "ms_per_step": ms_per_step,
            "kernel_bytes_per_pixel_iter": kbpp, "kernel_bytes_frac": achieved * kbpp / bpp / peak,
            "traffic": None if traffic_bpp is None else traffic_bpp * px / n}


def step_bandwidth(n_streams, ms_per_step, flags=0):
    """The pixel kernels' algorithmic bytes of one timed step over the step's
    time: a lower bound of their bandwidth as they run in the timed region,
    where the slot groups' pixel kernels overlap one another and the FP64
    steps (the roofline's per-launch figure times launches in isolation)."""
    peak, peak_kind = measured_peaks()
    bpp, _ = bytes_per_pixel_iter(flags)
    achieved = bpp * PIXEL_ITERS_PER_FRAME * n_streams / (ms_per_step / 1000.0) / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "bytes_per_pixel_iter": bpp}


class Runner:
    """Streams of the benchmark on one device: frame k of stream i shows loop
    frame (offset_i + k) mod 100 at time (offset_i + k) / 30 s."""

    def __init__(self, seq, imu, d_dev, i_dev, d_pin, i_pin, offsets, dev, tiles=None, groups=None,
                 flags=0, imu_mode=0, track_mode=0, occlusion_thr=0.0):
        import torch
        from paper_2207_10940_gb300 import dri
        self.dri, self.torch = dri, torch
        self.dev = dev
        self.d_dev, self.i_dev, self.d_pin, self.i_pin = d_dev, i_dev, d_pin, i_pin
        self.ts = torch.cuda.Stream(dev)
        cfg = dri_config(seq, flags, imu_mode, track_mode, occlusion_thr)
        self.offsets = list(offsets)
        self.streams = [dri.Stream(cfg, dri.state_from_dict(initial_state_at(seq, o), o / FPS), self.ts)
                        for o in self.offsets]
        arr = dri.imu_array(imu)
        for st in self.streams:
            dri.dri_push_imu(st.handle, arr)
        if tiles or groups:
            dri.dri_batch_set_options([st.handle for st in self.streams], rows_per_thread=tiles,
                                      groups=groups)
        self.k = 0

    def upload(self, device_inputs=True):
        dri = self.dri
        for st, o in zip(self.streams, self.offsets):
            j = (o + self.k) % N_UNIQUE
            t = (o + self.k) / FPS
            if device_inputs:
                dri.dri_upload_frame(st.handle, t, self.d_dev[j], self.i_dev[j], mem_kind=dri.DRI_DEVICE)
            else:
                dri.dri_upload_frame(st.handle, t, self.d_pin[j], self.i_pin[j], mem_kind=dri.DRI_HOST)
        self.k += 1

    def step(self, device_inputs=True, wait=False):
        self.upload(device_inputs)
        if len(self.streams) == 1:
            return self.dri.dri_track(self.streams[0].handle, wait=wait)
        return self.dri.dri_track_batch(self.streams, wait=wait)

    def close(self):
        for st in self.streams:
            st.close()


def max_over_ranks(x, device, world):
    """The largest value of x over the ranks (the job's time is its slowest rank's)."""
    import torch
    if world <= 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job units/s: every rank processes units_per_rank (replicas, weak
    scaling) and the job takes its slowest rank's time."""
    return world * units_per_rank / (ms_max / 1000.0)


MM_COUNTERS = ("pgmigrate_success", "compact_isolated", "compact_migrate_scanned", "compact_stall",
               "thp_collapse_alloc", "numa_hint_faults")


def mm_counters(path="/proc/vmstat"):
    """The host kernel's page-migration and compaction counters (None where the
    file is unreadable)."""
    try:
        with open(path) as f:
            d = dict(line.split() for line in f)
    except OSError:
        return None
    return {k: int(d[k]) for k in MM_COUNTERS if k in d}


def mm_delta(a, b):
    if a is None or b is None:
        return None
    return {k: b[k] - a[k] for k in b if k in a}


def wait_mm_quiet(max_s=20.0, period=0.5):
    """Waits until the host kernel has stopped migrating and compacting pages
    (two consecutive samples `period` apart without a migrated page), at most
    max_s; returns the seconds waited.  Migration unmaps the pages it moves,
    and on this machine the GPU's reads of host memory (pinned frames, copies)
    stalled for tens to hundreds of ms while the kernel compacted the memory
    freed by the frame-rendering processes."""
    t = time.perf_counter()
    prev = mm_counters()
    if prev is None:
        return 0.0
    quiet = 0
    while time.perf_counter() - t < max_s:
        time.sleep(period)
        cur = mm_counters()
        moved = cur.get("pgmigrate_success", 0) - prev.get("pgmigrate_success", 0) + \
            cur.get("compact_isolated", 0) - prev.get("compact_isolated", 0)
        quiet = quiet + 1 if moved == 0 else 0
        prev = cur
        if quiet >= 2:
            break
    return time.perf_counter() - t


def cpu_throttle(root="/sys/fs/cgroup"):
    """The process's CPU-bandwidth throttling counters from its cgroup (v2
    cpu.stat / cpu.max, else v1 cpu/cpu.stat and the CFS quota): throttled
    periods, throttled milliseconds and the quota in CPUs (None: no quota).
    A throttled period stops every thread of the process until it ends."""
    def read(path):
        try:
            with open(path) as f:
                return f.read()
        except OSError:
            return None
    stat, scale, quota = read(os.path.join(root, "cpu.stat")), 1e-3, None
    if stat is not None and "nr_throttled" in stat:
        m = (read(os.path.join(root, "cpu.max")) or "").split()
        if len(m) == 2 and m[0] != "max":
            quota = float(m[0]) / float(m[1])
    else:
        stat, scale = read(os.path.join(root, "cpu", "cpu.stat")), 1e-6
        q, per = read(os.path.join(root, "cpu", "cpu.cfs_quota_us")), read(os.path.join(root, "cpu", "cpu.cfs_period_us"))
        if q and per and int(q) > 0:
            quota = int(q) / int(per)
    if not stat:
        return None
    kv = dict(line.split()[:2] for line in stat.splitlines() if len(line.split()) >= 2)
    t = kv.get("throttled_usec", kv.get("throttled_time", "0"))
    return {"periods": int(kv.get("nr_periods", 0)), "throttled_periods": int(kv.get("nr_throttled", 0)),
            "throttled_ms": float(t) * scale, "quota_cpus": quota}


def throttle_delta(a, b):
    if a is None or b is None:
        return None
    return {"throttled_periods": b["throttled_periods"] - a["throttled_periods"],
            "throttled_ms": b["throttled_ms"] - a["throttled_ms"], "periods": b["periods"] - a["periods"],
            "quota_cpus": b["quota_cpus"]}


class NoCyclicGC:
    """The harness's cyclic garbage collector frozen and off: a full pass over
    the interpreter's heap (torch's objects included) can hold the thread that
    enqueues the steps for tens of milliseconds, longer than the plan's ring of
    launches in flight lets the GPU run ahead."""

    def __enter__(self):
        gc.collect()
        gc.freeze()
        gc.disable()
        return self

    def __exit__(self, *a):
        gc.enable()
        gc.unfreeze()


def timed_pass(run, steps, world, local):
    """Device time of `steps` steps (CUDA events on the library's stream)."""
    torch, dri = run.torch, run.dri
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    h0 = run.streams[0].handle
    n0 = dri.dri_launch_count(h0)
    barrier(run.dev, world)
    thr0 = cpu_throttle()
    with ClockSampler(local) as clk, NoCyclicGC():
        with torch.cuda.stream(run.ts):
            evs[0].record(run.ts)
        for i in range(steps):
            run.step()
            with torch.cuda.stream(run.ts):
                evs[i + 1].record(run.ts)
        barrier(run.dev, world)
    launches = dri.dri_launch_count(h0) - n0
    per = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(steps)])
    total_ms = evs[0].elapsed_time(evs[-1])
    summary = dict(clk.summary(), host_cpu_throttle=throttle_delta(thr0, cpu_throttle()))
    return max_over_ranks(total_ms, run.dev, world), per, launches, summary


def profiled_pass(run, steps):
    dri = run.dri
    h0 = run.streams[0].handle
    dri.dri_profile_enable(h0, True)
    for _ in range(steps):
        run.step()
    prof = dri.dri_profile_read(h0)
    dri.dri_profile_enable(h0, False)
    return prof


def e2e_pass(run, steps, world):
    barrier(run.dev, world)
    with NoCyclicGC():
        t = time.perf_counter()
        for _ in range(steps):
            run.step(device_inputs=False, wait=True)
        barrier(run.dev, world)
        el = time.perf_counter() - t
    h2d = d2h = 0
    for st in run.streams:
        a, b = run.dri.dri_io_bytes(st.handle)
        h2d += a
        d2h += b
    return el, h2d, d2h


def frame_counts(run):
    ok = failed = 0
    for st in run.streams:
        a, b = run.dri.dri_frame_counts(st.handle)
        ok += a
        failed += b
    return ok, failed


def barrier(dev, world):
    import torch
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()


SERVE_STREAMS = 256
SERVE_CLASSES = ((320, 240), (640, 480), (1280, 720))   # stream i: class i mod 3
SERVE_LOOP = 30                                         # frames of each class's looping sequence
SERVE_BUDGET = 120 << 30


def _render_class(args):
    from paper_2207_10940_gb300 import synth
    c, i = args
    seq = _serve_sequence(c, render=False)
    return c, i, synth.render_frame(seq, i, seed=SERVE_SEED + c)


SERVE_SEED = 500


def _serve_sequence(c, render=False):
    from paper_2207_10940_gb300 import synth
    w, h = SERVE_CLASSES[c]
    cam = {320: synth.CAM_320, 640: synth.CAM_640, 1280: synth.CAM_1280}[w]
    return synth.sinusoid_sequence(seed=SERVE_SEED + c, cam=cam, n_frames=SERVE_LOOP, rate=400.0,
                                   period_frames=SERVE_LOOP, render_frames=render)


def tick_summary(trace):
    """Phases of the serving loop's ticks from their host timestamps: staging
    (IMU samples and frame uploads enqueued), launch (the batched frame
    enqueued), GPU (until the worker saw the results) and the gap before the
    next tick; percentiles, and the slowest tick with its phases."""
    if not trace:
        return None
    ph = {"stage": [t.staged_ms - t.dequeue_ms for t in trace],
          "launch": [t.launched_ms - t.staged_ms for t in trace],
          "gpu": [t.done_ms - t.launched_ms for t in trace],
          "device": [t.device_ms for t in trace],
          "tick": [t.done_ms - t.dequeue_ms for t in trace],
          "gap": [b.dequeue_ms - a.done_ms for a, b in zip(trace, trace[1:])] or [0.0]}
    out = {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)),
               "max": float(np.max(v))} for k, v in ph.items()}
    w = max(trace, key=lambda t: t.done_ms - t.dequeue_ms)
    out["slowest"] = {"at_ms": w.dequeue_ms - trace[0].dequeue_ms, "requests": int(w.requests),
                      "stage_ms": w.staged_ms - w.dequeue_ms, "launch_ms": w.launched_ms - w.staged_ms,
                      "gpu_ms": w.done_ms - w.launched_ms, "device_ms": w.device_ms}
    out["ticks"] = len(trace)
    out["ticks_over_50ms"] = int(sum(1 for v in ph["tick"] if v > 50.0))
    return out


def serve_frames(workers):
    """The serving classes' looping sequences (320x240, 640x480, 1280x720) and
    their SERVE_LOOP rendered frames, rendered once for the served, mixed-batch
    and 320x240-pair passes."""
    seqs = [_serve_sequence(c) for c in range(len(SERVE_CLASSES))]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        out = pool.map(_render_class, [(c, i) for c in range(len(SERVE_CLASSES)) for i in range(SERVE_LOOP)])
    frames = [[None] * SERVE_LOOP for _ in SERVE_CLASSES]
    for c, i, f in out:
        frames[c][i] = f
    return seqs, frames


class ClassRunner:
    """Streams of the serving classes tracked with dri_track_batch (or dri_track
    for one stream): stream j of class c starts at loop frame (7 j + 3 c) mod
    SERVE_LOOP; frames come from device memory (timed passes) or pinned host
    memory (end-to-end pass)."""

    def __init__(self, rendered, counts, dev, levels=LEVELS, iters=ITERS, n_frames=400, flags=0):
        import torch
        from paper_2207_10940_gb300 import dri, synth
        self.dri, self.torch, self.dev = dri, torch, dev
        seqs, frames = rendered
        self.D = [torch.stack([torch.from_numpy(f[0]) for f in fc]).to(dev) for fc in frames]
        self.I = [torch.stack([torch.from_numpy(f[1]) for f in fc]).to(dev) for fc in frames]
        self.Dp = [torch.stack([torch.from_numpy(f[0]) for f in fc]).pin_memory() for fc in frames]
        self.Ip = [torch.stack([torch.from_numpy(f[1]) for f in fc]).pin_memory() for fc in frames]
        torch.cuda.synchronize(dev)
        self.ts = torch.cuda.Stream(dev)
        self.streams, self.cls, self.off = [], [], []
        for c, count in enumerate(counts):
            if not count:
                continue
            s = seqs[c]
            cam = s.cam
            cfg = dri.config_for(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels, iters,
                                 q_CS=synth.matrix_to_quat(s.R_CS), r_CS=s.r_CS, precision_flags=flags)
            imu = dri.imu_array(synth.sequence_imu(s, (SERVE_LOOP + n_frames + 2) / FPS, seed=SERVE_SEED + c))
            for j in range(count):
                o = (7 * j + 3 * c) % SERVE_LOOP
                g = s.gt[o]
                x0 = dict(t=o / FPS, r_WC=np.zeros(3), q_WC=np.array([1.0, 0, 0, 0]), v_I=g["v_I"].copy(),
                          bg=np.zeros(3), ba=np.zeros(3), q_IW=synth.matrix_to_quat(g["R_IW"]))
                st = dri.Stream(cfg, dri.state_from_dict(x0, o / FPS), self.ts)
                dri.dri_push_imu(st.handle, imu)
                self.streams.append(st)
                self.cls.append(c)
                self.off.append(o)
        self.k = 0

    def step(self, device_inputs=True, wait=False):
        dri = self.dri
        for st, c, o in zip(self.streams, self.cls, self.off):
            j = o + self.k
            if device_inputs:
                dri.dri_upload_frame(st.handle, j / FPS, self.D[c][j % SERVE_LOOP], self.I[c][j % SERVE_LOOP],
                                     mem_kind=dri.DRI_DEVICE)
            else:
                dri.dri_upload_frame(st.handle, j / FPS, self.Dp[c][j % SERVE_LOOP], self.Ip[c][j % SERVE_LOOP],
                                     mem_kind=dri.DRI_HOST)
        self.k += 1
        if len(self.streams) == 1:
            return dri.dri_track(self.streams[0].handle, wait=wait)
        return dri.dri_track_batch(self.streams, wait=wait)

    def close(self):
        for st in self.streams:
            st.close()


def config_pass(rendered, counts, dev, steps, warmup, world, local, levels=LEVELS, iters=ITERS, flags=0,
                what=""):
    """frames/s of one step = one frame of each stream of `counts` (per serving
    class), the step-level 56 B roofline on its pixel-iterations, and the same
    metric end to end from pinned host frames."""
    n_frames = 1 + warmup + steps + max(3, steps // 4) + 4
    run = ClassRunner(rendered, counts, dev, levels, iters, n_frames, flags)
    run.step(wait=True)
    for _ in range(warmup):
        run.step()
    total_ms, per, launches, clocks = timed_pass(run, steps, world, local)
    ok, failed = frame_counts(run)
    e2e_steps = max(3, steps // 4)
    e2e_s, h2d, d2h = e2e_pass(run, e2e_steps, world)
    n = len(run.streams)
    px = sum(cnt * sum((w >> l) * (h >> l) * iters[l] for l in range(levels))
             for cnt, (w, h) in zip(counts, SERVE_CLASSES))
    peak, peak_kind = measured_peaks()
    bpp, _ = bytes_per_pixel_iter(flags)
    achieved = bpp * px / (total_ms / steps / 1000.0) / 1e9
    run.close()
    return {"workload": what, "streams": n, "value": job_throughput(n * steps, world, total_ms),
            "unit": "frames/s", "steps": steps, "ms_per_step": total_ms / steps,
            "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
            "pixel_iters_per_step": px,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "bytes_per_pixel_iter": bpp,
                         "over": "the whole step (every kernel of the frame)"},
            "e2e": {"value": world * n * e2e_steps / e2e_s, "unit": "frames/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "frames_ok": int(ok), "frames_failed": int(failed), "gpu_launches": int(launches), "clocks": clocks}


def served_pass(args, dev, workers, rendered=None):
    """Serving loop: SERVE_STREAMS streams (resolution by id mod 3), 30 Hz each with
    exponential arrival jitter, for args.serve_seconds of arrivals.  Frames are
    rendered in advance into pinned host memory and each request's frame is
    uploaded by the server (DRI_HOST); one client thread submits on schedule and
    one polls tickets.  Then a saturation run: every stream keeps two requests
    queued (the next is submitted as one completes) for args.saturate_seconds."""
    import threading
    import torch
    from paper_2207_10940_gb300 import dri, synth
    seqs, frames = rendered if rendered is not None else serve_frames(workers)
    D = [torch.stack([torch.from_numpy(f[0]) for f in fc]).pin_memory() for fc in frames]
    I = [torch.stack([torch.from_numpy(f[1]) for f in fc]).pin_memory() for fc in frames]
    secs = float(args.serve_seconds)
    sat_secs = float(args.saturate_seconds)
    n_per = int(secs * FPS)
    n_sat = int(max(sat_secs, 0.0) * FPS * 3) + 4           # frames a stream may use when saturated
    t_end = (SERVE_LOOP + n_per + n_sat + 2) / FPS
    imu = [synth.sequence_imu(s, t_end, seed=SERVE_SEED + c) for c, s in enumerate(seqs)]
    imu_t = [m[:, 0] for m in imu]
    ts = torch.cuda.Stream(dev)
    srv = dri.dri_server_create(SERVE_BUDGET, SERVE_STREAMS, ts)
    rng = np.random.default_rng(SERVE_SEED)
    handles, cls, off = [], [], []
    for i in range(SERVE_STREAMS):
        c = i % len(SERVE_CLASSES)
        o = (7 * i) % SERVE_LOOP
        s = seqs[c]
        cam = s.cam
        cfg = dri.config_for(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, LEVELS, ITERS,
                             q_CS=synth.matrix_to_quat(s.R_CS), r_CS=s.r_CS,
                             precision_flags=args.precision_flags, imu_mode=args.imu_mode,
                             occlusion_thr=args.occlusion_thr)
        g = s.gt[o]
        x0 = dict(t=o / FPS, r_WC=np.zeros(3), q_WC=np.array([1.0, 0, 0, 0]), v_I=g["v_I"].copy(),
                  bg=np.zeros(3), ba=np.zeros(3), q_IW=synth.matrix_to_quat(g["R_IW"]))
        handles.append(dri.dri_server_open_stream(srv, cfg, dri.state_from_dict(x0, o / FPS)))
        cls.append(c)
        off.append(o)
    covering = []   # per class: index of the first sample at or after each frame time
    for c in range(len(SERVE_CLASSES)):
        ft = (np.arange(SERVE_LOOP + n_per + n_sat + 1)) / FPS
        covering.append(np.searchsorted(imu_t[c], ft))
    lib = dri.load_library()
    frame_bytes = [2 * 4 * w * h for w, h in SERVE_CLASSES]

    def request(i, k):
        """Arguments of stream i's frame k (its k-th request): time, pinned host
        images and the IMU samples since its previous frame."""
        c, o = cls[i], off[i]
        j = o + k                                      # global frame index of the class
        lo = 0 if k == 0 else covering[c][j - 1] + 1
        hi = covering[c][j] + 1
        arr = dri.imu_array(imu[c][lo:hi]) if hi > lo else None
        return (handles[i], float(j / FPS), ctypes.c_void_p(D[c][j % SERVE_LOOP].data_ptr()),
                ctypes.c_void_p(I[c][j % SERVE_LOOP].data_ptr()), arr, 0 if arr is None else len(arr))

    # arrival schedule: stream i's frame k at phase_i + k / 30 s + Exp(3 ms) jitter
    phase = rng.uniform(0.0, 1.0 / FPS, SERVE_STREAMS)
    events = []
    for i in range(SERVE_STREAMS):
        jit = np.minimum(rng.exponential(0.003, n_per), 0.02)
        for k in range(n_per):
            events.append((phase[i] + k / FPS + jit[k], i, k))
    events.sort()
    # every request's arguments are built before the run, so the client thread
    # only sleeps and calls the library (no allocation on its path)
    reqs = [(ta,) + request(i, k) for (ta, i, k) in events]
    n_req = len(reqs)
    tickets = [0] * n_req
    statuses = [0] * n_req
    submitted = [0]
    lock = threading.Condition()
    lag = [0.0, 0.0]

    def client():
        tk = ctypes.c_uint64()
        t0 = time.perf_counter() + 0.2
        for idx, (ta, h, t, dp, ip, arr, n) in enumerate(reqs):
            now = time.perf_counter()
            if t0 + ta > now:
                time.sleep(t0 + ta - now)
            elif now - (t0 + ta) > lag[0]:
                lag[0], lag[1] = now - (t0 + ta), ta      # submitted late by the client itself
            code = lib.dri_server_submit(srv, h, t, dp, ip, 0, dri.DRI_HOST, arr, n, ctypes.byref(tk))
            tickets[idx] = tk.value if code == dri.DRI_OK else 0
            statuses[idx] = 0 if code == dri.DRI_OK else code
            with lock:
                submitted[0] = idx + 1
                lock.notify()

    def poller():
        res = dri.dri_track_result()
        for n in range(n_req):
            with lock:
                while n >= submitted[0]:
                    lock.wait()
            if tickets[n]:
                statuses[n] = lib.dri_server_poll(srv, ctypes.c_uint64(tickets[n]), ctypes.byref(res), -1)

    # the host kernel compacts the memory the rendering processes freed: let it
    # finish before the offered load starts (bounded; the wait is reported)
    quiet_s = wait_mm_quiet()
    th = [threading.Thread(target=client), threading.Thread(target=poller)]
    # the client and poller are Python threads: a pass of the cyclic garbage
    # collector over the bench's objects can hold them for hundreds of ms and
    # release a burst of requests at once, a stall of the harness, not of the
    # server; the collector is frozen and off while requests are offered
    gc.collect()
    gc.freeze()
    gc.disable()
    t_start = time.perf_counter()
    for t in th:
        t.start()
    # latency after the warm-up: 2 s, and until the backlog of the start (plan
    # building, pinned buffers, graph instantiation, tuning on the first tracked
    # frames) is drained to at most one request per stream, within half the run
    t_w = time.perf_counter()
    time.sleep(min(2.0, secs / 4))
    while time.perf_counter() - t_w < secs / 2:
        st = dri.dri_server_stats_read(srv)
        if st.submitted - st.completed <= SERVE_STREAMS:
            break
        time.sleep(0.05)
    warm_s = time.perf_counter() - t_w
    dri.dri_server_stats_read(srv, reset=True)
    thr0 = cpu_throttle()
    mm0 = mm_counters()
    mon = ServeMonitor(dev.index if dev.index is not None else 0)
    with mon:
        t0_wall = time.time()
        for t in th:
            t.join()
        t1_wall = time.time()
    thr = throttle_delta(thr0, cpu_throttle())
    mm = mm_delta(mm0, mm_counters())
    wall = time.perf_counter() - t_start
    trace = dri.dri_server_trace_read(srv)             # read before the reset clears it
    st = dri.dri_server_stats_read(srv, reset=True)
    ticks = tick_summary(trace)
    # wall time of each tick over 50 ms (the trace's first tick is the first
    # after the stats reset, t0_wall)
    stalls = [] if not trace else [
        (t0_wall + (t.dequeue_ms - trace[0].dequeue_ms) / 1e3, t.done_ms - t.dequeue_ms)
        for t in trace if t.done_ms - t.dequeue_ms > 50.0]
    bad = sum(1 for s in statuses if s != 0)
    served = {
        "streams": SERVE_STREAMS, "mix": "stream i: " + ", ".join(f"{w}x{h}" for w, h in SERVE_CLASSES)
        + " by i mod 3", "rate_hz_per_stream": FPS, "arrival_jitter": "exponential, mean 3 ms",
        "seconds": secs, "offered_frames_per_s": SERVE_STREAMS * FPS,
        "requests": len(events), "wall_s": wall, "value": st.frames_per_s, "unit": "frames/s",
        "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "max_ms": st.max_ms, "failed": int(bad),
        "mean_batch": st.mean_batch, "ticks": int(st.ticks), "hbm_used_gb": st.hbm_used / 1e9,
        "hbm_budget_gb": SERVE_BUDGET / 1e9,
        "inputs": "frames rendered in advance into pinned host memory (30-frame loops per resolution, "
                  "period-30 sinusoid), uploaded per request by the server (DRI_HOST); IMU copied per "
                  "request",
        "h2d_bytes_per_s": st.frames_per_s * float(np.mean(frame_bytes)),
        "warmup_s": warm_s, "client_max_lag_ms": 1000.0 * lag[0], "client_max_lag_at_s": lag[1],
        "host_cpu_throttle": thr, "host_mm_counters": mm, "mm_quiet_wait_s": quiet_s,
        "tick_phases_ms": ticks,
        "monitor": mon.summary(t0_wall, t1_wall, stalls),
        "latency_from": "submit to result (warm-up excluded: 2 s and until the start's backlog is "
                        "drained)"}

    # saturation: each stream keeps two requests queued; the poller submits a
    # stream's next frame when one of its requests completes
    if sat_secs > 0:
        from collections import deque
        nxt = [n_per] * SERVE_STREAMS                  # next frame index per stream
        fifo = deque()
        tk = ctypes.c_uint64()
        res = dri.dri_track_result()
        sat_bad = [0]

        def submit(i):
            h, t, dp, ip, arr, n = request(i, nxt[i])
            nxt[i] += 1
            code = lib.dri_server_submit(srv, h, t, dp, ip, 0, dri.DRI_HOST, arr, n, ctypes.byref(tk))
            if code == dri.DRI_OK:
                fifo.append((tk.value, i))
            else:
                sat_bad[0] += 1

        t_s = time.perf_counter()
        for _ in range(2):
            for i in range(SERVE_STREAMS):
                submit(i)
        while fifo:
            ticket, i = fifo.popleft()
            if lib.dri_server_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(res), -1) != dri.DRI_OK:
                sat_bad[0] += 1
            if time.perf_counter() - t_s < sat_secs:
                submit(i)
        sat_wall = time.perf_counter() - t_s
        sat_trace = dri.dri_server_trace_read(srv)
        st2 = dri.dri_server_stats_read(srv)
        served["saturation"] = {
            "seconds": sat_wall, "queued_per_stream": 2, "value": st2.frames_per_s, "unit": "frames/s",
            "completed": int(st2.completed), "failed": int(sat_bad[0]), "p50_ms": st2.p50_ms,
            "p99_ms": st2.p99_ms, "mean_batch": st2.mean_batch, "ticks": int(st2.ticks),
            "tick_phases_ms": tick_summary(sat_trace),
            "note": "latency here includes the queueing of two requests per stream"}
    gc.enable()
    gc.unfreeze()
    dri.dri_server_destroy(srv)
    return served


PRECISION_VARIANTS = (("fp32_pixel_fp64_partials", 0), ("fp32_pixel_fp32_partials", 2),
                      ("fp16_maps_fp64_partials", 1), ("fp16_maps_fp32_partials", 3))


def _norm_errors(H_g, b_g, H_o, b_o, cost):
    """max |dH_ij| / sqrt(H_ii H_jj) and max |db_i| / sqrt(H_ii C) (the parity
    tolerance's normalisation, bar 1e-5)."""
    H_g, b_g, H_o, b_o = (np.asarray(a, dtype=np.float64) for a in (H_g, b_g, H_o, b_o))
    d = np.sqrt(np.maximum(np.diag(H_o), 1e-300))
    eh = float(np.max(np.abs(H_g - H_o) / np.outer(d, d)))
    eb = float(np.max(np.abs(b_g - b_o) / (d * np.sqrt(max(cost, 1e-300)))))
    return eh, eb


def precision_study(seq, frames, imu, dev, n_frames):
    """Each precision variant against the exact FP64 oracle on the 640x480
    sequence: the level-0 systems of frame 1 against frame 0 at the ground-truth
    states, and the pose after tracking frames 0 .. n_frames - 1."""
    import torch
    from oracle import gn, imu as imu_mod, maps
    from oracle.params import TrackerConfig
    from oracle.so3 import State, log_so3
    from paper_2207_10940_gb300 import dri, synth
    cam = seq.cam
    ocfg = TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=LEVELS,
                         iters=ITERS, R_CS=seq.R_CS, r_CS=seq.r_CS)
    x_init = synth.initial_state(seq)
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(imu)
    tr.track(frames[0][0], frames[0][1], 0.0)
    x0, x1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    lv = maps.frame_levels(frames[1][0], frames[1][1], ocfg)
    W, _ = imu_mod.weight(x0, tr.imu, 0.0, 1.0 / FPS, ocfg)
    H_o, b_o, parts = tr.linearise_all(lv, 0, x0, x1, 0.0, 1.0 / FPS, W)
    lin = parts["lin"]
    t = time.perf_counter()
    for i in range(1, n_frames):
        x_o = tr.track(frames[i][0], frames[i][1], i / FPS)["x1"]
    t_oracle = time.perf_counter() - t
    out = {"workload": f"640x480 sinusoid sequence, frames 0-{n_frames - 1}; systems: level 0 of "
                       f"frame 1 against frame 0 at the ground-truth states",
           "oracle": "exact FP64 (maps not rounded)", "solve": "FP64 on the GPU in every variant",
           "normalisation": "max |dH_ij|/sqrt(H_ii H_jj), max |db_i|/sqrt(H_ii C); bar 1e-5",
           "parity_bars": {
               "fp32 maps (flags 0, 2)": "systems 1e-5 normalised, pose 1e-6 rad / 1e-6 m, against "
                                         "the FP64 oracle (tests)",
               "fp16 maps (flags 1, 3)": "systems 2^-11 normalised, pose 1e-5 rad / 1e-5 m (10x the "
                                         "FP32 pose bar), against an oracle that rounds the stored "
                                         "normals and gradients to FP16 as the library does (tests); "
                                         "FP32- and FP64-computed normals can round to neighbouring "
                                         "half-precision values"},
           "oracle_track_s": t_oracle, "variants": {}}
    for name, flags in PRECISION_VARIANTS:
        cfg = dri_config(seq, flags)
        st = dri.Stream(cfg, dri.state_from_dict(x_init), torch.cuda.Stream(dev))
        dri.dri_push_imu(st.handle, imu)
        dri.dri_upload_frame(st.handle, 0.0, frames[0][0], frames[0][1])
        dri.dri_track(st.handle)
        dri.dri_upload_frame(st.handle, 1.0 / FPS, frames[1][0], frames[1][1])
        g, _ = dri.dri_linearise(st.handle, 0, dri.state_from_dict(x0.to_dict()),
                                 dri.state_from_dict(x1.to_dict()))
        e_icp = _norm_errors(np.array(g.H_icp).reshape(6, 6), g.b_icp, lin["H_icp"], lin["b_icp"],
                             lin["cost_icp"])
        e_rgb = _norm_errors(np.array(g.H_rgb).reshape(6, 6), g.b_rgb, lin["H_rgb"][6:, 6:],
                             lin["b_rgb"][6:], lin["cost_rgb"])
        e_joint = _norm_errors(np.array(g.H).reshape(34, 34), g.b, H_o, b_o,
                               lin["cost_icp"] + lin["cost_rgb"] + parts["cost_imu"])
        for i in range(1, n_frames):
            dri.dri_upload_frame(st.handle, i / FPS, frames[i][0], frames[i][1])
            r = dri.dri_track(st.handle)
        xg = State.from_dict(dri.state_to_dict(r.x1))
        out["variants"][name] = {
            "flags": flags, "H_icp": e_icp[0], "b_icp": e_icp[1], "H_rgb": e_rgb[0], "b_rgb": e_rgb[1],
            "H_joint": e_joint[0], "b_joint": e_joint[1],
            "n_icp": int(g.n_icp), "n_icp_oracle": int(lin["n_icp"]),
            "n_rgb": int(g.n_rgb), "n_rgb_oracle": int(lin["n_rgb"]),
            "pose_err_rad": float(np.linalg.norm(log_so3(xg.R @ x_o.R.T))),
            "pose_err_m": float(np.linalg.norm(xg.r - x_o.r)), "status": int(r.status)}
        st.close()
    return out


def run_ours(args):
    rank, local, world = dist_env()
    plain_steps = args.plain_steps
    n_frames = max(BATCH_OFFSET * (BATCH - 1) % N_UNIQUE, N_UNIQUE) + 2 * (
        args.warmup + 2 * max(args.steps, plain_steps) + args.profile_frames + 8)
    seq, frames, imu = make_inputs(n_frames, min(16, os.cpu_count() or 4))
    import torch
    from paper_2207_10940_gb300 import build, dri
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    d_dev = torch.stack([torch.from_numpy(f[0]) for f in frames]).to(dev)
    i_dev = torch.stack([torch.from_numpy(f[1]) for f in frames]).to(dev)
    d_pin = torch.stack([torch.from_numpy(f[0]) for f in frames]).pin_memory()
    i_pin = torch.stack([torch.from_numpy(f[1]) for f in frames]).pin_memory()
    torch.cuda.synchronize(dev)      # the library reads these on its own stream
    out = {}
    passes = [("batched", args.batch, args.steps)]
    if plain_steps > 0:
        passes.append(("plain", 1, plain_steps))
    for mode, n_streams, steps in passes:
        offsets = [(BATCH_OFFSET * i) % N_UNIQUE for i in range(n_streams)]
        run = Runner(seq, imu, d_dev, i_dev, d_pin, i_pin, offsets, dev,
                     args.rows_per_thread if n_streams > 1 else None,
                     args.groups if n_streams > 1 else None, args.precision_flags, args.imu_mode, 0,
                     args.occlusion_thr)
        res = run.step(wait=True)
        for _ in range(args.warmup):
            run.step()
        total_ms, per, launches, clocks = timed_pass(run, steps, world, local)
        ok, failed = frame_counts(run)
        prof = profiled_pass(run, max(3, args.profile_frames // (8 if n_streams > 1 else 1)))
        e2e_steps = max(3, steps // 4)
        e2e_s, h2d, d2h = e2e_pass(run, e2e_steps, world)
        opts = dri.dri_batch_get_options([s.handle for s in run.streams])
        tiles = list(opts.rows_per_thread)
        out[mode] = {
            "value": job_throughput(n_streams * steps, world, total_ms), "steps": steps,
            "streams": n_streams, "ms_per_step": total_ms / steps,
            "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
            "slowest_steps": [[int(k), float(per[k])] for k in np.argsort(per)[::-1][:5]],
            "gpu_launches": int(launches), "frames_ok": int(ok), "frames_failed": int(failed),
            "roofline": roofline(prof, dri, track_traffic(), n_streams, total_ms / steps,
                                 args.precision_flags),
            "kernel_classes": kernel_classes(prof, dri),
            "e2e": {"value": world * n_streams * e2e_steps / e2e_s, "unit": "frames/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "clocks": clocks, "rows_per_thread": tiles[:LEVELS], "groups": opts.groups,
            "step_bandwidth": step_bandwidth(n_streams, total_ms / steps, args.precision_flags),
        }
        run.close()
        del run
        torch.cuda.synchronize(dev)
    odo_states = odo_rgbd = odo_occ = odo_gyro = None
    n_odo = min(args.odometry_frames, n_frames - 2)
    if n_odo > 1 and rank == 0:
        odo_states = odometry_pass(seq, imu, d_dev, i_dev, d_pin, i_pin, dev, n_odo, args.precision_flags,
                                   args.imu_mode, occlusion_thr=args.occlusion_thr)
        # the vision-only, pose-only baseline the paper compares with (same frames)
        odo_rgbd = odometry_pass(seq, imu, d_dev, i_dev, d_pin, i_pin, dev, n_odo, args.precision_flags,
                                 args.imu_mode, track_mode=1, occlusion_thr=args.occlusion_thr)
        # the gyroscope-only setup (accelerometer residuals ignored), between the two
        odo_gyro = odometry_pass(seq, imu, d_dev, i_dev, d_pin, i_pin, dev, n_odo, args.precision_flags,
                                 args.imu_mode, track_mode=2, occlusion_thr=args.occlusion_thr)
        # the joint tracker with the occlusion test (when the timed passes run without it)
        if args.occlusion_thr <= 0:
            odo_occ = odometry_pass(seq, imu, d_dev, i_dev, d_pin, i_pin, dev, n_odo, args.precision_flags,
                                    args.imu_mode, occlusion_thr=ODOMETRY_OCCLUSION_THR)
        torch.cuda.synchronize(dev)
    rendered = None
    if args.serve_seconds > 0 or args.config_steps > 0:
        rendered = serve_frames(min(16, os.cpu_count() or 4))
    mixed = pair320 = None
    if args.config_steps > 0:
        # the mixed batch of uneven sizes: 24 x 320x240, 32 x 640x480, 8 x 1280x720
        mixed = config_pass(rendered, (24, 32, 8), dev, args.config_steps, args.warmup, world, local,
                            flags=args.precision_flags,
                            what="24 x 320x240 + 32 x 640x480 + 8 x 1280x720 streams per step (one "
                                 "dri_track_batch call), 3 levels 10/5/4")
        # the 320x240 pair workload: one stream, 2 levels 10/5, one frame per step
        pair320 = config_pass(rendered, (1, 0, 0), dev, args.config_steps * 4, args.warmup, world, local,
                              levels=2, iters=(10, 5), flags=args.precision_flags,
                              what="one 320x240 stream, 2 levels 10/5 (dri_track), one frame per step")
        torch.cuda.synchronize(dev)
    served = None
    if args.serve_seconds > 0:
        served = served_pass(args, dev, min(16, os.cpu_count() or 4), rendered)
    precision = None
    if args.precision_frames > 1 and rank == 0:
        precision = precision_study(seq, frames, imu, dev, args.precision_frames)
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    budget = float(os.environ.get("DRI_BENCH_ORACLE_SECONDS", "15"))
    o_fps, o_n, o_t, o_states = oracle_frames_per_s(seq, frames, imu, budget)
    n_cores = os.cpu_count() or 1
    a_fps, a_t, a_rows = oracle_all_cores(frames, imu, min(budget, 10.0), n_cores)
    b, p = out["batched"], out.get("plain")
    line = {
        "metric": "tracked frames/s at 640x480 (batched vs plain)",
        "value": b["value"], "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(args.precision_flags),
        "data": "synthetic", "config": config_json(args),
        "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"], "slowest_steps": b["slowest_steps"],
        "gpu_launches": b["gpu_launches"],
        "frames_failed": b["frames_failed"], "frames_ok": b["frames_ok"],
        "roofline": b["roofline"], "step_bandwidth": b["step_bandwidth"],
        "kernel_classes": b["kernel_classes"], "e2e": b["e2e"],
        "rows_per_thread": b["rows_per_thread"], "groups": b["groups"],
        "plain": None if p is None else {
            k: p[k] for k in ("value", "steps", "ms_per_step", "p50_ms", "p99_ms", "gpu_launches",
                              "frames_ok", "frames_failed", "roofline", "kernel_classes", "e2e",
                              "rows_per_thread")},
        "batched_over_plain": None if p is None else b["value"] / p["value"],
        "mixed_batch": mixed, "pair_320x240": pair320,
        "odometry": None if odo_states is None else odometry_report(seq, odo_states, o_states),
        "odometry_rgbd_only": None if odo_rgbd is None else rgbd_only_report(seq, odo_rgbd),
        "odometry_gyro_only": None if odo_gyro is None else rgbd_only_report(seq, odo_gyro),
        "odometry_occlusion": None if odo_occ is None else dict(
            rgbd_only_report(seq, odo_occ), occlusion_thr_m=ODOMETRY_OCCLUSION_THR),
        "precision": precision,
        "cpu_baseline": {"value": o_fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "impl": "FP64 numpy oracle (vectorised over pixels; not a C++ program)",
                         "sample": f"{o_n} whole frames of the same sequence tracked by the FP64 "
                                   f"numpy oracle in {o_t:.1f} s"},
        "cpu_baseline_all_cores": {"value": a_fps, "unit": "frames/s", "cores": n_cores, "kind": "oracle",
                                   "sample": f"{n_cores} processes, each repeating the oracle's linearisation "
                                             f"of all terms on its own {a_rows} level-0 rows of frame 1 for "
                                             f"{a_t:.1f} s; frames/s = pixel-iterations / wall time / "
                                             f"{PIXEL_ITERS_PER_FRAME}"},
        "clocks": b["clocks"], "clocks_plain": None if p is None else p["clocks"],
        # last, so that the end of the line (which logs keep) shows the serving results
        "served": served,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--plain-steps", type=int, default=600,
                    help="frames of the plain single-stream pass (0: skip it)")
    ap.add_argument("--batch", type=int, default=BATCH, help="streams of the batched pass")
    ap.add_argument("--precision-frames", type=int, default=3,
                    help="frames of the precision study against the FP64 oracle (< 2: skip it)")
    ap.add_argument("--serve-seconds", type=float, default=30.0,
                    help="seconds of arrivals in the serving pass (0: skip it)")
    ap.add_argument("--saturate-seconds", type=float, default=10.0,
                    help="seconds of the serving saturation run after it (0: skip it)")
    ap.add_argument("--config-steps", type=int, default=40,
                    help="timed steps of the mixed-size batch and of the 320x240 pair stream (0: skip)")
    ap.add_argument("--rows-per-thread", type=lambda v: [int(x) for x in v.split(",")], default=None,
                    help="pixel-kernel rows per thread per level for the batched pass, e.g. 8,8,8 "
                         "(default: the plan's autotuner)")
    ap.add_argument("--groups", type=int, default=None,
                    help="slot groups of the batched Gauss-Newton loop (default: the library's)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--imu-mode", type=int, default=0, choices=(0, 1),
                    help="IMU term per Gauss-Newton iteration of the timed streams: 0 re-integrate "
                         "(default), 1 first-order bias update (DRI_IMU_FIRST_ORDER)")
    ap.add_argument("--occlusion-thr", type=float, default=0.0,
                    help="photometric occlusion test of the timed streams, m (default 0: off)")
    ap.add_argument("--precision-flags", type=int, default=0,
                    help="precision_flags of the timed streams: 1 FP16 maps, 2 FP32 partials, 3 both "
                         "(default 0: FP32 maps, FP64 partials)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--profile-frames", type=int, default=60)
    ap.add_argument("--odometry-frames", type=int, default=300,
                    help="frames of the odometry pass against ground truth (< 2: skip it)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
