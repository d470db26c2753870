"""Host-side helpers of the benchmark (no GPU): cgroup CPU-throttling counters
in both cgroup layouts, the step-bandwidth and throughput arithmetic."""
import os

import bench


def _write(path, text):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        f.write(text)


def test_cpu_throttle_cgroup_v2(tmp_path):
    root = str(tmp_path)
    _write(os.path.join(root, "cpu.stat"), "usage_usec 5\nnr_periods 40\nnr_throttled 3\nthrottled_usec 2500\n")
    _write(os.path.join(root, "cpu.max"), "400000 100000\n")
    a = bench.cpu_throttle(root)
    assert a == {"periods": 40, "throttled_periods": 3, "throttled_ms": 2.5, "quota_cpus": 4.0}
    _write(os.path.join(root, "cpu.stat"), "nr_periods 50\nnr_throttled 7\nthrottled_usec 12500\n")
    d = bench.throttle_delta(a, bench.cpu_throttle(root))
    assert d == {"throttled_periods": 4, "throttled_ms": 10.0, "periods": 10, "quota_cpus": 4.0}
    _write(os.path.join(root, "cpu.max"), "max 100000\n")
    assert bench.cpu_throttle(root)["quota_cpus"] is None


def test_cpu_throttle_cgroup_v1(tmp_path):
    root = str(tmp_path)
    _write(os.path.join(root, "cpu", "cpu.stat"), "nr_periods 9\nnr_throttled 2\nthrottled_time 3000000\n")
    _write(os.path.join(root, "cpu", "cpu.cfs_quota_us"), "-1\n")
    _write(os.path.join(root, "cpu", "cpu.cfs_period_us"), "100000\n")
    assert bench.cpu_throttle(root) == {"periods": 9, "throttled_periods": 2, "throttled_ms": 3.0,
                                        "quota_cpus": None}
    _write(os.path.join(root, "cpu", "cpu.cfs_quota_us"), "250000\n")
    assert bench.cpu_throttle(root)["quota_cpus"] == 2.5


def test_cpu_throttle_without_cgroup(tmp_path):
    assert bench.cpu_throttle(str(tmp_path)) is None
    assert bench.throttle_delta(None, None) is None


def test_step_bandwidth_and_throughput():
    sb = bench.step_bandwidth(64, 5.0)
    want = bench.BYTES_PER_PIXEL_ITER * bench.PIXEL_ITERS_PER_FRAME * 64 / 5e-3 / 1e9
    assert abs(sb["achieved"] - want) <= 1e-9 * want
    assert abs(sb["frac"] - sb["achieved"] / sb["peak"]) <= 1e-12
    # 640x480, 3 levels, 10/5/4 iterations
    assert bench.PIXEL_ITERS_PER_FRAME == 307200 * 10 + 76800 * 5 + 19200 * 4
    # whole-job units/s: every rank does units_per_rank in the slowest rank's time
    assert bench.job_throughput(200 * 64, 4, 1000.0) == 4 * 200 * 64


def test_tick_summary_phases():
    class T:
        def __init__(self, i, d, s, l, e, n=4):
            self.tick, self.requests, self.status = i, n, 0
            self.dequeue_ms, self.staged_ms, self.launched_ms, self.done_ms = d, s, l, e
            self.device_ms = e - l
    tr = [T(0, 0.0, 0.5, 1.0, 11.0), T(1, 11.2, 11.4, 12.0, 80.0, n=9), T(2, 80.1, 80.3, 80.9, 91.0)]
    s = bench.tick_summary(tr)
    assert s["ticks"] == 3 and s["ticks_over_50ms"] == 1
    assert abs(s["gpu"]["max"] - 68.0) < 1e-9 and abs(s["stage"]["max"] - 0.5) < 1e-9
    assert abs(s["gap"]["max"] - 0.2) < 1e-9
    assert s["slowest"]["requests"] == 9 and abs(s["slowest"]["at_ms"] - 11.2) < 1e-9
    assert bench.tick_summary([]) is None


def test_mm_counters_and_quiet_wait(tmp_path, monkeypatch):
    p = str(tmp_path / "vmstat")
    _write(p, "nr_free_pages 10\npgmigrate_success 7\ncompact_isolated 3\ncompact_stall 0\n")
    a = bench.mm_counters(p)
    assert a == {"pgmigrate_success": 7, "compact_isolated": 3, "compact_stall": 0}
    _write(p, "nr_free_pages 9\npgmigrate_success 19\ncompact_isolated 5\ncompact_stall 1\n")
    assert bench.mm_delta(a, bench.mm_counters(p)) == {"pgmigrate_success": 12, "compact_isolated": 2,
                                                       "compact_stall": 1}
    assert bench.mm_counters(str(tmp_path / "missing")) is None
    assert bench.mm_delta(None, a) is None
    # the wait ends after two quiet samples, or at its bound while pages keep moving
    seq = iter([{"pgmigrate_success": n, "compact_isolated": 0} for n in (0, 5, 9, 9, 9, 9)])
    monkeypatch.setattr(bench, "mm_counters", lambda path="/proc/vmstat": next(seq))
    waited = bench.wait_mm_quiet(max_s=5.0, period=0.01)
    assert 0.03 <= waited < 1.0
    moving = iter({"pgmigrate_success": n, "compact_isolated": 0} for n in range(10 ** 6))
    monkeypatch.setattr(bench, "mm_counters", lambda path="/proc/vmstat": next(moving))
    assert 0.1 <= bench.wait_mm_quiet(max_s=0.1, period=0.01) < 0.5


def test_serve_monitor_summary(tmp_path, monkeypatch):
    import datetime
    monkeypatch.setenv("DRI_CLOCKS_DIR", str(tmp_path))
    m = bench.ServeMonitor(0)
    t = datetime.datetime(2026, 1, 2, 3, 4, 5, 100000).timestamp()
    _write(m.paths[0], "2026/01/02 03:04:05.100, 2070, 2070, Not Active, Not Active, Not Active, Not Active\n"
                       "2026/01/02 03:04:05.200, 1500, 2070, Active, Not Active, Not Active, Not Active\n"
                       "2026/01/02 03:04:09.000, 2070, 2070, Not Active, Not Active, Not Active, Not Active\n")
    _write(m.paths[1], "4321, 500\n1234, 900\n")
    out = m.summary(t - 0.05, t + 1.0, [(t + 0.21, 80.0)])
    assert out["clock_samples"] == 2                    # the third sample is after the pass
    assert out["sm_mhz_min"] == 1500.0 and out["samples_below_95pct"] == 1
    assert out["reasons"] == ["hw_slowdown"]
    assert out["compute_pids"] == [1234, 4321]
    (st,) = out["stalled_ticks"]
    assert st["sm_mhz"] == 1500.0 and st["reasons"] == ["hw_slowdown"] and abs(st["sample_dt_s"] + 0.11) < 1e-3
