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
