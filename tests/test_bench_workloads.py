"""The benchmark's synthetic workloads have the shapes the growth plan states
(host logic only, no GPU)."""
import math

import numpy as np

import bench


def test_scan_runs_follow_the_stated_distributions():
    descs = [bench.scan_desc(i) for i in range(256)]
    assert bench.scan_steps(40) == 21053  # 40 periods at lambda/500, dt = 0.95 dx
    a0 = np.array([d["a0"] for d in descs])
    th = np.array([d["foil_thickness"] for d in descs])
    ne = np.array([d["ne"] for d in descs])
    ppc = np.array([d["ppc"] for d in descs])
    assert a0.min() >= 100 and a0.max() <= 600 and th.min() >= 0.5 and th.max() <= 2.0
    assert ne.min() >= 30 and ne.max() <= 150 and ppc.min() >= 32 and ppc.max() <= 256
    for key in ("polarization", "rr_on"):
        frac = np.mean([bool(d[key]) for d in descs])
        assert 0.35 < frac < 0.65  # 50/50
    n = np.array([bench.desc_particles(d, 500) // 2 for d in descs])
    assert 5_000 <= n.min() and n.max() <= 256_000  # about 5k..250k per species
    assert all(d["length_lambda"] == 30.0 and d["foil_x0"] == 10.0 for d in descs)
    assert len({d["seed"] for d in descs}) == 256
    # deterministic
    assert bench.scan_desc(17) == bench.scan_desc(17)


def test_request_stream_is_poisson_with_log_uniform_sizes():
    reqs = bench.serve_requests(20.0, 100.0, seed=5)
    t = np.array([r[0] for r in reqs])
    assert abs(len(reqs) - 2000) < 4 * math.sqrt(2000)  # Poisson count at 20/s over 100 s
    gaps = np.diff(t)
    assert abs(gaps.mean() - 0.05) < 0.005 and abs(gaps.std() / gaps.mean() - 1.0) < 0.1  # exponential gaps
    n = np.array([bench.desc_particles(d, 500) / 2 for _, d in reqs])
    assert n.min() > 0.7e4 and n.max() < 1.3e6
    logn = np.log10(n)
    assert abs(np.mean(logn) - 5.0) < 0.1  # log-uniform on [1e4, 1e6]
    periods = np.array([d["steps"] for _, d in reqs]) * 0.95 / 500
    assert periods.min() >= 20.0 - 1e-9 and periods.max() <= 200.0 + 0.01


def test_clock_samples_are_kept_only_inside_the_timed_region(tmp_path):
    import datetime

    c = bench.Clocks.__new__(bench.Clocks)  # no sampler process: feed a recorded trace
    rows = ["2026/12/03 03:12:55.000, 1400, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "2026/12/03 03:12:55.100, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "2026/12/03 03:12:55.150, 2070, 2070, 1250.0, 0x4, Not Active, Not Active, Not Active, Active",
            "2026/12/03 03:12:55.400, 1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    f = open(tmp_path / "clk.csv", "w+")
    f.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.f, c.p = f, Done()
    c.t0 = datetime.datetime(2026, 12, 3, 3, 12, 55, 50000)
    c.t1 = datetime.datetime(2026, 12, 3, 3, 12, 55, 300000)
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}


def test_both_arms_name_the_same_workload_and_traffic_is_keyed_by_shapes():
    assert "8000 ppc/species (32M e + 32M p)" in bench.large_workload()
    assert "1000 ppc/species (4M e + 4M p)" in bench.large_workload(1000)
    # measured DRAM bytes of one push launch stay close to the 40 B per particle-step the roofline counts
    # (below it by at most the 4 B cell slot a warp whose particles all stayed in their cells does not
    # rewrite, and by writes still in L2 when the kernel ends), and an entry applies only to the push
    # kernel it was measured on
    assert any(k[5] == bench.push_kernel_digest() for k in bench.PUSH_TRAFFIC)
    for (n, unit, interval, w, hot, digest), b in bench.PUSH_TRAFFIC.items():
        assert n == 64_000_000 and w in (2, 4) and 1 <= interval <= 96 and unit in (2048, 4096, 8192, 16384)
        assert hot is True and len(digest) == 12
        assert 0.8 < b / (bench.BYTES_PER_PARTICLE_STEP * n) < 1.05


def test_timed_window_follows_the_pulse():
    """The large run's timed window starts after the pulse front reached the foil
    and after the tuner's 840 trial steps; both arms name the same window."""
    assert bench.PULSE_AT_FOIL_STEP == 518
    assert bench.RUN_STEPS == 2000
    assert bench.TUNER_STEPS == 840
    assert bench.window_start(20, 5, 600) == 1980 and bench.window_start(384, 8, 600) == 1616
    assert bench.window_start(1500, 5, 600) == 600 + 840 + 5
    assert "timed steps 1980..1999" in bench.workload_with_window(1980, 20)
    assert bench.SCAN["shapes"] == (8192, 96, 2) and bench.SERVE["sort_interval"] == 64


class _FakeSim:
    """Steps, sorts and timing counters as the library keeps them (a sort after
    every `interval` steps; with timing on, fixed per-kernel times)."""

    def __init__(self, steps, interval, push=0.4, field=0.01, sort=0.7):
        self.steps, self.interval, self.timing = steps, interval, False
        self.push, self.field, self.sort = push, field, sort
        self.sorts = steps // interval
        self.c = dict(push_ms=0.0, field_ms=0.0, sort_ms=0.0, timed_push_launches=0)

    def set_timing(self, on):
        self.timing = bool(on)
        if on:
            self.c = dict(push_ms=0.0, field_ms=0.0, sort_ms=0.0, timed_push_launches=0)

    def step(self, n):
        for _ in range(n):
            self.steps += 1
            if self.timing:
                self.c["push_ms"] += self.push
                self.c["field_ms"] += self.field
                self.c["timed_push_launches"] += 1
            if self.steps % self.interval == 0:
                self.sorts += 1
                if self.timing:
                    self.c["sort_ms"] += self.sort

    def stats(self):
        return dict(self.c, steps=self.steps, sort_count=self.sorts, steps_since_sort=self.steps % self.interval)


def test_kernel_times_cover_whole_sort_intervals_after_the_window():
    s = _FakeSim(2000, 96)
    kt = bench.kernel_times(s, 96)
    assert (kt["first_step"], kt["last_step"]) == (2016, 2207)  # to the next sort, then two whole intervals
    assert abs(kt["push_ms"] - 0.4) < 1e-12 and abs(kt["field_ms_per_step"] - 0.01) < 1e-12
    assert abs(kt["sort_ms_mean"] - 0.7) < 1e-12
    assert abs(kt["steps_per_step_ms"] - (0.41 + 0.7 / 96)) < 1e-12
    assert not s.timing  # the window's step graphs hold no event nodes afterwards
    s = _FakeSim(1920, 64)  # already on a sort boundary
    assert bench.kernel_times(s, 64)["first_step"] == 1920
