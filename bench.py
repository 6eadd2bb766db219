"""Benchmark of the 1D laser-foil PIC step (fused gather + Boris + LL
radiation-reaction kick + charge-conserving deposit, Yee update with laser
injection, periodic cell sort) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload (N = 1): the large single run that saturates HBM — 100 wavelengths
at 2000 cells per wavelength (200,000 cells), a 2-wavelength hydrogen foil
at 0.25 wavelengths with n_e = 100 n_c and 8000 macro-particles per cell per
species (32M electrons + 32M protons), CP laser a0 = 500 with a 20-period
sin^2 envelope, radiation reaction on, dt = 0.95 dx.  Synthetic, seeded.
With N > 1 (torchrun) every rank steps its own replica: a single run does
not shard (there is no data-path collective); value = all ranks' particle
steps / max-over-ranks time.

--impl reference times the FP64 CPU oracle (the paper's method restated in
plain C, single thread) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+LL push+deposit) & runs/h; p50/p99 latency vs plain"
UNIT = "particle-steps/s"

# the large single run: 100 lambda, lambda/2000, foil 2 lambda thick at 0.25 lambda
LARGE = dict(length_lambda=100.0, cells_per_lambda=2000.0, cfl=0.95, lambda_um=0.8, rr_on=True,
             source_node=8, foil_x0=0.25, foil_thickness=2.0, ne=100.0, ppc=8000, a0=500.0, pol=1,
             duration=20.0, seed=4, sort_interval=8)
RUN_STEPS = 2000  # length of the large run
# step at which the pulse front reaches the foil: (foil front - source node) / cfl
PULSE_AT_FOIL_STEP = int(math.ceil((LARGE["foil_x0"] * LARGE["cells_per_lambda"] - LARGE["source_node"])
                                   / LARGE["cfl"]))
BYTES_PER_PARTICLE_STEP = 40  # cell + offset + 3 momenta, read and written (int32 + 4 x fp32)
# DRAM traffic of one push launch of this workload, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch, 64M particles,
# the push of step 1996) with the pulse in the foil, keyed by (particles,
# particles per unit, sort interval, particles per thread, whether the timed
# window starts after the pulse reached the foil, digest of the push
# kernel's source); a run that does not match every key, or a kernel changed
# since the capture, reports null
PUSH_TRAFFIC = {
    (64_000_000, 16384, 96, 4, True, "82e9ef27a5c0"): 1_282_509_568 + 964_495_872,
}


def push_kernel_digest():
    """First 12 hex digits of the SHA-256 of the push kernel's source: its file
    followed by the internal header that sets its window and unit bounds."""
    import hashlib

    h = hashlib.sha256()
    for name in ("k_push.cu", "picrr_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1008_1685_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:12]


def hot_fractions(sim, w):
    """Fractions of electrons and ions with kinetic energy above 1 keV (a
    one-bin spectrum through pic_spectra; counts are sum(w dx) / bin width)."""
    import numpy as np

    out = {}
    for sp, name in ((0, "electrons"), (1, "ions")):
        lo, hi = 1e-3, 1e7
        c, _ = sim.spectra(sp, 1, lo, hi)
        wdx = (w["ne"] / w["ppc"]) * (2 * math.pi / w["cells_per_lambda"])
        n_sp = w["ppc"] * int(round(w["foil_thickness"] * w["cells_per_lambda"]))
        out[name + "_above_1keV"] = float(np.sum(c) * (hi - lo) / wdx / n_sp)
    return out


def kernel_times(sim, interval, intervals=2):
    """Per-kernel CUDA-event times of the run's next whole sort intervals: with
    timing on, the step graphs hold an event-record node before and after every
    push, Yee update and sort (each pair leaves a gap of a few microseconds
    between the kernels), so the timed window runs without them and the kernel
    times come from these intervals of the same run, right after it."""
    k = sim.stats()["steps_since_sort"]
    if k:
        sim.step(interval - k)  # to a sort boundary: whole intervals follow, as graph launches
    s0 = sim.stats()
    sim.set_timing(True)
    sim.step(intervals * interval)
    st = sim.stats()
    sim.set_timing(False)
    n = intervals * interval
    return {"push_ms": st["push_ms"] / max(1, st["timed_push_launches"]), "field_ms_per_step": st["field_ms"] / n,
            "sort_ms_mean": st["sort_ms"] / max(1, st["sort_count"] - s0["sort_count"]),
            "steps_per_step_ms": (st["push_ms"] + st["field_ms"] + st["sort_ms"]) / n,
            "first_step": s0["steps"], "last_step": s0["steps"] + n - 1}


def rr_cost_leg(sim, interval, reps=3):
    """The radiation-reaction kick's cost on one state: whole sort intervals
    stepped alternately with the kick on and off (pic_set_rr), the push
    kernel's mean launch time and the whole step's time per rr setting."""
    per = {1: [], 0: []}
    step_ms = {1: [], 0: []}
    k = sim.stats()["steps_since_sort"]
    if k:
        sim.step(interval - k)  # to a sort boundary: whole intervals follow, as graph launches
    for _ in range(reps):
        for rr in (1, 0):
            sim.set_rr(rr)
            sim.set_timing(True)
            sim.step(interval)
            st = sim.stats()
            per[rr].append(st["push_ms"] / max(1, st["timed_push_launches"]))
            step_ms[rr].append((st["push_ms"] + st["field_ms"] + st["sort_ms"]) / interval)
    sim.set_rr(1)
    on, off = statistics.median(per[1]), statistics.median(per[0])
    son, soff = statistics.median(step_ms[1]), statistics.median(step_ms[0])
    return {"push_ms_rr_on": on, "push_ms_rr_off": off, "push_ratio": on / off,
            "step_ms_rr_on": son, "step_ms_rr_off": soff, "step_ratio": son / soff,
            "paper": "about +10 % computing time with the RR force (Sec. 3, last paragraph)",
            "how": "%d alternating pairs of %d-step intervals on the same run after the timed window; "
                   "medians; push = the fused kernel's mean launch time, step = push + Yee + sort per step"
                   % (reps, interval)}

# the batched scan: 256 independent runs, 30 lambda at lambda/500 (15,000 cells), foil front at
# 10 lambda, 40 periods each (21,053 steps), per-run parameters drawn from the run's seed
PLAIN_SHAPES = (4096, 8, 2)  # the library's default launch shapes
SCAN = dict(n_runs=256, length_lambda=30.0, cells_per_lambda=500.0, cfl=0.95, foil_x0=10.0, periods=40.0,
            duration=20.0, seed_base=1000, sort_interval=8, shapes=(8192, 96, 2))


def scan_steps(periods, w=SCAN):
    return int(math.ceil(periods * w["cells_per_lambda"] / w["cfl"] - 1e-9))


def scan_desc(i, w=SCAN):
    """Parameters of scan run i, drawn from seed base + i: a0 ~ U[100, 600],
    thickness ~ U[0.5, 2] lambda, n_e ~ U[30, 150] n_c, LP/CP and RR on/off at
    50/50, particles per cell ~ U{32..256}."""
    import numpy as np

    rng = np.random.default_rng(w["seed_base"] + i)
    return dict(length_lambda=w["length_lambda"], foil_x0=w["foil_x0"], foil_thickness=float(rng.uniform(0.5, 2.0)),
                ne=float(rng.uniform(30.0, 150.0)), a0=float(rng.uniform(100.0, 600.0)),
                polarization=int(rng.integers(0, 2)), rr_on=bool(rng.integers(0, 2)), ppc=int(rng.integers(32, 257)),
                duration=w["duration"], steps=scan_steps(w["periods"], w), seed=w["seed_base"] + i)


def desc_particles(d, cpl):
    return 2 * d["ppc"] * int(round(d["foil_thickness"] * cpl))


# the served request stream: Poisson arrivals, sizes log-uniform in 1e4..1e6
# particles per species, 20..200 periods, physical parameters as in the scan,
# admission by device memory under a 150 GB budget
SERVE = dict(rate=20.0, window_s=10.0, cap_s=40.0, budget=150 * 10**9, max_runs=256, chunk=64, seed=77,
             policy="sjf", resident=24_000_000, sort_interval=64)
# a second stream at a rate one GB300 keeps up with for this mix (its capacity is about 1 request/s)
SERVE_LOW = dict(SERVE, rate=0.5, window_s=20.0, cap_s=40.0)


def serve_requests(rate, window_s, seed, w=SCAN):
    """Arrival times (s) and run descriptions of the request stream."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out, t, i = [], 0.0, 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= window_s:
            return out
        n = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
        thick = float(rng.uniform(0.5, 2.0))
        ppc = max(1, int(round(n / (thick * w["cells_per_lambda"]))))
        periods = float(rng.uniform(20.0, 200.0))
        d = dict(length_lambda=w["length_lambda"], foil_x0=w["foil_x0"], foil_thickness=thick,
                 ne=float(rng.uniform(30.0, 150.0)), a0=float(rng.uniform(100.0, 600.0)),
                 polarization=int(rng.integers(0, 2)), rr_on=bool(rng.integers(0, 2)), ppc=ppc,
                 duration=w["duration"], steps=scan_steps(periods, w), seed=seed * 100000 + i)
        out.append((t, d))
        i += 1


def _latency_summary(lat, pending_ages, elapsed, n_req):
    import numpy as np

    done = np.array(sorted(lat)) if lat else np.zeros(0)
    cens = np.array(sorted(list(lat) + list(pending_ages)))
    q = lambda a, p: float(np.percentile(a, p)) if len(a) else None
    return {"requests": n_req, "completed": len(lat), "unfinished": len(pending_ages),
            "p50_s": q(done, 50), "p99_s": q(done, 99),
            "p50_s_with_unfinished_lower_bound": q(cens, 50), "p99_s_with_unfinished_lower_bound": q(cens, 99),
            "runs_per_hour": 3600.0 * len(lat) / elapsed}


def my_requests(picrr, cfg, w, rank, ws):
    """This rank's share of the request stream: each request goes, in arrival
    order, to the rank with the least work so far (pic_shard_runs)."""
    reqs = serve_requests(cfg["rate"], cfg["window_s"], cfg["seed"], w)
    if ws == 1 or not reqs:
        return reqs
    ranks, _ = shard(picrr, [d for _, d in reqs], ws, in_order=True, w=w)
    return [q for q, r in zip(reqs, ranks) if r == rank]


def serve_leg(picrr, device, cfg=SERVE, w=SCAN, rank=0, ws=1):
    """Continuous batching through pic_server: requests are submitted at their
    arrival times; latency = submission to spectra on the host."""
    import threading

    reqs = my_requests(picrr, cfg, w, rank, ws)
    srv = picrr.Server(w["cells_per_lambda"], max_runs=cfg["max_runs"], chunk_steps=cfg["chunk"], cfl=w["cfl"],
                       sort_interval=cfg["sort_interval"], device=device, hbm_budget_bytes=cfg["budget"])
    srv.set_policy(picrr.SERVE_SHORTEST_FIRST if cfg["policy"] == "sjf" else picrr.SERVE_FIFO, cfg["resident"])
    tickets = []
    t0 = time.perf_counter()

    def submitter():
        for ta, d in reqs:
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append((ta, srv.submit(nbins=200, ion_e_max=2000.0, el_e_max=2000.0, **d)))

    th = threading.Thread(target=submitter)
    th.start()
    lat, done = [], set()
    while time.perf_counter() - t0 < cfg["cap_s"]:
        for ta, t in list(tickets):
            if t not in done:
                r = srv.result(t, 0.0)
                if r is not None:
                    lat.append(r["latency_s"])
                    done.add(t)
        if len(done) == len(reqs):
            break
        time.sleep(0.01)
    th.join()
    el = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    pending = [el - ta for ta, t in tickets if t not in done]
    out = _latency_summary(lat, pending, el, len(reqs))
    work = sum(desc_particles(d, w["cells_per_lambda"]) * d["steps"] for _, d in reqs)
    out.update(elapsed_s=el, offered_particle_steps_per_s=work / cfg["window_s"],
               served_particle_steps_per_s=st["particle_steps"] / el,
               peak_device_bytes=st["peak_device_bytes"], batch_steps=st["batch_steps"])
    return out


def plain_serve_leg(picrr, device, cfg=SERVE, w=SCAN, rank=0, ws=1):
    """The same request stream served one run at a time through the
    single-run API (no batching), under the same time cap and the same order
    policy (arrival order, or the least work among the arrived requests)."""
    reqs = my_requests(picrr, cfg, w, rank, ws)
    work = [desc_particles(d, w["cells_per_lambda"]) * d["steps"] for _, d in reqs]
    t0 = time.perf_counter()
    lat, pending = [], list(range(len(reqs)))
    while pending and time.perf_counter() - t0 < cfg["cap_s"]:
        now = time.perf_counter() - t0
        arrived = [j for j in pending if reqs[j][0] <= now]
        if not arrived:
            time.sleep(max(0.0, reqs[pending[0]][0] - now))
            continue
        j = min(arrived, key=lambda q: (work[q], q)) if cfg["policy"] == "sjf" else arrived[0]
        ta, d = reqs[j]
        s = picrr.Sim(d["length_lambda"], w["cells_per_lambda"], cfl=w["cfl"], rr_on=d["rr_on"],
                      sort_interval=cfg["sort_interval"], seed=d["seed"], device=device)
        s.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"])
        s.inject_laser(d["a0"], d["polarization"], 0, d["duration"])
        left = d["steps"]
        while left > 0 and time.perf_counter() - t0 < cfg["cap_s"]:
            left -= s.step(min(left, 4096))
        if left == 0:
            s.spectra(1, 200, 0.0, 2000.0)
            s.spectra(0, 200, 0.0, 2000.0)
            s.energy()
            lat.append(time.perf_counter() - t0 - ta)
            pending.remove(j)
        s.close()
    el = time.perf_counter() - t0
    return _latency_summary(lat, [el - reqs[j][0] for j in pending if reqs[j][0] <= el], el, len(reqs))


def shard(picrr, descs, ranks, in_order=False, w=SCAN):
    """The rank of each run description (pic_shard_runs: least-work rank
    first, largest runs first unless in_order); every rank computes the same."""
    rd = [picrr.run_desc(d["length_lambda"], d["foil_x0"], d["foil_thickness"], d["ne"], d["a0"],
                         d["polarization"], d["duration"], d["steps"], rr_on=d["rr_on"], ppc=d["ppc"], seed=d["seed"])
          for d in descs]
    return picrr.shard_runs(rd, ranks, w["cells_per_lambda"], in_order=in_order)


def batched_scan(picrr, device, run_ids, w=SCAN, max_steps=None, shapes=None):
    """The scan runs run_ids (indices into the scan's seed sequence) in one
    batch (one launch per kernel per step for all of them), from creation to
    every run's ion spectrum on the host.  max_steps (for profiling) cuts
    every run short; shapes: (unit particles, sort interval, particles per
    thread) of the batch."""
    n_runs = len(run_ids)
    descs = [scan_desc(i, w) for i in run_ids]
    if max_steps:
        descs = [dict(d, steps=min(d["steps"], max_steps)) for d in descs]
    shapes = shapes or w["shapes"]
    t0 = time.perf_counter()
    b = picrr.Batch(w["cells_per_lambda"], max_runs=n_runs, cfl=w["cfl"], sort_interval=shapes[1], device=device)
    b.set_shapes(*shapes)
    ids = [b.add_run(d["length_lambda"], d["foil_x0"], d["foil_thickness"], d["ne"], d["a0"], d["polarization"],
                     d["duration"], d["steps"], rr_on=d["rr_on"], ppc=d["ppc"], seed=d["seed"]) for d in descs]
    while b.step(4096) > 0:
        pass
    for r in ids:
        b.spectra(r, 1, 200, 0.0, 2000.0)
    el = time.perf_counter() - t0
    st = b.stats()
    b.close()
    ps = sum(desc_particles(d, w["cells_per_lambda"]) * d["steps"] for d in descs)
    return dict(runs=n_runs, seconds=el, runs_per_hour=3600.0 * n_runs / el, particle_steps_per_s=ps / el,
                particles=sum(desc_particles(d, w["cells_per_lambda"]) for d in descs),
                push_launches=st["push_launches"], kernel_launches=st["kernel_launches"])


def plain_scan(picrr, device, run_ids, w=SCAN, shapes=None):
    """The same runs one at a time through the single-run API (create, foil,
    laser, step to the end, ion spectrum, destroy), on the same GPU, with the
    same launch shapes."""
    n_runs = len(run_ids)
    descs = [scan_desc(i, w) for i in run_ids]
    shapes = shapes or w["shapes"]
    t0 = time.perf_counter()
    for d in descs:
        s = picrr.Sim(d["length_lambda"], w["cells_per_lambda"], cfl=w["cfl"], rr_on=d["rr_on"],
                      sort_interval=shapes[1], seed=d["seed"], device=device)
        s.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"])
        s.inject_laser(d["a0"], d["polarization"], 0, d["duration"])
        s.set_shapes(*shapes)
        s.step(d["steps"])
        s.spectra(1, 200, 0.0, 2000.0)
        s.close()
    el = time.perf_counter() - t0
    ps = sum(desc_particles(d, w["cells_per_lambda"]) * d["steps"] for d in descs)
    return dict(runs=n_runs, seconds=el, runs_per_hour=3600.0 * n_runs / el, particle_steps_per_s=ps / el)


# thin, hot plasma: electrons with momenta of width 20 (m_e c) and cold-ish
# protons spread uniformly over 3.84M cells (the cells of the 256-run scan),
# about 6 particles per cell per species: the deposit's worst case, where
# nearly every lane of a warp holds its own anchor
THIN = dict(cells=3_840_000, per_species=22_500_000, p_e=20.0, p_i=0.05, shapes=(4096, 8, 2), warm=16, steps=24,
            seed=1)


def thin_leg(picrr, device, w=THIN):
    """The push kernel on synthetic thin, hot plasma (seeded), timed with CUDA
    events over `steps` steps after `warm`."""
    import numpy as np

    cpl = 500.0
    s = picrr.Sim(w["cells"] / cpl, cpl, cfl=0.95, rr_on=True, sort_interval=w["shapes"][1], seed=w["seed"],
                  device=device)
    rng = np.random.default_rng(w["seed"])
    n = w["per_species"]
    cell = np.sort(rng.integers(1000, w["cells"] - 1000, n)).astype(np.int32)
    off = rng.random(n, dtype=np.float32)
    for sp, (ps, q, m) in enumerate([(w["p_e"], -1.0, 1.0), (w["p_i"], 1.0, 1836.15267343)]):
        px, py, pz = (rng.standard_normal(n, dtype=np.float32) * np.float32(ps) for _ in range(3))
        s.load_particles_f32(sp, cell, off, px, py, pz, 0.01, q, m)
    s.set_shapes(*w["shapes"])
    s.step(w["warm"])
    s.set_timing(True)
    s.step(w["steps"])
    st = s.stats()
    s.close()
    push = st["push_ms"] / max(1, st["timed_push_launches"])
    peak, kind = _peaks()
    gbs = BYTES_PER_PARTICLE_STEP * 2 * n / (push / 1e3) / 1e9
    return {"push_ms": push, "achieved_gbs": gbs, "frac": gbs / peak, "peak_kind": kind,
            "field_ms": st["field_ms"] / w["steps"], "sort_ms_per_step": st["sort_ms"] / w["steps"],
            "workload": "%d cells, %dM electrons (momenta N(0, %g)) + %dM protons (N(0, %g)) uniform, units of %d, "
                        "sort every %d, %d per thread; %d steps timed after %d"
                        % (w["cells"], n // 10**6, w["p_e"], n // 10**6, w["p_i"], w["shapes"][0], w["shapes"][1],
                           w["shapes"][2], w["steps"], w["warm"])}


def parity_leg(picrr, device):
    """The GPU's errors against the FP64 oracle on small seeded cases, outside
    any timed region: the oracle's results are stored in
    tests/golden/oracle_parity_cases.json and oracle_small_run_ensemble.json
    (written by scripts there that call only the oracle); the inputs are
    regenerated from the same seeds by tests/synth.py."""
    import numpy as np

    from tests import synth
    from tests.spectrum_stats import balance, peak_fwhm

    gold = os.path.join(ROOT, "tests", "golden")
    G = json.load(open(os.path.join(gold, "oracle_parity_cases.json")))
    out = {}
    c = G["one_step"]
    g = picrr.Sim(seed=1, sort_interval=8, device=device, **c["box"])
    F = synth.random_fields(g.nx, **c["fields"])
    g.set_fields(*F)
    for sp, s in enumerate(c["species"]):
        p = synth.random_particles(s["n"], 2, g.nx - 2, s["pscale"], s["seed"])
        g.load_particles(sp, *p, s["weight"], s["charge"], s["mass"])
    g.step(1)
    worst_p, worst_x = 0.0, 0.0
    for sp in (0, 1):
        q, r = g.particles(sp), c["result"][sp]
        pg = np.stack([q["px"], q["py"], q["pz"]], 1)
        po = np.stack([np.array(r["px"]), np.array(r["py"]), np.array(r["pz"])], 1)
        scale = np.maximum(np.linalg.norm(po, axis=1), 1e-3 * c["fields"]["scale"] * g.dt)
        worst_p = max(worst_p, float(np.max(np.max(np.abs(pg - po), axis=1) / scale)))
        worst_x = max(worst_x, float(np.max(np.abs(q["x"] - np.array(r["x"]))) / g.dx))
    g.close()
    out["momentum_1_step"] = {"max_rel": worst_p, "tolerance": 1e-5,
                              "what": "per particle max-norm difference / max(|p|, 1e-3 F dt), 1000 e + 500 p"}
    out["position_1_step"] = {"max_cells": worst_x}
    c = G["fields_200"]
    g = picrr.Sim(seed=c["foil"]["seed"], sort_interval=8, device=device, **c["box"])
    f, la = c["foil"], c["laser"]
    g.load_foil(f["x0"], f["thickness"], f["ne"], f["Z"], f["A"], f["ppc"])
    g.inject_laser(la["a0"], la["polarization"], la["envelope"], la["duration"])
    g.step(c["steps"])
    groups = {"E_perp": (1, 2), "B_perp": (3, 4), "Ex": (0,)}
    l2 = {}
    for name, comps in groups.items():
        a = np.concatenate([g.field(k) for k in comps])
        b = np.concatenate([np.array(c["result"][k]) for k in comps])
        l2[name] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    g.close()
    out["fields_200_steps"] = {"rel_l2": l2, "tolerance": 1e-4}
    c = G["balance"]
    g = picrr.Sim(seed=c["foil"]["seed"], sort_interval=8, device=device, **c["box"])
    f, la = c["foil"], c["laser"]
    g.load_foil(f["x0"], f["thickness"], f["ne"], f["Z"], f["A"], f["ppc"])
    g.inject_laser(la["a0"], la["polarization"], la["envelope"], la["duration"])
    b, e = balance(g, c["steps"], c["every"])
    g.close()
    out["energy_balance"] = {"gpu_max_over_injected": float(np.max(np.abs(b)) / e[4]),
                             "oracle_max_over_injected": c["result"]["max_abs_over_injected"],
                             "tolerance": 1e-3, "what": "small single run, 4211 steps, time-centred balance"}
    E = json.load(open(os.path.join(gold, "oracle_small_run_ensemble.json")))
    seeds = E["seeds"]
    nb, e_max = E["bins"]["n"], E["bins"]["e_max"]
    bt = picrr.Batch(E["small"]["cells_per_lambda"], max_runs=len(seeds), sort_interval=8, device=device)
    f, la = E["foil"], E["laser"]
    ids = [bt.add_run(E["small"]["length_lambda"], f["x0"], f["thickness"], f["ne"], la["a0"], la["polarization"],
                      la["duration"], E["steps"], rr_on=True, ppc=f["ppc"], seed=sd) for sd in seeds]
    while bt.step(4096) > 0:
        pass
    spec_g = sum(bt.spectra(r, 1, nb, 0.0, e_max)[0] for r in ids)
    rad_g = float(np.mean([bt.energy(r)[3] for r in ids]))
    bt.close()
    spec_o = np.array(E["spectrum_sum"])
    pg, fg = peak_fwhm(spec_g, 0.0, e_max)
    po, fo = peak_fwhm(spec_o, 0.0, e_max)
    ec = (np.arange(nb) + 0.5) * e_max / nb
    mg, mo = float(spec_g @ ec / spec_g.sum()), float(spec_o @ ec / spec_o.sum())
    rad_o = float(np.mean(E["radiated"]))
    out["ensemble_%d_seeds" % len(seeds)] = {
        "peak_rel": pg / po - 1.0, "fwhm_rel": fg / fo - 1.0, "mean_energy_rel": mg / mo - 1.0,
        "radiated_rel": rad_g / rad_o - 1.0, "tolerance": 0.02,
        "what": "ion spectra of the small single run summed over foil seeds (full runs are chaotic)"}
    return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler (every 50 ms); only the samples stamped between
    begin() and end() (the timed region) are kept."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        # let the sampler start before the timed region
        for _ in range(40):
            if self.p is None or os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.05)

    def begin(self):
        self.t0 = datetime.datetime.now()

    def end(self):
        self.t1 = datetime.datetime.now()

    @staticmethod
    def _stamp(text):
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f")
        except ValueError:
            return None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if (lambda t: t is not None and self.t0 <= t <= self.t1)(self._stamp(r[0]))]
            if inside:
                rows = inside
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(steps, ppc=400, parallel=True):
    """The FP64 oracle on the large run's grid and foil with ppc per species,
    the first `steps` steps (the oracle's cost per particle does not depend on
    the state: it has no sort and skips nothing but frozen particles).
    parallel: the OpenMP timing build on all host cores (OMP_NUM_THREADS)."""
    import oracle

    par = parallel and oracle.parallel_available()
    w = LARGE
    o = oracle.OracleSim(w["length_lambda"], w["cells_per_lambda"], w["cfl"], w["lambda_um"], w["rr_on"],
                         w["source_node"], parallel=par)
    o.load_foil(w["foil_x0"], w["foil_thickness"], w["ne"], 1, 1.0, ppc, w["seed"])
    o.inject_laser(w["a0"], w["pol"], 0, w["duration"])
    n_part = 2 * ppc * int(round(w["foil_thickness"] * w["cells_per_lambda"]))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    cores = oracle.threads() if par else 1
    sample = ("large-run grid (200,000 cells) and foil with %d macro-particles per cell per species "
              "(%d particles), first %d steps, FP64, %d threads" % (ppc, n_part, steps, cores))
    return n_part * steps / dt, sample, cores


# the small single run (20 lambda at lambda/200, 1-lambda foil at 10 lambda, n_e = 64 n_c, 64 ppc per
# species, LP a0 = 200, 10-period sin^2 pulse, RR on, 4211 steps) and the paper-scale run (60 lambda at
# lambda/1000, 1-lambda foil at 10 lambda, n_e = 90 n_c, 400 ppc, a0 = 350 LP, 20-period pulse)
SMALL = dict(length_lambda=20.0, cells_per_lambda=200.0, foil_x0=10.0, foil_thickness=1.0, ne=64.0, ppc=64,
             a0=200.0, pol=0, duration=10.0, steps=4211, seed=1)
PAPER = dict(length_lambda=60.0, cells_per_lambda=1000.0, foil_x0=10.0, foil_thickness=1.0, ne=90.0, ppc=400,
             a0=350.0, pol=0, duration=20.0, steps=500, seed=11)


def _oracle_run(d, steps, parallel):
    import oracle

    o = oracle.OracleSim(d["length_lambda"], d["cells_per_lambda"], 0.95, 0.8, True, 8, parallel=parallel)
    o.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"], d["seed"])
    o.inject_laser(d["a0"], d["pol"], 0, d["duration"])
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    n = 2 * d["ppc"] * int(round(d["foil_thickness"] * d["cells_per_lambda"]))
    o.close()
    return el, n


def _oracle_scan_worker(args):
    i, steps = args
    d = scan_desc(i)
    run = dict(length_lambda=d["length_lambda"], cells_per_lambda=SCAN["cells_per_lambda"], foil_x0=d["foil_x0"],
               foil_thickness=d["foil_thickness"], ne=d["ne"], ppc=d["ppc"], a0=d["a0"], pol=d["polarization"],
               duration=d["duration"], seed=d["seed"])
    el, n = _oracle_run(run, steps, False)
    return el, n, d["steps"]


def cpu_plan_leg(scan_runs=16, scan_steps=800):
    """The oracle on the host cores for the workloads the GPU legs run: the
    small single run in full and the paper-scale run's first 500 steps (the
    OpenMP build, all cores), and 16 scan runs in 16 processes (the serial
    build, one run each) for their first scan_steps steps, extrapolated to
    the full run length and to the 256-run scan."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import oracle

    par = oracle.parallel_available()
    out = {"threads": oracle.threads() if par else 1, "nproc": os.cpu_count()}
    el, n = _oracle_run(SMALL, SMALL["steps"], par)
    out["small_run_full"] = {"seconds": el, "particle_steps_per_s": n * SMALL["steps"] / el,
                             "runs_per_hour": 3600.0 / el,
                             "what": "20 lambda at lambda/200, 12,800 + 12,800 particles, LP a0 = 200, all 4211 steps"}
    el, n = _oracle_run(PAPER, PAPER["steps"], par)
    out["paper_scale_500_steps"] = {"seconds": el, "particle_steps_per_s": n * PAPER["steps"] / el,
                                    "what": "60,000 cells, 400k + 400k particles, first 500 steps"}
    workers = min(scan_runs, os.cpu_count() or 1)
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_scan_worker, [(i, scan_steps) for i in range(scan_runs)]))
    wall = time.perf_counter() - t0
    full = sum(el * total / scan_steps for el, _, total in res)  # one core, all 16 runs in full
    ps = sum(n * scan_steps for _, n, _ in res)
    out["batched_scan"] = {
        "runs_timed": scan_runs, "steps_timed": scan_steps, "processes": workers, "wall_s": wall,
        "particle_steps_per_s": ps / wall,
        "runs_per_hour_extrapolated": 3600.0 * scan_runs / (full / workers),
        "what": "the scan's first %d runs, one process each (serial oracle), first %d of their 21,053 steps; "
                "runs/h extrapolated to full length and to %d processes running the 256 runs"
                % (scan_runs, scan_steps, workers)}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    vals = []
    oracle_sample(2, ppc=args.ref_ppc)
    for _ in range(max(1, args.steps)):
        v, sample, cores = oracle_sample(args.ref_steps, ppc=args.ref_ppc)
        vals.append(v)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_with_window(window_start(args.steps, args.warmup, args.preroll),
                                                        args.steps),
                       "cells": 200000},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def aggregate(torch, dist, ms, particle_steps):
    """Whole-job numbers across replicas: the slowest rank's time and the sum
    of all ranks' particle steps (all_reduce MAX / SUM; identity at N = 1)."""
    if dist is None or not dist.is_initialized():
        return ms, particle_steps
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    n = torch.tensor([particle_steps], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def large_workload(ppc=LARGE["ppc"]):
    """The name of the large single run (both arms report the same workload)."""
    n = ppc * int(round(LARGE["foil_thickness"] * LARGE["cells_per_lambda"]))
    return ("large single run: 200,000 cells (100 lambda, lambda/2000), 2-lambda H foil n_e=100 n_c, "
            "%d ppc/species (%.3gM e + %.3gM p), CP a0=500, RR on" % (ppc, n / 1e6, n / 1e6))


# steps the shape tuner takes (its trials are real steps): two particles-per-thread trials and four
# unit-size trials at the default interval of 8, then one trial per interval of 8, 16, 32, 64, 96;
# each trial is one warm-up interval plus TUNER_TRIAL steps rounded to whole intervals (at least one)
TUNER_TRIAL = 48
TUNER_STEPS = 6 * (8 + TUNER_TRIAL) + sum(i + max(i, TUNER_TRIAL // i * i) for i in (8, 16, 32, 64, 96))


def window_start(steps, warmup, preroll, tuned=True):
    """First timed step of the large run: the last `steps` of the 2000-step
    run when they fit after the pre-roll, the tuner and the warm-up;
    otherwise right after those."""
    now = preroll + (TUNER_STEPS if tuned else 0)
    return max(RUN_STEPS - steps, now + warmup)


def workload_with_window(start, steps, ppc=LARGE["ppc"]):
    return (large_workload(ppc) + "; timed steps %d..%d of the 2000-step run (the pulse front reaches the foil at "
            "step %d)" % (start, start + steps - 1, PULSE_AT_FOIL_STEP))


def make_sim(picrr, device, w=LARGE):
    s = picrr.Sim(w["length_lambda"], w["cells_per_lambda"], cfl=w["cfl"], lambda_um=w["lambda_um"],
                  rr_on=w["rr_on"], sort_interval=w["sort_interval"], seed=w["seed"], device=device,
                  source_node=w["source_node"])
    return s


def host_foil(np, torch, w=LARGE):
    """The large run's foil as pinned host SoA (seeded, cell-ordered, cold)."""
    cpl = w["cells_per_lambda"]
    c0, nc = int(round(w["foil_x0"] * cpl)), int(round(w["foil_thickness"] * cpl))
    rng = np.random.default_rng(w["seed"])
    cell = np.repeat(np.arange(c0, c0 + nc, dtype=np.int32), w["ppc"])
    off = rng.random(cell.size, dtype=np.float32)
    zero = np.zeros(cell.size, np.float32)
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    arrs = [pin(cell), pin(off), pin(zero), pin(zero.copy()), pin(zero.copy())]
    host = {0: arrs, 1: arrs,
            "species": {0: (w["ne"] / w["ppc"], -1.0, 1.0), 1: (w["ne"] / w["ppc"], 1.0, 1836.15267343)}}
    return host


def e2e_run(picrr, torch, device, steps, host, shapes=None):
    """Through the public C ABI with host buffers: create, upload the particles
    from pinned host memory, inject, step, read spectra + energy back."""
    w = LARGE
    t0 = time.perf_counter()
    s = make_sim(picrr, device)
    for sp in (0, 1):
        c, o, x, y, z = host[sp]
        s.load_particles_f32(sp, c, o, x, y, z, *host["species"][sp])
    s.inject_laser(w["a0"], w["pol"], 0, w["duration"])
    if shapes:
        s.set_shapes(shapes["unit_particles"], shapes["sort_interval"], shapes["particles_per_thread"])
    s.step(steps)
    counts, rad = s.spectra(1, 200, 0.0, 2000.0)
    en = s.energy()
    el = time.perf_counter() - t0
    n = s.stats()["active_particles"]
    s.close()
    h2d = sum(host[sp][k].nbytes for sp in (0, 1) for k in range(5))
    d2h = counts.nbytes + en.nbytes + 8
    return n * steps / el, h2d, d2h


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=384)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-steps", type=int, default=40, help="steps of each oracle sample")
    ap.add_argument("--ref-ppc", type=int, default=400, help="particles per cell per species of the oracle sample")
    ap.add_argument("--no-cpu-plan", action="store_true",
                    help="skip the oracle timings of the small run, the paper-scale run and the scan")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no tuner run)")
    ap.add_argument("--shapes", default=None,
                    help="UNIT,INTERVAL[,PARTICLES_PER_THREAD]: set these launch shapes instead of running the "
                         "tuner (profiling)")
    ap.add_argument("--scan-runs", type=int, default=SCAN["n_runs"], help="runs of the batched scan (0: skip)")
    ap.add_argument("--scan-steps", type=int, default=0, help="cut the scan runs to this many steps (profiling)")
    ap.add_argument("--scan-shapes", default=None, help="UNIT,INTERVAL,PARTICLES_PER_THREAD of the scan's batch")
    ap.add_argument("--plain-runs", type=int, default=8,
                    help="runs of the scan stepped one at a time for the plain comparison (0: skip)")
    ap.add_argument("--serve-window", type=float, default=SERVE["window_s"],
                    help="seconds of request arrivals of the serving leg (0: skip)")
    ap.add_argument("--serve-cap", type=float, default=SERVE["cap_s"], help="time cap of each serving arm (s)")
    ap.add_argument("--serve-rate", type=float, default=SERVE["rate"], help="request arrivals per second")
    ap.add_argument("--serve-low-rate", type=float, default=SERVE_LOW["rate"],
                    help="arrival rate of the second (sustainable) stream; 0 skips it")
    ap.add_argument("--serve-policy", default=SERVE["policy"], choices=["sjf", "fifo"],
                    help="admission order of both serving arms: least work first, or arrival order")
    ap.add_argument("--serve-sort-interval", type=int, default=SERVE["sort_interval"],
                    help="sort interval of the server's batch and of the plain arm")
    ap.add_argument("--serve-resident", type=int, default=SERVE["resident"],
                    help="particles stepping at once in the server (0: no cap)")
    ap.add_argument("--preroll", type=int, default=PULSE_AT_FOIL_STEP + 82,
                    help="untimed steps before the tuner; the timed window ends at step 2000 when it fits after "
                         "them")
    ap.add_argument("--no-rr-cost", action="store_true", help="skip the RR on/off timing after the window")
    ap.add_argument("--no-parity", action="store_true", help="skip the errors against the stored oracle results")
    ap.add_argument("--no-thin", action="store_true", help="skip the thin, hot plasma push timing")
    ap.add_argument("--ppc", type=int, default=LARGE["ppc"],
                    help="macro-particles per cell per species (smaller values give the profiling case)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = _dist()
    import numpy as np
    import torch

    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as picrr

    w = dict(LARGE, ppc=args.ppc)
    shapes = None
    if args.shapes:
        v = [int(x) for x in args.shapes.split(",")]
        shapes = {"unit_particles": v[0], "sort_interval": v[1], "particles_per_thread": v[2] if len(v) > 2 else 4,
                  "tuned": False}
    sim = make_sim(picrr, local, w)
    sim.load_foil(w["foil_x0"], w["foil_thickness"], w["ne"], 1, 1.0, w["ppc"])
    sim.inject_laser(w["a0"], w["pol"], 0, w["duration"])
    if shapes:
        sim.set_shapes(shapes["unit_particles"], shapes["sort_interval"], shapes["particles_per_thread"])
    stream = torch.cuda.current_stream()
    sim.set_stream(stream.cuda_stream)
    # untimed pre-roll: the pulse front reaches the foil at step ~518; the
    # tuner (whose trial steps are real steps of this run) and the timed
    # window both run with the pulse in the foil
    sim.step(args.preroll)
    if shapes is None and not args.no_tune:
        unit, interval, ppt, tms = sim.tune_shapes(TUNER_TRIAL)
        shapes = {"unit_particles": unit, "sort_interval": interval, "particles_per_thread": ppt, "tuned": True,
                  "tuned_from_step": sim.stats()["steps"],
                  "trial_ms_per_step": {"particles_per_thread_4_2": [round(v, 4) for v in tms[:2]],
                                        "unit_2048_4096_8192_16384": [round(v, 4) for v in tms[2:6]],
                                        "interval_8_16_32_64_96": [round(v, 4) for v in tms[6:]]}}
    interval = shapes["sort_interval"] if shapes else w["sort_interval"]
    # the timed window ends at the run's last step (2000) when it fits after
    # the pre-roll, the tuner and the warm-up; otherwise it starts right after them
    now = sim.stats()["steps"]
    start = max(RUN_STEPS - args.steps, now + args.warmup)
    sim.step(start - args.warmup - now)
    sim.step(args.warmup)
    hot = hot_fractions(sim, w)
    st0 = sim.stats()
    n_active = st0["active_particles"]

    def barrier():
        if dist is not None:
            dist.barrier()

    clocks = Clocks(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    sim.set_timing(False)  # no per-kernel event nodes inside the timed window (kernel_times below)
    st0 = sim.stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.begin()
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.end()
    barrier()
    ms_raw = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    st1 = sim.stats()
    n_active_end = st1["active_particles"]
    # kernel times (CUDA events on the launching stream) from the next two
    # whole sort intervals; the sorts that fell inside the K timed steps are
    # replaced by K / interval sorts of their mean duration, so that the value
    # holds the amortised sort at any K
    sorts_in = st1["sort_count"] - st0["sort_count"]
    kt = kernel_times(sim, interval)
    sort_ms_mean = kt["sort_ms_mean"]
    ms = ms_raw - sorts_in * sort_ms_mean + args.steps * sort_ms_mean / interval
    ms_max, total = aggregate(torch, dist, ms, float(n_active) * args.steps)
    value = total / (ms_max / 1e3)
    push_avg_ms = kt["push_ms"]
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_PARTICLE_STEP * n_active / (push_avg_ms / 1e3) / 1e9
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    traffic = None
    if shapes:
        traffic = PUSH_TRAFFIC.get((n_active, shapes["unit_particles"], shapes["sort_interval"],
                                    shapes["particles_per_thread"], start >= PULSE_AT_FOIL_STEP,
                                    push_kernel_digest()))
    window = {"first_step": start, "last_step": start + args.steps - 1, "ms_raw": ms_raw, "sorts_inside": sorts_in,
              "sort_ms_mean": sort_ms_mean, "sort_interval": interval,
              "ms_with_amortised_sort": ms, "kernel_launches_before": st0["kernel_launches"],
              "push_launches_before": st0["push_launches"],
              "kernel_times": {"first_step": kt["first_step"], "last_step": kt["last_step"],
                               "sum_of_kernel_ms_per_step": kt["steps_per_step_ms"],
                               "what": "per-kernel CUDA events (event-record nodes around every push, Yee update "
                                       "and sort in the step graphs) over the two whole sort intervals after the "
                                       "window; the window itself runs without them"}}
    rr_cost = None if args.no_rr_cost else rr_cost_leg(sim, interval)
    sim.close()

    e2e = None
    if not args.no_e2e:
        host = host_foil(np, torch)
        n_e2e = start + args.steps
        ev, h2d, d2h = e2e_run(picrr, torch, local, n_e2e, host, shapes)
        e2e = {"value": ev, "unit": UNIT, "h2d_bytes_per_step": h2d / n_e2e,
               "d2h_bytes_per_step": d2h / n_e2e, "steps": n_e2e,
               "what": "pic_create + pic_load_particles_f32 from pinned host SoA + pic_inject_laser + "
                       "pic_set_shapes (the tuned shapes) + pic_step_n(steps 0 .. end of the timed window) + "
                       "pic_spectra + pic_energy, host wall clock"}

    thin = thin_leg(picrr, local) if not args.no_thin else None

    scan = None
    if args.scan_runs > 0:
        # the scan's runs split over the ranks by work (strong scaling: the
        # whole job steps the same runs at any N)
        ranks, loads = shard(picrr, [scan_desc(i) for i in range(args.scan_runs)], ws)
        mine = [i for i, r in enumerate(ranks) if r == rank]
        scan_shapes = tuple(int(x) for x in args.scan_shapes.split(",")) if args.scan_shapes else SCAN["shapes"]
        scan = batched_scan(picrr, local, mine, max_steps=args.scan_steps or None, shapes=scan_shapes)
        scan["shapes"] = scan_shapes
        if args.plain_runs > 0:
            # runs one at a time take the library's default shapes (units of 4096, sort every 8), their better
            # choice: with the scan's (units of 8192, sort every 64) they run 25 % slower
            plain = plain_scan(picrr, local, mine[:args.plain_runs], shapes=PLAIN_SHAPES)
            plain["shapes"] = PLAIN_SHAPES
            scan["plain"] = plain
            scan["speedup_runs_per_hour"] = scan["runs_per_hour"] / plain["runs_per_hour"]
        scan["workload"] = ("%d runs, 15,000 cells (30 lambda, lambda/500), 21,053 steps each; a0 U[100,600], "
                            "thickness U[0.5,2] lambda, n_e U[30,150] n_c, LP/CP, RR on/off, ppc U{32..256}; "
                            "plain = the first %d of the same runs one at a time" % (args.scan_runs, args.plain_runs))
        ms_scan, _ = aggregate(torch, dist, scan["seconds"] * 1e3, 0.0)
        scan["runs_per_hour"] = 3600.0 * args.scan_runs / (ms_scan / 1e3)
        scan["scaling"] = "strong"
        scan["sharding"] = {"ranks": ws, "runs_per_rank": [ranks.count(r) for r in range(ws)],
                            "particle_steps_per_rank": [float(x) for x in loads]}

    serving = None
    if args.serve_window > 0:
        def one_stream(cfg):
            out = serve_leg(picrr, local, cfg, rank=rank, ws=ws)
            out["plain"] = plain_serve_leg(picrr, local, cfg, rank=rank, ws=ws)
            if ws > 1:
                ms_all, done_all = aggregate(torch, dist, out["elapsed_s"] * 1e3, float(out["completed"]))
                out["share"] = "rank 0's share of the stream (requests split over %d ranks as they arrive)" % ws
                out["completed_all_ranks"] = int(done_all)
                out["runs_per_hour_all_ranks"] = 3600.0 * done_all / (ms_all / 1e3)
            out["overloaded"] = out["unfinished"] > 0  # the queue had not drained when the cap ended the arm
            out["workload"] = ("Poisson arrivals at %g/s for %g s (seed %d), per species 1e4..1e6 particles "
                               "(log-uniform), 20..200 periods at lambda/500 in a 30-lambda box, parameters as in "
                               "the scan; 150 GB admission budget, %d slots, at most %d particles stepping at once, "
                               "%d-step chunks, sort every %d steps, admission %s in both arms; each arm capped "
                               "at %g s; latency = submission to ion + electron spectra on the host"
                               % (cfg["rate"], cfg["window_s"], cfg["seed"], cfg["max_runs"], cfg["resident"],
                                  cfg["chunk"], cfg["sort_interval"],
                                  "least work first" if cfg["policy"] == "sjf" else "in arrival order", cfg["cap_s"]))
            return out

        # one request stream split over the ranks as the requests arrive; rank 0 reports its share
        cfg = dict(SERVE, window_s=args.serve_window, cap_s=args.serve_cap, rate=args.serve_rate,
                   policy=args.serve_policy, resident=args.serve_resident, sort_interval=args.serve_sort_interval)
        serving = one_stream(cfg)
        if args.serve_low_rate > 0:
            low = dict(SERVE_LOW, cap_s=args.serve_cap, rate=args.serve_low_rate, policy=args.serve_policy,
                       resident=args.serve_resident, sort_interval=args.serve_sort_interval)
            serving["sustainable_rate"] = one_stream(low)

    parity = None
    if rank == 0 and not args.no_parity:
        parity = parity_leg(picrr, local)

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, sample, cores = oracle_sample(args.ref_steps, ppc=args.ref_ppc)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        if not args.no_cpu_plan:
            cpu["plan"] = cpu_plan_leg()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_with_window(start, args.steps, args.ppc),
                       "particles": n_active, "particles_end": n_active_end, "cells": 200000,
                       "sort_interval": interval,
                       "shapes": shapes, "hot_at_window_start": hot,
                       "l2": "inputs larger than L2: 2.56 GB particle state streamed per step",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_push_deposit", "kernel_ms": push_avg_ms,
                         "peak_kind": peak_kind,
                         "bytes_per_launch": BYTES_PER_PARTICLE_STEP * n_active},
            "step_breakdown_ms": {"push": push_avg_ms, "field": kt["field_ms_per_step"],
                                  "sort_amortised": sort_ms_mean / interval},
            "timed_window": window,
            "rr_cost": rr_cost,
            "runs_per_hour": 3600.0 / (2000 * ms_max / args.steps / 1e3) * ws,
            "thin_plasma": thin,
            "batched_scan": scan,
            "serving": serving,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "parity": parity,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
