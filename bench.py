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
BYTES_PER_PARTICLE_STEP = 40  # cell + offset + 3 momenta, read and written (int32 + 4 x fp32)


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
    """nvidia-smi sampler for the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

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


def oracle_sample(steps, ppc=50):
    """The FP64 oracle on the large run's grid and foil with ppc per species."""
    import oracle

    w = LARGE
    o = oracle.OracleSim(w["length_lambda"], w["cells_per_lambda"], w["cfl"], w["lambda_um"], w["rr_on"],
                         w["source_node"])
    o.load_foil(w["foil_x0"], w["foil_thickness"], w["ne"], 1, 1.0, ppc, w["seed"])
    o.inject_laser(w["a0"], w["pol"], 0, w["duration"])
    n_part = 2 * len(o.particles(0)["x"])
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    sample = ("large-run grid (200,000 cells) and foil with %d macro-particles per cell per species "
              "(%d particles), first %d steps, FP64, one thread" % (ppc, n_part, steps))
    return n_part * steps / dt, sample


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        oracle_sample(2)
    for _ in range(max(1, args.steps)):
        v, sample = oracle_sample(args.ref_steps)
        vals.append(v)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "large single run sample (oracle)", "cells": 200000},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def e2e_run(picrr, torch, device, steps, host):
    """Through the public C ABI with host buffers: create, upload the particles
    from pinned host memory, inject, step, read spectra + energy back."""
    w = LARGE
    t0 = time.perf_counter()
    s = make_sim(picrr, device)
    for sp in (0, 1):
        c, o, x, y, z = host[sp]
        s.load_particles_f32(sp, c, o, x, y, z, *host["species"][sp])
    s.inject_laser(w["a0"], w["pol"], 0, w["duration"])
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
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-steps", type=int, default=40)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
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
    sim = make_sim(picrr, local)
    sim.load_foil(w["foil_x0"], w["foil_thickness"], w["ne"], 1, 1.0, w["ppc"])
    sim.inject_laser(w["a0"], w["pol"], 0, w["duration"])
    stream = torch.cuda.current_stream()
    sim.set_stream(stream.cuda_stream)
    sim.step(args.warmup)
    st0 = sim.stats()
    n_active = st0["active_particles"]

    def barrier():
        if dist is not None:
            dist.barrier()

    clocks = Clocks(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    sim.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    st1 = sim.stats()
    n_active_end = st1["active_particles"]
    ms_max, total = aggregate(torch, dist, ms, float(n_active) * args.steps)
    value = total / (ms_max / 1e3)
    push_avg_ms = st1["push_ms"] / max(1, st1["timed_push_launches"])
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_PARTICLE_STEP * n_active / (push_avg_ms / 1e3) / 1e9
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    sim.close()

    e2e = None
    if not args.no_e2e:
        host = host_foil(np, torch)
        ev, h2d, d2h = e2e_run(picrr, torch, local, args.steps, host)
        e2e = {"value": ev, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps,
               "what": "pic_create + pic_load_particles_f32 from pinned host SoA + pic_inject_laser + "
                       "pic_step_n(steps) + pic_spectra + pic_energy, host wall clock"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, sample = oracle_sample(args.ref_steps)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "large single run: 200,000 cells (100 lambda, lambda/2000), 2-lambda H foil "
                                   "n_e=100 n_c, 8000 ppc/species (32M e + 32M p), CP a0=500, RR on",
                       "particles": n_active, "particles_end": n_active_end, "cells": 200000,
                       "sort_interval": w["sort_interval"],
                       "l2": "inputs larger than L2: 2.56 GB particle state streamed per step",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "k_push_deposit", "kernel_ms": push_avg_ms,
                         "peak_kind": peak_kind,
                         "bytes_per_launch": BYTES_PER_PARTICLE_STEP * n_active},
            "step_breakdown_ms": {"push": st1["push_ms"] / args.steps, "field": st1["field_ms"] / args.steps,
                                  "sort": st1["sort_ms"] / args.steps},
            "runs_per_hour": 3600.0 / (2000 * ms_max / args.steps / 1e3) * ws,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
