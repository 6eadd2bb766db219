"""GPU parity on whole runs and at full benchmark size.

- small single run (20 lambda, lambda/200, 12,800 + 12,800 particles, LP a0 = 200,
  4211 steps = 20 periods): energy bookkeeping within 1e-3 of the injected
  energy; ion spectra of 1024-seed ensembles (the oracle's stored): peak,
  FWHM, mean ion energy and mean radiated energy within 2 %;
- paper-scale grid (60,000 cells, 400 + 400 particles per cell) over its first
  500 steps, with the foil and a short pulse placed so that the pulse peak
  reaches the foil inside the window;
- the large benchmark run (200,000 cells, 32M + 32M particles) in the launch
  configuration bench.py times: sampled particles recomputed one by one by
  the oracle from the GPU's own fields, plus Gauss's law over the whole grid.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests.spectrum_stats import balance, peak_fwhm

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


SMALL = dict(length_lambda=20, cells_per_lambda=200, cfl=0.95, lambda_um=0.8, rr_on=True, source_node=8)
SMALL_STEPS = 4211
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_small_run_ensemble.json")


def test_small_single_run_energy_bookkeeping(picrr):
    """Seed 1 on both sides: the time-centred energy balance (field + kinetic
    + radiated + outflow = injected) holds within 1e-3 of the injected energy
    along the whole run, on the GPU as in the oracle, and the two balances
    agree within 1e-3."""
    g = picrr.Sim(seed=1, sort_interval=8, **SMALL)
    o = oracle.OracleSim(**SMALL)
    g.load_foil(10.0, 1.0, 64.0, 1, 1.0, 64)
    o.load_foil(10.0, 1.0, 64.0, 1, 1.0, 64, 1)
    for s in (g, o):
        s.inject_laser(200.0, picrr.LP, picrr.ENV_SIN2, 10.0)
    bg, eg = balance(g, SMALL_STEPS, 199)
    bo, eo = balance(o, SMALL_STEPS, 199)
    g.close()
    o.close()
    u_in = eo[4]
    assert u_in > 1e5 and eg[4] == pytest.approx(u_in, rel=1e-5)
    assert np.max(np.abs(bo)) < 1e-3 * u_in
    assert np.max(np.abs(bg)) < 1e-3 * u_in
    assert np.max(np.abs(bg - bo)) < 1e-3 * u_in


def test_small_run_seed_ensembles_within_2_percent(picrr):
    """Full runs are chaotic: a single- and a double-precision run from the
    same seed end as different as runs from different seeds.  So the
    ion spectra are compared as ensembles over foil seeds: the oracle's
    (stored by tests/golden/make_oracle_ensemble.py, which calls only the
    oracle) against the GPU's for the same seeds, all stepped as one batch.
    With 1024 seeds the ensemble-to-ensemble spread is a few tenths of a
    percent, so the peak energy, the FWHM and the mean ion energy are held
    to 2 %, and the mean radiated energy too."""
    G = json.load(open(GOLDEN))
    seeds = G["seeds"]
    nb, e_max = G["bins"]["n"], G["bins"]["e_max"]
    assert len(seeds) >= 1024 and G["steps"] == SMALL_STEPS
    b = picrr.Batch(SMALL["cells_per_lambda"], max_runs=len(seeds), sort_interval=8)
    f, la = G["foil"], G["laser"]
    ids = [b.add_run(SMALL["length_lambda"], f["x0"], f["thickness"], f["ne"], la["a0"], la["polarization"],
                     la["duration"], G["steps"], rr_on=True, ppc=f["ppc"], seed=s) for s in seeds]
    while b.step(4096) > 0:
        pass
    spec_g = sum(b.spectra(r, picrr.ION, nb, 0.0, e_max)[0] for r in ids)
    rad_g = np.mean([b.energy(r)[3] for r in ids])
    b.close()
    spec_o = np.array(G["spectrum_sum"])
    rad_o = np.mean(G["radiated"])
    pg, fg = peak_fwhm(spec_g, 0.0, e_max)
    po, fo = peak_fwhm(spec_o, 0.0, e_max)
    assert po > 150.0  # the foil has been accelerated
    assert pg == pytest.approx(po, rel=0.02), (pg, po)
    assert fg == pytest.approx(fo, rel=0.02), (fg, fo)
    e = (np.arange(nb) + 0.5) * e_max / nb
    assert (spec_g @ e) / spec_g.sum() == pytest.approx((spec_o @ e) / spec_o.sum(), rel=0.02)
    assert rad_g == pytest.approx(rad_o, rel=0.02)


PAPER_KW = dict(length_lambda=60, cells_per_lambda=1000, cfl=0.95, lambda_um=0.8, source_node=8)
PAPER_CASES = [(a0, pol, rr) for a0 in (200.0, 350.0, 500.0) for pol in (0, 1) for rr in (True, False)]
# the pulse front reaches the foil (node 100) after ~97 steps; by step 250 the
# rising front (a ~ 0.5 a0 in vacuum) has driven the skin layer relativistically
EARLY_STEPS = 250


def oracle_paper_scale(case):
    """The oracle's first 500 steps of one paper-scale case (process-pool worker)."""
    import oracle as orc

    a0, pol, rr = case
    o = orc.OracleSim(rr_on=rr, **PAPER_KW)
    o.load_foil(0.1, 1.0, 90.0, 1, 1.0, 400, 11)
    o.inject_laser(a0, pol, orc.ENV_SIN2, 0.6)
    o.step(EARLY_STEPS)
    early = o.particles(0)
    o.step(500 - EARLY_STEPS)
    out = dict(fields=[o.field(c) for c in range(5)], px=o.particles(0)["px"],
               early=[early[k] for k in ("px", "py", "pz")])
    o.close()
    return out


def test_paper_scale_grid_first_500_steps(picrr):
    """The paper-scale grid (60,000 cells, 400 + 400 particles per cell) for
    a0 in {200, 350, 500}, LP and CP, RR on and off: fields after 500 steps
    within 1e-4 (relative L2 per group) and electron momenta within 1e-4 in
    the median, and every electron's momentum after the first 250 steps (the
    front has then driven the skin layer for ~150 steps) within 1e-4 in the
    R12 norm.  A 0.6-period sin^2 pulse peaks 0.3 periods (300 cells) behind
    its front, so its peak reaches the foil inside the window."""
    import concurrent.futures as cf
    import multiprocessing as mp

    with cf.ProcessPoolExecutor(max_workers=min(len(PAPER_CASES), os.cpu_count() or 4),
                                mp_context=mp.get_context("spawn")) as ex:
        ref = list(ex.map(oracle_paper_scale, PAPER_CASES))
    for (a0, pol, rr), o in zip(PAPER_CASES, ref):
        g = picrr.Sim(seed=11, sort_interval=8, rr_on=rr, **PAPER_KW)
        g.load_foil(0.1, 1.0, 90.0, 1, 1.0, 400)
        g.inject_laser(a0, pol, picrr.ENV_SIN2, 0.6)
        g.step(EARLY_STEPS)
        e = g.particles(0)
        pg = np.stack([e["px"], e["py"], e["pz"]], 1)
        po = np.stack(o["early"], 1)
        scale = np.maximum(np.linalg.norm(po, axis=1), 1e-3 * a0 * g.dt)
        err = np.max(np.abs(pg - po), axis=1) / scale
        assert np.max(err) <= 1e-4, (a0, pol, rr, float(np.max(err)), float(np.max(np.abs(po))))
        assert np.max(np.abs(po)) > 1.0  # the front has driven the skin layer relativistically
        g.step(500 - EARLY_STEPS)
        for comps in ((picrr.EY, picrr.EZ), (picrr.BY, picrr.BZ), (picrr.EX,)):
            a = np.concatenate([g.field(c) for c in comps])
            b = np.concatenate([o["fields"][c] for c in comps])
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), (a0, pol, rr, comps)
        px_g = g.particles(0)["px"]
        g.close()
        assert np.max(np.abs(o["px"])) > 0.02 * a0  # the pulse has driven the skin layer
        d = np.abs(px_g - o["px"]) / (1.0 + np.abs(o["px"]))
        assert np.median(d) < 1e-4, (a0, pol, rr)


def test_large_run_sampled_against_oracle(picrr):
    # the benchmark's run and launch configuration
    import bench

    w = bench.LARGE
    g = bench.make_sim(picrr, 0)
    g.load_foil(w["foil_x0"], w["foil_thickness"], w["ne"], 1, 1.0, w["ppc"])
    g.inject_laser(w["a0"], w["pol"], picrr.ENV_SIN2, w["duration"])
    g.tune_shapes(48)  # the launch shapes the benchmark times, picked the same way (its trials are real steps)
    g.step(4000 - g.stats()["steps"])  # the front reaches the foil after ~520 steps; 4000 steps: a ~ 0.07 a0 in it
    fields = [g.field(c) for c in range(5)]
    before = [g.particles(sp) for sp in (0, 1)]
    g.step(1)
    after = [g.particles(sp) for sp in (0, 1)]
    nx, dx = g.nx, g.dx
    assert len(before[0]["x"]) == 32_000_000
    rng = np.random.default_rng(0)
    kw = dict(length_lambda=w["length_lambda"], cells_per_lambda=w["cells_per_lambda"], cfl=w["cfl"],
              lambda_um=w["lambda_um"], rr_on=w["rr_on"], source_node=w["source_node"])
    o = oracle.OracleSim(**kw)
    o.set_fields(*fields)
    idx = {}
    species = {0: (w["ne"] / w["ppc"], -1.0, 1.0), 1: (w["ne"] / w["ppc"], 1.0, 1836.15267343)}
    for sp in (0, 1):
        b = before[sp]
        # sample: half uniformly, half among the most strongly driven particles
        strong = np.argsort(-np.abs(b["px"]))[:10000]
        pick = np.unique(np.concatenate([rng.choice(len(b["x"]), 10000, replace=False), strong]))
        idx[sp] = pick
        xi = b["x"][pick] / dx
        cell = np.floor(xi).astype(np.int32)
        off = xi - cell
        o.load_particles(sp, cell, off, b["px"][pick], b["py"][pick], b["pz"][pick], *species[sp])
    o.step(1)
    for sp in (0, 1):
        po = o.particles(sp)
        a = after[sp]
        pg = np.stack([a["px"][idx[sp]], a["py"][idx[sp]], a["pz"][idx[sp]]], 1)
        pr = np.stack([po["px"], po["py"], po["pz"]], 1)
        scale = np.maximum(np.linalg.norm(pr, axis=1), 1e-3 * w["a0"] * g.dt)
        err = np.max(np.abs(pg - pr), axis=1) / scale
        assert np.max(err) <= 1e-5, (sp, np.max(err))
        assert np.max(np.abs(a["x"][idx[sp]] - po["x"])) <= 2e-6 * dx
    # the laser is in the foil: skin-layer electrons carry transverse momentum
    assert max(np.max(np.abs(before[0]["py"])), np.max(np.abs(before[0]["pz"]))) > 1.0
    # Gauss's law on the whole grid after the step (all 64M particles)
    rho = np.zeros(nx + 3)
    for sp, q in ((0, -1.0), (1, 1.0)):
        xi = after[sp]["x"] / dx
        c = np.floor(xi).astype(np.int64)
        f = xi - c
        rho += q * species[sp][0] * (np.bincount(c, weights=1 - f, minlength=nx + 3)[: nx + 3]
                                     + np.bincount(c + 1, weights=f, minlength=nx + 3)[: nx + 3])
    ex = g.field(picrr.EX)
    div = (ex[1:] - ex[:-1]) / dx
    assert np.max(np.abs(div - rho[1:nx])) <= 1e-4 * np.max(np.abs(rho[: nx + 1]))
