"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances (single-precision particles and fields):
  - momenta after one step: per particle, max-norm difference <= 1e-5 of
    max(|p|, 1e-3 F dt), F the field scale;
  - fields after 200 steps: relative L2 per component <= 1e-4;
  - full runs (tests/test_gpu_fullrun.py): energy bookkeeping within 1e-3 of
    the injected energy; ion spectra compared as 1024-seed ensembles (full
    runs are chaotic): peak, FWHM and mean energy within 2 %.
"""
import math

import numpy as np
import pytest

import oracle
from tests import synth

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


def pair(picrr, seed=1, sort_interval=8, **kw):
    kw.setdefault("cfl", 0.95)
    kw.setdefault("lambda_um", 0.8)
    kw.setdefault("source_node", 8)
    g = picrr.Sim(seed=seed, sort_interval=sort_interval, **kw)
    o = oracle.OracleSim(**kw)
    return g, o


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def check_momenta(pg, po, fscale, dt, tol=1e-5):
    p_g = np.stack([pg["px"], pg["py"], pg["pz"]], 1)
    p_o = np.stack([po["px"], po["py"], po["pz"]], 1)
    scale = np.maximum(np.linalg.norm(p_o, axis=1), 1e-3 * fscale * dt)
    err = np.max(np.abs(p_g - p_o), axis=1) / scale
    assert np.max(err) <= tol, (np.max(err), np.argmax(err))
    assert rel_l2(p_g, p_o) <= tol
    return np.max(err)


@pytest.mark.parametrize("rr", [True, False])
def test_one_step_random_particles_and_fields(picrr, rr):
    # ragged counts (not multiples of 4 or of a unit), cells over the whole box
    nx_l, cpl = 8, 100
    g, o = pair(picrr, length_lambda=nx_l, cells_per_lambda=cpl, rr_on=rr)
    nx = g.nx
    F = synth.random_fields(nx, scale=80.0, seed=5)
    for s in (g, o):
        s.set_fields(*F)
    parts = {}
    for sp, (n, q, m, w) in enumerate([(4999, -1.0, 1.0, 0.01), (3001, 1.0, 1836.15267343, 0.01)]):
        cell, off, px, py, pz = synth.random_particles(n, 2, nx - 2, pscale=60.0 if sp == 0 else 2.0,
                                                       seed=10 + sp)
        parts[sp] = (cell, off)
        for s in (g, o):
            s.load_particles(sp, cell, off, px, py, pz, w, q, m)
    g.step(1)
    o.step(1)
    for sp in (0, 1):
        pg, po = g.particles(sp), o.particles(sp)
        check_momenta(pg, po, 80.0, g.dt)
        assert np.max(np.abs(pg["x"] - po["x"])) <= 2e-6 * g.dx
        assert np.array_equal(pg["flag"], po["flag"])
    for comp in range(8):
        a, b = g.field(comp), o.field(comp)
        assert rel_l2(a, b) <= 2e-6, comp
    if rr:
        eg, eo = g.energy(), o.energy()
        assert eg[3] == pytest.approx(eo[3], rel=1e-4)


@pytest.mark.parametrize("nx", [100, 255, 256, 257, 511, 512, 513, 1025])
def test_one_step_fields_at_every_node_across_block_edges(picrr, nx):
    # the Yee kernel tiles the grid into blocks of a power-of-two number of nodes that
    # recompute their neighbours' guard values: grids just below, at and above a multiple
    # of the block, and shorter than one block, compared node by node after one step
    g, o = pair(picrr, length_lambda=nx / 100.0, cells_per_lambda=100, rr_on=True)
    assert g.nx == nx
    F = synth.random_fields(nx, scale=50.0, seed=nx)
    for s in (g, o):
        s.set_fields(*F)
    for sp, (n, q, m) in enumerate([(3 * nx + 7, -1.0, 1.0), (nx + 3, 1.0, 1836.15267343)]):
        cell, off, px, py, pz = synth.random_particles(n, 2, nx - 2, pscale=30.0 if sp == 0 else 1.0, seed=nx + sp)
        for s in (g, o):
            s.load_particles(sp, cell, off, px, py, pz, 0.01, q, m)
    g.step(1)
    o.step(1)
    for comp in range(8):
        a, b = g.field(comp), o.field(comp)
        assert np.max(np.abs(a - b)) <= 4e-6 * max(np.max(np.abs(b)), 1e-30), (comp, np.argmax(np.abs(a - b)))


@pytest.mark.parametrize("ppt", [2, 4])
def test_one_step_dense_tiles_split_into_units(picrr, ppt):
    """Dense cells (about 250 particles each): every 64-cell tile splits into
    units of 1024 particles whose ends fall inside the slots of 2 or 4
    particles a thread takes, so the partial-slot loads and stores at unit
    boundaries and the merged warp records of crowded cells are all on the
    path; one step against the oracle."""
    g, o = pair(picrr, length_lambda=4, cells_per_lambda=100, rr_on=True)
    nx = g.nx
    F = synth.random_fields(nx, scale=80.0, seed=6)
    for s in (g, o):
        s.set_fields(*F)
    for sp, (n, q, m, w) in enumerate([(20011, -1.0, 1.0, 0.002), (19997, 1.0, 1836.15267343, 0.002)]):
        cell, off, px, py, pz = synth.random_particles(n, 150, 230, pscale=60.0 if sp == 0 else 2.0, seed=20 + sp)
        for s in (g, o):
            s.load_particles(sp, cell, off, px, py, pz, w, q, m)
    g.set_shapes(1024, 8, ppt)
    assert g.stats()["n_units"] >= 2 * (20000 // 1024)  # both species split into many units
    g.step(1)
    o.step(1)
    for sp in (0, 1):
        pg, po = g.particles(sp), o.particles(sp)
        check_momenta(pg, po, 80.0, g.dt)
        assert np.max(np.abs(pg["x"] - po["x"])) <= 2e-6 * g.dx
        assert np.array_equal(pg["flag"], po["flag"])
    for comp in range(8):
        a, b = g.field(comp), o.field(comp)
        assert rel_l2(a, b) <= 2e-6, comp
    eg, eo = g.energy(), o.energy()
    assert eg[3] == pytest.approx(eo[3], rel=1e-4)


def laser_foil_pair(picrr, rr=True, pol=0, a0=200.0, ne=64.0, ppc=32, sort_interval=8, seed=7):
    g, o = pair(picrr, seed=seed, sort_interval=sort_interval, length_lambda=3, cells_per_lambda=200,
                rr_on=rr)
    g.load_foil(0.2, 0.5, ne, 1, 1.0, ppc)
    o.load_foil(0.2, 0.5, ne, 1, 1.0, ppc, seed)
    for s in (g, o):
        s.inject_laser(a0, pol, 0, 3.0)
    return g, o


@pytest.mark.parametrize("rr,pol", [(True, 0), (True, 1), (False, 0)])
def test_fields_after_200_steps(picrr, rr, pol):
    g, o = laser_foil_pair(picrr, rr=rr, pol=pol)
    g.step(200)
    o.step(200)
    groups = {"Eperp": (picrr.EY, picrr.EZ), "Bperp": (picrr.BY, picrr.BZ), "Ex": (picrr.EX,)}
    for name, comps in groups.items():
        a = np.concatenate([g.field(c) for c in comps])
        b = np.concatenate([o.field(c) for c in comps])
        assert rel_l2(a, b) <= 1e-4, (name, rel_l2(a, b))
    pe_g, pe_o = g.particles(0), o.particles(0)
    assert np.std(pe_o["px"]) > 0.3  # the electrons have been driven (CP drives them least)
    eg, eo = g.energy(), o.energy()
    np.testing.assert_allclose(eg[[0, 1, 2, 4, 5]], eo[[0, 1, 2, 4, 5]], rtol=2e-4, atol=1e-6 * eo[4])
    if rr:
        assert eg[3] == pytest.approx(eo[3], rel=2e-3)


def charge_density(x, dx, nx, qw):
    """rho on nodes from positions with the linear shape (test-side check)."""
    xi = x / dx
    c = np.floor(xi).astype(int)
    f = xi - c
    rho = np.zeros(nx + 3)
    np.add.at(rho, c, qw * (1 - f))
    np.add.at(rho, c + 1, qw * f)
    return rho[: nx + 1]


def test_gpu_gauss_law(picrr):
    g, _ = laser_foil_pair(picrr)
    g.step(300)
    e, i = g.particles(0), g.particles(1)
    w = 64.0 / 32
    rho = charge_density(e["x"], g.dx, g.nx, -w) + charge_density(i["x"], g.dx, g.nx, w)
    ex = g.field(picrr.EX)
    div = (ex[1:] - ex[:-1]) / g.dx
    err = np.max(np.abs(div - rho[1:-1])) / np.max(np.abs(rho))
    assert np.max(np.abs(rho)) > 1.0
    assert err <= 1e-4, err


def test_determinism_bit_identical(picrr):
    runs = []
    for _ in range(2):
        g, _o = laser_foil_pair(picrr)
        g.step(237)
        runs.append((g.particles(0), g.particles(1), [g.field(c) for c in range(8)], g.energy()))
        g.close()
    a, b = runs
    for sp in (0, 1):
        for k in ("x", "px", "py", "pz", "flag"):
            assert np.array_equal(a[sp][k], b[sp][k]), (sp, k)
    for c in range(8):
        assert np.array_equal(a[2][c], b[2][c]), c
    assert np.array_equal(a[3], b[3])


def test_sort_interval_changes_only_rounding(picrr):
    res = []
    for si in (1, 3, 16):
        g, _o = laser_foil_pair(picrr, sort_interval=si)
        g.step(160)
        res.append((np.concatenate([g.field(c) for c in range(5)]), g.particles(0)))
        assert g.stats()["sort_count"] == 160 // si
    for f, p in res[1:]:
        assert rel_l2(f, res[0][0]) <= 1e-5
        assert np.max(np.abs(p["px"] - res[0][1]["px"])) <= 1e-3 * (1 + np.max(np.abs(res[0][1]["px"])))


def test_vacuum_energy_balance(picrr):
    g, o = pair(picrr, length_lambda=6, cells_per_lambda=100, rr_on=True)
    for s in (g, o):
        s.inject_laser(50.0, picrr.CP, picrr.ENV_TRAPEZOID, 3.0, 1.0)
    n = int(10 * TWO_PI / g.dt)
    for _ in range(4):
        g.step(n // 4)
        o.step(n // 4)
        e, eo = g.energy(), o.energy()
        assert abs(e[0] - e[4] + e[5]) <= 2e-6 * max(e[4], 1.0)
        assert e[4] == pytest.approx(eo[4], rel=1e-5)
    assert e[5] > 0.99 * e[4]


def test_spectra_exact_bins(picrr):
    g, o = pair(picrr, length_lambda=4, cells_per_lambda=50)
    m = 1836.15267343
    rng = np.random.default_rng(3)
    # bin centres of 50 bins over [0, 500) MeV, energies stored as float momenta
    e_mev = (rng.integers(0, 50, 777) + 0.5) * 10.0
    gam = 1 + e_mev / (m * 0.51099895)
    px = np.float32(np.sqrt(gam**2 - 1)).astype(np.float64)
    n = len(px)
    cell = rng.integers(10, 190, n).astype(np.int32)
    off = np.full(n, 0.25)
    z = np.zeros(n)
    for s in (g, o):
        s.load_particles(1, cell, off, px, z, z, 0.5, 1.0, m)
    cg, _ = g.spectra(1, 50, 0.0, 500.0)
    co, _ = o.spectra(1, 50, 0.0, 500.0)
    np.testing.assert_allclose(cg, co, rtol=1e-14)
    assert cg.sum() > 0


def test_walls_freeze_like_oracle(picrr):
    g, o = pair(picrr, length_lambda=2, cells_per_lambda=50)
    nx = g.nx
    cell = np.array([nx - 1, nx - 2, 0, 1, 50], np.int32)
    off = np.array([0.9, 0.5, 0.1, 0.3, 0.5])
    px = np.array([40.0, 40.0, -40.0, -40.0, 0.0])
    z = np.zeros(5)
    for s in (g, o):
        s.load_particles(0, cell, off, px, z, z, 1e-3, -1.0, 1.0)
    g.step(5)
    o.step(5)
    pg, po = g.particles(0), o.particles(0)
    assert list(pg["flag"]) == list(po["flag"]) == [1, 1, -1, -1, 0]
    np.testing.assert_allclose(pg["x"], po["x"], rtol=0, atol=1e-6 * g.dx)


def test_state_errors_and_budget(picrr):
    g = picrr.Sim(length_lambda=2, cells_per_lambda=50)
    g.load_foil(0.5, 0.5, 10.0, 1, 1.0, 4)
    g.step(2)
    with pytest.raises(picrr.PicError) as e:
        g.inject_laser(1.0, 0, 0, 1.0)
    assert e.value.status == -2
    with pytest.raises(picrr.PicError) as e:
        g.load_foil(0.5, 0.5, 10.0, 1, 1.0, 4)
    assert e.value.status == -2
    st = g.stats()
    assert st["push_launches"] == 2 and st["steps"] == 2
    g.close()
    small = picrr.Sim(length_lambda=2, cells_per_lambda=50, hbm_budget_bytes=2 << 20)
    with pytest.raises(picrr.PicError) as e:
        small.load_foil(0.5, 1.0, 10.0, 1, 1.0, 4096)
    assert e.value.status == -3
    small.load_foil(0.5, 0.1, 10.0, 1, 1.0, 4)  # the failed call left the handle usable
    small.step(1)


def test_particle_upload_is_checked_on_the_device(picrr):
    """Uploaded particles are checked on the GPU: a cell outside the grid, an
    offset outside [0, 1) or a non-finite momentum is rejected and leaves the
    species unloaded; particles not in cell order are put in order (their
    read-out keeps the load order)."""
    g = picrr.Sim(length_lambda=2, cells_per_lambda=50)
    nx = g.nx
    n = 1001
    rng = np.random.default_rng(3)
    cell = np.sort(rng.integers(0, nx, n)).astype(np.int32)
    off = rng.random(n).astype(np.float32)
    p = rng.normal(size=(3, n)).astype(np.float32)
    bad = [("cell", cell.copy()), ("off", off.copy()), ("px", p[0].copy())]
    bad[0][1][500] = nx
    bad[1][1][7] = 1.0
    bad[2][1][1000] = np.inf
    for what, arr in bad:
        args = dict(cell=cell, off=off, px=p[0])
        args[what] = arr
        with pytest.raises(picrr.PicError) as e:
            g.load_particles_f32(0, args["cell"], args["off"], args["px"], p[1], p[2], 0.01, -1.0, 1.0)
        assert e.value.status == -1, what
    perm = rng.permutation(n)  # out of cell order: sorted on the way in
    g.load_particles_f32(0, cell[perm], off[perm], p[0][perm], p[1][perm], p[2][perm], 0.01, -1.0, 1.0)
    got = g.particles(0)
    np.testing.assert_array_equal(got["px"], p[0][perm])
    np.testing.assert_allclose(got["x"], (cell[perm] + off[perm].astype(np.float64)) * g.dx, rtol=1e-6)
    g.step(3)
    g.close()


def test_empty_and_single_species(picrr):
    g, o = pair(picrr, length_lambda=2, cells_per_lambda=50)
    cell, off, px, py, pz = synth.random_particles(5, 10, 90, pscale=3.0, seed=2)
    for s in (g, o):
        s.load_particles(0, cell, off, px, py, pz, 0.1, -1.0, 1.0)
        s.inject_laser(5.0, 0, 0, 1.0)
    g.step(40)
    o.step(40)
    check_momenta(g.particles(0), o.particles(0), 5.0, g.dt, tol=1e-4)
    assert g.particles(1)["x"].size == 0


def test_gpu_foil_generator_is_the_published_splitmix64(picrr):
    """The CUDA foil loader draws the same published SplitMix64 outputs as the
    oracle's (cells 0..4 of a one-particle-per-cell foil from cell 0, seed
    1234567): each offset is the output's top 24 bits over 2^24."""
    import json
    import os

    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "splitmix64_published.json")))
    g = picrr.Sim(length_lambda=1.0, cells_per_lambda=64, seed=gold["seed"])
    g.load_foil(0.0, 0.25, 1.0, 1, 1.0, 1)
    xi = g.particles(0)["x"] / g.dx
    g.close()
    for c, out in enumerate(gold["outputs"]):
        assert round((xi[c] - c) * 2 ** 24) == int(out) >> 40, c
