"""The oracle's parallel timing build (OpenMP over the particles of each
species, per-thread currents added in thread order) against the serial
oracle: the same arithmetic per particle, so one step agrees to FP64
round-off and 300 laser-driven steps to round-off amplified by the
dynamics (measured ~1e-13 relative in the fields, ~1e-10 in the momenta)."""
import os

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def parallel():
    if not oracle.parallel_available():
        pytest.skip("no OpenMP C compiler")
    return True


def laser_foil(par, steps, ppc=64):
    o = oracle.OracleSim(3, 200, rr_on=True, parallel=par)
    o.load_foil(0.2, 0.5, 64.0, 1, 1.0, ppc, 7)
    o.inject_laser(200.0, oracle.LP, oracle.ENV_SIN2, 3.0)
    o.step(steps)
    return o


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("steps,tol_f,tol_p", [(1, 1e-14, 1e-14), (300, 1e-9, 1e-8)])
def test_parallel_build_matches_serial(parallel, steps, tol_f, tol_p):
    if oracle.threads() < 2:
        pytest.skip("one thread only")
    # 6400 particles per species: above the size the parallel loop starts at
    a, b = laser_foil(False, steps), laser_foil(True, steps)
    for c in range(8):
        assert rel(b.field(c), a.field(c)) <= tol_f, c
    for sp in (0, 1):
        pa, pb = a.particles(sp), b.particles(sp)
        assert np.array_equal(pa["flag"], pb["flag"])
        for k in ("x", "px", "py", "pz"):
            assert rel(pb[k], pa[k]) <= tol_p, (sp, k)
    np.testing.assert_allclose(b.energy(), a.energy(), rtol=tol_f, atol=tol_f * a.energy()[4])
    if steps > 1:
        assert np.std(a.particles(0)["px"]) > 0.3  # the laser has driven the electrons


def test_parallel_build_drops_no_particle_block(parallel, monkeypatch):
    """Several thread counts (blocks of uneven size) give the same run."""
    res = []
    for t in ("2", "3", "5"):
        monkeypatch.setenv("OMP_NUM_THREADS", t)
        # the thread count is read when the shared object starts its runtime;
        # run each count in its own process
        import subprocess
        import sys

        code = ("import sys; sys.path.insert(0, %r); import oracle, numpy as np; "
                "o = oracle.OracleSim(3, 200, rr_on=True, parallel=True); "
                "o.load_foil(0.2, 0.5, 64.0, 1, 1.0, 64, 7); o.inject_laser(200.0, 0, 0, 3.0); o.step(20); "
                "print(oracle.threads()); np.save(sys.argv[1], np.concatenate([o.field(c) for c in range(8)]))"
                % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        out = os.path.join(os.environ.get("TMPDIR", "/tmp"), "omp_%s_%d.npy" % (t, os.getpid()))
        r = subprocess.run([sys.executable, "-c", code, out], capture_output=True, text=True,
                           env=dict(os.environ, OMP_NUM_THREADS=t))
        assert r.returncode == 0, r.stderr
        assert r.stdout.strip() == t
        res.append(np.load(out))
        os.unlink(out)
    ref = laser_foil(False, 20)
    f = np.concatenate([ref.field(c) for c in range(8)])
    for r in res:
        assert rel(r, f) <= 1e-12
