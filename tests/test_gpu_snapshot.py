"""GPU parity of the skin-layer snapshot (friction coefficient d of
Eq. (damping), quantum parameter chi) against the FP64 oracle.

Single precision evaluates the bracket of Eq. (damping) as a sum of squares
(f_L^2 + |p x f_L|^2), the oracle its literal form; both cancel differently
for co-moving particles, so each value is judged against the size of the
terms, eps (gamma^2 |E|^2 + |p|^2 |B|^2) with the field scale F: per particle
|d_gpu - d_oracle| <= 2e-5 eps (1 + |p|^2) F^2.
"""
import numpy as np
import pytest

import oracle
from tests import synth
from tests.test_gpu_parity import laser_foil_pair, pair

pytestmark = pytest.mark.gpu
EPS = oracle.eps_rr(0.8)
ECR = oracle.ecr(0.8)


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


def test_snapshot_random_state(picrr):
    g, o = pair(picrr, length_lambda=8, cells_per_lambda=100, rr_on=True)
    nx, F = g.nx, 80.0
    fields = synth.random_fields(nx, scale=F, seed=5)
    for s in (g, o):
        s.set_fields(*fields)
    for sp, (n, q, m, ps) in enumerate([(4999, -1.0, 1.0, 60.0), (3001, 1.0, 1836.15267343, 2.0)]):
        cell, off, px, py, pz = synth.random_particles(n, 2, nx - 2, pscale=ps, seed=20 + sp)
        for s in (g, o):
            s.load_particles(sp, cell, off, px, py, pz, 0.01, q, m)
    for sp in (0, 1):
        gs, os_ = g.snapshot(sp, chi_flag=0.0), o.snapshot(sp)
        p = o.particles(sp)
        p2 = p["px"] ** 2 + p["py"] ** 2 + p["pz"] ** 2
        floor = EPS * (1.0 + p2) * F ** 2
        assert np.max(np.abs(gs["d"] - os_["d"]) / floor) <= 2e-5
        assert np.max(np.abs(gs["chi"] - os_["chi"]) / (np.sqrt(floor / EPS) / ECR)) <= 2e-5
        assert gs["d_max"] == pytest.approx(np.max(os_["d"]), rel=1e-5)
        assert gs["chi_max"] == pytest.approx(np.max(os_["chi"]), rel=1e-5)
        assert gs["d_max"] == np.max(gs["d"]) and gs["chi_max"] == np.max(gs["chi"])
        np.testing.assert_allclose(gs["px"], p["px"], rtol=0, atol=0)
        np.testing.assert_allclose(gs["pperp"], np.hypot(p["py"], p["pz"]), rtol=1e-12)
        assert gs["n_flagged"] == gs["n"]  # chi >= 0 for every particle
        # the count above a threshold: equal to the oracle's away from rounding ties
        flag = float(np.median(os_["chi"]))
        near = np.sum(np.abs(os_["chi"] - flag) <= 1e-4 * flag)
        got = g.snapshot(sp, chi_flag=flag, per_particle=False)["n_flagged"]
        assert abs(got - int(np.sum(os_["chi"] >= flag))) <= near
    g.close()


def test_snapshot_after_laser_steps(picrr):
    g, o = laser_foil_pair(picrr, rr=True, pol=0, a0=300.0)
    g.step(200)
    o.step(200)
    gs, os_ = g.snapshot(0), o.snapshot(0)
    assert np.max(os_["d"]) > 1e-3  # the pulse drives the skin layer
    assert gs["d_max"] == pytest.approx(np.max(os_["d"]), rel=1e-3)
    assert gs["chi_max"] == pytest.approx(np.max(os_["chi"]), rel=1e-3)
    big = os_["d"] > 1e-3 * np.max(os_["d"])
    rel = np.abs(gs["d"][big] - os_["d"][big]) / os_["d"][big]
    assert np.median(rel) < 1e-3
    g.close()
