"""GPU single-electron integrators (pic_electron_scan) against the FP64
oracle's: the leapfrog pusher of Sec. 3 and RK4 on Eq. (3dLL) in analytic
plane waves, each in double precision on both sides (the paths share no
code; results agree to rounding: 1e-9 relative over 10^4 steps, since plane-
wave motion is not chaotic).  A scan over amplitude then reproduces the
paper's single-electron accuracy test (Sec. 3, last paragraph) on the GPU:
the leapfrog against RK4 on the full Eq. (3dLL) for p_x0 = -200, a0 = 350,
dt = 0.01 over 500/omega.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
EPS = oracle.eps_rr(0.8)


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


CASES = [
    dict(wave=0, a0=350.0, x0=0.0, p0=(-200.0, 0.0, 0.0)),
    dict(wave=1, a0=200.0, x0=0.3, p0=(-50.0, 10.0, -5.0)),
    dict(wave=2, a0=300.0, tau=40.0, x0=-1.0, p0=(0.0, 0.0, 0.0)),
    dict(wave=0, a0=20.0, x0=0.0, p0=(5.0, 0.0, 1.0)),
]


def close(a, b, rtol):
    scale = np.max(np.abs(b), axis=0) + 1.0
    return np.max(np.abs(a - b) / scale) <= rtol


@pytest.mark.parametrize("integrator,rr,deriv", [(0, True, False), (0, False, False), (1, True, True),
                                                 (1, True, False), (1, False, False)])
def test_scan_matches_oracle(picrr, integrator, rr, deriv):
    dt, n, every = 0.01, 10000, 100
    got = picrr.electron_scan(CASES, integrator=integrator, rr=rr, deriv=deriv, dt=dt, nsteps=n, every=every)
    for c, g in zip(CASES, got):
        if integrator == 0:
            ref = oracle.pw_leapfrog(c["wave"], c["a0"], c["x0"], np.array(c["p0"]), dt, n, every=every, eps=EPS,
                                     rr=rr, tau=c.get("tau", 0.0))
        else:
            ref = oracle.pw_rk4(c["wave"], c["a0"], c["x0"], np.array(c["p0"]), dt, n, every=every, eps=EPS, rr=rr,
                                deriv=deriv, tau=c.get("tau", 0.0))
        assert np.array_equal(g[:, 0], ref[:, 0])
        assert close(g[:, 1:], ref[:, 1:], 1e-9), (c, np.max(np.abs(g - ref)))


def test_paper_accuracy_test_on_gpu(picrr):
    """Leapfrog vs RK4 (full Eq. 3dLL, dt/10) for the paper's case and a scan
    of amplitudes around it: the relative displacement difference stays of
    the order the paper reports (~4e-4 at a0 = 350) and the p_x phase lag
    well below a period."""
    a0s = [200.0, 275.0, 350.0, 425.0, 500.0]
    T, dt = 500.0, 0.01
    cases = [dict(wave=0, a0=a, x0=0.0, p0=(-200.0, 0.0, 0.0)) for a in a0s]
    lf = picrr.electron_scan(cases, integrator=0, rr=True, dt=dt, nsteps=int(T / dt), every=50)
    rk = picrr.electron_scan(cases, integrator=1, rr=True, deriv=True, dt=dt / 10, nsteps=int(T / dt) * 10,
                             every=500)
    res = {}
    for k, a in enumerate(a0s):
        x_l, x_r = lf[k, -1, 1], rk[k, -1, 1]
        rel = abs(x_l - x_r) / abs(x_r)
        # p_x phase: time shift minimising the mismatch over the last 20/omega
        sel = lf[k, :, 0] > T - 20
        t_l, px_l = lf[k, sel, 0] - 0.5 * dt, lf[k, sel, 2]
        t_r, px_r = rk[k, :, 0], rk[k, :, 2]
        shifts = np.linspace(-3.0, 3.0, 601)
        mis = [np.sum((np.interp(t_l + s, t_r, px_r) - px_l) ** 2) for s in shifts]
        res[a] = (rel, abs(shifts[int(np.argmin(mis))]) / (2 * math.pi))
    print("a0: (relative displacement difference, p_x phase lag in periods)", res)
    # the paper's case: errors of the size it reports (~4e-4, ~0.1 period), as the oracle pin holds them
    assert res[350.0][0] < 2.5 * 4e-4 and res[350.0][1] < 2 * 0.1, res[350.0]
    # the scheme is first order where RR is strong: the errors grow with the amplitude but stay bounded
    assert all(r < 1e-2 and lag < 0.5 for r, lag in res.values()), res


def test_scan_throughput_smoke(picrr):
    # thousands of cases in one launch
    rng = np.random.default_rng(0)
    cases = [dict(wave=int(rng.integers(0, 2)), a0=float(rng.uniform(100, 600)), x0=0.0,
                  p0=tuple(rng.normal(scale=50.0, size=3))) for _ in range(4096)]
    out = picrr.electron_scan(cases, integrator=1, rr=True, deriv=True, dt=0.01, nsteps=2000, every=2000)
    assert out.shape == (4096, 1, 5) and np.all(np.isfinite(out))
    with pytest.raises(picrr.PicError):
        picrr.electron_scan(cases[:2], integrator=0, deriv=True)  # the derivative term is an RK4 option
