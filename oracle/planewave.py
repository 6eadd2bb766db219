"""Closed-form motion of one electron in a plane wave, with and without the
radiation-reaction force of Eq. (f_r) (Sec. 3), used to pin the oracle's
pusher.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For a wave E_perp(phi), B = x_hat x E, phi = t - x, travelling along +x, and
an electron (charge -1, mass 1) the light-front variable u = gamma - p_x obeys
(derived from Eq. f_r, with gamma^2 (1 - v_x) = ... identities below):

  Lorentz force only:  du/dphi = 0,  dp_perp/dphi = -E_perp
  with Eq. (f_r):      du/dphi = -eps u^2 |E_perp|^2,
                       dp_perp/dphi = -E_perp - eps u |E_perp|^2 p_perp
  field-derivative term of Eq. (3dLL) adds -eps u dE_perp/dphi to dp_perp/dphi
  and nothing to du/dphi.

Hence, with h(phi) = 1 + eps u0 int_{phi0}^{phi} |E_perp|^2:
  u = u0 / h,
  h p_perp = p_perp0 - int h E_perp dphi  [- eps u0 (E_perp(phi) - E_perp(phi0))],
  p_x = (1 + p_perp^2 - u^2) / (2 u),  gamma = u + p_x,
  dt/dphi = gamma / u,  dx/dphi = p_x / u.
The identities used are f_L x B - (v.E)E = -(1 - v_x)|E|^2 x_hat and
f_L^2 - (v.E)^2 = (1 - v_x)^2 |E|^2 in a plane wave.  Eps = 0 gives the
textbook figure-eight motion (drift speed a0^2/(4 + a0^2) for an electron
initially at rest in an LP wave with zero vector potential at the start).

The quadratures int |E|^2, int h E, int gamma/u, int p_x/u are evaluated by
scipy's adaptive DOP853 integrator at tight tolerance; nothing else is
integrated numerically.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq


def wave(kind: int, a0: float, tau: float, phi):
    """E_perp(phi) = (Ey, Ez) and its phi-derivative for the three wave kinds
    that ``or_planewave`` also implements (LP cos, CP, LP with sin^2 envelope)."""
    phi = np.asarray(phi, dtype=float)
    if kind == 0:
        ey, ez = a0 * np.cos(phi), 0.0 * phi
        dey, dez = -a0 * np.sin(phi), 0.0 * phi
    elif kind == 1:
        a = a0 / math.sqrt(2.0)
        ey, ez = a * np.cos(phi), a * np.sin(phi)
        dey, dez = -a * np.sin(phi), a * np.cos(phi)
    else:
        inside = (phi >= 0.0) & (phi <= tau)
        sn, cs = np.sin(np.pi * phi / tau), np.cos(np.pi * phi / tau)
        g, dg = sn * sn, 2.0 * sn * cs * np.pi / tau
        ey = np.where(inside, a0 * g * np.cos(phi), 0.0)
        dey = np.where(inside, a0 * (dg * np.cos(phi) - g * np.sin(phi)), 0.0)
        ez, dez = 0.0 * phi, 0.0 * phi
    return np.array([ey, ez]), np.array([dey, dez])


class ClosedForm:
    """Exact trajectory from initial data (t0, x0, p0), evaluated at any t >= t0."""

    def __init__(self, kind, a0, t0, x0, p0, eps=0.0, deriv=False, tau=0.0, t_max=100.0,
                 rtol=1e-13):
        self.kind, self.a0, self.tau, self.eps, self.deriv = kind, a0, tau, eps, deriv
        p0 = np.asarray(p0, dtype=float)
        g0 = math.sqrt(1.0 + p0 @ p0)
        self.u0 = g0 - p0[0]
        self.pp0 = p0[1:].copy()
        self.phi0 = t0 - x0
        self.E0, _ = wave(kind, a0, tau, self.phi0)
        self.t0, self.x0 = t0, x0

        def rhs(phi, y):
            # y = (I1, Iy, Iz, T, X) with I1 = int |E|^2, I = int h E
            E, _ = wave(kind, a0, tau, phi)
            h = 1.0 + eps * self.u0 * y[0]
            u, pp = self._state(phi, y)
            px = (1.0 + pp @ pp - u * u) / (2.0 * u)
            gam = u + px
            return [E @ E, h * E[0], h * E[1], gam / u, px / u]

        def hit(phi, y):
            return y[3] - t_max

        hit.terminal = True
        hit.direction = 1
        # phi advances at the rate u/gamma <= 1, so t_max bounds the phi range
        # only loosely; the terminal event stops the integration at t_max.
        span = (self.phi0, self.phi0 + 4.0 * (t_max - t0) * max(1.0, self.u0) + 10.0)
        self.sol = solve_ivp(rhs, span, [0.0, 0.0, 0.0, t0, x0], method="DOP853", rtol=rtol,
                             atol=1e-13, dense_output=True, events=hit)
        if self.sol.status < 0:
            raise RuntimeError("closed-form quadrature failed: " + self.sol.message)
        self.phi_end = self.sol.t[-1]

    def _state(self, phi, y):
        h = 1.0 + self.eps * self.u0 * y[0]
        u = self.u0 / h
        pp = self.pp0 - np.array([y[1], y[2]])
        if self.deriv:
            E, _ = wave(self.kind, self.a0, self.tau, phi)
            pp = pp - self.eps * self.u0 * (E - self.E0)
        return u, pp / h

    def at_phi(self, phi):
        y = self.sol.sol(phi)
        u, pp = self._state(phi, y)
        px = (1.0 + pp @ pp - u * u) / (2.0 * u)
        return dict(t=y[3], x=y[4], p=np.array([px, pp[0], pp[1]]), u=u, gamma=u + px)

    def phi_of_t(self, t):
        f = lambda ph: self.sol.sol(ph)[3] - t
        lo, hi = self.phi0, self.phi_end
        if f(hi) < 0:
            raise ValueError("t beyond the integrated range")
        return brentq(f, lo, hi, xtol=1e-14, rtol=1e-15, maxiter=500)

    def at_t(self, t):
        return self.at_phi(self.phi_of_t(t))


def leapfrog_start(kind, a0, x0, p0, dt, eps=0.0, tau=0.0, t_max=100.0, deriv=False):
    """Exact trajectory whose momentum at t = -dt/2 is p0; returns the closed
    form and the position it has at t = 0, i.e. consistent leapfrog initial
    data (x^0, p^{-1/2}) lying on one exact trajectory."""
    g0 = math.sqrt(1.0 + float(np.dot(p0, p0)))
    xa = x0 - 0.5 * dt * p0[0] / g0
    cf = ClosedForm(kind, a0, -0.5 * dt, xa, p0, eps=eps, tau=tau, t_max=t_max, deriv=deriv)
    return cf, cf.at_t(0.0)["x"]


def lp_drift_velocity(a0: float) -> float:
    """Mean longitudinal velocity of an electron starting at rest where the
    vector potential vanishes in an LP wave: a0^2 / (4 + a0^2)."""
    return a0 * a0 / (4.0 + a0 * a0)


def gamma_uniform_B_rr(gamma0: float, B: float, eps: float, t):
    """Electron gyrating in a uniform magnetic field B (momentum normal to B)
    with the force of Eq. (f_r): f_R = -eps B^2 gamma^2 v, so
    d gamma/dt = -eps B^2 (gamma^2 - 1), i.e.
    (gamma - 1)/(gamma + 1) = (gamma0 - 1)/(gamma0 + 1) exp(-2 eps B^2 t)."""
    k = (gamma0 - 1.0) / (gamma0 + 1.0) * np.exp(-2.0 * eps * B * B * np.asarray(t, dtype=float))
    return (1.0 + k) / (1.0 - k)
