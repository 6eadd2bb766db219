"""Pins of the oracle's skin-layer observables: the friction coefficient d of
Eq. (damping) and the quantum parameter chi (classical validity, Sec. 2).

- in crossed fields of a plane wave (E = a y, B = a z) the bracket of
  Eq. (damping) is a^2 (1 - v_x)^2 for any velocity, which gives the limits the
  paper states after Eq. (damping): d -> 0 for v_x -> 1, d -> 4 eps gamma^2 a^2
  for v_x -> -1 and d = eps gamma^2 a^2 for transverse motion;
- for any uniform fields, gamma^2 [f_L^2 - (v.f_L)^2] equals the Lorentz
  invariant |gamma E + p x B|^2 - (p.E)^2 (the spatial part of F u squared
  minus its time part), computed here with numpy from the same vectors;
- linear fields are gathered exactly, so the same invariant holds with the
  fields evaluated at the particle's position;
- d >= 0, d = eps (chi E_cr)^2, frozen particles give 0.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleSim

EPS = oracle.eps_rr(0.8)
ECR = oracle.ecr(0.8)


def test_ecr_value():
    # E_cr / (m omega c / e) = m c^2 / (hbar omega) = lambda / (2 pi lambda_C); 3.297e5 at 0.8 um
    assert ECR == pytest.approx(0.8 / (2 * math.pi * 3.8615926796e-7), rel=1e-12)
    assert 3.29e5 < ECR < 3.30e5


def load(s, sp, cells, offs, p, w=0.01):
    q, m = (-1.0, 1.0) if sp == 0 else (1.0, 1836.15267343)
    s.load_particles(sp, cells.astype(np.int32), offs, p[:, 0], p[:, 1], p[:, 2], w, q, m)


def test_plane_wave_crossed_fields_closed_form():
    s = OracleSim(4, 50, 0.9, rr_on=True, source_node=8)
    nx, a = s.nx, 250.0
    s.set_fields(np.zeros(nx), np.full(nx + 1, a), np.zeros(nx + 1), np.zeros(nx), np.full(nx, a))
    rng = np.random.default_rng(3)
    n = 64
    p = rng.normal(scale=100.0, size=(n, 3))
    p[0] = [-300.0, 0, 0]   # counter-propagating: d -> 4 eps gamma^2 a^2
    p[1] = [300.0, 0, 0]    # co-moving: d -> 0
    p[2] = [0, 0, 300.0]    # transverse: d = eps gamma^2 a^2
    p[3] = [0, 300.0, 0]
    cells = rng.integers(5, nx - 5, n)
    offs = rng.random(n)
    load(s, 0, cells, offs, p)
    out = s.snapshot(0)
    g = np.sqrt(1 + np.sum(p * p, 1))
    vx = p[:, 0] / g
    ref = EPS * g ** 2 * a ** 2 * (1 - vx) ** 2
    # the literal bracket of Eq. (damping) cancels for co-moving particles:
    # judge against the size of its terms, eps gamma^2 a^2
    scale = EPS * g ** 2 * a ** 2
    assert np.max(np.abs(out["d"] - ref) / scale) <= 1e-12
    assert np.max(np.abs(out["chi"] * ECR - g * a * (1 - vx)) / (g * a)) <= 1e-6
    assert out["d"][0] == pytest.approx(4 * EPS * g[0] ** 2 * a ** 2, rel=2e-5)
    assert out["d"][1] < 1e-9 * out["d"][0]
    assert out["d"][2] == pytest.approx(EPS * g[2] ** 2 * a ** 2, rel=1e-12)
    assert out["d"][3] == pytest.approx(EPS * g[3] ** 2 * a ** 2, rel=1e-12)


def invariant(E, B, p):
    g = np.sqrt(1 + np.sum(p * p, -1))
    sp = g[:, None] * E + np.cross(p, B)
    return np.sum(sp * sp, -1) - np.sum(p * E, -1) ** 2


def test_uniform_fields_lorentz_invariant():
    s = OracleSim(4, 50, 0.9, rr_on=True, source_node=8)
    nx = s.nx
    E = np.array([12.0, -40.0, 25.0])
    B = np.array([0.0, 31.0, -18.0])
    s.set_fields(np.full(nx, E[0]), np.full(nx + 1, E[1]), np.full(nx + 1, E[2]), np.full(nx, B[1]),
                 np.full(nx, B[2]))
    rng = np.random.default_rng(4)
    n = 200
    p = rng.normal(scale=30.0, size=(n, 3))
    cells = rng.integers(5, nx - 5, n)
    load(s, 1, cells, rng.random(n), p)
    out = s.snapshot(1)
    inv = invariant(np.tile(E, (n, 1)), np.tile(B, (n, 1)), p)
    np.testing.assert_allclose(out["d"], EPS * inv, rtol=1e-10)
    np.testing.assert_allclose(EPS * (out["chi"] * ECR) ** 2, out["d"], rtol=1e-10)
    assert np.all(out["d"] >= 0)


def test_linear_fields_at_the_particle():
    s = OracleSim(4, 50, 0.9, rr_on=True, source_node=8)
    nx, dx = s.nx, s.dx
    i = np.arange(nx + 1.0)
    j = np.arange(nx) + 0.5
    coef = {"Ex": (0.3, 0.11), "Ey": (-2.0, 0.7), "Ez": (1.5, -0.5), "By": (0.7, 0.3), "Bz": (-1.1, 0.2)}
    lin = lambda k, pos: coef[k][0] + coef[k][1] * pos
    s.set_fields(lin("Ex", j), lin("Ey", i), lin("Ez", i), lin("By", j), lin("Bz", j))
    rng = np.random.default_rng(6)
    n = 80
    cells = rng.integers(3, nx - 3, n)
    offs = rng.random(n)
    p = rng.normal(scale=20.0, size=(n, 3))
    load(s, 0, cells, offs, p)
    out = s.snapshot(0)
    xi = cells + offs
    E = np.stack([lin("Ex", xi), lin("Ey", xi), lin("Ez", xi)], 1)
    B = np.stack([np.zeros(n), lin("By", xi), lin("Bz", xi)], 1)
    np.testing.assert_allclose(out["d"], EPS * invariant(E, B, p), rtol=1e-9)


def test_frozen_particles_and_zero_fields():
    s = OracleSim(4, 50, 0.9, rr_on=True, source_node=8)
    nx = s.nx
    s.set_fields(np.full(nx, 5.0), np.full(nx + 1, 5.0), np.zeros(nx + 1), np.zeros(nx), np.full(nx, 5.0))
    p = np.array([[-50.0, 0.0, 0.0], [50.0, 0.0, 0.0]])
    load(s, 0, np.array([0, nx - 1]), np.array([0.001, 0.999]), p)
    s.step(1)  # both leave the box and freeze at the walls
    assert list(s.particles(0)["flag"]) == [-1, 1]
    out = s.snapshot(0)
    assert np.all(out["d"] == 0.0) and np.all(out["chi"] == 0.0)
    s2 = OracleSim(4, 50, 0.9, rr_on=True, source_node=8)
    load(s2, 0, np.array([10, 20]), np.array([0.3, 0.6]), np.array([[5.0, 1.0, 2.0], [0.0, 0.0, 0.0]]))
    out = s2.snapshot(0)  # no fields: no friction
    assert np.all(out["d"] == 0.0)
