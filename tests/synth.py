"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

Holds no arithmetic of the method: it only draws random particles and fields
(values rounded to single precision, so both paths start from identical
numbers).
"""
import numpy as np


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def random_particles(n, cell_lo, cell_hi, pscale, seed):
    """n particles with cells uniform in [cell_lo, cell_hi), offsets in [0, 1)
    and Gaussian momenta of width pscale, all single-precision values."""
    rng = np.random.default_rng(seed)
    cell = rng.integers(cell_lo, cell_hi, n).astype(np.int32)
    off = _f32(rng.random(n))
    off = np.where(off >= 1.0, 0.0, off)
    px, py, pz = (_f32(rng.normal(size=n) * pscale) for _ in range(3))
    return cell, off, px, py, pz


def random_fields(nx, scale, seed):
    """Ex, Ey, Ez, By, Bz of a 1D grid with nx cells: node arrays have nx+1
    values, half-node arrays nx; smooth random modes plus noise."""
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate((nx, nx + 1, nx + 1, nx, nx)):
        x = np.arange(n) / n
        f = sum(rng.normal() * np.sin(2 * np.pi * (m + 1) * x + rng.random() * 6.28) for m in range(6))
        f = scale * (f / 3.0 + 0.1 * rng.normal(size=n))
        out.append(_f32(f))
    return out
