"""FP64 CPU oracle for the 1D laser-foil PIC step with the leapfrog
Landau-Lifshitz radiation-reaction pusher (Tamburini et al., arXiv 1008.1685).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import this package.
It shares no code with the CUDA library and the CUDA library never calls it.

The arithmetic lives in ``pic_oracle.c`` (plain C, IEEE double, no FMA
contraction); this module only loads the shared object and marshals
arguments.  ``pic_oracle_omp.c`` builds the same code a second time with the
particle loop split over OpenMP threads: a timing build for the CPU baseline,
checked against the serial build, never the checker itself.  ``planewave.py`` holds the closed-form plane-wave solutions used
to pin the pusher.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "pic_oracle.c")
# the parallel timing build (OpenMP over the particles of each species)
_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")
_SRC_OMP = os.path.join(_HERE, "pic_oracle_omp.c")

LP, CP = 0, 1
ENV_SIN2, ENV_TRAPEZOID = 0, 1
ELECTRON, ION = 0, 1
EX, EY, EZ, BY, BZ, JX, JY, JZ = range(8)


def ecr(lambda_um):
    """E_cr = m c^2/(hbar omega) in the field unit m omega c/|e|."""
    return lib().or_ecr(lambda_um)


def _stale(so, srcs):
    return not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(f) for f in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (ISO C11, -O2, no FP contraction), and its
    parallel timing build with -fopenmp where the compiler supports it."""
    hdr = os.path.join(_HERE, "oracle.h")
    flags = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    if force or _stale(_SO, [_SRC, hdr]):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    if force or _stale(_SO_OMP, [_SRC, _SRC_OMP, hdr]):
        tmp = _SO_OMP + ".tmp%d" % os.getpid()
        r = subprocess.run(["gcc", *flags, "-fopenmp", "-o", tmp, _SRC_OMP, "-lm"], capture_output=True)
        if r.returncode == 0:
            os.replace(tmp, _SO_OMP)
    return _SO


def parallel_available() -> bool:
    build()
    return os.path.exists(_SO_OMP)


class _Config(C.Structure):
    _fields_ = [
        ("length_lambda", C.c_double),
        ("cells_per_lambda", C.c_double),
        ("cfl", C.c_double),
        ("lambda_um", C.c_double),
        ("rr_on", C.c_int),
        ("source_node", C.c_int),
    ]


_libs = {}


def lib(parallel: bool = False):
    """The oracle's shared object; parallel=True: the OpenMP timing build."""
    if parallel not in _libs:
        build()
        if parallel and not os.path.exists(_SO_OMP):
            raise RuntimeError("the parallel oracle build needs a C compiler with OpenMP")
        L = C.CDLL(_SO_OMP if parallel else _SO)
        if parallel:
            L.or_threads.restype = C.c_int
        dp = C.POINTER(C.c_double)
        L.or_eps_rr.restype = C.c_double
        L.or_eps_rr.argtypes = [C.c_double]
        L.or_push_boris_rr.restype = C.c_double
        L.or_push_boris_rr.argtypes = [dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_int, dp]
        L.or_pw_leapfrog.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, dp, C.c_double,
                                     C.c_int64, C.c_int, C.c_double, C.c_int, dp, C.c_int64]
        L.or_pw_rk4.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, dp, C.c_double,
                                C.c_int64, C.c_int, C.c_double, C.c_int, C.c_int, dp, C.c_int64]
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Config)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_nx.argtypes = [C.c_void_p]
        L.or_dx.restype = C.c_double
        L.or_dx.argtypes = [C.c_void_p]
        L.or_dt.restype = C.c_double
        L.or_dt.argtypes = [C.c_void_p]
        L.or_load_foil.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int,
                                   C.c_double, C.c_int, C.c_uint64]
        L.or_load_particles.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.POINTER(C.c_int32), dp,
                                        dp, dp, dp, C.c_double, C.c_double, C.c_double]
        L.or_set_fields.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.or_inject_laser.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_double,
                                      C.c_double]
        L.or_step_n.argtypes = [C.c_void_p, C.c_int64]
        L.or_steps_done.restype = C.c_int64
        L.or_steps_done.argtypes = [C.c_void_p]
        L.or_energy.argtypes = [C.c_void_p, dp]
        L.or_spectra.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, dp, dp]
        L.or_read_particles.restype = C.c_int64
        L.or_read_particles.argtypes = [C.c_void_p, C.c_int, C.c_int64, dp, dp, dp, dp,
                                        C.POINTER(C.c_int32)]
        L.or_snapshot.restype = C.c_int64
        L.or_snapshot.argtypes = [C.c_void_p, C.c_int, C.c_int64, dp, dp]
        L.or_ecr.restype = C.c_double
        L.or_ecr.argtypes = [C.c_double]
        L.or_read_fields.restype = C.c_int64
        L.or_read_fields.argtypes = [C.c_void_p, C.c_int, C.c_int64, dp]
        _libs[parallel] = L
    return _libs[parallel]


def threads() -> int:
    """OpenMP threads the parallel build uses (OMP_NUM_THREADS, else all cores)."""
    return lib(True).or_threads()


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def eps_rr(lambda_um: float = 0.8) -> float:
    """(4/3) pi r_e / lambda, the radiation constant of Eq. (3dLL)."""
    return lib().or_eps_rr(lambda_um)


def push(p, E, B, qm=-1.0, dt=0.01, eps=None, rr=True, lambda_um=0.8):
    """One pusher step of Sec. 3 for a single particle; returns (p_new, p_L, radiated)."""
    if eps is None:
        eps = eps_rr(lambda_um)
    p = _f64(p).copy()
    pL = np.zeros(3)
    rad = lib().or_push_boris_rr(_dp(p), _dp(_f64(E)), _dp(_f64(B)), qm, dt, eps, int(rr), _dp(pL))
    return p, pL, rad


def pw_leapfrog(kind, a0, x0, p0, dt, nsteps, every=1, eps=0.0, rr=False, tau=0.0):
    """Electron in an analytic plane wave with the leapfrog pusher.  Returns an
    array of rows (t_n, x^n, px, py, pz) with p = p^{n-1/2}."""
    nout = nsteps // every
    out = np.zeros((nout, 5))
    rc = lib().or_pw_leapfrog(kind, a0, tau, x0, _dp(_f64(p0)), dt, nsteps, every, eps, int(rr),
                              _dp(out), nout)
    assert rc == 0
    return out


def pw_rk4(kind, a0, x0, p0, dt, nsteps, every=1, eps=0.0, rr=False, deriv=False, tau=0.0):
    """Electron in an analytic plane wave, RK4 on Eq. (3dLL).  Rows (t, x, px, py, pz)."""
    nout = nsteps // every
    out = np.zeros((nout, 5))
    rc = lib().or_pw_rk4(kind, a0, tau, x0, _dp(_f64(p0)), dt, nsteps, every, eps, int(rr),
                         int(deriv), _dp(out), nout)
    assert rc == 0
    return out


class OracleSim:
    """The FP64 1D PIC with the same call sequence as the CUDA library."""

    def __init__(self, length_lambda, cells_per_lambda, cfl=0.95, lambda_um=0.8, rr_on=True,
                 source_node=8, parallel=False):
        cfg = _Config(length_lambda, cells_per_lambda, cfl, lambda_um, int(rr_on), source_node)
        self._L = lib(parallel)
        self._h = self._L.or_create(C.byref(cfg))
        if not self._h:
            raise ValueError("oracle: invalid configuration")
        self.nx = self._L.or_nx(self._h)
        self.dx = self._L.or_dx(self._h)
        self.dt = self._L.or_dt(self._h)

    def close(self):
        if self._h:
            self._L.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError("oracle %s failed (%d)" % (what, rc))

    def load_foil(self, x0_lambda, thickness_lambda, ne_over_nc, ion_Z, ion_A, ppc, seed):
        self._check(self._L.or_load_foil(self._h, x0_lambda, thickness_lambda, ne_over_nc, ion_Z,
                                         ion_A, ppc, seed), "load_foil")

    def load_particles(self, species, cell, off, px, py, pz, weight, charge, mass):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        off, px, py, pz = (_f64(a) for a in (off, px, py, pz))
        self._check(self._L.or_load_particles(
            self._h, species, len(cell), cell.ctypes.data_as(C.POINTER(C.c_int32)), _dp(off),
            _dp(px), _dp(py), _dp(pz), weight, charge, mass), "load_particles")

    def set_fields(self, Ex, Ey, Ez, By, Bz):
        arrs = [_f64(a) for a in (Ex, Ey, Ez, By, Bz)]
        self._check(self._L.or_set_fields(self._h, *[_dp(a) for a in arrs]), "set_fields")

    def inject_laser(self, a0, polarization, envelope, duration_periods, rise_periods=0.0):
        self._check(self._L.or_inject_laser(self._h, a0, polarization, envelope, duration_periods,
                                            rise_periods), "inject_laser")

    def step(self, n):
        self._check(self._L.or_step_n(self._h, n), "step_n")

    @property
    def steps_done(self):
        return self._L.or_steps_done(self._h)

    def energy(self):
        out = np.zeros(6)
        self._check(self._L.or_energy(self._h, _dp(out)), "energy")
        return out

    def spectra(self, species, nbins, e_min, e_max):
        counts = np.zeros(nbins)
        uo = np.zeros(2)
        self._check(self._L.or_spectra(self._h, species, nbins, e_min, e_max, _dp(counts),
                                       _dp(uo)), "spectra")
        return counts, uo

    def snapshot(self, species):
        """Friction coefficient d (Eq. damping) and quantum parameter chi per particle."""
        n = self._L.or_snapshot(self._h, species, 0, None, None)
        d, chi = np.zeros(n), np.zeros(n)
        self._L.or_snapshot(self._h, species, n, _dp(d), _dp(chi))
        return dict(d=d, chi=chi)

    def particles(self, species):
        n = self._L.or_read_particles(self._h, species, 0, None, None, None, None, None)
        x, px, py, pz = (np.zeros(n) for _ in range(4))
        flag = np.zeros(n, dtype=np.int32)
        self._L.or_read_particles(self._h, species, n, _dp(x), _dp(px), _dp(py), _dp(pz),
                                  flag.ctypes.data_as(C.POINTER(C.c_int32)))
        return dict(x=x, px=px, py=py, pz=pz, flag=flag)

    def field(self, comp):
        out = np.zeros(self.nx + 1)
        n = self._L.or_read_fields(self._h, comp, len(out), _dp(out))
        if n < 0:
            raise RuntimeError("oracle read_fields failed")
        return out[:n].copy()
