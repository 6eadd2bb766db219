"""ctypes binding of libpicrr.so with the same names as the C ABI.

Argument marshalling only: the arithmetic of every step runs on the GPU in
the library's kernels.  Missing library or a failing call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpicrr.so")

LP, CP = 0, 1
ENV_SIN2, ENV_TRAPEZOID = 0, 1
ELECTRON, ION = 0, 1
EX, EY, EZ, BY, BZ, JX, JY, JZ = range(8)

STATUS = {0: "PIC_OK", -1: "PIC_ERR_INVALID_ARG", -2: "PIC_ERR_STATE", -3: "PIC_ERR_OOM",
          -4: "PIC_ERR_CUDA", -5: "PIC_ERR_TIMEOUT", -6: "PIC_ERR_UNSUPPORTED"}

# exported symbols of include/picrr.h
SYMBOLS = ("pic_create", "pic_set_stream", "pic_load_foil", "pic_load_particles", "pic_load_particles_f32",
           "pic_set_fields",
           "pic_inject_laser", "pic_step_n", "pic_spectra", "pic_energy", "pic_read_particles",
           "pic_read_fields", "pic_stats", "pic_set_timing", "pic_last_error", "pic_destroy",
           "pic_spectrum_noalloc")
NOALLOC_MAX_BINS = 65536


class PicError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class Config(C.Structure):
    _fields_ = [
        ("length_lambda", C.c_double),
        ("cells_per_lambda", C.c_double),
        ("cfl", C.c_double),
        ("lambda_um", C.c_double),
        ("rr_on", C.c_int),
        ("sort_interval", C.c_int),
        ("seed", C.c_uint64),
        ("device", C.c_int),
        ("source_node", C.c_int),
        ("hbm_budget_bytes", C.c_size_t),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64),
        ("kernel_launches", C.c_int64),
        ("push_launches", C.c_int64),
        ("sort_count", C.c_int64),
        ("active_particles", C.c_int64),
        ("push_ms", C.c_double),
        ("field_ms", C.c_double),
        ("sort_ms", C.c_double),
        ("timed_push_launches", C.c_int64),
        ("device_bytes", C.c_int64),
        ("n_units", C.c_int32),
        ("fp_bits", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _LIB_PATH


def library():
    """Load libpicrr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libpicrr.so is not built: run __graft_entry__.build() "
                              "(or python paper_1008_1685_gb300/build.py)")
        L = C.CDLL(_LIB_PATH)
        dp, vp, i64 = C.POINTER(C.c_double), C.c_void_p, C.c_int64
        L.pic_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
        L.pic_set_stream.argtypes = [vp, vp]
        L.pic_load_foil.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int]
        L.pic_load_particles.argtypes = [vp, C.c_int, i64, C.POINTER(C.c_int32), dp, dp, dp, dp,
                                         C.c_double, C.c_double, C.c_double]
        fp = C.POINTER(C.c_float)
        L.pic_load_particles_f32.argtypes = [vp, C.c_int, i64, C.POINTER(C.c_int32), fp, fp, fp, fp,
                                             C.c_double, C.c_double, C.c_double]
        L.pic_set_fields.argtypes = [vp, dp, dp, dp, dp, dp]
        L.pic_inject_laser.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double]
        L.pic_step_n.argtypes = [vp, i64, C.POINTER(i64)]
        L.pic_spectra.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, dp, dp]
        L.pic_energy.argtypes = [vp, dp]
        L.pic_read_particles.argtypes = [vp, C.c_int, i64, dp, dp, dp, dp, C.POINTER(C.c_int32),
                                         C.POINTER(i64)]
        L.pic_read_fields.argtypes = [vp, C.c_int, i64, dp, C.POINTER(i64)]
        L.pic_stats.argtypes = [vp, C.POINTER(Stats)]
        L.pic_set_timing.argtypes = [vp, C.c_int]
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = C.c_char_p
        L.pic_destroy.argtypes = [vp]
        L.pic_spectrum_noalloc.argtypes = [vp, vp, vp, i64, C.c_double, C.c_double, C.c_int, C.c_double,
                                           C.c_double, vp, vp]
        for name in SYMBOLS:
            if name != "pic_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def spectrum_noalloc(px_ptr, py_ptr, pz_ptr, n, mass_me, weight_dx, nbins, e_min, e_max, counts_ptr,
                     stream_ptr=0):
    """pic_spectrum_noalloc on device pointers (integers); returns the status
    and, on failure, the library's message."""
    L = library()
    rc = L.pic_spectrum_noalloc(C.c_void_p(px_ptr), C.c_void_p(py_ptr), C.c_void_p(pz_ptr), n, mass_me,
                                weight_dx, nbins, e_min, e_max, C.c_void_p(counts_ptr), C.c_void_p(stream_ptr))
    return rc, (L.pic_last_error(None).decode() if rc else "")


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Sim:
    """One simulation handle (pic_create ... pic_destroy)."""

    def __init__(self, length_lambda, cells_per_lambda, cfl=0.95, lambda_um=0.8, rr_on=True,
                 sort_interval=8, seed=1, device=0, source_node=8, hbm_budget_bytes=0):
        self._L = library()
        cfg = Config(length_lambda, cells_per_lambda, cfl, lambda_um, int(rr_on), sort_interval, seed,
                     device, source_node, hbm_budget_bytes)
        h = C.c_void_p()
        rc = self._L.pic_create(C.byref(cfg), C.byref(h))
        if rc != 0:
            raise PicError(rc, self._L.pic_last_error(None).decode())
        self._h = h
        self.cells_per_lambda = cells_per_lambda
        self.nx = int(round(length_lambda * cells_per_lambda))
        self.dx = 2 * np.pi / cells_per_lambda
        self.dt = cfl * self.dx

    def _check(self, rc):
        if rc != 0:
            raise PicError(rc, self._L.pic_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.pic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- setup --------------------------------------------------------------
    def set_stream(self, stream_ptr):
        self._check(self._L.pic_set_stream(self._h, C.c_void_p(stream_ptr)))

    def load_foil(self, x0_lambda, thickness_lambda, ne_over_nc, ion_Z=1, ion_A=1.0, ppc=64):
        self._check(self._L.pic_load_foil(self._h, x0_lambda, thickness_lambda, ne_over_nc, ion_Z, ion_A, ppc))

    def load_particles(self, species, cell, off, px, py, pz, weight, charge, mass):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        off, px, py, pz = (_f64(a) for a in (off, px, py, pz))
        self._check(self._L.pic_load_particles(
            self._h, species, len(cell), cell.ctypes.data_as(C.POINTER(C.c_int32)), _dp(off), _dp(px),
            _dp(py), _dp(pz), weight, charge, mass))

    def load_particles_f32(self, species, cell, off, px, py, pz, weight, charge, mass):
        """Single-precision host arrays (numpy float32 / int32, pinned or not) copied as they are."""
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (off, px, py, pz)]
        fpp = C.POINTER(C.c_float)
        self._check(self._L.pic_load_particles_f32(
            self._h, species, len(cell), cell.ctypes.data_as(C.POINTER(C.c_int32)),
            *[a.ctypes.data_as(fpp) for a in arrs], weight, charge, mass))

    def set_fields(self, Ex=None, Ey=None, Ez=None, By=None, Bz=None):
        arrs = [_f64(a) for a in (Ex, Ey, Ez, By, Bz)]
        self._check(self._L.pic_set_fields(self._h, *[_dp(a) for a in arrs]))

    def inject_laser(self, a0, polarization, envelope, duration_periods, rise_periods=0.0):
        self._check(self._L.pic_inject_laser(self._h, a0, polarization, envelope, duration_periods,
                                             rise_periods))

    # -- stepping -----------------------------------------------------------
    def step(self, n):
        done = C.c_int64(0)
        self._check(self._L.pic_step_n(self._h, n, C.byref(done)))
        return done.value

    # -- read-outs ----------------------------------------------------------
    def energy(self):
        out = np.zeros(6)
        self._check(self._L.pic_energy(self._h, _dp(out)))
        return out

    def spectra(self, species, nbins, e_min, e_max):
        counts = np.zeros(nbins)
        rad = C.c_double(0.0)
        self._check(self._L.pic_spectra(self._h, species, nbins, e_min, e_max, _dp(counts), C.byref(rad)))
        return counts, rad.value

    def particles(self, species):
        n = C.c_int64(0)
        self._check(self._L.pic_read_particles(self._h, species, 0, None, None, None, None, None,
                                               C.byref(n)))
        n = n.value
        x, px, py, pz = (np.zeros(n) for _ in range(4))
        flag = np.zeros(n, dtype=np.int32)
        self._check(self._L.pic_read_particles(self._h, species, n, _dp(x), _dp(px), _dp(py), _dp(pz),
                                               flag.ctypes.data_as(C.POINTER(C.c_int32)), None))
        return dict(x=x, px=px, py=py, pz=pz, flag=flag)

    def field(self, comp):
        out = np.zeros(self.nx + 1)
        n = C.c_int64(0)
        self._check(self._L.pic_read_fields(self._h, comp, len(out), _dp(out), C.byref(n)))
        return out[: n.value].copy()

    def stats(self):
        st = Stats()
        self._check(self._L.pic_stats(self._h, C.byref(st)))
        return st.as_dict()

    def set_timing(self, on=True):
        self._check(self._L.pic_set_timing(self._h, int(on)))
