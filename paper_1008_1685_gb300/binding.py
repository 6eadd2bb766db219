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
SERVE_FIFO, SERVE_SHORTEST_FIRST = 0, 1
ELECTRON, ION = 0, 1
EX, EY, EZ, BY, BZ, JX, JY, JZ = range(8)

STATUS = {0: "PIC_OK", -1: "PIC_ERR_INVALID_ARG", -2: "PIC_ERR_STATE", -3: "PIC_ERR_OOM",
          -4: "PIC_ERR_CUDA", -5: "PIC_ERR_TIMEOUT", -6: "PIC_ERR_UNSUPPORTED"}

# exported symbols of include/picrr.h
SYMBOLS = ("pic_create", "pic_set_stream", "pic_load_foil", "pic_load_particles", "pic_load_particles_f32",
           "pic_set_fields",
           "pic_inject_laser", "pic_step_n", "pic_spectra", "pic_energy", "pic_read_particles",
           "pic_read_fields", "pic_stats", "pic_set_timing", "pic_last_error", "pic_destroy",
           "pic_spectrum_noalloc", "pic_batch_create", "pic_batch_set_stream", "pic_batch_add_run",
           "pic_batch_step", "pic_batch_run_status", "pic_batch_energy", "pic_batch_spectra",
           "pic_batch_read_particles", "pic_batch_read_fields", "pic_batch_release_run", "pic_batch_stats",
           "pic_batch_set_timing", "pic_batch_last_error", "pic_batch_destroy", "pic_batch_run_footprint",
           "pic_server_create", "pic_server_submit", "pic_server_result", "pic_server_stats",
           "pic_server_last_error", "pic_server_destroy", "pic_tune_shapes",
           "pic_batch_tune_shapes", "pic_set_shapes", "pic_batch_set_shapes", "pic_server_set_policy",
           "pic_snapshot", "pic_batch_snapshot",
           "pic_electron_scan", "pic_selftest_wait_timeout", "pic_batch_stop_run", "pic_server_cancel",
           "pic_save", "pic_restore", "pic_get_config", "pic_set_rr", "pic_shard_runs")
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


class ElectronCase(C.Structure):
    _fields_ = [("wave", C.c_int), ("a0", C.c_double), ("tau", C.c_double), ("x0", C.c_double),
                ("p0", C.c_double * 3)]


INTEGRATOR_LEAPFROG, INTEGRATOR_RK4 = 0, 1
ELECTRON_RR, ELECTRON_DERIV = 1, 2


class RunDesc(C.Structure):
    _fields_ = [
        ("length_lambda", C.c_double),
        ("source_node", C.c_int),
        ("rr_on", C.c_int),
        ("seed", C.c_uint64),
        ("foil_x0_lambda", C.c_double),
        ("foil_thickness_lambda", C.c_double),
        ("ne_over_nc", C.c_double),
        ("ion_Z", C.c_int),
        ("ion_A", C.c_double),
        ("ppc", C.c_int),
        ("a0", C.c_double),
        ("polarization", C.c_int),
        ("envelope", C.c_int),
        ("duration_periods", C.c_double),
        ("rise_periods", C.c_double),
        ("steps", C.c_int64),
    ]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "admitted", "completed", "failed", "queued", "running",
                                          "batch_steps", "particle_steps")] + \
               [("busy_s", C.c_double), ("device_bytes", C.c_int64), ("peak_device_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


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
        ("graph_launches", C.c_int64),
        ("steps_since_sort", C.c_int32),
        ("reserved", C.c_int32),
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
        L.pic_batch_create.argtypes = [C.POINTER(Config), C.c_int, C.POINTER(vp)]
        L.pic_batch_set_stream.argtypes = [vp, vp]
        L.pic_batch_add_run.argtypes = [vp, C.POINTER(RunDesc), C.POINTER(C.c_int)]
        L.pic_batch_step.argtypes = [vp, i64, C.POINTER(i64)]
        L.pic_batch_run_status.argtypes = [vp, C.c_int, C.POINTER(i64), C.POINTER(C.c_int)]
        L.pic_batch_energy.argtypes = [vp, C.c_int, dp]
        L.pic_batch_spectra.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, dp, dp]
        L.pic_batch_read_particles.argtypes = [vp, C.c_int, C.c_int, i64, dp, dp, dp, dp, C.POINTER(C.c_int32),
                                               C.POINTER(i64)]
        L.pic_batch_read_fields.argtypes = [vp, C.c_int, C.c_int, i64, dp, C.POINTER(i64)]
        L.pic_batch_release_run.argtypes = [vp, C.c_int]
        L.pic_batch_stats.argtypes = [vp, C.POINTER(Stats)]
        L.pic_batch_set_timing.argtypes = [vp, C.c_int]
        L.pic_batch_last_error.argtypes = [vp]
        L.pic_batch_last_error.restype = C.c_char_p
        L.pic_batch_destroy.argtypes = [vp]
        L.pic_batch_run_footprint.argtypes = [vp, C.POINTER(RunDesc), C.POINTER(C.c_size_t)]
        L.pic_server_create.argtypes = [C.POINTER(Config), C.c_int, i64, C.POINTER(vp)]
        L.pic_server_submit.argtypes = [vp, C.POINTER(RunDesc), C.c_int, C.c_double, C.c_double, C.POINTER(i64)]
        L.pic_server_result.argtypes = [vp, i64, C.c_double, dp, dp, dp, dp]
        L.pic_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.pic_server_last_error.argtypes = [vp]
        L.pic_server_last_error.restype = C.c_char_p
        L.pic_server_destroy.argtypes = [vp]
        ip = C.POINTER(C.c_int)
        L.pic_tune_shapes.argtypes = [vp, i64, ip, ip, ip, dp]
        L.pic_batch_tune_shapes.argtypes = [vp, i64, ip, ip, ip, dp]
        L.pic_set_shapes.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.pic_batch_set_shapes.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.pic_server_set_policy.argtypes = [vp, C.c_int, i64]
        L.pic_electron_scan.argtypes = [C.POINTER(ElectronCase), i64, C.c_int, C.c_int, C.c_double, i64, C.c_int,
                                        C.c_double, C.c_int, dp, i64]
        L.pic_selftest_wait_timeout.argtypes = [C.c_int, dp]
        L.pic_batch_stop_run.argtypes = [vp, C.c_int]
        L.pic_save.argtypes = [vp, C.c_char_p]
        L.pic_restore.argtypes = [C.c_char_p, C.c_int, C.c_int, C.POINTER(vp)]
        L.pic_get_config.argtypes = [vp, C.POINTER(Config)]
        L.pic_set_rr.argtypes = [vp, C.c_int]
        L.pic_shard_runs.argtypes = [C.POINTER(Config), C.POINTER(RunDesc), C.c_int, C.c_int, C.c_int, C.c_size_t,
                                     C.POINTER(C.c_int), dp]
        L.pic_server_cancel.argtypes = [vp, i64]
        L.pic_snapshot.argtypes = [vp, C.c_int, C.c_double, i64, dp, dp, dp, dp, dp, dp, C.POINTER(i64)]
        L.pic_batch_snapshot.argtypes = [vp, C.c_int, C.c_int, C.c_double, i64, dp, dp, dp, dp, dp, dp,
                                         C.POINTER(i64)]
        for name in SYMBOLS:
            if name not in ("pic_last_error", "pic_batch_last_error", "pic_server_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def selftest_wait_timeout(device=0):
    """Run the device wait self-test; returns (status, seconds).  The expected
    status is -5 (PIC_ERR_TIMEOUT): the bounded wait gave up."""
    sec = C.c_double(0.0)
    rc = library().pic_selftest_wait_timeout(device, C.byref(sec))
    return rc, sec.value


def electron_scan(cases, integrator=INTEGRATOR_RK4, rr=True, deriv=False, dt=0.01, nsteps=1000, every=1,
                  lambda_um=0.8, device=0):
    """Single electrons in analytic plane waves on the GPU (pic_electron_scan).
    cases: iterable of dicts with wave, a0, x0, p0 (3) and tau (wave 2).
    Returns an array [n][nsteps // every][5] of rows (t, x, px, py, pz)."""
    cases = list(cases)
    arr = (ElectronCase * max(1, len(cases)))()
    for k, c in enumerate(cases):
        arr[k].wave = int(c["wave"])
        arr[k].a0 = float(c["a0"])
        arr[k].tau = float(c.get("tau", 0.0))
        arr[k].x0 = float(c.get("x0", 0.0))
        for j in range(3):
            arr[k].p0[j] = float(c["p0"][j])
    ns = nsteps // every
    out = np.zeros((len(cases), ns, 5))
    flags = (ELECTRON_RR if rr else 0) | (ELECTRON_DERIV if deriv else 0)
    rc = library().pic_electron_scan(arr, len(cases), integrator, flags, dt, nsteps, every, lambda_um, device,
                                     _dp(out), ns)
    if rc != 0:
        raise PicError(rc, library().pic_last_error(None).decode())
    return out


def shard_runs(descs, n_ranks, cells_per_lambda, in_order=False, budget_per_rank=0, cfl=0.95):
    """pic_shard_runs: the rank of each run (list of RunDesc) and the
    particle-steps assigned to each rank."""
    L = library()
    n = len(descs)
    arr = (RunDesc * max(1, n))(*descs)
    cfg = Config(1.0, cells_per_lambda, cfl, 0.8, 1, 8, 1, 0, 8, 0)
    ranks = (C.c_int * max(1, n))()
    work = np.zeros(n_ranks)
    rc = L.pic_shard_runs(C.byref(cfg), arr, n, n_ranks, int(bool(in_order)), budget_per_rank, ranks, _dp(work))
    if rc != 0:
        raise PicError(rc, L.pic_last_error(None).decode())
    return [ranks[i] for i in range(n)], work


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


def _snapshot(call, check, per_particle):
    n = C.c_int64(0)
    summ = np.zeros(3)
    check(call(0, None, None, None, None, None, _dp(summ), C.byref(n)))
    out = dict(d_max=summ[0], chi_max=summ[1], n_flagged=int(summ[2]), n=n.value)
    if per_particle and n.value:
        arr = {k: np.zeros(n.value) for k in ("x", "px", "pperp", "d", "chi")}
        check(call(n.value, _dp(arr["x"]), _dp(arr["px"]), _dp(arr["pperp"]), _dp(arr["d"]), _dp(arr["chi"]), None,
                   None))
        out.update(arr)
    return out


class Sim:
    """One simulation handle (pic_create ... pic_destroy)."""

    def __init__(self, length_lambda, cells_per_lambda, cfl=0.95, lambda_um=0.8, rr_on=True,
                 sort_interval=8, seed=1, device=0, source_node=8, hbm_budget_bytes=0, _handle=None):
        self._L = library()
        if _handle is None:
            cfg = Config(length_lambda, cells_per_lambda, cfl, lambda_um, int(rr_on), sort_interval, seed,
                         device, source_node, hbm_budget_bytes)
            h = C.c_void_p()
            rc = self._L.pic_create(C.byref(cfg), C.byref(h))
            if rc != 0:
                raise PicError(rc, self._L.pic_last_error(None).decode())
        else:
            h = _handle
        self._h = h
        self.cells_per_lambda = cells_per_lambda
        self.nx = int(round(length_lambda * cells_per_lambda))
        self.dx = 2 * np.pi / cells_per_lambda
        self.dt = cfl * self.dx

    @classmethod
    def restore(cls, path, device=0, sort_interval=0):
        """A new handle in the state saved by save() (pic_restore)."""
        L = library()
        h = C.c_void_p()
        rc = L.pic_restore(os.fsencode(path), device, sort_interval, C.byref(h))
        if rc != 0:
            raise PicError(rc, L.pic_last_error(None).decode())
        cfg = Config()
        L.pic_get_config(h, C.byref(cfg))
        return cls(cfg.length_lambda, cfg.cells_per_lambda, cfg.cfl, _handle=h)

    def save(self, path):
        self._check(self._L.pic_save(self._h, os.fsencode(path)))

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

    def snapshot(self, species, chi_flag=0.1, per_particle=True):
        """d (Eq. damping) and chi per particle (load order) with x, p_x, p_perp,
        and the summary (max d, max chi, particles with chi >= chi_flag)."""
        return _snapshot(lambda *a: self._L.pic_snapshot(self._h, species, chi_flag, *a), self._check, per_particle)

    def field(self, comp):
        out = np.zeros(self.nx + 1)
        n = C.c_int64(0)
        self._check(self._L.pic_read_fields(self._h, comp, len(out), _dp(out), C.byref(n)))
        return out[: n.value].copy()

    def stats(self):
        st = Stats()
        self._check(self._L.pic_stats(self._h, C.byref(st)))
        return st.as_dict()

    def tune_shapes(self, steps_per_candidate=64):
        """Pick the fastest particles per thread, work-unit size and sort interval
        by timing real steps.  Returns (unit_particles, sort_interval,
        particles_per_thread, ms_per_step[11])."""
        u, c, w = C.c_int(0), C.c_int(0), C.c_int(0)
        ms = np.full(11, -1.0)
        self._check(self._L.pic_tune_shapes(self._h, steps_per_candidate, C.byref(u), C.byref(c), C.byref(w),
                                            _dp(ms)))
        return u.value, c.value, w.value, ms

    def set_shapes(self, unit_particles, sort_interval, particles_per_thread=2):
        self._check(self._L.pic_set_shapes(self._h, unit_particles, sort_interval, particles_per_thread))

    def set_rr(self, on):
        """Radiation-reaction kick of the electrons on or off from the next step (pic_set_rr)."""
        self._check(self._L.pic_set_rr(self._h, int(on)))

    def set_timing(self, on=True):
        self._check(self._L.pic_set_timing(self._h, int(on)))


def run_desc(length_lambda, foil_x0, foil_thickness, ne, a0, polarization, duration, steps, rr_on=True, ppc=64,
             ion_Z=1, ion_A=1.0, envelope=ENV_SIN2, rise=0.0, seed=1, source_node=8):
    return RunDesc(length_lambda, source_node, int(rr_on), seed, foil_x0, foil_thickness, ne, ion_Z, ion_A, ppc,
                   a0, polarization, envelope, duration, rise, steps)


class Batch:
    """Many independent runs stepped together (pic_batch_*)."""

    def __init__(self, cells_per_lambda, max_runs, cfl=0.95, lambda_um=0.8, sort_interval=8, device=0,
                 hbm_budget_bytes=0):
        self._L = library()
        cfg = Config(1.0, cells_per_lambda, cfl, lambda_um, 1, sort_interval, 0, device, 0, hbm_budget_bytes)
        h = C.c_void_p()
        rc = self._L.pic_batch_create(C.byref(cfg), max_runs, C.byref(h))
        if rc != 0:
            raise PicError(rc, self._L.pic_batch_last_error(None).decode())
        self._h = h
        self.dx = 2 * np.pi / cells_per_lambda
        self.dt = cfl * self.dx
        self.cells_per_lambda = cells_per_lambda
        self._nx = {}

    def _check(self, rc):
        if rc != 0:
            raise PicError(rc, self._L.pic_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.pic_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        self._check(self._L.pic_batch_set_stream(self._h, C.c_void_p(stream_ptr)))

    def add_run(self, length_lambda, foil_x0, foil_thickness, ne, a0, polarization, duration, steps, rr_on=True,
                ppc=64, ion_Z=1, ion_A=1.0, envelope=ENV_SIN2, rise=0.0, seed=1, source_node=8):
        d = run_desc(length_lambda, foil_x0, foil_thickness, ne, a0, polarization, duration, steps, rr_on, ppc,
                     ion_Z, ion_A, envelope, rise, seed, source_node)
        rid = C.c_int(-1)
        self._check(self._L.pic_batch_add_run(self._h, C.byref(d), C.byref(rid)))
        self._nx[rid.value] = int(round(length_lambda * self.cells_per_lambda))
        return rid.value

    def step(self, n):
        done = C.c_int64(0)
        self._check(self._L.pic_batch_step(self._h, n, C.byref(done)))
        return done.value

    def run_status(self, run):
        done, fin = C.c_int64(0), C.c_int(0)
        self._check(self._L.pic_batch_run_status(self._h, run, C.byref(done), C.byref(fin)))
        return done.value, bool(fin.value)

    def energy(self, run):
        out = np.zeros(6)
        self._check(self._L.pic_batch_energy(self._h, run, _dp(out)))
        return out

    def spectra(self, run, species, nbins, e_min, e_max):
        counts = np.zeros(nbins)
        rad = C.c_double(0.0)
        self._check(self._L.pic_batch_spectra(self._h, run, species, nbins, e_min, e_max, _dp(counts),
                                              C.byref(rad)))
        return counts, rad.value

    def particles(self, run, species):
        n = C.c_int64(0)
        self._check(self._L.pic_batch_read_particles(self._h, run, species, 0, None, None, None, None, None,
                                                     C.byref(n)))
        n = n.value
        x, px, py, pz = (np.zeros(n) for _ in range(4))
        flag = np.zeros(n, dtype=np.int32)
        self._check(self._L.pic_batch_read_particles(self._h, run, species, n, _dp(x), _dp(px), _dp(py), _dp(pz),
                                                     flag.ctypes.data_as(C.POINTER(C.c_int32)), None))
        return dict(x=x, px=px, py=py, pz=pz, flag=flag)

    def snapshot(self, run, species, chi_flag=0.1, per_particle=True):
        return _snapshot(lambda *a: self._L.pic_batch_snapshot(self._h, run, species, chi_flag, *a), self._check,
                         per_particle)

    def nx(self, run):
        return self._nx[run]

    def field(self, run, comp):
        out = np.zeros(self._nx[run] + 1)
        n = C.c_int64(0)
        self._check(self._L.pic_batch_read_fields(self._h, run, comp, len(out), _dp(out), C.byref(n)))
        return out[: n.value].copy()

    def footprint(self, **desc):
        d = run_desc(**desc)
        out = C.c_size_t(0)
        rc = self._L.pic_batch_run_footprint(self._h, C.byref(d), C.byref(out))
        if rc != 0:
            raise PicError(rc, self._L.pic_batch_last_error(None).decode())
        return out.value

    def stop_run(self, run):
        self._check(self._L.pic_batch_stop_run(self._h, run))

    def release_run(self, run):
        self._check(self._L.pic_batch_release_run(self._h, run))

    def stats(self):
        st = Stats()
        self._check(self._L.pic_batch_stats(self._h, C.byref(st)))
        return st.as_dict()

    def tune_shapes(self, steps_per_candidate=64):
        u, c, w = C.c_int(0), C.c_int(0), C.c_int(0)
        ms = np.full(11, -1.0)
        self._check(self._L.pic_batch_tune_shapes(self._h, steps_per_candidate, C.byref(u), C.byref(c),
                                                  C.byref(w), _dp(ms)))
        return u.value, c.value, w.value, ms

    def set_shapes(self, unit_particles, sort_interval, particles_per_thread=2):
        self._check(self._L.pic_batch_set_shapes(self._h, unit_particles, sort_interval, particles_per_thread))

    def set_timing(self, on=True):
        self._check(self._L.pic_batch_set_timing(self._h, int(on)))


class Server:
    """Request loop over a batch (pic_server_*): submit run descriptions, fetch
    their spectra and energy read-outs when they finish."""

    def __init__(self, cells_per_lambda, max_runs, chunk_steps=64, cfl=0.95, lambda_um=0.8, sort_interval=8,
                 device=0, hbm_budget_bytes=0):
        self._L = library()
        cfg = Config(1.0, cells_per_lambda, cfl, lambda_um, 1, sort_interval, 0, device, 0, hbm_budget_bytes)
        h = C.c_void_p()
        rc = self._L.pic_server_create(C.byref(cfg), max_runs, chunk_steps, C.byref(h))
        if rc != 0:
            raise PicError(rc, self._L.pic_server_last_error(None).decode())
        self._h = h
        self._nbins = {}

    def _err(self, rc):
        return PicError(rc, self._L.pic_server_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.pic_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, nbins=200, ion_e_max=2000.0, el_e_max=2000.0, **desc):
        d = run_desc(**desc)
        t = C.c_int64(0)
        rc = self._L.pic_server_submit(self._h, C.byref(d), nbins, ion_e_max, el_e_max, C.byref(t))
        if rc != 0:
            raise self._err(rc)
        self._nbins[t.value] = nbins
        return t.value

    def result(self, ticket, wait_s=0.0):
        """dict(ion, el, energy, latency_s) when finished, None if not yet."""
        nb = self._nbins[ticket]
        ion, el, en = np.zeros(nb), np.zeros(nb), np.zeros(6)
        lat = C.c_double(0.0)
        rc = self._L.pic_server_result(self._h, ticket, wait_s, _dp(ion), _dp(el), _dp(en), C.byref(lat))
        if rc == -5:
            return None
        del self._nbins[ticket]
        if rc != 0:
            raise self._err(rc)
        return dict(ion=ion, el=el, energy=en, latency_s=lat.value)

    def set_policy(self, policy=SERVE_FIFO, max_resident_particles=0):
        rc = self._L.pic_server_set_policy(self._h, policy, max_resident_particles)
        if rc != 0:
            raise self._err(rc)

    def cancel(self, ticket):
        rc = self._L.pic_server_cancel(self._h, ticket)
        if rc != 0:
            raise self._err(rc)

    def stats(self):
        st = ServerStats()
        rc = self._L.pic_server_stats(self._h, C.byref(st))
        if rc != 0:
            raise self._err(rc)
        return st.as_dict()
