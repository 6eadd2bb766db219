"""GB300-native (sm_103a) 1D laser-foil PIC step with the leapfrog
Landau-Lifshitz radiation-reaction pusher of Tamburini et al. (arXiv
1008.1685), behind the C ABI declared in ``include/picrr.h``.

This package is the thin Python binding: argument marshalling only.  Every
step of the method runs in the CUDA kernels of ``libpicrr.so``; there is no
CPU fallback, and importing the binding raises if the library is missing.
"""
from .binding import (  # noqa: F401
    BY, BZ, CP, ELECTRON, ENV_SIN2, ENV_TRAPEZOID, EX, EY, EZ, ION, JX, JY, JZ, LP, SERVE_FIFO,
    SERVE_SHORTEST_FIRST, INTEGRATOR_LEAPFROG, INTEGRATOR_RK4, ElectronCase, electron_scan, selftest_wait_timeout, shard_runs,
    Batch, PicError, RunDesc, Server, ServerStats, Sim, Stats, library, library_path, run_desc,
)
