"""Read-out statistics shared by the full-run tests and the benchmark's
parity record: peak energy and FWHM of a binned spectrum, and the
time-centred energy balance sampled along a run.  Neither is part of the
method: both only post-process what a run reports.
"""
import numpy as np


def peak_fwhm(counts, e_min, e_max, sigma_bins=6.0):
    """Peak energy and FWHM of a binned spectrum after Gaussian smoothing
    (sigma in bins); parabolic peak interpolation, linear interpolation of the
    half-maximum crossings on each side of the peak."""
    nb = len(counts)
    w = (e_max - e_min) / nb
    x = np.arange(-int(4 * sigma_bins), int(4 * sigma_bins) + 1)
    k = np.exp(-0.5 * (x / sigma_bins) ** 2)
    s = np.convolve(counts, k / k.sum(), mode="same")
    i = int(np.argmax(s))
    d = 0.0
    if 0 < i < nb - 1:
        a, b, c = s[i - 1], s[i], s[i + 1]
        den = a - 2 * b + c
        d = 0.5 * (a - c) / den if den != 0 else 0.0
    peak = e_min + (i + 0.5 + d) * w
    half = 0.5 * s[i]
    lo = i
    while lo > 0 and s[lo] > half:
        lo -= 1
    hi = i
    while hi < nb - 1 and s[hi] > half:
        hi += 1
    x_lo = lo + (half - s[lo]) / (s[lo + 1] - s[lo]) if s[lo + 1] != s[lo] else lo
    x_hi = hi - 1 + (s[hi - 1] - half) / (s[hi - 1] - s[hi]) if s[hi - 1] != s[hi] else hi
    return peak, (x_hi - x_lo) * w


def balance(sim, steps, every):
    """Time-centred energy balance sampled along a run (two reads per sample):
    field + kinetic + radiated + outflow - injected, kinetic and radiated
    averaged over the two reads around the field's time level."""
    out = []
    done = 0
    while done + every + 1 <= steps:
        sim.step(every)
        e0 = sim.energy()
        sim.step(1)
        e1 = sim.energy()
        done += every + 1
        out.append(e0[0] + 0.5 * (e0[1] + e1[1] + e0[2] + e1[2] + e0[3] + e1[3]) + e0[5] - e0[4])
    if steps > done:
        sim.step(steps - done)
    return np.array(out), sim.energy()
