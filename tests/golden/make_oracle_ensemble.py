"""Write oracle_small_run_ensemble.json: the FP64 oracle's ion spectra and
energy read-outs of the small single run (20 wavelengths at 200 cells per
wavelength, a 1-wavelength hydrogen foil at 10 wavelengths with n_e = 64 n_c
and 64 macro-particles per cell per species, LP a0 = 200 with a 10-period
sin^2 envelope, radiation reaction on, 4211 steps = 20 periods) for foil
seeds 1..N.  Full runs are chaotic, so GPU and oracle are compared as
ensembles; this script calls only the oracle.

    python tests/golden/make_oracle_ensemble.py [N] [workers]
"""
import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_small_run_ensemble.json")

SMALL = dict(length_lambda=20, cells_per_lambda=200, cfl=0.95, lambda_um=0.8, rr_on=True, source_node=8)
FOIL = dict(x0=10.0, thickness=1.0, ne=64.0, Z=1, A=1.0, ppc=64)
LASER = dict(a0=200.0, polarization=0, envelope=0, duration=10.0)
STEPS = 4211
BINS = dict(n=400, e_min=0.0, e_max=2000.0)


def one(seed):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle

    o = oracle.OracleSim(**SMALL)
    o.load_foil(FOIL["x0"], FOIL["thickness"], FOIL["ne"], FOIL["Z"], FOIL["A"], FOIL["ppc"], seed)
    o.inject_laser(LASER["a0"], LASER["polarization"], LASER["envelope"], LASER["duration"])
    o.step(STEPS)
    spec = o.spectra(oracle.ION, BINS["n"], BINS["e_min"], BINS["e_max"])[0]
    e = o.energy()
    o.close()
    return seed, [float(v) for v in spec], [float(v) for v in e]


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 256
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 4)
    sys.path.insert(0, ROOT)
    import oracle

    oracle.build()
    t0 = time.time()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = sorted(ex.map(one, range(1, n + 1)))
    spec = [0.0] * BINS["n"]
    for _, s, _ in res:
        spec = [a + b for a, b in zip(spec, s)]
    out = {
        "what": "FP64 oracle, small single run, ion spectra dN/dE (weights per unit energy) summed over seeds",
        "small": SMALL, "foil": FOIL, "laser": LASER, "steps": STEPS, "bins": BINS,
        "seeds": [r[0] for r in res],
        "spectrum_sum": [float("%.12g" % v) for v in spec],
        "energy_labels": ["field", "kinetic_e", "kinetic_i", "radiated", "injected_net", "boundary_out"],
        "energy_mean": [float("%.12g" % (sum(r[2][k] for r in res) / len(res))) for k in range(6)],
        "radiated": [float("%.10g" % r[2][3]) for r in res],
        "seconds": time.time() - t0,
    }
    json.dump(out, open(OUT, "w"))
    print("wrote", OUT, "seeds", n, "%.0f s" % out["seconds"])


if __name__ == "__main__":
    main()
