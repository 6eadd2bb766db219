"""Write oracle_parity_cases.json: the FP64 oracle's results on three small
seeded cases, which the benchmark compares with the GPU's on the same inputs
to report its errors against the oracle.  This script calls only the oracle;
the inputs come from tests/synth.py (seeds stored in the file).

  one_step   8 wavelengths at 100 cells per wavelength, random fields of
             scale 80 (seed 5), 1000 electrons (seed 10, momenta of width 60)
             and 500 protons (seed 11, width 2), RR on: positions and momenta
             after one step;
  fields_200 3 wavelengths at 200 cells per wavelength, a 0.5-wavelength
             hydrogen foil at 0.2 wavelengths (n_e = 64 n_c, 32 particles per
             cell per species, foil seed 7), LP a0 = 200 with a 3-period sin^2
             envelope, RR on: the five field components after 200 steps;
  balance    the small single run (20 wavelengths at 200 cells per
             wavelength, foil seed 1; as in oracle_small_run_ensemble.json):
             the largest time-centred energy-balance error along the 4211
             steps, sampled every 200 steps, relative to the injected energy.

    python tests/golden/make_parity_cases.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_parity_cases.json")

ONE_STEP = dict(box=dict(length_lambda=8, cells_per_lambda=100, cfl=0.95, lambda_um=0.8, rr_on=True, source_node=8),
                fields=dict(scale=80.0, seed=5),
                species=[dict(n=1000, charge=-1.0, mass=1.0, weight=0.01, pscale=60.0, seed=10),
                         dict(n=500, charge=1.0, mass=1836.15267343, weight=0.01, pscale=2.0, seed=11)])
FIELDS_200 = dict(box=dict(length_lambda=3, cells_per_lambda=200, cfl=0.95, lambda_um=0.8, rr_on=True,
                           source_node=8),
                  foil=dict(x0=0.2, thickness=0.5, ne=64.0, Z=1, A=1.0, ppc=32, seed=7),
                  laser=dict(a0=200.0, polarization=0, envelope=0, duration=3.0), steps=200)
BALANCE = dict(box=dict(length_lambda=20, cells_per_lambda=200, cfl=0.95, lambda_um=0.8, rr_on=True, source_node=8),
               foil=dict(x0=10.0, thickness=1.0, ne=64.0, Z=1, A=1.0, ppc=64, seed=1),
               laser=dict(a0=200.0, polarization=0, envelope=0, duration=10.0), steps=4211, every=199)


def one_step_inputs(nx):
    """The one-step case's inputs (test-side generators only)."""
    from tests import synth

    F = synth.random_fields(nx, **ONE_STEP["fields"])
    parts = [synth.random_particles(s["n"], 2, nx - 2, s["pscale"], s["seed"]) for s in ONE_STEP["species"]]
    return F, parts


def r10(a):
    return [float("%.10e" % v) for v in a]


def main():
    sys.path.insert(0, ROOT)
    import oracle
    from tests.spectrum_stats import balance

    out = {"what": __doc__.split("\n\n")[0], "one_step": ONE_STEP, "fields_200": FIELDS_200, "balance": BALANCE}
    o = oracle.OracleSim(**ONE_STEP["box"])
    F, parts = one_step_inputs(o.nx)
    o.set_fields(*F)
    for sp, (s, p) in enumerate(zip(ONE_STEP["species"], parts)):
        o.load_particles(sp, *p, s["weight"], s["charge"], s["mass"])
    o.step(1)
    res = []
    for sp in (0, 1):
        q = o.particles(sp)
        res.append({k: r10(q[k]) for k in ("x", "px", "py", "pz")})
    out["one_step"]["result"] = res
    o.close()

    c = FIELDS_200
    o = oracle.OracleSim(**c["box"])
    f = c["foil"]
    o.load_foil(f["x0"], f["thickness"], f["ne"], f["Z"], f["A"], f["ppc"], f["seed"])
    la = c["laser"]
    o.inject_laser(la["a0"], la["polarization"], la["envelope"], la["duration"])
    o.step(c["steps"])
    out["fields_200"]["result"] = [r10(o.field(k)) for k in range(5)]
    o.close()

    c = BALANCE
    o = oracle.OracleSim(**c["box"])
    f = c["foil"]
    o.load_foil(f["x0"], f["thickness"], f["ne"], f["Z"], f["A"], f["ppc"], f["seed"])
    la = c["laser"]
    o.inject_laser(la["a0"], la["polarization"], la["envelope"], la["duration"])
    b, e = balance(o, c["steps"], c["every"])
    out["balance"]["result"] = {"max_abs_over_injected": float(abs(b).max() / e[4]), "injected": float(e[4])}
    o.close()
    json.dump(out, open(OUT, "w"))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
