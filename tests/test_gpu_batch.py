"""Batched runs (pic_batch_*): independent runs of uneven sizes stepped
together, one launch per kernel per step for all of them.  Each run's result
must be the same alone and in the mix.

Particle and field arithmetic of a run does not depend on the other runs of its
batch: its work units are built from its own cell counts, its current is
summed in exact integer arithmetic, and it sorts on the same steps as when it
runs alone (runs join at sort boundaries).  So particles, fields, spectra and
the boundary fluxes of each run are bit-identical to the same run stepped on
its own.  The radiated-energy tally is the same sum of per-unit partials, but
the partials are flushed into it whenever any run of the batch ends, so it is
grouped differently: equal to 1e-12 relative.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CPL = 100
RUNS = [
    dict(length_lambda=8, foil_x0=3.0, foil_thickness=0.5, ne=40.0, a0=150.0, polarization=0, duration=3.0,
         steps=704, rr_on=True, ppc=24, seed=5),
    dict(length_lambda=12, foil_x0=4.0, foil_thickness=1.0, ne=90.0, a0=300.0, polarization=1, duration=4.0,
         steps=1000, rr_on=False, ppc=48, seed=6),
    dict(length_lambda=6, foil_x0=2.0, foil_thickness=0.3, ne=120.0, a0=500.0, polarization=0, duration=2.0,
         steps=453, rr_on=True, ppc=16, seed=7),
]
# the foil sits near the laser source, so the pulse is in it within ~50 steps
EARLY = dict(length_lambda=6, foil_x0=0.5, foil_thickness=0.5, ne=80.0, a0=300.0, polarization=1, duration=2.0,
             steps=240, rr_on=True, ppc=32, seed=9)
LATE = dict(length_lambda=10, foil_x0=3.5, foil_thickness=0.8, ne=70.0, a0=400.0, polarization=1, duration=3.0,
            steps=620, rr_on=True, ppc=32, seed=8)


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


def solo(picrr, d):
    g = picrr.Sim(length_lambda=d["length_lambda"], cells_per_lambda=CPL, rr_on=d["rr_on"], sort_interval=8,
                  seed=d["seed"])
    g.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"])
    g.inject_laser(d["a0"], d["polarization"], picrr.ENV_SIN2, d["duration"])
    g.step(d["steps"])
    out = snapshot(g.particles, g.field, g.energy, g.spectra)
    g.close()
    return out


def snapshot(particles, field, energy, spectra):
    return dict(p=[particles(sp) for sp in (0, 1)], f=[field(c) for c in range(8)], e=energy(),
                s=spectra(1, 200, 0.0, 400.0)[0])


def batch_snapshot(b, rid):
    return snapshot(lambda sp: b.particles(rid, sp), lambda c: b.field(rid, c), lambda: b.energy(rid),
                    lambda sp, n, lo, hi: b.spectra(rid, sp, n, lo, hi))


def assert_same(a, b, what):
    for sp in (0, 1):
        for k in ("x", "px", "py", "pz", "flag"):
            assert np.array_equal(a["p"][sp][k], b["p"][sp][k]), (what, sp, k)
    for c in range(8):
        assert np.array_equal(a["f"][c], b["f"][c]), (what, c)
    assert np.array_equal(a["e"][[0, 1, 2, 4, 5]], b["e"][[0, 1, 2, 4, 5]]), what
    assert a["e"][3] == pytest.approx(b["e"][3], rel=1e-12, abs=1e-300), what
    assert np.array_equal(a["s"], b["s"]), what


def add(b, d):
    return b.add_run(d["length_lambda"], d["foil_x0"], d["foil_thickness"], d["ne"], d["a0"], d["polarization"],
                     d["duration"], d["steps"], rr_on=d["rr_on"], ppc=d["ppc"], seed=d["seed"])


def test_batch_runs_equal_solo_runs(picrr):
    b = picrr.Batch(CPL, max_runs=4, sort_interval=8)
    ids = [add(b, d) for d in RUNS]
    # step in pieces that do not line up with the sort interval or the run ends
    done = 0
    while True:
        n = b.step(97)
        done += n
        if n < 97:
            break
    assert done == max(d["steps"] for d in RUNS)
    for rid, d in zip(ids, RUNS):
        assert b.run_status(rid) == (d["steps"], True)
    st = b.stats()
    assert st["push_launches"] == done  # one push launch per step for all runs
    for rid, d in zip(ids, RUNS):
        ref = solo(picrr, d)
        got = batch_snapshot(b, rid)
        assert np.max(np.abs(ref["p"][0]["px"])) > 1.0  # the laser reached the foil
        assert_same(got, ref, rid)
    assert b.step(10) == 0  # nothing left to step
    b.close()


def test_late_joiner_and_slot_reuse(picrr):
    b = picrr.Batch(CPL, max_runs=3, sort_interval=8)
    r0, r1 = add(b, RUNS[0]), add(b, RUNS[2])
    assert b.step(160) == 160  # a multiple of the sort interval: the join needs no extra sort
    r2 = add(b, LATE)
    while b.step(1000) > 0:
        pass
    with pytest.raises(picrr.PicError) as e:
        add(b, RUNS[1])  # no free slot
    assert e.value.status == -2
    for rid, d in ((r0, RUNS[0]), (r1, RUNS[2]), (r2, LATE)):
        assert_same(batch_snapshot(b, rid), solo(picrr, d), rid)
    # a released slot takes a new run, which again matches its solo run
    b.release_run(r1)
    with pytest.raises(picrr.PicError) as e:
        b.energy(r1)
    assert e.value.status == -1
    r3 = add(b, RUNS[1])
    assert r3 == r1
    while b.step(1000) > 0:
        pass
    assert_same(batch_snapshot(b, r3), solo(picrr, RUNS[1]), r3)
    b.close()


def test_join_between_sorts_changes_only_rounding(picrr):
    """A run that joins between two sorts forces an early sort of the runs
    already stepping: their particles are reordered a few steps early, which
    changes only the order of single-precision sums."""
    b = picrr.Batch(CPL, max_runs=2, sort_interval=8)
    r0 = add(b, EARLY)
    b.step(101)
    r1 = add(b, LATE)
    while b.step(1000) > 0:
        pass
    assert_same(batch_snapshot(b, r1), solo(picrr, LATE), r1)
    # the early run: 139 steps after the extra sort (the runs are chaotic, so
    # rounding differences grow over longer spans)
    got, ref = batch_snapshot(b, r0), solo(picrr, EARLY)
    assert np.max(np.abs(ref["p"][0]["px"])) > 1.0
    for grp in ((1, 2), (3, 4), (0,)):
        a = np.concatenate([got["f"][c] for c in grp])
        r = np.concatenate([ref["f"][c] for c in grp])
        assert np.linalg.norm(a - r) <= 1e-4 * np.linalg.norm(r), grp
    for sp in (0, 1):
        d = np.abs(got["p"][sp]["px"] - ref["p"][sp]["px"])
        assert np.max(d) <= 1e-3 * (1.0 + np.max(np.abs(ref["p"][sp]["px"]))), sp
    b.close()


def test_batch_energy_balance_each_run(picrr):
    b = picrr.Batch(CPL, max_runs=3, sort_interval=8)
    ids = [add(b, d) for d in RUNS]
    while b.step(1000) > 0:
        pass
    for rid in ids:
        e = b.energy(rid)
        u_in = e[4]
        assert u_in > 0
        # field + kinetic + radiated + outflow = injected, to the scheme's drift
        assert abs(e[0] + e[1] + e[2] + e[3] + e[5] - u_in) < 2e-2 * u_in, (rid, e)
    b.close()


def test_batch_argument_errors(picrr):
    b = picrr.Batch(CPL, max_runs=1)
    with pytest.raises(picrr.PicError) as e:
        b.add_run(4, 1.0, 0.5, 10.0, 10.0, 0, 2.0, steps=0)
    assert e.value.status == -1
    with pytest.raises(picrr.PicError) as e:
        b.add_run(4, 3.9, 0.5, 10.0, 10.0, 0, 2.0, steps=10)  # foil beyond the box
    assert e.value.status == -1
    rid = b.add_run(4, 1.0, 0.5, 10.0, 10.0, 0, 2.0, steps=50, ppc=4)
    b.step(5)
    with pytest.raises(picrr.PicError) as e:
        b.release_run(rid)  # still stepping
    assert e.value.status == -2
    with pytest.raises(picrr.PicError) as e:
        b.energy(7)
    assert e.value.status == -1
    assert b.step(100) == 45
    b.release_run(rid)
    b.close()


def test_graph_chunks_equal_single_launches(picrr):
    """Whole sort intervals run as one captured CUDA graph; step calls shorter
    than an interval launch every kernel on its own; with timing on, the graphs
    carry event-record nodes that time every push, Yee update and sort.  Same
    results in all three modes."""
    d = RUNS[0]
    out, st = [], []
    for mode in ("graphs", "single", "graphs+timing"):
        g = picrr.Sim(length_lambda=d["length_lambda"], cells_per_lambda=CPL, rr_on=d["rr_on"], sort_interval=8,
                      seed=d["seed"])
        g.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"])
        g.inject_laser(d["a0"], d["polarization"], picrr.ENV_SIN2, d["duration"])
        g.set_timing(mode == "graphs+timing")
        if mode == "single":
            left = d["steps"]
            while left > 0:  # calls of fewer steps than a sort interval never form a graph chunk
                g.step(min(7, left))
                left -= 7
        else:
            for n in (5, 3, 200, d["steps"] - 208):  # chunks start only on sort boundaries
                g.step(n)
        out.append(snapshot(g.particles, g.field, g.energy, g.spectra))
        st.append(g.stats())
        g.close()
    chunks = (d["steps"] - 8) // 8
    assert st[0]["graph_launches"] == chunks and st[1]["graph_launches"] == 0 and st[2]["graph_launches"] == chunks
    # (each short step call also flushes the radiated-energy partials: one launch more)
    assert st[0]["kernel_launches"] == st[2]["kernel_launches"] <= st[1]["kernel_launches"]
    # every push of the timed run was timed, inside the graphs as well as outside
    assert st[2]["timed_push_launches"] == st[2]["push_launches"] == d["steps"]
    assert st[2]["push_ms"] > 0 and st[2]["field_ms"] > 0 and st[2]["sort_ms"] > 0
    assert st[0]["timed_push_launches"] == 0
    assert_same(out[0], out[1], "graph vs single launches")
    assert_same(out[0], out[2], "graph vs timed graph")


def test_shape_tuner(picrr):
    """The tuner times real steps with 4 and 2 particles per thread, then at
    unit sizes 2048..16384, then at sort intervals 8..96, and keeps the
    fastest shapes; its trials are ordinary steps of the run: replaying the
    same shape changes and step counts by hand gives the same bits."""
    d = EARLY  # the pulse is in the foil from step ~50 on
    slots, units, intervals = (4, 2), (2048, 4096, 8192, 16384), (8, 16, 32, 64, 96)
    res = []
    for tune in (True, False):
        g = picrr.Sim(length_lambda=d["length_lambda"], cells_per_lambda=CPL, rr_on=d["rr_on"], sort_interval=8,
                      seed=d["seed"])
        g.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"])
        g.inject_laser(d["a0"], d["polarization"], picrr.ENV_SIN2, d["duration"])
        if tune:
            unit, interval, w, ms = g.tune_shapes(8)
            assert unit in units and interval in intervals and w in slots
            assert np.all(ms > 0)
            picks = (slots[int(np.argmin(ms[:2]))], units[int(np.argmin(ms[2:6]))], intervals[int(np.argmin(ms[6:]))])
            assert (w, unit, interval) == picks
            done = g.stats()["steps"]
            # warm-up interval + trial for each candidate (a trial is at least one interval)
            assert done == 2 * (8 + 8) + 4 * (8 + 8) + (8 + 8) + (16 + 16) + (32 + 32) + (64 + 64) + (96 + 96)
        else:
            bw, bu, bi = picks
            for s_ in slots:
                g.set_shapes(4096, 8, s_)
                g.step(16)
            for u in units:
                g.set_shapes(u, 8, bw)
                g.step(16)
            for i in intervals:
                g.set_shapes(bu, i, bw)
                g.step(i + max(i, 8 // i * i))
            g.set_shapes(bu, bi, bw)
            assert g.stats()["steps"] == done
        g.step(640 - done)
        res.append([g.field(c) for c in range(5)] + [g.particles(0)["px"]])
        g.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_set_shapes_changes_only_rounding(picrr):
    d = EARLY
    out = []
    for unit, interval, w in ((1024, 8, 4), (16384, 4, 2), (4096, 16, 2), (16384, 64, 4), (8192, 96, 2)):
        g = picrr.Sim(length_lambda=d["length_lambda"], cells_per_lambda=CPL, rr_on=d["rr_on"], sort_interval=8,
                      seed=d["seed"])
        g.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"])
        g.inject_laser(d["a0"], d["polarization"], picrr.ENV_SIN2, d["duration"])
        g.step(13)
        g.set_shapes(unit, interval, w)  # mid-interval: sorted first
        g.step(187)
        out.append((np.concatenate([g.field(c) for c in range(5)]), g.particles(0)))
        g.close()
    for f, p in out[1:]:
        assert np.linalg.norm(f - out[0][0]) <= 1e-5 * np.linalg.norm(out[0][0])
        assert np.max(np.abs(p["px"] - out[0][1]["px"])) <= 1e-3 * (1 + np.max(np.abs(out[0][1]["px"])))
    with pytest.raises(picrr.PicError):
        g = picrr.Sim(length_lambda=4, cells_per_lambda=CPL)
        g.set_shapes(3000, 8, 4)


def test_scan_split_over_ranks_gives_the_same_runs(picrr):
    """A scan split over two GPUs by pic_shard_runs (here the two shares run
    one after the other on this GPU, as two batches) gives every run the same
    result as the whole scan in one batch: the split changes only which runs
    share a batch."""
    descs = RUNS + [EARLY, LATE] + [dict(d, seed=d["seed"] + 20, steps=d["steps"] // 2 + 8) for d in RUNS]
    rd = [picrr.run_desc(d["length_lambda"], d["foil_x0"], d["foil_thickness"], d["ne"], d["a0"], d["polarization"],
                         d["duration"], d["steps"], rr_on=d["rr_on"], ppc=d["ppc"], seed=d["seed"]) for d in descs]
    ranks, work = picrr.shard_runs(rd, 2, CPL)
    assert set(ranks) == {0, 1}

    def run(subset):
        b = picrr.Batch(CPL, max_runs=len(subset), sort_interval=8)
        ids = {i: add(b, descs[i]) for i in subset}
        while b.step(500) > 0:
            pass
        out = {i: batch_snapshot(b, r) for i, r in ids.items()}
        b.close()
        return out

    whole = run(list(range(len(descs))))
    for rank in (0, 1):
        part = run([i for i, r in enumerate(ranks) if r == rank])
        for i, snap in part.items():
            assert_same(snap, whole[i], (rank, i))
