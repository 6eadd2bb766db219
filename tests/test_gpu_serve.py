"""The request loop (pic_server_*): run requests arrive while others are
stepping, are admitted by batch slots and device memory, join the running
batch between step chunks, and come back as spectra and energy read-outs.
Each result must be the same alone and in the mix: a request's run is packed
into shared launches but none of its arithmetic changes, so its spectra and
energy equal those of the same run stepped alone (the radiated-energy tally
to 1e-12 relative: its per-unit partials are grouped differently)."""
import time

import numpy as np
import pytest

from tests.test_gpu_batch import CPL, EARLY, LATE, RUNS

pytestmark = pytest.mark.gpu
NB, ION_MAX, EL_MAX = 120, 400.0, 600.0


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


def desc(d):
    return dict(length_lambda=d["length_lambda"], foil_x0=d["foil_x0"], foil_thickness=d["foil_thickness"],
                ne=d["ne"], a0=d["a0"], polarization=d["polarization"], duration=d["duration"], steps=d["steps"],
                rr_on=d["rr_on"], ppc=d["ppc"], seed=d["seed"])


def solo(picrr, d):
    g = picrr.Sim(length_lambda=d["length_lambda"], cells_per_lambda=CPL, rr_on=d["rr_on"], sort_interval=8,
                  seed=d["seed"])
    g.load_foil(d["foil_x0"], d["foil_thickness"], d["ne"], 1, 1.0, d["ppc"])
    g.inject_laser(d["a0"], d["polarization"], picrr.ENV_SIN2, d["duration"])
    g.step(d["steps"])
    out = dict(ion=g.spectra(1, NB, 0.0, ION_MAX)[0], el=g.spectra(0, NB, 0.0, EL_MAX)[0], energy=g.energy())
    g.close()
    return out


def assert_same(res, ref, what):
    assert np.array_equal(res["ion"], ref["ion"]), what
    assert np.array_equal(res["el"], ref["el"]), what
    assert np.array_equal(res["energy"][[0, 1, 2, 4, 5]], ref["energy"][[0, 1, 2, 4, 5]]), what
    assert res["energy"][3] == pytest.approx(ref["energy"][3], rel=1e-12, abs=1e-300), what
    assert res["ion"].sum() > 0 and res["latency_s"] > 0


def test_requests_overlap_and_equal_solo_runs(picrr):
    srv = picrr.Server(CPL, max_runs=4, chunk_steps=64)
    first = [RUNS[0], RUNS[2]]
    tickets = [srv.submit(nbins=NB, ion_e_max=ION_MAX, el_e_max=EL_MAX, **desc(d)) for d in first]
    t0 = time.time()
    while srv.stats()["batch_steps"] < 128 and time.time() - t0 < 60:
        time.sleep(0.002)
    st = srv.stats()
    assert st["running"] == 2 and st["completed"] == 0  # both still stepping
    later = [LATE, RUNS[1], EARLY]
    tickets += [srv.submit(nbins=NB, ion_e_max=ION_MAX, el_e_max=EL_MAX, **desc(d)) for d in later]
    results = [srv.result(t, wait_s=300.0) for t in tickets]
    st = srv.stats()
    assert st["completed"] == 5 and st["failed"] == 0 and st["queued"] == 0 and st["running"] == 0
    descs = first + later
    # the runs overlapped: far fewer batch steps than one run after another
    assert st["batch_steps"] < sum(d["steps"] for d in descs) - 1000
    assert st["particle_steps"] == sum(2 * d["ppc"] * round(d["foil_thickness"] * CPL) * d["steps"] for d in descs)
    for res, d in zip(results, descs):
        assert_same(res, solo(picrr, d), d["seed"])
    srv.close()


def test_admission_by_device_memory(picrr):
    same = [dict(RUNS[0], seed=s, a0=a) for s, a in ((21, 150.0), (22, 250.0), (23, 350.0))]
    probe = picrr.Batch(CPL, max_runs=3)
    base = probe.stats()["device_bytes"]
    fp = probe.footprint(**desc(same[0]))
    probe.close()
    # room for one of these runs, not for two
    budget = base + fp + fp // 4
    srv = picrr.Server(CPL, max_runs=3, chunk_steps=32, hbm_budget_bytes=budget)
    tickets = [srv.submit(nbins=NB, ion_e_max=ION_MAX, el_e_max=EL_MAX, **desc(d)) for d in same]
    with pytest.raises(picrr.PicError) as e:  # larger than the whole budget
        srv.submit(**desc(dict(RUNS[1], ppc=4000)))
    assert e.value.status == -3
    bad = srv.submit(**desc(dict(RUNS[0], foil_x0=7.9)))  # foil beyond the box: fails at admission
    results = [srv.result(t, wait_s=300.0) for t in tickets]
    with pytest.raises(picrr.PicError) as e:
        srv.result(bad, wait_s=60.0)
    assert e.value.status == -1
    st = srv.stats()
    assert st["completed"] == 3 and st["failed"] == 1
    assert 0 < st["peak_device_bytes"] <= budget
    # one run at a time: the batch steps add up to the runs' step counts
    assert st["batch_steps"] == sum(d["steps"] for d in same)
    for res, d in zip(results, same):
        assert_same(res, solo(picrr, d), d["seed"])
    srv.close()


def test_unknown_ticket_and_poll(picrr):
    srv = picrr.Server(CPL, max_runs=1)
    t = srv.submit(nbins=NB, **desc(RUNS[2]))
    assert srv.result(t, wait_s=0.0) is None  # not finished yet
    assert srv.result(t, wait_s=300.0) is not None
    with pytest.raises(KeyError):
        srv.result(t)
    srv.close()


@pytest.mark.parametrize("policy", ["fifo", "sjf"])
def test_admission_order_policy(picrr, policy):
    """One run resident at a time (particle cap); while the first request runs,
    a medium and then a small request queue up.  Arrival order serves the
    medium one first, least-work-first the small one."""
    big = dict(RUNS[1], seed=31)                    # admitted at once, runs while the others queue
    medium = dict(RUNS[0], seed=32)                 # 1200 particles per species, 704 steps
    small = dict(RUNS[2], seed=33, steps=300)       # 480 particles per species, 300 steps
    srv = picrr.Server(CPL, max_runs=3, chunk_steps=32)
    # room for the medium run, not for medium + small; the big run is admitted alone
    cap = 2 * medium["ppc"] * round(medium["foil_thickness"] * CPL)
    srv.set_policy(picrr.SERVE_SHORTEST_FIRST if policy == "sjf" else picrr.SERVE_FIFO, cap)
    kw = dict(nbins=NB, ion_e_max=ION_MAX, el_e_max=EL_MAX)
    tb = srv.submit(**kw, **desc(big))
    t0 = time.time()
    while srv.stats()["running"] < 1 and time.time() - t0 < 60:
        time.sleep(0.001)
    tm = srv.submit(**kw, **desc(medium))
    ts = srv.submit(**kw, **desc(small))
    rb, rm, rs = (srv.result(t, wait_s=300.0) for t in (tb, tm, ts))
    st = srv.stats()
    assert st["completed"] == 3
    # one at a time: the batch steps add up
    assert st["batch_steps"] == big["steps"] + medium["steps"] + small["steps"]
    if policy == "sjf":
        assert rs["latency_s"] < rm["latency_s"]
    else:
        assert rm["latency_s"] < rs["latency_s"]
    for res, d in ((rb, big), (rm, medium), (rs, small)):
        assert_same(res, solo(picrr, d), d["seed"])
    srv.close()


def test_cancel_queued_and_running(picrr):
    """A cancelled queued request is dropped; a cancelled running one leaves the
    batch at the end of the step chunk and frees its memory; the others are
    unaffected (their results equal their solo runs)."""
    long_run = dict(RUNS[1], seed=41, steps=4000)
    other = dict(RUNS[0], seed=42)
    queued = dict(RUNS[2], seed=43)
    srv = picrr.Server(CPL, max_runs=2, chunk_steps=32)
    kw = dict(nbins=NB, ion_e_max=ION_MAX, el_e_max=EL_MAX)
    # only one run at a time: the queued request waits behind the first
    srv.set_policy(picrr.SERVE_FIFO, 2 * long_run["ppc"] * round(long_run["foil_thickness"] * CPL))
    ta = srv.submit(**kw, **desc(long_run))
    tq = srv.submit(**kw, **desc(queued))
    tb = srv.submit(**kw, **desc(other))
    srv.cancel(tq)
    with pytest.raises(picrr.PicError) as e:
        srv.result(tq, wait_s=10.0)
    assert e.value.status == -2 and "cancelled" in str(e.value)
    t0 = time.time()
    while srv.stats()["batch_steps"] < 200 and time.time() - t0 < 60:
        time.sleep(0.001)
    srv.cancel(ta)
    with pytest.raises(picrr.PicError) as e:
        srv.result(ta, wait_s=60.0)
    assert e.value.status == -2
    rb = srv.result(tb, wait_s=300.0)
    st = srv.stats()
    assert st["completed"] == 1 and st["failed"] == 2 and st["running"] == 0
    assert st["batch_steps"] < long_run["steps"]  # the long run did not run to its end
    assert_same(rb, solo(picrr, other), other["seed"])
    with pytest.raises(picrr.PicError) as e:
        srv.cancel(tb)
    assert e.value.status == -1  # already fetched: unknown ticket
    srv.close()
