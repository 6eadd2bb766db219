"""Checkpoint and restore (pic_save / pic_restore): a run saved on a sort
step and restored into a new handle continues bit-identically to the
uninterrupted run (particles, fields, spectra, energy bookkeeping); saved
between sorts it is sorted first, which changes only rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
KW = dict(length_lambda=6, cells_per_lambda=100, rr_on=True, sort_interval=8, seed=9)


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


def fresh(picrr):
    g = picrr.Sim(**KW)
    g.load_foil(0.5, 0.5, 80.0, 1, 1.0, 32)
    g.inject_laser(300.0, picrr.CP, picrr.ENV_SIN2, 2.0)
    return g


def state(g):
    return dict(p=[g.particles(sp) for sp in (0, 1)], f=[g.field(c) for c in range(8)], e=g.energy(),
                s=g.spectra(1, 100, 0.0, 400.0)[0])


def test_restore_on_a_sort_step_is_bit_identical(picrr, tmp_path):
    ref = fresh(picrr)
    ref.step(360)
    want = state(ref)
    ref.close()
    g = fresh(picrr)
    g.step(160)  # a multiple of the sort interval
    path = str(tmp_path / "run.ck")
    g.save(path)
    g.close()
    r = picrr.Sim.restore(path)
    assert r.nx == 600
    r.step(200)
    got = state(r)
    r.close()
    for sp in (0, 1):
        for k in ("x", "px", "py", "pz", "flag"):
            assert np.array_equal(got["p"][sp][k], want["p"][sp][k]), (sp, k)
    for c in range(8):
        assert np.array_equal(got["f"][c], want["f"][c]), c
    assert np.array_equal(got["e"][[0, 1, 2, 4, 5]], want["e"][[0, 1, 2, 4, 5]])
    assert got["e"][3] == pytest.approx(want["e"][3], rel=1e-12)
    assert np.array_equal(got["s"], want["s"])


def test_restore_between_sorts_changes_only_rounding(picrr, tmp_path):
    ref = fresh(picrr)
    ref.step(300)
    want = state(ref)
    ref.close()
    g = fresh(picrr)
    g.step(157)
    path = str(tmp_path / "run2.ck")
    g.save(path)
    g.close()
    r = picrr.Sim.restore(path)
    r.step(143)
    got = state(r)
    r.close()
    for c in range(5):
        assert np.linalg.norm(got["f"][c] - want["f"][c]) <= 1e-4 * max(np.linalg.norm(want["f"][c]), 1e-30), c
    assert got["e"][4] == pytest.approx(want["e"][4], rel=1e-6)


def test_restore_rejects_other_files(picrr, tmp_path):
    bad = tmp_path / "bad.ck"
    bad.write_bytes(b"not a checkpoint" * 10)
    with pytest.raises(picrr.PicError) as e:
        picrr.Sim.restore(str(bad))
    assert e.value.status == -1
