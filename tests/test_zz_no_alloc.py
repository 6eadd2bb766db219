"""pic_spectrum_noalloc: the ion spectrum from device-resident momenta with no
device allocation by the library (for callers that cannot allocate when they
need a spectrum, e.g. code that must not synchronise the GPU or whose device
memory belongs to another allocator).  Its output must equal pic_spectra's on
the same particles, on two calls in a row (the shared counter array is
cleared by each call).  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_spectrum_matches_pic_spectra_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as picrr
    from paper_1008_1685_gb300 import binding

    ne, ppc = 20.0, 16
    g = picrr.Sim(length_lambda=4, cells_per_lambda=100, seed=3, sort_interval=4)
    g.load_foil(1.0, 0.5, ne, 1, 1.0, ppc)
    g.inject_laser(120.0, picrr.LP, picrr.ENV_SIN2, 3.0)
    g.step(400)
    nbins, e_min, e_max = 300, 0.0, 60.0
    ref, _ = g.spectra(picrr.ION, nbins, e_min, e_max)
    ions = g.particles(picrr.ION)
    assert np.count_nonzero(ref) > 10  # the ions have a spread of energies
    dev = torch.device("cuda", 0)
    px, py, pz = (torch.tensor(ions[k], dtype=torch.float32, device=dev) for k in ("px", "py", "pz"))
    out = torch.empty(nbins, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    weight_dx = ne / ppc * g.dx
    for _ in range(2):
        out.fill_(-1.0)
        rc, msg = binding.spectrum_noalloc(px.data_ptr(), py.data_ptr(), pz.data_ptr(), px.numel(),
                                           1836.15267343, weight_dx, nbins, e_min, e_max, out.data_ptr(),
                                           stream.cuda_stream)
        assert rc == 0, msg
        torch.cuda.synchronize(dev)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0.0)
    # beyond the fixed counter array: rejected, nothing launched
    rc, msg = binding.spectrum_noalloc(px.data_ptr(), py.data_ptr(), pz.data_ptr(), px.numel(), 1836.15267343,
                                       weight_dx, binding.NOALLOC_MAX_BINS + 1, e_min, e_max, out.data_ptr(),
                                       stream.cuda_stream)
    assert rc == -1 and "nbins" in msg
    g.close()
