"""The velocity power spectrum (Sect. 3.3) on the GPU (sub-cell sampling
kernel, cuFFT real-to-complex transform, shell sums of the half spectrum)
against the oracle (its own sampling, numpy's full complex FFT), on even and
odd grid sizes, and its argument checks."""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1602_09079_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("n,order,sub", [(8, 3, 4), (6, 4, 3), (5, 2, 3), (4, 1, 1)])
def test_spectrum_matches_oracle(dg, n, order, sub):
    g = syn.GAMMA
    s = dg.Solver((n, n, n), order, g)
    o = oracle.Oracle((n, n, n), order - 1, g)
    w = syn.random_state((n, n, n), s.N, g, seed=70 + n, high=0.05)
    s.set_state(w)
    E = s.velocity_spectrum(sub)
    Eo = o.velocity_spectrum(w, sub)
    assert E.shape == Eo.shape
    assert np.abs(E - Eo).max() <= 1e-12 * Eo.sum()
    # bin by bin: an FFT coefficient carries an absolute rounding error of
    # order eps |v|, so a bin holding a fraction f of the power is accurate
    # to about eps / sqrt(f) relative; every bin above 1e-8 of the total
    # agrees to 1e-9 of itself
    big = Eo > 1e-8 * Eo.sum()
    assert big.sum() >= 3
    assert np.all(np.abs(E[big] - Eo[big]) <= 1e-9 * Eo[big])
    # the same call again gives the same result (bins cleared per call)
    assert np.abs(s.velocity_spectrum(sub) - E).max() <= 1e-14 * Eo.sum()


def test_spectrum_arguments(dg):
    s = dg.Solver((4, 4, 5), 2, syn.GAMMA)
    with pytest.raises(dg.DGError) as e:
        dg.dg_spectrum_sizes(s.ctx, 2)
    assert e.value.code == dg.DG_ERR_ARG
    s2 = dg.Solver((4, 4, 4), 2, syn.GAMMA)
    for sub in (0, 9):
        with pytest.raises(dg.DGError) as e:
            dg.dg_spectrum_sizes(s2.ctx, sub)
        assert e.value.code == dg.DG_ERR_ARG
