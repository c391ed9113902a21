"""The density PDF (Sect. 4.4) on the GPU against the oracle: integer
counts, bit-exact (both sides bin ln(rho) in FP64 with the same formula)."""
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


@pytest.mark.parametrize("n,order,sub,nb", [(8, 3, 4, 128), (5, 4, 3, 50), (4, 2, 1, 7)])
def test_density_pdf_matches_oracle(dg, n, order, sub, nb):
    g = syn.GAMMA
    s = dg.Solver((n, n, n), order, g)
    o = oracle.Oracle((n, n, n), order - 1, g)
    w = syn.random_state((n, n, n), s.N, g, seed=90 + n, high=0.05)
    s.set_state(w)
    lo, hi = -0.25, 0.2
    c = s.density_pdf(sub, lo, hi, nb)
    co = o.density_pdf(w, sub, lo, hi, nb)
    assert c.sum() == (n * sub) ** 3
    assert np.array_equal(c, co), np.nonzero(c - co)
    with pytest.raises(dg.DGError):
        s.density_pdf(sub, 1.0, 0.5, nb)
