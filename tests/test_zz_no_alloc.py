"""dg_rhs_noalloc: the allocation-free R(y) entry point, for callers whose
device memory is owned and budgeted by a host application or another
framework's allocator and who may not call cudaMalloc/cudaFree themselves.
It must give what dg_rhs gives, call after call, although every call reuses
the same fixed device array. Collected last on purpose (file name), so a run
that stops at the first failure has run every other test before it."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 2e-5


def _normwise(a, b, N):
    a = a.reshape(5, N, -1)
    b = b.reshape(5, N, -1)
    return max(float(np.abs(a[i] - b[i]).max() / np.abs(b[i]).max()) for i in range(5))


@pytest.mark.parametrize("order,n,prec", [(3, (12, 9, 7), 0), (4, (10, 9, 8), 0), (2, (16, 13, 11), 1),
                                          (3, (9, 8, 7), 1), (4, (8, 7, 6), 1), (1, (9, 8, 7), 0)])
def test_noalloc_rhs_matches_dg_rhs_on_consecutive_calls(order, n, prec):
    import torch
    import paper_1602_09079_gb300 as dg

    g = syn.GAMMA
    s = dg.Solver(n, order, g, length=(1.0, 0.9, 1.2))
    s.set_precision(prec)
    tol = TOL64 if prec == dg.DG_PREC_FP64 else TOLMIX
    for call, seed in enumerate((21, 22)):  # two calls in a row, different states
        w = syn.random_state(n, s.N, g, seed=seed + order, high=0.01)
        s.set_state(w)
        ref = s.rhs(canonical=False)
        out = torch.full_like(ref, float("nan"))
        dg.dg_rhs_noalloc(n, order, g, prec, s.y, out, s.stream.cuda_stream, length=(1.0, 0.9, 1.2))
        torch.cuda.synchronize()
        assert torch.isfinite(out).all(), call
        assert _normwise(out.cpu().numpy(), ref.cpu().numpy(), s.N) <= tol, call


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    import paper_1602_09079_gb300 as dg

    n, order = (64, 64, 64), 3  # 15 * 9 * 262144 * 8 bytes > 32 MiB
    y = torch.zeros(5 * 10 * 64 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_noalloc(n, order, syn.GAMMA, dg.DG_PREC_FP64, y, y, 0)
    assert e.value.code == dg.DG_ERR_TOO_LARGE
    assert "32 MiB" in str(e.value)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_nan_input_then_finite_call(prec):
    """A non-finite input gives a non-finite R and DG_OK (no device-side
    error reporting); the next call on a finite state is unaffected by what
    the first one left in the shared array and matches dg_rhs again."""
    import torch
    import paper_1602_09079_gb300 as dg

    n, order, g = (7, 6, 5), 3, syn.GAMMA
    s = dg.Solver(n, order, g)
    s.set_precision(prec)
    w = syn.random_state(n, s.N, g, seed=41, high=0.01)
    bad = w.copy()
    bad[2, 3, 4, 4, 0] = np.nan
    s.set_state(bad)
    out = torch.zeros_like(s.y)
    dg.dg_rhs_noalloc(n, order, g, prec, s.y, out, s.stream.cuda_stream)
    torch.cuda.synchronize()
    assert not torch.isfinite(out).all()
    s.set_state(w)
    ref = s.rhs(canonical=False)
    out = torch.full_like(ref, float("nan"))
    dg.dg_rhs_noalloc(n, order, g, prec, s.y, out, s.stream.cuda_stream)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    assert _normwise(out.cpu().numpy(), ref.cpu().numpy(), s.N) <= (TOL64 if prec == 0 else TOLMIX)
