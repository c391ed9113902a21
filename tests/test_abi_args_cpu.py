"""Error behaviour of the C ABI that include/dg.h states, checked without a
GPU: every call that takes a context returns DG_ERR_ARG for a NULL context
before touching the device, dg_init and dg_rhs_noalloc reject invalid meshes,
orders and gammas with DG_ERR_ARG (and dg_rhs_noalloc a mesh beyond its fixed
scratch with DG_ERR_TOO_LARGE), dg_destroy(NULL) is a no-op, and
dg_indicator_sizes returns the feature and parameter counts of the network
the header describes."""
import ctypes as C
import math

import pytest

import paper_1602_09079_gb300 as dg

# calls without a context argument, checked one by one below
NO_CTX = {"dg_strerror", "dg_destroy", "dg_init", "dg_rhs_noalloc", "dg_indicator_sizes", "dg_indicator_forward",
          "dg_indicator_backward", "dg_indicator_adam", "dg_probe_fma_peak", "dg_selftest_conversions"}


@pytest.fixture(scope="module")
def lib():
    return dg.load()


def _dummy(a):
    if a in (C.c_int, C.c_int64, C.c_longlong, C.c_size_t, C.c_ulonglong):
        return 1
    if a in (C.c_double, C.c_float):
        return 1.0
    if a is C.c_void_p:
        return None
    return a()  # NULL pointer of that type


def test_null_context_is_an_argument_error(lib):
    names = [n for n, (_, args) in dg._SIGS.items() if n not in NO_CTX]
    assert len(names) >= 25
    for name in names:
        res, args = dg._SIGS[name]
        assert args[0] is C.c_void_p, name
        vals = [_dummy(a) for a in args]
        vals[0] = None
        assert getattr(lib, name)(*vals) == dg.DG_ERR_ARG, name
    lib.dg_destroy(None)


def _mesh(n, length=(1.0, 1.0, 1.0)):
    m = dg.dg_mesh()
    for a in range(3):
        m.n[a] = n[a]
        m.length[a] = length[a]
    return m


BAD = [
    ((4, 4, 4), (1.0, 1.0, 1.0), 0, 1.4),
    ((4, 4, 4), (1.0, 1.0, 1.0), 5, 1.4),
    ((4, 4, 4), (1.0, 1.0, 1.0), 3, 1.0),
    ((4, 4, 4), (1.0, 1.0, 1.0), 3, math.nan),
    ((4, 4, 4), (1.0, 1.0, 1.0), 3, math.inf),
    ((0, 4, 4), (1.0, 1.0, 1.0), 3, 1.4),
    ((4, -1, 4), (1.0, 1.0, 1.0), 3, 1.4),
    ((4, 4, 4), (1.0, 0.0, 1.0), 3, 1.4),
    ((4, 4, 4), (1.0, 1.0, math.inf), 3, 1.4),
    ((4, 4, 4), (math.nan, 1.0, 1.0), 3, 1.4),
]


@pytest.mark.parametrize("n,length,order,gamma", BAD)
def test_init_rejects_invalid_arguments(lib, n, length, order, gamma):
    out = C.c_void_p()
    m = _mesh(n, length)
    assert lib.dg_init(C.byref(m), order, gamma, C.byref(out)) == dg.DG_ERR_ARG
    assert out.value is None
    assert lib.dg_rhs_noalloc(C.byref(m), order, gamma, dg.DG_PREC_FP64, C.c_void_p(16), C.c_void_p(16),
                              None) == dg.DG_ERR_ARG


def test_init_rejects_null_pointers_and_huge_meshes(lib):
    out = C.c_void_p()
    m = _mesh((4, 4, 4))
    assert lib.dg_init(None, 3, 1.4, C.byref(out)) == dg.DG_ERR_ARG
    assert lib.dg_init(C.byref(m), 3, 1.4, None) == dg.DG_ERR_ARG
    big = _mesh((2048, 2048, 1024))  # 2^32 cells: beyond the 32-bit cell index
    assert lib.dg_init(C.byref(big), 3, 1.4, C.byref(out)) == dg.DG_ERR_ARG


def test_cell_count_overflow_is_an_argument_error(lib):
    """Three axes whose product wraps a 64-bit count to 0 (2^21 x 2^21 x
    2^22 = 2^64): rejected before the product is formed, by dg_init and by
    dg_rhs_noalloc, without touching the device."""
    out = C.c_void_p()
    p = C.c_void_p(16)
    for n in [(1 << 21, 1 << 21, 1 << 22), (1 << 30, 4, 1), (65536, 65536, 2)]:
        m = _mesh(n)
        assert lib.dg_init(C.byref(m), 3, 1.4, C.byref(out)) == dg.DG_ERR_ARG, n
        assert out.value is None
        assert lib.dg_rhs_noalloc(C.byref(m), 3, 1.4, dg.DG_PREC_FP64, p, p, None) == dg.DG_ERR_ARG, n


def test_noalloc_argument_and_size_errors(lib):
    m = _mesh((8, 8, 8))
    p = C.c_void_p(16)
    assert lib.dg_rhs_noalloc(None, 3, 1.4, dg.DG_PREC_FP64, p, p, None) == dg.DG_ERR_ARG
    assert lib.dg_rhs_noalloc(C.byref(m), 3, 1.4, dg.DG_PREC_FP64, None, p, None) == dg.DG_ERR_ARG
    assert lib.dg_rhs_noalloc(C.byref(m), 3, 1.4, dg.DG_PREC_FP64, p, None, None) == dg.DG_ERR_ARG
    assert lib.dg_rhs_noalloc(C.byref(m), 3, 1.4, 7, p, p, None) == dg.DG_ERR_ARG
    # the face fluxes of 256^3 cells at order 4 (15 x 16 doubles per cell,
    # 32 GB) cannot fit the fixed scratch: rejected before any device work
    huge = _mesh((256, 256, 256))
    assert lib.dg_rhs_noalloc(C.byref(huge), 4, 1.4, dg.DG_PREC_FP64, p, p, None) == dg.DG_ERR_TOO_LARGE
    assert dg.dg_strerror(dg.DG_ERR_TOO_LARGE).startswith("problem too large")


def test_indicator_sizes_match_the_header(lib):
    for order in (2, 3, 4):
        N = order * (order + 1) * (order + 2) // 6
        F = 5 * (N - 1) + 2 + 5 + 26 * 5
        Fp = (F + 31) // 32 * 32
        nf, npad, npar, wb = C.c_int(), C.c_int(), C.c_size_t(), C.c_size_t()
        assert lib.dg_indicator_sizes(order, C.byref(nf), C.byref(npad), C.byref(npar), C.byref(wb)) == dg.DG_OK
        assert nf.value == F and npad.value == Fp
        assert npar.value == 64 * Fp + 64 + 64 * 64 + 64 + 64 + 1
        assert wb.value >= 4 * (npar.value + 1)
    for order in (0, 1, 5):
        assert lib.dg_indicator_sizes(order, None, None, None, None) == dg.DG_ERR_ARG


def test_device_free_calls_reject_bad_arguments(lib):
    p = C.c_void_p(16)
    assert lib.dg_indicator_forward(3, None, 4, p, p, None) == dg.DG_ERR_ARG
    assert lib.dg_indicator_forward(3, p, -1, p, p, None) == dg.DG_ERR_ARG
    assert lib.dg_indicator_forward(1, p, 4, p, p, None) == dg.DG_ERR_ARG
    assert lib.dg_indicator_backward(3, p, p, 0, 1.0, p, p, p, 1 << 20, None) == dg.DG_ERR_ARG
    assert lib.dg_indicator_backward(3, p, p, 4, 0.0, p, p, p, 1 << 20, None) == dg.DG_ERR_ARG
    assert lib.dg_indicator_adam(p, p, p, p, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == dg.DG_ERR_ARG
    assert lib.dg_indicator_adam(None, p, p, p, 10, 1e-3, 0.9, 0.999, 1e-8, 1, None) == dg.DG_ERR_ARG
    mm = C.c_longlong()
    assert lib.dg_selftest_conversions(-1, 0, C.byref(mm)) == dg.DG_ERR_ARG
    assert lib.dg_selftest_conversions(10, 0, None) == dg.DG_ERR_ARG
    assert lib.dg_probe_fma_peak(1, None) == dg.DG_ERR_ARG
