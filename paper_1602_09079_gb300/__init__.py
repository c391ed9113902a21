"""GB300 (sm_103a) modal discontinuous Galerkin solver for the 3D Euler
equations on periodic Cartesian meshes, after Bauer et al.,
arXiv:1602.09079 (TENET), Sect. 2-3.

The compute path is the CUDA library ``libdg_gb300.so`` behind the C ABI of
``include/dg.h``. This module is a thin ctypes binding with the same function
names (argument marshalling only), plus ``Solver``, which allocates the
caller-owned device buffers with PyTorch and binds them on the current torch
CUDA stream. There is no CPU fallback: every call fails loudly if the
library cannot be built or loaded, or if no CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import _build

DG_OK, DG_ERR_ARG, DG_ERR_NOT_BOUND, DG_ERR_CUDA = 0, -1, -2, -3
DG_ERR_NONFINITE, DG_ERR_POSITIVITY, DG_ERR_NEWTON, DG_ERR_TOO_LARGE = -4, -5, -6, -7
DG_PREC_FP64, DG_PREC_MIXED = 0, 1
DG_FLUX_HLLC, DG_FLUX_EXACT = 0, 1
DG_LIMIT_S, DG_LIMIT_S_VOLUME = 0, 1
DG_FEATURE_FORCING = 1

_lock = threading.Lock()
_lib = None


class DGError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {dg_strerror(code)} ({code})")


class dg_mesh(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("length", C.c_double * 3)]


_SIGS = {
    "dg_strerror": (C.c_char_p, [C.c_int]),
    "dg_init": (C.c_int, [C.POINTER(dg_mesh), C.c_int, C.c_double, C.POINTER(C.c_void_p)]),
    "dg_destroy": (None, [C.c_void_p]),
    "dg_sizes": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "dg_bind": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dg_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_quadrature_points": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_project": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_project_range": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "dg_quadrature_points_range": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]),
    "dg_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_step": (C.c_int, [C.c_void_p, C.c_double]),
    "dg_limit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "dg_cfl_dt": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "dg_set_precision": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_set_flux": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_set_limiter_points": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_set_eps": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    "dg_set_forcing": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dg_energy_reset": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.POINTER(C.c_double)]),
    "dg_totals": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_diagnostics": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dg_spectrum_sizes": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "dg_velocity_spectrum": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dg_density_pdf": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p]),
    "dg_check": (C.c_int, [C.c_void_p]),
    "dg_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_kernel_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_probe_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "dg_selftest_conversions": (C.c_int, [C.c_longlong, C.c_ulonglong, C.POINTER(C.c_longlong)]),
    "dg_rhs_noalloc": (C.c_int, [C.POINTER(dg_mesh), C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "dg_indicator_sizes": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t),
                                     C.POINTER(C.c_size_t)]),
    "dg_indicator_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_indicator_forward": (C.c_int, [C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_indicator_backward": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dg_indicator_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                    C.c_float, C.c_float, C.c_float, C.c_int, C.c_void_p]),
    "dg_set_indicator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_float]),
    "dg_indicator_capture": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_limiter_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
}

DG_KCLASS_COUNT = 6
KERNEL_CLASSES = ("limiter", "face_flux", "volume", "cfl", "energy_reset", "other")


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed) libdg_gb300.so; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            lib = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(code, where):
    if code != DG_OK:
        raise DGError(code, where)


def _ptr(x):
    """Raw address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


# ------------------------------------------------ C-ABI mirror (same names)

def dg_strerror(code: int) -> str:
    return load().dg_strerror(code).decode()


def dg_init(n, order, gamma, length=(1.0, 1.0, 1.0)):
    m = dg_mesh()
    for a in range(3):
        m.n[a] = int(n[a])
        m.length[a] = float(length[a])
    ctx = C.c_void_p()
    _check(load().dg_init(C.byref(m), int(order), float(gamma), C.byref(ctx)), "dg_init")
    return ctx


def dg_destroy(ctx):
    load().dg_destroy(ctx)


def dg_sizes(ctx, features=0):
    a, b = C.c_size_t(0), C.c_size_t(0)
    _check(load().dg_sizes(ctx, int(features), C.byref(a), C.byref(b)), "dg_sizes")
    return a.value, b.value


def dg_bind(ctx, y_dev, scratch_dev, scratch_bytes, stream):
    _check(load().dg_bind(ctx, _ptr(y_dev), _ptr(scratch_dev), int(scratch_bytes), _ptr(stream)), "dg_bind")


def dg_set_state(ctx, src, is_device):
    _check(load().dg_set_state(ctx, _ptr(src), int(is_device)), "dg_set_state")


def dg_get_state(ctx, dst, is_device):
    _check(load().dg_get_state(ctx, _ptr(dst), int(is_device)), "dg_get_state")


def dg_quadrature_points(ctx, xyz_host):
    _check(load().dg_quadrature_points(ctx, _ptr(xyz_host)), "dg_quadrature_points")


def dg_project(ctx, q_points_dev):
    _check(load().dg_project(ctx, _ptr(q_points_dev)), "dg_project")


def dg_project_range(ctx, q_points_dev, first, count):
    _check(load().dg_project_range(ctx, _ptr(q_points_dev), int(first), int(count)), "dg_project_range")


def dg_quadrature_points_range(ctx, first, count, xyz_host):
    _check(load().dg_quadrature_points_range(ctx, int(first), int(count), _ptr(xyz_host)),
           "dg_quadrature_points_range")


def dg_rhs(ctx, y_dev, R_dev):
    _check(load().dg_rhs(ctx, _ptr(y_dev), _ptr(R_dev)), "dg_rhs")


def dg_step(ctx, dt):
    _check(load().dg_step(ctx, float(dt)), "dg_step")


def dg_limit(ctx, flags_dev=None, want_count=False):
    n = C.c_int64(0)
    _check(load().dg_limit(ctx, _ptr(flags_dev), C.byref(n) if want_count else None), "dg_limit")
    return n.value if want_count else None


def dg_cfl_dt(ctx, courant):
    dt = C.c_double(0.0)
    _check(load().dg_cfl_dt(ctx, float(courant), C.byref(dt)), "dg_cfl_dt")
    return dt.value


def dg_set_precision(ctx, mode):
    _check(load().dg_set_precision(ctx, int(mode)), "dg_set_precision")


def dg_set_limiter_points(ctx, mode):
    _check(load().dg_set_limiter_points(ctx, int(mode)), "dg_set_limiter_points")


def dg_set_flux(ctx, flux):
    _check(load().dg_set_flux(ctx, int(flux)), "dg_set_flux")


def dg_set_eps(ctx, eps_rho, eps_p):
    _check(load().dg_set_eps(ctx, float(eps_rho), float(eps_p)), "dg_set_eps")


def dg_set_forcing(ctx, nvec, ahat):
    if nvec is None or len(nvec) == 0:
        _check(load().dg_set_forcing(ctx, 0, None, None), "dg_set_forcing")
        return
    nv = np.ascontiguousarray(nvec, dtype=np.int32).reshape(-1, 3)
    ah = np.ascontiguousarray(ahat, dtype=np.float64).reshape(-1, 6)
    _check(load().dg_set_forcing(ctx, len(nv), nv.ctypes.data, ah.ctypes.data), "dg_set_forcing")


def dg_energy_reset(ctx, c_iso, rho0=1.0, want_dissipated=False):
    d = C.c_double(0.0)
    _check(load().dg_energy_reset(ctx, float(c_iso), float(rho0), C.byref(d) if want_dissipated else None),
           "dg_energy_reset")
    return d.value if want_dissipated else None


def dg_diagnostics(ctx):
    out = np.zeros(3)
    _check(load().dg_diagnostics(ctx, out.ctypes.data), "dg_diagnostics")
    return out


def dg_spectrum_sizes(ctx, sub):
    b, nb = C.c_size_t(0), C.c_int(0)
    _check(load().dg_spectrum_sizes(ctx, int(sub), C.byref(b), C.byref(nb)), "dg_spectrum_sizes")
    return b.value, nb.value


def dg_velocity_spectrum(ctx, sub, work, work_bytes, n_bins):
    out = np.zeros(n_bins)
    _check(load().dg_velocity_spectrum(ctx, int(sub), _ptr(work), int(work_bytes), out.ctypes.data),
           "dg_velocity_spectrum")
    return out


def dg_density_pdf(ctx, sub, lo, hi, n_bins):
    out = np.zeros(n_bins + 2, dtype=np.int64)
    _check(load().dg_density_pdf(ctx, int(sub), float(lo), float(hi), int(n_bins), out.ctypes.data),
           "dg_density_pdf")
    return out


def dg_totals(ctx):
    out = np.zeros(5)
    _check(load().dg_totals(ctx, out.ctypes.data), "dg_totals")
    return out


def dg_check(ctx):
    _check(load().dg_check(ctx), "dg_check")


def dg_set_timing(ctx, on):
    _check(load().dg_set_timing(ctx, int(bool(on))), "dg_set_timing")


def dg_kernel_stats(ctx):
    """{class: (launches, ms)} since the last call; synchronises."""
    n = np.zeros(DG_KCLASS_COUNT, dtype=np.int64)
    ms = np.zeros(DG_KCLASS_COUNT)
    _check(load().dg_kernel_stats(ctx, n.ctypes.data, ms.ctypes.data), "dg_kernel_stats")
    return {name: (int(n[i]), float(ms[i])) for i, name in enumerate(KERNEL_CLASSES)}


def dg_rhs_noalloc(n, order, gamma, precision, y_dev, R_dev, stream, length=(1.0, 1.0, 1.0)):
    """R(y) into R_dev using the library's fixed device scratch instead of a
    caller allocation (see include/dg.h)."""
    m = dg_mesh()
    for a in range(3):
        m.n[a] = int(n[a])
        m.length[a] = float(length[a])
    _check(load().dg_rhs_noalloc(C.byref(m), int(order), float(gamma), int(precision), _ptr(y_dev), _ptr(R_dev),
                                 _ptr(stream)), "dg_rhs_noalloc")


def dg_indicator_sizes(order):
    """(n_features, n_padded, n_params, work_bytes)"""
    a, b, c, d = C.c_int(0), C.c_int(0), C.c_size_t(0), C.c_size_t(0)
    _check(load().dg_indicator_sizes(int(order), C.byref(a), C.byref(b), C.byref(c), C.byref(d)),
           "dg_indicator_sizes")
    return a.value, b.value, c.value, d.value


def dg_indicator_features(ctx, y_dev, X_dev):
    _check(load().dg_indicator_features(ctx, _ptr(y_dev), _ptr(X_dev)), "dg_indicator_features")


def dg_indicator_forward(order, X_dev, n, params_dev, logits_dev, stream):
    _check(load().dg_indicator_forward(int(order), _ptr(X_dev), int(n), _ptr(params_dev), _ptr(logits_dev),
                                       _ptr(stream)), "dg_indicator_forward")


def dg_indicator_backward(order, X_dev, labels_dev, n, pos_weight, params_dev, grads_dev, work_dev, work_bytes,
                          stream):
    _check(load().dg_indicator_backward(int(order), _ptr(X_dev), _ptr(labels_dev), int(n), float(pos_weight),
                                        _ptr(params_dev), _ptr(grads_dev), _ptr(work_dev), int(work_bytes),
                                        _ptr(stream)), "dg_indicator_backward")


def dg_indicator_adam(params, m, v, grads, n_params, lr, beta1, beta2, eps, step, stream):
    _check(load().dg_indicator_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grads), int(n_params), float(lr),
                                    float(beta1), float(beta2), float(eps), int(step), _ptr(stream)),
           "dg_indicator_adam")


def dg_set_indicator(ctx, params_dev, threshold=0.5):
    _check(load().dg_set_indicator(ctx, _ptr(params_dev), float(threshold)), "dg_set_indicator")


def dg_indicator_capture(ctx, dt, X_dev, flags_dev, screen_dev):
    _check(load().dg_indicator_capture(ctx, float(dt), _ptr(X_dev), _ptr(flags_dev), _ptr(screen_dev)),
           "dg_indicator_capture")


def dg_limiter_counts(ctx):
    q, f = C.c_int64(0), C.c_int64(0)
    _check(load().dg_limiter_counts(ctx, C.byref(q), C.byref(f)), "dg_limiter_counts")
    return q.value, f.value


def dg_selftest_conversions(n, seed=0):
    v = C.c_longlong(0)
    _check(load().dg_selftest_conversions(int(n), int(seed), C.byref(v)), "dg_selftest_conversions")
    return v.value


def dg_probe_fma_peak(fp64):
    v = C.c_double(0.0)
    _check(load().dg_probe_fma_peak(int(bool(fp64)), C.byref(v)), "dg_probe_fma_peak")
    return v.value


# ------------------------------------------------------------- convenience

def nmodes(k: int) -> int:
    return (k + 1) * (k + 2) * (k + 3) // 6


class Solver:
    """One mesh + degree on the current CUDA device. Allocates the state
    (state layout, [5][N][n_cells] FP64) and the scratch with torch and binds
    them with the current torch stream. Canonical-layout arrays
    ([nz][ny][nx][5][N]) go in and out through set_state/get_state."""

    def __init__(self, n, order, gamma, length=(1.0, 1.0, 1.0), forcing=False, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1602_09079_gb300 needs a CUDA device; there is no CPU fallback")
        load()
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n = tuple(int(v) for v in n)
        self.order = int(order)
        self.k = self.order - 1
        self.N = nmodes(self.k)
        self.Q = self.k + 1
        self.gamma = float(gamma)
        self.length = tuple(float(v) for v in length)
        self.ncells = self.n[0] * self.n[1] * self.n[2]
        with torch.cuda.device(self.device):
            self.ctx = dg_init(self.n, self.order, self.gamma, self.length)
            state_len, scratch = dg_sizes(self.ctx, DG_FEATURE_FORCING if forcing else 0)
            self.y = torch.empty(state_len, dtype=torch.float64, device=self.device)
            self.scratch = torch.empty(scratch, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device)
            dg_bind(self.ctx, self.y, self.scratch, scratch, self.stream.cuda_stream)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and _lib is not None:
            _lib.dg_destroy(ctx)
            self.ctx = None

    @property
    def state_shape(self):
        return (self.n[2], self.n[1], self.n[0], 5, self.N)

    # canonical <-> bound state
    def set_state(self, w):
        """w: canonical-layout state, a host array or a CUDA tensor (moved to
        this solver's device if it lives on another one)."""
        if hasattr(w, "data_ptr") and w.is_cuda:
            w = w.to(device=self.device, dtype=self.torch.float64).contiguous()
            if w.numel() != self.y.numel():
                raise ValueError(f"state has {w.numel()} values, the mesh needs {self.y.numel()}")
            dg_set_state(self.ctx, w, 1)
            self._keep = w  # the copy is enqueued on the bound stream
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            if w.size != self.y.numel():
                raise ValueError(f"state has {w.size} values, the mesh needs {self.y.numel()}")
            dg_set_state(self.ctx, w, 0)

    def get_state(self):
        out = np.empty(self.state_shape)
        dg_get_state(self.ctx, out, 0)
        return out

    def quadrature_points(self):
        xyz = np.empty((self.ncells, self.Q ** 3, 3))
        dg_quadrature_points(self.ctx, xyz)
        return xyz

    def project_fn(self, fn, chunk_cells=1 << 20):
        """Project a callable fn(x, y, z) -> (5, ...) at this library's own
        quadrature points (device-side projection), chunk_cells cells at a
        time."""
        Q3 = self.Q ** 3
        for first in range(0, self.ncells, chunk_cells):
            count = min(chunk_cells, self.ncells - first)
            xyz = np.empty((count, Q3, 3))
            dg_quadrature_points_range(self.ctx, first, count, xyz)
            vals = np.asarray(fn(xyz[..., 0], xyz[..., 1], xyz[..., 2]), dtype=np.float64)
            f = np.ascontiguousarray(np.moveaxis(vals, 0, 1))  # [count][5][Q3]
            fd = self.torch.from_numpy(f).to(self.device)
            dg_project_range(self.ctx, fd, first, count)
            self.stream.synchronize()

    def rhs(self, canonical=True):
        R = self.torch.empty_like(self.y)
        dg_rhs(self.ctx, None, R)
        if not canonical:
            return R
        return R.view(5 * self.N, self.ncells).t().contiguous().cpu().numpy().reshape(self.state_shape)

    def step(self, dt):
        dg_step(self.ctx, dt)

    def limit(self, want_flags=False):
        flags = self.torch.zeros(self.ncells, dtype=self.torch.int8, device=self.device) if want_flags else None
        n = dg_limit(self.ctx, flags, want_count=True)
        if want_flags:
            return n, flags.cpu().numpy()
        return n

    def cfl_dt(self, courant):
        return dg_cfl_dt(self.ctx, courant)

    def set_precision(self, mode):
        dg_set_precision(self.ctx, mode)

    def set_flux(self, flux):
        dg_set_flux(self.ctx, flux)

    def set_limiter_points(self, mode):
        dg_set_limiter_points(self.ctx, mode)

    def set_eps(self, eps_rho, eps_p):
        dg_set_eps(self.ctx, eps_rho, eps_p)

    def set_forcing(self, nvec, ahat):
        dg_set_forcing(self.ctx, nvec, ahat)

    def energy_reset(self, c_iso, rho0=1.0, want_dissipated=False):
        return dg_energy_reset(self.ctx, c_iso, rho0, want_dissipated)

    def totals(self):
        return dg_totals(self.ctx)

    def velocity_spectrum(self, sub=4):
        """Shell-summed velocity power spectrum on sub^3 samples per cell
        (work area allocated with torch for the call)."""
        nbytes, nb = dg_spectrum_sizes(self.ctx, sub)
        work = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)
        return dg_velocity_spectrum(self.ctx, sub, work, nbytes, nb)

    def density_pdf(self, sub, lo, hi, n_bins):
        """Counts of ln(rho) at sub^3 sub-cell centres per cell: [below lo,
        n_bins bins of [lo, hi), at or above hi]."""
        return dg_density_pdf(self.ctx, sub, lo, hi, n_bins)

    def diagnostics(self):
        """(rms Mach of the cell means, kinetic energy of the means,
        power of the driving force)."""
        return dg_diagnostics(self.ctx)

    def check(self):
        dg_check(self.ctx)

    def set_timing(self, on):
        dg_set_timing(self.ctx, on)

    def kernel_stats(self):
        return dg_kernel_stats(self.ctx)
