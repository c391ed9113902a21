"""Memory safety of the DG kernels, checked on the CPU: the role
compute-sanitizer plays on a GPU, with the kernel sources compiled by g++
under AddressSanitizer and UndefinedBehaviorSanitizer in a host emulation of
the CUDA thread model (tests/host_emulation: one OS thread per CUDA thread,
barriers for __syncthreads and warp shuffles, shared memory poisoned). Every
global, shared and table access of the face, volume, stage, limiter, energy
reset, forcing-field, CFL, diagnostics and spectrum/PDF kernels is
bounds-checked on meshes whose cell
count leaves ragged tiles, at every degree and in both precisions, with the
launch sizes of the library's launchers and in the order the C ABI issues
the kernels. The results are compared with the oracle only to confirm that
the emulation ran the kernels' arithmetic; parity of the GPU path itself is
what the -m gpu tests check."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_09079_gb300", "csrc")
EMU = os.path.join(ROOT, "tests", "host_emulation")
FLAGS = ["-std=c++20", "-O1", "-g", "-pthread", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
         "-fno-omit-frame-pointer"]


_DYN_SMEM = re.compile(r"extern __shared__ (?:__align__\(\d+\) )?([A-Za-z_][\w ]*?) (\w+)\[\];")


def _host_smem(src):
    """Dynamic shared memory (extern __shared__ T name[];) taken from the
    emulated block's buffer."""
    s = _DYN_SMEM.sub(lambda m: f"{m.group(1)}* {m.group(2)} = reinterpret_cast<{m.group(1)}*>(emu::dyn_smem());",
                      src)
    assert "extern __shared__" not in s
    return s


def _generate(dst):
    """The kernel headers with host dynamic shared memory, the table builder
    of dg_api.cu and the analysis kernels of dg_spectrum.cu."""
    for f in ("dg_common.cuh", "dg_kernels.cuh", "dg_fused.cuh", "dg_launch.h"):
        open(os.path.join(dst, f), "w").write(_host_smem(open(os.path.join(CSRC, f)).read()))
    api = open(os.path.join(CSRC, "dg_api.cu")).read()
    a = api.index("// ----------------------------------------------------------------- tables")
    b = api.index("Launchers launchers_for(int k)")
    open(os.path.join(dst, "tables.inc"), "w").write(api[a:b] + "}  // namespace\n")
    # the analysis kernels of dg_spectrum.cu (without the cuFFT plan helper)
    sp = open(os.path.join(CSRC, "dg_spectrum.cu")).read()
    a = sp.index("namespace {\n") + len("namespace {\n")
    b = sp.index("}  // namespace\n", a)
    body = sp[a:b]
    p0 = body.index("// cuFFT plan of")
    p1 = body.index("\n}\n", p0) + 3
    open(os.path.join(dst, "spectrum_kernels.inc"), "w").write(_host_smem(body[:p0] + body[p1:]))
    # the C ABI's own helper kernels (layout transposes, reductions)
    a = api.index("// ------------------------------------------------------ helper kernels")
    b = api.index("size_t align256(size_t b)")
    open(os.path.join(dst, "api_kernels.inc"), "w").write(_host_smem(api[a:b]))
    # the indicator's kernels (dg_mlp.cu up to its host dispatch), with the
    # inline-PTX mma.sync replaced by the emulation's warp-level product
    ml = open(os.path.join(CSRC, "dg_mlp.cu")).read()
    a = ml.index("namespace {\n") + len("namespace {\n")
    b = ml.index("// ------------------------------------------------------------ dispatch")
    body = ml[a:b]
    m0 = body.index("__device__ __forceinline__ void mma(")
    m1 = body.index("\n}\n", m0) + 3
    body = body[:m0] + ("__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], "
                        "const uint32_t (&b)[2]) {\n  emu::mma_bf16(d, a, b);\n}\n") + body[m1:]
    assert "asm" not in body
    open(os.path.join(dst, "mlp_kernels.inc"), "w").write(_host_smem(body))


@pytest.fixture(scope="module")
def drivers():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="dg_host_emu_")
    _generate(d)

    def build(k):
        exe = os.path.join(d, f"driver_k{k}")
        cmd = ["g++", *FLAGS, "-I", EMU, "-I", d, "-include", os.path.join(EMU, "emu.h"), f"-DDG_K={k}",
               os.path.join(EMU, "driver.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-4000:]
        return exe

    with cf.ThreadPoolExecutor(4) as ex:
        exes = list(ex.map(build, range(4)))
    yield d, exes
    shutil.rmtree(d, ignore_errors=True)


def _layout(w):
    nc = w.shape[0] * w.shape[1] * w.shape[2]
    return np.ascontiguousarray(w.reshape(nc, 5, w.shape[-1]).transpose(1, 2, 0))


def _canonical(y, shape):
    nc = shape[0] * shape[1] * shape[2]
    return y.reshape(5, shape[-1], nc).transpose(2, 0, 1).reshape(shape)


def _run(exe, args, d):
    r = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=900, cwd=d)
    assert r.returncode == 0, (r.returncode, r.stderr[-4000:])
    return dict(kv.split("=") for kv in r.stdout.split())


def normwise(a, b):
    return max(np.max(np.abs(a[..., i, :] - b[..., i, :])) / np.max(np.abs(b[..., i, :])) for i in range(5))


N_MESH = (5, 3, 7)  # 105 cells: ragged tiles of 8, 32 and 256 cells


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_rhs_kernels_clean(drivers, k, prec):
    d, exes = drivers
    g = syn.GAMMA
    w = syn.random_state(N_MESH, oracle.nmodes(k), g, seed=40 + k, high=0.01)
    fin, fout = os.path.join(d, f"r{k}{prec}.in"), os.path.join(d, f"r{k}{prec}.out")
    _layout(w).tofile(fin)
    info = _run(exes[k], ["rhs", *N_MESH, prec, repr(g), fin, fout], d)
    assert info["err"] == "0"
    R = _canonical(np.fromfile(fout), w.shape)
    assert normwise(R, oracle.Oracle(N_MESH, k, g).rhs(w)) <= (1e-12 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_step_kernels_clean(drivers, k, prec):
    """A driven step whose high modes are large enough for the limiter to
    act in every stage (queued cells, theta1 and theta2), then the energy
    reset and the CFL reduction; against the oracle's step and reset (FP64
    to 1e-9: the pressure Newton iteration near the 1e-12 floor is
    ill-conditioned, mixed to 1e-5)."""
    d, exes = drivers
    g = syn.GAMMA
    n = N_MESH
    w = syn.random_state(n, oracle.nmodes(k), g, seed=50 + k, high=0.3)
    nv = syn.driving_modes(1.0, 2.0)
    ah = np.random.default_rng(60 + k).normal(size=(len(nv), 6)) * 0.5
    o = oracle.Oracle(n, k, g)
    o.set_forcing(nv, ah)
    st, dt = o.cfl_dt(w, 0.3)
    assert st == 0
    st, w1 = o.step(w, dt)
    assert st == 0
    st, w2, dref = o.energy_reset(w1, 0.7, 1.0)
    assert st == 0
    fin, fout, fm = (os.path.join(d, f"s{k}{prec}.{x}") for x in ("in", "out", "modes"))
    _layout(w).tofile(fin)
    np.ascontiguousarray(np.concatenate([nv.astype(np.float64), ah], axis=1)).tofile(fm)
    info = _run(exes[k], ["step", *n, prec, repr(g), fin, fout, repr(dt), len(nv), fm, 0.7, 1.0, 0], d)
    assert info["err"] == "0"
    y = _canonical(np.fromfile(fout), w.shape)
    assert normwise(y, w2) <= (1e-9 if prec == 0 else 1e-5)
    assert abs(float(info["dissipated"]) - dref) <= (1e-9 if prec == 0 else 1e-5) * abs(dref)
    # the CFL reduction saw the reset state
    assert float(info["smax"]) > 0


def test_step_with_volume_limiter_points_clean(drivers):
    d, exes = drivers
    g, k, n = syn.GAMMA, 2, N_MESH
    w = syn.random_state(n, oracle.nmodes(k), g, seed=70, high=0.3)
    o = oracle.Oracle(n, k, g, limiter_points=oracle.LIMIT_S_VOLUME)
    st, dt = o.cfl_dt(w, 0.3)
    st, w1 = o.step(w, dt)
    assert st == 0
    st, w2, dref = o.energy_reset(w1, 0.7, 1.0)
    fin, fout = os.path.join(d, "v.in"), os.path.join(d, "v.out")
    _layout(w).tofile(fin)
    info = _run(exes[k], ["step", *n, 1, repr(g), fin, fout, repr(dt), 0, fin, 0.7, 1.0, 1], d)
    assert info["err"] == "0"
    assert normwise(_canonical(np.fromfile(fout), w.shape), w2) <= 1e-5


def _hllc(exe, d, g, UL, UR, tmp):
    info = _run(exe, ["hllc", d, repr(g), *(repr(float(x)) for x in UL), *(repr(float(x)) for x in UR)], tmp)
    return (np.array([float(x) for x in info["f32"].split(",")]),
            np.array([float(x) for x in info["f64"].split(",")]))


def _cons(rho, v, p, g):
    return [rho, rho * v[0], rho * v[1], rho * v[2], p / (g - 1) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)]


def test_fp32_hllc_receding_vacuum_states(drivers):
    """FP32 traces of a state limited in FP64 can round both face pressures
    to <= 0; the sound speeds are then clamped to zero, and in a receding
    flow (u_L < 0 < u_R) both HLLC wave speeds equal the fluid velocities,
    so the contact-speed denominator vanishes. The flux must stay finite:
    (0, p_L e_d, 0), the flux at a vacuum interface. Away from that case
    the FP32 flux equals the FP64 one to FP32 rounding."""
    d, exes = drivers
    g = syn.GAMMA
    for dirn in range(3):
        vL, vR = np.zeros(3), np.zeros(3)
        vL[dirn], vR[dirn] = -0.24, 0.12
        vL[(dirn + 1) % 3] = 0.07
        pL = -1e-4  # pressures below zero, as FP32 rounding can leave them
        UL = _cons(0.9989, vL, pL, g)
        UR = _cons(0.9451, vR, -3e-4, g)
        f32, _ = _hllc(exes[2], dirn, g, UL, UR, d)
        assert np.all(np.isfinite(f32)), f32
        expect = np.zeros(5)
        expect[1 + dirn] = pL
        assert np.max(np.abs(f32 - expect)) <= 1e-7, f32
        # and the mirrored pair (the contact speed from the other side)
        f32m, _ = _hllc(exes[2], dirn, g, UR, UL, d)
        assert np.all(np.isfinite(f32m))
    rng = np.random.default_rng(3)
    for _ in range(20):
        dirn = int(rng.integers(3))
        UL = _cons(rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.2, 2), g)
        UR = _cons(rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.2, 2), g)
        f32, f64 = _hllc(exes[2], dirn, g, UL, UR, d)
        assert np.max(np.abs(f32 - f64)) <= 1e-5 * max(1.0, np.max(np.abs(f64)))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_exact_flux_rhs_clean(drivers, k, prec):
    """The exact-Riemann-solver face kernels (dg_set_flux) on strong jumps
    between neighbouring cell means (limited first, as a step would)."""
    d, exes = drivers
    g = syn.GAMMA
    w = syn.random_state(N_MESH, oracle.nmodes(k), g, seed=80 + k, high=0.1, rho_mean=(0.2, 2.0),
                         v_mean=(-2.0, 2.0), p_mean=(0.1, 2.0))
    o = oracle.Oracle(N_MESH, k, g, flux=oracle.FLUX_EXACT)
    st, w, _, _ = o.limit(w)
    assert st == 0
    fin, fout = os.path.join(d, f"e{k}{prec}.in"), os.path.join(d, f"e{k}{prec}.out")
    _layout(w).tofile(fin)
    info = _run(exes[k], ["rhs", *N_MESH, prec, repr(g), fin, fout, 1], d)
    assert info["err"] == "0"
    R = _canonical(np.fromfile(fout), w.shape)
    assert normwise(R, o.rhs(w)) <= (1e-12 if prec == 0 else 2e-5)


@pytest.mark.parametrize("mode", ["hllc", "exact"])
def test_fp32_fluxes_finite_near_vacuum(drivers, mode):
    """Near-vacuum face states (pressures at, near or rounded below zero;
    receding, approaching and resting flows; every direction): the FP32
    fluxes are finite and the exact solver's Newton iteration converges."""
    d, exes = drivers
    g = syn.GAMMA
    for pl, pr in ((-1e-4, -3e-4), (-2e-9, -6e-9), (1e-9, -6e-9), (0.0, 0.0), (1e-12, 1e-12), (1e-30, 1e-20)):
        for ul, ur in ((-0.24, 0.12), (0.3, -0.2), (-2.0, 2.0), (0.0, 0.0)):
            for dirn in range(3):
                vL, vR = [0.0] * 3, [0.0] * 3
                vL[dirn], vR[dirn] = ul, ur
                vL[(dirn + 1) % 3] = 0.07
                info = _run(exes[2], [mode, dirn, repr(g), *(repr(float(x)) for x in _cons(0.9989, vL, pl, g)),
                                      *(repr(float(x)) for x in _cons(0.9451, vR, pr, g))], d)
                f32 = np.array([float(x) for x in info["f32"].split(",")])
                assert np.all(np.isfinite(f32)) and info["e32"] == "0", (mode, pl, pr, ul, ur, dirn, f32)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_analysis_kernels_clean(drivers, k):
    """Diagnostics partial sums (FP64 and FP32 driving field), the velocity
    sampling, ln(rho) histogram and shell-sum kernels of the spectrum and
    PDF (the FFT between them taken by numpy), on a 3^3 mesh with 3^3
    samples per cell."""
    d, exes = drivers
    g, n, sub, nb, lo, hi = syn.GAMMA, 3, 3, 24, -0.3, 0.3
    N = oracle.nmodes(k)
    w = syn.random_state((n, n, n), N, g, seed=90 + k, high=0.05)
    nv = syn.driving_modes(1.0, 2.0)
    ah = np.random.default_rng(91 + k).normal(size=(len(nv), 6)) * 0.5
    o = oracle.Oracle((n, n, n), k, g)
    o.set_forcing(nv, ah)
    M = n * sub
    vel = [o.sample_velocity(w, sub, c) for c in range(3)]
    spec = np.stack([np.fft.rfftn(v) for v in vel])  # [3][M][M][M/2+1], layout [z][y][x]
    fin, fout, fm, fs = (os.path.join(d, f"a{k}.{x}") for x in ("in", "out", "modes", "spec"))
    _layout(w).tofile(fin)
    np.ascontiguousarray(np.concatenate([nv.astype(np.float64), ah], axis=1)).tofile(fm)
    np.ascontiguousarray(spec.astype(np.complex128)).view(np.float64).tofile(fs)
    _run(exes[k], ["analysis", n, repr(g), fin, fout, sub, lo, hi, nb, len(nv), fm, fs], d)
    out = np.fromfile(fout)
    ref = o.diagnostics(w)
    assert np.max(np.abs(out[0:3] - ref) / np.maximum(np.abs(ref), 1e-300)) <= 1e-12
    assert np.max(np.abs(out[3:6] - ref) / np.maximum(np.abs(ref), 1e-300)) <= 1e-5
    M3 = M ** 3
    for c in range(3):
        got = out[6 + c * M3: 6 + (c + 1) * M3]
        assert np.max(np.abs(got - vel[c].ravel())) <= 1e-13 * np.max(np.abs(vel[c]))
    cnt = out[6 + 3 * M3: 6 + 3 * M3 + nb + 2]
    assert np.array_equal(cnt.astype(np.int64), o.density_pdf(w, sub, lo, hi, nb))
    bins = out[6 + 3 * M3 + nb + 2:]
    E = o.velocity_spectrum(w, sub)
    assert len(bins) == len(E) and np.max(np.abs(bins - E)) <= 1e-12 * E.sum()


@pytest.mark.parametrize("k", [2, 3])
def test_kernels_race_free_under_tsan(k, tmp_path):
    """The same kernels under ThreadSanitizer (shared-memory races between
    the emulated CUDA threads of a block: a missing __syncthreads, a buffer
    reused too early): R and a driven step with the limiter active, both
    precisions."""
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = str(tmp_path)
    _generate(d)
    exe = os.path.join(d, "tsan")
    flags = [f for f in FLAGS if not f.startswith("-fsanitize") and f != "-fno-sanitize-recover=undefined"]
    r = subprocess.run(["g++", *flags, "-fsanitize=thread", "-I", EMU, "-I", d, "-include", os.path.join(EMU, "emu.h"),
                        f"-DDG_K={k}", os.path.join(EMU, "driver.cpp"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    g, n = syn.GAMMA, N_MESH
    w = syn.random_state(n, oracle.nmodes(k), g, seed=100 + k, high=0.3)
    fin, fout = os.path.join(d, "t.in"), os.path.join(d, "t.out")
    _layout(w).tofile(fin)
    st, dt = oracle.Oracle(n, k, g).cfl_dt(w, 0.3)
    assert st == 0
    for prec in (0, 1):
        for args in (["rhs", *n, prec, repr(g), fin, fout],
                     ["step", *n, prec, repr(g), fin, fout, repr(dt), 0, fin, 0.7, 1.0, 0]):
            rr = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=1800,
                                env=dict(os.environ, TSAN_OPTIONS="halt_on_error=1"))
            if "unexpected memory mapping" in rr.stderr:
                pytest.skip("ThreadSanitizer cannot run on this host's memory layout")
            assert rr.returncode == 0 and "WARNING: ThreadSanitizer" not in rr.stderr, rr.stderr[-4000:]


@pytest.mark.parametrize("lim_vol", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_limiter_with_flags_clean(drivers, k, lim_vol):
    """dg_limit's kernel with per-cell flags on states whose polynomials
    leave the positive set (floors 1e-2), both point sets: flags bit-exact
    and the state within 1e-12 of the oracle's limiter."""
    d, exes = drivers
    g, n, eps = 1.4, N_MESH, 1e-2
    w = syn.random_state(n, oracle.nmodes(k), g, seed=110 + k, high=0.5)
    o = oracle.Oracle(n, k, g, eps_rho=eps, eps_p=eps, limiter_points=lim_vol)
    st, ref, fref, nref = o.limit(w)
    assert st == 0 and nref > 5
    fin, fout, ffl = (os.path.join(d, f"l{k}{lim_vol}.{x}") for x in ("in", "out", "flags"))
    _layout(w).tofile(fin)
    info = _run(exes[k], ["limit", *n, repr(g), repr(eps), lim_vol, fin, fout, ffl], d)
    assert info["err"] == "0" and int(info["n_limited"]) == nref
    assert np.array_equal(np.fromfile(ffl, dtype=np.int8), np.asarray(fref, dtype=np.int8).ravel())
    assert normwise(_canonical(np.fromfile(fout), w.shape), ref) <= 1e-12


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_projection_range_clean(drivers, k):
    """dg_project_range's kernel on a range of cells that ends in a ragged
    block: the projected weights of those cells equal the oracle's
    projection of the same point values."""
    d, exes = drivers
    g, n = syn.GAMMA, N_MESH
    o = oracle.Oracle(n, k, g)
    fn = syn.solenoidal_velocity(seed=5, mach=0.3)
    xyz = o.volume_points()
    vals = np.moveaxis(np.asarray(fn(xyz[..., 0], xyz[..., 1], xyz[..., 2])), 0, 1)  # [nc][5][Q^3]
    ref = o.project(vals).reshape(o.ncells, 5, -1)
    first, count = 17, 61
    fin, fout = os.path.join(d, f"p{k}.in"), os.path.join(d, f"p{k}.out")
    np.ascontiguousarray(vals[first:first + count]).tofile(fin)
    _run(exes[k], ["project", *n, repr(g), first, count, fin, fout], d)
    y = _canonical(np.fromfile(fout), (n[2], n[1], n[0], 5, oracle.nmodes(k))).reshape(o.ncells, 5, -1)
    assert np.all(np.isnan(y[:first])) and np.all(np.isnan(y[first + count:]))  # other cells untouched
    assert np.max(np.abs(y[first:first + count] - ref[first:first + count])) <= 1e-14 * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def mlp_drivers(drivers):
    d, _ = drivers

    def build(k):
        exe = os.path.join(d, f"mlp_k{k}")
        cmd = ["g++", *FLAGS, "-I", EMU, "-I", d, "-include", os.path.join(EMU, "emu.h"), f"-DDG_K={k}",
               os.path.join(EMU, "mlp_driver.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-4000:]
        return exe

    with cf.ThreadPoolExecutor(3) as ex:
        exes = dict(zip((1, 2, 3), ex.map(build, (1, 2, 3))))
    return d, exes


@pytest.mark.parametrize("order", [2, 3, 4])
def test_indicator_kernels_clean(mlp_drivers, order):
    """The learned indicator's features, BF16 forward and backward kernels
    (mma.sync m16n8k16 emulated at the warp from its documented fragment
    layout): bounds-checked, and within the GPU tests' criteria of the
    oracle (features within one BF16 ulp, logits within 5e-3 of their scale,
    gradients within 2e-2 relative L2 and 0.999 cosine)."""
    torch = pytest.importorskip("torch")
    import test_gpu_indicator as T  # the mirrored-oracle helpers (numpy / torch on the CPU)
    from oracle import mlp
    d, exes = mlp_drivers
    k, g = order - 1, syn.GAMMA
    F = mlp.n_features_padded(k)
    exe = exes[k]

    def bits(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).view(torch.int16).numpy()

    def unbits(b):
        return torch.from_numpy(b).view(torch.bfloat16).to(torch.float64).numpy()

    n = (7, 6, 5)
    nc = n[0] * n[1] * n[2]
    w = syn.random_state(n, oracle.nmodes(k), g, seed=120 + order, high=0.05)
    f = lambda x: os.path.join(d, f"i{order}.{x}")  # noqa: E731
    _layout(w).tofile(f("in"))
    _run_plain(exe, ["features", *n, repr(g), f("in"), f("X")], d)
    got = unbits(np.fromfile(f("X"), dtype=np.int16).reshape(nc, F))
    ref = T.bf16(mlp.features(w, k, g))
    assert np.all(np.abs(got - ref) <= np.abs(ref) * 2.0 ** -7 + 1e-30)

    rng = np.random.default_rng(130 + order)
    N = 300  # three 128-row tiles, the last ragged
    X = T.bf16(rng.normal(size=(N, F)))
    P = T.rand_params(F, 131 + order)
    bits(X).tofile(f("fx"))
    T.flat(P).tofile(f("P"))
    _run_plain(exe, ["forward", N, f("fx"), f("P"), f("lg")], d)
    lg = np.fromfile(f("lg"), dtype=np.float32).astype(np.float64)
    Q = T.mirrored(P)
    cache = T.forward_mirrored(Q, X)
    assert np.all(np.isfinite(lg))
    assert np.max(np.abs(lg - cache["logit"])) <= 5e-3 * np.max(np.abs(cache["logit"])) + 1e-4

    y = (rng.uniform(size=N) < 0.3).astype(np.float64)
    a = 3.0
    y.astype(np.float32).tofile(f("y"))
    _run_plain(exe, ["backward", N, repr(a), f("fx"), f("y"), f("P"), f("G")], d)
    gv = np.fromfile(f("G"), dtype=np.float32).astype(np.float64)
    npar = len(T.flat(P))
    assert abs(gv[npar] - mlp.loss(cache["logit"], y, a)) <= 1e-3 * abs(mlp.loss(cache["logit"], y, a))
    got = T.unflat(gv[:npar], F)
    gref = mlp.backward(Q, X, cache, y, a)
    for key in gref:
        r, q = gref[key].ravel(), got[key].ravel()
        rel = np.linalg.norm(q - r) / max(np.linalg.norm(r), 1e-30)
        cos = q @ r / max(np.linalg.norm(q) * np.linalg.norm(r), 1e-30)
        assert rel <= 2e-2 and cos >= 0.999, (key, rel, cos)


def _run_plain(exe, args, d):
    r = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=900, cwd=d)
    assert r.returncode == 0, (r.returncode, r.stderr[-4000:])


def test_indicator_gate_and_adam_clean(mlp_drivers):
    """The gate kernel (features and forward of the limiter queue, cells
    whose logit reaches the threshold appended with atomics) and the Adam
    kernel, order 3: the gated set equals the oracle's away from the
    threshold; Adam equals the update written out in numpy."""
    pytest.importorskip("torch")
    import test_gpu_indicator as T
    from oracle import mlp
    d, exes = mlp_drivers
    k, g, n = 2, syn.GAMMA, (7, 6, 5)
    nc = n[0] * n[1] * n[2]
    F = mlp.n_features_padded(k)
    w = syn.random_state(n, oracle.nmodes(k), g, seed=140, high=0.05)
    P = T.rand_params(F, 141)
    queue = np.sort(np.random.default_rng(142).choice(nc, size=150, replace=False)).astype(np.int32)
    logit = T.forward_mirrored(T.mirrored(P), T.bf16(mlp.features(w, k, g)[queue]))["logit"]
    thr = float(np.median(logit))
    f = lambda x: os.path.join(d, f"gate.{x}")  # noqa: E731
    _layout(w).tofile(f("in"))
    queue.tofile(f("list"))
    T.flat(P).tofile(f("P"))
    _run_plain(exes[k], ["gate", *n, repr(g), f("in"), f("list"), len(queue), f("P"), repr(thr), f("out")], d)
    got = set(np.fromfile(f("out"), dtype=np.int32).tolist())
    margin = 5e-3 * np.max(np.abs(logit)) + 1e-4
    assert set(queue[logit >= thr + margin].tolist()) <= got
    assert not (got & set(queue[logit < thr - margin].tolist()))
    assert got <= set(queue.tolist())

    rng = np.random.default_rng(143)
    m_ = 1000
    p, m, v, gr = (rng.normal(size=m_).astype(np.float32) for _ in range(4))
    v = np.abs(v)
    for arr, x in ((p, "p"), (m, "m"), (v, "v"), (gr, "g")):
        arr.tofile(f(x))
    step, lr = 3, 1e-3
    _run_plain(exes[k], ["adam", m_, step, repr(lr), f("p"), f("m"), f("v"), f("g")], d)
    out = np.fromfile(f("g"), dtype=np.float32).reshape(3, m_).astype(np.float64)
    b1, b2, eps = 0.9, 0.999, 1e-8
    m1 = b1 * m + (1 - b1) * gr
    v1 = b2 * v + (1 - b2) * gr.astype(np.float64) ** 2
    p1 = p - lr * (m1 / (1 - b1 ** step)) / (np.sqrt(v1 / (1 - b2 ** step)) + eps)
    for got_, ref in zip(out, (p1, m1, v1)):
        assert np.max(np.abs(got_ - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("k", [1, 3])
def test_layout_and_totals_kernels_clean(drivers, k):
    """The C ABI's canonical <-> state transposes (32 x 8 thread blocks,
    32 x 33 shared tiles; ragged in cells and in rows 5 N) round-trip a
    state exactly, and the totals reduction matches the cell-mean sums."""
    d, exes = drivers
    n = (5, 3, 7)
    nc = n[0] * n[1] * n[2]
    w = syn.random_state(n, oracle.nmodes(k), syn.GAMMA, seed=150 + k, high=0.1)
    fin, fout = os.path.join(d, f"y{k}.in"), os.path.join(d, f"y{k}.out")
    np.ascontiguousarray(w).tofile(fin)
    _run_plain(exes[k], ["layout", *n, fin, fout], d)
    out = np.fromfile(fout)
    R = 5 * oracle.nmodes(k)
    st, back, sums = out[:nc * R], out[nc * R:2 * nc * R], out[2 * nc * R:]
    assert np.array_equal(st, _layout(w).ravel())
    assert np.array_equal(back, w.ravel())
    ref = w.reshape(nc, 5, -1)[:, :, 0].sum(axis=0) / nc
    assert np.max(np.abs(sums - ref)) <= 1e-14 * np.max(np.abs(ref))
