"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle (element by element where the
oracle finishes in seconds; sampled kernels and sampled destinations at the full 96^3 and 192^3 sizes).

Tolerances (relative L2 of the field after the stated steps, and per-kernel relative L2):
FP64 path <= 1e-12, FP32 <= 1e-5, FP16/BF16 storage <= 1e-3 with the total mass exact to 1e-12.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_11376_gb300 import FDiRW, FdirwError, fdirw, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()                      # no-op when libfdirw.so is up to date

FIELD_TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-3}
KERNEL_TOL = {"fp64": 1e-13, "fp32": 1e-5, "fp16": 2e-3, "bf16": 8e-3}
DEV = "cuda:0"


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(shape, seed, kind="two_phase", porosity=0.4, d_solid=1e-5):
    if kind == "rough":
        return synth.random_diffusivity(shape, seed, 6.0)
    p = synth.sphere_packing(shape, porosity, seed, r_range=(1.5, 3.5))
    return synth.diffusivity_two_phase(p, 1.0, d_solid) if kind == "two_phase" else synth.diffusivity_per_sphere(p)


def _gpu_run(shape, D, dt_sub, R, n_sub, c0, steps, prec, sources=None, parts=0):
    Dd = torch.from_numpy(D).to(DEV)
    cin = torch.from_numpy(np.ascontiguousarray(c0)).to(DEV)
    cout = torch.empty_like(cin)
    with FDiRW(shape, Dd, n_sub * dt_sub, R, n_sub, prec, march_parts=parts) as f:
        m = f.step(cin, cout, steps, want_mass=True)
        ks = f.read_kernels(sources) if sources is not None else None
        info = f.info()
    return cout.cpu().numpy(), m, ks, info


def _oracle_steps(shape, D, lam, R, n_sub, c0, steps):
    c = c0.copy()
    for _ in range(steps):
        c = oracle.superpose(shape, D, lam, R, n_sub, c)
    return c


def _oracle_at(shape, D, lam, R, n_sub, c, dests):
    """c'(x) for listed destinations: sum over the sources within L-inf distance R of x of c(s) k_s(x)."""
    nx, ny, nz = shape
    cond = oracle.Conductance(shape, D)
    out = []
    for x in dests:
        xx, xy, xz = x % nx, (x // nx) % ny, x // (nx * ny)
        src, offs = [], []
        for sz in range(max(xz - R, 0), min(xz + R, nz - 1) + 1):
            for sy in range(max(xy - R, 0), min(xy + R, ny - 1) + 1):
                for sx in range(max(xx - R, 0), min(xx + R, nx - 1) + 1):
                    src.append(sx + nx * (sy + ny * sz))
                    offs.append((xz - sz + R, xy - sy + R, xx - sx + R))
        ks, _ = oracle.kernels(shape, D, lam, R, n_sub, src, cond)
        out.append(sum(c[s] * ks[q][o] for q, (s, o) in enumerate(zip(src, offs))))
    return np.array(out)


# ------------------------------------------------------------------------- kernels, element by element

@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape,R,n_sub", [((20, 18, 16), 3, 50), ((21, 19, 18), 8, 60)])
def test_kernels_match_oracle(prec, shape, R, n_sub):
    D = _case(shape, 11)
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    src = np.arange(N)
    _, _, ks, _ = _gpu_run(shape, D, lam, R, n_sub, np.zeros(N), 0, prec, src)
    ref, _ = oracle.kernels(shape, D, lam, R, n_sub, src)
    ks = ks.reshape(N, -1)
    ref = ref.reshape(N, -1)
    err = np.linalg.norm(ks - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= KERNEL_TOL[prec], (prec, err.max())
    # FP64 renormalisation: every stored kernel times sigma sums to 1.
    assert np.max(np.abs(ks.sum(axis=1) - 1.0)) <= 1e-12
    assert ks.min() >= 0.0


@pytest.mark.parametrize("R", [9, 10])
def test_large_radius_mappings_agree_bitwise(R):
    """R = 9, 10 run on mapping 4 (2x2 blocks, one source per CTA), mapping 5 (one column per thread) and
    mapping 7 (column pairs): same bits."""
    shape = (23, 22, 21)
    D = _case(shape, 83, "per_sphere")
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    c0 = synth.random_field(N, 84)
    src = np.arange(1, N, 29)
    runs = [_gpu_run(shape, D, lam, R, 31, c0, 2, "fp32", src, parts=P) for P in (4, 5, 7)]
    assert [r[3]["march_parts"] for r in runs] == [4, 5, 7]
    for got, m, ks, info in runs[1:]:
        assert np.array_equal(runs[0][0], got) and np.array_equal(runs[0][2], ks)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("R", [9, 10])
def test_large_radius_kernels_match_oracle(prec, R):
    """R = 9, 10 (only the TMEM-face mapping): sampled kernels element by element, windows clipped by the
    domain on some sides and not on others."""
    shape = (25, 23, 22)
    D = _case(shape, 12, "per_sphere")
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    src = np.arange(3, N, 37)
    _, _, ks, info = _gpu_run(shape, D, lam, R, 45, np.zeros(N), 0, prec, src)
    assert info["march_parts"] in (4, 5)
    ref, _ = oracle.kernels(shape, D, lam, R, 45, src)
    ks = ks.reshape(len(src), -1)
    ref = ref.reshape(len(src), -1)
    err = np.linalg.norm(ks - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= KERNEL_TOL[prec], (prec, err.max())
    assert np.max(np.abs(ks.sum(axis=1) - 1.0)) <= 1e-12 and ks.min() >= 0.0


@pytest.mark.parametrize("R", [9, 10])
def test_large_radius_steps_match_oracle(R):
    shape = (16, 13, 12)
    D = _case(shape, 23, "two_phase")
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    c0 = synth.random_field(N, 24, 0.0, 2.0)
    for prec in ("fp32", "bf16"):
        got, m, _, _ = _gpu_run(shape, D, lam, R, 30, c0, 2, prec)
        ref = _oracle_steps(shape, D, lam, R, 30, c0, 2)
        assert _rel(got, ref) <= FIELD_TOL[prec], (prec, _rel(got, ref))
        assert abs(m - c0.sum()) <= 1e-12 * c0.sum()


# ------------------------------------------------------------------------- steps, element by element

@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape,R,n_sub,kind", [
    ((24, 16, 12), 3, 40, "two_phase"),   # aligned x: vectorised gather, several CTAs and batches
    ((13, 11, 9), 2, 25, "rough"),        # ragged x: scalar gather path
    ((16, 9, 7), 5, 30, "per_sphere"),    # windows larger than most of the domain
])
def test_steps_match_oracle(prec, shape, R, n_sub, kind):
    D = _case(shape, 21, kind)
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    c0 = synth.random_field(N, 22, 0.0, 2.0)
    got, m, _, _ = _gpu_run(shape, D, lam, R, n_sub, c0, 2, prec)
    ref = _oracle_steps(shape, D, lam, R, n_sub, c0, 2)
    assert _rel(got, ref) <= FIELD_TOL[prec], (prec, _rel(got, ref))
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workload_32_full(prec):
    """32^3, porosity 0.4, D 1/1e-5, R=3, n_sub=50 at the stability limit, 2 macro steps, c=1 in solid."""
    w = synth.WORKLOADS["fdirw-32c-r3"]
    p, D, c0 = w.make()
    shape = (w.n,) * 3
    lam = oracle.stable_dt_sub(shape, D)
    got, m, _, _ = _gpu_run(shape, D, lam, w.R, w.n_sub, c0, w.steps, prec)
    ref = _oracle_steps(shape, D, lam, w.R, w.n_sub, c0, w.steps)
    assert _rel(got, ref) <= FIELD_TOL[prec]
    assert abs(m - oracle.mass(c0)) <= 1e-12 * oracle.mass(c0)


# ------------------------------------------------------------------------- degenerate and edge cases

def test_window_covers_domain_equals_full_march():
    shape = (5, 4, 3)
    D = _case(shape, 31, "rough")
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(60, 32)
    for prec in ("fp64", "fp32"):
        got, _, _, _ = _gpu_run(shape, D, lam, 8, 17, c0, 1, prec)
        ref = oracle.full_march(shape, D, lam, 17, c0)
        assert _rel(got, ref) <= FIELD_TOL[prec]


@pytest.mark.parametrize("shape,R,n_sub,D_zero", [
    ((6, 5, 4), 2, 0, False),    # n_sub = 0
    ((6, 5, 4), 0, 9, False),    # R = 0
    ((6, 5, 4), 3, 9, True),     # D = 0 everywhere
    ((1, 1, 1), 4, 9, False),    # one cell
])
def test_identity_cases(shape, R, n_sub, D_zero):
    N = int(np.prod(shape))
    D = np.zeros(N) if D_zero else _case(shape, 41, "rough")
    c0 = synth.random_field(N, 42)
    for prec in ("fp64", "fp32", "bf16"):
        dt = oracle.stable_dt_sub(shape, D)
        dt = 0.1 if not np.isfinite(dt) else dt        # no faces at all: any substep is stable
        got, m, _, _ = _gpu_run(shape, D, dt, R, n_sub, c0, 3, prec)
        # FP64: exact; mixed path: the chat split keeps ~48 bits per step
        tol = 0.0 if prec == "fp64" else 1e-13
        assert np.allclose(got, c0, rtol=0, atol=tol * np.abs(c0).max()), prec


def test_one_dimensional_chain():
    shape = (64, 1, 1)
    D = _case(shape, 43, "rough")
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(64, 44)
    got, _, _, _ = _gpu_run(shape, D, lam, 6, 33, c0, 3, "fp64")
    assert _rel(got, _oracle_steps(shape, D, lam, 6, 33, c0, 3)) <= 1e-12


@pytest.mark.parametrize("R", [2, 5, 8])
def test_thread_mappings_agree_bitwise(R):
    """Every thread mapping of the FP32 march (1, 2 or 3 threads per window column, 2x2 column blocks
    with TMEM-resident coefficients, one column per thread with TMEM-resident lateral faces, one column
    of a source pair per thread in packed f32x2 arithmetic, or column pairs with TMEM-resident faces and
    diagonals) gives the same bits."""
    shape = (19, 17, 13)
    D = _case(shape, 81, "per_sphere")
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    c0 = synth.random_field(N, 82)
    src = np.arange(0, N, 7)
    runs = [_gpu_run(shape, D, lam, R, 37, c0, 2, "fp32", src, parts=P) for P in (1, 2, 3, 4, 5, 6, 7)]
    for got, m, ks, info in runs[1:]:
        assert np.array_equal(got, runs[0][0]) and np.array_equal(ks, runs[0][2]) and m == runs[0][1]
    assert [r[3]["march_parts"] for r in runs] == [1, 2, 3, 4, 5, 6, 7]
    ref, _ = oracle.kernels(shape, D, lam, R, 37, src)
    err = np.linalg.norm((runs[0][2] - ref).reshape(len(src), -1), axis=1) / np.linalg.norm(ref.reshape(len(src), -1), axis=1)
    assert err.max() <= KERNEL_TOL["fp32"]


@pytest.mark.parametrize("shape", [(1, 1, 40), (1, 37, 1), (33, 1, 1), (4, 1, 23), (1, 6, 19)])
def test_thin_domains_every_mapping(shape):
    """Grids one cell thick in one or two axes, so every window is clipped to a single column or row of
    columns (R = 3, and R = 8 beyond the thin extents): each FP32 thread mapping gives the same bits, the
    kernels of every source match the oracle, and so do two macro steps."""
    D = _case(shape, 91, "rough")
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    c0 = synth.random_field(N, 92)
    src = np.arange(N)
    for R in (3, 8):
        runs = [_gpu_run(shape, D, lam, R, 21, c0, 2, "fp32", src, parts=P) for P in (1, 2, 3, 4, 5, 6, 7)]
        for got, m, ks, info in runs[1:]:
            assert np.array_equal(got, runs[0][0]) and np.array_equal(ks, runs[0][2]) and m == runs[0][1]
        ref, _ = oracle.kernels(shape, D, lam, R, 21, src)
        err = np.linalg.norm((runs[0][2] - ref).reshape(N, -1), axis=1) / np.linalg.norm(ref.reshape(N, -1), axis=1)
        assert err.max() <= KERNEL_TOL["fp32"], (R, err.max())
        assert _rel(runs[0][0], _oracle_steps(shape, D, lam, R, 21, c0, 2)) <= FIELD_TOL["fp32"]


def test_deterministic_bitwise():
    shape = (24, 16, 12)
    D = _case(shape, 51)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(24 * 16 * 12, 52)
    for prec in ("fp64", "bf16"):
        a, ma, _, _ = _gpu_run(shape, D, lam, 4, 30, c0, 3, prec)
        b, mb, _, _ = _gpu_run(shape, D, lam, 4, 30, c0, 3, prec)
        assert np.array_equal(a, b) and ma == mb


def test_host_pointers_and_in_place():
    shape = (16, 12, 10)
    D = _case(shape, 61)
    lam = oracle.stable_dt_sub(shape, D)
    N = 1920
    c0 = synth.random_field(N, 62)
    dev, _, _, _ = _gpu_run(shape, D, lam, 3, 20, c0, 2, "fp32")
    with FDiRW(shape, D, 20 * lam, 3, 20, "fp32") as f:          # host D
        host_out = np.empty(N)
        m = f.step(c0, host_out, 2, want_mass=True)             # host in, host out
        assert np.array_equal(host_out, dev)
        assert m == f.mass(host_out)
        t = torch.from_numpy(c0.copy()).to(DEV)
        f.step(t, t, 2)                                         # in place on the device
        assert np.array_equal(t.cpu().numpy(), dev)
        t0 = torch.from_numpy(c0).to(DEV)
        f.step(t0, host_out, 2)                                 # device in, host out
        assert np.array_equal(host_out, dev)


def test_errors_are_reported():
    shape = (8, 8, 8)
    D = _case(shape, 71)
    lam = oracle.stable_dt_sub(shape, D)
    with pytest.raises(FdirwError) as e:
        FDiRW(shape, D, 10 * lam * 1.01, 2, 10)
    assert e.value.code == fdirw.FDIRW_ERR_UNSTABLE
    bad = D.copy()
    bad[5] = np.nan
    with pytest.raises(FdirwError) as e:
        FDiRW(shape, bad, 10 * lam, 2, 10)
    assert e.value.code == fdirw.FDIRW_ERR_ARG
    bad[5] = -1.0
    with pytest.raises(FdirwError) as e:
        FDiRW(shape, torch.from_numpy(bad).to(DEV), 10 * lam, 2, 10)
    assert e.value.code == fdirw.FDIRW_ERR_ARG
    with FDiRW(shape, D, 10 * lam, 2, 10) as f:
        base = f.info()["device_bytes"]                                    # everything but the cache
    plane = 125 * 64 * 4                                                   # one z-plane of FP32 kernels
    with FDiRW(shape, D, 10 * lam, 2, 10, mem_limit=base + 512 * 8 + plane - 1) as f:
        with pytest.raises(FdirwError) as e:                               # not even one plane fits
            f.kernels()
        assert e.value.code == fdirw.FDIRW_ERR_NOMEM
    with FDiRW(shape, D, 10 * lam, 2, 10, mem_limit=base + 512 * 8 + plane) as f:
        f.kernels()                                                        # one plane: 8 streamed slabs
        assert f.info()["n_chunks"] == 8
    with FDiRW(shape, D, 10 * lam, 2, 10) as f:
        with pytest.raises(FdirwError) as e:
            f.read_kernels([0])
        assert e.value.code == fdirw.FDIRW_ERR_STATE
        f.kernels()
        with pytest.raises(FdirwError) as e:
            f.read_kernels([512])
        assert e.value.code == fdirw.FDIRW_ERR_ARG
    assert abs(fdirw.fdirw_stable_dt(shape, D) - lam) <= 1e-15 * lam


# ------------------------------------------------------------------------- full-size workloads, sampled

def _sample_sources(shape, n_random, seed):
    nx, ny, nz = shape
    corners = [x + nx * (y + ny * z) for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)]
    edges = [nx // 2, nx * (ny // 2), nx * ny * (nz // 2) + nx - 1, (nx * ny * nz) // 2 + nx // 3]
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([corners, edges, rng.integers(0, nx * ny * nz, n_random)]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workload_96_sampled(prec):
    """96^3, porosity 0.35, per-sphere log10 D ratio U[3,8], R=6, n_sub=120, Gaussian blob."""
    w = synth.WORKLOADS["fdirw-96c-r6"]
    _, D, c0 = w.make()
    shape = (w.n,) * 3
    lam = oracle.stable_dt_sub(shape, D)
    src = _sample_sources(shape, 40, 96)
    got, m, ks, _ = _gpu_run(shape, D, lam, w.R, w.n_sub, c0, 1, prec, src)
    ref, _ = oracle.kernels(shape, D, lam, w.R, w.n_sub, src)
    err = np.linalg.norm((ks - ref).reshape(len(src), -1), axis=1) / np.linalg.norm(ref.reshape(len(src), -1), axis=1)
    assert err.max() <= KERNEL_TOL[prec]
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()
    N = w.n ** 3
    centre = (w.n // 2) * (1 + w.n + w.n * w.n)
    dests = np.array([0, N - 1, centre, centre + 7, centre - 5 * w.n])
    ref_at = _oracle_at(shape, D, lam, w.R, w.n_sub, c0, dests)
    assert np.max(np.abs(got[dests] - ref_at)) <= FIELD_TOL[prec] * np.abs(ref_at).max()


def test_workload_256_sampled():
    """256^3 with the 192^3 recipe (the surrogate comparison's second size), BF16 storage: sampled kernels
    and destinations against the oracle, mass budget."""
    w = synth.WORKLOADS["fdirw-256c-r8"]
    _, D, c0 = w.make()
    shape = (w.n,) * 3
    lam = oracle.stable_dt_sub(shape, D)
    src = _sample_sources(shape, 16, 256)
    got, m, ks, info = _gpu_run(shape, D, lam, w.R, w.n_sub, c0, 1, "bf16", src)
    ref, _ = oracle.kernels(shape, D, lam, w.R, w.n_sub, src)
    err = np.linalg.norm((ks - ref).reshape(len(src), -1), axis=1) / np.linalg.norm(ref.reshape(len(src), -1), axis=1)
    assert err.max() <= KERNEL_TOL["bf16"]
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()
    N = w.n ** 3
    dests = np.array([7, N - 8, (w.n // 2) * (1 + w.n + w.n * w.n)])
    ref_at = _oracle_at(shape, D, lam, w.R, w.n_sub, c0, dests)
    assert np.max(np.abs(got[dests] - ref_at)) <= FIELD_TOL["bf16"] * np.abs(ref_at).max()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_workload_192_sampled(prec):
    """192^3, porosity 0.4, D 1/1e-6, R=8, n_sub=200, c=1 in solid: the benchmark's launch configuration."""
    w = synth.WORKLOADS["fdirw-192c-r8"]
    _, D, c0 = w.make()
    shape = (w.n,) * 3
    lam = oracle.stable_dt_sub(shape, D)
    src = _sample_sources(shape, 24, 192)
    got, m, ks, info = _gpu_run(shape, D, lam, w.R, w.n_sub, c0, 1, prec, src)
    assert info["kernels_ms"] > 0
    ref, _ = oracle.kernels(shape, D, lam, w.R, w.n_sub, src)
    err = np.linalg.norm((ks - ref).reshape(len(src), -1), axis=1) / np.linalg.norm(ref.reshape(len(src), -1), axis=1)
    assert err.max() <= KERNEL_TOL[prec]
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()
    N = w.n ** 3
    dests = np.array([0, N - 1, (w.n // 2) * (1 + w.n + w.n * w.n)])
    ref_at = _oracle_at(shape, D, lam, w.R, w.n_sub, c0, dests)
    assert np.max(np.abs(got[dests] - ref_at)) <= FIELD_TOL[prec] * np.abs(ref_at).max()


# ------------------------------------------------------------------------- streamed cache (z-slabs)

@pytest.mark.parametrize("prec,accum", [("fp32", "ff"), ("bf16", "fp32"), ("fp64", "ff"), ("fp16", "ff")])
@pytest.mark.parametrize("n_steps", [1, 2, 3])
def test_streamed_cache_equals_resident_bitwise(prec, accum, n_steps):
    """A mem_limit that leaves room for about a third of the cache makes the context stream it by
    z-slabs (every step re-marches each slab's sources): fields, masses and the in-place call equal the
    resident cache's bit for bit, and the streamed context reports its slabs and no resident kernels."""
    shape, R, n_sub = (24, 16, 21), 4, 30
    D = _case(shape, 160, "per_sphere")
    lam = oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    c0 = synth.random_field(N, 161)
    Dd = torch.from_numpy(D).to(DEV)
    with FDiRW(shape, Dd, n_sub * lam, R, n_sub, prec, accum=accum) as f:
        f.kernels()
        info = f.info()
        cin = torch.from_numpy(c0).to(DEV)
        ref = torch.empty_like(cin)
        m_ref = f.step(cin, ref, n_steps, want_mass=True)
    limit = info["device_bytes"] - info["cache_bytes"] + info["cache_bytes"] // 3 + 8 * N
    with FDiRW(shape, Dd, n_sub * lam, R, n_sub, prec, mem_limit=limit, accum=accum) as f:
        out = torch.empty_like(cin)
        m = f.step(cin, out, n_steps, want_mass=True)
        sinfo = f.info()
        with pytest.raises(FdirwError) as e:
            f.read_kernels([0])
        assert e.value.code == fdirw.FDIRW_ERR_STATE
        inplace = cin.clone()
        f.step(inplace, inplace, n_steps)
        host = np.empty_like(c0)
        f.step(c0, host, n_steps)
    assert sinfo["n_chunks"] >= 3 and sinfo["cache_bytes"] < info["cache_bytes"]
    assert torch.equal(out, ref) and torch.equal(inplace, ref) and m == m_ref
    assert np.array_equal(host, ref.cpu().numpy())
