"""GPU parity of the convection path (fdirw_set_velocity; Sec. 5, a steady flow folded into the spreading
kernels with the superposition unchanged) against the FP64 oracle's upwind march: kernels element by
element, macro steps, the no-flow limit bit for bit, exact Courant-1 shifts, the largest radii, and the
argument and stability errors."""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_11376_gb300 import FDiRW, FdirwError, fdirw, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KERNEL_TOL = {"fp32": 1e-5, "bf16": 8e-3}      # per-kernel relative L2, as the diffusion-only path
FIELD_TOL = {"fp32": 1e-5, "bf16": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(shape, seed, amp=0.5, mean=(0.3, -0.2, 0.1)):
    p = synth.sphere_packing(shape, 0.45, seed, r_range=(1.5, 3.5))
    D = synth.diffusivity_two_phase(p, 1.0, 1e-3)
    w = synth.face_velocity(shape, seed + 1, mean, amp, p.solid)
    return D, w


def _oracle_kernels(shape, D, w, lam, R, n_sub, sources):
    return np.stack([oracle.source_kernel_adv(shape, D, w, lam, lam, R, n_sub, int(s))[0] for s in sources])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("shape,R,n_sub,every", [((20, 18, 16), 3, 40, 1), ((21, 19, 18), 8, 60, 5)])
def test_flow_kernels_match_oracle(prec, shape, R, n_sub, every):
    D, w = _case(shape, 120)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    N = int(np.prod(shape))
    src = np.arange(0, N, every)
    with FDiRW(shape, torch.from_numpy(D).to(DEV), n_sub * lam, R, n_sub, prec) as f:
        f.set_velocity(torch.from_numpy(w.reshape(-1)).to(DEV))
        f.kernels()
        ks = f.read_kernels(src).reshape(len(src), -1)
        assert f.info()["march_parts"] == 5
    ref = _oracle_kernels(shape, D, w, lam, R, n_sub, src).reshape(len(src), -1)
    err = np.linalg.norm(ks - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= KERNEL_TOL[prec], err.max()
    assert np.max(np.abs(ks.sum(axis=1) - 1.0)) <= 1e-12 and ks.min() >= 0.0


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_flow_steps_match_oracle(prec):
    shape, R, n_sub = (19, 17, 16), 4, 30
    D, w = _case(shape, 122, amp=0.8)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 123, 0.0, 2.0)
    ref = oracle.superpose_adv(shape, D, w, lam, lam, R, n_sub, oracle.superpose_adv(shape, D, w, lam, lam, R, n_sub, c0))
    with FDiRW(shape, D, n_sub * lam, R, n_sub, prec) as f:
        f.set_velocity(w)                               # host velocity
        cin = torch.from_numpy(c0).to(DEV)
        cout = torch.empty_like(cin)
        m = f.step(cin, cout, 2, want_mass=True)
        host = np.empty_like(c0)
        f.step(c0, host, 2)                             # host field, same result
    got = cout.cpu().numpy()
    assert np.array_equal(got, host)
    assert _rel(got, ref) <= FIELD_TOL[prec], _rel(got, ref)
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()       # upwind fluxes conserve mass within closed windows


@pytest.mark.parametrize("R", [3, 8, 9, 10])
def test_no_flow_is_bitwise_the_diffusion_path(R):
    """w = 0 gives the diffusion-only coefficients bit for bit, and mapping 5 with direction-dependent
    faces makes the same FP32 operations as every diffusion mapping: same kernels, same steps."""
    shape = (22, 21, 20)
    D = synth.random_diffusivity(shape, 124, 3.0)
    lam = oracle.stable_dt_sub(shape, D)
    N = D.size
    c0 = synth.random_field(N, 125)
    src = np.arange(3, N, 37)
    out = []
    for flow in (False, True):
        with FDiRW(shape, D, 25 * lam, R, 25, "fp32") as f:
            if flow:
                f.set_velocity(np.zeros(3 * N))
            c = np.empty_like(c0)
            f.step(c0, c, 2)
            out.append((c, f.read_kernels(src)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_courant_one_is_an_exact_shift(sign):
    """D = 0, w = +-1, lam_a = 1: each substep moves every value one cell (the FP32 march is exact on 0/1,
    so the kernel is bit for bit the one-hot shift), and the closed window and domain edges hold what
    reaches them; the step agrees with the oracle to the float-float gather's rounding."""
    shape, R, n_sub = (16, 3, 2), 5, 3
    N = 96
    D = np.zeros(N)
    w = synth.face_velocity(shape, 0, (sign, 0.0, 0.0))
    c0 = synth.random_field(N, 126)
    with FDiRW(shape, D, float(n_sub), R, n_sub, "fp32") as f:
        f.set_velocity(w)
        c = np.empty_like(c0)
        f.step(c0, c, 1)
        ks = f.read_kernels([7])
    ref = oracle.superpose_adv(shape, D, w, 1.0, 1.0, R, n_sub, c0)
    assert np.all(np.abs(c - ref) <= 1e-13 * np.abs(ref))
    assert np.count_nonzero(ref == 0.0) == 3 * 3 * 2    # the three planes the flow leaves empty
    want = np.zeros((11, 11, 11))
    want[5, 5, 5 + int(sign) * 3] = 1.0
    assert np.array_equal(ks[0], want)


def test_velocity_replaced_and_errors():
    shape = (12, 11, 10)
    N = 1320
    D = synth.random_diffusivity(shape, 127, 2.0)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    w1 = synth.face_velocity(shape, 128, (0.2, 0.0, 0.0), 0.2)
    w2 = synth.face_velocity(shape, 129, (0.0, -0.3, 0.0), 0.2)
    c0 = synth.random_field(N, 130)
    ref = oracle.superpose_adv(shape, D, w2, lam, lam, 3, 20, c0)
    with FDiRW(shape, D, 20 * lam, 3, 20) as f:
        f.set_velocity(w1)
        c = np.empty_like(c0)
        f.step(c0, c, 1)
        f.set_velocity(w2)                               # replaces w1; kernels recomputed on the next step
        with pytest.raises(FdirwError):
            f.read_kernels([0])                          # the cache of w1 is gone
        f.step(c0, c, 1)
        assert _rel(c, ref) <= FIELD_TOL["fp32"]
        with pytest.raises(FdirwError) as e:
            f.set_velocity(np.full(3 * N, 1e3))          # outflow sum far above 1
        assert e.value.code == fdirw.FDIRW_ERR_UNSTABLE
        c2 = np.empty_like(c0)
        f.step(c0, c2, 1)                                # w2 still in place
        assert np.array_equal(c, c2)
        bad = w2.reshape(-1).copy()
        bad[17] = np.nan
        with pytest.raises(FdirwError) as e:
            f.set_velocity(bad)
        assert e.value.code == fdirw.FDIRW_ERR_ARG
        f.step(c0, c2, 1)                                # w2 still in place
        assert np.array_equal(c, c2)
        with pytest.raises(ValueError):
            f.set_velocity(np.zeros(N))
    with FDiRW(shape, D, 20 * lam, 3, 20, "fp64") as f:
        with pytest.raises(FdirwError):
            f.set_velocity(w1)


def test_flow_kernels_at_the_benchmark_size():
    """192^3 two-phase packing, R = 8, n_sub = 220 and the bench's flow (mean 0.03 along +x, noise 0.03,
    zero on solid faces): sampled kernels (corner, face, centre, random) against the oracle's upwind march."""
    w = synth.WORKLOADS["fdirw-192c-r8"]
    packing, D, _ = w.make()
    shape = (w.n,) * 3
    lam = oracle.stable_dt_sub(shape, D)
    n_sub = -(-11 * w.n_sub // 10)
    dt = w.n_sub * lam                                   # the workload's macro step, split into n_sub substeps
    vel = synth.face_velocity(shape, w.seed + 40, (0.03, 0.0, 0.0), 0.03, packing.solid)
    N = w.n ** 3
    rng = np.random.default_rng(162)
    src = np.concatenate([[0, N - 1, (w.n // 2) * (1 + w.n + w.n * w.n), 7 + w.n * 3], rng.integers(0, N, 4)])
    with FDiRW(shape, torch.from_numpy(D).to(DEV), dt, w.R, n_sub, "bf16") as f:
        f.set_velocity(torch.from_numpy(vel.reshape(-1)).to(DEV))
        f.kernels()
        ks = f.read_kernels(src).reshape(len(src), -1)
    lam_sub = dt / n_sub
    ref = _oracle_kernels(shape, D, vel, lam_sub, w.R, n_sub, src).reshape(len(src), -1)
    err = np.linalg.norm(ks - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= KERNEL_TOL["bf16"], err.max()
