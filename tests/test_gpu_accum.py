"""GPU parity of the FP32-accumulation superposition (fdirw_opts.accum = FDIRW_ACCUM_FP32; Sec. 3.3's
low-precision products summed in FP32) against the FP64 oracle: fields after several macro steps, the
total mass restored every step, the float-float mode beside it, the scalar (ragged nx) path, zero and
mixed-sign fields, determinism, and the 192^3 benchmark configuration on sampled destinations."""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_11376_gb300 import FDiRW, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FIELD_TOL = {"fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(shape, seed):
    p = synth.sphere_packing(shape, 0.4, seed, r_range=(1.5, 3.5))
    return synth.diffusivity_per_sphere(p)


def _run(shape, D, lam, R, n_sub, c0, steps, prec, accum):
    with FDiRW(shape, torch.from_numpy(D).to(DEV), n_sub * lam, R, n_sub, prec, accum=accum) as f:
        cin = torch.from_numpy(np.ascontiguousarray(c0)).to(DEV)
        cout = torch.empty_like(cin)
        m = f.step(cin, cout, steps, want_mass=True)
        assert f.info()["accum"] == (1 if accum == "fp32" else 0)
    return cout.cpu().numpy(), m


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("shape,R,n_sub", [((24, 18, 16), 3, 40), ((16, 17, 18), 8, 60), ((13, 11, 9), 2, 25)])
def test_fp32_accum_steps_match_oracle(prec, shape, R, n_sub):
    """Vector gather (nx a multiple of the vector width) and the scalar one (nx = 13): three macro steps
    within the storage tolerance of the oracle, the total mass equal to the input's to FP64 rounding."""
    D = _case(shape, 150 + R)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 151, 0.0, 2.0)
    ref = c0
    for _ in range(3):
        ref = oracle.superpose(shape, D, lam, R, n_sub, ref)
    got, m = _run(shape, D, lam, R, n_sub, c0, 3, prec, "fp32")
    assert _rel(got, ref) <= FIELD_TOL[prec], _rel(got, ref)
    assert abs(m - c0.sum()) <= 1e-13 * c0.sum()
    assert abs(got.sum() - c0.sum()) <= 1e-13 * c0.sum()


def test_fp32_accum_close_to_float_float():
    """Same kernels, two accumulations: the FP32 rows stay within a few 1e-7 of the float-float rows."""
    shape, R, n_sub = (32, 24, 20), 4, 50
    D = _case(shape, 152)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 153)
    a, ma = _run(shape, D, lam, R, n_sub, c0, 5, "fp32", "fp32")
    b, mb = _run(shape, D, lam, R, n_sub, c0, 5, "fp32", "ff")
    assert _rel(a, b) <= 1e-6, _rel(a, b)
    assert abs(ma - mb) <= 1e-13 * mb


def test_fp32_accum_zero_and_mixed_sign_fields():
    """A zero field stays exactly zero (no restoration factor from 0/0); a field whose positive and
    negative parts nearly cancel keeps its total to FP64 rounding of sum |c| without amplifying errors."""
    shape, R, n_sub = (16, 16, 16), 3, 30
    D = _case(shape, 154)
    lam = oracle.stable_dt_sub(shape, D)
    z, _ = _run(shape, D, lam, R, n_sub, np.zeros(D.size), 2, "bf16", "fp32")
    assert not z.any()
    c0 = synth.random_field(D.size, 155, -1.0, 1.0)
    c0 -= c0.mean()
    a, _ = _run(shape, D, lam, R, n_sub, c0, 2, "fp32", "fp32")
    b, _ = _run(shape, D, lam, R, n_sub, c0, 2, "fp32", "ff")
    assert abs(a.sum() - c0.sum()) <= 1e-13 * np.abs(c0).sum()
    assert np.max(np.abs(a - b)) <= 1e-6 * np.abs(b).max()


def test_fp32_accum_host_buffers_and_identity_cases():
    """Host fields give the device result bit for bit; n_steps = 0 and R = 0 copy the field unchanged."""
    shape, R, n_sub = (16, 12, 10), 3, 25
    D = _case(shape, 158)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 159)
    with FDiRW(shape, D, n_sub * lam, R, n_sub, "bf16", accum="fp32") as f:
        dev_in = torch.from_numpy(c0).to(DEV)
        dev_out = torch.empty_like(dev_in)
        f.step(dev_in, dev_out, 2)
        host = np.empty_like(c0)
        f.step(c0, host, 2)
        same = np.empty_like(c0)
        f.step(c0, same, 0)
    assert np.array_equal(dev_out.cpu().numpy(), host)
    assert np.array_equal(same, c0)
    with FDiRW(shape, D, n_sub * lam, 0, n_sub, "fp32", accum="fp32") as f:
        out = np.empty_like(c0)
        f.step(c0, out, 3)
    assert np.array_equal(out, c0)


def test_fp32_accum_deterministic():
    shape, R, n_sub = (24, 16, 16), 5, 40
    D = _case(shape, 156)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 157)
    a, ma = _run(shape, D, lam, R, n_sub, c0, 3, "bf16", "fp32")
    b, mb = _run(shape, D, lam, R, n_sub, c0, 3, "bf16", "fp32")
    assert np.array_equal(a, b) and ma == mb


def test_fp32_accum_workload_192_sampled():
    """The benchmark configuration (192^3, R = 8, n_sub = 200, BF16 cache): sampled destinations of one
    macro step against the oracle, and the mass of 20 macro steps."""
    w = synth.WORKLOADS["fdirw-192c-r8"]
    _, D, c0 = w.make()
    shape = (w.n,) * 3
    lam = oracle.stable_dt_sub(shape, D)
    with FDiRW(shape, torch.from_numpy(D).to(DEV), w.n_sub * lam, w.R, w.n_sub, "bf16", accum="fp32") as f:
        cin = torch.from_numpy(c0).to(DEV)
        cout = torch.empty_like(cin)
        f.step(cin, cout, 1)
        got = cout.cpu().numpy()
        m20 = f.step(cin, cout, w.steps, want_mass=True)
    N = w.n ** 3
    dests = np.array([0, N - 1, (w.n // 2) * (1 + w.n + w.n * w.n), 12345, N // 3])
    nx = ny = nz = w.n
    cond = oracle.Conductance(shape, D)
    want = []
    for x in dests:
        xx, xy, xz = x % nx, (x // nx) % ny, x // (nx * ny)
        src, offs = [], []
        for sz in range(max(xz - w.R, 0), min(xz + w.R, nz - 1) + 1):
            for sy in range(max(xy - w.R, 0), min(xy + w.R, ny - 1) + 1):
                for sx in range(max(xx - w.R, 0), min(xx + w.R, nx - 1) + 1):
                    src.append(sx + nx * (sy + ny * sz))
                    offs.append((xz - sz + w.R, xy - sy + w.R, xx - sx + w.R))
        ks, _ = oracle.kernels(shape, D, lam, w.R, w.n_sub, src, cond)
        want.append(sum(c0[s] * ks[q][o] for q, (s, o) in enumerate(zip(src, offs))))
    want = np.array(want)
    assert np.max(np.abs(got[dests] - want)) <= FIELD_TOL["bf16"] * np.abs(want).max()
    assert abs(m20 - c0.sum()) <= 1e-13 * c0.sum()
