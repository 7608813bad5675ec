"""Pins of the surrogate's CPU oracle (no GPU): library correlation, finite differences, torch BF16."""
import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

from oracle import surrogate as so
from paper_2408_11376_gb300 import synth


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    # exact ties between two BF16 values (low 16 bits 0x8000), with an even and an odd upper half
    ties = np.array([0x3F808000, 0x3F818000, 0xBF808000, 0xBF818000, 0x00018000], dtype=np.uint32).view(np.float32)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-30, 100), [0.0, -0.0, 1.0, 65504.0, 3e38],
                        ties.astype(np.float64)])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(so.bf16_round(x), ref)


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(so.C, so.P, so.P, so.P))
    W = rng.normal(size=(27, so.C, so.C))
    b = rng.normal(size=so.C)
    z = so.conv3d_same(a, W, b)
    for co in (0, 5, 15):
        ref = np.full((so.P,) * 3, b[co])
        for ci in range(so.C):
            k = np.zeros((3, 3, 3))
            for t in range(27):
                k[t // 9, (t // 3) % 3, t % 3] = W[t, co, ci]      # [dz+1, dy+1, dx+1]
            ref += ndi.correlate(a[ci], k, mode="constant", cval=0.0)
        assert np.allclose(z[co], ref, rtol=0, atol=1e-10)


def _smooth_case(seed):
    rng = np.random.default_rng(seed)
    shape = (21, 19, 18)
    D = synth.random_diffusivity(shape, seed, 6.0)
    feat = so.features(D, shape, 7 + 21 * (9 + 19 * 9))
    Ws, bs = so.init_params(seed)
    Ws = [W + rng.normal(0, 0.02, W.shape) for W in Ws]
    Ws[-1][13, 0, 0] = 3.0
    bs = [b + rng.normal(0, 0.1, b.shape) for b in bs]
    bs[-1][0] = -3.0
    k = rng.random((so.P,) * 3)
    k /= k.sum()
    return feat, Ws, bs, k


def test_backward_matches_finite_differences():
    feat, Ws, bs, k = _smooth_case(2)

    def L(Ws_, bs_):
        _, _, c = so.forward(feat, Ws_, bs_, emulate_bf16=False)
        return so.loss_grad(c, k)[0]

    _, _, cache = so.forward(feat, Ws, bs, emulate_bf16=False)
    _, dz = so.loss_grad(cache, k)
    dWs, dbs = so.backward(Ws, cache, dz, emulate_bf16=False)
    rng = np.random.default_rng(3)
    h = 1e-6
    rel = []
    for l in range(so.LAYERS):
        co_max = 1 if l == so.LAYERS - 1 else so.C
        for _ in range(6):
            t, co, ci = rng.integers(27), rng.integers(co_max), rng.integers(so.C)
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][t, co, ci] += h
            Wm[l][t, co, ci] -= h
            fd = (L(Wp, bs) - L(Wm, bs)) / (2 * h)
            rel.append(abs(dWs[l][t, co, ci] - fd) / max(1.0, abs(fd)))
        co = rng.integers(co_max)
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][co] += h
        bm[l][co] -= h
        fd = (L(Ws, bp) - L(Ws, bm)) / (2 * h)
        rel.append(abs(dbs[l][co] - fd) / max(1.0, abs(fd)))
    # A relu kink inside the +-h step can spoil one entry; a wrong term or index spoils all of them.
    assert np.median(rel) <= 1e-6 and max(rel) <= 1e-2, rel


def test_features_and_gate():
    shape = (10, 9, 8)
    D = np.ones(720)
    D[0] = 1e-8
    D[1] = 0.0
    f = so.features(D, shape, 0)                  # corner source: most of the patch is outside
    assert f[2, 8, 8, 8] == 1.0 and f[2].sum() == 1.0
    assert f[1].sum() == 9 * 9 * 8                # in-domain cells of the clipped patch (x, y, z)
    assert f[0, 8, 8, 8] == 0.0 and f[0, 8, 8, 9] == -0.5 and f[0, 8, 8, 10] == 1.0
    assert so.gate(1.0009) and not so.gate(1.0011) and not so.gate(0.998)


def test_delta_prior_forward_closed_form():
    """With no noise the prior carries the source marker through the relu layers unchanged (centre taps
    1), and layer 4 gives z = bf16(L) a0 - fp32(L), L = -ln(eps): in closed form the head is
    exp(bf16(L) - fp32(L)) at the source, exp(-fp32(L)) on the other in-domain cells and 0 outside the
    domain.  An edge source puts part of the patch outside."""
    shape = (12, 11, 10)
    s = 0 + 12 * (5 + 11 * 9)                    # x = 0, y = 5, z = 9: patch outside in -x and +z
    feat = so.features(np.ones(12 * 11 * 10), shape, s)
    Ws, bs = so.init_params(0, noise=0.0)
    y, m, _ = so.forward(feat, Ws, bs)
    L = -np.log(so.EPS)
    Lb = float(so.bf16_round(np.array([L]))[0])
    Lf = float(np.float32(L))
    inside = feat[1] > 0.5
    want = np.where(inside, np.exp(-Lf), 0.0)
    want[so.HALF, so.HALF, so.HALF] = np.exp(Lb - Lf)
    assert np.allclose(y, want, rtol=1e-14, atol=0)
    assert inside.sum() == 9 * 11 * 9               # x in [0, 8], y in [0, 10], z in [1, 9]
    assert m == pytest.approx(np.exp(Lb - Lf) + (inside.sum() - 1) * np.exp(-Lf), rel=1e-14)
