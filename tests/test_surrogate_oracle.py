"""Pins of the surrogate's CPU oracle (no GPU): library correlation, float64 autograd through torch's conv3d,
finite differences, torch BF16."""
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


def _torch_weight(W):
    """[27 taps][co][ci] (tap = (dx+1) + 3(dy+1) + 9(dz+1)) -> torch's conv3d layout [co][ci][dz+1][dy+1][dx+1]."""
    return torch.tensor(np.ascontiguousarray(np.asarray(W).reshape(3, 3, 3, so.C, so.C).transpose(3, 4, 0, 1, 2)),
                        dtype=torch.float64)


def _autograd(feat, Ws, bs, k):
    """The same four-layer network and loss written with torch's float64 conv3d and differentiated by
    autograd, independent of the oracle's hand-derived backward: returns (loss, dWs [27][co][ci], dbs)."""
    Wt = [_torch_weight(W).requires_grad_(True) for W in Ws]
    bt = [torch.tensor(np.asarray(b, dtype=np.float64), requires_grad=True) for b in bs]
    h = torch.tensor(feat[None], dtype=torch.float64)
    for l in range(so.LAYERS):
        z = torch.nn.functional.conv3d(h, Wt[l], bt[l], padding=1)
        h = torch.relu(z) if l + 1 < so.LAYERS else z
    mask = torch.tensor(feat[1] > 0.5)
    kk = torch.tensor(np.asarray(k, dtype=np.float64))
    z = h[0, 0]
    klnk = torch.where(kk > 0, kk * torch.log(torch.where(kk > 0, kk, torch.ones_like(kk))), torch.zeros_like(kk))
    loss = torch.where(mask, torch.exp(z) - kk * z + klnk - kk, torch.zeros_like(kk)).sum()
    loss.backward()
    dWs = [W.grad.numpy().transpose(2, 3, 4, 0, 1).reshape(27, so.C, so.C) for W in Wt]
    return float(loss.item()), dWs, [b.grad.numpy() for b in bt]


def _edge_case(seed):
    """A corner-adjacent source on a rough D: the patch runs off the domain on three sides, so the head
    mask, the zero padding and every edge tap take part."""
    feat, Ws, bs, k = _smooth_case(seed)
    shape = (21, 19, 18)
    D = synth.random_diffusivity(shape, seed + 50, 6.0)
    return so.features(D, shape, 2 + 21 * (17 + 19 * 1)), Ws, bs, k


@pytest.mark.parametrize("case", [_smooth_case, _edge_case])
def test_backward_matches_float64_autograd(case):
    """Every weight and bias gradient of the oracle's hand-derived backward equals float64 autograd through
    torch's conv3d on every entry: relative error <= 1e-12, measured against the entry itself or, for
    entries smaller than 1e-3 of their layer's largest, against that thousandth (FP64 sums in two
    different orders cancel differently there)."""
    feat, Ws, bs, k = case(2)
    _, _, cache = so.forward(feat, Ws, bs, emulate_bf16=False)
    loss, dz = so.loss_grad(cache, k)
    dWs, dbs = so.backward(Ws, cache, dz, emulate_bf16=False)
    ref_loss, ref_W, ref_b = _autograd(feat, Ws, bs, k)
    assert abs(loss - ref_loss) <= 1e-13 * ref_loss
    for l in range(so.LAYERS):
        for got, ref in ((dWs[l], ref_W[l]), (dbs[l], ref_b[l])):
            floor = 1e-3 * np.abs(ref).max()
            assert floor > 0.0
            assert np.all(np.abs(got - ref) <= 1e-12 * np.maximum(np.abs(ref), floor)), (l, np.abs(got - ref).max())


def test_forward_bf16_matches_torch_chain():
    """The BF16-emulating forward rounds exactly where the GPU does (features, weights and every relu
    output, not the head): the same chain in torch float64 with torch's own BF16 cast at those points."""
    feat, Ws, bs, _ = _edge_case(4)
    r = lambda t: t.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    h = r(torch.tensor(feat[None], dtype=torch.float64))
    for l in range(so.LAYERS):
        z = torch.nn.functional.conv3d(h, r(_torch_weight(Ws[l])), torch.tensor(bs[l], dtype=torch.float64), padding=1)
        h = r(torch.relu(z)) if l + 1 < so.LAYERS else z
    y, m, (acts, zs, mask) = so.forward(feat, Ws, bs)
    ref = h[0, 0].numpy()
    assert np.allclose(zs[-1][0], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    want = np.where(mask, np.exp(ref), 0.0)
    assert np.allclose(y, want, rtol=1e-11, atol=0) and m == pytest.approx(want.sum(), rel=1e-11)


def test_backward_matches_finite_differences():
    """Central differences of the forward pass (a smoke check beside the exact autograd pin): every sampled
    weight and bias whose +-h step leaves every relu on the same side agrees to 1e-6; a step that crosses
    a relu kink (where no derivative exists) is redrawn."""
    feat, Ws, bs, k = _smooth_case(2)

    def L(Ws_, bs_):
        _, _, c = so.forward(feat, Ws_, bs_, emulate_bf16=False)
        return so.loss_grad(c, k)[0], [z > 0.0 for z in c[1][:-1]]

    _, _, cache = so.forward(feat, Ws, bs, emulate_bf16=False)
    _, dz = so.loss_grad(cache, k)
    dWs, dbs = so.backward(Ws, cache, dz, emulate_bf16=False)
    rng = np.random.default_rng(3)
    h = 1e-6
    rel, redrawn = [], 0

    def fd(Wp, bp, Wm, bm):
        lp, mp = L(Wp, bp)
        lm, mm = L(Wm, bm)
        if any(not np.array_equal(a, b) for a, b in zip(mp, mm)):
            return None
        return (lp - lm) / (2 * h)

    for l in range(so.LAYERS):
        co_max = 1 if l == so.LAYERS - 1 else so.C
        done = 0
        while done < 6:
            t, co, ci = rng.integers(27), rng.integers(co_max), rng.integers(so.C)
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][t, co, ci] += h
            Wm[l][t, co, ci] -= h
            g = fd(Wp, bs, Wm, bs)
            if g is None:
                redrawn += 1
                continue
            rel.append(abs(dWs[l][t, co, ci] - g) / max(1.0, abs(g)))
            done += 1
        co = rng.integers(co_max)
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][co] += h
        bm[l][co] -= h
        g = fd(Ws, bp, Ws, bm)
        if g is not None:
            rel.append(abs(dbs[l][co] - g) / max(1.0, abs(g)))
    assert redrawn <= 8 and len(rel) >= 24
    assert max(rel) <= 1e-6, rel


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


def test_offset_channels():
    """Channels 3-6 encode each voxel's offset o from the source: channel 3 grows by exactly 1/8 per cell
    along x and not at all along y or z (4 along y, 5 along z), all three vanish at the source and are odd
    about it, channel 6 equals (c3^2 + c4^2 + c5^2) / 4 = |o|^2 / 256, every value is a BF16 number, and none
    depends on the domain or on where the source sits in it."""
    shape = (10, 9, 8)
    D = np.ones(720)
    corner = so.features(D, shape, 0)
    inner = so.features(synth.random_diffusivity(shape, 3, 6.0), shape, 4 + 10 * (4 + 9 * 4))
    assert np.array_equal(corner[3:7], inner[3:7])
    f = inner
    for ch, axis in ((3, 3), (4, 2), (5, 1)):              # f is [channel, z, y, x]
        d = np.diff(f[ch], axis=axis - 1)
        assert np.all(d == 0.125), ch
        for other in {1, 2, 3} - {axis}:
            assert np.all(np.diff(f[ch], axis=other - 1) == 0.0), (ch, other)
        assert f[ch, 8, 8, 8] == 0.0
        assert np.array_equal(f[ch], -np.flip(f[ch], axis=axis - 1))
    assert np.array_equal(f[6], (f[3] ** 2 + f[4] ** 2 + f[5] ** 2) / 4.0)
    assert f[6].max() == 192.0 / 256.0 and f[6, 8, 8, 8] == 0.0
    assert np.array_equal(so.bf16_round(f), f)
    assert not f[7:].any()


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
