"""GPU parity of the learned surrogate (tensor-core convolutions) against its CPU oracle, and the gate with
FD fallback inside the kernel-cache build."""
import numpy as np
import pytest
import torch

import oracle
from oracle import surrogate as so
from paper_2408_11376_gb300 import FDiRW, Net, fdirw, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()


def _domain(shape, seed, kind="per_sphere"):
    p = synth.sphere_packing(shape, 0.4, seed, r_range=(1.5, 3.5))
    return synth.diffusivity_per_sphere(p) if kind == "per_sphere" else synth.diffusivity_two_phase(p, 1.0, 1e-6)


def _random_params(seed):
    Ws, bs = so.init_params(seed, noise=0.05)
    rng = np.random.default_rng(seed + 100)
    bs = [b + rng.normal(0, 0.05, b.shape) for b in bs]
    Ws[-1][13, 0, 0] = 4.0                      # moderate head so that y spans a few decades
    bs[-1][1:] = 0.0
    bs[-1][0] = -4.0
    return Ws, bs


# Tolerances of the element-by-element checks, derived from the arithmetic.  Each convolution output is a
# sum of K = 27 x 16 = 432 exact BF16 x BF16 products (and the FP32 bias) accumulated in FP32 on the tensor
# cores.  The accumulation is bounded by the standard recursive-summation bound gamma_K * S, S the sum of
# the absolute terms, with the unit taken as 2^-23 (twice FP32's rounding unit, which also covers a
# truncating accumulator).  A BF16 output is then rounded to nearest, so GPU and reference may land on
# neighbouring BF16 values: one BF16 ulp, at most 2^-7 of the value.  The reference layer is applied to the
# GPU's own input of that layer, so errors do not compound from layer to layer.
U_ACC = 2.0 ** -23
ULP_BF16 = 2.0 ** -7


def _gamma(k):
    return k * U_ACC / (1.0 - k * U_ACC)


def _bits(u16):
    return (np.asarray(u16, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def _layer_check(got, ref, S, K, bf16_out, what, max_mismatch=0.05):
    d = _gamma(K) * S
    tol = d + (ULP_BF16 * (np.abs(ref) + d) if bf16_out else 2.0 ** -24 * np.abs(ref))
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (what, int(bad.sum()), float(np.abs(got - ref)[bad].max()))
    if bf16_out:
        frac = float(np.mean(got != ref))
        assert frac <= max_mismatch, (what, frac)


def _edge_sources(shape, n, seed):
    """Corners, edge midpoints and face centres of the grid, then random cells: n sources in all."""
    nx, ny, nz = shape
    cells = set()
    for x in (0, nx // 2, nx - 1):
        for y in (0, ny // 2, ny - 1):
            for z in (0, nz // 2, nz - 1):
                cells.add(x + nx * (y + ny * z))
    rng = np.random.default_rng(seed)
    while len(cells) < n:
        cells.add(int(rng.integers(0, nx * ny * nz)))
    return np.array(sorted(cells))[:n]


def _b32(b):
    return np.asarray(b, dtype=np.float32).astype(np.float64)


def test_forward_layers_match_oracle_element_by_element():
    """64 sources (the 27 corner, edge-midpoint and face-centre cells and random ones): the features bit
    for bit, every layer's BF16 output and the head's pre-exponential z against the oracle's layer applied
    to the GPU's input of that layer, within the bounds above; the predicted kernels are exp(z)."""
    shape = (24, 22, 20)
    D = _domain(shape, 5)
    Ws, bs = _random_params(1)
    src = _edge_sources(shape, 64, 3)
    with FDiRW(shape, D, 0.1, 8, 1, "fp32") as f:            # march settings unused here
        net = Net(fdirw.pack_params(Ws, bs))
        acts, z, _, _, _ = net.trace(f.ctx, src)
        k, m, _ = net.predict(f.ctx, src)
        net.close()
    Wb = [so.bf16_round(W) for W in Ws]
    Wa = [np.abs(W) for W in Wb]
    for q, s in enumerate(src):
        a = [_bits(acts[l, q]).reshape(16, 17, 17, 17) for l in range(4)]
        assert np.array_equal(a[0], so.features(D, shape, int(s))), q
        for l in range(3):
            ref = so.bf16_round(np.maximum(so.conv3d_same(a[l], Wb[l], _b32(bs[l])), 0.0))
            S = so.conv3d_same(np.abs(a[l]), Wa[l], np.abs(_b32(bs[l])))
            _layer_check(a[l + 1], ref, S, 27 * 16 + 1, True, ("layer", l, q))
        zr = so.conv3d_same(a[3], Wb[3], _b32(bs[3]))[0]
        S = so.conv3d_same(np.abs(a[3]), Wa[3], np.abs(_b32(bs[3])))[0]
        _layer_check(z[q].astype(np.float64).reshape(17, 17, 17), zr, S, 27 * 16 + 1, False, ("head", q))
        inside = a[0][1] > 0.5
        y = np.where(inside, np.exp(z[q].astype(np.float64).reshape(17, 17, 17)), 0.0)
        assert np.allclose(k[q], y, rtol=2.0 ** -21, atol=0), q
        assert abs(m[q] - k[q].sum()) <= 1e-12 * m[q]


def test_backward_layers_match_oracle_element_by_element():
    """The same 64 sources with random targets: the head gradient, every layer's BF16 input gradient
    (masked by the relu) against the oracle's transposed convolution of the GPU's gradient of the layer
    above, and every weight and bias gradient against the oracle's FP64 sums of the GPU's activations and
    gradients, each within its accumulation bound; the loss to FP64 rounding."""
    shape = (24, 22, 20)
    D = _domain(shape, 6)
    Ws, bs = _random_params(2)
    src = _edge_sources(shape, 64, 4)
    n = len(src)
    rng = np.random.default_rng(7)
    tg = rng.random((n, 17, 17, 17)) * 1e-3
    with FDiRW(shape, D, 0.1, 8, 1, "fp32") as f:
        net = Net(fdirw.pack_params(Ws, bs))
        acts, z, grads, pg, loss = net.trace(f.ctx, src, tg)
        g2, loss2 = net.gradients(f.ctx, src, tg)
        net.close()
    assert np.array_equal(pg, g2) and loss == loss2           # the traced pass is the training pass
    Wb = [so.bf16_round(W) for W in Ws]
    dW = [np.zeros((27, 16, 16)) for _ in range(4)]
    SW = [np.zeros((27, 16, 16)) for _ in range(4)]
    db = [np.zeros(16) for _ in range(4)]
    Sb = [np.zeros(16) for _ in range(4)]
    lo = 0.0
    for q in range(n):
        a = [_bits(acts[l, q]).reshape(16, 17, 17, 17) for l in range(4)]
        g = [_bits(grads[l, q]).reshape(16, 17, 17, 17) for l in range(4)]
        zq = z[q].astype(np.float64).reshape(17, 17, 17)
        inside = a[0][1] > 0.5
        kq = tg[q]
        yq = np.exp(zq)
        lo += float(np.where(inside, yq - kq * zq + kq * np.log(kq) - kq, 0.0).sum())
        head = np.zeros((16, 17, 17, 17))
        head[0] = so.bf16_round(np.where(inside, yq - kq, 0.0))
        _layer_check(g[3], head, np.zeros_like(head), 0, True, ("head gradient", q), max_mismatch=1e-3)
        for l in (2, 1, 0):
            ref = so.bf16_round(so.conv3d_same_grad_input(g[l + 1], Wb[l + 1]) * (a[l + 1] > 0.0))
            S = so.conv3d_same_grad_input(np.abs(g[l + 1]), np.abs(Wb[l + 1]))
            _layer_check(g[l], ref, S, 27 * 16, True, ("input gradient", l, q))
        for l in range(4):
            dW[l] += so.conv3d_same_grad_weight(a[l], g[l])
            SW[l] += so.conv3d_same_grad_weight(np.abs(a[l]), np.abs(g[l]))
            db[l] += g[l].sum(axis=(1, 2, 3))
            Sb[l] += np.abs(g[l]).sum(axis=(1, 2, 3))
    assert abs(loss - lo / n) <= 1e-12 * lo / n
    gW, gb = fdirw.unpack_params(pg)
    # Weight and bias gradients: each of 152 CTAs takes a contiguous range of 32-row units (192 per patch);
    # groups of 8 units (256 rows) accumulate in TMEM, the group sums are added in FP32 registers, and the
    # 152 partials are summed in order: a chain of at most 256 + ceil(units / 8) + 152 additions.
    per = 8 * 32 + -(-(-(-n * 192 // 152)) // 8) + 152
    for l in range(4):
        _layer_check(gW[l], dW[l], SW[l], per, False, ("weight gradient", l))
        _layer_check(gb[l], db[l], Sb[l], per, False, ("bias gradient", l))


def test_bounded_wait_runs_out_and_the_net_recovers():
    """The convolutions' MMA wait is bounded: with the test hook withholding the MMAs (nothing in flight),
    a prediction returns FDIRW_ERR_TIMEOUT after the 2 ms budget, the kernel frees its tensor memory, and
    the next prediction on the same network, hook cleared, returns the same kernels as before."""
    shape = (24, 22, 20)
    D = _domain(shape, 5)
    Ws, bs = _random_params(1)
    src = np.array([0, 10 + 24 * (11 + 22 * 10), 24 * 22 * 20 - 1])
    with FDiRW(shape, D, 0.1, 8, 1, "fp32") as f:
        net = Net(fdirw.pack_params(Ws, bs))
        k0, m0, a0 = net.predict(f.ctx, src)
        net.test_wait(wait_ns=2_000_000, withhold_mma=True)
        with pytest.raises(fdirw.FdirwError) as e:
            net.predict(f.ctx, src)
        assert e.value.code == fdirw.FDIRW_ERR_TIMEOUT
        net.test_wait(0, False)
        k1, m1, a1 = net.predict(f.ctx, src)
        net.close()
    assert np.array_equal(k0, k1) and np.array_equal(m0, m1) and np.array_equal(a0, a1)


def test_bounded_wait_in_training_runs_out_and_the_net_recovers():
    """The same hook on a training pass: the convolutions and the weight-gradient kernel (whose drain warps
    wait for accumulators that never fill, and whose producer waits for stages that are never released)
    all run out of their 2 ms budget with nothing in flight, the call returns FDIRW_ERR_TIMEOUT, and the
    next pass on the same network, hook cleared, returns the gradients and loss of a fresh network."""
    shape = (24, 22, 20)
    D = _domain(shape, 6)
    Ws, bs = _random_params(2)
    src = _edge_sources(shape, 64, 4)
    tg = np.random.default_rng(7).random((len(src), 17, 17, 17)) * 1e-3
    with FDiRW(shape, D, 0.1, 8, 1, "fp32") as f:
        ref = Net(fdirw.pack_params(Ws, bs))
        g0, l0 = ref.gradients(f.ctx, src, tg)
        ref.close()
        net = Net(fdirw.pack_params(Ws, bs))
        net.test_wait(wait_ns=2_000_000, withhold_mma=True)
        with pytest.raises(fdirw.FdirwError) as e:
            net.gradients(f.ctx, src, tg)
        assert e.value.code == fdirw.FDIRW_ERR_TIMEOUT
        net.test_wait(0, False)
        g1, l1 = net.gradients(f.ctx, src, tg)
        net.close()
    assert np.array_equal(g0, g1) and l0 == l1


def _gate_params():
    """Hand-set weights: a source-marker path gives z = 0 at the source cell (y = 1) and z = -30
    elsewhere, and a log-D path adds 0.5 at pore sources (f0 = 1 -> relu(f0 - 0.5) = 0.5): solid sources
    predict a delta (accepted), pore sources predict e^0.5 at the centre (rejected)."""
    Ws = [np.zeros((27, 16, 16)) for _ in range(4)]
    bs = [np.zeros(16) for _ in range(4)]
    c = 13                                      # centre tap
    Ws[0][c, 0, 2] = 1.0                        # ch0 <- source marker
    Ws[0][c, 1, 0] = 1.0                        # ch1 <- f0 - 0.5
    bs[0][1] = -0.5
    for l in (1, 2):
        Ws[l][c, 0, 0] = 1.0
        Ws[l][c, 1, 1] = 1.0
    Ws[3][c, 0, 0] = 30.0
    Ws[3][c, 0, 1] = 1.0
    bs[3][0] = -30.0
    return Ws, bs


def test_kernel_cache_with_gate_and_fd_fallback():
    shape = (24, 20, 16)
    D = _domain(shape, 9, "two_phase")
    N = int(np.prod(shape))
    lam = oracle.stable_dt_sub(shape, D)
    Ws, bs = _gate_params()
    net = Net(fdirw.pack_params(Ws, bs))
    src = np.arange(N)
    with FDiRW(shape, D, 60 * lam, 8, 60, "fp32") as fd, FDiRW(shape, D, 60 * lam, 8, 60, "fp32") as sg:
        fd.kernels()
        kfd = fd.read_kernels(src)
        accepted = net.build_kernels(sg.ctx)
        ksg = sg.read_kernels(src)
        _, m, acc = net.predict(sg.ctx, src[:1024])
    net.close()
    solid = D < 0.5
    assert accepted == int(solid.sum())
    assert np.array_equal(acc, solid[:1024])
    # rejected (pore) sources come from the FD march, bit for bit
    assert np.array_equal(ksg[~solid], kfd[~solid])
    # accepted (solid) sources hold the renormalised prediction: a delta up to e^-30 entries
    ctr = ksg[solid][:, 8, 8, 8]
    assert np.all(np.abs(ctr - 1.0) <= 1e-9)
    assert np.max(np.abs(ksg[solid].reshape(int(solid.sum()), -1).sum(axis=1) - 1.0)) <= 1e-12


def test_training_lowers_the_loss():
    from paper_2408_11376_gb300 import surrogate as sg
    shape = (24, 22, 20)
    D = _domain(shape, 11, "two_phase")
    lam = oracle.stable_dt_sub(shape, D)
    rng = np.random.default_rng(3)
    src = rng.integers(0, int(np.prod(shape)), 64)
    with FDiRW(shape, D, 60 * lam, 8, 60, "fp32") as f:
        f.kernels()
        tg = f.read_kernels(src)
        net = Net(sg.init_params(4))
        losses = [net.train_step(f.ctx, src, tg, 3e-3) for _ in range(60)]
        net.close()
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.5 * losses[0], losses
