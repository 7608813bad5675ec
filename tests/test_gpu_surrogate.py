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


def test_forward_matches_oracle():
    shape = (24, 22, 20)
    D = _domain(shape, 5)
    Ws, bs = _random_params(1)
    src = np.array([0, 23, 24 * 22 * 20 - 1, 10 + 24 * (11 + 22 * 10), 5 + 24 * (3 + 22 * 17)])
    with FDiRW(shape, D, 0.1, 8, 1, "fp32") as f:            # march settings unused here
        net = Net(fdirw.pack_params(Ws, bs))
        k, m, _ = net.predict(f.ctx, src)
        net.close()
    for q, s in enumerate(src):
        y, mo, _ = so.forward(so.features(D, shape, int(s)), Ws, bs)
        assert np.max(np.abs(k[q] - y)) <= 2e-2 * np.abs(y).max(), (q, np.max(np.abs(k[q] - y)), np.abs(y).max())
        assert abs(m[q] - mo) <= 2e-2 * mo


def test_gradients_match_oracle():
    shape = (24, 22, 20)
    D = _domain(shape, 6)
    Ws, bs = _random_params(2)
    src = np.array([3, 10 + 24 * (11 + 22 * 10), 5 + 24 * (3 + 22 * 17)])
    rng = np.random.default_rng(7)
    tg = rng.random((len(src), 17, 17, 17)) * 1e-3
    with FDiRW(shape, D, 0.1, 8, 1, "fp32") as f:            # march settings unused here
        net = Net(fdirw.pack_params(Ws, bs))
        g, loss = net.gradients(f.ctx, src, tg)
        net.close()
    dW = [np.zeros((27, 16, 16)) for _ in range(4)]
    db = [np.zeros(16) for _ in range(4)]
    lo = 0.0
    for q, s in enumerate(src):
        _, _, cache = so.forward(so.features(D, shape, int(s)), Ws, bs)
        l, dz = so.loss_grad(cache, tg[q])
        lo += l
        w_, b_ = so.backward(Ws, cache, dz)
        for i in range(4):
            dW[i] += w_[i]
            db[i] += b_[i]
    gW, gb = fdirw.unpack_params(g)
    assert abs(loss - lo / len(src)) <= 1e-2 * lo / len(src)
    for i in range(4):
        ref = np.concatenate([dW[i].ravel(), db[i]])
        got = np.concatenate([gW[i].ravel(), gb[i]])
        if np.linalg.norm(ref) == 0.0:
            continue
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 3e-2, (i, rel)


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
