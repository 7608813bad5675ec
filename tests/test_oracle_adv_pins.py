"""Pins of the oracle's convection (Sec. 5: steady flow folded into the kernels): exact upwind shifts at
Courant number 1, the closed window stopping the shift, the diffusion-only limit, and the first moment
advancing by exactly lam_a w per substep."""
import numpy as np
import pytest

import oracle
from paper_2408_11376_gb300 import synth


def _w(n, wx=0.0, wy=0.0, wz=0.0):
    return (np.full(n, wx), np.full(n, wy), np.full(n, wz))


@pytest.mark.parametrize("w,shift", [(1.0, 3), (-1.0, -3)])
def test_courant_one_is_an_exact_shift(w, shift):
    n = 15
    k, m = oracle.source_kernel_adv((n, 1, 1), np.zeros(n), _w(n, w), 0.0, 1.0, 5, 3, 7)
    want = np.zeros(11)
    want[5 + shift] = 1.0
    assert np.array_equal(k[5, 5], want) and m == 1.0


def test_closed_window_stops_the_shift():
    """Seven substeps of a unit shift in a window of radius 5: the mass waits at the window's edge."""
    n = 20
    k, _ = oracle.source_kernel_adv((n, 1, 1), np.zeros(n), _w(n, 1.0), 0.0, 1.0, 5, 7, 9)
    assert k[5, 5, 10] == 1.0 and k.sum() == 1.0


def test_no_flow_is_the_diffusion_kernel():
    shape = (9, 8, 7)
    D = synth.random_diffusivity(shape, 110, 3.0)
    lam = oracle.stable_dt_sub(shape, D)
    for s in (0, 100, 503):
        a, ma = oracle.source_kernel_adv(shape, D, _w(504), lam, 0.7, 3, 11, s)
        b, mb = oracle.source_kernel(shape, D, lam, 3, 11, s)
        assert np.array_equal(a, b) and ma == mb


def test_first_moment_advances_by_lam_a_w():
    """Uniform D and flow, source far from every edge: sum_x x k(x) moves by lam_a w per substep exactly
    (the upwind flux is conservative and diffusion keeps the mean)."""
    shape = (41, 21, 21)
    N = 41 * 21 * 21
    D = np.ones(N)
    lam, lama, wx, wy, n_sub = 0.05, 0.5, 0.4, -0.2, 10
    s = 20 + 41 * (10 + 21 * 10)
    k, m = oracle.source_kernel_adv(shape, D, _w(N, wx, wy), lam, lama, 18, n_sub, s)
    R = 18
    ox = np.arange(-R, R + 1)
    assert (k.sum(axis=(0, 1)) * ox).sum() == pytest.approx(n_sub * lama * wx, abs=1e-12)
    assert (k.sum(axis=(0, 2)) * ox).sum() == pytest.approx(n_sub * lama * wy, abs=1e-12)
    assert m == pytest.approx(1.0, abs=1e-13) and k.min() >= 0.0


def test_superpose_adv_conserves_mass():
    shape = (10, 9, 8)
    D = synth.random_diffusivity(shape, 111, 3.0)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    rng = np.random.default_rng(112)
    w = tuple(rng.uniform(-0.3, 0.3, 720) for _ in range(3))
    c = synth.random_field(720, 113)
    out = oracle.superpose_adv(shape, D, w, lam, 0.5, 3, 9, c)
    assert out.sum() == pytest.approx(c.sum(), rel=1e-13) and out.min() >= 0.0
