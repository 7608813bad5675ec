"""Pins of the oracle's per-source window radius (batched variant): the radius rule against values worked
out by hand, and the variable-radius superposition against hand-derived chains, the uniform-radius
superposition and the full-domain march."""
import numpy as np
import pytest

import oracle
from paper_2408_11376_gb300 import synth


def test_radius_rule_hand_values():
    # R = clamp(ceil(2 sqrt(2 D dt) / h), R_min, R_max)
    D = np.array([1.0, 0.5, 2.0, 0.125, 0.0, 1e-3, 0.5, 4.5])
    dt = np.array([12.5, 1.0, 1.0, 1.0, 5.0, 12.5, 12.5, 1.0])
    want = {  # (D, dt, h) -> unclamped ceil
        0: 10,   # 2 sqrt(25) = 10 exactly
        1: 2,    # 2 sqrt(1) = 2 exactly: no rounding up
        2: 4,    # 2 sqrt(4) = 4
        3: 1,    # 2 sqrt(0.25) = 1
        4: 0,    # D = 0
        5: 1,    # 2 sqrt(0.025) = 0.316...
        6: 8,    # 2 sqrt(12.5) = 7.07...
        7: 6,    # 2 sqrt(9) = 6
    }
    for i, r in want.items():
        assert oracle.radius_map(D[i:i + 1], dt[i], 1.0, 0, 99)[0] == r, i
        assert oracle.radius_map(D[i:i + 1], dt[i], 1.0, 3, 7)[0] == min(max(r, 3), 7), i
    # h scales the length: 2 sqrt(2 * 2 * 1) / 2 = 2; / 0.5 -> 8
    assert oracle.radius_map(np.array([2.0]), 1.0, 2.0, 0, 99)[0] == 2
    assert oracle.radius_map(np.array([2.0]), 1.0, 0.5, 0, 99)[0] == 8


def test_radius_rule_on_two_phase_workload():
    """Pore D = 1 at dt_macro = 75 / 6 gives R = 10; solid D <= 1e-3 falls to R_min = 3."""
    p = synth.sphere_packing((20, 20, 20), 0.4, 5)
    D = synth.diffusivity_per_sphere(p)
    R = oracle.radius_map(D, 75.0 / 6.0, 1.0, 3, 10)
    assert set(np.unique(R)) <= {3, 10}
    assert np.array_equal(R == 10, D == 1.0)


def _chain_cond(lam):
    shape = (3, 1, 1)
    return shape, np.ones(3), lam


@pytest.mark.parametrize("n_sub", [1, 2])
def test_rmap_chain_middle_source_only(n_sub):
    """3-cell chain, D = 1 (face conductance 1), radii [0, 1, 0]: only the middle source spreads."""
    shape, D, lam = _chain_cond(0.25)
    c = np.array([0.7, 1.3, 0.4])
    M = np.array([[1 - lam, lam, 0.0], [lam, 1 - 2 * lam, lam], [0.0, lam, 1 - lam]])
    u = np.linalg.matrix_power(M, n_sub) @ np.array([0.0, 1.0, 0.0])
    want = np.array([c[0] + c[1] * u[0], c[1] * u[1], c[2] + c[1] * u[2]])
    got = oracle.superpose_rmap(shape, D, lam, [0, 1, 0], n_sub, c)
    assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_rmap_chain_uses_the_source_radius():
    """Radii [1, 0, 0]: source 0 spreads over its clipped window {0, 1}; cell 1 keeps its own mass
    (a destination-radius reading would give a different field)."""
    shape, D, lam = _chain_cond(0.3)
    c = np.array([0.9, 0.2, 0.5])
    got = oracle.superpose_rmap(shape, D, lam, [1, 0, 0], 1, c)
    want = np.array([c[0] * (1 - lam), c[1] + c[0] * lam, c[2]])
    assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_rmap_constant_equals_uniform_window():
    shape = (9, 8, 7)
    D = synth.random_diffusivity(shape, 3, 4.0)
    lam = oracle.stable_dt_sub(shape, D)
    c = synth.random_field(int(np.prod(shape)), 4)
    for R in (0, 2, 3):
        a = oracle.superpose_rmap(shape, D, lam, np.full(c.size, R), 11, c)
        b = oracle.superpose(shape, D, lam, R, 11, c)
        assert np.array_equal(a, b), R


def test_rmap_large_radius_is_full_march():
    shape = (6, 5, 4)
    D = synth.random_diffusivity(shape, 5, 4.0)
    lam = oracle.stable_dt_sub(shape, D)
    c = synth.random_field(120, 6)
    Rmap = np.random.default_rng(7).integers(6, 9, size=120)     # every window covers the domain
    got = oracle.superpose_rmap(shape, D, lam, Rmap, 9, c)
    ref = oracle.full_march(shape, D, lam, 9, c)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-15)


def test_rmap_mass_and_positivity():
    shape = (11, 10, 9)
    p = synth.sphere_packing(shape, 0.4, 8, r_range=(1.5, 3.0))
    D = synth.diffusivity_per_sphere(p)
    lam = oracle.stable_dt_sub(shape, D)
    Rmap = oracle.radius_map(D, 7 * lam, 1.0, 1, 4)
    c = synth.random_field(D.size, 9, 0.0, 1.0)
    got = oracle.superpose_rmap(shape, D, lam, Rmap, 7, c)
    assert abs(got.sum() - c.sum()) <= 1e-13 * c.sum()
    assert got.min() >= 0.0
    assert len(np.unique(Rmap)) >= 2
