"""Pins of the oracle against the paper's Table 1 (Sec. 2): the dimensionless lattice numbers the table's
parameters give, lambda_L = D_L (A_L/RT) dt_fd / dh^2 = 0.1 as the text states and lambda_S = 1e-4, and
dt / dt_fd = 1000 FD substeps per macro step; the oracle's stability limit admits both phases at those
numbers, and a liquid source marched 1000 substeps at lambda = 0.1 in a window it cannot leave keeps its
unit mass, spreads with the random walk's exact variance 2 lambda n and stays non-negative."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _table1():
    vals = {}
    with open(os.path.join(HERE, "golden", "table1_parameters.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_lattice_numbers_from_table1():
    t = _table1()
    dt_fd = t["dt_fd_us"] * 1e-6
    lam_L = t["D_L_m2_s"] * t["A_L_over_RT"] * dt_fd / t["dh_m"] ** 2
    lam_S = t["D_S_m2_s"] * t["A_S_over_RT"] * dt_fd / t["dh_m"] ** 2
    assert lam_L == pytest.approx(t["lambda_L"], rel=1e-12)
    assert lam_S == pytest.approx(1e-4, rel=1e-12)
    assert t["dt_us"] / t["dt_fd_us"] == 1000.0


def test_oracle_stability_admits_table1_numbers():
    """Uniform lattice D = 1: the oracle's largest stable dt_sub is 1/6 (six unit faces), so lambda_L = 0.1
    and the solid's 1e-4 are inside it; a two-phase grid keeps the liquid's limit."""
    shape = (6, 5, 4)
    assert oracle.stable_dt_sub(shape, np.ones(120)) == pytest.approx(1.0 / 6.0, rel=1e-15)
    D = np.where(np.arange(120) % 3 == 0, 1e-3, 1.0)
    assert oracle.stable_dt_sub(shape, D) >= 1.0 / 6.0 * (1 - 1e-15)
    assert _table1()["lambda_L"] <= 1.0 / 6.0


def test_liquid_source_over_one_macro_step_of_table1():
    """lambda = 0.1 and the table's 1000 substeps on a uniform liquid chain with a window of radius 120
    (8.5 standard deviations of the walk, whose tail beyond it is below 1e-16): the kernel keeps mass 1,
    mean 0 and the lazy random walk's exact variance 2 * 0.1 * 1000 = 200, and stays non-negative."""
    lam, n_sub, R = _table1()["lambda_L"], 1000, 120
    n = 2 * R + 1
    k, m = oracle.source_kernel((n, 1, 1), np.ones(n), lam, R, n_sub, R)
    px = k.reshape(-1, n).sum(axis=0)
    ox = np.arange(-R, R + 1)
    assert m == pytest.approx(1.0, abs=1e-12) and px.min() >= 0.0
    assert (px * ox).sum() == pytest.approx(0.0, abs=1e-10)
    assert (px * ox * ox).sum() == pytest.approx(2 * lam * n_sub, rel=1e-10)
