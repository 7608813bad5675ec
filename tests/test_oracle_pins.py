"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms (discrete heat kernel in
the DCT-II basis, lazy-random-walk moments, the random-walk Gaussian of Sec. 1), invariants (mass
conservation, Sec. 3.1 / Eq. 7; positivity; symmetry of the FD propagator), brute force (linearity,
Eq. 8: with windows covering the domain one superposition step equals one full-domain FD march), a
library matmul, and homogenisation of a layered 1D medium (which singles out the harmonic face rule).
"""
import numpy as np
import pytest

import oracle
from paper_2408_11376_gb300 import synth


def _grid_dct_kernel(m, s, lamD, n_sub):
    """Discrete heat kernel of the uniform-D zero-flux box of sides m=(mx,my,mz) from source s, by its
    eigen-decomposition: 1D Neumann Laplacian eigenvectors cos(pi k (j+1/2)/m), eigenvalues
    -4 sin^2(pi k / (2m)); the 3D propagator (I + lamD * L)^n is diagonal in the product basis."""
    phis, mus = [], []
    for ma in m:
        k = np.arange(ma)[:, None]
        j = np.arange(ma)[None, :]
        phi = np.sqrt((2.0 - (k == 0)) / ma) * np.cos(np.pi * k * (j + 0.5) / ma)
        phis.append(phi)
        mus.append(4.0 * np.sin(np.pi * np.arange(ma) / (2.0 * ma)) ** 2)
    mx, my, mz = m
    lam_tot = mus[0][None, None, :] + mus[1][None, :, None] + mus[2][:, None, None]   # [kz, ky, kx]
    amp = (1.0 - lamD * lam_tot) ** n_sub
    cx, cy, cz = (phis[0][:, s[0]], phis[1][:, s[1]], phis[2][:, s[2]])
    coef = amp * cz[:, None, None] * cy[None, :, None] * cx[None, None, :]
    # field[z, y, x] = sum_k coef[kz,ky,kx] phi_z[kz,z] phi_y[ky,y] phi_x[kx,x]
    return np.einsum("cba,cz,by,ax->zyx", coef, phis[2], phis[1], phis[0])


def _kernel_box(k, R, s, shape):
    """Cut the (2R+1)^3 offset-layout kernel down to the window box clipped to the domain."""
    nx, ny, nz = shape
    sx, sy, sz = s
    lo = [max(v - R, 0) for v in (sx, sy, sz)]
    hi = [min(v + R, n - 1) for v, n in zip((sx, sy, sz), (nx, ny, nz))]
    return k[lo[2] - sz + R:hi[2] - sz + R + 1, lo[1] - sy + R:hi[1] - sy + R + 1, lo[0] - sx + R:hi[0] - sx + R + 1]


def _dense_P(shape, D, lam, R, n_sub):
    """Dense matrix P[x, s] = k_s(x) assembled from the oracle's per-source kernels."""
    nx, ny, nz = shape
    N = nx * ny * nz
    ks, _ = oracle.kernels(shape, D, lam, R, n_sub, np.arange(N))
    P = np.zeros((N, N))
    W1 = 2 * R + 1
    oz, oy, ox = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    for s in range(N):
        sx, sy, sz = s % nx, (s // nx) % ny, s // (nx * ny)
        x, y, z = sx + ox, sy + oy, sz + oz
        ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
        P[(x + nx * (y + ny * z))[ok], s] = ks[s][ok]
    assert ks.shape[1] == W1
    return P


def _rough_D(shape, seed, decades=6.0):
    return synth.random_diffusivity(shape, seed, decades)


# ---------------------------------------------------------------- mass, positivity, symmetry

def test_kernel_mass_conservation_and_positivity():
    shape = (9, 8, 7)
    D = _rough_D(shape, 1)
    R, n_sub = 2, 30
    lam = oracle.stable_dt_sub(shape, D)          # exactly at the limit
    N = np.prod(shape)
    ks, masses = oracle.kernels(shape, D, lam, R, n_sub, np.arange(N))
    W = (2 * R + 1) ** 3
    # The flux form moves mass between cells and never creates it (Sec. 3.1; Eq. 7 conserves totals).
    assert np.max(np.abs(masses - 1.0)) <= n_sub * W * 1e-16
    assert np.max(np.abs(ks.reshape(N, -1).sum(axis=1) - 1.0)) <= 1e-14
    # At lam * max(sum g) <= 1 every explicit coefficient is >= 0, hence every kernel entry is.
    assert ks.min() >= 0.0


def test_kernel_symmetry_when_window_is_domain():
    shape = (5, 4, 3)
    D = _rough_D(shape, 2)
    lam = 0.9 * oracle.stable_dt_sub(shape, D)
    P = _dense_P(shape, D, lam, R=4, n_sub=23)
    # Symmetric face conductances and equal cell volumes make the FD propagator symmetric.
    assert np.max(np.abs(P - P.T)) <= 1e-14


def _box_propagator(shape, D, lam, n_sub, lo, hi):
    """(I + lam A_B)^n_sub for the box [lo, hi] (inclusive, x fastest): A_B is the graph Laplacian of the
    faces with both cells in the box, each of conductance 2 D_a D_b / (D_a + D_b), assembled densely here
    and raised to the power with numpy's matrix_power."""
    nx, ny, _ = shape
    Dg = np.asarray(D).reshape(shape[2], ny, nx)
    cells = [(x, y, z) for z in range(lo[2], hi[2] + 1) for y in range(lo[1], hi[1] + 1) for x in range(lo[0], hi[0] + 1)]
    at = {c: i for i, c in enumerate(cells)}
    A = np.zeros((len(cells), len(cells)))
    for (x, y, z), i in at.items():
        for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            j = at.get((x + d[0], y + d[1], z + d[2]))
            if j is None:
                continue
            a, b = Dg[z, y, x], Dg[z + d[2], y + d[1], x + d[0]]
            g = 2.0 * a * b / (a + b) if a + b > 0 else 0.0
            A[i, j] += g
            A[j, i] += g
            A[i, i] -= g
            A[j, j] -= g
    return np.linalg.matrix_power(np.eye(len(cells)) + lam * A, n_sub), cells


@pytest.mark.parametrize("s", [(4, 4, 3), (0, 7, 6), (8, 0, 3)])
def test_windowed_kernel_is_a_column_of_the_box_propagator(s):
    """Sec. 3.1 with a window smaller than the domain and a rough D: the kernel of s is column s of the
    box propagator (I + lam A_B)^n_sub of its clipped window B_s, divided by that column's sum, and the box
    propagator is symmetric (symmetric faces, equal cell volumes).  An interior window, a corner and an
    edge."""
    shape, R, n_sub = (9, 8, 7), 2, 13
    D = _rough_D(shape, 5)
    lam = 0.8 * oracle.stable_dt_sub(shape, D)
    lo = [max(v - R, 0) for v in s]
    hi = [min(v + R, n - 1) for v, n in zip(s, shape)]
    M, cells = _box_propagator(shape, D, lam, n_sub, lo, hi)
    assert np.max(np.abs(M - M.T)) <= 1e-15
    col = M[:, cells.index(tuple(s))]
    k, m = oracle.source_kernel(shape, D, lam, R, n_sub, s[0] + shape[0] * (s[1] + shape[1] * s[2]))
    got = np.array([k[z - s[2] + R, y - s[1] + R, x - s[0] + R] for x, y, z in cells])
    assert m == pytest.approx(col.sum(), abs=1e-14)
    assert np.max(np.abs(got - col / col.sum())) <= 1e-15
    assert k.sum() == pytest.approx(got.sum(), abs=1e-15)          # nothing outside the clipped window


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("shape,R,s", [
    ((6, 5, 4), 5, None),            # window = domain, every source
    ((20, 20, 20), 3, (10, 10, 10)),  # window strictly inside the domain (zero flux at the window faces)
    ((20, 20, 20), 3, (1, 0, 18)),    # window clipped at a domain corner
])
def test_uniform_D_matches_dct_heat_kernel(shape, R, s):
    Dval, n_sub = 0.7, 13
    nx, ny, nz = shape
    D = np.full(nx * ny * nz, Dval)
    lam = 0.8 * oracle.stable_dt_sub(shape, D)
    cond = oracle.Conductance(shape, D)
    srcs = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)] if s is None else [s]
    for (sx, sy, sz) in srcs:
        k, _ = oracle.source_kernel(shape, D, lam, R, n_sub, sx + nx * (sy + ny * sz), cond)
        lo = [max(v - R, 0) for v in (sx, sy, sz)]
        hi = [min(v + R, n - 1) for v, n in zip((sx, sy, sz), shape)]
        m = tuple(h - l + 1 for l, h in zip(lo, hi))
        expect = _grid_dct_kernel(m, (sx - lo[0], sy - lo[1], sz - lo[2]), lam * Dval, n_sub)
        got = _kernel_box(k, R, (sx, sy, sz), shape)
        assert got.shape == expect.shape
        assert np.max(np.abs(got - expect)) <= 1e-13
        # and nothing outside the clipped window
        outside = np.ones_like(k, dtype=bool)
        _kernel_box(outside, R, (sx, sy, sz), shape)[...] = False
        assert np.all(k[outside] == 0.0)


@pytest.mark.parametrize("p", [1.0 / 12.0, 1.0 / 6.0])
def test_uniform_D_lazy_random_walk_moments(p):
    # D = 1, lam = p: each substep moves the walker one cell along one of 6 directions with probability
    # p each, else it stays.  With R >= n_sub the window edge is never reached, so the kernel is exactly
    # the law of this walk after n_sub steps.
    n_sub, R = 8, 8
    shape = (17, 17, 17)
    D = np.ones(17 ** 3)
    k, _ = oracle.source_kernel(shape, D, p, R, n_sub, 8 + 17 * (8 + 17 * 8))
    o = np.arange(-R, R + 1, dtype=np.float64)
    oz, oy, ox = np.meshgrid(o, o, o, indexing="ij")
    E = lambda f: float((k * f).sum())
    n, q = n_sub, 2.0 * p
    for a in (ox, oy, oz):
        assert abs(E(a)) <= 1e-14
        assert abs(E(a ** 2) - q * n) <= 1e-13
        assert abs(E(a ** 4) - (q * n + 3 * n * (n - 1) * q * q)) <= 1e-12
    assert abs(E(ox * oy)) <= 1e-14
    assert abs(E(ox ** 2 * oy ** 2) - n * (n - 1) * q * q) <= 1e-12


def test_uniform_D_approaches_random_walk_gaussian():
    # Sec. 1: the Random-Walk model's analytical long-time solution for isotropic diffusion.
    Dval, lam, n_sub, R = 1.0, 1.0 / 12.0, 300, 30
    W1 = 2 * R + 1
    shape = (W1, W1, W1)
    D = np.full(W1 ** 3, Dval)
    k, _ = oracle.source_kernel(shape, D, lam, R, n_sub, R + W1 * (R + W1 * R))
    Dt = Dval * lam * n_sub                     # = 25 cells^2
    o = np.arange(-R, R + 1, dtype=np.float64)
    oz, oy, ox = np.meshgrid(o, o, o, indexing="ij")
    g = (4.0 * np.pi * Dt) ** -1.5 * np.exp(-(ox ** 2 + oy ** 2 + oz ** 2) / (4.0 * Dt))
    assert np.max(np.abs(k - g)) <= 0.02 * g.max()


def test_two_cell_closed_form():
    D, lam, n = 0.8, 0.4, 7
    k, _ = oracle.source_kernel((2, 1, 1), np.array([D, D]), lam, 1, n, 0)
    mu = 1.0 - 2.0 * lam * D
    got = k[1, 1, 1:]      # offsets ox = 0, +1
    assert np.allclose(got, [(1 + mu ** n) / 2, (1 - mu ** n) / 2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_harmonic_face_rule_reproduces_layered_medium_homogenisation(axis):
    # Cells with period-3 diffusivities along one axis; the two other axes are 2 cells wide, so the face
    # rule must pair each cell with its neighbour along that axis and not along another.  Homogenisation
    # of a layered medium in series gives D_eff with 1/D_eff = mean(1/D).  The long-time variance of the
    # point-source solution along the layered axis grows as 2 D_eff t, so its slope pins the face rule
    # (an arithmetic-mean face rule gives ~0.36 here, against 0.123).  The marginal along that axis is a
    # 1D chain exactly (the faces across the other axes only move mass within a layer); the full-domain
    # march stands for a window covering the domain, which the solution does not reach in 3000 substeps.
    period = np.array([1.0, 0.3, 0.05])
    n = 801
    layer = np.tile(period, n // 3 + 1)[:n]
    dims = [2, 2, 2]
    dims[axis] = n
    shape = tuple(dims)
    coord = np.meshgrid(np.arange(dims[0]), np.arange(dims[1]), np.arange(dims[2]), indexing="ij")[axis]
    D = layer[coord].transpose(2, 1, 0).reshape(-1)          # x fastest
    lam = oracle.stable_dt_sub(shape, D)
    cond = oracle.Conductance(shape, D)
    x = np.arange(n, dtype=np.float64)
    slopes = []
    for s in (399, 400, 401):                   # three phases of the period
        c0 = np.zeros(D.size)
        at = [0, 0, 0]
        at[axis] = s
        c0[at[0] + dims[0] * (at[1] + dims[1] * at[2])] = 1.0
        c1 = oracle.full_march(shape, D, lam, 1500, c0, cond)
        c2 = oracle.full_march(shape, D, lam, 1500, c1, cond)
        var = []
        for c in (c1, c2):
            kk = c.reshape(dims[2], dims[1], dims[0]).sum(axis=tuple(a for a in (0, 1, 2) if a != 2 - axis))
            mean = (kk * x).sum()
            var.append((kk * (x - mean) ** 2).sum())
        slopes.append((var[1] - var[0]) / (2.0 * lam * 1500))
    d_eff = 1.0 / np.mean(1.0 / period)
    assert abs(np.mean(slopes) - d_eff) <= 0.01 * d_eff


def test_grid_spacing_scales_out():
    # The diffusion equation is unchanged by x -> x / h, t -> t / h^2: with lam = (dt_macro / n_sub) / h^2
    # the lazy walk's exact variance 2 lam n_sub (cells^2), times h^2, is the continuum 2 D dt_macro for
    # every h (window never reached: R >= n_sub).  The largest stable dt_sub turns back into 1 / (max face
    # sum) through the same lam.
    D, n_sub, R = 1.0, 8, 8
    W1 = 2 * R + 1
    shape = (W1, W1, W1)
    Dm = np.full(W1 ** 3, D)
    o = np.arange(-R, R + 1, dtype=np.float64)
    for h, dt_macro in ((0.5, 0.2), (2.0, 3.2), (1.0, 0.8)):
        lam = oracle.lam_of(dt_macro, n_sub, h)
        assert lam == pytest.approx(0.1, rel=1e-15)
        k, _ = oracle.source_kernel(shape, Dm, lam, R, n_sub, R + W1 * (R + W1 * R))
        var_x = float((k.sum(axis=(0, 1)) * o * o).sum())
        assert var_x * h * h == pytest.approx(2.0 * D * dt_macro, rel=1e-13)
        dts = oracle.stable_dt_sub(shape, Dm, h)
        assert oracle.lam_of(dts * n_sub, n_sub, h) == pytest.approx(1.0 / 6.0, rel=1e-15)


def test_stability_limit_closed_form():
    # Uniform D on a 3^3 grid: the centre cell has 6 faces of conductance D.
    D = np.full(27, 2.5)
    assert oracle.max_face_sum((3, 3, 3), D) == 6 * 2.5
    assert oracle.stable_dt_sub((3, 3, 3), D, h=2.0) == 4.0 / 15.0


# ---------------------------------------------------------------- linearity / brute force / matmul

@pytest.mark.parametrize("seed", [3, 4])
def test_superposition_equals_full_domain_march(seed):
    shape = (5, 4, 3)
    D = _rough_D(shape, seed) if seed == 3 else synth.diffusivity_two_phase(
        synth.sphere_packing(shape, 0.4, seed, r_range=(1.0, 2.0)), 1.0, 1e-5)
    lam = oracle.stable_dt_sub(shape, D)
    c = synth.random_field(60, seed + 10)
    got = oracle.superpose(shape, D, lam, 4, 17, c)
    ref = oracle.full_march(shape, D, lam, 17, c)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-13


def test_superpose_matches_dense_matmul_and_is_not_symmetric():
    shape = (6, 5, 4)
    D = _rough_D(shape, 5)
    lam = oracle.stable_dt_sub(shape, D)
    R, n_sub = 2, 9
    P = _dense_P(shape, D, lam, R, n_sub)
    # With windows smaller than the domain P is not symmetric, so a transposed gather would fail below.
    assert np.max(np.abs(P - P.T)) > 1e-6
    c = synth.random_field(P.shape[0], 6)
    got = oracle.superpose(shape, D, lam, R, n_sub, c)
    ref = P @ c
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-13
    assert abs(oracle.mass(got) - oracle.mass(c)) <= 1e-13 * oracle.mass(c)


# ---------------------------------------------------------------- degenerate cases, determinism

def test_degenerate_cases_are_identity():
    shape = (4, 3, 3)
    N = 36
    D = _rough_D(shape, 7)
    lam = oracle.stable_dt_sub(shape, D)
    c = synth.random_field(N, 8)
    assert np.array_equal(oracle.superpose(shape, D, lam, 2, 0, c), c)          # n_sub = 0
    assert np.array_equal(oracle.superpose(shape, D, lam, 0, 11, c), c)         # R = 0
    assert np.array_equal(oracle.superpose(shape, np.zeros(N), 0.3, 2, 11, c), c)  # D = 0


def test_determinism_bitwise():
    shape = (7, 6, 5)
    D = _rough_D(shape, 9)
    lam = oracle.stable_dt_sub(shape, D)
    c = synth.random_field(210, 10)
    a = oracle.superpose(shape, D, lam, 2, 12, c)
    b = oracle.superpose(shape, D, lam, 2, 12, c)
    assert np.array_equal(a, b)
    oracle.set_threads(1)
    k1, _ = oracle.kernels(shape, D, lam, 2, 12, np.arange(210))
    oracle.set_threads(4)
    k4, _ = oracle.kernels(shape, D, lam, 2, 12, np.arange(210))
    assert np.array_equal(k1, k4)


def test_bad_arguments_are_rejected():
    shape = (3, 3, 3)
    D = np.ones(27)
    with pytest.raises(ValueError):
        oracle.source_kernel(shape, D, 0.1, 1, 3, 27)
    with pytest.raises(ValueError):
        oracle.source_kernel(shape, D, 0.1, -1, 3, 0)


# ---------------------------------------------------------------- input generator (not the method)

def test_sphere_packing_reaches_porosity_and_is_seeded():
    p1 = synth.sphere_packing((32, 32, 32), 0.4, 20240821)
    p2 = synth.sphere_packing((32, 32, 32), 0.4, 20240821)
    p3 = synth.sphere_packing((32, 32, 32), 0.4, 20240822)
    assert np.array_equal(p1.solid, p2.solid)
    assert not np.array_equal(p1.solid, p3.solid)
    assert 0.39 <= p1.porosity <= 0.41
    d = synth.diffusivity_per_sphere(p1)
    assert np.all((d[p1.solid] <= 1e-3 + 1e-15) & (d[p1.solid] >= 1e-8 - 1e-20))
    assert np.all(d[~p1.solid] == 1.0)
