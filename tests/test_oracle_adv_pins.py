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


def test_kernel_is_a_column_of_the_upwind_box_propagator():
    """Sec. 5 with a rough D and a non-uniform flow: the kernel of s is column s of (I + lam A_B + lam_a V_B)^n_sub
    for its clipped window B_s, divided by the column's sum.  A_B is the diffusive graph Laplacian of the
    faces inside the box (harmonic-mean conductances); V_B is the upwind operator: through the face from
    a lower cell l to the upper cell u with velocity w, u gains w+ u_l - w- u_u and l loses it.  Both are
    assembled densely here and raised with numpy's matrix_power."""
    shape, R, n_sub, lama = (8, 7, 6), 2, 9, 0.3
    nx, ny, nz = shape
    N = nx * ny * nz
    D = synth.random_diffusivity(shape, 117, 4.0)
    rng = np.random.default_rng(118)
    w = tuple(rng.uniform(-0.3, 0.3, N) for _ in range(3))
    lam = 0.3 * oracle.stable_dt_sub(shape, D)         # diffusion 0.3 + outflow at most 6 * 0.3 * 0.3: below 1
    Dg = D.reshape(nz, ny, nx)
    for s in ((4, 3, 3), (0, 6, 5), (7, 0, 2)):
        lo = [max(v - R, 0) for v in s]
        hi = [min(v + R, n - 1) for v, n in zip(s, shape)]
        cells = [(x, y, z) for z in range(lo[2], hi[2] + 1) for y in range(lo[1], hi[1] + 1)
                 for x in range(lo[0], hi[0] + 1)]
        at = {c: i for i, c in enumerate(cells)}
        A = np.zeros((len(cells), len(cells)))
        V = np.zeros_like(A)
        for (x, y, z), l in at.items():
            for axis, d in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                u = at.get((x + d[0], y + d[1], z + d[2]))
                if u is None:
                    continue
                a, b = Dg[z, y, x], Dg[z + d[2], y + d[1], x + d[0]]
                g = 2.0 * a * b / (a + b) if a + b > 0 else 0.0
                A[l, u] += g
                A[u, l] += g
                A[l, l] -= g
                A[u, u] -= g
                wf = w[axis][x + nx * (y + ny * z)]
                wp, wm = max(wf, 0.0), max(-wf, 0.0)
                V[u, l] += wp
                V[l, l] -= wp
                V[l, u] += wm
                V[u, u] -= wm
        step = np.eye(len(cells)) + lam * A + lama * V
        assert np.diag(step).min() >= 0.0                  # every explicit coefficient non-negative
        M = np.linalg.matrix_power(step, n_sub)
        col = M[:, at[s]]
        k, m = oracle.source_kernel_adv(shape, D, w, lam, lama, R, n_sub, s[0] + nx * (s[1] + ny * s[2]))
        got = np.array([k[z - s[2] + R, y - s[1] + R, x - s[0] + R] for x, y, z in cells])
        assert m == pytest.approx(col.sum(), abs=1e-14)
        assert np.max(np.abs(got - col / col.sum())) <= 1e-15
        assert k.min() >= 0.0 and k.sum() == pytest.approx(1.0, abs=1e-14)


def test_superpose_adv_moves_the_mean_by_lam_a_w():
    """Eq. 8 with convection on a field that is a point mass a: the step gives a times that source's
    kernel, so the mass stays a and the first moment moves by a n_sub lam_a w exactly (n_sub <= R: no
    walker reaches a window face), with lam != lam_a."""
    shape, a = (25, 9, 9), 3.0
    N = 25 * 9 * 9
    lam, lama, wx, wy, n_sub, R = 0.05, 0.5, 0.4, -0.2, 4, 4
    s = 12 + 25 * (4 + 9 * 4)
    c = np.zeros(N)
    c[s] = a
    out = oracle.superpose_adv(shape, np.ones(N), _w(N, wx, wy), lam, lama, R, n_sub, c).reshape(9, 9, 25)
    x, y = np.arange(25) - 12, np.arange(9) - 4
    assert out.sum() == pytest.approx(a, rel=1e-14) and out.min() >= 0.0
    assert (out.sum(axis=(0, 1)) * x).sum() == pytest.approx(a * n_sub * lama * wx, abs=1e-12)
    assert (out.sum(axis=(0, 2)) * y).sum() == pytest.approx(a * n_sub * lama * wy, abs=1e-12)


# ---------------------------------------------------------------- convection on the coarse (liquid) path

def _packing(shape, seed):
    p = synth.sphere_packing(shape, 0.45, seed, r_range=(1.5, 3.0))
    return synth.diffusivity_per_sphere(p), (~p.solid).astype(np.uint8)


def test_coarse_no_flow_is_the_diffusion_matrix():
    shape = (12, 11, 10)
    D, liquid = _packing(shape, 112)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    w0 = _w(D.size)
    assert np.array_equal(oracle.coarse_kernels(shape, D, liquid, 3, lam, 2, 12, w=w0),
                          oracle.coarse_kernels(shape, D, liquid, 3, lam, 2, 12))
    assert np.array_equal(oracle.coarse_kernels_open(shape, D, liquid, 3, lam, 2, 12, w=w0),
                          oracle.coarse_kernels_open(shape, D, liquid, 3, lam, 2, 12))
    assert np.array_equal(oracle.coarse_pbc(shape, D, liquid, 3, lam, 12, w=w0),
                          oracle.coarse_pbc(shape, D, liquid, 3, lam, 12))


def test_coarse_unit_blocks_are_the_fine_upwind_kernels():
    """B = 1 on an all-liquid grid: column J of P is the fine kernel of source J with the same flow."""
    shape = (9, 8, 7)
    N = 504
    D = synth.random_diffusivity(shape, 113, 2.0)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    w = synth.face_velocity(shape, 114, (0.3, -0.2, 0.1), 0.3)
    P = oracle.coarse_kernels(shape, D, np.ones(N, np.uint8), 1, lam, 2, 15, w=w)
    for J in (0, 77, 250, 503):
        k, _ = oracle.source_kernel_adv(shape, D, w, lam, lam, 2, 15, J)
        assert np.array_equal(P[J], k), J


def test_coarse_flow_columns_conserve_and_stay_positive():
    """Closed windows: every column carries its block's liquid cells exactly (sum_I P[I][J] N_I = N_J),
    the flow moves mass downstream (the +x neighbour block gains against the no-flow matrix), and with
    the outer faces open the columns only lose mass."""
    shape = (15, 9, 9)
    D, liquid = _packing(shape, 115)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    B, R, n_sub = 3, 3, 20
    w = synth.face_velocity(shape, 116, (0.6, 0.0, 0.0), 0.0)
    P = oracle.coarse_kernels(shape, D, liquid, B, lam, R, n_sub, w=w)
    P0 = oracle.coarse_kernels(shape, D, liquid, B, lam, R, n_sub)
    Po = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, n_sub, w=w)
    cnt = oracle.coarse_counts(shape, liquid, B)
    ncx, ncy, ncz = 5, 3, 3
    Rc = 1
    for J in np.flatnonzero(cnt):
        bx, by, bz = J % ncx, (J // ncx) % ncy, J // (ncx * ncy)
        tot = 0.0
        for dz in range(-Rc, Rc + 1):
            for dy in range(-Rc, Rc + 1):
                for dx in range(-Rc, Rc + 1):
                    cx, cy, cz = bx + dx, by + dy, bz + dz
                    if 0 <= cx < ncx and 0 <= cy < ncy and 0 <= cz < ncz:
                        tot += P[J, dz + Rc, dy + Rc, dx + Rc] * cnt[cx + ncx * (cy + ncy * cz)]
        assert tot == pytest.approx(cnt[J], rel=1e-12)
    assert P.min() >= 0.0 and Po.min() >= 0.0
    assert np.all(Po.reshape(len(cnt), -1).sum(1) <= P.reshape(len(cnt), -1).sum(1) * (1 + 1e-12) + 1e-15)
    downstream = P[:, Rc, Rc, Rc + 1] - P0[:, Rc, Rc, Rc + 1]
    assert downstream[np.flatnonzero(cnt)].sum() > 0.0


def test_radius_map_superposition_with_flow():
    """The per-source-radius superposition with flow: w = 0 gives superpose_rmap bit for bit, and a
    constant radius map gives superpose_adv bit for bit (both follow from the definitions)."""
    shape = (10, 9, 8)
    N = 720
    D = synth.random_diffusivity(shape, 117, 3.0)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    c = synth.random_field(N, 118)
    Rmap = (np.arange(N) % 3 + 1).astype(np.int32)
    assert np.array_equal(oracle.superpose_rmap_adv(shape, D, _w(N), lam, lam, Rmap, 9, c),
                          oracle.superpose_rmap(shape, D, lam, Rmap, 9, c))
    w = synth.face_velocity(shape, 119, (0.2, 0.1, -0.1), 0.2)
    assert np.array_equal(oracle.superpose_rmap_adv(shape, D, w, lam, lam, np.full(N, 2, np.int32), 9, c),
                          oracle.superpose_adv(shape, D, w, lam, lam, 2, 9, c))
