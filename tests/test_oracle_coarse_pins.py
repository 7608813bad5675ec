"""Pins of the oracle's coarse-mesh FDiRW (Sec. 3.1, Eqs. 10-15): hand-worked chains, the reduction to
the fine windowed FDiRW when every block is one cell, a single-block domain, and mass conservation with
a liquid mask and clipped blocks."""
import numpy as np
import pytest

import oracle
from paper_2408_11376_gb300 import synth


def test_chain_two_blocks_by_hand():
    """6 cells in a row, all liquid, D = 1 (face conductance 1), B = 3, one substep of lam:
    u0 = 1 on block 0 -> [1, 1, 1 - lam, lam, 0, 0], so P[0][0] = 1 - lam/3 and P[1][0] = lam/3."""
    lam = 0.2
    shape = (6, 1, 1)
    P = oracle.coarse_kernels(shape, np.ones(6), np.ones(6), 3, lam, 3, 1)
    Rc = oracle.coarse_radius(3, 3)
    assert P.shape == (2, 2 * Rc + 1, 2 * Rc + 1, 2 * Rc + 1)
    assert P[0][Rc, Rc, Rc] == pytest.approx(1 - lam / 3, abs=1e-15)
    assert P[0][Rc, Rc, Rc + 1] == pytest.approx(lam / 3, abs=1e-15)
    assert P[1][Rc, Rc, Rc] == pytest.approx(1 - lam / 3, abs=1e-15)
    assert P[1][Rc, Rc, Rc - 1] == pytest.approx(lam / 3, abs=1e-15)
    assert np.count_nonzero(P) == 4
    c = np.array([0.3, 0.9, 0.6, 2.0, 1.0, 0.0])
    C = np.array([0.6, 1.0])                                     # block means (Eq. 13)
    Cn = np.array([(1 - lam / 3) * C[0] + lam / 3 * C[1], lam / 3 * C[0] + (1 - lam / 3) * C[1]])
    got = oracle.coarse_step(shape, np.ones(6), 3, 3, P, c)
    assert np.allclose(got, np.repeat(Cn, 3), rtol=0, atol=1e-15)   # re-mapping (Eq. 15)


def test_non_liquid_cell_blocks_flux_and_keeps_its_value():
    """Chain [L, L, S, L], B = 1: the solid cell is no fast-diffusion node and cuts the chain."""
    lam = 0.25
    shape = (4, 1, 1)
    liquid = np.array([1, 1, 0, 1])
    P = oracle.coarse_kernels(shape, np.ones(4), liquid, 1, lam, 2, 1)
    Rc = 2
    assert P[0][Rc, Rc, Rc] == pytest.approx(1 - lam) and P[0][Rc, Rc, Rc + 1] == pytest.approx(lam)
    assert P[3][Rc, Rc, Rc] == 1.0 and not P[2].any()
    c = np.array([1.0, 0.0, 5.0, 2.0])
    got = oracle.coarse_step(shape, liquid, 1, 2, P, c)
    assert np.allclose(got, [1 - lam, lam, 5.0, 2.0], rtol=0, atol=1e-15)


def test_unit_blocks_reduce_to_the_fine_windowed_fdirw():
    """B = 1 with every cell liquid: the representative nodes are the cells and P is p (Eq. 8)."""
    shape = (9, 8, 7)
    D = synth.random_diffusivity(shape, 61, 4.0)
    lam = oracle.stable_dt_sub(shape, D)
    c = synth.random_field(D.size, 62)
    liquid = np.ones(D.size)
    P = oracle.coarse_kernels(shape, D, liquid, 1, lam, 3, 13)
    ks, _ = oracle.kernels(shape, D, lam, 3, 13, np.arange(D.size))
    assert np.allclose(P, ks, rtol=0, atol=1e-15)
    got = oracle.coarse_step(shape, liquid, 1, 3, P, c)
    assert np.allclose(got, oracle.superpose(shape, D, lam, 3, 13, c), rtol=1e-14, atol=0)


def test_one_block_is_the_liquid_mean():
    shape = (5, 4, 3)
    D = synth.random_diffusivity(shape, 63, 3.0)
    liquid = (np.random.default_rng(64).random(60) < 0.7).astype(np.uint8)
    lam = oracle.stable_dt_sub(shape, D)
    P = oracle.coarse_kernels(shape, D, liquid, 5, lam, 4, 9)
    c = synth.random_field(60, 65)
    got = oracle.coarse_step(shape, liquid, 5, 4, P, c)
    Rc = oracle.coarse_radius(4, 5)
    assert P[0][Rc, Rc, Rc] == pytest.approx(1.0, abs=1e-15)
    lq = liquid.astype(bool)
    assert np.allclose(got[lq], c[lq].mean(), rtol=1e-15) and np.array_equal(got[~lq], c[~lq])


def test_mass_conservation_with_mask_and_clipped_blocks():
    shape = (13, 12, 11)
    p = synth.sphere_packing(shape, 0.4, 66, r_range=(1.5, 3.0))
    D = synth.diffusivity_per_sphere(p)
    liquid = ~p.solid
    lam = oracle.stable_dt_sub(shape, D)
    for B, R in ((5, 8), (3, 4)):
        P = oracle.coarse_kernels(shape, D, liquid, B, lam, R, 20)
        cnt = oracle.coarse_counts(shape, liquid, B)
        # every column carries its block's mass: sum_I N_I P[I][J] = N_J
        Rc = oracle.coarse_radius(R, B)
        ncx, ncy, ncz = ((n + B - 1) // B for n in shape)
        for J in np.flatnonzero(cnt)[::3]:
            bx, by, bz = J % ncx, (J // ncx) % ncy, J // (ncx * ncy)
            tot = 0.0
            for dz in range(-Rc, Rc + 1):
                for dy in range(-Rc, Rc + 1):
                    for dx in range(-Rc, Rc + 1):
                        cx, cy, cz = bx + dx, by + dy, bz + dz
                        if 0 <= cx < ncx and 0 <= cy < ncy and 0 <= cz < ncz:
                            I = cx + ncx * (cy + ncy * cz)
                            tot += cnt[I] * P[J][dz + Rc, dy + Rc, dx + Rc]
            assert tot == pytest.approx(cnt[J], rel=1e-13)
        c = synth.random_field(D.size, 67, 0.0, 2.0)
        got = oracle.coarse_step(shape, liquid, B, R, P, c)
        assert abs(got.sum() - c.sum()) <= 1e-13 * c.sum()
        assert P.min() >= 0.0


# ------------------------------------------------------------------ far-field boundary (Eq. 7, P_BC c_far)

def test_open_chain_by_hand():
    """3 x 1 x 1 grid, all liquid, D = 1: every cell has 4 open lateral faces and the end cells one more,
    so gb = [5, 4, 5].  One substep: u = 1 - lam gb from the unit block (ghost 0), u = lam gb from the
    ghosts at 1 (field 0); with one block of 3 cells P = (3 - 14 lam) / 3 and P_BC = 14 lam / 3."""
    lam = 0.05
    shape = (3, 1, 1)
    assert np.array_equal(oracle.boundary_conductance(shape, np.ones(3), np.ones(3)), [5.0, 4.0, 5.0])
    P = oracle.coarse_kernels_open(shape, np.ones(3), np.ones(3), 3, lam, 3, 1)
    pbc = oracle.coarse_pbc(shape, np.ones(3), np.ones(3), 3, lam, 1)
    Rc = oracle.coarse_radius(3, 3)
    assert P[0][Rc, Rc, Rc] == pytest.approx((3 - 14 * lam) / 3, abs=1e-15)
    assert pbc[0] == pytest.approx(14 * lam / 3, abs=1e-15)


def test_uniform_far_field_is_a_fixed_point():
    """With windows covering the grid, a liquid at c_far stays at c_far: P 1 + P_BC = 1 on every node."""
    shape = (9, 8, 7)
    D = synth.random_diffusivity(shape, 90, 3.0)
    liquid = (np.random.default_rng(91).random(D.size) < 0.8).astype(np.uint8)
    lam = 0.8 * oracle.stable_dt_sub(shape, D) * 4 / 5      # leave room for the open faces
    B, R = 3, 9
    P = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, 12)
    pbc = oracle.coarse_pbc(shape, D, liquid, B, lam, 12)
    c = np.where(liquid > 0, 0.7, 0.0)
    out, _ = oracle.coarse_step_far(shape, liquid, B, R, P, pbc, 100.0, 0.7, c)
    assert np.allclose(out[liquid > 0], 0.7, rtol=0, atol=1e-14)


def test_far_field_conserves_the_total_and_closes_without_open_faces():
    shape = (12, 11, 10)
    p = synth.sphere_packing(shape, 0.4, 92, r_range=(1.5, 3.0))
    D = synth.diffusivity_per_sphere(p)
    liquid = (~p.solid).astype(np.uint8)
    lam = 0.8 * oracle.stable_dt_sub(shape, D) * 4 / 5
    B, R, n_sub, V_far = 3, 4, 15, 500.0
    P = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, n_sub)
    pbc = oracle.coarse_pbc(shape, D, liquid, B, lam, n_sub)
    c = synth.random_field(D.size, 93, 0.0, 1.0)
    cf = 0.25
    total = c.sum() + V_far * cf
    for _ in range(3):
        c, cf = oracle.coarse_step_far(shape, liquid, B, R, P, pbc, V_far, cf, c)
        assert c.sum() + V_far * cf == pytest.approx(total, rel=1e-14)
    # A liquid phase that never touches the outer surface has no open face: P_BC = 0 and P is the
    # closed coarse matrix.
    inner = liquid.copy().reshape(shape[::-1])
    inner[0, :, :] = inner[-1, :, :] = 0
    inner[:, 0, :] = inner[:, -1, :] = 0
    inner[:, :, 0] = inner[:, :, -1] = 0
    inner = inner.reshape(-1)
    assert not oracle.coarse_pbc(shape, D, inner, B, lam, n_sub).any()
    assert np.allclose(oracle.coarse_kernels_open(shape, D, inner, B, lam, R, n_sub),
                       oracle.coarse_kernels(shape, D, inner, B, lam, R, n_sub), rtol=1e-13, atol=1e-16)


# ------------------------------------------------------------------ coupled macro step (Eqs. 1-7)

def test_absorption_by_hand():
    """Liquid cell at 3 cL_eq next to a solid cell at cS_eq / 4: f_L = 2, f_S = 3/4, m = k f_L f_S dt."""
    k, cS, cL, dt = 0.05, 1.0, 1e-5, 1e-4
    c = np.array([3e-5, 0.25])
    got = oracle.absorb((2, 1, 1), [1, 0], k, cS, cL, dt, c)
    m = k * 2.0 * 0.75 * dt
    assert got[0] == pytest.approx(3e-5 - m, rel=1e-14) and got[1] == pytest.approx(0.25 + m, rel=1e-15)
    # no reaction below the liquid equilibrium or at / above the solid one
    assert np.array_equal(oracle.absorb((2, 1, 1), [1, 0], k, cS, cL, dt, np.array([0.5e-5, 0.25])), [0.5e-5, 0.25])
    assert np.array_equal(oracle.absorb((2, 1, 1), [1, 0], k, cS, cL, dt, np.array([3e-5, 1.2])), [3e-5, 1.2])


def test_absorption_counts_every_interface_face_and_conserves():
    """A liquid cell between two solid cells loses to both; the total is unchanged."""
    k, cS, cL, dt = 0.01, 1.0, 1e-3, 0.1
    c = np.array([0.5, 5e-3, 0.2])
    got = oracle.absorb((3, 1, 1), [0, 1, 0], k, cS, cL, dt, c)
    fL = (5e-3 - 1e-3) / 1e-3
    m0, m2 = k * fL * 0.5 * dt, k * fL * 0.8 * dt
    assert got == pytest.approx([0.5 + m0, 5e-3 - m0 - m2, 0.2 + m2], abs=1e-17)
    shape = (9, 8, 7)
    liquid = (np.random.default_rng(97).random(504) < 0.5).astype(np.uint8)
    c = synth.random_field(504, 98, 0.0, 1e-2)
    assert oracle.absorb(shape, liquid, k, cS, cL, dt, c).sum() == pytest.approx(c.sum(), rel=1e-14)


def test_absorption_only_across_interface_faces_in_every_direction():
    """The reaction of Eqs. 4-6 acts on the solid/liquid interface only: a grid of one phase is left as it
    is whatever its values.  A liquid cell whose six face neighbours are solid (3^3 grid, liquid centre)
    loses m to each of them, m = k f_L f_S dt with f_L = (4e-3 - 1e-3) / 1e-3 = 3 and f_S = (1 - 0.2) / 1
    = 0.8; the edge and corner cells touch no liquid and keep their values."""
    k, cS, cL, dt = 0.01, 1.0, 1e-3, 0.1
    shape = (3, 3, 3)
    c = np.full(27, 0.2)
    c[13] = 4e-3
    for liquid in (np.ones(27), np.zeros(27)):
        assert np.array_equal(oracle.absorb(shape, liquid, k, cS, cL, dt, c), c)
    liquid = np.zeros(27)
    liquid[13] = 1
    got = oracle.absorb(shape, liquid, k, cS, cL, dt, c)
    m = 0.01 * 3.0 * 0.8 * 0.1
    want = np.full(27, 0.2)
    want[[4, 10, 12, 14, 16, 22]] = 0.2 + m         # the six face neighbours of cell 13
    want[13] = 4e-3 - 6 * m
    assert got == pytest.approx(want, abs=1e-17)


def test_solid_march_is_the_full_march_of_the_solid():
    shape = (7, 6, 5)
    D = synth.random_diffusivity(shape, 99, 3.0)
    lam = oracle.stable_dt_sub(shape, D)
    c = synth.random_field(D.size, 100)
    none_liquid = np.zeros(D.size)
    assert np.allclose(oracle.solid_march(shape, D, none_liquid, lam, 9, c), oracle.full_march(shape, D, lam, 9, c),
                       rtol=1e-14, atol=0)
    all_liquid = np.ones(D.size)
    assert np.array_equal(oracle.solid_march(shape, D, all_liquid, lam, 9, c), c)   # no solid face: unchanged


def test_coupled_step_by_hand():
    """Chain solid, solid, liquid (cells of 1, B = 1, closed: P_BC = 0).  The reading's order within the
    macro step: the Eq. 4-6 exchange on the pre-step values first, f_L = (1 - 0.5) / 0.5 = 1,
    f_S = (1 - 0) / 1 = 1, m = k f_L f_S dt = 0.5 * 0.2 = 0.1; then one solid substep of lam_s = 0.25
    across the solid-solid face (conductance 1) moves 0.25 * 0.1 to the first cell; then the coarse step
    of the lone liquid node (P = 1) keeps 0.9, and Eq. 7 leaves c_far unchanged (the near-field total is
    unchanged).  Marching the solid before the exchange would leave the first cell at 0."""
    shape, liquid, D = (3, 1, 1), np.array([0, 0, 1], np.uint8), np.ones(3)
    P = oracle.coarse_kernels(shape, D, liquid, 1, 0.1, 1, 4)
    assert P[2, 1, 1, 1] == 1.0 and np.count_nonzero(P) == 1
    c, cf = oracle.coupled_step(shape, D, liquid, 1, 1, P, np.zeros(3), 10.0, 0.3, 0.5, 1.0, 0.5, 0.2, 0.25, 1,
                                np.array([0.0, 0.0, 1.0]))
    assert c == pytest.approx([0.025, 0.075, 0.9], abs=1e-16)
    assert cf == pytest.approx(0.3, abs=1e-16)


def test_coupled_step_conserves_the_total():
    shape = (12, 11, 10)
    p = synth.sphere_packing(shape, 0.45, 101, r_range=(1.5, 3.0))
    liquid = (~p.solid).astype(np.uint8)
    D = np.where(liquid > 0, 1.0, 1e-3)
    lam = 0.6 * oracle.stable_dt_sub(shape, D)
    B, R, n_sub, V_far = 3, 4, 12, 800.0
    P = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, n_sub)
    pbc = oracle.coarse_pbc(shape, D, liquid, B, lam, n_sub)
    c = np.where(liquid > 0, 2e-3, 1e-6)
    cf = 2e-3
    total = c.sum() + V_far * cf
    for _ in range(3):
        c, cf = oracle.coupled_step(shape, D, liquid, B, R, P, pbc, V_far, cf, 1e-7, 1.0, 1e-5, n_sub * lam,
                                    lam, 2, c)
        assert c.sum() + V_far * cf == pytest.approx(total, rel=1e-13)
    assert c[liquid == 0].sum() > 1e-6 * (liquid == 0).sum()       # the solid absorbed


def _liquid_operator(shape, D, liquid, lo, hi, gb=None):
    """Dense graph Laplacian of the box [lo, hi] (x fastest) over the faces whose two cells are both inside
    the box and both liquid (harmonic-mean conductances), minus gb_i on the diagonal when the open faces
    lose to a ghost (gb: conductance to the far field per cell)."""
    nx, ny, nz = shape
    Dg = np.asarray(D).reshape(nz, ny, nx)
    Lg = np.asarray(liquid).reshape(nz, ny, nx)
    cells = [(x, y, z) for z in range(lo[2], hi[2] + 1) for y in range(lo[1], hi[1] + 1) for x in range(lo[0], hi[0] + 1)]
    at = {c: i for i, c in enumerate(cells)}
    A = np.zeros((len(cells), len(cells)))
    for (x, y, z), i in at.items():
        for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            j = at.get((x + d[0], y + d[1], z + d[2]))
            if j is None or not (Lg[z, y, x] and Lg[z + d[2], y + d[1], x + d[0]]):
                continue
            a, b = Dg[z, y, x], Dg[z + d[2], y + d[1], x + d[0]]
            g = 2.0 * a * b / (a + b)
            A[i, j] += g
            A[j, i] += g
            A[i, i] -= g
            A[j, j] -= g
        if gb is not None:
            A[i, i] -= gb[x + nx * (y + ny * z)]
    return A, cells


def test_coarse_columns_from_the_block_window_propagator():
    """Eqs. 10-12 on a rough D with a liquid mask, blocks of B = 2 (the last ones clipped) and R = 2: column J
    is the unit on J's liquid cells pushed through (I + lam A_W)^n_sub on J's window W (the block widened
    by R, clipped; liquid-liquid faces only), summed over the liquid cells of each block I and mapped to
    N_J S_I / (m N_I).  With the outer faces open to a ghost at 0 (each open face of conductance D_i) the
    column is S_I / N_I; and P_BC is the whole grid marched from 0 with the ghost at 1, mean per block.
    The propagators are assembled densely here and raised with numpy's matrix_power."""
    shape, B, R, n_sub = (7, 5, 4), 2, 2, 6
    nx, ny, nz = shape
    N = nx * ny * nz
    D = synth.random_diffusivity(shape, 131, 3.0)
    liquid = (np.random.default_rng(132).random(N) < 0.75).astype(np.uint8)
    lam = 0.8 * oracle.stable_dt_sub(shape, D)
    ncx, ncy, ncz = (nx + B - 1) // B, (ny + B - 1) // B, (nz + B - 1) // B
    Rc = oracle.coarse_radius(R, B)
    cnt = oracle.coarse_counts(shape, liquid, B)
    gb = oracle.boundary_conductance(shape, D, liquid)
    closed = oracle.coarse_kernels(shape, D, liquid, B, lam, R, n_sub)
    opened = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, n_sub)
    Lg = liquid.reshape(nz, ny, nx)
    checked = 0
    for J in range(ncx * ncy * ncz):
        if cnt[J] == 0:
            assert not closed[J].any() and not opened[J].any()
            continue
        bx, by, bz = J % ncx, (J // ncx) % ncy, J // (ncx * ncy)
        lo = [max(b * B - R, 0) for b in (bx, by, bz)]
        hi = [min(b * B + B - 1 + R, n - 1) for b, n in zip((bx, by, bz), shape)]
        for open_, P in ((False, closed), (True, opened)):
            A, cells = _liquid_operator(shape, D, liquid, lo, hi, gb if open_ else None)
            u0 = np.array([1.0 if (x // B, y // B, z // B) == (bx, by, bz) and Lg[z, y, x] else 0.0
                           for x, y, z in cells])
            u = np.linalg.matrix_power(np.eye(len(cells)) + lam * A, n_sub) @ u0
            m = u.sum()
            want = np.zeros((2 * Rc + 1,) * 3)
            for (x, y, z), v in zip(cells, u):
                if Lg[z, y, x]:
                    want[z // B - bz + Rc, y // B - by + Rc, x // B - bx + Rc] += v
            for dz in range(-Rc, Rc + 1):
                for dy in range(-Rc, Rc + 1):
                    for dx in range(-Rc, Rc + 1):
                        cx, cy, cz = bx + dx, by + dy, bz + dz
                        inside = 0 <= cx < ncx and 0 <= cy < ncy and 0 <= cz < ncz
                        I = cx + ncx * (cy + ncy * cz) if inside else -1
                        o = (dz + Rc, dy + Rc, dx + Rc)
                        if not inside or cnt[I] == 0:
                            want[o] = 0.0
                        else:
                            want[o] = want[o] / cnt[I] if open_ else cnt[J] * want[o] / (m * cnt[I])
            assert np.max(np.abs(P[J] - want)) <= 1e-14, (J, open_)
        checked += 1
    assert checked >= 20
    A, cells = _liquid_operator(shape, D, liquid, (0, 0, 0), (nx - 1, ny - 1, nz - 1), gb)
    step = np.eye(N) + lam * A
    u = np.zeros(N)
    for _ in range(n_sub):
        u = step @ u + lam * gb                       # cells in x-fastest order, as the field
    want = np.zeros(ncx * ncy * ncz)
    for i in range(N):
        if liquid[i]:
            x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
            want[x // B + ncx * (y // B + ncy * (z // B))] += u[i]
    want = np.where(cnt > 0, want / np.maximum(cnt, 1), 0.0)
    assert np.max(np.abs(oracle.coarse_pbc(shape, D, liquid, B, lam, n_sub) - want)) <= 1e-14
