"""GPU parity of the coarse-mesh FDiRW (fdirw_create_coarse, Eqs. 10-15) against the FP64 oracle: every
column of the coarse matrix, macro steps element by element (non-liquid cells bit for bit unchanged),
unit blocks against the fine windowed FDiRW, the largest window, and argument errors."""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_11376_gb300 import FDiRWCoarse, FdirwError, fdirw, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
P_TOL = 1e-5          # FP32 march, FP64 mapping: per-column relative L2
FIELD_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(shape, seed):
    p = synth.sphere_packing(shape, 0.4, seed, r_range=(1.5, 3.5))
    D = synth.diffusivity_per_sphere(p)
    return D, (~p.solid).astype(np.uint8)


@pytest.mark.parametrize("shape,B,R,n_sub", [((23, 21, 19), 5, 3, 30), ((17, 16, 15), 3, 4, 25)])
def test_coarse_matrix_matches_oracle(shape, B, R, n_sub):
    """Clipped blocks on every face (sides not multiples of B), a liquid mask from a sphere packing."""
    D, liquid = _case(shape, 70 + B)
    lam = oracle.stable_dt_sub(shape, D)
    ref = oracle.coarse_kernels(shape, D, liquid, B, lam, R, n_sub)
    with FDiRWCoarse(shape, torch.from_numpy(D).to(DEV), torch.from_numpy(liquid).to(DEV), B, n_sub * lam, R,
                     n_sub) as f:
        f.kernels()
        info = f.info()
        got = f.read_coarse(np.arange(ref.shape[0]))
    cnt = oracle.coarse_counts(shape, liquid, B)
    assert info["coarse_block"] == B and info["coarse_nodes"] == int(np.count_nonzero(cnt))
    for J in range(ref.shape[0]):
        if cnt[J] == 0:
            assert not got[J].any()
            continue
        assert _rel(got[J], ref[J]) <= P_TOL, (J, _rel(got[J], ref[J]))
        assert (got[J] >= 0).all()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_coarse_steps_match_oracle(prec):
    shape, B, R, n_sub = (24, 20, 18), 5, 4, 30
    D, liquid = _case(shape, 80)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 81, 0.0, 2.0)
    P = oracle.coarse_kernels(shape, D, liquid, B, lam, R, n_sub)
    ref = c0
    for _ in range(3):
        ref = oracle.coarse_step(shape, liquid, B, R, P, ref)
    with FDiRWCoarse(shape, D, liquid, B, n_sub * lam, R, n_sub, prec) as f:
        cin = torch.from_numpy(c0).to(DEV)
        cout = torch.empty_like(cin)
        m = f.step(cin, cout, 3, want_mass=True)
        got = cout.cpu().numpy()
        host = np.empty_like(c0)
        f.step(c0, host, 3)                       # host pointers, same result
    assert np.array_equal(got, host)
    assert _rel(got, ref) <= FIELD_TOL, _rel(got, ref)
    solid = liquid == 0
    assert np.array_equal(got[solid], c0[solid])
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()


def test_unit_blocks_are_the_fine_windowed_fdirw():
    shape = (14, 13, 12)
    D = synth.random_diffusivity(shape, 82, 4.0)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 83)
    with FDiRWCoarse(shape, D, None, 1, 20 * lam, 3, 20) as f:
        out = np.empty_like(c0)
        f.step(c0, out, 2)
    ref = oracle.superpose(shape, D, lam, 3, 20, oracle.superpose(shape, D, lam, 3, 20, c0))
    assert _rel(out, ref) <= FIELD_TOL


def test_largest_window_matches_oracle():
    """B = 5, R = 8: window radius 10 (21^3), the configuration of the 192^3 coarse leg."""
    shape, B, R, n_sub = (26, 25, 24), 5, 8, 40
    D, liquid = _case(shape, 84)
    lam = oracle.stable_dt_sub(shape, D)
    ref = oracle.coarse_kernels(shape, D, liquid, B, lam, R, n_sub)
    blocks = np.flatnonzero(oracle.coarse_counts(shape, liquid, B))[::4]
    with FDiRWCoarse(shape, D, liquid, B, n_sub * lam, R, n_sub) as f:
        f.kernels()
        got = f.read_coarse(blocks)
    for q, J in enumerate(blocks):
        assert _rel(got[q], ref[J]) <= P_TOL


def test_coarse_argument_errors():
    shape = (10, 10, 10)
    D = np.ones(1000)
    for B, R, prec in ((4, 2, "fp32"), (0, 2, "fp32"), (5, 9, "fp32"), (5, 2, "fp64"), (1, 0, "fp32")):
        with pytest.raises(FdirwError):
            FDiRWCoarse(shape, D, None, B, 0.1, R, 2, prec)
    with FDiRWCoarse(shape, D, None, 5, 0.1, 2, 2) as f:
        with pytest.raises(FdirwError) as e:
            f.read_coarse([0])
        assert e.value.code == fdirw.FDIRW_ERR_STATE
        f.kernels()
        with pytest.raises(FdirwError):
            f.read_kernels([0])
        with pytest.raises(FdirwError):
            f.read_coarse([8])                    # 2 x 2 x 2 blocks


# ------------------------------------------------------------------ far-field boundary (Eq. 7, P_BC c_far)

def test_far_field_matches_oracle():
    shape, B, R, n_sub, V_far, cf0 = (22, 19, 17), 5, 4, 24, 3000.0, 0.4
    D, liquid = _case(shape, 95)
    lam = 0.8 * oracle.stable_dt_sub(shape, D) * 4 / 5
    P = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, n_sub)
    pbc = oracle.coarse_pbc(shape, D, liquid, B, lam, n_sub)
    c0 = synth.random_field(D.size, 96, 0.0, 1.0)
    ref, cf = c0, cf0
    refs = []
    for _ in range(3):
        ref, cf = oracle.coarse_step_far(shape, liquid, B, R, P, pbc, V_far, cf, ref)
        refs.append((ref, cf))
    with FDiRWCoarse(shape, D, liquid, B, n_sub * lam, R, n_sub) as f:
        f.far_field(V_far, cf0)
        f.kernels()
        gotP = f.read_coarse(np.arange(P.shape[0]))
        gotpbc = f.read_pbc()
        out = np.empty_like(c0)
        cur = c0
        for t in range(3):
            f.step(cur, out, 1)
            cur = out.copy()
            assert _rel(cur, refs[t][0]) <= FIELD_TOL
            # c_far moves by the step's mass change over V_far, so its error is the field's mass error / V_far
            assert abs(f.c_far() - refs[t][1]) <= FIELD_TOL * np.abs(refs[t][0]).sum() / V_far
            assert cur.sum() + V_far * f.c_far() == pytest.approx(c0.sum() + V_far * cf0, rel=1e-12)
    cnt = oracle.coarse_counts(shape, liquid, B)
    for J in np.flatnonzero(cnt):
        assert _rel(gotP[J], P[J]) <= P_TOL
    assert _rel(gotpbc, pbc) <= P_TOL
    assert np.array_equal(cur[liquid == 0], c0[liquid == 0])


def test_far_field_errors():
    shape = (10, 10, 10)
    D = np.full((10, 10, 10), 1e-3)
    D[0], D[-1], D[:, 0], D[:, -1], D[:, :, 0], D[:, :, -1] = 1.0, 1.0, 1.0, 1.0, 1.0, 1.0
    D = D.reshape(-1)
    dt = oracle.stable_dt_sub(shape, D)          # closed limit, set by the outer layer's in-layer faces
    with FDiRWCoarse(shape, D, None, 5, dt, 2, 1) as f:
        with pytest.raises(FdirwError) as e:
            f.far_field(100.0, 0.0)              # the open faces of the outer layer push it over
        assert e.value.code == fdirw.FDIRW_ERR_UNSTABLE
    D = np.ones(1000)
    with FDiRWCoarse(shape, D, None, 5, 0.1, 2, 1) as f:
        with pytest.raises(FdirwError):
            f.c_far()
        with pytest.raises(FdirwError):
            f.far_field(0.0, 1.0)


# ------------------------------------------------------------------ coupled macro step (Eqs. 1-7)

def test_coupled_steps_match_oracle():
    shape, B, R, n_sub, V_far = (20, 18, 16), 5, 4, 20, 2000.0
    p = synth.sphere_packing(shape, 0.45, 102, r_range=(1.5, 3.0))
    liquid = (~p.solid).astype(np.uint8)
    D = np.where(liquid > 0, 1.0, 1e-3)                      # effective D_m A_m / RT per phase
    lam = 0.6 * oracle.stable_dt_sub(shape, D)
    dt = n_sub * lam
    kin = dict(k=1e-7, cS_eq=1.0, cL_eq=1e-5)
    P = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, n_sub)
    pbc = oracle.coarse_pbc(shape, D, liquid, B, lam, n_sub)
    c0 = np.where(liquid > 0, 2e-3, 1e-6)
    cf0 = 2e-3
    ref, cf = c0.copy(), cf0
    QLr, QSr = [], []
    for _ in range(3):
        ref, cf = oracle.coupled_step(shape, D, liquid, B, R, P, pbc, V_far, cf, kin["k"], kin["cS_eq"], kin["cL_eq"],
                                      dt, dt / 2 / 1.0, 2, ref)
        QLr.append(ref[liquid > 0].sum())
        QSr.append(ref[liquid == 0].sum())
    with FDiRWCoarse(shape, D, liquid, B, dt, R, n_sub) as f:
        f.far_field(V_far, cf0)
        field = torch.from_numpy(c0).to(DEV)
        QL, QS, c_far = f.coupled_step(field, 3, kin["k"], kin["cS_eq"], kin["cL_eq"], dt, 2)
        got = field.cpu().numpy()
    assert _rel(got, ref) <= FIELD_TOL, _rel(got, ref)
    assert np.allclose(QS, QSr, rtol=FIELD_TOL) and np.allclose(QL, QLr, rtol=FIELD_TOL)
    assert abs(c_far - cf) <= FIELD_TOL * np.abs(ref).sum() / V_far
    total0 = c0.sum() + V_far * cf0
    assert got.sum() + V_far * c_far == pytest.approx(total0, rel=1e-12)
    assert QS[-1] > QS[0] > (liquid == 0).sum() * 1e-6          # the solid keeps absorbing


def test_coupled_exchange_and_solid_march_are_exact():
    """With unit blocks and no substeps the FDiRW part is the identity, so the step is exchange + solid
    march, both FP64 in the oracle's order: bit for bit."""
    shape, B, R = (9, 8, 7), 1, 2
    liquid = np.zeros(504, dtype=np.uint8)
    liquid[::5] = 1
    D = np.where(liquid > 0, 1.0, 0.05)
    dt = 0.4
    c0 = np.where(liquid > 0, 3e-5, 0.3) + synth.random_field(504, 103, 0.0, 1e-6)
    ref = oracle.solid_march(shape, D, liquid, dt / 2, 2, oracle.absorb(shape, liquid, 0.02, 1.0, 1e-5, dt, c0))
    with FDiRWCoarse(shape, D, liquid, B, dt, R, 0) as f:         # B = 1, n_sub = 0: the liquid step is the identity
        f.far_field(100.0, 0.0)
        field = c0.copy()
        f.coupled_step(field, 1, 0.02, 1.0, 1e-5, dt, 2)
    assert np.array_equal(field, ref)


# ------------------------------------------------------------------ convection on the coarse path (Sec. 5)

def _flow(shape, seed, liquid, mean=(0.25, -0.1, 0.05), amp=0.2):
    return synth.face_velocity(shape, seed, mean, amp, liquid == 0)


def test_coarse_flow_matrix_and_steps_match_oracle():
    shape, B, R, n_sub = (23, 21, 19), 5, 3, 24
    D, liquid = _case(shape, 170)
    lam = 0.5 * oracle.stable_dt_sub(shape, D)
    w = _flow(shape, 171, liquid)
    P = oracle.coarse_kernels(shape, D, liquid, B, lam, R, n_sub, w=w)
    c0 = synth.random_field(D.size, 172, 0.0, 2.0)
    ref = c0
    for _ in range(3):
        ref = oracle.coarse_step(shape, liquid, B, R, P, ref)
    with FDiRWCoarse(shape, D, liquid, B, n_sub * lam, R, n_sub) as f:
        f.set_velocity(w)
        f.kernels()
        got = f.read_coarse(np.arange(P.shape[0]))
        out = np.empty_like(c0)
        m = f.step(c0, out, 3, want_mass=True)
    cnt = oracle.coarse_counts(shape, liquid, B)
    for J in np.flatnonzero(cnt):
        assert _rel(got[J], P[J]) <= P_TOL, (J, _rel(got[J], P[J]))
    assert _rel(out, ref) <= FIELD_TOL
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()
    assert np.array_equal(out[liquid == 0], c0[liquid == 0])


def test_coarse_no_flow_is_bitwise_the_diffusion_path():
    shape, B, R, n_sub = (17, 16, 15), 3, 4, 20
    D, liquid = _case(shape, 173)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 174)
    outs = []
    for flow in (False, True):
        with FDiRWCoarse(shape, D, liquid, B, n_sub * lam, R, n_sub) as f:
            f.far_field(1000.0, 0.3)
            if flow:
                f.set_velocity(np.zeros(3 * D.size))
            o = np.empty_like(c0)
            f.step(c0, o, 2)
            outs.append((o, f.read_coarse(np.arange(10)), f.read_pbc(), f.c_far()))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_coarse_flow_far_field_matches_oracle():
    shape, B, R, n_sub, V_far, cf0 = (22, 19, 17), 5, 4, 24, 3000.0, 0.4
    D, liquid = _case(shape, 175)
    lam = 0.4 * oracle.stable_dt_sub(shape, D)
    w = _flow(shape, 176, liquid)
    P = oracle.coarse_kernels_open(shape, D, liquid, B, lam, R, n_sub, w=w)
    pbc = oracle.coarse_pbc(shape, D, liquid, B, lam, n_sub, w=w)
    c0 = synth.random_field(D.size, 177, 0.0, 1.0)
    ref, cf = c0, cf0
    for _ in range(3):
        ref, cf = oracle.coarse_step_far(shape, liquid, B, R, P, pbc, V_far, cf, ref)
    with FDiRWCoarse(shape, D, liquid, B, n_sub * lam, R, n_sub) as f:
        f.far_field(V_far, cf0)
        f.set_velocity(w)
        f.kernels()
        gotP = f.read_coarse(np.arange(P.shape[0]))
        gotpbc = f.read_pbc()
        out = np.empty_like(c0)
        f.step(c0, out, 3)
        cfar = f.c_far()
    for J in np.flatnonzero(oracle.coarse_counts(shape, liquid, B)):
        assert _rel(gotP[J], P[J]) <= P_TOL
    assert _rel(gotpbc, pbc) <= P_TOL
    assert _rel(out, ref) <= FIELD_TOL
    assert abs(cfar - cf) <= FIELD_TOL * np.abs(ref).sum() / V_far
    assert out.sum() + V_far * cfar == pytest.approx(c0.sum() + V_far * cf0, rel=1e-12)


def test_coarse_flow_ordering_and_stability_errors():
    shape = (10, 10, 10)
    D = np.ones(1000)
    with FDiRWCoarse(shape, D, None, 5, 0.05, 2, 1) as f:
        f.set_velocity(np.zeros(3000))
        with pytest.raises(FdirwError) as e:
            f.far_field(100.0, 0.0)                     # the far field must come first
        assert e.value.code == fdirw.FDIRW_ERR_STATE
    with FDiRWCoarse(shape, D, None, 5, 0.1, 2, 1) as f:
        f.far_field(100.0, 0.0)                         # lam sum = 0.1 * (6 + open faces) <= 0.9
        with pytest.raises(FdirwError) as e:
            f.set_velocity(np.full(3000, 2.0))          # the flow pushes a boundary cell's outflow over 1
        assert e.value.code == fdirw.FDIRW_ERR_UNSTABLE
