"""GPU parity of the batched, per-source-radius path (fdirw_create_batch) against the FP64 oracle:
the radius map bit for bit, sampled kernels element by element, macro steps element by element per
structure, chunked execution against single-chunk execution bit for bit, and the one-structure,
one-radius batch against the uniform-window context bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_11376_gb300 import FDiRW, FDiRWBatch, FdirwError, fdirw, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FIELD_TOL = {"fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-3}
KERNEL_TOL = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 8e-3}


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()


def _structures(seed, shapes, porosity=0.38):
    Ds, cs = [], []
    for i, shape in enumerate(shapes):
        p = synth.sphere_packing(shape, porosity, seed + i, r_range=(1.5, 3.5))
        Ds.append(synth.diffusivity_per_sphere(p))
        cs.append(synth.random_field(int(np.prod(shape)), seed + 100 + i, 0.0, 2.0))
    return Ds, cs


def _dt_sub(shapes, Ds, hs):
    return min(oracle.stable_dt_sub(s, D, h) for s, D, h in zip(shapes, Ds, hs))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SHAPES = [(17, 13, 11), (24, 9, 10), (12, 16, 14)]
HS = [1.0, 1.0, 0.9]


def _batch_case(n_sub=24, R_min=2, R_max=6, seed=300):
    Ds, cs = _structures(seed, SHAPES)
    dt_macro = n_sub * _dt_sub(SHAPES, Ds, HS)
    return Ds, cs, dt_macro


def test_radius_map_matches_oracle_bitwise():
    Ds, _, dt = _batch_case()
    with FDiRWBatch(SHAPES, [torch.from_numpy(D).to(DEV) for D in Ds], dt, 2, 6, 24, "fp32", hs=HS) as b:
        got = b.radius()
    ref = np.concatenate([oracle.radius_map(D, dt, h, 2, 6) for D, h in zip(Ds, HS)])
    assert np.array_equal(got, ref)
    assert len(np.unique(ref)) >= 2


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_kernels_match_oracle(prec):
    Ds, _, dt = _batch_case()
    n_sub = 24
    with FDiRWBatch(SHAPES, Ds, dt, 2, 6, n_sub, prec, hs=HS) as b:
        b.kernels()
        info = b.info()
        assert info["n_structures"] == 3 and info["n_chunks"] == 1 and info["kernels_ready"] == 1
        Rmap = b.radius()
        src = np.arange(5, b.n, 11)
        ks = b.read_kernels(src)
    Rm = 6
    for q, s in enumerate(src):
        i = int(np.searchsorted(b.offsets, s, side="right") - 1)
        ls = int(s - b.offsets[i])
        r = int(Rmap[s])
        lam = (dt / n_sub) / (HS[i] * HS[i])
        ref, _ = oracle.source_kernel(SHAPES[i], Ds[i], lam, r, n_sub, ls)
        got = ks[q][Rm - r:Rm + r + 1, Rm - r:Rm + r + 1, Rm - r:Rm + r + 1]
        assert _rel(got, ref) <= KERNEL_TOL[prec], (s, r)
        assert abs(ks[q].sum() - 1.0) <= 1e-12 and ks[q].min() >= 0.0
        outside = ks[q].copy()
        outside[Rm - r:Rm + r + 1, Rm - r:Rm + r + 1, Rm - r:Rm + r + 1] = 0.0
        assert not outside.any()


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_batch_steps_match_oracle(prec):
    Ds, cs, dt = _batch_case()
    n_sub = 24
    c0 = np.concatenate(cs)
    with FDiRWBatch(SHAPES, Ds, dt, 2, 6, n_sub, prec, hs=HS) as b:
        cin = torch.from_numpy(c0).to(DEV)
        cout = torch.empty_like(cin)
        m = b.step(cin, cout, 2, want_mass=True)
        got = cout.cpu().numpy()
        Rmap = b.radius()
        assert b.info()["graph_launches"] == 1
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()
    for i, shape in enumerate(SHAPES):
        sl = slice(int(b.offsets[i]), int(b.offsets[i + 1]))
        lam = (dt / n_sub) / (HS[i] * HS[i])
        ref = cs[i]
        for _ in range(2):
            ref = oracle.superpose_rmap(shape, Ds[i], lam, Rmap[sl], n_sub, ref)
        assert _rel(got[sl], ref) <= FIELD_TOL[prec], (prec, i, _rel(got[sl], ref))


def test_chunked_equals_resident_bitwise_and_graph_replays():
    Ds, cs, dt = _batch_case(seed=310)
    c0 = torch.from_numpy(np.concatenate(cs)).to(DEV)
    with FDiRWBatch(SHAPES, Ds, dt, 2, 6, 24, "bf16", hs=HS) as b:
        one = torch.empty_like(c0)
        b.step(c0, one, 3)
        one2 = torch.empty_like(c0)
        b.step(c0, one2, 3)                       # same arguments: the captured graph is replayed
        info1 = b.info()
    assert torch.equal(one, one2)
    assert info1["n_chunks"] == 1 and info1["graph_launches"] == 2
    # A memory cap that holds the fixed buffers but only part of the kernels forces several chunks.
    limit = info1["device_bytes"] - info1["cache_bytes"] + info1["cache_bytes"] // 2
    with FDiRWBatch(SHAPES, Ds, dt, 2, 6, 24, "bf16", hs=HS, mem_limit=limit) as b:
        many = torch.empty_like(c0)
        m = b.step(c0, many, 3, want_mass=True)
        info2 = b.info()
        with pytest.raises(FdirwError) as e:
            b.read_kernels([0])
        assert e.value.code == fdirw.FDIRW_ERR_STATE
    assert info2["n_chunks"] >= 2
    assert torch.equal(one, many)
    assert abs(m - float(c0.sum())) <= 1e-12 * float(c0.sum())


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_layouts_match_oracle(prec):
    """Log-uniform D gives radii 1..6 with one common radius (destination-indexed cache) and several rare
    ones (source-indexed cache); fields, sampled kernels and chunked execution against the oracle."""
    shapes = [(16, 12, 10), (11, 14, 9)]
    Ds = [synth.random_diffusivity(s, 340 + i, 4.0) for i, s in enumerate(shapes)]
    n_sub = 20
    dt = n_sub * min(oracle.stable_dt_sub(s, D) for s, D in zip(shapes, Ds))
    c0 = np.concatenate([synth.random_field(int(np.prod(s)), 350 + i) for i, s in enumerate(shapes)])
    with FDiRWBatch(shapes, Ds, dt, 1, 6, n_sub, prec) as b:
        out = np.empty_like(c0)
        m = b.step(c0, out, 2, want_mass=True)
        Rmap = b.radius()
        info = b.info()
        src = np.arange(2, b.n, 9)
        ks = b.read_kernels(src)
    present = set(int(r) for r in np.unique(Rmap))
    dest = {r for r in present if (info["dest_indexed_radii"] >> r) & 1}
    assert dest and (present - dest), (present, dest)        # both cache layouts in use
    assert abs(m - c0.sum()) <= 1e-12 * c0.sum()
    offs = b.offsets
    for i, shape in enumerate(shapes):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        ref = c0[sl]
        for _ in range(2):
            ref = oracle.superpose_rmap(shape, Ds[i], dt / n_sub, Rmap[sl], n_sub, ref)
        assert _rel(out[sl], ref) <= FIELD_TOL[prec], (prec, i, _rel(out[sl], ref))
    for q, s in enumerate(src):
        i = int(np.searchsorted(offs, s, side="right") - 1)
        r = int(Rmap[s])
        ref, _ = oracle.source_kernel(shapes[i], Ds[i], dt / n_sub, r, n_sub, int(s - offs[i]))
        got = ks[q][6 - r:7 + r, 6 - r:7 + r, 6 - r:7 + r]
        assert _rel(got, ref) <= KERNEL_TOL[prec], (s, r)
    limit = info["device_bytes"] - info["cache_bytes"] + info["cache_bytes"] * 2 // 3
    with FDiRWBatch(shapes, Ds, dt, 1, 6, n_sub, prec, mem_limit=limit) as b:
        out2 = np.empty_like(c0)
        b.step(c0, out2, 2)
        assert b.info()["n_chunks"] == 2
    assert np.array_equal(out, out2)


@pytest.mark.parametrize("R", [3, 9])
def test_single_structure_single_radius_equals_uniform_bitwise(R):
    shape = (20, 14, 12)
    p = synth.sphere_packing(shape, 0.4, 320, r_range=(1.5, 3.0))
    D = synth.diffusivity_two_phase(p, 1.0, 1e-5)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = torch.from_numpy(synth.random_field(D.size, 321)).to(DEV)
    src = np.arange(0, D.size, 13)
    with FDiRW(shape, D, 30 * lam, R, 30, "fp32") as u:
        a = torch.empty_like(c0)
        u.step(c0, a, 2)
        ka = u.read_kernels(src)
        parts = u.info()["march_parts"]
    with FDiRWBatch([shape], [D], 30 * lam, R, R, 30, "fp32", march_parts=parts) as b:
        b_out = torch.empty_like(c0)
        b.step(c0, b_out, 2)
        kb = b.read_kernels(src)
    assert np.array_equal(ka, kb)
    assert torch.equal(a, b_out)


def test_zero_radius_sources_and_identity_cases():
    """R_min = 0: cells with D = 0 keep their own mass (identity kernel) next to marched sources."""
    shape = (14, 12, 10)
    D = synth.random_diffusivity(shape, 330, 3.0)
    D[::7] = 0.0
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 331)
    with FDiRWBatch([shape], [D], 10 * lam, 0, 4, 10, "fp32") as b:
        out = np.empty_like(c0)
        b.step(c0, out, 1)                        # host pointers in and out
        Rmap = b.radius()
    assert (Rmap[::7] == 0).all() and Rmap.max() >= 2
    ref = oracle.superpose_rmap(shape, D, lam, Rmap, 10, c0)
    assert _rel(out, ref) <= FIELD_TOL["fp32"]
    for R_max, n_sub in ((0, 10), (4, 0)):        # every kernel is the identity
        with FDiRWBatch([shape], [D], 10 * lam, 0, R_max, n_sub, "bf16") as b:
            out = np.empty_like(c0)
            b.step(c0, out, 2)
        assert np.array_equal(out, c0)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fp32_accum_batch_matches_oracle_and_keeps_every_structure_mass(prec):
    """FDIRW_ACCUM_FP32 on a batch mixing both cache layouts: fields per structure against the oracle,
    every structure's total restored to its input's, and chunked execution bit for bit the resident one."""
    shapes = [(16, 12, 10), (11, 14, 9), (24, 16, 8)]
    Ds = [synth.random_diffusivity(s, 360 + i, 4.0) for i, s in enumerate(shapes)]
    n_sub = 20
    dt = n_sub * min(oracle.stable_dt_sub(s, D) for s, D in zip(shapes, Ds))
    c0 = np.concatenate([synth.random_field(int(np.prod(s)), 370 + i, 0.0, 2.0) for i, s in enumerate(shapes)])
    with FDiRWBatch(shapes, Ds, dt, 1, 6, n_sub, prec, accum="fp32") as b:
        out = np.empty_like(c0)
        b.step(c0, out, 3)
        Rmap = b.radius()
        info = b.info()
        offs = b.offsets
    assert info["accum"] == fdirw.FDIRW_ACCUM_FP32
    present = set(int(r) for r in np.unique(Rmap))
    dest = {r for r in present if (info["dest_indexed_radii"] >> r) & 1}
    assert dest and (present - dest)
    for i, shape in enumerate(shapes):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        ref = c0[sl]
        for _ in range(3):
            ref = oracle.superpose_rmap(shape, Ds[i], dt / n_sub, Rmap[sl], n_sub, ref)
        assert _rel(out[sl], ref) <= FIELD_TOL[prec], (prec, i, _rel(out[sl], ref))
        assert abs(out[sl].sum() - c0[sl].sum()) <= 1e-13 * c0[sl].sum()
    limit = info["device_bytes"] - info["cache_bytes"] + info["cache_bytes"] * 2 // 3
    with FDiRWBatch(shapes, Ds, dt, 1, 6, n_sub, prec, mem_limit=limit, accum="fp32") as b:
        out2 = np.empty_like(c0)
        b.step(c0, out2, 3)
        assert b.info()["n_chunks"] >= 2
    assert np.array_equal(out, out2)


@pytest.mark.parametrize("accum", ["ff", "fp32"])
def test_batch_flow_matches_oracle(accum):
    """Convection on a batch mixing both cache layouts: each structure's field after two macro steps
    against the oracle's per-source-radius upwind superposition, chunked execution bit for bit the
    resident one, and w = 0 bit for bit the diffusion-only batch."""
    shapes = [(16, 12, 10), (11, 14, 9), (24, 16, 8)]
    Ds = [synth.random_diffusivity(s, 380 + i, 4.0) for i, s in enumerate(shapes)]
    n_sub = 30
    dt = n_sub * 0.6 * min(oracle.stable_dt_sub(s, D) for s, D in zip(shapes, Ds))
    ws = [synth.face_velocity(s, 390 + i, (0.2, -0.1, 0.05), 0.15) for i, s in enumerate(shapes)]
    w_all = np.concatenate([w for w in ws], axis=1)          # (3, total): structure i at its offset
    c0 = np.concatenate([synth.random_field(int(np.prod(s)), 400 + i) for i, s in enumerate(shapes)])
    with FDiRWBatch(shapes, Ds, dt, 1, 6, n_sub, "fp32", accum=accum) as b:
        b.set_velocity(w_all)
        out = np.empty_like(c0)
        b.step(c0, out, 2)
        Rmap = b.radius()
        info = b.info()
        offs = b.offsets
    for i, shape in enumerate(shapes):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        lam = dt / n_sub
        ref = c0[sl]
        for _ in range(2):
            ref = oracle.superpose_rmap_adv(shape, Ds[i], ws[i], lam, lam, Rmap[sl], n_sub, ref)
        assert _rel(out[sl], ref) <= FIELD_TOL["fp32"], (i, _rel(out[sl], ref))
        assert abs(out[sl].sum() - c0[sl].sum()) <= 1e-12 * c0[sl].sum()
    limit = info["device_bytes"] - info["cache_bytes"] + info["cache_bytes"] * 2 // 3
    with FDiRWBatch(shapes, Ds, dt, 1, 6, n_sub, "fp32", mem_limit=limit, accum=accum) as b:
        b.set_velocity(w_all)
        out2 = np.empty_like(c0)
        b.step(c0, out2, 2)
        assert b.info()["n_chunks"] >= 2
    assert np.array_equal(out, out2)
    outs = []
    for flow in (False, True):
        with FDiRWBatch(shapes, Ds, dt, 1, 6, n_sub, "bf16", accum=accum) as b:
            o = np.empty_like(c0)
            b.step(c0, o, 1)                                  # builds and captures without a velocity
            if flow:
                b.set_velocity(np.zeros_like(w_all))          # drops the graph; the kernels are rebuilt
                b.step(c0, o, 1)
            outs.append(o)
    assert np.array_equal(outs[0], outs[1])


def test_batch_argument_errors():
    shape = (8, 8, 8)
    D = np.ones(512)
    with pytest.raises(FdirwError):
        FDiRWBatch([shape], [D], 0.1, 3, 11, 2, "fp32")          # R_max > 10
    with pytest.raises(FdirwError):
        FDiRWBatch([shape], [D], 0.1, 4, 3, 2, "fp32")           # R_min > R_max
    with pytest.raises(FdirwError):
        FDiRWBatch([shape], [D], 0.1, 1, 3, 2, "fp64")           # FP64 march has no batch path
    with pytest.raises(FdirwError) as e:
        FDiRWBatch([shape], [D], 10.0, 1, 3, 2, "fp32")          # dt_sub = 5 > 1/6
    assert e.value.code == fdirw.FDIRW_ERR_UNSTABLE
    with pytest.raises(FdirwError) as e:
        FDiRWBatch([shape], [D], 0.1, 8, 8, 2, "fp32", mem_limit=600_000)
    assert e.value.code == fdirw.FDIRW_ERR_NOMEM
    bad = D.copy()
    bad[3] = -1.0
    with pytest.raises(FdirwError):
        FDiRWBatch([shape, shape], [D, bad], 0.1, 1, 3, 2, "fp32")


def test_batch_workload_full_size():
    """The benchmark's batched workload at full size (64 structures, 5.4e7 cells, chunked): one macro step,
    the mass budget, and three structures checked against single-structure contexts bit for bit and, for
    sampled sources of every radius, against the oracle's kernels."""
    bw = synth.BATCH_WORKLOADS["fdirw-batch64-r3to10"]
    shapes, Ds, cs = bw.make()
    dt = bw.n_sub * min(oracle.stable_dt_sub(s, D) for s, D in zip(shapes, Ds))
    c0 = torch.from_numpy(np.concatenate(cs)).to(DEV)
    with FDiRWBatch(shapes, [torch.from_numpy(D).to(DEV) for D in Ds], dt, bw.R_min, bw.R_max, bw.n_sub, "bf16") as b:
        out = torch.empty_like(c0)
        m = b.step(c0, out, 1, want_mass=True)
        info = b.info()
        offs = b.offsets
    assert info["n_structures"] == 64 and info["n_chunks"] >= 2
    assert abs(m - float(c0.sum())) <= 1e-12 * float(c0.sum())
    rng = np.random.default_rng(105)
    for i in (0, 31, 63):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        with FDiRWBatch([shapes[i]], [Ds[i]], dt, bw.R_min, bw.R_max, bw.n_sub, "bf16") as one:
            single = torch.empty_like(c0[sl])
            one.step(c0[sl].contiguous(), single, 1)
            Rmap = one.radius()
            src = np.concatenate([rng.choice(np.flatnonzero(Rmap == r), 2, replace=False) for r in np.unique(Rmap)])
            ks = one.read_kernels(src)
        assert torch.equal(out[sl], single)
        lam = dt / bw.n_sub
        for q, s in enumerate(src):
            r = int(Rmap[s])
            ref, _ = oracle.source_kernel(shapes[i], Ds[i], lam, r, bw.n_sub, int(s))
            got = ks[q][10 - r:11 + r, 10 - r:11 + r, 10 - r:11 + r]
            assert _rel(got, ref) <= KERNEL_TOL["bf16"], (i, s, r)
