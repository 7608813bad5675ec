"""Checkpoint and resume (the paper has none): the state of a run is the diffusivity map, the parameters and
the FP64 field c; the kernels are recomputed from D.  A run saved to a file after two macro steps and
resumed in a new context matches the uninterrupted four-step run.  With FP64 and with the float-float
accumulation every step is a function of the field alone, so the match is bit for bit.  The FP32
accumulation restores each step's mass to the FP64 total of its call's input, so a resumed call aims at
the saved field's total, which differs from the original input's by FP64 rounding; the fields then agree
to that rounding."""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_11376_gb300 import FDiRW, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()


@pytest.mark.parametrize("prec,accum", [("fp64", "ff"), ("fp32", "ff"), ("bf16", "ff"), ("bf16", "fp32")])
def test_resume_from_a_saved_field(tmp_path, prec, accum):
    shape, R, n_sub = (24, 18, 16), 3, 40
    p = synth.sphere_packing(shape, 0.4, 171, r_range=(1.5, 3.5))
    D = synth.diffusivity_per_sphere(p)
    lam = oracle.stable_dt_sub(shape, D)
    c0 = synth.random_field(D.size, 172, 0.0, 2.0)

    def context():
        return FDiRW(shape, torch.from_numpy(D).to(DEV), n_sub * lam, R, n_sub, prec, accum=accum)

    cin = torch.from_numpy(c0).to(DEV)
    with context() as f:
        full = torch.empty_like(cin)
        f.step(cin, full, 4)
        half = torch.empty_like(cin)
        f.step(cin, half, 2)
    path = tmp_path / "c_after_2.npy"
    np.save(path, half.cpu().numpy())
    with context() as g:
        saved = torch.from_numpy(np.load(path)).to(DEV)
        resumed = torch.empty_like(saved)
        g.step(saved, resumed, 2)
    a, b = resumed.cpu().numpy(), full.cpu().numpy()
    if accum == "ff":
        assert np.array_equal(a, b)
    else:
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
        assert abs(a.sum() - c0.sum()) <= 1e-13 * c0.sum()
