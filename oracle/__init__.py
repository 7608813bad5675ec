"""FP64 CPU oracle for the windowed FDiRW hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
package.  The product path (``paper_2408_11376_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``fdirw_oracle.c`` (plain C, FP64, no FMA contraction); this module compiles it
with gcc on first use and marshals numpy arrays.  Section/equation citations refer to the paper
(Mao, Hu, Li, "A GPU accelerated mixed-precision FDiRW solver"):

* ``face_conductance``  -- Eq. 1 discretised by finite differences (harmonic-mean face rule: a reading;
  the paper does not state the face rule).
* ``stable_dt_sub``, ``lam_of`` -- largest substep keeping every explicit coefficient non-negative;
  lam = dt_sub / h^2.
* ``source_kernel`` / ``kernels`` -- Sec. 3.1: column s of p is an explicit FD march from a unit point
  source at s; here on the window of radius R, zero flux at window and domain faces, renormalised to
  unit mass in FP64.
* ``superpose``         -- Eq. 8 / Eq. 14: c' = p c.
* ``full_march``        -- the fine-mesh FD solver of Sec. 4.1 over the whole domain (linearity pin).
* ``mass``              -- Eq. 7: total mass.
* ``radius_map`` / ``superpose_rmap`` -- Eq. 8 with a window radius per source (the batched variant's
  radius rule is a reading).
* ``coarse_counts``, ``coarse_kernels``, ``coarse_step`` -- the coarse mesh, Eqs. 10-15.
* ``boundary_conductance``, ``coarse_kernels_open``, ``coarse_pbc``, ``coarse_step_far`` -- the far-field
  boundary: the P_BC c_far term of Eqs. 10 and 14 and the Eq. 7 update of c_far.
* ``absorb``, ``solid_march``, ``coupled_step`` -- the coupled macro step of Sec. 2 (Eqs. 1-7).
* ``source_kernel_adv``, ``superpose_adv``, ``superpose_rmap_adv`` and the ``w=`` forms of the coarse
  functions -- convection (Sec. 5) as upwind faces in the march.

Parity status: every function above is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``
(closed forms, hand-worked cases, invariants, brute force); ``tests/test_oracle_mutants.py`` checks that
those pins fail on plausible mistakes planted in a copy of this package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdirw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, -ffp-contract=off). Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.fo_face_conductance.argtypes = [ctypes.c_int] * 3 + [_D] * 4
            lib.fo_face_conductance.restype = None
            lib.fo_max_face_sum.argtypes = [ctypes.c_int] * 3 + [_D] * 3
            lib.fo_max_face_sum.restype = ctypes.c_double
            lib.fo_source_kernel.argtypes = [ctypes.c_int] * 3 + [_D] * 3 + [ctypes.c_double, ctypes.c_int,
                                                                            ctypes.c_int, ctypes.c_int64, _D, _D]
            lib.fo_source_kernel.restype = ctypes.c_int
            lib.fo_kernels.argtypes = [ctypes.c_int] * 3 + [_D] * 3 + [ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                                      _I64, ctypes.c_int64, _D, _D]
            lib.fo_kernels.restype = ctypes.c_int
            lib.fo_superpose.argtypes = [ctypes.c_int] * 3 + [_D] * 3 + [ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                                        _D, _D]
            lib.fo_superpose.restype = ctypes.c_int
            lib.fo_full_march.argtypes = [ctypes.c_int] * 3 + [_D] * 3 + [ctypes.c_double, ctypes.c_int, _D, _D]
            lib.fo_full_march.restype = ctypes.c_int
            lib.fo_radius_map.argtypes = [ctypes.c_int64, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, _I32]
            lib.fo_radius_map.restype = None
            lib.fo_superpose_rmap.argtypes = [ctypes.c_int] * 3 + [_D] * 3 + [ctypes.c_double, _I32, ctypes.c_int,
                                                                             _D, _D]
            lib.fo_superpose_rmap.restype = ctypes.c_int
            _U8 = ctypes.POINTER(ctypes.c_uint8)
            lib.fo_mask_faces.argtypes = [ctypes.c_int] * 3 + [_U8, _D, _D, _D]
            lib.fo_mask_faces.restype = None
            lib.fo_coarse_counts.argtypes = [ctypes.c_int] * 3 + [_U8, ctypes.c_int, _I64]
            lib.fo_coarse_counts.restype = None
            lib.fo_coarse_kernels.argtypes = [ctypes.c_int] * 3 + [_D] * 3 + [_U8, ctypes.c_int, ctypes.c_double,
                                                                             ctypes.c_int, ctypes.c_int, _D]
            lib.fo_coarse_kernels.restype = ctypes.c_int
            lib.fo_coarse_step.argtypes = [ctypes.c_int] * 3 + [_U8, ctypes.c_int, ctypes.c_int, _D, _D, _D]
            lib.fo_coarse_step.restype = ctypes.c_int
            lib.fo_boundary_conductance.argtypes = [ctypes.c_int] * 3 + [_D, _U8, _D]
            lib.fo_boundary_conductance.restype = None
            lib.fo_coarse_kernels_open.argtypes = [ctypes.c_int] * 3 + [_D] * 4 + [_U8, ctypes.c_int, ctypes.c_double,
                                                                                  ctypes.c_int, ctypes.c_int, _D]
            lib.fo_coarse_kernels_open.restype = ctypes.c_int
            lib.fo_coarse_pbc.argtypes = [ctypes.c_int] * 3 + [_D] * 4 + [_U8, ctypes.c_int, ctypes.c_double,
                                                                         ctypes.c_int, _D]
            lib.fo_coarse_pbc.restype = ctypes.c_int
            lib.fo_superpose_rmap_adv.argtypes = [ctypes.c_int] * 3 + [_D] * 6 + [ctypes.c_double, ctypes.c_double,
                                                                                 _I32, ctypes.c_int, _D, _D]
            lib.fo_superpose_rmap_adv.restype = ctypes.c_int
            lib.fo_coarse_kernels_adv.argtypes = [ctypes.c_int] * 3 + [_D] * 6 + [ctypes.c_double, _U8, ctypes.c_int,
                                                                                 ctypes.c_double, ctypes.c_int,
                                                                                 ctypes.c_int, _D]
            lib.fo_coarse_kernels_adv.restype = ctypes.c_int
            lib.fo_coarse_kernels_open_adv.argtypes = [ctypes.c_int] * 3 + [_D] * 6 + [ctypes.c_double, _D, _U8,
                                                                                      ctypes.c_int, ctypes.c_double,
                                                                                      ctypes.c_int, ctypes.c_int, _D]
            lib.fo_coarse_kernels_open_adv.restype = ctypes.c_int
            lib.fo_coarse_pbc_adv.argtypes = [ctypes.c_int] * 3 + [_D] * 6 + [ctypes.c_double, _D, _U8, ctypes.c_int,
                                                                             ctypes.c_double, ctypes.c_int, _D]
            lib.fo_coarse_pbc_adv.restype = ctypes.c_int
            lib.fo_coarse_step_far.argtypes = [ctypes.c_int] * 3 + [_U8, ctypes.c_int, ctypes.c_int, _D, _D,
                                                                   ctypes.c_double, ctypes.c_double, _D, _D, _D]
            lib.fo_coarse_step_far.restype = ctypes.c_int
            lib.fo_absorb.argtypes = [ctypes.c_int] * 3 + [_U8] + [ctypes.c_double] * 4 + [_D, _D]
            lib.fo_absorb.restype = None
            lib.fo_solid_march.argtypes = [ctypes.c_int] * 3 + [_D, _U8, ctypes.c_double, ctypes.c_int, _D, _D]
            lib.fo_solid_march.restype = ctypes.c_int
            lib.fo_source_kernel_adv.argtypes = [ctypes.c_int] * 3 + [_D] * 6 + [ctypes.c_double, ctypes.c_double,
                                                                                ctypes.c_int, ctypes.c_int,
                                                                                ctypes.c_int64, _D, _D]
            lib.fo_source_kernel_adv.restype = ctypes.c_int
            lib.fo_superpose_adv.argtypes = [ctypes.c_int] * 3 + [_D] * 6 + [ctypes.c_double, ctypes.c_double,
                                                                            ctypes.c_int, ctypes.c_int, _D, _D]
            lib.fo_superpose_adv.restype = ctypes.c_int
            lib.fo_mass.argtypes = [_D, ctypes.c_int64]
            lib.fo_mass.restype = ctypes.c_double
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Conductance:
    """Face conductances of a grid (gx, gy, gz: +x/+y/+z face of each cell).  With a liquid mask, faces
    with a non-liquid cell on either side carry none (the coarse-mesh path)."""

    def __init__(self, shape, D, liquid=None):
        self.shape = tuple(int(v) for v in shape)
        nx, ny, nz = self.shape
        self.D = _f64(D).reshape(-1)
        if self.D.size != nx * ny * nz:
            raise ValueError("D has the wrong size")
        self.gx = np.empty_like(self.D)
        self.gy = np.empty_like(self.D)
        self.gz = np.empty_like(self.D)
        _load().fo_face_conductance(nx, ny, nz, _p(self.D), _p(self.gx), _p(self.gy), _p(self.gz))
        if liquid is not None:
            self.liquid = _u8(liquid, self.D.size)
            _load().fo_mask_faces(nx, ny, nz, _pu8(self.liquid), _p(self.gx), _p(self.gy), _p(self.gz))

    @property
    def args(self):
        nx, ny, nz = self.shape
        return (nx, ny, nz, _p(self.gx), _p(self.gy), _p(self.gz))


def face_conductance(shape, D):
    """(gx, gy, gz) float64 arrays: harmonic-mean conductance of each cell's +x/+y/+z face."""
    g = Conductance(shape, D)
    return g.gx, g.gy, g.gz


def max_face_sum(shape, D) -> float:
    g = Conductance(shape, D)
    return float(_load().fo_max_face_sum(*g.args))


def stable_dt_sub(shape, D, h: float = 1.0) -> float:
    """Largest dt_sub with dt_sub * max_cell(sum of face conductances) / h^2 <= 1."""
    m = max_face_sum(shape, D)
    return float("inf") if m == 0.0 else h * h / m


def lam_of(dt_macro: float, n_sub: int, h: float = 1.0) -> float:
    """lam = dt_sub / h^2 with dt_sub = dt_macro / n_sub."""
    return 0.0 if n_sub == 0 else (dt_macro / n_sub) / (h * h)


def source_kernel(shape, D, lam: float, R: int, n_sub: int, s: int, cond: Conductance | None = None):
    """(kernel, mass_before): kernel is a (2R+1,2R+1,2R+1) array indexed [oz+R, oy+R, ox+R]."""
    g = cond or Conductance(shape, D)
    W1 = 2 * R + 1
    out = np.empty(W1 ** 3, dtype=np.float64)
    m = ctypes.c_double(0.0)
    rc = _load().fo_source_kernel(*g.args, float(lam), int(R), int(n_sub), int(s), _p(out), ctypes.byref(m))
    if rc != 0:
        raise ValueError("fo_source_kernel rejected its arguments")
    return out.reshape(W1, W1, W1), m.value


def kernels(shape, D, lam: float, R: int, n_sub: int, sources, cond: Conductance | None = None):
    """(kernels [n, 2R+1, 2R+1, 2R+1], masses_before [n]) for a list of sources (OpenMP over sources)."""
    g = cond or Conductance(shape, D)
    src = np.ascontiguousarray(sources, dtype=np.int64).reshape(-1)
    W1 = 2 * R + 1
    out = np.empty((src.size, W1, W1, W1), dtype=np.float64)
    masses = np.empty(src.size, dtype=np.float64)
    rc = _load().fo_kernels(*g.args, float(lam), int(R), int(n_sub), src.ctypes.data_as(_I64), src.size,
                            _p(out), _p(masses))
    if rc != 0:
        raise ValueError("fo_kernels rejected its arguments")
    return out, masses


def superpose(shape, D, lam: float, R: int, n_sub: int, c, cond: Conductance | None = None) -> np.ndarray:
    """One macro step c' = p c (Eq. 8) with windowed kernels."""
    g = cond or Conductance(shape, D)
    c = _f64(c).reshape(-1)
    out = np.empty_like(c)
    if _load().fo_superpose(*g.args, float(lam), int(R), int(n_sub), _p(c), _p(out)) != 0:
        raise ValueError("fo_superpose failed")
    return out


def radius_map(D, dt_macro: float, h: float, R_min: int, R_max: int) -> np.ndarray:
    """Per-source window radius clamp(ceil(2 sqrt(2 D dt_macro) / h), R_min, R_max) (int32, FP64 rule)."""
    D = _f64(D).reshape(-1)
    out = np.empty(D.size, dtype=np.int32)
    _load().fo_radius_map(D.size, _p(D), float(dt_macro), float(h), int(R_min), int(R_max),
                          out.ctypes.data_as(_I32))
    return out


def superpose_rmap(shape, D, lam: float, Rmap, n_sub: int, c, cond: Conductance | None = None) -> np.ndarray:
    """One macro step of Eq. 8 where source s uses its own window radius Rmap[s]."""
    g = cond or Conductance(shape, D)
    c = _f64(c).reshape(-1)
    Rm = np.ascontiguousarray(Rmap, dtype=np.int32).reshape(-1)
    if Rm.size != c.size:
        raise ValueError("Rmap has the wrong size")
    out = np.empty_like(c)
    if _load().fo_superpose_rmap(*g.args, float(lam), Rm.ctypes.data_as(_I32), int(n_sub), _p(c), _p(out)) != 0:
        raise ValueError("fo_superpose_rmap failed")
    return out


def superpose_rmap_adv(shape, D, w, lam: float, lama: float, Rmap, n_sub: int, c) -> np.ndarray:
    """superpose_rmap whose kernels include the upwind convection of face velocities w (Sec. 5)."""
    g = Conductance(shape, D)
    wx, wy, wz = (_f64(a).reshape(-1) for a in w)
    c = _f64(c).reshape(-1)
    Rm = np.ascontiguousarray(Rmap, dtype=np.int32).reshape(-1)
    if Rm.size != c.size:
        raise ValueError("Rmap has the wrong size")
    out = np.empty_like(c)
    if _load().fo_superpose_rmap_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lam), float(lama),
                                     Rm.ctypes.data_as(_I32), int(n_sub), _p(c), _p(out)) != 0:
        raise ValueError("fo_superpose_rmap_adv failed")
    return out


def _u8(a, n: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
    if a.size != n:
        raise ValueError("liquid mask has the wrong size")
    return a


def _pu8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def coarse_radius(R: int, B: int) -> int:
    """Block radius of the coarse matrix band: ceil(R / B)."""
    return (R + B - 1) // B


def coarse_counts(shape, liquid, B: int) -> np.ndarray:
    """Liquid cells per B^3 block (int64, block index bx + ncx (by + ncy bz))."""
    nx, ny, nz = shape
    nc = ((nx + B - 1) // B) * ((ny + B - 1) // B) * ((nz + B - 1) // B)
    out = np.empty(nc, dtype=np.int64)
    lq = _u8(liquid, nx * ny * nz)
    _load().fo_coarse_counts(nx, ny, nz, _pu8(lq), int(B), out.ctypes.data_as(_I64))
    return out


def _liquid_velocity(shape, w, liquid):
    """Copies of the face velocities (wx, wy, wz) with the faces that touch a non-liquid cell zeroed (the
    liquid path's reading of Sec. 5: no flux of either kind there)."""
    nx, ny, nz = shape
    out = [np.array(_f64(a).reshape(-1)) for a in w]
    lq = _u8(liquid, out[0].size)
    _load().fo_mask_faces(nx, ny, nz, _pu8(lq), _p(out[0]), _p(out[1]), _p(out[2]))
    return out


def coarse_kernels(shape, D, liquid, B: int, lam: float, R: int, n_sub: int, w=None, lama=None) -> np.ndarray:
    """Coarse matrix P of Eq. 10 in its band layout [n_blocks, Wc, Wc, Wc] (source block J, offsets
    [dz+Rc, dy+Rc, dx+Rc] to the destination block), Wc = 2 ceil(R/B) + 1.  With face velocities w (and
    lama = dt_sub / h, default lam) the block-source march carries the upwind faces (Sec. 5)."""
    nx, ny, nz = shape
    g = Conductance(shape, D, liquid)
    Wc = 2 * coarse_radius(R, B) + 1
    nc = ((nx + B - 1) // B) * ((ny + B - 1) // B) * ((nz + B - 1) // B)
    out = np.empty((nc, Wc, Wc, Wc), dtype=np.float64)
    if w is None:
        rc = _load().fo_coarse_kernels(*g.args, _pu8(g.liquid), int(B), float(lam), int(R), int(n_sub), _p(out))
    else:
        wx, wy, wz = _liquid_velocity(shape, w, g.liquid)
        rc = _load().fo_coarse_kernels_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lam if lama is None else lama),
                                           _pu8(g.liquid), int(B), float(lam), int(R), int(n_sub), _p(out))
    if rc != 0:
        raise ValueError("fo_coarse_kernels rejected its arguments")
    return out


def coarse_step(shape, liquid, B: int, R: int, P_band, c) -> np.ndarray:
    """One coarse-mesh FDiRW step (Eqs. 13-15, no boundary term)."""
    nx, ny, nz = shape
    lq = _u8(liquid, nx * ny * nz)
    c = _f64(c).reshape(-1)
    P = _f64(P_band)
    out = np.empty_like(c)
    if _load().fo_coarse_step(nx, ny, nz, _pu8(lq), int(B), int(R), _p(P), _p(c), _p(out)) != 0:
        raise ValueError("fo_coarse_step failed")
    return out


def boundary_conductance(shape, D, liquid) -> np.ndarray:
    """Open-face conductance of every cell: D_i times its faces on the grid's outer surface (liquid only)."""
    nx, ny, nz = shape
    Dv = _f64(D).reshape(-1)
    lq = _u8(liquid, Dv.size)
    out = np.empty_like(Dv)
    _load().fo_boundary_conductance(nx, ny, nz, _p(Dv), _pu8(lq), _p(out))
    return out


def coarse_kernels_open(shape, D, liquid, B: int, lam: float, R: int, n_sub: int, w=None, lama=None) -> np.ndarray:
    """Coarse matrix with the grid's outer faces open to the far field (no renormalisation); face
    velocities w add the upwind faces inside the grid (the open faces stay diffusive)."""
    nx, ny, nz = shape
    g = Conductance(shape, D, liquid)
    gb = boundary_conductance(shape, D, liquid)
    Wc = 2 * coarse_radius(R, B) + 1
    nc = ((nx + B - 1) // B) * ((ny + B - 1) // B) * ((nz + B - 1) // B)
    out = np.empty((nc, Wc, Wc, Wc), dtype=np.float64)
    if w is None:
        rc = _load().fo_coarse_kernels_open(*g.args, _p(gb), _pu8(g.liquid), int(B), float(lam), int(R), int(n_sub),
                                            _p(out))
    else:
        wx, wy, wz = _liquid_velocity(shape, w, g.liquid)
        rc = _load().fo_coarse_kernels_open_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lam if lama is None else lama),
                                                _p(gb), _pu8(g.liquid), int(B), float(lam), int(R), int(n_sub),
                                                _p(out))
    if rc != 0:
        raise ValueError("fo_coarse_kernels_open rejected its arguments")
    return out


def coarse_pbc(shape, D, liquid, B: int, lam: float, n_sub: int, w=None, lama=None) -> np.ndarray:
    """P_BC of Eq. 10 on the blocks: the liquid marched from 0 with every far-field ghost at 1, mapped;
    face velocities w add the upwind faces inside the grid."""
    nx, ny, nz = shape
    g = Conductance(shape, D, liquid)
    gb = boundary_conductance(shape, D, liquid)
    nc = ((nx + B - 1) // B) * ((ny + B - 1) // B) * ((nz + B - 1) // B)
    out = np.empty(nc, dtype=np.float64)
    if w is None:
        rc = _load().fo_coarse_pbc(*g.args, _p(gb), _pu8(g.liquid), int(B), float(lam), int(n_sub), _p(out))
    else:
        wx, wy, wz = _liquid_velocity(shape, w, g.liquid)
        rc = _load().fo_coarse_pbc_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lam if lama is None else lama), _p(gb),
                                       _pu8(g.liquid), int(B), float(lam), int(n_sub), _p(out))
    if rc != 0:
        raise ValueError("fo_coarse_pbc failed")
    return out


def coarse_step_far(shape, liquid, B: int, R: int, P_band, PBC, V_far: float, c_far: float, c):
    """One coarse step with the far-field term and the Eq. 7 update: returns (c', c_far')."""
    nx, ny, nz = shape
    lq = _u8(liquid, nx * ny * nz)
    c = _f64(c).reshape(-1)
    out = np.empty_like(c)
    cf = ctypes.c_double(0.0)
    if _load().fo_coarse_step_far(nx, ny, nz, _pu8(lq), int(B), int(R), _p(_f64(P_band)), _p(_f64(PBC)),
                                  float(V_far), float(c_far), _p(c), _p(out), ctypes.byref(cf)) != 0:
        raise ValueError("fo_coarse_step_far failed")
    return out, cf.value


def absorb(shape, liquid, k: float, cS_eq: float, cL_eq: float, dt: float, c) -> np.ndarray:
    """Interface exchange of Eqs. 4-6 over one macro step on every liquid/solid face."""
    nx, ny, nz = shape
    lq = _u8(liquid, nx * ny * nz)
    c = _f64(c).reshape(-1)
    out = np.empty_like(c)
    _load().fo_absorb(nx, ny, nz, _pu8(lq), float(k), float(cS_eq), float(cL_eq), float(dt), _p(c), _p(out))
    return out


def solid_march(shape, D, liquid, lam: float, n_sub: int, c) -> np.ndarray:
    """Slow diffusion of the solid phase: explicit flux-form march over solid-solid faces only."""
    nx, ny, nz = shape
    Dv = _f64(D).reshape(-1)
    lq = _u8(liquid, Dv.size)
    c = _f64(c).reshape(-1)
    out = np.empty_like(c)
    if _load().fo_solid_march(nx, ny, nz, _p(Dv), _pu8(lq), float(lam), int(n_sub), _p(c), _p(out)) != 0:
        raise ValueError("fo_solid_march failed")
    return out


def coupled_step(shape, D, liquid, B: int, R: int, P_band, PBC, V_far: float, c_far: float, k: float,
                 cS_eq: float, cL_eq: float, dt: float, lam_s: float, n_sub_s: int, c):
    """One coupled macro step: interface exchange, slow solid march, coarse FDiRW with the far field.
    Returns (c', c_far')."""
    c1 = absorb(shape, liquid, k, cS_eq, cL_eq, dt, c)
    c2 = solid_march(shape, D, liquid, lam_s, n_sub_s, c1)
    return coarse_step_far(shape, liquid, B, R, P_band, PBC, V_far, c_far, c2)


def source_kernel_adv(shape, D, w, lam: float, lama: float, R: int, n_sub: int, s: int):
    """(kernel, mass_before) with convection: w = (wx, wy, wz) face velocities (+a face of each cell),
    lama = dt_sub / h; kernel indexed [oz+R, oy+R, ox+R]."""
    g = Conductance(shape, D)
    wx, wy, wz = (_f64(a).reshape(-1) for a in w)
    W1 = 2 * R + 1
    out = np.empty(W1 ** 3, dtype=np.float64)
    m = ctypes.c_double(0.0)
    if _load().fo_source_kernel_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lam), float(lama), int(R), int(n_sub),
                                    int(s), _p(out), ctypes.byref(m)) != 0:
        raise ValueError("fo_source_kernel_adv rejected its arguments")
    return out.reshape(W1, W1, W1), m.value


def superpose_adv(shape, D, w, lam: float, lama: float, R: int, n_sub: int, c) -> np.ndarray:
    """One macro step of Eq. 8 whose kernels include the upwind convection of face velocities w."""
    g = Conductance(shape, D)
    wx, wy, wz = (_f64(a).reshape(-1) for a in w)
    c = _f64(c).reshape(-1)
    out = np.empty_like(c)
    if _load().fo_superpose_adv(*g.args, _p(wx), _p(wy), _p(wz), float(lam), float(lama), int(R), int(n_sub),
                                _p(c), _p(out)) != 0:
        raise ValueError("fo_superpose_adv failed")
    return out


def full_march(shape, D, lam: float, n_sub: int, c, cond: Conductance | None = None) -> np.ndarray:
    """Brute-force explicit FD march of the whole field over the full domain."""
    g = cond or Conductance(shape, D)
    c = _f64(c).reshape(-1)
    out = np.empty_like(c)
    if _load().fo_full_march(*g.args, float(lam), int(n_sub), _p(c), _p(out)) != 0:
        raise ValueError("fo_full_march failed")
    return out


def mass(c) -> float:
    """Total mass sum(c) (Eq. 7)."""
    c = _f64(c).reshape(-1)
    return float(_load().fo_mass(_p(c), c.size))


def set_threads(n: int) -> None:
    """Sets the OpenMP thread count used by ``kernels`` (via omp_set_num_threads from libgomp)."""
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(int(n))
    except OSError:
        os.environ["OMP_NUM_THREADS"] = str(int(n))
