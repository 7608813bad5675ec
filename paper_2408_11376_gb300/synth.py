"""Seeded synthetic inputs for FDiRW workloads.

The paper runs on phase-field porous particles (Sec. 2, Fig. 1) that are not available; seeded
overlapping-sphere packings with the paper's diffusivity contrast of 3 to 8 decades (Sec. 1) stand in
for them.  This module only *makes inputs* -- a solid/pore mask, a cell diffusivity map D and an
initial concentration field -- and holds none of the method's arithmetic (no face conductances, no
finite-difference march, no superposition).  Both the CUDA path and the CPU oracle consume what it
returns; neither is imported here.

Layout: every field is a flat float64 array of N = nx*ny*nz cells, x fastest
(index i = x + nx*(y + ny*z)), i.e. a C-order numpy array of shape (nz, ny, nx) flattened.

Random numbers come from one splitmix64 stream per structure (Steele, Lea & Flood 2014, the
published 64-bit mixing constants), drawn in a fixed order, five per sphere:
centre x, centre y, centre z (each U[0, n)), radius U[r_lo, r_hi], log10 diffusivity ratio U[lo, hi]
(the fifth draw is taken even when the workload does not use it, so the geometry of a seed does not
depend on the diffusivity recipe).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator: state += golden gamma; output = two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """53-bit uniform double in [lo, hi)."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (2.0 ** -53))


@dataclasses.dataclass
class Packing:
    """A porous microstructure: solid grains (overlapping spheres) in a pore space."""
    shape: tuple            # (nx, ny, nz)
    solid: np.ndarray       # bool, flat, x fastest
    log10_ratio: np.ndarray  # float64, flat: per-cell max over covering spheres of their drawn ratio (0 in pore)
    n_spheres: int

    @property
    def porosity(self) -> float:
        return 1.0 - float(self.solid.mean())


def sphere_packing(shape, porosity: float, seed: int, r_range=(2.0, 5.0), ratio_range=(3.0, 8.0),
                   max_spheres: int | None = None) -> Packing:
    """Overlapping spheres added one at a time until the solid fraction reaches 1 - porosity.

    A cell with integer centre (x, y, z) is solid when it lies within radius r of some sphere centre
    (distance <= r); spheres are not periodic.  For each solid cell the largest log10 ratio of the
    spheres covering it is kept (overlap takes the smallest diffusivity, an order-free rule).
    """
    nx, ny, nz = (int(v) for v in shape)
    n = nx * ny * nz
    if not (0.0 <= porosity <= 1.0):
        raise ValueError("porosity must be in [0, 1]")
    rng = SplitMix64(seed)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    ratio = np.zeros((nz, ny, nx), dtype=np.float64)
    target = (1.0 - porosity) * n
    count = 0
    k = 0
    cap = max_spheres if max_spheres is not None else 50 * n + 1000
    zs = np.arange(nz, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    xs = np.arange(nx, dtype=np.float64)
    while count < target:
        if k >= cap:
            raise RuntimeError("sphere packing did not reach the requested solid fraction")
        cx = rng.uniform(0.0, nx)
        cy = rng.uniform(0.0, ny)
        cz = rng.uniform(0.0, nz)
        r = rng.uniform(*r_range)
        u = rng.uniform(*ratio_range)
        k += 1
        x0, x1 = max(0, math.ceil(cx - r)), min(nx - 1, math.floor(cx + r))
        y0, y1 = max(0, math.ceil(cy - r)), min(ny - 1, math.floor(cy + r))
        z0, z1 = max(0, math.ceil(cz - r)), min(nz - 1, math.floor(cz + r))
        if x0 > x1 or y0 > y1 or z0 > z1:
            continue
        dz2 = (zs[z0:z1 + 1] - cz) ** 2
        dy2 = (ys[y0:y1 + 1] - cy) ** 2
        dx2 = (xs[x0:x1 + 1] - cx) ** 2
        inside = (dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :]) <= r * r
        box = (slice(z0, z1 + 1), slice(y0, y1 + 1), slice(x0, x1 + 1))
        sub = solid[box]
        count += int(np.count_nonzero(inside & ~sub))
        sub |= inside
        rsub = ratio[box]
        np.maximum(rsub, np.where(inside, u, 0.0), out=rsub)
    return Packing((nx, ny, nz), solid.reshape(-1), ratio.reshape(-1), k)


def diffusivity_two_phase(p: Packing, d_pore: float = 1.0, d_solid: float = 1e-5) -> np.ndarray:
    """D = d_pore in pore cells and d_solid in solid cells."""
    return np.where(p.solid, d_solid, d_pore).astype(np.float64)


def diffusivity_per_sphere(p: Packing, d_pore: float = 1.0) -> np.ndarray:
    """D = d_pore in pore; in solid D = d_pore * 10**(-u) with u the cell's drawn log10 ratio."""
    return np.where(p.solid, d_pore * np.power(10.0, -p.log10_ratio), d_pore).astype(np.float64)


def field_solid_one(p: Packing) -> np.ndarray:
    """c = 1 in solid cells, 0 in pore cells."""
    return p.solid.astype(np.float64)


def field_blob(p: Packing, sigma: float = 10.0) -> np.ndarray:
    """c = exp(-r^2 / (2 sigma^2)) on solid cells, r measured from the domain centre; 0 in pore."""
    nx, ny, nz = p.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - (nx - 1) / 2.0) ** 2 + (y - (ny - 1) / 2.0) ** 2 + (z - (nz - 1) / 2.0) ** 2
    c = np.exp(-r2 / (2.0 * sigma * sigma)).reshape(-1)
    return np.where(p.solid, c, 0.0)


def random_field(n: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """A seeded uniform field (for linearity and parity cases)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n)


def random_diffusivity(shape, seed: int, decades: float = 6.0, d_max: float = 1.0) -> np.ndarray:
    """Independent per-cell log-uniform D in [d_max * 10**-decades, d_max] (a rough, unstructured map)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return d_max * np.power(10.0, -rng.uniform(0.0, decades, size=nx * ny * nz))


def face_velocity(shape, seed: int, mean=(0.0, 0.0, 0.0), amp: float = 0.0, solid=None) -> np.ndarray:
    """A seeded steady face-velocity field, (3, n): a uniform mean flow plus independent uniform noise in
    [-amp, amp] on every face, w[a, i] through the +a face of cell i; zero on faces touching a solid cell
    when a solid mask is given (the flow runs in the pore space)."""
    nx, ny, nz = shape
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    w = np.asarray(mean, dtype=np.float64)[:, None] + rng.uniform(-amp, amp, size=(3, n))
    if solid is not None:
        sol = np.asarray(solid, dtype=bool).reshape(nz, ny, nx)
        for a, axis in enumerate((2, 1, 0)):
            touch = sol | np.roll(sol, -1, axis=axis)        # cell i or its +a neighbour is solid
            w[a][touch.reshape(-1)] = 0.0
    return w


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic FDiRW workload: geometry, diffusivity recipe, method parameters, initial field."""
    name: str
    n: int                  # cube side (cells)
    porosity: float
    d_mode: str             # "two_phase" or "per_sphere"
    d_solid: float          # two_phase only
    R: int                  # window radius (window (2R+1)^3)
    n_sub: int              # explicit substeps per macro step (at the stability limit)
    steps: int              # macro steps
    field: str              # "solid_one" or "blob"
    seed: int

    def make(self):
        """Returns (packing, D, c0)."""
        p = sphere_packing((self.n,) * 3, self.porosity, self.seed)
        if self.d_mode == "two_phase":
            d = diffusivity_two_phase(p, 1.0, self.d_solid)
        elif self.d_mode == "per_sphere":
            d = diffusivity_per_sphere(p, 1.0)
        else:
            raise ValueError(self.d_mode)
        c0 = field_solid_one(p) if self.field == "solid_one" else field_blob(p, 10.0)
        return p, d, c0


_S0 = 20240821
WORKLOADS = {
    # 32^3, porosity 0.4, D 1 / 1e-5, R=3, n_sub=50 at the stability limit, 2 steps, c = 1 in solid.
    "fdirw-32c-r3": Workload("fdirw-32c-r3", 32, 0.40, "two_phase", 1e-5, 3, 50, 2, "solid_one", _S0 + 0),
    # 96^3, porosity 0.35, per-sphere log10 ratio U[3,8], R=6, n_sub=120, 10 steps, Gaussian blob sigma=10.
    "fdirw-96c-r6": Workload("fdirw-96c-r6", 96, 0.35, "per_sphere", 0.0, 6, 120, 10, "blob", _S0 + 1),
    # 192^3, porosity 0.4, D 1 / 1e-6, R=8, n_sub=200, 20 steps, c = 1 in solid.
    "fdirw-192c-r8": Workload("fdirw-192c-r8", 192, 0.40, "two_phase", 1e-6, 8, 200, 20, "solid_one", _S0 + 2),
    # 256^3 with the 192^3 recipe (the surrogate's second size).
    "fdirw-256c-r8": Workload("fdirw-256c-r8", 256, 0.40, "two_phase", 1e-6, 8, 200, 20, "solid_one", _S0 + 5),
    # 64^3 with the 192^3 recipe: small profiling case of the same kernels.
    "fdirw-64c-r8": Workload("fdirw-64c-r8", 64, 0.40, "two_phase", 1e-6, 8, 200, 2, "solid_one", _S0 + 6),
}


@dataclasses.dataclass
class BatchWorkload:
    """Many independent structures with per-source window radii: cube sides drawn uniformly from
    `sides`, porosity from U[porosity_range], per-sphere log10 D ratio U[3, 8] (pore D = 1), c = 1 in
    solid; the radius rule clamps to [R_min, R_max]; dt_macro = n_sub * (smallest stable substep)."""
    name: str
    n_struct: int
    sides: tuple
    porosity_range: tuple
    R_min: int
    R_max: int
    n_sub: int
    steps: int
    seed: int

    def layout(self):
        """[(side, porosity, structure seed)] for every structure (cheap: no geometry)."""
        rng = SplitMix64(self.seed)
        out = []
        for i in range(self.n_struct):
            side = self.sides[min(int(rng.uniform(0.0, len(self.sides))), len(self.sides) - 1)]
            por = rng.uniform(*self.porosity_range)
            out.append((side, por, self.seed * 1000 + i))
        return out

    def make(self):
        """Returns (shapes, Ds, c0s): one entry per structure."""
        shapes, Ds, cs = [], [], []
        for side, por, s in self.layout():
            p = sphere_packing((side,) * 3, por, s)
            shapes.append((side,) * 3)
            Ds.append(diffusivity_per_sphere(p, 1.0))
            cs.append(field_solid_one(p))
        return shapes, Ds, cs


BATCH_WORKLOADS = {
    # 64 structures, sides 32..128 step 16, porosity U[0.35, 0.4], radius 3..10 by the rule, n_sub = 75
    # at the stability limit (pore R = 10, solid R = 3), 10 macro steps.
    "fdirw-batch64-r3to10": BatchWorkload("fdirw-batch64-r3to10", 64, (32, 48, 64, 80, 96, 112, 128), (0.35, 0.40),
                                          3, 10, 75, 10, _S0 + 3),
    # Two 48^3 structures of the same recipe, one macro step: small profiling case of the batched kernels.
    "fdirw-batch2x48c-r3to10": BatchWorkload("fdirw-batch2x48c-r3to10", 2, (48,), (0.35, 0.40), 3, 10, 75, 1, _S0 + 4),
}
