"""ctypes binding of libfdirw (the C ABI declared in include/fdirw.h): argument marshalling only.

Every step of the FDiRW hot path runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing or cannot be loaded, importing this module's functions raises.

Fields may be numpy arrays (host memory) or torch tensors (host or CUDA); both are passed to the library
as raw pointers and must be contiguous float64 with N = nx*ny*nz elements, x fastest.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

FDIRW_OK = 0
FDIRW_ERR_ARG = -1
FDIRW_ERR_UNSTABLE = -2
FDIRW_ERR_NOMEM = -3
FDIRW_ERR_CUDA = -4
FDIRW_ERR_TIMEOUT = -5
FDIRW_ERR_STATE = -6

FDIRW_FP64 = 0
FDIRW_FP32 = 1
FDIRW_FP32_STORE_FP16 = 2
FDIRW_FP32_STORE_BF16 = 3
PRECISIONS = {"fp64": FDIRW_FP64, "fp32": FDIRW_FP32, "fp16": FDIRW_FP32_STORE_FP16, "bf16": FDIRW_FP32_STORE_BF16}
FDIRW_ACCUM_FF = 0
FDIRW_ACCUM_FP32 = 1
ACCUMS = {"ff": FDIRW_ACCUM_FF, "fp32": FDIRW_ACCUM_FP32}

EXPORTED = ("fdirw_stable_dt", "fdirw_create", "fdirw_kernels", "fdirw_step", "fdirw_mass", "fdirw_read_kernels",
            "fdirw_get_info", "fdirw_destroy", "fdirw_last_error", "fdirw_mass_noalloc", "fdirw_net_create",
            "fdirw_net_params", "fdirw_net_destroy", "fdirw_net_predict", "fdirw_net_gradients", "fdirw_net_train_step",
            "fdirw_kernels_surrogate", "fdirw_create_batch", "fdirw_read_radius", "fdirw_create_coarse",
            "fdirw_read_coarse", "fdirw_coarse_far_field", "fdirw_coarse_get_far_field", "fdirw_read_coarse_pbc",
            "fdirw_coupled_step", "fdirw_set_velocity", "fdirw_net_trace", "fdirw_net_test_wait",
            "fdirw_probe_peaks", "fdirw_net_timing")
NET_NPARAM = 4 * 27 * 16 * 16 + 4 * 16
NET_KV = 17 ** 3

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfdirw.so")


class FdirwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fdirw error {code}: {msg}")
        self.code = code


class fdirw_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("h", ctypes.c_double)]


class fdirw_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("mem_limit", ctypes.c_uint64), ("march_parts", ctypes.c_int32), ("accum", ctypes.c_int32)]


class fdirw_coupled_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("cS_eq", ctypes.c_double), ("cL_eq", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_sub_solid", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fdirw_info(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("window_R", ctypes.c_int32), ("n_sub", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("kernels_ready", ctypes.c_int32), ("dt_sub", ctypes.c_double),
                ("lam", ctypes.c_double), ("max_face_sum", ctypes.c_double), ("cache_bytes", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("window_cells", ctypes.c_double),
                ("kernels_ms", ctypes.c_float), ("last_gather_ms", ctypes.c_float),
                ("last_mass_in", ctypes.c_double), ("last_mass_out", ctypes.c_double),
                ("march_parts", ctypes.c_int32), ("accum", ctypes.c_int32),
                ("n_structures", ctypes.c_int32), ("n_chunks", ctypes.c_int32), ("window_R_min", ctypes.c_int32),
                ("graph_launches", ctypes.c_int32), ("dest_indexed_radii", ctypes.c_int32),
                ("coarse_block", ctypes.c_int32), ("coarse_nodes", ctypes.c_int64),
                ("last_restore_drift", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Loads libfdirw.so (built by ``paper_2408_11376_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libfdirw.so not found at {p}: run paper_2408_11376_gb300.build.build() "
                              "(the CUDA path has no fallback)")
        lib = ctypes.CDLL(p)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.fdirw_stable_dt.argtypes = [ctypes.POINTER(fdirw_grid), vp, i32, dp]
        lib.fdirw_create.argtypes = [ctypes.POINTER(fdirw_grid), vp, ctypes.c_double, i32, i32,
                                     ctypes.POINTER(fdirw_opts), ctypes.POINTER(vp)]
        lib.fdirw_kernels.argtypes = [vp]
        lib.fdirw_step.argtypes = [vp, vp, vp, i32, dp]
        lib.fdirw_mass.argtypes = [vp, vp, dp]
        lib.fdirw_read_kernels.argtypes = [vp, vp, i64, vp]
        lib.fdirw_get_info.argtypes = [vp, ctypes.POINTER(fdirw_info)]
        lib.fdirw_destroy.argtypes = [vp]
        lib.fdirw_destroy.restype = None
        lib.fdirw_last_error.argtypes = [vp]
        lib.fdirw_last_error.restype = ctypes.c_char_p
        lib.fdirw_mass_noalloc.argtypes = [vp, i64, vp, vp]
        lib.fdirw_net_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
        lib.fdirw_net_params.argtypes = [vp, vp]
        lib.fdirw_net_destroy.argtypes = [vp]
        lib.fdirw_net_destroy.restype = None
        lib.fdirw_net_predict.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        lib.fdirw_net_gradients.argtypes = [vp, vp, vp, i64, vp, vp, dp]
        lib.fdirw_net_train_step.argtypes = [vp, vp, vp, i64, vp, ctypes.c_float, dp]
        lib.fdirw_kernels_surrogate.argtypes = [vp, vp, ctypes.POINTER(i64)]
        lib.fdirw_net_trace.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp, dp]
        lib.fdirw_net_test_wait.argtypes = [vp, ctypes.c_uint64, i32]
        lib.fdirw_probe_peaks.argtypes = [i32, dp, dp]
        lib.fdirw_net_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.fdirw_create_batch.argtypes = [i32, ctypes.POINTER(fdirw_grid), ctypes.POINTER(vp), ctypes.c_double, i32,
                                           i32, i32, ctypes.POINTER(fdirw_opts), ctypes.POINTER(vp)]
        lib.fdirw_read_radius.argtypes = [vp, vp]
        lib.fdirw_create_coarse.argtypes = [ctypes.POINTER(fdirw_grid), vp, vp, i32, ctypes.c_double, i32, i32,
                                            ctypes.POINTER(fdirw_opts), ctypes.POINTER(vp)]
        lib.fdirw_read_coarse.argtypes = [vp, vp, i64, vp]
        lib.fdirw_coarse_far_field.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        lib.fdirw_coarse_get_far_field.argtypes = [vp, dp]
        lib.fdirw_read_coarse_pbc.argtypes = [vp, vp]
        lib.fdirw_coupled_step.argtypes = [vp, ctypes.POINTER(fdirw_coupled_params), vp, i32, vp, vp, dp]
        lib.fdirw_set_velocity.argtypes = [vp, vp]
        for name in EXPORTED:
            if name not in ("fdirw_destroy", "fdirw_last_error", "fdirw_net_destroy"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int, ctx=None):
    if rc != FDIRW_OK:
        msg = load().fdirw_last_error(ctx)
        raise FdirwError(rc, msg.decode() if msg else "")


def _ptr(a) -> int:
    """Raw data pointer of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)!r}")


def _check_f64(a, n: int):
    dt = getattr(a, "dtype", None)
    if isinstance(a, np.ndarray):
        ok = a.dtype == np.float64
    else:
        ok = str(dt) == "torch.float64"
    if not ok:
        raise TypeError("fields must be float64")
    size = a.size if isinstance(a, np.ndarray) else a.numel()
    if size != n:
        raise ValueError(f"field has {size} elements, expected {n}")


# --------------------------------------------------------------------------- C-ABI mirrors

def fdirw_stable_dt(shape, D, h: float = 1.0, device: int = -1) -> float:
    lib = load()
    nx, ny, nz = (int(v) for v in shape)
    _check_f64(D, nx * ny * nz)
    g = fdirw_grid(nx, ny, nz, float(h))
    out = ctypes.c_double(0.0)
    _check(lib.fdirw_stable_dt(ctypes.byref(g), ctypes.c_void_p(_ptr(D)), int(device), ctypes.byref(out)))
    return out.value


def fdirw_create(shape, D, dt_macro: float, window_R: int, n_sub: int, prec="fp32", h: float = 1.0,
                 device: int = -1, stream=None, mem_limit: int = 0, march_parts: int = 0, accum="ff") -> int:
    """Returns the context handle (an integer address); release it with fdirw_destroy.  accum: "ff"
    (float-float rows, the default) or "fp32" (FP32 rows with the mass restored every step)."""
    lib = load()
    nx, ny, nz = (int(v) for v in shape)
    _check_f64(D, nx * ny * nz)
    g = fdirw_grid(nx, ny, nz, float(h))
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    st = 0 if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    acc = ACCUMS[accum] if isinstance(accum, str) else int(accum)
    o = fdirw_opts(p, int(device), ctypes.c_void_p(st), int(mem_limit), int(march_parts), acc)
    ctx = ctypes.c_void_p(0)
    _check(lib.fdirw_create(ctypes.byref(g), ctypes.c_void_p(_ptr(D)), float(dt_macro), int(window_R), int(n_sub),
                            ctypes.byref(o), ctypes.byref(ctx)))
    return ctx.value


def fdirw_create_batch(shapes, Ds, dt_macro: float, R_min: int, R_max: int, n_sub: int, prec="fp32", hs=None,
                       device: int = -1, stream=None, mem_limit: int = 0, march_parts: int = 0, accum="ff") -> int:
    """Context for a batch of structures with per-source radii; fields are the concatenation of the
    structures' fields.  Returns the handle; release it with fdirw_destroy."""
    lib = load()
    n = len(shapes)
    if len(Ds) != n:
        raise ValueError("one D map per structure")
    hs = [1.0] * n if hs is None else list(hs)
    grids = (fdirw_grid * n)()
    ptrs = (ctypes.c_void_p * n)()
    for i, (shape, D) in enumerate(zip(shapes, Ds)):
        nx, ny, nz = (int(v) for v in shape)
        _check_f64(D, nx * ny * nz)
        grids[i] = fdirw_grid(nx, ny, nz, float(hs[i]))
        ptrs[i] = _ptr(D)
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    st = 0 if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    acc = ACCUMS[accum] if isinstance(accum, str) else int(accum)
    o = fdirw_opts(p, int(device), ctypes.c_void_p(st), int(mem_limit), int(march_parts), acc)
    ctx = ctypes.c_void_p(0)
    _check(lib.fdirw_create_batch(int(n), grids, ptrs, float(dt_macro), int(R_min), int(R_max), int(n_sub),
                                  ctypes.byref(o), ctypes.byref(ctx)))
    return ctx.value


def fdirw_create_coarse(shape, D, liquid, block: int, dt_macro: float, window_R: int, n_sub: int, prec="fp32",
                        h: float = 1.0, device: int = -1, stream=None, mem_limit: int = 0) -> int:
    """Coarse-mesh context (Eqs. 10-15): liquid = N bytes (nonzero = liquid) or None for all liquid."""
    lib = load()
    nx, ny, nz = (int(v) for v in shape)
    _check_f64(D, nx * ny * nz)
    lq_ptr = None
    if liquid is not None:
        if isinstance(liquid, np.ndarray):
            liquid = np.ascontiguousarray(liquid, dtype=np.uint8).reshape(-1)
        n = liquid.size if isinstance(liquid, np.ndarray) else liquid.numel()
        if n != nx * ny * nz:
            raise ValueError("liquid mask has the wrong size")
        lq_ptr = ctypes.c_void_p(_ptr(liquid))
    g = fdirw_grid(nx, ny, nz, float(h))
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    st = 0 if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    o = fdirw_opts(p, int(device), ctypes.c_void_p(st), int(mem_limit), 0, 0)
    ctx = ctypes.c_void_p(0)
    _check(lib.fdirw_create_coarse(ctypes.byref(g), ctypes.c_void_p(_ptr(D)), lq_ptr, int(block), float(dt_macro),
                                   int(window_R), int(n_sub), ctypes.byref(o), ctypes.byref(ctx)))
    return ctx.value


def fdirw_read_coarse(ctx: int, blocks, Rc: int) -> np.ndarray:
    """Coarse-matrix columns of the listed blocks, [n, Wc, Wc, Wc] indexed [dz+Rc, dy+Rc, dx+Rc]."""
    b = np.ascontiguousarray(blocks, dtype=np.int64).reshape(-1)
    Wc = 2 * int(Rc) + 1
    out = np.empty((b.size, Wc, Wc, Wc), dtype=np.float64)
    _check(load().fdirw_read_coarse(ctypes.c_void_p(ctx), ctypes.c_void_p(b.ctypes.data), b.size,
                                    ctypes.c_void_p(out.ctypes.data)), ctypes.c_void_p(ctx))
    return out


def fdirw_read_radius(ctx: int, n_cells: int) -> np.ndarray:
    """Window radius of every source (int32 [n_cells])."""
    out = np.empty(int(n_cells), dtype=np.int32)
    _check(load().fdirw_read_radius(ctypes.c_void_p(ctx), ctypes.c_void_p(out.ctypes.data)), ctypes.c_void_p(ctx))
    return out


def fdirw_kernels(ctx: int) -> None:
    _check(load().fdirw_kernels(ctypes.c_void_p(ctx)), ctypes.c_void_p(ctx))


def fdirw_step(ctx: int, c_in, c_out, n_steps: int = 1, want_mass: bool = False):
    """Advances c_in by n_steps macro steps into c_out; returns the FP64 total of c_out if want_mass."""
    m = ctypes.c_double(0.0)
    _check(load().fdirw_step(ctypes.c_void_p(ctx), ctypes.c_void_p(_ptr(c_in)), ctypes.c_void_p(_ptr(c_out)),
                             int(n_steps), ctypes.byref(m) if want_mass else None), ctypes.c_void_p(ctx))
    return m.value if want_mass else None


def fdirw_mass(ctx: int, c) -> float:
    m = ctypes.c_double(0.0)
    _check(load().fdirw_mass(ctypes.c_void_p(ctx), ctypes.c_void_p(_ptr(c)), ctypes.byref(m)), ctypes.c_void_p(ctx))
    return m.value


def fdirw_read_kernels(ctx: int, sources, R: int) -> np.ndarray:
    """Renormalised kernels of the given sources, shape [n, 2R+1, 2R+1, 2R+1] indexed [oz+R, oy+R, ox+R]."""
    src = np.ascontiguousarray(sources, dtype=np.int64).reshape(-1)
    W1 = 2 * int(R) + 1
    out = np.empty((src.size, W1, W1, W1), dtype=np.float64)
    _check(load().fdirw_read_kernels(ctypes.c_void_p(ctx), ctypes.c_void_p(src.ctypes.data), src.size,
                                     ctypes.c_void_p(out.ctypes.data)), ctypes.c_void_p(ctx))
    return out


def fdirw_get_info(ctx: int) -> dict:
    info = fdirw_info()
    _check(load().fdirw_get_info(ctypes.c_void_p(ctx), ctypes.byref(info)), ctypes.c_void_p(ctx))
    return info.as_dict()


def fdirw_destroy(ctx: int) -> None:
    if ctx:
        load().fdirw_destroy(ctypes.c_void_p(ctx))


def fdirw_probe_peaks(device: int = -1) -> dict:
    """Measured FP32 FMA rate (flop/s) and streaming HBM read bandwidth (bytes/s) of a GPU."""
    f, r = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().fdirw_probe_peaks(int(device), ctypes.byref(f), ctypes.byref(r)))
    return {"fp32_flops": f.value, "read_bytes_per_s": r.value}


def fdirw_mass_noalloc(c, mass_out, stream=None) -> None:
    """FP64 total of the device field c written into the one-element device tensor mass_out, with no
    allocation inside the library (fixed scratch; fields of up to 2^30 cells).  Asynchronous on stream."""
    n = c.numel() if hasattr(c, "numel") else int(np.asarray(c).size)
    st = 0 if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    _check(load().fdirw_mass_noalloc(ctypes.c_void_p(_ptr(c)), int(n), ctypes.c_void_p(_ptr(mass_out)),
                                     ctypes.c_void_p(st)))


def fdirw_set_velocity(ctx: int, w, n: int) -> None:
    """Face velocities w (3 * n float64, host or device; w[a * n + i] through the +a face of cell i)."""
    if hasattr(w, "data_ptr"):
        if str(w.dtype) != "torch.float64" or w.numel() != 3 * n:
            raise ValueError("w must be a float64 tensor of 3 * n_cells values")
        _check(load().fdirw_set_velocity(ctypes.c_void_p(ctx), ctypes.c_void_p(_ptr(w))), ctx)
        return
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
    if a.size != 3 * n:
        raise ValueError("w must hold 3 * n_cells values")
    _check(load().fdirw_set_velocity(ctypes.c_void_p(ctx), ctypes.c_void_p(a.ctypes.data)), ctx)


def fdirw_last_error(ctx: int | None = None) -> str:
    m = load().fdirw_last_error(ctypes.c_void_p(ctx) if ctx else None)
    return m.decode() if m else ""


# --------------------------------------------------------------------------- convenience owner

class FDiRW:
    """Owns one context: ``FDiRW(shape, D, dt_macro, R, n_sub, prec)``; ``step(c_in, c_out, n)``; ``close()``."""

    def __init__(self, shape, D, dt_macro: float, window_R: int, n_sub: int, prec="fp32", h: float = 1.0,
                 device: int = -1, stream=None, mem_limit: int = 0, march_parts: int = 0, accum="ff"):
        self.shape = tuple(int(v) for v in shape)
        self.R = int(window_R)
        self.n = self.shape[0] * self.shape[1] * self.shape[2]
        self.ctx = fdirw_create(self.shape, D, dt_macro, window_R, n_sub, prec, h, device, stream, mem_limit,
                                march_parts, accum)

    def kernels(self):
        fdirw_kernels(self.ctx)

    def step(self, c_in, c_out, n_steps: int = 1, want_mass: bool = False):
        _check_f64(c_in, self.n)
        _check_f64(c_out, self.n)
        return fdirw_step(self.ctx, c_in, c_out, n_steps, want_mass)

    def mass(self, c) -> float:
        _check_f64(c, self.n)
        return fdirw_mass(self.ctx, c)

    def read_kernels(self, sources) -> np.ndarray:
        return fdirw_read_kernels(self.ctx, sources, self.R)

    def set_velocity(self, w):
        """Steady face velocities (3, n) or (3 * n,) float64, host or device (Sec. 5 convection)."""
        fdirw_set_velocity(self.ctx, w, self.n)

    def info(self) -> dict:
        return fdirw_get_info(self.ctx)

    def close(self):
        if self.ctx:
            fdirw_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FDiRWBatch(FDiRW):
    """Owns one batch context: ``FDiRWBatch(shapes, Ds, dt_macro, R_min, R_max, n_sub, prec)``.  Fields are
    the concatenation of the structures' fields (``offsets[i]`` is structure i's first cell)."""

    def __init__(self, shapes, Ds, dt_macro: float, R_min: int, R_max: int, n_sub: int, prec="fp32", hs=None,
                 device: int = -1, stream=None, mem_limit: int = 0, march_parts: int = 0, accum="ff"):
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        sizes = [a * b * c for a, b, c in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        self.R = int(R_max)
        self.ctx = fdirw_create_batch(self.shapes, Ds, dt_macro, R_min, R_max, n_sub, prec, hs, device, stream,
                                      mem_limit, march_parts, accum)

    def radius(self) -> np.ndarray:
        return fdirw_read_radius(self.ctx, self.n)


class FDiRWCoarse(FDiRW):
    """Owns one coarse-mesh context: ``FDiRWCoarse(shape, D, liquid, block, dt_macro, R, n_sub)``."""

    def __init__(self, shape, D, liquid, block: int, dt_macro: float, window_R: int, n_sub: int, prec="fp32",
                 h: float = 1.0, device: int = -1, stream=None, mem_limit: int = 0):
        self.shape = tuple(int(v) for v in shape)
        self.n = self.shape[0] * self.shape[1] * self.shape[2]
        self.R = int(window_R)
        self.B = int(block)
        self.ctx = fdirw_create_coarse(self.shape, D, liquid, block, dt_macro, window_R, n_sub, prec, h, device,
                                       stream, mem_limit)
        self.Rc = (self.R + self.B - 1) // self.B        # block >= 1 once the library accepted it

    def read_coarse(self, blocks) -> np.ndarray:
        return fdirw_read_coarse(self.ctx, blocks, self.Rc)

    def far_field(self, V_far: float, c_far: float) -> None:
        """Open the outer surface onto a far field of V_far cell volumes at c_far (Eqs. 7, 10, 14)."""
        _check(load().fdirw_coarse_far_field(ctypes.c_void_p(self.ctx), float(V_far), float(c_far)),
               ctypes.c_void_p(self.ctx))

    def c_far(self) -> float:
        v = ctypes.c_double(0.0)
        _check(load().fdirw_coarse_get_far_field(ctypes.c_void_p(self.ctx), ctypes.byref(v)), ctypes.c_void_p(self.ctx))
        return v.value

    def coupled_step(self, field, n_steps: int, k: float, cS_eq: float, cL_eq: float, dt: float, n_sub_solid: int):
        """n_steps coupled macro steps in place on field; returns (QL [n], QS [n], c_far)."""
        _check_f64(field, self.n)
        prm = fdirw_coupled_params(float(k), float(cS_eq), float(cL_eq), float(dt), int(n_sub_solid), 0)
        QL = np.empty(max(int(n_steps), 0))
        QS = np.empty(max(int(n_steps), 0))
        cf = ctypes.c_double(0.0)
        _check(load().fdirw_coupled_step(ctypes.c_void_p(self.ctx), ctypes.byref(prm), ctypes.c_void_p(_ptr(field)),
                                         int(n_steps), ctypes.c_void_p(QL.ctypes.data), ctypes.c_void_p(QS.ctypes.data),
                                         ctypes.byref(cf)), ctypes.c_void_p(self.ctx))
        return QL, QS, cf.value

    def read_pbc(self) -> np.ndarray:
        nb = 1
        for n in self.shape:
            nb *= (n + self.B - 1) // self.B
        out = np.empty(nb, dtype=np.float64)
        _check(load().fdirw_read_coarse_pbc(ctypes.c_void_p(self.ctx), ctypes.c_void_p(out.ctypes.data)),
               ctypes.c_void_p(self.ctx))
        return out


# --------------------------------------------------------------------------- learned surrogate

class Net:
    """The surrogate network (C ABI fdirw_net_*).  params: float32 [NET_NPARAM] (weights [4][27][16][16]
    as [layer][tap][co][ci], then biases [4][16])."""

    def __init__(self, params, device: int = -1):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if p.size != NET_NPARAM:
            raise ValueError(f"expected {NET_NPARAM} parameters")
        h = ctypes.c_void_p(0)
        _check(load().fdirw_net_create(ctypes.c_void_p(p.ctypes.data), int(device), ctypes.byref(h)))
        self.h = h.value

    def params(self) -> np.ndarray:
        out = np.empty(NET_NPARAM, dtype=np.float32)
        _check(load().fdirw_net_params(ctypes.c_void_p(self.h), ctypes.c_void_p(out.ctypes.data)))
        return out

    @staticmethod
    def _src(sources):
        return np.ascontiguousarray(sources, dtype=np.int64).reshape(-1)

    def predict(self, ctx: int, sources):
        """(kernels [n, 17, 17, 17] (unnormalised y), masses [n], accepted [n] bool)."""
        src = self._src(sources)
        k = np.empty((src.size, 17, 17, 17))
        m = np.empty(src.size)
        a = np.empty(src.size, dtype=np.int32)
        _check(load().fdirw_net_predict(ctypes.c_void_p(ctx), ctypes.c_void_p(self.h), ctypes.c_void_p(src.ctypes.data),
                                        src.size, ctypes.c_void_p(k.ctypes.data), ctypes.c_void_p(m.ctypes.data),
                                        ctypes.c_void_p(a.ctypes.data)), ctypes.c_void_p(ctx))
        return k, m, a.astype(bool)

    def gradients(self, ctx: int, sources, targets):
        src = self._src(sources)
        t = np.ascontiguousarray(targets, dtype=np.float64)
        g = np.empty(NET_NPARAM, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(load().fdirw_net_gradients(ctypes.c_void_p(ctx), ctypes.c_void_p(self.h), ctypes.c_void_p(src.ctypes.data),
                                          src.size, ctypes.c_void_p(_ptr(t)), ctypes.c_void_p(g.ctypes.data),
                                          ctypes.byref(loss)), ctypes.c_void_p(ctx))
        return g, loss.value

    def train_step(self, ctx: int, sources, targets, lr: float) -> float:
        src = self._src(sources)
        loss = ctypes.c_double(0.0)
        t = targets if hasattr(targets, "data_ptr") else np.ascontiguousarray(targets, dtype=np.float64)
        _check(load().fdirw_net_train_step(ctypes.c_void_p(ctx), ctypes.c_void_p(self.h), ctypes.c_void_p(src.ctypes.data),
                                           src.size, ctypes.c_void_p(_ptr(t)), float(lr), ctypes.byref(loss)),
               ctypes.c_void_p(ctx))
        return loss.value

    def trace(self, ctx: int, sources, targets=None):
        """fdirw_net_trace: (acts [4, n, 16, 17^3] uint16 BF16 patterns, z [n, 17^3] float32, grads
        [4, n, 16, 17^3] uint16 or None, parameter gradients [NET_NPARAM] float32 or None, mean loss or None)."""
        src = self._src(sources)
        n = src.size
        acts = np.empty((4, n, 16, 17 ** 3), dtype=np.uint16)
        z = np.empty((n, 17 ** 3), dtype=np.float32)
        grads = pg = t = None
        loss = ctypes.c_double(0.0)
        if targets is not None:
            t = np.ascontiguousarray(targets, dtype=np.float64)
            grads = np.empty((4, n, 16, 17 ** 3), dtype=np.uint16)
            pg = np.empty(NET_NPARAM, dtype=np.float32)
        _check(load().fdirw_net_trace(ctypes.c_void_p(ctx), ctypes.c_void_p(self.h), ctypes.c_void_p(src.ctypes.data), n,
                                      ctypes.c_void_p(t.ctypes.data if t is not None else 0),
                                      ctypes.c_void_p(acts.ctypes.data), ctypes.c_void_p(z.ctypes.data),
                                      ctypes.c_void_p(grads.ctypes.data if grads is not None else 0),
                                      ctypes.c_void_p(pg.ctypes.data if pg is not None else 0),
                                      ctypes.byref(loss) if t is not None else None), ctypes.c_void_p(ctx))
        return acts, z, grads, pg, (loss.value if t is not None else None)

    def conv_ms(self) -> float:
        """fdirw_net_timing: device time of the last forward pass's four convolutions (ms)."""
        v = ctypes.c_float(0.0)
        _check(load().fdirw_net_timing(ctypes.c_void_p(self.h), ctypes.byref(v)))
        return float(v.value)

    def test_wait(self, wait_ns: int = 0, withhold_mma: bool = False) -> None:
        """fdirw_net_test_wait: the MMA-wait budget (0 = default) and the withhold-MMA test hook."""
        _check(load().fdirw_net_test_wait(ctypes.c_void_p(self.h), int(wait_ns), 1 if withhold_mma else 0))

    def build_kernels(self, ctx: int) -> int:
        """fdirw_kernels_surrogate: returns the number of accepted sources."""
        acc = ctypes.c_int64(0)
        _check(load().fdirw_kernels_surrogate(ctypes.c_void_p(ctx), ctypes.c_void_p(self.h), ctypes.byref(acc)),
               ctypes.c_void_p(ctx))
        return acc.value

    def close(self):
        if self.h:
            load().fdirw_net_destroy(ctypes.c_void_p(self.h))
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_params(Ws, bs) -> np.ndarray:
    """Weights [4][27][16][16] and biases [4][16] (any float arrays) into the flat parameter vector."""
    return np.concatenate([np.asarray(Ws, dtype=np.float32).reshape(-1), np.asarray(bs, dtype=np.float32).reshape(-1)])


def unpack_params(p):
    p = np.asarray(p, dtype=np.float64)
    return p[:NET_NPARAM - 64].reshape(4, 27, 16, 16), p[NET_NPARAM - 64:].reshape(4, 16)
