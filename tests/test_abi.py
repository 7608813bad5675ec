"""C-ABI library checks that need no GPU: it loads, exports every declared symbol, validates arguments on
the host, and the product path has no route to the oracle or a CPU fallback."""
import ast
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2408_11376_gb300 import build as libbuild
from paper_2408_11376_gb300 import fdirw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fdirw.h")).read()
    return re.findall(r"FDIRW_API\s+[\w\s\*]+?\b(fdirw_\w+)\s*\(", src)


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return fdirw.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) == len(set(names)) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fdirw.EXPORTED)


def test_host_side_argument_checks(lib):
    D = np.ones(64)
    bad = [((0, 4, 4), 1.0, 2, 3, 1.0), ((4, 4, 4), float("nan"), 2, 3, 1.0), ((4, 4, 4), 1.0, 11, 3, 1.0),
           ((4, 4, 4), 1.0, -1, 3, 1.0), ((4, 4, 4), 1.0, 2, -3, 1.0), ((4, 4, 4), -1.0, 2, 3, 1.0),
           ((4, 4, 4), 1.0, 2, 3, 0.0)]
    for shape, dt, R, n_sub, h in bad:
        g = fdirw.fdirw_grid(*shape, h)
        ctx = ctypes.c_void_p(1234)
        rc = lib.fdirw_create(ctypes.byref(g), ctypes.c_void_p(D.ctypes.data), dt, R, n_sub, None, ctypes.byref(ctx))
        assert rc == fdirw.FDIRW_ERR_ARG, (shape, dt, R, n_sub, h)
        assert ctx.value is None
        assert fdirw.fdirw_last_error()
    g = fdirw.fdirw_grid(4, 4, 4, 1.0)
    assert lib.fdirw_create(ctypes.byref(g), None, 1.0, 2, 3, None, ctypes.byref(ctypes.c_void_p())) == fdirw.FDIRW_ERR_ARG
    for R, bad_opts in ((2, fdirw.fdirw_opts(7, -1, None, 0, 0, 0)), (2, fdirw.fdirw_opts(1, -1, None, 0, 8, 0)),
                        (9, fdirw.fdirw_opts(fdirw.FDIRW_FP64, -1, None, 0, 0, 0)),
                        (2, fdirw.fdirw_opts(fdirw.FDIRW_FP32, -1, None, 0, 0, 2)),                  # unknown accum
                        (2, fdirw.fdirw_opts(fdirw.FDIRW_FP64, -1, None, 0, 0, fdirw.FDIRW_ACCUM_FP32))):
        rc = lib.fdirw_create(ctypes.byref(g), ctypes.c_void_p(D.ctypes.data), 1.0, R, 3, ctypes.byref(bad_opts),
                              ctypes.byref(ctypes.c_void_p()))
        assert rc == fdirw.FDIRW_ERR_ARG
    assert lib.fdirw_kernels(None) == fdirw.FDIRW_ERR_ARG
    assert lib.fdirw_step(None, None, None, 1, None) == fdirw.FDIRW_ERR_ARG
    lib.fdirw_destroy(None)   # NULL-safe


def test_batch_host_side_argument_checks(lib):
    D = np.ones(64)
    g = (fdirw.fdirw_grid * 2)(fdirw.fdirw_grid(4, 4, 4, 1.0), fdirw.fdirw_grid(4, 4, 4, 1.0))
    ptrs = (ctypes.c_void_p * 2)(D.ctypes.data, D.ctypes.data)
    huge = (fdirw.fdirw_grid * 1)(fdirw.fdirw_grid(1024, 1024, 256, 1.0))     # 2^28 cells
    fp64 = fdirw.fdirw_opts(fdirw.FDIRW_FP64, -1, None, 0, 0, 0)
    parts8 = fdirw.fdirw_opts(fdirw.FDIRW_FP32, -1, None, 0, 8, 0)
    bad_grid = (fdirw.fdirw_grid * 1)(fdirw.fdirw_grid(4, 0, 4, 1.0))
    acc_bad = fdirw.fdirw_opts(fdirw.FDIRW_FP32, -1, None, 0, 0, 2)
    cases = [(0, g, ptrs, 1.0, 1, 3, 2, None), (2, None, ptrs, 1.0, 1, 3, 2, None), (2, g, None, 1.0, 1, 3, 2, None),
             (2, g, ptrs, 1.0, 1, 11, 2, None), (2, g, ptrs, 1.0, 4, 3, 2, None), (2, g, ptrs, 1.0, -1, 3, 2, None),
             (2, g, ptrs, -1.0, 1, 3, 2, None), (2, g, ptrs, 1.0, 1, 3, -2, None), (1, huge, ptrs, 1.0, 1, 3, 2, None),
             (2, g, ptrs, 1.0, 1, 3, 2, fp64), (2, g, ptrs, 1.0, 1, 3, 2, parts8), (1, bad_grid, ptrs, 1.0, 1, 3, 2, None),
             (2, g, ptrs, 1.0, 1, 3, 2, acc_bad)]
    for n, grids, dm, dt, rmin, rmax, n_sub, opts in cases:
        ctx = ctypes.c_void_p(1234)
        rc = lib.fdirw_create_batch(n, grids, dm, dt, rmin, rmax, n_sub, ctypes.byref(opts) if opts else None,
                                    ctypes.byref(ctx))
        assert rc == fdirw.FDIRW_ERR_ARG, (n, dt, rmin, rmax, n_sub)
        assert ctx.value is None
    null_ptrs = (ctypes.c_void_p * 2)(D.ctypes.data, None)
    assert lib.fdirw_create_batch(2, g, null_ptrs, 1.0, 1, 3, 2, None, ctypes.byref(ctypes.c_void_p())) == \
        fdirw.FDIRW_ERR_ARG
    assert lib.fdirw_read_radius(None, None) == fdirw.FDIRW_ERR_ARG


def test_coarse_host_side_argument_checks(lib):
    D = np.ones(64)
    g = fdirw.fdirw_grid(4, 4, 4, 1.0)
    fp64 = fdirw.fdirw_opts(fdirw.FDIRW_FP64, -1, None, 0, 0, 0)
    acc32 = fdirw.fdirw_opts(fdirw.FDIRW_FP32, -1, None, 0, 0, fdirw.FDIRW_ACCUM_FP32)
    for block, R, opts in ((2, 2, None), (0, 2, None), (-1, 2, None), (5, 9, None), (1, 0, None), (3, -1, None),
                           (3, 2, fp64), (3, 2, acc32)):
        ctx = ctypes.c_void_p(1234)
        rc = lib.fdirw_create_coarse(ctypes.byref(g), ctypes.c_void_p(D.ctypes.data), None, block, 0.1, R, 2,
                                     ctypes.byref(opts) if opts else None, ctypes.byref(ctx))
        assert rc == fdirw.FDIRW_ERR_ARG, (block, R)
        assert ctx.value is None
    assert lib.fdirw_create_coarse(ctypes.byref(g), None, None, 3, 0.1, 2, 2, None,
                                   ctypes.byref(ctypes.c_void_p())) == fdirw.FDIRW_ERR_ARG
    assert lib.fdirw_read_coarse(None, None, 0, None) == fdirw.FDIRW_ERR_ARG
    assert lib.fdirw_coarse_far_field(None, 1.0, 0.0) == fdirw.FDIRW_ERR_ARG
    assert lib.fdirw_coarse_get_far_field(None, None) == fdirw.FDIRW_ERR_ARG
    assert lib.fdirw_read_coarse_pbc(None, None) == fdirw.FDIRW_ERR_ARG


def test_binding_fails_loudly_without_library(tmp_path):
    saved = fdirw._lib
    try:
        fdirw._lib = None
        with pytest.raises(ImportError):
            fdirw.load(str(tmp_path / "missing.so"))
    finally:
        fdirw._lib = saved


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2408_11376_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                tree = ast.parse(open(os.path.join(dirpath, f)).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), f
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", f
            if f.endswith((".cu", ".h", ".cpp", ".c")):
                assert "fdirw_oracle" not in open(os.path.join(dirpath, f)).read(), f


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """The ctypes structures and constants of the binding against the C header, compiled with gcc: every
    field at the same offset with the same size, the same struct sizes, the same constant values."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = (fdirw.fdirw_grid, fdirw.fdirw_opts, fdirw.fdirw_coupled_params, fdirw.fdirw_info)
    consts = ("FDIRW_OK", "FDIRW_ERR_ARG", "FDIRW_ERR_UNSTABLE", "FDIRW_ERR_NOMEM", "FDIRW_ERR_CUDA",
              "FDIRW_ERR_TIMEOUT", "FDIRW_ERR_STATE", "FDIRW_FP64", "FDIRW_FP32", "FDIRW_FP32_STORE_FP16",
              "FDIRW_FP32_STORE_BF16", "FDIRW_ACCUM_FF", "FDIRW_ACCUM_FP32")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fdirw.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'    printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'    printf("{n}.{f} %zu %zu\\n", offsetof({n}, {f}), sizeof((({n}*)0)->{f}));')
    for c in consts:
        lines.append(f'    printf("{c} %d\\n", (int)({c}));')
    lines.append('    printf("FDIRW_NET_NPARAM %d\\n", (int)(FDIRW_NET_NPARAM));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        k, *v = l.split()
        got[k] = tuple(int(x) for x in v)
    for st in structs:
        n = st.__name__
        assert got[n] == (ctypes.sizeof(st),), n
        for f, t in st._fields_:
            assert got[f"{n}.{f}"] == (getattr(st, f).offset, ctypes.sizeof(t)), (n, f)
    for c in consts:
        assert got[c] == (getattr(fdirw, c),), c
    assert got["FDIRW_NET_NPARAM"] == (fdirw.NET_NPARAM,)


_SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64, "double": ctypes.c_double, "float": ctypes.c_float,
            "int": ctypes.c_int}
_POINTEES = {"double": ctypes.c_double, "int64_t": ctypes.c_int64, "float": ctypes.c_float, "fdirw_grid": fdirw.fdirw_grid,
             "fdirw_opts": fdirw.fdirw_opts, "fdirw_info": fdirw.fdirw_info,
             "fdirw_coupled_params": fdirw.fdirw_coupled_params}


def _prototypes():
    """(return type, name, [parameter types]) of every FDIRW_API declaration in the header."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "fdirw.h")).read(), flags=re.S)
    out = []
    for ret, name, params in re.findall(r"FDIRW_API\s+([\w\s\*]+?)\s*\b(fdirw_\w+)\s*\(([^)]*)\)\s*;", src):
        types = []
        for p in params.split(","):
            p = " ".join(p.split())
            if p == "void":
                continue
            m = re.match(r"^(.*?)(\w+)$", p)
            types.append(m.group(1).replace("const", "").replace(" ", ""))
        out.append((ret.replace("const", "").replace(" ", ""), name, types))
    return out


def test_binding_argtypes_match_the_header_prototypes(lib):
    """Every entry point's ctypes signature against its C prototype: the same arity, the same scalar types
    (an int64 passed where the C side reads an int32 would shift every later argument), and pointers
    declared as pointers (of the same pointee where the binding names one)."""
    protos = _prototypes()
    assert {n for _, n, _ in protos} == set(fdirw.EXPORTED)
    for ret, name, types in protos:
        f = getattr(lib, name)
        assert len(f.argtypes) == len(types), name
        for i, (ct, at) in enumerate(zip(types, f.argtypes)):
            if "*" in ct:
                base = ct.rstrip("*")
                if at is ctypes.c_void_p:
                    continue
                assert hasattr(at, "_type_") and ct.count("*") >= 1, (name, i, ct, at)
                if ct.count("*") == 2 or base in ("void", "fdirw_ctx", "fdirw_net"):
                    assert at._type_ is ctypes.c_void_p, (name, i, ct, at)      # pointer to a handle
                else:
                    assert at._type_ is _POINTEES[base], (name, i, ct, at)
            else:
                assert at is _SCALARS[ct], (name, i, ct, at)
        if ret == "int":
            assert f.restype is ctypes.c_int, name
        elif ret == "void":
            assert f.restype is None, name
        else:
            assert ret == "char*" and f.restype is ctypes.c_char_p, name
