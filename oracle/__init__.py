"""CPU FP64 oracle for the second-order nested-grid thin-disk force.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library under ``paper_1603_03142_gb300``) never imports this package, and
this package imports nothing from it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over targets):
a direct O(N^4) sum, over every source cell of every level, of the exact cell
integrals of the linear density of Eq. (eqnSigma) against the force kernel
(Sec. 2.1).  This module only builds and loads that library and marshals numpy
arrays.  Nest descriptors are duck-typed: any object with ``n``, ``levels``,
``x0``, ``y0``, ``h0`` and ``off`` (a sequence of ``(ox, oy)`` per level,
entry 0 unused) works.  Forests (several patches per level) are objects with
``n``, ``x0``, ``y0``, ``h0``, ``level`` and ``org`` (per patch: its level and
its corner in cells of that level from (x0, y0)) and ``levels`` = the number of
patches: every per-level list below is then a per-patch list.

Parity status of each function is stated in the design notes; every function
here is pinned by a ``-m "not gpu"`` test against quadrature, closed forms or
invariants (tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB = _HERE / "liboracle.so"
MAX_LEVELS = 8
MAX_PATCHES = 16


class _Nest(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("levels", ctypes.c_int),
        ("x0", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("h0", ctypes.c_double),
        ("off", (ctypes.c_int * 2) * MAX_LEVELS),
    ]


class _Forest(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("patches", ctypes.c_int),
        ("x0", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("h0", ctypes.c_double),
        ("level", ctypes.c_int * MAX_PATCHES),
        ("org", (ctypes.c_int * 2) * MAX_PATCHES),
    ]


def build_oracle(force: bool = False) -> Path:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", str(tmp), str(_SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(str(_LIB))
        dp = ctypes.POINTER(ctypes.c_double)
        dpp = ctypes.POINTER(dp)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_cell_integrals.argtypes = [ctypes.c_double] * 4 + [dp]
        lib.oracle_cell_integrals.restype = None
        lib.oracle_validate.argtypes = [ctypes.POINTER(_Nest)]
        lib.oracle_validate.restype = ctypes.c_int
        lib.oracle_prepare.argtypes = [ctypes.POINTER(_Nest), dpp, dpp, dpp, dpp]
        lib.oracle_prepare.restype = ctypes.c_int
        lib.oracle_force_targets.argtypes = [ctypes.POINTER(_Nest), dpp, dpp, dpp, ctypes.c_long,
                                             ip, ip, ip, dp, dp, ctypes.c_int]
        lib.oracle_force_targets.restype = ctypes.c_int
        lib.oracle_potential_targets.argtypes = [ctypes.POINTER(_Nest), dpp, dpp, dpp, ctypes.c_long,
                                                 ip, ip, ip, dp, ctypes.c_int]
        lib.oracle_potential_targets.restype = ctypes.c_int
        lib.oracle_cell_integrals_potential.argtypes = [ctypes.c_double] * 4 + [dp]
        lib.oracle_cell_integrals_potential.restype = None
        fp = ctypes.POINTER(_Forest)
        lib.oracle_forest_validate.argtypes = [fp]
        lib.oracle_forest_validate.restype = ctypes.c_int
        lib.oracle_forest_prepare.argtypes = [fp, dpp, dpp, dpp, dpp]
        lib.oracle_forest_prepare.restype = ctypes.c_int
        lib.oracle_forest_force_targets.argtypes = [fp, dpp, dpp, dpp, ctypes.c_long, ip, ip, ip, dp, dp,
                                                    ctypes.c_int]
        lib.oracle_forest_force_targets.restype = ctypes.c_int
        lib.oracle_forest_potential_targets.argtypes = [fp, dpp, dpp, dpp, ctypes.c_long, ip, ip, ip, dp,
                                                        ctypes.c_int]
        lib.oracle_forest_potential_targets.restype = ctypes.c_int
        lib.oracle_force_row.argtypes = [ctypes.POINTER(_Nest), dp, dp, dp, ctypes.c_int, ctypes.c_long, ip,
                                         dp, dp, ctypes.c_int]
        lib.oracle_force_row.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        for name in ("oracle_genconv_case2", "oracle_genconv_case3"):
            fn = getattr(lib, name)
            fn.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
            fn.restype = None
        _lib = lib
    return _lib


def _nest(desc) -> _Nest:
    g = _Nest()
    g.n, g.levels = int(desc.n), int(desc.levels)
    g.x0, g.y0, g.h0 = float(desc.x0), float(desc.y0), float(desc.h0)
    for l in range(1, int(desc.levels)):
        g.off[l][0], g.off[l][1] = int(desc.off[l][0]), int(desc.off[l][1])
    return g


def _is_forest(desc) -> bool:
    return hasattr(desc, "org") and hasattr(desc, "level")


def _forest(desc) -> _Forest:
    f = _Forest()
    K = len(desc.level)
    if K > MAX_PATCHES:
        raise ValueError(f"{K} patches, at most {MAX_PATCHES}")
    f.n, f.patches = int(desc.n), K
    f.x0, f.y0, f.h0 = float(desc.x0), float(desc.y0), float(desc.h0)
    for p in range(K):
        f.level[p] = int(desc.level[p])
        f.org[p][0], f.org[p][1] = int(desc.org[p][0]), int(desc.org[p][1])
    return f


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr_array(arrs):
    return (ctypes.POINTER(ctypes.c_double) * len(arrs))(*[_dp(a) for a in arrs])


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def cell_integrals(a: float, b: float, c: float, d: float) -> np.ndarray:
    """Exact integrals over [a,b]x[c,d] of u/r^3, v/r^3, u^2/r^3, v^2/r^3, uv/r^3."""
    out = np.zeros(5)
    _load().oracle_cell_integrals(a, b, c, d, _dp(out))
    return out


def cell_integrals_potential(a: float, b: float, c: float, d: float) -> np.ndarray:
    """Exact integrals over [a,b]x[c,d] of 1/r, u/r, v/r."""
    out = np.zeros(3)
    _load().oracle_cell_integrals_potential(a, b, c, d, _dp(out))
    return out


def validate(desc) -> bool:
    if _is_forest(desc):
        return _load().oracle_forest_validate(ctypes.byref(_forest(desc))) == 0
    return _load().oracle_validate(ctypes.byref(_nest(desc))) == 0


def prepare(desc, sigma):
    """Source fields of Eq. (eqnSigma) per level: (sig, dsig/dx, dsig/dy), covered cells 0."""
    n, L = int(desc.n), int(desc.levels)
    sin = [np.ascontiguousarray(s, dtype=np.float64).reshape(n, n) for s in sigma]
    if len(sin) != L:
        raise ValueError("need one sigma array per level")
    sig = [np.zeros((n, n)) for _ in range(L)]
    dsx = [np.zeros((n, n)) for _ in range(L)]
    dsy = [np.zeros((n, n)) for _ in range(L)]
    if _is_forest(desc):
        rc = _load().oracle_forest_prepare(ctypes.byref(_forest(desc)), _ptr_array(sin), _ptr_array(sig),
                                           _ptr_array(dsx), _ptr_array(dsy))
    else:
        rc = _load().oracle_prepare(ctypes.byref(_nest(desc)), _ptr_array(sin), _ptr_array(sig),
                                    _ptr_array(dsx), _ptr_array(dsy))
    if rc:
        raise ValueError(f"invalid nest descriptor (oracle_prepare rc={rc})")
    return sig, dsx, dsy


def force_at(desc, sigma, levels, ii, jj, nthreads: int = 0, prepared=None):
    """(Fx, Fy) at target cells (levels[k], ii[k], jj[k]); covered targets give 0."""
    lib = _load()
    sig, dsx, dsy = prepared if prepared is not None else prepare(desc, sigma)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    iv = np.ascontiguousarray(ii, dtype=np.int32)
    jv = np.ascontiguousarray(jj, dtype=np.int32)
    nt = lv.size
    fx = np.zeros(nt)
    fy = np.zeros(nt)
    ip = ctypes.POINTER(ctypes.c_int)
    fn, g = ((lib.oracle_forest_force_targets, _forest(desc)) if _is_forest(desc)
             else (lib.oracle_force_targets, _nest(desc)))
    rc = fn(ctypes.byref(g), _ptr_array(sig), _ptr_array(dsx),
                                  _ptr_array(dsy), nt, lv.ctypes.data_as(ip), iv.ctypes.data_as(ip),
                                  jv.ctypes.data_as(ip), _dp(fx), _dp(fy), int(nthreads))
    if rc:
        raise ValueError(f"oracle_force_targets failed rc={rc}")
    return fx, fy


def force(desc, sigma, nthreads: int = 0):
    """Full direct sum: lists of (n, n) arrays Fx[l], Fy[l]; covered cells are 0."""
    n, L = int(desc.n), int(desc.levels)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lv = np.repeat(np.arange(L), n * n)
    iv = np.tile(ii.ravel(), L)
    jv = np.tile(jj.ravel(), L)
    fx, fy = force_at(desc, sigma, lv, iv, jv, nthreads=nthreads)
    return [fx[l * n * n:(l + 1) * n * n].reshape(n, n) for l in range(L)], \
           [fy[l * n * n:(l + 1) * n * n].reshape(n, n) for l in range(L)]


def force_row(desc, sigma, jt: int, ii=None, nthreads: int = 0, prepared=None):
    """(Fx, Fy) at the targets (ii[k], jt) of row jt (every column if ii is None)
    of a single-level grid: the direct sum of oracle_force_targets, with the cell
    integrals of each source row evaluated once per cell offset from the target
    and shared by the row's targets (oracle.c, oracle_force_row)."""
    if _is_forest(desc) or int(desc.levels) != 1:
        raise ValueError("force_row takes a single-level grid")
    n = int(desc.n)
    sig, dsx, dsy = prepared if prepared is not None else prepare(desc, sigma)
    iv = np.arange(n, dtype=np.int32) if ii is None else np.ascontiguousarray(ii, dtype=np.int32)
    fx = np.zeros(iv.size)
    fy = np.zeros(iv.size)
    rc = _load().oracle_force_row(ctypes.byref(_nest(desc)), _dp(sig[0]), _dp(dsx[0]), _dp(dsy[0]), int(jt),
                                  iv.size, iv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(fx), _dp(fy),
                                  int(nthreads))
    if rc:
        raise ValueError(f"oracle_force_row rc={rc}")
    return fx, fy


def force_col(desc, sigma, it: int, jj=None, nthreads: int = 0):
    """(Fx, Fy) at the targets (it, jj[k]) of column it (every row if jj is None)
    of a single-level grid, by the x <-> y symmetry of the method: the grid with
    sigma transposed has the slope fields of sigma swapped and transposed (the
    slope rule treats x and y alike), its kernels are those of the original with
    the roles of u and v exchanged, so its row it holds (Fy, Fx) of column it."""
    if _is_forest(desc) or int(desc.levels) != 1:
        raise ValueError("force_col takes a single-level grid")
    sig, dsx, dsy = prepare(desc, sigma)
    tr = ([np.ascontiguousarray(sig[0].T)], [np.ascontiguousarray(dsy[0].T)], [np.ascontiguousarray(dsx[0].T)])
    gy, gx = force_row(desc, None, it, jj, nthreads=nthreads, prepared=tr)
    return gx, gy


def genconv_case2(b, c, m: int, nout: int) -> np.ndarray:
    """a_k = sum_j b_{m k - j} c_j  (Eq. eqnbmnn), k = 0..nout-1."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros(nout)
    _load().oracle_genconv_case2(_dp(b), b.size, _dp(c), c.size, int(m), _dp(out), int(nout))
    return out


def genconv_case3(b, c, m: int, nout: int) -> np.ndarray:
    """a_k = sum_j b_{k - m j} c_j  (Eq. eqnbnmn), k = 0..nout-1."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros(nout)
    _load().oracle_genconv_case3(_dp(b), b.size, _dp(c), c.size, int(m), _dp(out), int(nout))
    return out


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build_oracle(force="--force" in sys.argv))


def potential_at(desc, sigma, levels, ii, jj, nthreads: int = 0, prepared=None):
    """Potential (G = 1) at target cells (levels[k], ii[k], jj[k]); covered targets give 0."""
    lib = _load()
    sig, dsx, dsy = prepared if prepared is not None else prepare(desc, sigma)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    iv = np.ascontiguousarray(ii, dtype=np.int32)
    jv = np.ascontiguousarray(jj, dtype=np.int32)
    out = np.zeros(len(lv))
    ip = ctypes.POINTER(ctypes.c_int)
    fn, g = ((lib.oracle_forest_potential_targets, _forest(desc)) if _is_forest(desc)
             else (lib.oracle_potential_targets, _nest(desc)))
    rc = fn(ctypes.byref(g), _ptr_array(sig), _ptr_array(dsx),
                                      _ptr_array(dsy), len(lv), lv.ctypes.data_as(ip), iv.ctypes.data_as(ip),
                                      jv.ctypes.data_as(ip), _dp(out), int(nthreads))
    if rc:
        raise ValueError(f"oracle_potential_targets rc={rc}")
    return out


def potential(desc, sigma, nthreads: int = 0):
    """Potential at every cell of every level, as a list of (n, n) arrays."""
    n, L = int(desc.n), int(desc.levels)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lv = np.repeat(np.arange(L), n * n)
    out = potential_at(desc, sigma, lv, np.tile(ii.ravel(), L), np.tile(jj.ravel(), L), nthreads)
    return [out[l * n * n:(l + 1) * n * n].reshape(n, n) for l in range(L)]
