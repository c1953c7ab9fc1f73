"""CPU oracle for SpMSpV and BFS (test infrastructure only).

This package is the plain, sequential statement of what the GPU path
computes (Azad & Buluc, arXiv 1610.07902): a Gustavson column walk into a
sparse accumulator (Sec. I, Sec. II-F), BFS as repeated masked
(min, select2nd) SpMSpV (Sec. IV-D), and the pull (matrix-driven) form of a
BFS level (Sec. II-B), and the definitions the SpMSpV-built graph algorithms
of Sec. I reach: connected components (smallest vertex id per component) and
the maximal independent set of Luby's rounds with fixed priorities (the
greedy set in priority order), and the cardinality of a maximum bipartite
matching between rows and columns (augmenting paths).  The arithmetic lives in ``oracle.c``; this module
only compiles it with gcc and marshals numpy arrays.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PLUS_TIMES = 0
MIN_SELECT2ND = 1
OR_AND = 2

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so (sequential, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    p = ctypes.c_void_p
    lib.oracle_spmspv.restype = ctypes.c_int64
    lib.oracle_spmspv.argtypes = [ctypes.c_int32, ctypes.c_int32, p, p, p, ctypes.c_int,
                                  p, p, ctypes.c_int32, p, ctypes.c_int, p, p, p, p]
    lib.oracle_bfs.restype = ctypes.c_int32
    lib.oracle_bfs.argtypes = [ctypes.c_int32, p, p, ctypes.c_int32, p, p, p, p]
    lib.oracle_bfs_pull.restype = ctypes.c_int32
    lib.oracle_bfs_pull.argtypes = [ctypes.c_int32, p, p, ctypes.c_int32, p, p]
    lib.oracle_cc.restype = ctypes.c_int32
    lib.oracle_cc.argtypes = [ctypes.c_int32, p, p, p]
    lib.oracle_mis.restype = ctypes.c_int32
    lib.oracle_mis.argtypes = [ctypes.c_int32, p, p, p, p]
    lib.oracle_mcm.restype = ctypes.c_int32
    lib.oracle_mcm.argtypes = [ctypes.c_int32, ctypes.c_int32, p, p, p, p]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def load_variant(path: str):
    """Bind another build of oracle.c (used by tests that plant a mistake in
    a copy of the oracle to show that the pins catch it)."""
    return _bind(ctypes.CDLL(path))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class SpMSpVResult:
    """y in sorted list form plus the oracle's multiply count."""

    def __init__(self, idx, val, absum, nmult):
        self.idx = idx        # int32[nnz_y], ascending
        self.val = val        # float64[] (plus,times), int32[] (min,select2nd) or None
        self.absum = absum    # float64[]: sum_j |A(i,j) x(j)| per output (plus,times)
        self.nmult = nmult    # multiply count = sum of selected column lengths


def spmspv(m, colptr, rowidx, val, semiring, x_idx, x_val=None, mask=None,
           complement=True, lib=None, with_absum=True) -> SpMSpVResult:
    """y <- A (+).(x) x under an optional mask (bool/uint8 array of length m).

    colptr/rowidx int32, val float32 or None (pattern matrix), x_idx int32,
    x_val float32 (plus,times) / int32 (min,select2nd) / ignored (or,and).
    """
    lib = lib or _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    n = colptr.shape[0] - 1
    x_idx = np.ascontiguousarray(x_idx, dtype=np.int32)
    f = x_idx.shape[0]
    if val is not None:
        val = np.ascontiguousarray(val, dtype=np.float32)
    if semiring == PLUS_TIMES:
        x_val = np.ascontiguousarray(x_val, dtype=np.float32)
    elif semiring == MIN_SELECT2ND:
        x_val = np.ascontiguousarray(x_val, dtype=np.int32)
    else:
        x_val = None
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        assert mask.shape[0] == m
    if f and (x_idx.min() < 0 or x_idx.max() >= n):
        cap = m  # the C side reports the bad index
    else:
        cap = int(min(m, int(np.sum(colptr[x_idx + 1] - colptr[x_idx]))) if f else 0)
    y_idx = np.empty(max(cap, 1), dtype=np.int32)
    if semiring == PLUS_TIMES:
        y_val = np.empty(max(cap, 1), dtype=np.float64)
        absum = np.empty(max(cap, 1), dtype=np.float64) if with_absum else None
    elif semiring == MIN_SELECT2ND:
        y_val = np.empty(max(cap, 1), dtype=np.int32)
        absum = None
    else:
        y_val = None
        absum = None
    nnz_y = ctypes.c_int32(0)
    nm = lib.oracle_spmspv(m, n, _ptr(colptr), _ptr(rowidx), _ptr(val), semiring, _ptr(x_idx),
                           _ptr(x_val), f, _ptr(mask), 1 if complement else 0, _ptr(y_idx),
                           _ptr(y_val), _ptr(absum), ctypes.byref(nnz_y))
    if nm < 0:
        raise ValueError("oracle_spmspv failed with code %d" % nm)
    k = nnz_y.value
    return SpMSpVResult(y_idx[:k].copy(), None if y_val is None else y_val[:k].copy(),
                        None if absum is None else absum[:k].copy(), int(nm))


def bfs(colptr, rowidx, src, lib=None):
    """Levels and parents of BFS from src by iterated masked (min,select2nd) SpMSpV.

    Returns (level int32[n], parent int32[n], nlevels, total_mult, level_sizes).
    """
    lib = lib or _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    n = colptr.shape[0] - 1
    level = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    sizes = np.zeros(n + 1, dtype=np.int32)
    tm = ctypes.c_int64(0)
    nl = lib.oracle_bfs(n, _ptr(colptr), _ptr(rowidx), int(src), _ptr(level), _ptr(parent),
                        ctypes.byref(tm), _ptr(sizes))
    if nl < 0:
        raise ValueError("oracle_bfs failed with code %d" % nl)
    return level, parent, int(nl), int(tm.value), sizes[:nl].copy()


def cc(colptr, rowidx, lib=None):
    """Connected components: (label int32[n], number of components), label[v]
    the smallest vertex id of v's component (pattern-symmetric A)."""
    lib = lib or _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    n = colptr.shape[0] - 1
    label = np.empty(n, dtype=np.int32)
    k = lib.oracle_cc(n, _ptr(colptr), _ptr(rowidx), _ptr(label))
    if k < 0:
        raise ValueError("oracle_cc failed with code %d" % k)
    return label, int(k)


def mis(colptr, rowidx, prio, lib=None):
    """Maximal independent set reached by Luby's rounds with these distinct
    priorities: (in_set int32[n] of 0/1, size)."""
    lib = lib or _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    prio = np.ascontiguousarray(prio, dtype=np.int32)
    n = colptr.shape[0] - 1
    in_set = np.empty(n, dtype=np.int32)
    k = lib.oracle_mis(n, _ptr(colptr), _ptr(rowidx), _ptr(prio), _ptr(in_set))
    if k < 0:
        raise ValueError("oracle_mis failed with code %d" % k)
    return in_set, int(k)


def mcm(m, colptr, rowidx, lib=None):
    """Maximum-cardinality matching between the m rows and the columns:
    (mate_r int32[m], mate_c int32[n], cardinality)."""
    lib = lib or _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    n = colptr.shape[0] - 1
    mate_r = np.empty(m, dtype=np.int32)
    mate_c = np.empty(n, dtype=np.int32)
    k = lib.oracle_mcm(m, n, _ptr(colptr), _ptr(rowidx), _ptr(mate_r), _ptr(mate_c))
    if k < 0:
        raise ValueError("oracle_mcm failed with code %d" % k)
    return mate_r, mate_c, int(k)


def bfs_pull(colptr, rowidx, src, lib=None):
    """BFS with every level computed in the matrix-driven (pull) form."""
    lib = lib or _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    n = colptr.shape[0] - 1
    level = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    nl = lib.oracle_bfs_pull(n, _ptr(colptr), _ptr(rowidx), int(src), _ptr(level), _ptr(parent))
    if nl < 0:
        raise ValueError("oracle_bfs_pull failed with code %d" % nl)
    return level, parent, int(nl)
