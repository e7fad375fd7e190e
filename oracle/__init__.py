"""CPU oracle for parallel uniform-grid construction (Algorithm 1, Sec. 3).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  Nothing in the product
package imports this module, and this module imports nothing from the product
package; the two share no code.  The arithmetic lives in ``oracle.c`` (plain
sequential C, built with ``-O2 -ffp-contract=off``); this file only compiles
it, marshals numpy arrays and chains the steps.

Entry points (numpy in, numpy out):

* ``bounds`` / ``plan`` / ``cell_boxes`` / ``exclusive_sum`` - the per-object
  steps (boxes, grid metadata M, CountCells, ExclusiveSum);
* ``object_order_pairs`` - MakeObjectIds, InclusiveSum, SegmentedExclusiveSum
  and MakeCellIds: the (C, O) lists of Fig. 4a/4b in object order;
* ``sort_pairs`` - RadixSort(C, O) as a stable sort by cell;
* ``ranges`` - RunLengthEncode, NonEmptyCells, ExclusiveSum -> G;
* ``build_grid`` - the whole chain, either literally (``method="alg1"``) or by the
  counting placement (``method="counting"``, O(NO), for large scenes);
* ``grid_bruteforce`` - every (cell, object) pair tested directly (tiny only);
* ``tri_cell_separated`` / ``cull_pairs`` / ``place_stable`` and
  ``build_grid(..., cull=True)`` - the false-intersection culling mode (a
  triangle/cell separating-axis test before the sort, Sec. 6's future work).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

OK, EINVAL, ENOMEM, EOVERFLOW = 0, -1, -2, -3

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def compile_source(src: str, out: str) -> str:
    """gcc -O2 without FMA contraction or fast-math -> shared library."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_library(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (if stale)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def _bind(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    for name, args in {
        "or_bounds": [P, I64, P, I64, P, P],
        "or_plan": [P, P, I64, ctypes.c_float, P, P, P],
        "or_cell_boxes": [P, P, I64, P, P, P, P, P, P],
        "or_exclusive_sum": [P, I64, P, P],
        "or_object_order_pairs": [P, P, P, I64, I64, P, P, P],
        "or_sort_pairs": [P, P, I64],
        "or_ranges": [P, I64, I64, P],
        "or_grid_counting": [P, P, I64, P, I64, P, P],
        "or_grid_bruteforce": [P, P, I64, P, P, P, I64, P],
        "or_tri_cell_separated": [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
        "or_cull_pairs": [P, P, I64, P, P, P, P, P, I64, P, P, P, P],
        "or_place_stable": [P, P, I64, I64, P, P],
    }.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return lib


_PAR_SRC = os.path.join(_HERE, "cpu_parallel.c")
_PAR_LIB = os.path.join(_BUILD_DIR, "libcpu_parallel.so")
_par = None


def build_parallel_library(force: bool = False) -> str:
    """Compile the multi-core CPU baseline (cpu_parallel.c with the oracle's
    own steps, OpenMP) into _build/libcpu_parallel.so (if stale)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_PAR_LIB)
            and os.path.getmtime(_PAR_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_PAR_SRC))):
        return _PAR_LIB
    tmp = _PAR_LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                    "-o", tmp, _PAR_SRC, _SRC, "-lm"], check=True)
    os.replace(tmp, _PAR_LIB)
    return _PAR_LIB


def _load_parallel():
    global _par
    with _lock:
        if _par is None:
            lib = ctypes.CDLL(build_parallel_library())
            P, I64 = ctypes.c_void_p, ctypes.c_int64
            lib.cp_threads.argtypes = [ctypes.c_int]
            lib.cp_threads.restype = ctypes.c_int
            lib.cp_build_grid.argtypes = [P, I64, P, I64, ctypes.c_float, P, I64, P, I64, P, P]
            lib.cp_build_grid.restype = ctypes.c_int
            _par = lib
    return _par


def parallel_threads(nthreads: int = 0) -> int:
    """Threads the multi-core baseline uses (0: every host core)."""
    return int(_load_parallel().cp_threads(int(nthreads)))


def grid_parallel(verts, tris, lam: float, nthreads: int = 0):
    """The multi-core CPU baseline (a benchmark reference point, not a pin):
    the oracle's steps under OpenMP with an atomic counting placement and a
    per-cell sort.  Returns (G, refs, NO), equal to build_grid's."""
    lib = _load_parallel()
    lib.cp_threads(int(nthreads))
    v = _c(verts, np.float32, (-1, 3))
    t = _c(tris, np.int32, (-1, 3))
    nc = np.zeros(1, np.int64)
    nr = np.zeros(1, np.int64)
    G = np.zeros(1, np.int32)
    rc = lib.cp_build_grid(_p(v), v.shape[0], _p(t), t.shape[0], ctypes.c_float(lam), _p(G), 0, None, 0,
                           _p(nc), _p(nr))
    if rc not in (OK, EOVERFLOW):
        _check(rc, "grid_parallel")
    G = np.zeros(int(nc[0]) + 1, np.int32)
    refs = np.zeros(max(int(nr[0]), 1), np.int32)
    _check(lib.cp_build_grid(_p(v), v.shape[0], _p(t), t.shape[0], ctypes.c_float(lam), _p(G), G.shape[0],
                             _p(refs), refs.shape[0], _p(nc), _p(nr)), "grid_parallel")
    return G, refs[: int(nr[0])].copy(), int(nr[0])


def use_library(path: str) -> None:
    """Points this module at another build of oracle.c (the mutation tests
    plant mistakes in copies of it to show the pins catch them)."""
    global _lib
    with _lock:
        _lib = _bind(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build_library()))
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(code: int, what: str):
    if code != OK:
        raise OracleError(code, what)


def _c(a, dtype, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


@dataclasses.dataclass
class Plan:
    lo: np.ndarray      # float32[3] scene bounds
    hi: np.ndarray      # float32[3]
    res: np.ndarray     # int32[3] cells per axis
    scale: np.ndarray   # float32[3] res / extent (0 on a flat axis)
    ncells: int


def bounds(verts, tris):
    """Per-triangle boxes' union -> (lo, hi) float32[3]."""
    lib = _load()
    v = _c(verts, np.float32, (-1, 3))
    t = _c(tris, np.int32, (-1, 3))
    lo = np.zeros(3, np.float32)
    hi = np.zeros(3, np.float32)
    _check(lib.or_bounds(_p(v), v.shape[0], _p(t), t.shape[0], _p(lo), _p(hi)), "bounds")
    return lo, hi


def plan(lo, hi, n: int, lam: float) -> Plan:
    """Grid resolution and scale from the density rule."""
    lib = _load()
    lo = _c(lo, np.float32)
    hi = _c(hi, np.float32)
    res = np.zeros(3, np.int32)
    scale = np.zeros(3, np.float32)
    nc = np.zeros(1, np.int64)
    _check(lib.or_plan(_p(lo), _p(hi), int(n), ctypes.c_float(lam), _p(res), _p(scale), _p(nc)),
           "plan")
    return Plan(lo, hi, res, scale, int(nc[0]))


def cell_boxes(verts, tris, p: Plan):
    """CountCells: (clo int32[n,3], chi int32[n,3], V int64[n])."""
    lib = _load()
    v = _c(verts, np.float32, (-1, 3))
    t = _c(tris, np.int32, (-1, 3))
    n = t.shape[0]
    clo = np.zeros((n, 3), np.int32)
    chi = np.zeros((n, 3), np.int32)
    V = np.zeros(n, np.int64)
    _check(lib.or_cell_boxes(_p(v), _p(t), n, _p(p.lo), _p(p.scale), _p(p.res),
                             _p(clo), _p(chi), _p(V)), "cell_boxes")
    return clo, chi, V


def exclusive_sum(V):
    """ExclusiveSum(V) -> (offsets int64[n], NO)."""
    lib = _load()
    V = _c(V, np.int64)
    off = np.zeros(V.shape[0], np.int64)
    tot = np.zeros(1, np.int64)
    _check(lib.or_exclusive_sum(_p(V), V.shape[0], _p(off), _p(tot)), "exclusive_sum")
    return off, int(tot[0])


def object_order_pairs(clo, chi, offsets, NO: int, res):
    """(C, O) int32[NO] in object order (Fig. 4a/4b)."""
    lib = _load()
    clo = _c(clo, np.int32, (-1, 3))
    chi = _c(chi, np.int32, (-1, 3))
    off = _c(offsets, np.int64)
    res = _c(res, np.int32)
    C = np.zeros(NO, np.int32)
    O = np.zeros(NO, np.int32)
    _check(lib.or_object_order_pairs(_p(clo), _p(chi), _p(off), clo.shape[0], NO, _p(res),
                                     _p(C), _p(O)), "object_order_pairs")
    return C, O


def sort_pairs(C, O):
    """Stable sort of (C, O) by C -> new arrays."""
    lib = _load()
    C = np.array(C, dtype=np.int32, copy=True)
    O = np.array(O, dtype=np.int32, copy=True)
    _check(lib.or_sort_pairs(_p(C), _p(O), C.shape[0]), "sort_pairs")
    return C, O


def ranges(C_sorted, ncells: int):
    """G int32[ncells + 1] from the cell-sorted C."""
    lib = _load()
    C = _c(C_sorted, np.int32)
    G = np.zeros(ncells + 1, np.int32)
    _check(lib.or_ranges(_p(C), C.shape[0], ncells, _p(G)), "ranges")
    return G


def grid_counting(clo, chi, p: Plan, NO: int):
    lib = _load()
    clo = _c(clo, np.int32, (-1, 3))
    chi = _c(chi, np.int32, (-1, 3))
    G = np.zeros(p.ncells + 1, np.int32)
    refs = np.zeros(NO, np.int32)
    _check(lib.or_grid_counting(_p(clo), _p(chi), clo.shape[0], _p(p.res), p.ncells,
                                _p(G), _p(refs)), "grid_counting")
    return G, refs


def grid_bruteforce(clo, chi, p: Plan, cap: int | None = None):
    lib = _load()
    clo = _c(clo, np.int32, (-1, 3))
    chi = _c(chi, np.int32, (-1, 3))
    if cap is None:
        cap = max(1, p.ncells * clo.shape[0])
    G = np.zeros(p.ncells + 1, np.int32)
    refs = np.zeros(cap, np.int32)
    nr = np.zeros(1, np.int64)
    _check(lib.or_grid_bruteforce(_p(clo), _p(chi), clo.shape[0], _p(p.res), _p(G), _p(refs),
                                  cap, _p(nr)), "grid_bruteforce")
    return G, refs[: int(nr[0])].copy()


def tri_cell_separated(q, x: int, y: int, z: int) -> bool:
    """The culling test: is the triangle with grid-space vertices q
    (float32[3, 3], row = vertex) separated from cell (x, y, z)?"""
    lib = _load()
    q = _c(q, np.float32, (9,))
    return bool(lib.or_tri_cell_separated(_p(q), int(x), int(y), int(z)))


def grid_space(verts, tris, p: Plan):
    """q float32[n, 3, 3]: each triangle's vertices in grid coordinates,
    min((v - lo) * scale, res) with each operation rounded to FP32 (numpy
    float32 arithmetic: one rounding per operation)."""
    v = _c(verts, np.float32, (-1, 3))
    t = _c(tris, np.int32, (-1, 3))
    q = ((v[t] - p.lo[None, None, :]).astype(np.float32) * p.scale[None, None, :]).astype(np.float32)
    return np.minimum(q, p.res.astype(np.float32)[None, None, :])


def cull_pairs(verts, tris, p: Plan, clo, chi, cap: int):
    """Box-placement pairs minus the culled ones, in object order:
    (C int32[NOk], O int32[NOk], kept int64[n])."""
    lib = _load()
    v = _c(verts, np.float32, (-1, 3))
    t = _c(tris, np.int32, (-1, 3))
    clo = _c(clo, np.int32, (-1, 3))
    chi = _c(chi, np.int32, (-1, 3))
    n = t.shape[0]
    C = np.zeros(max(cap, 1), np.int32)
    O = np.zeros(max(cap, 1), np.int32)
    kept = np.zeros(n, np.int64)
    nk = np.zeros(1, np.int64)
    _check(lib.or_cull_pairs(_p(v), _p(t), n, _p(p.lo), _p(p.scale), _p(p.res), _p(clo), _p(chi), cap,
                             _p(C), _p(O), _p(kept), _p(nk)), "cull_pairs")
    k = int(nk[0])
    return C[:k].copy(), O[:k].copy(), kept


def place_stable(C, O, ncells: int):
    """Stable counting placement of object-order pairs -> (G, refs)."""
    lib = _load()
    C = _c(C, np.int32)
    O = _c(O, np.int32)
    G = np.zeros(ncells + 1, np.int32)
    refs = np.zeros(max(C.shape[0], 1), np.int32)
    _check(lib.or_place_stable(_p(C), _p(O), C.shape[0], ncells, _p(G), _p(refs)), "place_stable")
    return G, refs[: C.shape[0]].copy()


@dataclasses.dataclass
class Grid:
    plan: Plan
    G: np.ndarray       # int32[ncells + 1]
    refs: np.ndarray    # int32[NO] object ids in cell order
    NO: int
    clo: np.ndarray | None = None
    chi: np.ndarray | None = None
    V: np.ndarray | None = None
    offsets: np.ndarray | None = None


def build_grid(verts, tris, lam: float, method: str = "alg1", cull: bool = False) -> Grid:
    """BuildParallelGrid: boxes -> M -> ... -> (G, O).  With cull, the pairs a
    triangle/cell separating-axis test rejects are removed before the sort
    (the culling mode; NO is then the kept count and V the kept counts per
    object): "alg1" sorts the kept lists with the stable sort + range steps,
    any other method uses the stable counting placement."""
    lo, hi = bounds(verts, tris)
    n = int(np.asarray(tris).reshape(-1, 3).shape[0])
    p = plan(lo, hi, n, lam)
    clo, chi, V = cell_boxes(verts, tris, p)
    off, NO = exclusive_sum(V)
    if cull:
        C, O, kept = cull_pairs(verts, tris, p, clo, chi, NO)
        if method == "alg1":
            Cs, Os = sort_pairs(C, O)
            G, refs = ranges(Cs, p.ncells), Os
        else:
            G, refs = place_stable(C, O, p.ncells)
        koff, NOk = exclusive_sum(kept)
        return Grid(p, G, refs, NOk, clo, chi, kept, koff)
    if method == "alg1":
        C, O = object_order_pairs(clo, chi, off, NO, p.res)
        Cs, Os = sort_pairs(C, O)
        G = ranges(Cs, p.ncells)
        refs = Os
    elif method == "counting":
        G, refs = grid_counting(clo, chi, p, NO)
    elif method == "bruteforce":
        G, refs = grid_bruteforce(clo, chi, p, cap=NO)
    else:
        raise ValueError(method)
    return Grid(p, G, refs, NO, clo, chi, V, off)
