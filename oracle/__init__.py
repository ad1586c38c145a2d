"""CPU oracle for batched 2-D distance reporting along a space-filling curve (arXiv 2508.19891).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the cpu_baseline /
reference leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library and the CUDA library never calls it.

The heavy parts (keys, the sort, Alg. 1, brute force, the early-termination quadtree, the 3-D
Z curve) are plain C in ``oracle.c``, compiled
here with gcc into ``liboracle.so`` and called through ctypes; this module only marshals
numpy arrays.  ``learned.py`` holds the fp64 reference of the learned-bounds model and
``dynamic.py`` the rebuild-from-scratch oracle of the dynamic setting.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` (hand-enumerated
order-1/order-2 curve tables under ``tests/golden/``, curve invariants, brute force, the
library sort); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CURVE_Z = 0
CURVE_HILBERT = 1
OMEGA = 30  # bits per coordinate on the GPU path
OMEGA3 = 21  # bits per coordinate of 3-D points on the GPU path (63-bit keys)


NORM_DISC = 0     # closed disc dx^2 + dy^2 <= delta^2 (problem statement)
NORM_SQUARE = 1   # closed square max(|dx|, |dy|) <= delta (the experiments' windows)


def norm_id(norm) -> int:
    if norm in (NORM_DISC, "disc", "l2"):
        return NORM_DISC
    if norm in (NORM_SQUARE, "square", "box", "linf"):
        return NORM_SQUARE
    raise ValueError(f"unknown norm {norm!r}")


def curve_id(curve) -> int:
    if curve in (CURVE_Z, "z", "Z", "morton"):
        return CURVE_Z
    if curve in (CURVE_HILBERT, "h", "H", "hilbert"):
        return CURVE_HILBERT
    raise ValueError(f"unknown curve {curve!r}")


def build_lib(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2, no target-specific flags) into liboracle.so."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp]
            )
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        u64, u32, i32, c_int = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int
        P = ctypes.c_void_p
        lib.oracle_key_z.restype = u64
        lib.oracle_key_z.argtypes = [u32, u32, c_int]
        lib.oracle_key_h.restype = u64
        lib.oracle_key_h.argtypes = [u32, u32, c_int]
        lib.oracle_keys.restype = None
        lib.oracle_keys.argtypes = [P, u64, c_int, c_int, P]
        lib.oracle_build.restype = c_int
        lib.oracle_build.argtypes = [P, u64, c_int, c_int, P, P, P]
        lib.oracle_lower_bound.restype = u64
        lib.oracle_lower_bound.argtypes = [P, u64, u64]
        lib.oracle_level.restype = c_int
        lib.oracle_level.argtypes = [ctypes.c_int64, c_int]
        lib.oracle_cells.restype = c_int
        lib.oracle_cells.argtypes = [i32, i32, i32, c_int, c_int, P, P, P]
        lib.oracle_cells_refined.restype = c_int
        lib.oracle_cells_refined.argtypes = [i32, i32, i32, c_int, c_int, c_int, P, P, c_int]
        lib.oracle_occupancy.restype = None
        lib.oracle_occupancy.argtypes = [P, u64, c_int, c_int, P]
        lib.oracle_cell_occupied.restype = c_int
        lib.oracle_cell_occupied.argtypes = [P, c_int, c_int, c_int, u64]
        lib.oracle_query_norm.restype = c_int
        lib.oracle_query_norm.argtypes = [P, P, P, u64, P, P, u64, c_int, c_int, c_int, P, P, P, P, c_int]
        lib.oracle_brute_norm.restype = c_int
        lib.oracle_brute_norm.argtypes = [P, u64, P, P, u64, c_int, c_int, P, P, P, c_int]
        lib.oracle_cells_refined_norm.restype = c_int
        lib.oracle_cells_refined_norm.argtypes = [i32, i32, i32, c_int, c_int, c_int, c_int, P, P, c_int]
        lib.oracle_key_z3.restype = u64
        lib.oracle_key_z3.argtypes = [u32, u32, u32, c_int]
        lib.oracle_build3.restype = c_int
        lib.oracle_build3.argtypes = [P, u64, c_int, P, P, P]
        lib.oracle_cells3.restype = c_int
        lib.oracle_cells3.argtypes = [i32, i32, i32, i32, c_int, P, P, P]
        lib.oracle_cells3_refined.restype = c_int
        lib.oracle_cells3_refined.argtypes = [i32, i32, i32, i32, c_int, c_int, P, P, c_int]
        lib.oracle_query3.restype = c_int
        lib.oracle_query3.argtypes = [P, P, P, u64, P, P, u64, c_int, P, P, P]
        lib.oracle_brute3.restype = c_int
        lib.oracle_brute3.argtypes = [P, u64, P, P, u64, c_int, P, P, P]
        lib.oracle_query.restype = c_int
        lib.oracle_query.argtypes = [P, P, P, u64, P, P, u64, c_int, c_int, P, P, P, P, c_int]
        lib.oracle_brute.restype = c_int
        lib.oracle_brute.argtypes = [P, u64, P, P, u64, c_int, P, P, P, c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------------------
# Keys (Alg. 2 for Z; Sec. 2.1 for Hilbert)
# --------------------------------------------------------------------------------------

def key_z(x: int, y: int, w: int = OMEGA) -> int:
    return int(_L().oracle_key_z(int(x), int(y), int(w)))


def key_h(x: int, y: int, w: int = OMEGA) -> int:
    return int(_L().oracle_key_h(int(x), int(y), int(w)))


def keys(xy: np.ndarray, w: int = OMEGA, curve="z") -> np.ndarray:
    xy = _c(xy, np.int32).reshape(-1, 2)
    out = np.empty(xy.shape[0], dtype=np.uint64)
    _L().oracle_keys(_ptr(xy), xy.shape[0], int(w), curve_id(curve), _ptr(out))
    return out


# --------------------------------------------------------------------------------------
# Construction and query
# --------------------------------------------------------------------------------------

class Index:
    """The sorted array A_P (Sec. 2): keys, input indices and coordinates sorted by (key, id)."""

    def __init__(self, keys, ids, xy, w, curve):
        self.keys, self.ids, self.xy, self.w, self.curve = keys, ids, xy, w, curve

    @property
    def n(self):
        return int(self.keys.shape[0])


def build(xy: np.ndarray, w: int = OMEGA, curve="z") -> Index:
    xy = _c(xy, np.int32).reshape(-1, 2)
    n = xy.shape[0]
    sk = np.empty(n, np.uint64)
    si = np.empty(n, np.uint32)
    sxy = np.empty((n, 2), np.int32)
    rc = _L().oracle_build(_ptr(xy), n, int(w), curve_id(curve), _ptr(sk), _ptr(si), _ptr(sxy))
    if rc != 0:
        raise MemoryError("oracle_build failed")
    return Index(sk, si, sxy, int(w), curve_id(curve))


def lower_bound(keys_sorted: np.ndarray, t: int) -> int:
    k = _c(keys_sorted, np.uint64)
    return int(_L().oracle_lower_bound(_ptr(k), k.shape[0], int(t)))


def level(delta: int, w: int = OMEGA) -> int:
    return int(_L().oracle_level(int(delta), int(w)))


def cells(qx: int, qy: int, delta: int, w: int = OMEGA, curve="z"):
    """Key intervals [lo, hi] of cells(Q), sorted by lo, and the level l."""
    lo = np.zeros(4, np.uint64)
    hi = np.zeros(4, np.uint64)
    lv = ctypes.c_int(0)
    cnt = _L().oracle_cells(int(qx), int(qy), int(delta), int(w), curve_id(curve),
                            _ptr(lo), _ptr(hi), ctypes.byref(lv))
    if cnt < 0:
        raise AssertionError("more than four cells")
    return [(int(lo[i]), int(hi[i])) for i in range(cnt)], int(lv.value)


def cells_refined(qx: int, qy: int, delta: int, w: int = OMEGA, curve="z", drop: int = 1, norm="disc"):
    """Key intervals of the cells one (or `drop`) quadtree levels below cells(Q) that contain
    an integer point of the closed window (disc or square), sorted by lo (not merged)."""
    maxc = (2 ** drop + 1) ** 2
    lo = np.zeros(maxc, np.uint64)
    hi = np.zeros(maxc, np.uint64)
    cnt = _L().oracle_cells_refined_norm(int(qx), int(qy), int(delta), int(w), curve_id(curve), int(drop),
                                         norm_id(norm), _ptr(lo), _ptr(hi), maxc)
    if cnt < 0:
        raise AssertionError("more cells than (2^drop + 1)^2")
    return [(int(lo[i]), int(hi[i])) for i in range(cnt)]


def occupancy_words(D: int) -> int:
    """32-bit words of the early-termination bitmap of depth D (all depths 0..D)."""
    return ((4 ** (D + 1) - 1) // 3 + 31) // 32


def occupancy(keys_arr: np.ndarray, D: int, w: int = OMEGA) -> np.ndarray:
    """The early-termination quadtree's booleans (Sec. 2.2), one bit per node, depth after
    depth (depth t from bit (4^t - 1) / 3)."""
    k = _c(keys_arr, np.uint64)
    out = np.empty(occupancy_words(D), np.uint32)
    _L().oracle_occupancy(_ptr(k), k.shape[0], int(w), int(D), _ptr(out))
    return out


def occupancy_bit(bits: np.ndarray, t: int, v: int) -> int:
    b = (4 ** t - 1) // 3 + int(v)
    return int((int(bits[b // 32]) >> (b % 32)) & 1)


def cell_occupied(bits: np.ndarray, D: int, l: int, lo: int, w: int = OMEGA) -> bool:
    b = _c(bits, np.uint32)
    return bool(_L().oracle_cell_occupied(_ptr(b), int(w), int(D), int(l), int(lo)))


def merge_abutting(intervals):
    out = []
    for a, z in intervals:
        if out and out[-1][1] + 1 == a:
            out[-1] = (out[-1][0], z)
        else:
            out.append((a, z))
    return out


def query(index: Index, q: np.ndarray, delta: np.ndarray, threads: int = 1, want_scanned=False,
          norm="disc"):
    """Alg. 1 for every query.  Returns (offsets u64[m+1], ids u32[offsets[m]]) with each
    query's ids in ascending (key, id) order, plus the scanned counts if asked.  norm: the
    closed disc of radius delta (default) or the closed square of half-side delta."""
    q = _c(q, np.int32).reshape(-1, 2)
    delta = _c(delta, np.int32).reshape(-1)
    m = q.shape[0]
    assert delta.shape[0] == m
    counts = np.empty(m, np.uint64)
    scanned = np.empty(m, np.uint64)
    L = _L()
    nm = norm_id(norm)
    L.oracle_query_norm(_ptr(index.keys), _ptr(index.ids), _ptr(index.xy), index.n, _ptr(q),
                        _ptr(delta), m, index.w, index.curve, nm, _ptr(counts), None, None,
                        _ptr(scanned), int(threads))
    offsets = np.zeros(m + 1, np.uint64)
    np.cumsum(counts, out=offsets[1:])
    ids = np.empty(int(offsets[m]), np.uint32)
    L.oracle_query_norm(_ptr(index.keys), _ptr(index.ids), _ptr(index.xy), index.n, _ptr(q),
                        _ptr(delta), m, index.w, index.curve, nm, None, _ptr(offsets), _ptr(ids),
                        None, int(threads))
    if want_scanned:
        return offsets, ids, scanned
    return offsets, ids


def brute(xy: np.ndarray, q: np.ndarray, delta: np.ndarray, w: int = OMEGA, threads: int = 1,
          norm="disc"):
    """O(n*m) reporting straight from the problem statement; ids ascending per query."""
    xy = _c(xy, np.int32).reshape(-1, 2)
    q = _c(q, np.int32).reshape(-1, 2)
    delta = _c(delta, np.int32).reshape(-1)
    m = q.shape[0]
    counts = np.empty(m, np.uint64)
    L = _L()
    nm = norm_id(norm)
    L.oracle_brute_norm(_ptr(xy), xy.shape[0], _ptr(q), _ptr(delta), m, int(w), nm, _ptr(counts), None,
                        None, int(threads))
    offsets = np.zeros(m + 1, np.uint64)
    np.cumsum(counts, out=offsets[1:])
    ids = np.empty(int(offsets[m]), np.uint32)
    L.oracle_brute_norm(_ptr(xy), xy.shape[0], _ptr(q), _ptr(delta), m, int(w), nm, None, _ptr(offsets),
                        _ptr(ids), int(threads))
    return offsets, ids


def sorted_lists(offsets: np.ndarray, ids: np.ndarray):
    """Per-query id lists, each sorted ascending (the unique part of a result)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    return [np.sort(ids[offsets[i]:offsets[i + 1]]) for i in range(offsets.shape[0] - 1)]


# --------------------------------------------------------------------------------------
# d = 3 (the Z curve in Z^3)
# --------------------------------------------------------------------------------------

def key_z3(x: int, y: int, z: int, w: int = OMEGA3) -> int:
    return int(_L().oracle_key_z3(int(x), int(y), int(z), int(w)))


def keys3(xyz: np.ndarray, w: int = OMEGA3) -> np.ndarray:
    xyz = _c(xyz, np.int64).reshape(-1, 3)
    return np.array([key_z3(a, b, c, w) for a, b, c in xyz], dtype=np.uint64)


def build3(xyz: np.ndarray, w: int = OMEGA3) -> Index:
    xyz = _c(xyz, np.int32).reshape(-1, 3)
    n = xyz.shape[0]
    sk = np.empty(n, np.uint64)
    si = np.empty(n, np.uint32)
    sxyz = np.empty((n, 3), np.int32)
    if _L().oracle_build3(_ptr(xyz), n, int(w), _ptr(sk), _ptr(si), _ptr(sxyz)) != 0:
        raise MemoryError("oracle_build3 failed")
    return Index(sk, si, sxyz, int(w), CURVE_Z)


def cells3(qx: int, qy: int, qz: int, delta: int, w: int = OMEGA3):
    """Key intervals [lo, hi] of cells(Q) in 3-D, sorted by lo, and the level l."""
    lo = np.zeros(8, np.uint64)
    hi = np.zeros(8, np.uint64)
    lv = ctypes.c_int(0)
    cnt = _L().oracle_cells3(int(qx), int(qy), int(qz), int(delta), int(w), _ptr(lo), _ptr(hi), ctypes.byref(lv))
    if cnt < 0:
        raise AssertionError("more than eight cells")
    return [(int(lo[i]), int(hi[i])) for i in range(cnt)], int(lv.value)


def cells3_refined(qx: int, qy: int, qz: int, delta: int, w: int = OMEGA3, drop: int = 1):
    """Key intervals of the cells `drop` levels below cells(Q) in 3-D that contain an integer
    point of the closed ball, sorted by lo (not merged)."""
    maxc = (2 ** drop + 1) ** 3
    lo = np.zeros(maxc, np.uint64)
    hi = np.zeros(maxc, np.uint64)
    cnt = _L().oracle_cells3_refined(int(qx), int(qy), int(qz), int(delta), int(w), int(drop), _ptr(lo), _ptr(hi), maxc)
    if cnt < 0:
        raise AssertionError("more cells than (2^drop + 1)^3")
    return [(int(lo[i]), int(hi[i])) for i in range(cnt)]


def query3(index: Index, q: np.ndarray, delta: np.ndarray):
    """Alg. 1 in 3-D (closed ball); offsets u64[m+1], ids in ascending (key, id) order."""
    q = _c(q, np.int32).reshape(-1, 3)
    delta = _c(delta, np.int32).reshape(-1)
    m = q.shape[0]
    counts = np.empty(m, np.uint64)
    L = _L()
    L.oracle_query3(_ptr(index.keys), _ptr(index.ids), _ptr(index.xy), index.n, _ptr(q), _ptr(delta), m,
                    index.w, _ptr(counts), None, None)
    offsets = np.zeros(m + 1, np.uint64)
    np.cumsum(counts, out=offsets[1:])
    ids = np.empty(int(offsets[m]), np.uint32)
    L.oracle_query3(_ptr(index.keys), _ptr(index.ids), _ptr(index.xy), index.n, _ptr(q), _ptr(delta), m,
                    index.w, None, _ptr(offsets), _ptr(ids))
    return offsets, ids


def brute3(xyz: np.ndarray, q: np.ndarray, delta: np.ndarray, w: int = OMEGA3):
    xyz = _c(xyz, np.int32).reshape(-1, 3)
    q = _c(q, np.int32).reshape(-1, 3)
    delta = _c(delta, np.int32).reshape(-1)
    m = q.shape[0]
    counts = np.empty(m, np.uint64)
    L = _L()
    L.oracle_brute3(_ptr(xyz), xyz.shape[0], _ptr(q), _ptr(delta), m, int(w), _ptr(counts), None, None)
    offsets = np.zeros(m + 1, np.uint64)
    np.cumsum(counts, out=offsets[1:])
    ids = np.empty(int(offsets[m]), np.uint32)
    L.oracle_brute3(_ptr(xyz), xyz.shape[0], _ptr(q), _ptr(delta), m, int(w), None, _ptr(offsets), _ptr(ids))
    return offsets, ids
