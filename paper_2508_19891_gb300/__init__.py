"""Python binding of libsfc (include/sfc.h): batched 2-D distance reporting over points sorted
along a space-filling curve, on GB300 (sm_103a).

Argument marshalling only.  Every function has the name of the C entry point it calls;
tensors are used for device memory and torch's current stream is passed as the CUDA stream.
Every step of the method runs in the library's CUDA kernels; there is no CPU path, and
importing this module fails loudly if the compiled library is missing.

dtypes at this boundary: points/queries int32 [n, 2]; radii int32 [m]; keys and offsets are
held in int64 tensors (keys are < 2^60 and offsets < 2^63, so the bit patterns are the
unsigned values); ids in int32 tensors (read them as uint32).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsfc.so")

SFC_OK = 0
SFC_ERR_INVALID = -1
SFC_ERR_OOM = -2
SFC_ERR_CAPACITY = -3
SFC_ERR_NOT_FOUND = -4
SFC_ERR_TIMEOUT = -5
SFC_ERR_CUDA = -6
SFC_ERR_STATE = -7

SFC_CURVE_Z = 0
SFC_CURVE_HILBERT = 1
SFC_BOUNDS_BINARY = 0
SFC_BOUNDS_LEARNED = 1
SFC_ROOT_PWL = 0
SFC_ROOT_MLP = 1

SFC_DEV_BAD_POINT = 0x1
SFC_DEV_BAD_QUERY = 0x2
SFC_DEV_CAPACITY = 0x4
SFC_DEV_TIMEOUT = 0x8
SFC_DEV_NOT_FOUND = 0x10


class sfc_options(ctypes.Structure):
    _fields_ = [("bounds", ctypes.c_int), ("leaves", ctypes.c_int), ("train_steps", ctypes.c_int),
                ("train_samples", ctypes.c_int), ("learning_rate", ctypes.c_float),
                ("chunk", ctypes.c_int), ("mask_budget_mb", ctypes.c_int),
                ("reorder_queries", ctypes.c_int), ("profile", ctypes.c_int), ("root", ctypes.c_int),
                ("cover_refine", ctypes.c_int), ("occupancy_depth", ctypes.c_int),
                ("query_norm", ctypes.c_int)]


SFC_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
SFC_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class sfc_allocator(ctypes.Structure):
    _fields_ = [("alloc", SFC_ALLOC_FN), ("free", SFC_FREE_FN), ("ctx", ctypes.c_void_p)]


class TorchAllocator:
    """sfc_allocator callbacks backed by PyTorch's CUDA caching allocator, so that torch owns
    all of an index's device memory (torch.cuda.memory_allocated() counts it).  Keeps a
    record of the blocks handed out (address -> bytes) and of every request and release."""

    def __init__(self, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.live = {}
        self.allocs = 0
        self.frees = 0
        self.bytes_requested = 0

        def _alloc(nbytes, stream, ctx):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device.index, int(stream or 0))
            except Exception:
                return None
            self.live[int(p)] = int(nbytes)
            self.allocs += 1
            self.bytes_requested += int(nbytes)
            return int(p)

        def _free(ptr, stream, ctx):
            self.live.pop(int(ptr), None)
            self.frees += 1
            torch.cuda.caching_allocator_delete(int(ptr))

        # the ctypes function objects must outlive every index built with this allocator
        self._alloc = SFC_ALLOC_FN(_alloc)
        self._free = SFC_FREE_FN(_free)
        self.struct = sfc_allocator(self._alloc, self._free, None)

    def owns(self, ptr: int, nbytes: int = 1) -> bool:
        """Whether [ptr, ptr + nbytes) lies inside a block handed out and not yet returned."""
        return any(a <= ptr and ptr + nbytes <= a + b for a, b in self.live.items())


class sfc_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double)]


class SfcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {sfc_status_string(status)} ({status})")


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsfc.so is not built ({LIB_PATH}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, u64, u32, i32, ci = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                ctypes.c_int)
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "sfc_default_options": (None, [ctypes.POINTER(sfc_options)]),
            "sfc_build": (ci, [PP, P, u64, ci, ctypes.POINTER(sfc_options), ctypes.POINTER(sfc_allocator), P]),
            "sfc_build_host": (ci, [PP, P, u64, ci, ctypes.POINTER(sfc_options), ctypes.POINTER(sfc_allocator), P]),
            "sfc_destroy": (None, [P]),
            "sfc_query_count": (ci, [P, P, P, u64, P, P]),
            "sfc_query_write": (ci, [P, P, P, u64, P, P, u64, P]),
            "sfc_query_batch": (ci, [P, P, P, u64, P, P, u64, P]),
            "sfc_query_batch_host": (ci, [P, P, P, u64, P, P, u64, P]),
            "sfc_reserve_queries": (ci, [P, u64, P]),
            "sfc_set_bounds_mode": (ci, [P, ci]),
            "sfc_set_cover": (ci, [P, ci]),
            "sfc_model_fence": (ci, [P, P, P, P]),
            "sfc_model_fence_fine": (ci, [P, P, P, P]),
            "sfc_build3": (ci, [PP, P, u64, ctypes.POINTER(sfc_options), ctypes.POINTER(sfc_allocator), P]),
            "sfc_build3_host": (ci, [PP, P, u64, ctypes.POINTER(sfc_options), ctypes.POINTER(sfc_allocator), P]),
            "sfc_index_dim": (ci, [P]),
            "sfc_keys3": (ci, [P, u64, P, P]),
            "sfc_set_query_norm": (ci, [P, ci]),
            "sfc_get_occupancy": (ci, [P, P, u64, P, P]),
            "sfc_query_cell_stats": (ci, [P, P, P, P]),
            "sfc_cover_refine": (ci, [P]),
            "sfc_query_max_intervals": (ci, [P]),
            "sfc_train_model": (ci, [P, P]),
            "sfc_model_hidden": (ci, []),
            "sfc_model_params": (ci, [ci]),
            "sfc_model_loss_grad": (ci, [ci, P, P, P, u64, P, P, P]),
            "sfc_model_adam_step": (ci, [P, P, P, P, ci, ci, ctypes.c_float, P]),
            "sfc_model_get": (ci, [P, P, P, P, P, P, P, P, P, P, P]),
            "sfc_model_stats": (ci, [P, P, P, P, P]),
            "sfc_update": (ci, [P, P, u64, P, u64, P, P]),
            "sfc_get_sorted": (ci, [P, PP, PP, PP, ctypes.POINTER(ctypes.c_uint64)]),
            "sfc_device_status": (ci, [P, ctypes.POINTER(ctypes.c_uint32), P]),
            "sfc_keys": (ci, [P, u64, ci, P, P]),
            "sfc_decode": (ci, [P, u64, ci, P, P]),
            "sfc_sort_pairs": (ci, [P, P, u64, P, P, P]),
            "sfc_exclusive_scan": (ci, [P, u64, P, P]),
            "sfc_exclusive_scan_noalloc": (ci, [P, u64, P, P]),
            "sfc_exclusive_scan_noalloc_status": (ci, [P, P]),
            "sfc_query_ranges": (ci, [P, P, P, u64, P, P, P, P, P, P]),
            "sfc_launch_count": (u64, []),
            "sfc_pool_bytes_in_use": (u64, []),
            "sfc_autotune": (ci, [P, P, P, u64, ci, P, P, P, P]),
            "sfc_set_tuning": (ci, [P, ci, ci, ci]),
            "sfc_rebuild": (ci, [P, P, u64, P]),
            "sfc_rebuild_host": (ci, [P, P, u64, P]),
            "sfc_reserve": (ci, [P, u64, u64, P]),
            "sfc_graph_capture": (ci, [P, ctypes.c_uint, P, u64, P, P, u64, P, P, u64, PP, P]),
            "sfc_graph_launch": (ci, [P, P]),
            "sfc_graph_destroy": (None, [P]),
            "sfc_query_stats": (ci, [P, P, P, P, P]),
            "sfc_profile_enable": (ci, [P, ci]),
            "sfc_profile_read": (ci, [P, P, ci, P, ci, P]),
            "sfc_status_string": (ctypes.c_char_p, [ci]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# --------------------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------------------

def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    if a is None:
        return None
    return ctypes.c_void_p(a.ctypes.data)


def _check(status, what):
    if status != SFC_OK:
        raise SfcError(status, what)


def _curve(c):
    if c in (SFC_CURVE_Z, "z", "Z", "morton"):
        return SFC_CURVE_Z
    if c in (SFC_CURVE_HILBERT, "h", "H", "hilbert"):
        return SFC_CURVE_HILBERT
    raise ValueError(f"unknown curve {c!r}")


def _bounds(b):
    if b in (SFC_BOUNDS_BINARY, "binary"):
        return SFC_BOUNDS_BINARY
    if b in (SFC_BOUNDS_LEARNED, "learned"):
        return SFC_BOUNDS_LEARNED
    raise ValueError(f"unknown bounds mode {b!r}")


def _pts(t, dim: int = 2):
    assert t.dtype == torch.int32 and t.dim() == 2 and t.shape[1] == dim, f"points must be int32 [n, {dim}]"
    return t.contiguous()


class _CudaView:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3,
                                         "strides": None, "stream": None}


def sfc_status_string(status: int) -> str:
    return lib().sfc_status_string(int(status)).decode()


def _root(r):
    if r in (SFC_ROOT_PWL, "pwl"):
        return SFC_ROOT_PWL
    if r in (SFC_ROOT_MLP, "mlp"):
        return SFC_ROOT_MLP
    raise ValueError(f"unknown root kind {r!r}")


def sfc_default_options(**overrides) -> sfc_options:
    o = sfc_options()
    lib().sfc_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "bounds":
            v = _bounds(v)
        if k == "root":
            v = _root(v)
        if k == "query_norm":
            v = _norm(v)
        setattr(o, k, v)
    return o


def sfc_launch_count() -> int:
    return int(lib().sfc_launch_count())


def sfc_pool_bytes_in_use() -> int:
    """Device bytes held from the library's own pool (not from a caller's allocator)."""
    return int(lib().sfc_pool_bytes_in_use())


# --------------------------------------------------------------------------------------
# index
# --------------------------------------------------------------------------------------

class Index:
    """Owns an sfc_index handle (and keeps the allocator it was built with alive)."""

    def __init__(self, handle: ctypes.c_void_p, curve: int, device, dim: int = 2, allocator=None):
        self._h = handle
        self.curve = curve
        self.device = device
        self.dim = dim
        self.allocator = allocator

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().sfc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _alloc_ptr(allocator):
    return ctypes.byref(allocator.struct) if allocator is not None else None


def sfc_build(points: torch.Tensor, curve="z", options: sfc_options | None = None, stream=None,
              allocator: TorchAllocator | None = None, **opts) -> Index:
    """allocator: e.g. TorchAllocator() to take all of the index's device memory from
    PyTorch's caching allocator (None: the library's own pool)."""
    points = _pts(points)
    o = options if options is not None else sfc_default_options(**opts)
    h = ctypes.c_void_p()
    _check(lib().sfc_build(ctypes.byref(h), _dptr(points), points.shape[0], _curve(curve),
                           ctypes.byref(o), _alloc_ptr(allocator), _stream(stream)), "sfc_build")
    return Index(h, _curve(curve), points.device, allocator=allocator)


def sfc_build_host(points: np.ndarray, curve="z", options: sfc_options | None = None, stream=None,
                   allocator: TorchAllocator | None = None, **opts) -> Index:
    points = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 2)
    o = options if options is not None else sfc_default_options(**opts)
    h = ctypes.c_void_p()
    _check(lib().sfc_build_host(ctypes.byref(h), _hptr(points), points.shape[0], _curve(curve),
                                ctypes.byref(o), _alloc_ptr(allocator), _stream(stream)), "sfc_build_host")
    return Index(h, _curve(curve), torch.device("cuda", torch.cuda.current_device()), allocator=allocator)


def sfc_build3(points: torch.Tensor, options: sfc_options | None = None, stream=None,
               allocator: TorchAllocator | None = None, **opts) -> Index:
    """3-D index of int32 [n, 3] points (Z curve in Z^3, coordinates in [0, 2^21))."""
    points = _pts(points, 3)
    o = options if options is not None else sfc_default_options(**opts)
    h = ctypes.c_void_p()
    _check(lib().sfc_build3(ctypes.byref(h), _dptr(points), points.shape[0], ctypes.byref(o),
                            _alloc_ptr(allocator), _stream(stream)), "sfc_build3")
    return Index(h, SFC_CURVE_Z, points.device, dim=3, allocator=allocator)


def sfc_build3_host(points: np.ndarray, options: sfc_options | None = None, stream=None,
                    allocator: TorchAllocator | None = None, **opts) -> Index:
    points = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 3)
    o = options if options is not None else sfc_default_options(**opts)
    h = ctypes.c_void_p()
    _check(lib().sfc_build3_host(ctypes.byref(h), _hptr(points), points.shape[0], ctypes.byref(o),
                                 _alloc_ptr(allocator), _stream(stream)), "sfc_build3_host")
    return Index(h, SFC_CURVE_Z, torch.device("cuda", torch.cuda.current_device()), dim=3, allocator=allocator)


def sfc_keys3(points: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    points = _pts(points, 3)
    if out is None:
        out = torch.empty(points.shape[0], dtype=torch.int64, device=points.device)
    _check(lib().sfc_keys3(_dptr(points), points.shape[0], _dptr(out), _stream(stream)), "sfc_keys3")
    return out


def sfc_destroy(index: Index):
    index.close()


def sfc_rebuild(index: Index, points: torch.Tensor, stream=None):
    points = _pts(points, index.dim)
    _check(lib().sfc_rebuild(index.handle, _dptr(points), points.shape[0], _stream(stream)), "sfc_rebuild")


def sfc_rebuild_host(index: Index, points: np.ndarray, stream=None):
    """Rebuilds the index over host points (int32 [n, 2], or [n, 3] for a 3-D index); the
    array must stay unchanged until the stream has run the copy when it is page-locked."""
    points = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, index.dim)
    _check(lib().sfc_rebuild_host(index.handle, _hptr(points), points.shape[0], _stream(stream)),
           "sfc_rebuild_host")


def sfc_reserve(index: Index, n_max: int, m_max: int, stream=None):
    _check(lib().sfc_reserve(index.handle, int(n_max), int(m_max), _stream(stream)), "sfc_reserve")


SFC_GRAPH_REBUILD = 0x1
SFC_GRAPH_QUERY = 0x2


class Graph:
    """A captured pipeline (sfc_graph); keeps the tensors it reads and writes alive."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(lib().sfc_graph_launch(self._h, _stream(stream)), "sfc_graph_launch")

    def close(self):
        if self._h:
            lib().sfc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfc_graph_capture(index: Index, points: torch.Tensor | None, q: torch.Tensor | None,
                      delta: torch.Tensor | None, out_offsets: torch.Tensor | None,
                      out_ids: torch.Tensor | None, capacity: int | None = None, stream=None) -> Graph:
    flags = (SFC_GRAPH_REBUILD if points is not None else 0) | (SFC_GRAPH_QUERY if q is not None else 0)
    n = points.shape[0] if points is not None else 0
    m = q.shape[0] if q is not None else 0
    cap = (out_ids.numel() if out_ids is not None else 0) if capacity is None else int(capacity)
    h = ctypes.c_void_p()
    _check(lib().sfc_graph_capture(index.handle, flags, _dptr(points), n, _dptr(q), _dptr(delta), m,
                                   _dptr(out_offsets), _dptr(out_ids) if (out_ids is not None and out_ids.numel()) else None,
                                   cap, ctypes.byref(h), _stream(stream)), "sfc_graph_capture")
    return Graph(h, (index, points, q, delta, out_offsets, out_ids))


def sfc_query_count(index: Index, q: torch.Tensor, delta: torch.Tensor,
                    out_offsets: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    q = _pts(q, index.dim)
    delta = delta.contiguous()
    m = q.shape[0]
    if out_offsets is None:
        out_offsets = torch.empty(m + 1, dtype=torch.int64, device=q.device)
    _check(lib().sfc_query_count(index.handle, _dptr(q), _dptr(delta), m, _dptr(out_offsets),
                                 _stream(stream)), "sfc_query_count")
    return out_offsets


def sfc_query_write(index: Index, q: torch.Tensor, delta: torch.Tensor, out_offsets: torch.Tensor,
                    out_ids: torch.Tensor, capacity: int | None = None, stream=None) -> torch.Tensor:
    cap = out_ids.numel() if capacity is None else int(capacity)
    _check(lib().sfc_query_write(index.handle, _dptr(q), _dptr(delta), q.shape[0], _dptr(out_offsets),
                                 _dptr(out_ids) if out_ids.numel() else None, cap, _stream(stream)),
           "sfc_query_write")
    return out_ids


def sfc_query_batch(index: Index, q: torch.Tensor, delta: torch.Tensor, out_offsets: torch.Tensor,
                    out_ids: torch.Tensor, capacity: int | None = None, stream=None):
    q = _pts(q, index.dim)
    delta = delta.contiguous()
    cap = out_ids.numel() if capacity is None else int(capacity)
    _check(lib().sfc_query_batch(index.handle, _dptr(q), _dptr(delta), q.shape[0], _dptr(out_offsets),
                                 _dptr(out_ids) if out_ids.numel() else None, cap, _stream(stream)),
           "sfc_query_batch")
    return out_offsets, out_ids


def query(index: Index, q: torch.Tensor, delta: torch.Tensor, stream=None):
    """Count, read the total, allocate, write: returns (offsets int64[m+1], ids int32[total])."""
    q = _pts(q, index.dim)
    delta = delta.contiguous()
    off = sfc_query_count(index, q, delta, stream=stream)
    total = int(off[-1].item())
    ids = torch.empty(total, dtype=torch.int32, device=q.device)
    sfc_query_write(index, q, delta, off, ids, stream=stream)
    return off, ids


def sfc_query_batch_host(index: Index, q: np.ndarray, delta: np.ndarray, capacity: int,
                         out_offsets: np.ndarray | None = None, out_ids: np.ndarray | None = None,
                         stream=None):
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1, index.dim)
    delta = np.ascontiguousarray(delta, dtype=np.int32).reshape(-1)
    m = q.shape[0]
    if out_offsets is None:
        out_offsets = np.empty(m + 1, np.uint64)
    if out_ids is None:
        out_ids = np.empty(max(int(capacity), 1), np.uint32)
    st = lib().sfc_query_batch_host(index.handle, _hptr(q), _hptr(delta), m, _hptr(out_offsets),
                                    _hptr(out_ids), int(capacity), _stream(stream))
    _check(st, "sfc_query_batch_host")
    return out_offsets, out_ids[:int(out_offsets[m])]


def sfc_autotune(index: Index, q: torch.Tensor, delta: torch.Tensor, force: bool = False, stream=None) -> dict:
    q = _pts(q, index.dim)
    delta = delta.contiguous()
    c, b, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().sfc_autotune(index.handle, _dptr(q), _dptr(delta), q.shape[0], int(bool(force)), ctypes.byref(c),
                              ctypes.byref(b), ctypes.byref(w), _stream(stream)), "sfc_autotune")
    return {"chunk": c.value, "batch": b.value, "qbatch": w.value,
            "cover": int(lib().sfc_cover_refine(index.handle))}


def sfc_set_tuning(index: Index, chunk: int, batch: int, qbatch: int):
    _check(lib().sfc_set_tuning(index.handle, int(chunk), int(batch), int(qbatch)), "sfc_set_tuning")


def sfc_reserve_queries(index: Index, m: int, stream=None):
    _check(lib().sfc_reserve_queries(index.handle, int(m), _stream(stream)), "sfc_reserve_queries")


def sfc_set_bounds_mode(index: Index, mode):
    _check(lib().sfc_set_bounds_mode(index.handle, _bounds(mode)), "sfc_set_bounds_mode")


def sfc_get_occupancy(index: Index, depth: int, stream=None) -> torch.Tensor:
    """The early-termination bitmap as int32 words (bit layout in include/sfc.h)."""
    words = ((4 ** (depth + 1) - 1) // 3 + 31) // 32
    out = torch.empty(words, dtype=torch.int32, device=index.device)
    d = ctypes.c_int()
    _check(lib().sfc_get_occupancy(index.handle, _dptr(out), words, ctypes.byref(d), _stream(stream)),
           "sfc_get_occupancy")
    return out


def sfc_query_cell_stats(index: Index, stream=None) -> dict:
    c, e = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().sfc_query_cell_stats(index.handle, ctypes.byref(c), ctypes.byref(e), _stream(stream)),
           "sfc_query_cell_stats")
    return {"cells": c.value, "empty": e.value}


SFC_NORM_DISC = 0
SFC_NORM_SQUARE = 1


def _norm(norm) -> int:
    if norm in (SFC_NORM_DISC, "disc", "l2"):
        return SFC_NORM_DISC
    if norm in (SFC_NORM_SQUARE, "square", "box", "linf"):
        return SFC_NORM_SQUARE
    raise ValueError(f"unknown query norm {norm!r}")


def sfc_set_query_norm(index: Index, norm):
    _check(lib().sfc_set_query_norm(index.handle, _norm(norm)), "sfc_set_query_norm")


def sfc_set_cover(index: Index, refine: int):
    _check(lib().sfc_set_cover(index.handle, int(refine)), "sfc_set_cover")


def sfc_cover_refine(index: Index) -> int:
    return int(lib().sfc_cover_refine(index.handle))


def sfc_query_max_intervals(index: Index) -> int:
    return int(lib().sfc_query_max_intervals(index.handle))


def sfc_train_model(index: Index, stream=None):
    _check(lib().sfc_train_model(index.handle, _stream(stream)), "sfc_train_model")


def sfc_model_hidden() -> int:
    return int(lib().sfc_model_hidden())


def sfc_model_params(root="pwl") -> int:
    return int(lib().sfc_model_params(_root(root)))


def sfc_model_loss_grad(params: np.ndarray, keys: torch.Tensor, y: torch.Tensor, root="pwl", stream=None):
    npar = sfc_model_params(root)
    p = np.ascontiguousarray(params, np.float32)
    assert p.shape == (npar,)
    loss = np.zeros(1, np.float32)
    grad = np.zeros(npar, np.float32)
    _check(lib().sfc_model_loss_grad(_root(root), _hptr(p), _dptr(keys), _dptr(y), keys.numel(), _hptr(loss),
                                     _hptr(grad), _stream(stream)), "sfc_model_loss_grad")
    return float(loss[0]), grad


def sfc_model_adam_step(params, m, v, grad, t: int, lr: float, stream=None):
    p = np.array(params, np.float32)
    mm = np.array(m, np.float32)
    vv = np.array(v, np.float32)
    g = np.ascontiguousarray(grad, np.float32)
    _check(lib().sfc_model_adam_step(_hptr(p), _hptr(mm), _hptr(vv), _hptr(g), p.size, int(t), float(lr),
                                     _stream(stream)), "sfc_model_adam_step")
    return p, mm, vv


def sfc_model_get(index: Index, stream=None) -> dict:
    nl = ctypes.c_int(0)
    kind = ctypes.c_int(0)
    _check(lib().sfc_model_get(index.handle, ctypes.byref(kind), None, ctypes.byref(nl), None, None, None, None,
                               None, None, _stream(stream)), "sfc_model_get")
    L = nl.value
    out = {"root": "mlp" if kind.value == SFC_ROOT_MLP else "pwl",
           "params": np.zeros(sfc_model_params(kind.value), np.float32), "first": np.zeros(L, np.uint32),
           "end": np.zeros(L, np.uint32), "slope": np.zeros(L, np.float32),
           "icpt": np.zeros(L, np.float32), "err_lo": np.zeros(L, np.int32),
           "err_hi": np.zeros(L, np.int32)}
    _check(lib().sfc_model_get(index.handle, None, _hptr(out["params"]), ctypes.byref(nl),
                               _hptr(out["first"]), _hptr(out["end"]), _hptr(out["slope"]),
                               _hptr(out["icpt"]), _hptr(out["err_lo"]), _hptr(out["err_hi"]),
                               _stream(stream)), "sfc_model_get")
    return out


def sfc_model_fence(index: Index, stream=None) -> np.ndarray:
    """uint64[leaves, 16]: the fence keys of every leaf."""
    nl = ctypes.c_int(0)
    _check(lib().sfc_model_fence(index.handle, None, ctypes.byref(nl), _stream(stream)), "sfc_model_fence")
    out = np.zeros((nl.value, 16), np.uint64)
    _check(lib().sfc_model_fence(index.handle, _hptr(out), ctypes.byref(nl), _stream(stream)), "sfc_model_fence")
    return out


def sfc_model_fence_fine(index: Index, stream=None) -> np.ndarray:
    """uint64[leaves, 256]: the fine fence keys of every leaf."""
    nl = ctypes.c_int(0)
    _check(lib().sfc_model_fence_fine(index.handle, None, ctypes.byref(nl), _stream(stream)), "sfc_model_fence_fine")
    out = np.zeros((nl.value, 256), np.uint64)
    _check(lib().sfc_model_fence_fine(index.handle, _hptr(out), ctypes.byref(nl), _stream(stream)),
           "sfc_model_fence_fine")
    return out


def sfc_model_stats(index: Index, stream=None):
    e, m, w = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().sfc_model_stats(index.handle, ctypes.byref(e), ctypes.byref(m), ctypes.byref(w),
                                 _stream(stream)), "sfc_model_stats")
    return {"endpoints": e.value, "misses": m.value, "window_sum": w.value}


def sfc_query_stats(index: Index, stream=None):
    s, g, h = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().sfc_query_stats(index.handle, ctypes.byref(s), ctypes.byref(g), ctypes.byref(h),
                                 _stream(stream)), "sfc_query_stats")
    return {"scanned": s.value, "chunks": g.value, "hits": h.value}


def sfc_profile_enable(index: Index, on: bool = True):
    _check(lib().sfc_profile_enable(index.handle, int(bool(on))), "sfc_profile_enable")


def sfc_profile_read(index: Index, reset: bool = True, stream=None) -> dict:
    """{step name: (runs, total ms)} of the steps recorded since the last reset."""
    buf = (sfc_profile_entry * 64)()
    cnt = ctypes.c_int(0)
    _check(lib().sfc_profile_read(index.handle, buf, 64, ctypes.byref(cnt), int(bool(reset)),
                                  _stream(stream)), "sfc_profile_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(min(cnt.value, 64))}


def sfc_update(index: Index, inserts: torch.Tensor | None, delete_ids: torch.Tensor | None,
               stream=None) -> int:
    first = ctypes.c_uint32(0)
    ins = _pts(inserts) if inserts is not None and inserts.numel() else None
    dels = delete_ids.contiguous() if delete_ids is not None and delete_ids.numel() else None
    _check(lib().sfc_update(index.handle, _dptr(ins), 0 if ins is None else ins.shape[0], _dptr(dels),
                            0 if dels is None else dels.numel(), ctypes.byref(first), _stream(stream)),
           "sfc_update")
    return int(first.value)


def sfc_get_sorted(index: Index, copy: bool = True):
    """(keys int64[n], ids int32[n], coordinates int32[n, 2] or, for a 3-D index, int32[n, 4]
    records x, y, z, 0) of the sorted array."""
    k, i, x = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    n = ctypes.c_uint64()
    _check(lib().sfc_get_sorted(index.handle, ctypes.byref(k), ctypes.byref(i), ctypes.byref(x),
                                ctypes.byref(n)), "sfc_get_sorted")
    n = n.value
    dev = index.device
    c = 4 if index.dim == 3 else 2
    if n == 0:
        return (torch.empty(0, dtype=torch.int64, device=dev), torch.empty(0, dtype=torch.int32, device=dev),
                torch.empty((0, c), dtype=torch.int32, device=dev))
    with torch.cuda.device(dev):
        kt = torch.as_tensor(_CudaView(k.value, (n,), "<i8"), device=dev)
        it = torch.as_tensor(_CudaView(i.value, (n,), "<i4"), device=dev)
        xt = torch.as_tensor(_CudaView(x.value, (n, c), "<i4"), device=dev)
    if copy:
        return kt.clone(), it.clone(), xt.clone()
    return kt, it, xt


def sfc_device_status(index: Index, stream=None):
    bits = ctypes.c_uint32(0)
    st = lib().sfc_device_status(index.handle, ctypes.byref(bits), _stream(stream))
    return int(st), int(bits.value)


def sfc_keys(points: torch.Tensor, curve="z", out: torch.Tensor | None = None, stream=None):
    points = _pts(points)
    if out is None:
        out = torch.empty(points.shape[0], dtype=torch.int64, device=points.device)
    _check(lib().sfc_keys(_dptr(points), points.shape[0], _curve(curve), _dptr(out), _stream(stream)),
           "sfc_keys")
    return out


def sfc_decode(keys: torch.Tensor, curve="z", out: torch.Tensor | None = None, stream=None):
    keys = keys.contiguous()
    if out is None:
        out = torch.empty((keys.numel(), 2), dtype=torch.int32, device=keys.device)
    _check(lib().sfc_decode(_dptr(keys), keys.numel(), _curve(curve), _dptr(out), _stream(stream)),
           "sfc_decode")
    return out


def sfc_sort_pairs(keys: torch.Tensor, ids: torch.Tensor | None = None, stream=None):
    keys = keys.contiguous()
    n = keys.numel()
    ko = torch.empty_like(keys)
    io = torch.empty(n, dtype=torch.int32, device=keys.device)
    _check(lib().sfc_sort_pairs(_dptr(keys), _dptr(ids.contiguous()) if ids is not None else None, n,
                                _dptr(ko), _dptr(io), _stream(stream)), "sfc_sort_pairs")
    return ko, io


def sfc_exclusive_scan(x: torch.Tensor, stream=None):
    x = x.contiguous()
    out = torch.empty(x.numel() + 1, dtype=torch.int64, device=x.device)
    _check(lib().sfc_exclusive_scan(_dptr(x), x.numel(), _dptr(out), _stream(stream)), "sfc_exclusive_scan")
    return out


def sfc_exclusive_scan_noalloc(x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Exclusive scan through the entry point that allocates no device memory (the output
    buffer, if not given, is allocated here by torch, outside the library call).  x: 32-bit
    integers (read as uint32); out: int64, contiguous, on x's device, at least n + 1 long."""
    if x.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise ValueError(f"x must hold 32-bit integers, not {x.dtype}")
    x = x.contiguous()
    if out is None:
        out = torch.empty(x.numel() + 1, dtype=torch.int64, device=x.device)
    if out.dtype != torch.int64:
        raise ValueError(f"out must be int64, not {out.dtype}")
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    if out.device != x.device or not x.is_cuda:
        raise ValueError(f"x and out must be on the same CUDA device ({x.device}, {out.device})")
    if out.numel() < x.numel() + 1:
        raise ValueError(f"out holds {out.numel()} elements; the scan of {x.numel()} writes {x.numel() + 1}")
    _check(lib().sfc_exclusive_scan_noalloc(_dptr(x), x.numel(), _dptr(out), _stream(stream)),
           "sfc_exclusive_scan_noalloc")
    return out


def sfc_exclusive_scan_noalloc_status(stream=None) -> int:
    """Status bits of the most recent no-allocation scan on the current device (synchronises
    the stream); raises SfcError(SFC_ERR_TIMEOUT) if a look-back wait gave up."""
    bits = ctypes.c_uint32(0)
    _check(lib().sfc_exclusive_scan_noalloc_status(ctypes.byref(bits), _stream(stream)),
           "sfc_exclusive_scan_noalloc_status")
    return int(bits.value)


def sfc_query_ranges(index: Index, q: torch.Tensor, delta: torch.Tensor, stream=None):
    q = _pts(q, index.dim)
    delta = delta.contiguous()
    m = q.shape[0]
    dev = q.device
    k = sfc_query_max_intervals(index)
    lo = torch.empty(k * m, dtype=torch.int64, device=dev)
    hi = torch.empty(k * m, dtype=torch.int64, device=dev)
    b = torch.empty(k * m, dtype=torch.int32, device=dev)
    e = torch.empty(k * m, dtype=torch.int32, device=dev)
    c = torch.empty(m, dtype=torch.int32, device=dev)
    _check(lib().sfc_query_ranges(index.handle, _dptr(q), _dptr(delta), m, _dptr(lo), _dptr(hi), _dptr(b),
                                  _dptr(e), _dptr(c), _stream(stream)), "sfc_query_ranges")
    return lo, hi, b, e, c
