"""Python binding of libesg, the GB300 (sm_103a) implementation of ESG
range-filtered approximate k-NN search (arxiv 2504.04018).

Argument marshalling only: every step of the search runs in the CUDA kernels
of ``libesg.so`` behind the C ABI of ``include/esg.h``; the functions here
keep its names. PyTorch provides device memory and streams. There is no CPU
fallback: importing a compute function without the compiled library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from . import _build_lib

__all__ = [
    "load_library", "Index", "esg_build", "esg_index_import", "esg_index_export", "esg_free",
    "esg_decompose_batch", "esg_search_batch", "esg_bruteforce_filtered_knn", "esg_bruteforce_plan",
    "esg_attr_to_rank_range", "esg_save", "esg_load", "EsgError", "METRIC", "STORAGE",
    "PIECE_GRAPH", "PIECE_SCAN", "Q_INVALID", "Q_TRUNCATED", "Q_OVERFLOW",
]

METRIC = {"l2": 0, "ip": 1}
STORAGE = {"f32": 0, "bf16": 1, "fp8": 2}
LAYOUT = {"tree": 0, "prefix": 1}
PIECE_NONE, PIECE_GRAPH, PIECE_SCAN = 0, 1, 2
Q_INVALID, Q_TRUNCATED, Q_OVERFLOW = 1, 2, 4

EXPORTED = [
    "esg_build_params_default", "esg_search_params_default", "esg_build", "esg_index_import",
    "esg_index_info", "esg_index_layout", "esg_index_export", "esg_free", "esg_decompose_batch", "esg_search_batch",
    "esg_bruteforce_filtered_knn", "esg_bruteforce_plan", "esg_attr_to_rank_range", "esg_save", "esg_load",
    "esg_status_str", "esg_last_error", "esg_profile_enable", "esg_profile_read", "esg_profile_tensor_work",
    "esg_index_export_storage", "esg_index_add_storage", "esg_batch_create", "esg_batch_buffers",
    "esg_batch_run", "esg_batch_free", "esg_autotune", "esg_search_batch_noalloc",
    "esg_train_params_default", "esg_train_predictor", "esg_predictor_set", "esg_predictor_get",
    "esg_mlp_num_params", "esg_mlp_num_features", "esg_mlp_blob_size", "esg_mlp_forward", "esg_mlp_loss_grad", "esg_mlp_adam_step",
    "esg_query_features", "esg_query_budget", "esg_index_export_rows",
]


class EsgError(RuntimeError):
    pass


class _BuildParams(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("n_entries", ctypes.c_int32),
                ("ef_construction", ctypes.c_int32), ("batch_div", ctypes.c_int32),
                ("fanout", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("layout", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _TrainParams(ctypes.Structure):
    _fields_ = [("target_recall", ctypes.c_float), ("per_query_recall", ctypes.c_float),
                ("quantile", ctypes.c_float), ("lr", ctypes.c_float), ("val_fraction", ctypes.c_float),
                ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("ef_lo", ctypes.c_int32),
                ("ef_hi", ctypes.c_int32), ("traversal", ctypes.c_int32), ("per_k_class", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class _SearchParams(ctypes.Structure):
    _fields_ = [("ef", ctypes.c_int32), ("max_expansions", ctypes.c_int32),
                ("rerank", ctypes.c_int32), ("use_learned", ctypes.c_int32),
                ("traversal", ctypes.c_int32), ("width", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("hash_slots", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("post_root", ctypes.c_int32),
                ("max_registers", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libesg.so (compiling it with nvcc first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build_lib.LIB
    if build_if_missing:
        path = _build_lib.build()
    if not os.path.exists(path):
        raise EsgError(f"libesg.so not built: {path}")
    lib = ctypes.CDLL(path)
    lib.esg_build_params_default.restype = _BuildParams
    lib.esg_search_params_default.restype = _SearchParams
    lib.esg_build.argtypes = [_P, _I64, _I32, _P, ctypes.POINTER(_BuildParams), ctypes.POINTER(_P)]
    lib.esg_index_import.argtypes = [_P, _P, _I64, _I32, _I32, _I32, _I32, _I32, _P, _I32, _I32, _P, _I32,
                                     _I32, ctypes.POINTER(_P)]
    lib.esg_index_info.argtypes = [_P] + [_P] * 8
    lib.esg_index_layout.argtypes = [_P] + [_P] * 4
    lib.esg_index_export.argtypes = [_P, _P, _P, _P]
    lib.esg_index_export_rows.argtypes = [_P, _I32, _I64, _I64, _P]
    lib.esg_index_export_storage.argtypes = [_P, _I32, _P, _P]
    lib.esg_index_add_storage.argtypes = [_P, _I32]
    lib.esg_free.argtypes = [_P]
    lib.esg_free.restype = None
    lib.esg_decompose_batch.argtypes = [_I64, _I32, _I32, _I32, _I32, _P, _P, _I64, _P, _P, _P]
    lib.esg_search_batch.argtypes = [_P, _P, _I64, _P, _P, _P, _I32, ctypes.POINTER(_SearchParams),
                                     _P, _P, _P, _P, _P, _P]
    lib.esg_bruteforce_filtered_knn.argtypes = [_P, _I64, _I32, _I32, _P, _I64, _P, _P, _I32, _P, _P,
                                                _P, _P]
    lib.esg_attr_to_rank_range.argtypes = [_P, _P, _P, _I64, _P, _P]
    lib.esg_bruteforce_plan.argtypes = [_I64, _I32, _P, _P, _I64, _I32, _P, _P, _P, _P, _P]
    lib.esg_save.argtypes = [_P, ctypes.c_char_p]
    lib.esg_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(_P)]
    lib.esg_profile_enable.argtypes = [_I32]
    lib.esg_profile_read.argtypes = [_P, _P, _P, _I32]
    lib.esg_profile_tensor_work.argtypes = [_P, _I32]
    lib.esg_train_params_default.restype = _TrainParams
    lib.esg_train_predictor.argtypes = [_P, _P, _I64, _P, _P, _P, _I32, _P, _P,
                                        ctypes.POINTER(_TrainParams), _P, _P]
    lib.esg_predictor_set.argtypes = [_P, _P, _I32, _I32]
    lib.esg_predictor_get.argtypes = [_P, _P, _P, _P]
    lib.esg_mlp_num_params.restype = _I32
    lib.esg_mlp_num_features.restype = _I32
    lib.esg_mlp_blob_size.restype = _I32
    lib.esg_mlp_forward.argtypes = [_P, _P, _P, _P, _I64, _P, _P]
    lib.esg_mlp_loss_grad.argtypes = [_P, _P, _P, _P, _P, _I64, ctypes.c_float, _P, _P, _P]
    lib.esg_mlp_adam_step.argtypes = [_P, _P, _P, _P, _I32, ctypes.c_float, _P]
    lib.esg_query_features.argtypes = [_P, _P, _I64, _P, _P, _P, _I32, _P, _P]
    lib.esg_query_budget.argtypes = [_P, _P, _I64, _P, _P, _P, _I32, _I32, _P, _P, _P]
    lib.esg_search_batch_noalloc.argtypes = [_P, _P, _I64, _P, _P, _P, _I32,
                                             ctypes.POINTER(_SearchParams), _P, _P, _P, _P, _P, _P]
    lib.esg_batch_create.argtypes = [_P, _I64, _I32, _I32, ctypes.POINTER(_SearchParams), ctypes.POINTER(_P)]
    lib.esg_batch_buffers.argtypes = [_P] + [ctypes.POINTER(_P)] * 9
    lib.esg_batch_run.argtypes = [_P, _I64, _P]
    lib.esg_batch_free.argtypes = [_P]
    lib.esg_batch_free.restype = None
    lib.esg_autotune.argtypes = [_P, _P, _I64, _P, _P, _P, _I32, _P, _P, ctypes.c_float,
                                 ctypes.POINTER(_SearchParams), ctypes.POINTER(_SearchParams), _P, _P]
    lib.esg_status_str.restype = ctypes.c_char_p
    lib.esg_status_str.argtypes = [_I32]
    lib.esg_last_error.restype = ctypes.c_char_p
    for name in ["esg_build", "esg_index_import", "esg_index_info", "esg_index_layout", "esg_index_export",
                 "esg_index_export_rows",
                 "esg_decompose_batch", "esg_search_batch", "esg_bruteforce_filtered_knn",
                 "esg_attr_to_rank_range", "esg_save", "esg_load", "esg_profile_enable",
                 "esg_profile_read", "esg_profile_tensor_work", "esg_index_export_storage", "esg_index_add_storage",
                 "esg_batch_create", "esg_batch_buffers", "esg_batch_run", "esg_autotune",
                 "esg_search_batch_noalloc", "esg_train_predictor", "esg_predictor_set",
                 "esg_predictor_get", "esg_mlp_forward", "esg_mlp_loss_grad", "esg_mlp_adam_step",
                 "esg_query_features", "esg_query_budget"]:
        getattr(lib, name).restype = _I32
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        lib = load_library()
        raise EsgError(f"{what}: {lib.esg_status_str(status).decode()} "
                       f"({lib.esg_last_error().decode()})")


def _np_ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P)


def _dev_ptr(t):
    if t is None:
        return None
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "need a contiguous CUDA tensor"
    return _P(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


class Index:
    """Owner of an esg_index handle (freed with esg_free)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        lib = load_library()
        n, d, L, R, E, leaf, metric, storage = (_I64(), _I32(), _I32(), _I32(), _I32(), _I32(),
                                                _I32(), _I32())
        _check(lib.esg_index_info(handle, *[ctypes.byref(x) for x in
                                            (n, d, L, R, E, leaf, metric, storage)]), "esg_index_info")
        self.n, self.d, self.L, self.R, self.E = n.value, d.value, L.value, R.value, E.value
        self.leaf_size, self.metric, self.storage = leaf.value, metric.value, storage.value
        layout, fanout, nodes, rows = _I32(), _I32(), _I64(), _I64()
        _check(lib.esg_index_layout(handle, *[ctypes.byref(x) for x in (layout, fanout, nodes, rows)]),
               "esg_index_layout")
        self.layout = {v: k for k, v in LAYOUT.items()}[layout.value]
        self.fanout, self.nodes, self.adj_rows = fanout.value, nodes.value, rows.value
        # the library builds and imports on the current CUDA device
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else None

    @property
    def handle(self):
        if self._h is None:
            raise EsgError("index already freed")
        return self._h

    def close(self):
        if self._h is not None:
            load_library().esg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def esg_build(vectors: np.ndarray, attr: Optional[np.ndarray] = None, *, M: int = 16,
              leaf_size: int = 256, n_entries: int = 16, ef_construction: int = 200,
              batch_div: int = 8, metric: str = "l2", storage: str = "f32", fanout: int = 2,
              layout: str = "tree") -> Index:
    """Build an index on the current CUDA device from host float32 vectors
    [n, d] (original order) and optional float64 attributes [n]: the segment
    tree of fanout f (layout "tree") or the prefix graphs of base `fanout`
    (layout "prefix", half-bounded ranges [0, r])."""
    lib = load_library()
    v = np.ascontiguousarray(vectors, dtype=np.float32)
    a = None if attr is None else np.ascontiguousarray(attr, dtype=np.float64)
    p = _BuildParams(M, leaf_size, n_entries, ef_construction, batch_div, fanout, METRIC[metric],
                     STORAGE[storage], LAYOUT[layout], 0)
    h = _P()
    _check(lib.esg_build(_np_ptr(v), v.shape[0], v.shape[1], _np_ptr(a), ctypes.byref(p),
                         ctypes.byref(h)), "esg_build")
    return Index(h)


def esg_index_import(vectors_ranked: np.ndarray, perm: Optional[np.ndarray], metric: str,
                     leaf_size: int, adj: np.ndarray, entries: np.ndarray,
                     storage: str = "f32", layout: str = "tree", fanout: int = 2) -> Index:
    """Create an index from host graphs in the stored layout (vectors in rank
    order; tree: adj [L, n, R] uint32, entries [(f^L - 1)/(f - 1), E] int32;
    prefix: adj [sum of n_i, R], entries [L, E])."""
    lib = load_library()
    v = np.ascontiguousarray(vectors_ranked, dtype=np.float32)
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    ent = np.ascontiguousarray(entries, dtype=np.int32)
    if layout == "tree":
        L, _, R = adj.shape if adj.ndim == 3 else (0, 0, 1)
    else:
        L, R = ent.shape[0], adj.shape[1]
    h = _P()
    _check(lib.esg_index_import(_np_ptr(v), _np_ptr(pm), v.shape[0], v.shape[1], METRIC[metric],
                                leaf_size, LAYOUT[layout], fanout, _np_ptr(adj) if L else None, L, R,
                                _np_ptr(ent) if L else None, ent.shape[1] if ent.ndim == 2 else 1,
                                STORAGE[storage], ctypes.byref(h)), "esg_index_import")
    return Index(h)


def esg_index_export(index: Index) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(adj uint32: tree [L, n, R], prefix [sum of n_i, R]; entries [nodes, E]
    int32; perm [n] int64)."""
    lib = load_library()
    shape = (index.L, index.n, index.R) if index.layout == "tree" else (index.adj_rows, index.R)
    adj = np.empty(shape, dtype=np.uint32)
    ent = np.empty((index.nodes, index.E), dtype=np.int32)
    perm = np.empty(index.n, dtype=np.int64)
    _check(lib.esg_index_export(index.handle, _np_ptr(adj) if adj.size else None,
                                _np_ptr(ent) if ent.size else None, _np_ptr(perm)),
           "esg_index_export")
    return adj, ent, perm


def esg_index_export_entries(index: Index) -> np.ndarray:
    """Entry ranks per graph node: int32 [nodes, E], -1 padded."""
    ent = np.empty((index.nodes, index.E), dtype=np.int32)
    _check(load_library().esg_index_export(index.handle, None, _np_ptr(ent) if ent.size else None, None),
           "esg_index_export")
    return ent


def esg_index_perm(index: Index) -> np.ndarray:
    """Original id of each rank: int64 [n]."""
    perm = np.empty(index.n, dtype=np.int64)
    _check(load_library().esg_index_export(index.handle, None, None, _np_ptr(perm)), "esg_index_export")
    return perm


def esg_index_export_rows(index: Index, level: int, row0: int, nrows: int) -> np.ndarray:
    """Rows row0 .. row0 + nrows - 1 of one graph level: uint32 [nrows, R]."""
    adj = np.empty((nrows, index.R), dtype=np.uint32)
    _check(load_library().esg_index_export_rows(index.handle, level, row0, nrows,
                                                _np_ptr(adj) if adj.size else None),
           "esg_index_export_rows")
    return adj


def esg_index_export_storage(index: Index, dtype: str):
    """Low-precision traversal rows in rank order: (uint16 [n, d] BF16 bits,
    None) or (uint8 [n, d] E4M3 codes, float32 [n] scales)."""
    lib = load_library()
    if dtype == "bf16":
        rows = np.empty((index.n, index.d), dtype=np.uint16)
        _check(lib.esg_index_export_storage(index.handle, STORAGE[dtype], _np_ptr(rows), None),
               "esg_index_export_storage")
        return rows, None
    rows = np.empty((index.n, index.d), dtype=np.uint8)
    scale = np.empty(index.n, dtype=np.float32)
    _check(lib.esg_index_export_storage(index.handle, STORAGE[dtype], _np_ptr(rows), _np_ptr(scale)),
           "esg_index_export_storage")
    return rows, scale


def esg_index_add_storage(index: Index, dtype: str):
    """Add a BF16 or FP8 copy of the rows for low-precision traversal."""
    _check(load_library().esg_index_add_storage(index.handle, STORAGE[dtype]), "esg_index_add_storage")


def esg_free(index: Index):
    index.close()


def esg_decompose_batch(n: int, leaf_size: int, l, r, stream=None, fanout: int = 2, layout: str = "tree",
                        post_root: int = 0):
    """Decomposition of query ranges on the device (elastic subranges of the
    fanout-f tree, the prefix graph of the prefix layout, or the root alone).
    l, r: CUDA int64 [nq]. Returns (pieces int64 [nq, 2, 6] raw esg_piece
    records, npieces int32 [nq])."""
    import torch
    lib = load_library()
    nq = l.numel()
    pieces = torch.empty((nq, 2, 6), dtype=torch.int64, device=l.device)
    npieces = torch.empty(nq, dtype=torch.int32, device=l.device)
    _check(lib.esg_decompose_batch(n, leaf_size, LAYOUT[layout], fanout, post_root, _dev_ptr(l), _dev_ptr(r),
                                   nq, _dev_ptr(pieces), _dev_ptr(npieces), _stream_ptr(stream)),
           "esg_decompose_batch")
    return pieces, npieces


def unpack_pieces(pieces):
    """Split raw esg_piece records into (node_l, node_r, pl, pr, heap, depth, kind)."""
    p64 = pieces
    p32 = pieces.view(dtype=__import__("torch").int32)
    return (p64[..., 0], p64[..., 1], p64[..., 2], p64[..., 3], p32[..., 8], p32[..., 9], p32[..., 10])


def _check_search_buffers(who: str, index: Index, queries, l, r, k, k_max: int, ids, dist, count,
                          status, stats):
    """Shape, dtype, device and layout of every buffer of a batched search,
    checked before the C call: the library trusts the sizes it is given, so a
    buffer that is too small would be read or written past its end."""
    import torch
    nq = queries.shape[0] if hasattr(queries, "shape") else -1
    want = [("queries", queries, (nq, index.d), torch.float32, True),
            ("l", l, (nq,), torch.int64, True), ("r", r, (nq,), torch.int64, True),
            ("k", k, (nq,), torch.int32, False),
            ("ids", ids, (nq, k_max), torch.int64, True), ("dist", dist, (nq, k_max), torch.float32, True),
            ("count", count, (nq,), torch.int32, True), ("status", status, (nq,), torch.int32, False),
            ("stats", stats, (nq, 6), torch.int64, False)]
    for name, t, shape, dtype, required in want:
        if t is None:
            if required:
                raise EsgError(f"{who}: {name} is required")
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise EsgError(f"{who}: {name} must be a CUDA tensor")
        if index.device is not None and t.device != index.device:
            raise EsgError(f"{who}: {name} is on {t.device}, the index on {index.device}")
        if t.dtype != dtype:
            raise EsgError(f"{who}: {name} must be {dtype}, got {t.dtype}")
        if tuple(t.shape) != shape:
            raise EsgError(f"{who}: {name} must have shape {shape}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise EsgError(f"{who}: {name} must be contiguous")


def search_params(ef: int = 64, max_expansions: int = 0, rerank: int = 1, use_learned: int = 0,
                  traversal: str = "f32", width: int = 1, warps_per_block: int = 0,
                  hash_slots: int = 0, lanes_per_row: int = 0, post_root: int = 0,
                  max_registers: int = 0) -> _SearchParams:
    """An esg_search_params record."""
    return _SearchParams(ef, max_expansions, rerank, use_learned,
                         STORAGE[traversal] if isinstance(traversal, str) else traversal, width,
                         warps_per_block, hash_slots, lanes_per_row, post_root, max_registers)


def esg_search_batch(index: Index, queries, l, r, k=None, k_max: int = 10, *, ef: int = 64,
                     max_expansions: int = 0, rerank: int = 1, use_learned: int = 0,
                     traversal: str = "f32", width: int = 1, params=None, out=None,
                     want_status: bool = True, want_stats: bool = False, stream=None):
    """Range-filtered search of CUDA float32 queries [nq, d] with CUDA int64
    ranges [nq]. Returns (ids int64 [nq,k_max], dist f32, count int32,
    status int32 or None, stats int64 [nq,6] or None)."""
    import torch
    lib = load_library()
    nq = queries.shape[0]
    dev = queries.device
    if out is None:
        ids = torch.empty((nq, k_max), dtype=torch.int64, device=dev)
        dist = torch.empty((nq, k_max), dtype=torch.float32, device=dev)
        count = torch.empty(nq, dtype=torch.int32, device=dev)
        status = torch.empty(nq, dtype=torch.int32, device=dev) if want_status else None
        stats = torch.empty((nq, 6), dtype=torch.int64, device=dev) if want_stats else None
    else:
        ids, dist, count, status, stats = out
    p = params if params is not None else search_params(ef, max_expansions, rerank, use_learned,
                                                        traversal, width)
    _check_search_buffers("esg_search_batch", index, queries, l, r, k, k_max, ids, dist, count,
                          status, stats)
    _check(lib.esg_search_batch(index.handle, _dev_ptr(queries), nq, _dev_ptr(l), _dev_ptr(r),
                                _dev_ptr(k), k_max, ctypes.byref(p), _dev_ptr(ids), _dev_ptr(dist),
                                _dev_ptr(count), _dev_ptr(status), _dev_ptr(stats),
                                _stream_ptr(stream)), "esg_search_batch")
    return ids, dist, count, status, stats


def esg_bruteforce_filtered_knn(base, queries, l, r, k: int, metric: str = "l2", out=None,
                                stream=None):
    """Exact filtered k-NN by brute force on CUDA tensors. Returns
    (ids int64 [nq, k] row indices, dist f32 [nq, k], count int32 [nq])."""
    import torch
    lib = load_library()
    nq = queries.shape[0]
    dev = queries.device
    if out is None:
        ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
        dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
        count = torch.empty(nq, dtype=torch.int32, device=dev)
    else:
        ids, dist, count = out
    _check(lib.esg_bruteforce_filtered_knn(_dev_ptr(base), base.shape[0], base.shape[1],
                                           METRIC[metric], _dev_ptr(queries), nq, _dev_ptr(l),
                                           _dev_ptr(r), k, _dev_ptr(ids), _dev_ptr(dist),
                                           _dev_ptr(count), _stream_ptr(stream)),
           "esg_bruteforce_filtered_knn")
    return ids, dist, count


def esg_attr_to_rank_range(index: Index, lo: np.ndarray, hi: np.ndarray):
    lib = load_library()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    l = np.empty(lo.shape[0], dtype=np.int64)
    r = np.empty(lo.shape[0], dtype=np.int64)
    _check(lib.esg_attr_to_rank_range(index.handle, _np_ptr(lo), _np_ptr(hi), lo.shape[0],
                                      _np_ptr(l), _np_ptr(r)), "esg_attr_to_rank_range")
    return l, r


def esg_bruteforce_plan(n: int, d: int, l: np.ndarray, r: np.ndarray, ctas: int = 152):
    """Host work plan of the tensor-core exact search (no GPU work): returns
    (order [V], tiles [T], items [I, 4], cta_first [G + 1]) as int32 arrays."""
    lib = load_library()
    l = np.ascontiguousarray(l, dtype=np.int64)
    r = np.ascontiguousarray(r, dtype=np.int64)
    sizes = np.zeros(4, dtype=np.int64)
    args = (n, d, _np_ptr(l), _np_ptr(r), l.shape[0], ctas)
    _check(lib.esg_bruteforce_plan(*args, _np_ptr(sizes), None, None, None, None), "esg_bruteforce_plan")
    order = np.empty(sizes[0], dtype=np.int32)
    tiles = np.empty(sizes[1], dtype=np.int32)
    items = np.empty((sizes[2], 4), dtype=np.int32)
    cta_first = np.empty(sizes[3] + 1, dtype=np.int32)
    _check(lib.esg_bruteforce_plan(*args, _np_ptr(sizes), _np_ptr(order), _np_ptr(tiles), _np_ptr(items),
                                   _np_ptr(cta_first)), "esg_bruteforce_plan")
    return order, tiles, items, cta_first


def esg_save(index: Index, path: str):
    _check(load_library().esg_save(index.handle, path.encode()), "esg_save")


def esg_load(path: str) -> Index:
    h = _P()
    _check(load_library().esg_load(path.encode(), ctypes.byref(h)), "esg_load")
    return Index(h)


def esg_profile_enable(on: bool = True):
    """Record CUDA events around each search kernel (benchmark timing)."""
    _check(load_library().esg_profile_enable(1 if on else 0), "esg_profile_enable")


def esg_profile_read(reset: bool = True):
    """(summed search-kernel ms, kernels launched, timed launches) since the
    last reset; waits for the recorded events."""
    ms = ctypes.c_double()
    launches = _I64()
    timed = _I64()
    _check(load_library().esg_profile_read(ctypes.byref(ms), ctypes.byref(launches),
                                           ctypes.byref(timed), 1 if reset else 0),
           "esg_profile_read")
    return ms.value, launches.value, timed.value


def esg_profile_tensor_work(reset: bool = True) -> float:
    """FLOPs of the tensor-core MMAs issued by the brute force while
    profiling was enabled."""
    f = ctypes.c_double()
    _check(load_library().esg_profile_tensor_work(ctypes.byref(f), 1 if reset else 0),
           "esg_profile_tensor_work")
    return f.value


class Batch:
    """A CUDA-graph batch executor (esg_batch_*): device buffers for up to
    max_nq queries, replayed with one graph launch per run."""

    def __init__(self, index: Index, max_nq: int, k_max: int, params=None, use_k: bool = False):
        import torch
        lib = load_library()
        self.index, self.max_nq, self.k_max = index, max_nq, k_max
        p = params if params is not None else search_params()
        h = _P()
        _check(lib.esg_batch_create(index.handle, max_nq, k_max, 1 if use_k else 0, ctypes.byref(p),
                                    ctypes.byref(h)), "esg_batch_create")
        self._h = h
        ptrs = [_P() for _ in range(9)]
        _check(lib.esg_batch_buffers(h, *[ctypes.byref(x) for x in ptrs]), "esg_batch_buffers")
        self.ptrs = dict(zip(["queries", "l", "r", "k", "ids", "dist", "count", "status", "stats"],
                             [x.value for x in ptrs]))
        self._torch = torch

    def view(self, name: str, shape, dtype):
        """A torch tensor aliasing one of the batch's device buffers (no copy)."""
        torch = self._torch
        n = int(np.prod(shape))
        esize = torch.empty(0, dtype=dtype).element_size()

        class _Cuda:
            def __init__(self, ptr, nbytes):
                self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1",
                                                 "data": (ptr, False), "version": 3}
        raw = torch.as_tensor(_Cuda(self.ptrs[name], n * esize), device="cuda")
        return raw.view(dtype).view(*shape)

    def run(self, nq: int, stream=None):
        _check(load_library().esg_batch_run(self._h, nq, _stream_ptr(stream)), "esg_batch_run")

    def close(self):
        if getattr(self, "_h", None) is not None:
            load_library().esg_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def esg_autotune(index: Index, queries, l, r, gt_ids, gt_count, k_max: int = 10, k=None,
                 target_recall: float = 0.95, base=None, stream=None):
    """Choose ef, search width and launch shape for a recall target on sample
    queries with exact answers (CUDA tensors). Returns (params, recall, ms)."""
    lib = load_library()
    b = base if base is not None else search_params()
    out = _SearchParams()
    rep = np.zeros(2, dtype=np.float32)
    _check(lib.esg_autotune(index.handle, _dev_ptr(queries), queries.shape[0], _dev_ptr(l), _dev_ptr(r),
                            _dev_ptr(k), k_max, _dev_ptr(gt_ids), _dev_ptr(gt_count),
                            float(target_recall), ctypes.byref(b), ctypes.byref(out), _np_ptr(rep),
                            _stream_ptr(stream)), "esg_autotune")
    return out, float(rep[0]), float(rep[1])


def esg_search_batch_noalloc(index: Index, queries, l, r, out, k=None, k_max: int = 10,
                             params=None, stream=None):
    """esg_search_batch with no device allocation: scratch comes from the
    library's fixed device array. `out` = (ids, dist, count, status or None,
    stats or None) caller-allocated CUDA tensors."""
    lib = load_library()
    ids, dist, count, status, stats = out
    p = params if params is not None else search_params()
    _check_search_buffers("esg_search_batch_noalloc", index, queries, l, r, k, k_max, ids, dist,
                          count, status, stats)
    _check(lib.esg_search_batch_noalloc(index.handle, _dev_ptr(queries), queries.shape[0],
                                        _dev_ptr(l), _dev_ptr(r), _dev_ptr(k), k_max, ctypes.byref(p),
                                        _dev_ptr(ids), _dev_ptr(dist), _dev_ptr(count),
                                        _dev_ptr(status), _dev_ptr(stats), _stream_ptr(stream)),
           "esg_search_batch_noalloc")
    return out


def esg_train_predictor(index: Index, queries, l, r, gt_ids, gt_count, k_max: int = 10, k=None,
                        stream=None, **overrides):
    """Train and calibrate the learned search budget on CUDA tensors of
    queries with exact answers. Returns [train loss, held-out recall, ef
    margin, held-out distance evaluations per query]."""
    lib = load_library()
    tp = lib.esg_train_params_default()
    for key, v in overrides.items():
        setattr(tp, key, STORAGE[v] if key == "traversal" and isinstance(v, str) else v)
    rep = np.zeros(4, dtype=np.float32)
    _check(lib.esg_train_predictor(index.handle, _dev_ptr(queries), queries.shape[0], _dev_ptr(l),
                                   _dev_ptr(r), _dev_ptr(k), k_max, _dev_ptr(gt_ids), _dev_ptr(gt_count),
                                   ctypes.byref(tp), _np_ptr(rep), _stream_ptr(stream)),
           "esg_train_predictor")
    return rep


def esg_predictor_get(index: Index):
    lib = load_library()
    blob = np.empty(lib.esg_mlp_blob_size(), dtype=np.float32)
    lo, hi = _I32(), _I32()
    _check(lib.esg_predictor_get(index.handle, _np_ptr(blob), ctypes.byref(lo), ctypes.byref(hi)),
           "esg_predictor_get")
    return blob, lo.value, hi.value


def esg_predictor_set(index: Index, blob: np.ndarray, ef_lo: int, ef_hi: int):
    blob = np.ascontiguousarray(blob, dtype=np.float32)
    _check(load_library().esg_predictor_set(index.handle, _np_ptr(blob), ef_lo, ef_hi),
           "esg_predictor_set")


def esg_mlp_num_params() -> int:
    return int(load_library().esg_mlp_num_params())


def esg_mlp_num_features() -> int:
    return int(load_library().esg_mlp_num_features())


def esg_mlp_blob_size() -> int:
    """Floats of a predictor blob (esg_predictor_get / esg_predictor_set)."""
    return int(load_library().esg_mlp_blob_size())


def esg_mlp_forward(params, X, mu, sigma, stream=None):
    import torch
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
    _check(load_library().esg_mlp_forward(_dev_ptr(params), _dev_ptr(X), _dev_ptr(mu), _dev_ptr(sigma),
                                          X.shape[0], _dev_ptr(Y), _stream_ptr(stream)), "esg_mlp_forward")
    return Y


def esg_mlp_loss_grad(params, X, T, mu, sigma, quantile: float, stream=None):
    import torch
    g = torch.empty_like(params)
    loss = ctypes.c_float()
    _check(load_library().esg_mlp_loss_grad(_dev_ptr(params), _dev_ptr(X), _dev_ptr(T), _dev_ptr(mu),
                                            _dev_ptr(sigma), X.shape[0], float(quantile), _dev_ptr(g),
                                            ctypes.byref(loss), _stream_ptr(stream)), "esg_mlp_loss_grad")
    return loss.value, g


def esg_mlp_adam_step(params, grad, m, v, step: int, lr: float, stream=None):
    _check(load_library().esg_mlp_adam_step(_dev_ptr(params), _dev_ptr(grad), _dev_ptr(m), _dev_ptr(v),
                                            step, float(lr), _stream_ptr(stream)), "esg_mlp_adam_step")


def esg_query_features(index: Index, queries, l, r, k=None, k_max: int = 10, stream=None):
    import torch
    f = torch.empty((queries.shape[0], esg_mlp_num_features()), dtype=torch.float32,
                    device=queries.device)
    _check(load_library().esg_query_features(index.handle, _dev_ptr(queries), queries.shape[0],
                                             _dev_ptr(l), _dev_ptr(r), _dev_ptr(k), k_max, _dev_ptr(f),
                                             _stream_ptr(stream)), "esg_query_features")
    return f


def esg_query_budget(index: Index, queries, l, r, k=None, k_max: int = 10, ef_fixed: int = 64, stream=None):
    """Per-query (ef, expansion cap) the trained predictor gives, as CUDA
    int32 tensors [nq] (cap 0 = the default 16 ef_fixed + 256)."""
    import torch
    nq = queries.shape[0]
    ef = torch.empty(nq, dtype=torch.int32, device=queries.device)
    mx = torch.empty(nq, dtype=torch.int32, device=queries.device)
    _check(load_library().esg_query_budget(index.handle, _dev_ptr(queries), nq, _dev_ptr(l), _dev_ptr(r),
                                           _dev_ptr(k), k_max, ef_fixed, _dev_ptr(ef), _dev_ptr(mx),
                                           _stream_ptr(stream)), "esg_query_budget")
    return ef, mx
