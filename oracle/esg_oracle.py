"""Float64 CPU oracle for ESG (arxiv 2504.04018). TEST INFRASTRUCTURE ONLY.

Pure-Python/numpy parts: re-ranking, the elastic range decomposition of
Algorithm 4, the exact range-filtered k-NN of Definitions 1-2, the merge of
Algorithm 4, recall. Graph search (Algorithm 1) and the index build
(Algorithm 3) run in ``esg_oracle.c`` (plain single-threaded C, float64),
loaded through ctypes.

Conventions: ranks are 0-based and ranges inclusive ([l, r] with
0 <= l <= r <= N-1); the paper's ranks are 1-based (Definition 2). Row i of a
re-ranked matrix holds the point of rank i. Squared Euclidean distance
("l2") is sum (q - x)^2; inner-product distance ("ip") is -<q, x>. Orderings
are lexicographic on (distance, rank).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esg_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libesg_oracle.so")
NONE = 0xFFFFFFFF
METRICS = {"l2": 0, "ip": 1}

__all__ = [
    "build_c", "rerank", "is_leaf", "split", "children", "Piece", "decompose", "graph_depths",
    "tree_nodes", "prefix_sizes", "decompose_prefix", "decompose_root", "pieces_of",
    "build_prefix_index",
    "bruteforce", "merge_topk", "OracleIndex", "build_index", "graph_search", "graph_search_rows",
    "search", "recall_at_k", "distances", "METRICS", "NONE", "bf16_round", "bf16_to_float",
    "fp8_e4m3_grid", "fp8_quantize_rows", "fp8_to_float", "traversal_rows",
]


# ------------------------------------------------------------------ C part

def build_c(force: bool = False) -> str:
    """Compile esg_oracle.c into oracle/_build/libesg_oracle.so (gcc -O2)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _c():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_c())
        P = ctypes.c_void_p
        lib.oracle_graph_search.restype = ctypes.c_int
        lib.oracle_graph_search.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P,
                                            ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int,
                                            ctypes.c_int64, ctypes.c_int64, P, P, P, ctypes.c_int64,
                                            ctypes.c_int64]
        lib.oracle_build.restype = ctypes.c_int
        lib.oracle_build.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P,
                                     ctypes.c_int]
        lib.oracle_build_prefix.restype = ctypes.c_int
        lib.oracle_build_prefix.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------- re-ranking

def rerank(attr: np.ndarray) -> np.ndarray:
    """Rank order of the points (Section 1 footnote): ``perm[i]`` is the
    original row of the point with rank i, sorting by attribute value with
    ties broken by original row."""
    attr = np.asarray(attr, dtype=np.float64)
    return np.lexsort((np.arange(attr.shape[0]), attr)).astype(np.int64)


# ------------------------------------------------------------ segment tree

def is_leaf(l: int, r: int, leaf_size: int) -> bool:
    """A node [l, r] carries no graph when r - l < leaf_size (Algorithm 3
    and Algorithm 4, first test)."""
    return r - l < leaf_size


def split(l: int, r: int) -> int:
    """mid = floor((l + r) / 2); children are [l, mid] and [mid + 1, r]."""
    return (l + r) // 2


def children(l: int, r: int, fanout: int = 2) -> List[Tuple[int, int, int]]:
    """The non-empty children (a, b, j) of node [l, r] in a tree of fanout f:
    child j = [b_j, b_{j+1} - 1] with b_j = l + ceil(j * len / f), len = r - l + 1
    (the paper leaves the split points of a larger fanout open; this reading
    gives Algorithm 3's [l, mid], [mid + 1, r] for f = 2). Child j of heap
    node h is heap node f h + 1 + j."""
    n = r - l + 1
    b = [l + -(-j * n // fanout) for j in range(fanout + 1)]
    return [(b[j], b[j + 1] - 1, j) for j in range(fanout) if b[j] <= b[j + 1] - 1]


@dataclasses.dataclass(frozen=True)
class Piece:
    """One subrange chosen by Algorithm 4.

    kind: "graph" (search the graph of node [node_l, node_r]) or "scan"
    (linear scan). [pl, pr] is the part of the query range it answers.
    heap: the node's heap number (root 0; children of h are f h + 1 .. f h + f
    in a tree of fanout f; for a prefix index, the prefix graph's number);
    depth: its depth (root 0; for a prefix index, the level of the prefix
    graph).
    """
    kind: str
    node_l: int
    node_r: int
    pl: int
    pr: int
    heap: int
    depth: int


def decompose(n: int, leaf_size: int, lq: int, rq: int, fanout: int = 2) -> List[Piece]:
    """Query-2D-Index (Algorithm 4) restricted to the choice of subranges.

    Starting at the root [0, n-1]: a node with r - l < leaf_size is answered
    by a linear scan of its part of the query; a node that contains the query
    part with |[lq, rq]| / |[l, r]| >= c (c = 1/fanout, tested in integers as
    fanout * |[lq, rq]| >= |[l, r]|) is answered by its graph; otherwise the
    query part is clipped to each child it overlaps (left first) and each is
    resolved the same way. Lemma 3 (fanout 2) and Lemma 4 (fanout f with
    c = 1/f) bound the result to two pieces.
    """
    if not (0 <= lq <= rq <= n - 1):
        raise ValueError("need 0 <= lq <= rq <= n-1")
    out: List[Piece] = []

    def rec(l, r, a, b, h, depth):
        if is_leaf(l, r, leaf_size):
            out.append(Piece("scan", l, r, a, b, h, depth))
            return
        if l <= a and b <= r and fanout * (b - a + 1) >= (r - l + 1):
            out.append(Piece("graph", l, r, a, b, h, depth))
            return
        for (ca, cb, j) in children(l, r, fanout):
            if a <= cb and b >= ca:
                rec(ca, cb, max(a, ca), min(b, cb), fanout * h + 1 + j, depth + 1)

    rec(0, n - 1, lq, rq, 0, 0)
    return out


def graph_depths(n: int, leaf_size: int, fanout: int = 2) -> int:
    """Number of depths of the tree that hold at least one graph node."""
    L = 0
    frontier = [(0, n - 1)]
    while frontier:
        nxt = []
        any_graph = False
        for (l, r) in frontier:
            if not is_leaf(l, r, leaf_size):
                any_graph = True
                nxt += [(a, b) for (a, b, _) in children(l, r, fanout)]
        if not any_graph:
            break
        L += 1
        frontier = nxt
    return L


def tree_nodes(L: int, fanout: int = 2) -> int:
    """Heap slots of the depths 0..L-1: 1 + f + ... + f^(L-1)."""
    return sum(fanout ** t for t in range(L))


def prefix_sizes(n: int, base: int = 2) -> List[int]:
    """Sizes of the prefix graphs of the half-bounded index (ESG-1D, Section
    4.1): n_i = floor(n / B^i) for i = 0, 1, ... while n_i >= 1 (B = 2 in the
    paper's definition; base B is its extension)."""
    out, m = [], n
    while m >= 1:
        out.append(m)
        m //= base
    return out


def decompose_prefix(n: int, base: int, lq: int, rq: int) -> List[Piece]:
    """Query processing of the half-bounded index (Section 4.1, Lemma 2): a
    query [0, rq] is answered by the smallest prefix graph [0, n_i - 1] that
    contains it, i.e. the largest i with n_i = floor(n / B^i) >= rq + 1. Then
    |[0, rq]| / n_i > 1/B. (Lemma 2 as printed picks [1, N / 2^ceil(log r)],
    which is [1, 1] for r = N; this reading is the one its two claims,
    containment and ratio >= 1/2, fix.) Only prefix ranges are supported."""
    if not (lq == 0 and 0 <= rq <= n - 1):
        raise ValueError("the half-bounded index answers ranges [0, r] with 0 <= r <= n-1")
    sizes = prefix_sizes(n, base)
    i = max(j for j, m in enumerate(sizes) if m >= rq + 1)
    return [Piece("graph", 0, sizes[i] - 1, 0, rq, i, i)]


def decompose_root(n: int, leaf_size: int, lq: int, rq: int) -> List[Piece]:
    """POST on the root graph alone (the baseline of Section 3.1): every
    query is one piece of the root [0, n-1], scanned when the root is a leaf."""
    if not (0 <= lq <= rq <= n - 1):
        raise ValueError("need 0 <= lq <= rq <= n-1")
    kind = "scan" if is_leaf(0, n - 1, leaf_size) else "graph"
    return [Piece(kind, 0, n - 1, lq, rq, 0, 0)]


# ------------------------------------------------------------ exact k-NN

def distances(X: np.ndarray, q: np.ndarray, metric: str) -> np.ndarray:
    """Float64 distances from q to every row of X: squared Euclidean
    sum_j (q_j - x_j)^2, or negative inner product -sum_j q_j x_j."""
    X = np.asarray(X, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if metric == "l2":
        diff = X - q[None, :]
        return np.einsum("ij,ij->i", diff, diff)
    if metric == "ip":
        return -(X @ q)
    raise ValueError(metric)


def bruteforce(X: np.ndarray, q: np.ndarray, pl: int, pr: int, k: int, metric: str
               ) -> Tuple[np.ndarray, np.ndarray]:
    """Exact range-filtered k-NN (Definitions 1 and 2): the min(k, pr-pl+1)
    rows of X with rank in [pl, pr] closest to q, ascending by (distance,
    rank). Returns (ranks int64, distances float64)."""
    if pr < pl:
        return np.zeros(0, np.int64), np.zeros(0, np.float64)
    dd = distances(X[pl:pr + 1], q, metric)
    ranks = np.arange(pl, pr + 1, dtype=np.int64)
    order = np.lexsort((ranks, dd))[:k]
    return ranks[order], dd[order]


def merge_topk(parts: Sequence[Tuple[np.ndarray, np.ndarray]], k: int
               ) -> Tuple[np.ndarray, np.ndarray]:
    """Merge of per-piece results (Algorithm 4, last step): the k best of
    their union by (distance, rank). Pieces cover disjoint ranges, so no id
    appears twice."""
    if not parts:
        return np.zeros(0, np.int64), np.zeros(0, np.float64)
    ids = np.concatenate([p[0] for p in parts]).astype(np.int64)
    dd = np.concatenate([p[1] for p in parts]).astype(np.float64)
    order = np.lexsort((ids, dd))[:k]
    return ids[order], dd[order]


# ------------------------------------------------- low-precision storage

def bf16_round(x: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns of float32 values, rounding to nearest, ties to
    even (the upper 16 bits of the float32 pattern after adding 0x7FFF plus
    the lowest kept bit). NaN stays NaN."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    nan = np.isnan(np.asarray(x, dtype=np.float32))
    return np.where(nan, np.uint16(0x7FC0), rounded)


def bf16_to_float(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def fp8_e4m3_grid() -> np.ndarray:
    """The 127 non-negative finite FP8-E4M3 values in code order 0..126:
    code = (e << 3) | m, value = m/8 * 2^-6 for e = 0 (subnormal), else
    (1 + m/8) * 2^(e - 7); code 127 (e = 15, m = 7) is NaN, so 448 is the
    largest finite value."""
    vals = []
    for code in range(127):
        e, m = code >> 3, code & 7
        vals.append((m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(vals, dtype=np.float64)


_FP8_GRID = fp8_e4m3_grid()


def _fp8_code(v: np.ndarray) -> np.ndarray:
    """Saturating round-to-nearest-even of float32 values to E4M3 codes."""
    v = np.asarray(v, dtype=np.float32).astype(np.float64)
    a = np.minimum(np.abs(v), 448.0)
    hi = np.clip(np.searchsorted(_FP8_GRID, a, side="left"), 0, 126)
    lo = np.clip(hi - 1, 0, 126)
    dlo = a - _FP8_GRID[lo]
    dhi = _FP8_GRID[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo).astype(np.uint8)
    code = np.where(a == _FP8_GRID[hi], hi, code).astype(np.uint8)
    return np.where(np.signbit(v), code | 0x80, code).astype(np.uint8)


def fp8_quantize_rows(X: np.ndarray):
    """Per-row FP8-E4M3 storage: s_i = max_j |x_ij| / 448 and
    code_ij = satfinite RNE(x_ij / s_i), both divisions in float32 (code 0
    for an all-zero row). Returns (codes uint8 [n, d], scales float32 [n])."""
    X = np.asarray(X, dtype=np.float32)
    m = np.abs(X).max(axis=1)
    s = (m / np.float32(448.0)).astype(np.float32)
    safe = np.where(s > 0, s, np.float32(1.0)).astype(np.float32)
    v = (X / safe[:, None]).astype(np.float32)
    v = np.where(s[:, None] > 0, v, np.float32(0.0))
    return _fp8_code(v), s


def fp8_to_float(codes: np.ndarray) -> np.ndarray:
    codes = np.asarray(codes, dtype=np.uint8)
    mag = _FP8_GRID[np.minimum(codes & 0x7F, 126)]
    return np.where(codes & 0x80, -mag, mag)


def traversal_rows(X32: np.ndarray, dtype: str) -> np.ndarray:
    """Float64 values the traversal distances use for rows stored in `dtype`
    ("f32", "bf16" or "fp8")."""
    X32 = np.asarray(X32, dtype=np.float32)
    if dtype == "f32":
        return X32.astype(np.float64)
    if dtype == "bf16":
        return bf16_to_float(bf16_round(X32)).astype(np.float64)
    codes, s = fp8_quantize_rows(X32)
    return fp8_to_float(codes) * s.astype(np.float64)[:, None]


# ------------------------------------------------------------ index build

@dataclasses.dataclass
class OracleIndex:
    """Graphs of an ESG index in the layout the GPU library imports.

    X: float64 [n, d] in rank order; perm: rank -> original row.
    kind "tree" (ESG-2D, Algorithm 3; fanout f): adj uint32 [L, n, R]; row i of
    depth t lists the neighbour ranks of point i in the graph of the depth-t
    node that contains i (NONE-padded); entries int32 [(f^L - 1)/(f - 1), E]
    entry ranks per heap node (-1 padded; all -1 for leaves).
    kind "prefix" (ESG-1D, Algorithm 2; base B = fanout): adj uint32
    [sum of n_i, R], the rows of prefix graph i (ranks 0..n_i - 1) starting at
    row n_0 + ... + n_{i-1}; entries int32 [L, E].
    """
    X: np.ndarray
    perm: np.ndarray
    adj: np.ndarray
    entries: np.ndarray
    leaf_size: int
    M: int
    metric: str
    kind: str = "tree"
    fanout: int = 2

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def R(self) -> int:
        return self.adj.shape[-1]

    @property
    def L(self) -> int:
        return self.adj.shape[0] if self.kind == "tree" else len(prefix_sizes(self.n, self.fanout))

    def level(self, t: int) -> np.ndarray:
        """Rows of graph level t, indexed by rank."""
        if self.kind == "tree":
            return self.adj[t]
        sizes = prefix_sizes(self.n, self.fanout)
        off = sum(sizes[:t])
        return self.adj[off:off + sizes[t]]


def build_index(base: np.ndarray, attr: Optional[np.ndarray], metric: str, leaf_size: int,
                M: int, efc: int = 200, n_entries: int = 16, fanout: int = 2) -> OracleIndex:
    """Re-rank the points, then Build-2D-Index (Algorithm 3; fanout f, the
    extension of Section 4.2 for f > 2) with HNSW-style insertion into flat
    graphs (out-degree cap R = 2M, M neighbours chosen per insertion by edge
    occlusion, efc = construction beam width)."""
    n, d = base.shape
    perm = rerank(attr) if attr is not None else np.arange(n, dtype=np.int64)
    X = np.ascontiguousarray(base[perm].astype(np.float64))
    L = graph_depths(n, leaf_size, fanout)
    R = 2 * M
    adj = np.empty((max(L, 0), n, R), dtype=np.uint32)
    entries = np.empty((tree_nodes(L, fanout), n_entries), dtype=np.int32)
    rc = _c().oracle_build(_ptr(X), n, d, METRICS[metric], leaf_size, M, efc, n_entries, L,
                           _ptr(adj), _ptr(entries) if entries.size else None, fanout)
    if rc != 0:
        raise RuntimeError("oracle_build failed")
    return OracleIndex(X, perm, adj, entries, leaf_size, M, metric, "tree", fanout)


def build_prefix_index(base: np.ndarray, attr: Optional[np.ndarray], metric: str, M: int,
                       efc: int = 200, n_entries: int = 16, base_b: int = 2) -> OracleIndex:
    """Re-rank the points, then Build-1D-Index (Algorithm 2; base B, the
    extension of Section 4.1): prefix graphs of sizes floor(n / B^i), each a
    snapshot of one graph grown by inserting the points in rank order."""
    n, d = base.shape
    perm = rerank(attr) if attr is not None else np.arange(n, dtype=np.int64)
    X = np.ascontiguousarray(base[perm].astype(np.float64))
    sizes = prefix_sizes(n, base_b)
    R = 2 * M
    adj = np.empty((sum(sizes), R), dtype=np.uint32)
    entries = np.empty((len(sizes), n_entries), dtype=np.int32)
    rc = _c().oracle_build_prefix(_ptr(X), n, d, METRICS[metric], base_b, M, efc, n_entries, len(sizes),
                                  _ptr(adj), _ptr(entries))
    if rc != 0:
        raise RuntimeError("oracle_build_prefix failed")
    return OracleIndex(X, perm, adj, entries, 0, M, metric, "prefix", base_b)


def pieces_of(index: OracleIndex, lq: int, rq: int, mode: str = "elastic") -> List[Piece]:
    """The pieces a query range is answered by: the elastic choice of the
    index's kind (Algorithm 4 / Lemma 2), or POST on the root graph alone."""
    if mode == "root":
        return decompose_root(index.n, index.leaf_size, lq, rq)
    if index.kind == "prefix":
        return decompose_prefix(index.n, index.fanout, lq, rq)
    return decompose(index.n, index.leaf_size, lq, rq, index.fanout)


# -------------------------------------------------------------- search

def graph_search(index: OracleIndex, depth: int, heap: int, q: np.ndarray, ef: int,
                 pl: int, pr: int, counters: Optional[np.ndarray] = None,
                 X: Optional[np.ndarray] = None, max_expansions: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Algorithm 1 with POST filtering to [pl, pr] on the graph of heap node
    `heap` (at `depth`), from that node's entry points, over the rows X
    (default: the index's float64 rows). Returns up to ef (ranks, distances)
    ascending. max_expansions > 0 caps the expansions (a search budget)."""
    X = index.X if X is None else np.ascontiguousarray(X, dtype=np.float64)
    return graph_search_rows(X, index.level(depth), index.entries[heap], index.metric, q, ef, pl, pr,
                             counters, max_expansions=max_expansions)


def graph_search_rows(X: np.ndarray, adj: np.ndarray, entries: np.ndarray, metric: str, q: np.ndarray,
                      ef: int, pl: int, pr: int, counters: Optional[np.ndarray] = None,
                      row_base: int = 0, max_expansions: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Algorithm 1 with POST filtering to [pl, pr] on one graph given by its
    rows: X float64 and adj uint32 [rows, R] hold the ranks row_base,
    row_base + 1, ... (a whole level, or one node's rows, whose edges stay
    inside the node); entries are ranks (-1 padded). Returns up to ef
    (ranks, distances) ascending. counters (int64, 2 or 3 entries)
    accumulates expansions, distance evaluations and searches ended by the
    max_expansions cap (0 = no cap)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    q64 = np.ascontiguousarray(q, dtype=np.float64)
    entries = np.asarray(entries)
    ent = np.ascontiguousarray(entries[entries >= 0].astype(np.uint32))
    ids = np.empty(ef, dtype=np.uint32)
    dd = np.empty(ef, dtype=np.float64)
    cnt_arr = np.zeros(3, dtype=np.int64)
    cnt = _c().oracle_graph_search(_ptr(X), X.shape[0], X.shape[1], METRICS[metric],
                                   _ptr(adj), adj.shape[1], _ptr(ent) if len(ent) else None, len(ent),
                                   _ptr(q64), ef, pl, pr, _ptr(ids), _ptr(dd), _ptr(cnt_arr), row_base,
                                   max_expansions)
    if counters is not None:
        m = min(len(counters), 3)
        counters[:m] += cnt_arr[:m]
    return ids[:cnt].astype(np.int64), dd[:cnt].copy()


def search(index: OracleIndex, q: np.ndarray, lq: int, rq: int, k: int, ef: int,
           counters: Optional[np.ndarray] = None, trav_X: Optional[np.ndarray] = None,
           max_expansions: int = 0, mode: str = "elastic") -> Tuple[np.ndarray, np.ndarray]:
    """Query-2D-Index (Algorithm 4): decompose [lq, rq]; answer scan pieces
    exactly and graph pieces with Algorithm 1 + POST at beam width
    max(ef, k); merge into the top k by (distance, rank). Returns ranks.

    With `trav_X` (rows as stored in low precision, see traversal_rows) the
    traversal and scans use those rows, each piece keeps its best max(ef, k)
    in-range candidates, and these are re-ranked with the exact rows before
    the merge. max_expansions > 0 caps each graph piece's expansions.
    mode "root" answers every query by POST on the root graph alone."""
    parts = []
    w = max(ef, k)
    for p in pieces_of(index, lq, rq, mode):
        if trav_X is None:
            if p.kind == "scan":
                parts.append(bruteforce(index.X, q, p.pl, p.pr, k, index.metric))
            else:
                ids, dd = graph_search(index, p.depth, p.heap, q, w, p.pl, p.pr, counters,
                                       max_expansions=max_expansions)
                parts.append((ids[:k], dd[:k]))
            continue
        if p.kind == "scan":
            ids, _ = bruteforce(trav_X, q, p.pl, p.pr, w, index.metric)
        else:
            ids, _ = graph_search(index, p.depth, p.heap, q, w, p.pl, p.pr, counters, X=trav_X,
                                  max_expansions=max_expansions)
        exact = distances(index.X[ids], q, index.metric)
        order = np.lexsort((ids, exact))[:k]
        parts.append((ids[order], exact[order]))
    return merge_topk(parts, k)


def recall_at_k(found: Sequence[np.ndarray], truth: Sequence[np.ndarray]) -> float:
    """Mean over queries of |found ∩ truth| / |truth| (truth holds
    min(k, range width) ids per query)."""
    tot = 0.0
    for f, t in zip(found, truth):
        if len(t) == 0:
            tot += 1.0
            continue
        tot += len(set(np.asarray(f).tolist()) & set(np.asarray(t).tolist())) / len(t)
    return tot / max(1, len(truth))
