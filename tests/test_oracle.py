"""Pins for the CPU oracle: each test checks the oracle against something other
than itself (hand traces, closed forms, brute force, textbook routines)."""
import json
import os

import numpy as np
import pytest

import oracle as O
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------- re-ranking

def test_rerank_is_stable_sort_by_attribute():
    attr = np.array([3.0, 1.0, 2.0, 1.0, -5.0, 2.0])
    perm = O.rerank(attr)
    # rank 0 = smallest attribute; ties keep original order
    assert perm.tolist() == [4, 1, 3, 2, 5, 0]
    rng = np.random.default_rng(0)
    a = rng.integers(0, 20, size=500).astype(np.float64)
    assert np.array_equal(O.rerank(a), np.argsort(a, kind="stable"))


# ------------------------------------------------ decomposition (Alg 4)

def _all_nodes(n, leaf):
    """Every node of the segment tree as (l, r, depth, heap), by explicit
    breadth-first enumeration."""
    out, frontier, depth = [], [(0, n - 1, 0)], 0
    while frontier:
        nxt = []
        for (l, r, h) in frontier:
            out.append((l, r, depth, h))
            if r - l >= leaf:
                m = (l + r) // 2
                nxt += [(l, m, 2 * h + 1), (m + 1, r, 2 * h + 2)]
        frontier, depth = nxt, depth + 1
    return out


def _closed_form(nodes, leaf, lq, rq):
    """Independent statement of the decomposition: along the chain of nodes
    containing the query, take the shallowest that is a leaf or holds the query
    with ratio >= 1/2; if none, split at the mid of the deepest containing
    node and resolve each part the same way along its own chain."""
    def chain(a, b):
        return sorted([nd for nd in nodes if nd[0] <= a and b <= nd[1]], key=lambda t: t[2])

    def accept(nd, a, b):
        l, r = nd[0], nd[1]
        return (r - l < leaf) or (2 * (b - a + 1) >= r - l + 1)

    def resolve(a, b):
        for nd in chain(a, b):
            if accept(nd, a, b):
                kind = "scan" if nd[1] - nd[0] < leaf else "graph"
                return (kind, nd[0], nd[1], a, b, nd[3], nd[2])
        raise AssertionError("a suffix/prefix part always reaches an accepting node")

    ch = chain(lq, rq)
    for nd in ch:
        if accept(nd, lq, rq):
            kind = "scan" if nd[1] - nd[0] < leaf else "graph"
            return [(kind, nd[0], nd[1], lq, rq, nd[3], nd[2])]
    deepest = ch[-1]
    m = (deepest[0] + deepest[1]) // 2
    return [resolve(lq, m), resolve(m + 1, rq)]


@pytest.mark.parametrize("n,leaf", [(1, 1), (2, 1), (3, 1), (7, 1), (7, 2), (64, 1), (64, 4),
                                    (100, 3), (129, 8), (130, 16)])
def test_decompose_matches_closed_form_exhaustive(n, leaf):
    nodes = _all_nodes(n, leaf)
    for lq in range(n):
        for rq in range(lq, n):
            got = [(p.kind, p.node_l, p.node_r, p.pl, p.pr, p.heap, p.depth)
                   for p in O.decompose(n, leaf, lq, rq)]
            assert got == _closed_form(nodes, leaf, lq, rq), (n, leaf, lq, rq)


def _check_invariants(n, leaf, lq, rq, pieces):
    assert 1 <= len(pieces) <= 2                                   # Lemma 3
    # pieces partition [lq, rq] left to right
    assert pieces[0].pl == lq and pieces[-1].pr == rq
    for a, b in zip(pieces, pieces[1:]):
        assert b.pl == a.pr + 1
    for p in pieces:
        assert p.node_l <= p.pl <= p.pr <= p.node_r                 # piece inside its node
        size = p.node_r - p.node_l + 1
        if p.kind == "graph":
            assert size - 1 >= leaf
            assert 2 * (p.pr - p.pl + 1) >= size                     # elastic factor >= 1/2
        else:
            assert size - 1 < leaf


@pytest.mark.parametrize("n,leaf", [(1000, 16), (1023, 1), (257, 256), (256, 256)])
def test_decompose_invariants_exhaustive(n, leaf):
    for lq in range(n):
        for rq in range(lq, n):
            _check_invariants(n, leaf, lq, rq, O.decompose(n, leaf, lq, rq))


@pytest.mark.parametrize("n,leaf", [(2049, 1), (10_000, 256), (1_000_000, 256), (10_000_000, 256)])
def test_decompose_invariants_sampled(n, leaf):
    rng = np.random.default_rng(n)
    for _ in range(3000):
        a, b = sorted(rng.integers(0, n, size=2).tolist())
        _check_invariants(n, leaf, a, b, O.decompose(n, leaf, a, b))


def test_decompose_special_cases():
    # the full range is answered by the root graph alone
    assert O.decompose(1000, 16, 0, 999) == [O.Piece("graph", 0, 999, 0, 999, 0, 0)]
    # a single point inside a leaf is a scan of that point
    p = O.decompose(1000, 16, 5, 5)
    assert len(p) == 1 and p[0].kind == "scan" and (p[0].pl, p[0].pr) == (5, 5)
    # exactly half of the root, straddling mid: 500 points of [0,999] with
    # ratio 1/2 -> the root graph is accepted (the test is inclusive)
    p = O.decompose(1000, 16, 250, 749)
    assert p == [O.Piece("graph", 0, 999, 250, 749, 0, 0)]
    # one point less than half -> split at the root's mid (499)
    p = O.decompose(1000, 16, 251, 749)
    assert [(q.pl, q.pr) for q in p] == [(251, 499), (500, 749)]
    # whole tree is a leaf
    assert O.decompose(10, 16, 2, 7)[0].kind == "scan"


def test_graph_depths():
    assert O.graph_depths(10, 16) == 0
    assert O.graph_depths(17, 16) == 1
    assert O.graph_depths(10_000, 256) == 6      # 10000, 5000, ..., 313 > 256 >= 157
    assert O.graph_depths(1_000_000, 256) == 12


# --------------------------------------------------------- exact k-NN

def test_bruteforce_golden():
    g = json.load(open(os.path.join(GOLDEN, "alg1_traces.json")))["bruteforce"]
    X = np.array(g["points_1d"])[:, None]
    for c in g["cases"]:
        ranks, dd = O.bruteforce(X, np.array([c["q"]]), c["range"][0], c["range"][1], c["k"], c["metric"])
        assert ranks.tolist() == c["ranks"]
        assert np.allclose(dd, c["dist"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_bruteforce_vs_expanded_form(metric):
    """Against a differently-written distance (norm expansion) and argsort."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((400, 24))
    for _ in range(20):
        q = rng.standard_normal(24)
        l, r = sorted(rng.integers(0, 400, size=2).tolist())
        k = int(rng.integers(1, 30))
        ids, dd = O.bruteforce(X, q, l, r, k, metric)
        sub = X[l:r + 1]
        if metric == "l2":
            ref = (sub ** 2).sum(1) + (q ** 2).sum() - 2 * sub @ q
        else:
            ref = -np.array([sum(a * b for a, b in zip(row, q)) for row in sub])
        order = np.argsort(ref, kind="stable")[:k] + l
        assert ids.tolist() == order.tolist()
        assert len(ids) == min(k, r - l + 1)
        assert np.allclose(dd, ref[order - l], rtol=1e-9, atol=1e-9)


def test_merge_topk():
    a = (np.array([3, 9]), np.array([0.5, 2.0]))
    b = (np.array([12, 14, 15]), np.array([0.1, 2.0, 3.0]))
    ids, dd = O.merge_topk([a, b], 4)
    assert ids.tolist() == [12, 3, 9, 14]          # tie at 2.0 broken by rank
    assert dd.tolist() == [0.1, 0.5, 2.0, 2.0]


# ---------------------------------------------------- Algorithm 1 traces

def _path_index(points, adjacency, entries, metric):
    n = len(points)
    R = max(len(a) for a in adjacency)
    adj = np.full((1, n, R), O.NONE, dtype=np.uint32)
    for i, nb in enumerate(adjacency):
        adj[0, i, :len(nb)] = nb
    ent = np.full((1, len(entries)), -1, dtype=np.int32)
    ent[0, :] = entries
    X = np.array(points, dtype=np.float64)[:, None]
    return O.OracleIndex(X, np.arange(n), adj, ent, 1, R // 2 or 1, metric)


def test_graph_search_hand_traces():
    g = json.load(open(os.path.join(GOLDEN, "alg1_traces.json")))
    for c in g["cases"]:
        idx = _path_index(g["points_1d"], g["adjacency"], c["entries"], g["metric"])
        cnt = np.zeros(2, np.int64)
        ids, dd = O.graph_search(idx, 0, 0, np.array([c["q"]]), c["ef"], c["range"][0],
                                 c["range"][1], cnt)
        assert ids.tolist() == c["result_ranks"], c["why"]
        assert np.allclose(dd, c["result_dist"], atol=1e-12)
        assert int(cnt[0]) == c["expansions"], c["why"]
        assert int(cnt[1]) == c["distance_evals"], c["why"]


# --------------------------------------- build (Alg 3) + search (Alg 4)

@pytest.fixture(scope="module")
def small_index():
    w = synthetic.small_mixture(600, 16, 60, n_comp=8, seed=11, M=6, leaf_size=20)
    idx = O.build_index(w.base, w.attr, w.metric, w.leaf_size, w.M, efc=40, n_entries=4)
    return w, idx


def test_build_invariants(small_index):
    w, idx = small_index
    n, R = idx.n, idx.R
    assert idx.L == O.graph_depths(n, w.leaf_size)
    nodes = [nd for nd in _all_nodes(n, w.leaf_size) if nd[1] - nd[0] >= w.leaf_size]
    assert nodes and all(nd[2] < idx.L for nd in nodes)
    for (l, r, depth, h) in nodes:
        rows = idx.adj[depth, l:r + 1]
        for i, row in zip(range(l, r + 1), rows):
            nb = row[row != O.NONE].astype(np.int64)
            assert len(nb) <= R
            assert np.all(row[len(nb):] == O.NONE)          # packed to the left
            assert i not in nb                               # no self loops
            assert len(set(nb.tolist())) == len(nb)          # no duplicate edges
            assert np.all((nb >= l) & (nb <= r))             # edges stay inside the node
        ent = [e for e in idx.entries[h] if e >= 0]
        assert ent and all(l <= e <= r for e in ent)
        # almost every point is reachable from the entries; occlusion pruning
        # of reverse edges can orphan a few points, as in HNSW
        assert len(_reachable(idx, depth, h)) >= 0.99 * (r - l + 1)


def _reachable(idx, depth, h):
    ent = [int(e) for e in idx.entries[h] if e >= 0]
    seen, stack = set(ent), list(ent)
    while stack:
        u = stack.pop()
        for v in idx.adj[depth, u]:
            if v != O.NONE and int(v) not in seen:
                seen.add(int(v)); stack.append(int(v))
    return seen


def test_search_exact_when_ef_covers_node(small_index):
    """With ef >= node size, Algorithm 1 + POST visits every point reachable
    from the entries, so each graph piece returns the exact filtered k-NN of
    its reachable points and scan pieces the exact k-NN of the piece."""
    w, idx = small_index
    for i in range(len(w.queries)):
        l, r, k = int(w.l[i]), int(w.r[i]), 10
        q = w.queries[i]
        ids, dd = O.search(idx, q, l, r, k, ef=idx.n)
        parts = []
        for p in O.decompose(idx.n, idx.leaf_size, l, r):
            cand = np.arange(p.pl, p.pr + 1)
            if p.kind == "graph":
                reach = _reachable(idx, p.depth, p.heap)
                cand = np.array([c for c in cand if int(c) in reach], dtype=np.int64)
            dist = O.distances(idx.X[cand], q, w.metric)
            order = np.lexsort((cand, dist))[:k]
            parts.append((cand[order], dist[order]))
        gt, gd = O.merge_topk(parts, k)
        assert ids.tolist() == gt.tolist()
        assert np.allclose(dd, gd)


def test_search_result_properties(small_index):
    w, idx = small_index
    for i in range(len(w.queries)):
        l, r = int(w.l[i]), int(w.r[i])
        ids, dd = O.search(idx, w.queries[i], l, r, 10, ef=8)
        assert len(ids) >= min(10, r - l + 1) - 1
        assert np.all((ids >= l) & (ids <= r))
        assert len(set(ids.tolist())) == len(ids)
        assert np.all(np.diff(dd) >= 0)


def test_full_range_is_unfiltered_search(small_index):
    """A full-range query is answered by the root graph with no filtering:
    the same result as Algorithm 1 on the root from the root entries."""
    w, idx = small_index
    for i in range(10):
        ids, _ = O.search(idx, w.queries[i], 0, idx.n - 1, 10, ef=16)
        ids2, _ = O.graph_search(idx, 0, 0, w.queries[i], 16, 0, idx.n - 1)
        assert ids.tolist() == ids2[:10].tolist()


def test_leaf_range_is_exact_scan(small_index):
    w, idx = small_index
    for i in range(10):
        ids, _ = O.search(idx, w.queries[i], 100, 100 + w.leaf_size - 5, 5, ef=1)
        gt, _ = O.bruteforce(idx.X, w.queries[i], 100, 100 + w.leaf_size - 5, 5, w.metric)
        assert ids.tolist() == gt.tolist()


# ------------------------------------------------- low-precision storage

def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(50_000) * rng.choice([1e-3, 1.0, 1e2, 1e5], 50_000)).astype(np.float32)
    x = np.concatenate([x, np.float32([0.0, -0.0, 1.0, 1.00390625, 1.01171875])])  # exact ties
    ref = torch.tensor(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(O.bf16_round(x), ref)


def test_fp8_grid_and_codes():
    from oracle import esg_oracle as EO
    g = O.fp8_e4m3_grid()
    assert g[0] == 0.0 and g[1] == 2.0 ** -9 and g[8] == 2.0 ** -6 and g[126] == 448.0
    assert np.all(np.diff(g) > 0)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    v = (rng.standard_normal(100_000) * rng.choice([1e-4, 1e-2, 1.0, 50.0, 300.0], 100_000)).astype(np.float32)
    mids = ((g[1:] + g[:-1]) / 2).astype(np.float32)                 # exact ties -> even code
    v = np.concatenate([v, mids, -mids])
    v = v[np.abs(v) <= 448]
    ref = torch.tensor(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(EO._fp8_code(v), ref)
    # saturation (satfinite) beyond the largest finite value
    assert EO._fp8_code(np.float32([1e9, -1e9, 449.0])).tolist() == [126, 254, 126]


def test_fp8_rows_reconstruct_within_half_ulp():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((200, 24)).astype(np.float32)
    X[3] = 0.0
    codes, s = O.fp8_quantize_rows(X)
    assert s[3] == 0 and np.all(codes[3] == 0)
    rec = O.fp8_to_float(codes) * s[:, None]
    # relative step of E4M3 is 2^-3; the row maximum maps to 448 exactly
    err = np.abs(rec - X)
    assert np.all(err <= np.maximum(2.0 ** -4 * np.abs(X), 2.0 ** -10 * s[:, None]) + 1e-12)
    assert np.all(np.abs(O.fp8_to_float(codes).max(1)[s > 0]) <= 448)


def test_lowprec_search_reranks_exactly(small_index):
    """With traversal rows equal to the exact rows the re-ranked search is the
    plain search; with bf16 rows every returned distance is exact."""
    w, idx = small_index
    for i in range(10):
        a, _ = O.search(idx, w.queries[i], int(w.l[i]), int(w.r[i]), 10, 16)
        b, bd = O.search(idx, w.queries[i], int(w.l[i]), int(w.r[i]), 10, 16, trav_X=idx.X)
        assert a.tolist() == b.tolist()
        c, cd = O.search(idx, w.queries[i], int(w.l[i]), int(w.r[i]), 10, 16,
                         trav_X=O.traversal_rows(idx.X.astype(np.float32), "bf16"))
        assert np.allclose(cd, O.distances(idx.X[c], w.queries[i], w.metric))


# --------------------------------------------- learned predictor (MLP)

def test_mlp_gradient_matches_central_differences():
    from oracle import mlp
    rng = np.random.default_rng(4)
    F, B = 8, 37
    p = rng.standard_normal(mlp.n_params(F)) * 0.3
    X = rng.standard_normal((B, F)) * 3 + 1
    T = rng.standard_normal((B, 2))
    mu, sigma = X.mean(0), X.std(0) + 0.5
    for q in (0.5, 0.9):
        loss, g = mlp.loss_and_grad(p, X, T, mu, sigma, q)
        assert np.isclose(loss, mlp.pinball(mlp.forward(p, X, mu, sigma)[0], T, q))
        h = 1e-6
        idx = rng.choice(len(p), 120, replace=False)
        num = np.array([(mlp.pinball(mlp.forward(p + h * e, X, mu, sigma)[0], T, q) -
                         mlp.pinball(mlp.forward(p - h * e, X, mu, sigma)[0], T, q)) / (2 * h)
                        for e in np.eye(len(p))[idx]])
        assert np.allclose(g[idx], num, rtol=1e-4, atol=1e-8)


def test_mlp_pinball_quantile_property():
    """Minimising the pinball loss of a constant predicts the q-quantile."""
    from oracle import mlp
    t = np.linspace(0, 1, 1001)[:, None].repeat(2, 1)
    grid = np.linspace(0, 1, 201)
    best = grid[np.argmin([mlp.pinball(np.full_like(t, c), t, 0.9) for c in grid])]
    assert abs(best - 0.9) <= 0.005


def test_adam_first_step_moves_by_lr():
    from oracle import mlp
    p = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(5), np.zeros(5), 1, 0.01)
    # bias-corrected first step is lr * sign(g) (where g != 0)
    assert np.allclose(p1, -0.01 * np.sign(g), atol=1e-9)


# ------------------------------------------- Algorithm 3 hand-traced build

def _load_build_fn(lib_path):
    import ctypes
    lib = ctypes.CDLL(lib_path)
    P = ctypes.c_void_p
    lib.oracle_build.restype = ctypes.c_int
    lib.oracle_build.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P,
                                 ctypes.c_int]
    return lib.oracle_build


def _build_with(fn, X, metric, leaf, M, efc, E, fanout=2):
    """oracle_build through `fn` (the oracle's library or a mutant of it)."""
    n, d = X.shape
    L = O.graph_depths(n, leaf, fanout)
    adj = np.empty((L, n, 2 * M), np.uint32)
    ent = np.empty((O.tree_nodes(L, fanout), E), np.int32)
    X = np.ascontiguousarray(X, dtype=np.float64)
    assert fn(X.ctypes.data, n, d, O.METRICS[metric], leaf, M, efc, E, L, adj.ctypes.data,
              ent.ctypes.data, fanout) == 0
    return adj, ent


def _alg3_golden():
    g = json.load(open(os.path.join(GOLDEN, "alg3_build.json")))
    X = np.array(g["points_1d"], np.float64)[:, None]
    want = np.full((len(g["adjacency"]), len(X), 2 * g["M"]), O.NONE, np.uint32)
    for t, rows in enumerate(g["adjacency"]):
        for i, nb in enumerate(rows):
            want[t, i, :len(nb)] = nb
    return g, X, want


def _matches_golden(adj, ent, g, want):
    return adj.shape == want.shape and np.array_equal(adj, want) and \
        ent.tolist() == g["entries"]


def test_build_hand_trace():
    """Every row of every depth and every node's entries equal the hand trace
    of Algorithm 3 (tests/golden/alg3_build.json)."""
    g, X, want = _alg3_golden()
    idx = O.build_index(X, None, g["metric"], g["leaf_size"], g["M"], efc=g["efc"],
                        n_entries=g["n_entries"])
    for t in range(want.shape[0]):
        assert idx.adj[t].tolist() == want[t].tolist(), f"depth {t}"
    assert idx.entries.tolist() == g["entries"]


# Mistakes planted in a copy of the oracle's C source (compiled on the CPU);
# each must change the build of the hand-traced case. "fresh" rebuilds the
# left half by insertion instead of copying the left child's graph: the
# copy is only a saving of work, so that variant must give the same graph.
_ALG3_MUTANTS = {
    "no_copy": ("memcpy(row(c, depth, i), row(c, depth + 1, i), sizeof(uint32_t) * (size_t)c->R);",
                "(void)0;"),
    "right_half_descending": ("for (int64_t i = b1; i <= r; ++i) insert_point(c, depth, l, i);",
                              "for (int64_t i = r; i >= b1; --i) insert_point(c, depth, l, i);"),
    "full_row_drops_new_edge": ("if (du < c->R) { ru[du] = (uint32_t)v; continue; }",
                                "if (du < c->R) { ru[du] = (uint32_t)v; continue; } else continue;"),
    "full_row_keeps_nearest": ("int nk = select_neighbours(c->X, c->d, c->metric, cand, du + 1, c->R, keep);",
                               "int nk = 0; for (; nk < c->R && nk < du + 1; ++nk) keep[nk] = cand[nk].id;"),
    "occlusion_compares_to_kept": ("if (dist(c, X + (size_t)keep[s] * d, d, metric) < cand[i].d) { good = 0; break; }",
                                   "if (dist(c, X + (size_t)keep[s] * d, d, metric) > cand[i].d) { good = 0; break; }"),
    "fresh": ("if (first) {", "if (0) {"),
}


def _compile_mutant(tmp_path, name):
    import subprocess
    src = open(os.path.join(os.path.dirname(O.__file__), "esg_oracle.c")).read()
    old, new = _ALG3_MUTANTS[name]
    assert src.count(old) == 1, f"mutation site of {name} not found"
    p = tmp_path / f"{name}.c"
    p.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(p), "-o", str(so), "-lm"])
    return str(so)


@pytest.mark.parametrize("name", sorted(_ALG3_MUTANTS))
def test_build_hand_trace_rejects_planted_mistakes(tmp_path, name):
    g, X, want = _alg3_golden()
    fn = _load_build_fn(_compile_mutant(tmp_path, name))
    adj, ent = _build_with(fn, X, g["metric"], g["leaf_size"], g["M"], g["efc"], g["n_entries"])
    if name == "fresh":
        assert _matches_golden(adj, ent, g, want)
    else:
        assert not _matches_golden(adj, ent, g, want), name


# ------------------------------------- Adam, MLP forward, recall: hand values

# Three Adam steps worked by hand for beta1 = 0.5, beta2 = 0.75, eps = 0.25,
# lr = 0.1 from p = m = v = 0 with gradients g1, g2, g3 below:
#   step 1: m = [0.5, -1, 2], v = [0.25, 1, 4]; bias corrections 1/2, 1/4:
#           m^ = [1, -2, 4], v^ = [1, 4, 16], sqrt = [1, 2, 4];
#           p = -0.1 * [1/1.25, -2/2.25, 4/4.25] = [-2/25, 4/45, -8/85]
#   step 2: m = [1.75, 0.5, 1], v = [2.4375, 1.75, 3]; corrections 0.75, 0.4375:
#           m^ = [7/3, 2/3, 4/3], v^ = [39/7, 4, 48/7]
#   step 3: m = [0.375, 0.25, 1.5], v = [2.078125, 1.3125, 3.25];
#           corrections 0.875, 0.578125: m^ = [3/7, 2/7, 12/7],
#           v^ = [133/37, 84/37, 208/37]
_ADAM_G = [np.array([1.0, -2.0, 4.0]), np.array([3.0, 2.0, 0.0]), np.array([-1.0, 0.0, 2.0])]
_P1 = np.array([-2 / 25, 4 / 45, -8 / 85])
_P2 = _P1 - 0.1 * np.array([7 / 3, 2 / 3, 4 / 3]) / (np.sqrt([39 / 7, 4.0, 48 / 7]) + 0.25)
_P3 = _P2 - 0.1 * np.array([3 / 7, 2 / 7, 12 / 7]) / (np.sqrt([133 / 37, 84 / 37, 208 / 37]) + 0.25)
_ADAM_WANT = [_P1, _P2, _P3]
_ADAM_M = [np.array([0.5, -1.0, 2.0]), np.array([1.75, 0.5, 1.0]), np.array([0.375, 0.25, 1.5])]
_ADAM_V = [np.array([0.25, 1.0, 4.0]), np.array([2.4375, 1.75, 3.0]), np.array([2.078125, 1.3125, 3.25])]


def _adam_run(step_fn):
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    out = []
    for t, g in enumerate(_ADAM_G, start=1):
        p, m, v = step_fn(p, g, m, v, t, 0.1, beta1=0.5, beta2=0.75, eps=0.25)
        out.append((p.copy(), m.copy(), v.copy()))
    return out


def _adam_ok(out):
    return all(np.allclose(p, pw, rtol=0, atol=1e-12) and np.allclose(m, mw, atol=1e-12)
               and np.allclose(v, vw, atol=1e-12)
               for (p, m, v), pw, mw, vw in zip(out, _ADAM_WANT, _ADAM_M, _ADAM_V))


def test_adam_three_steps_hand_values():
    from oracle import mlp
    assert _adam_ok(_adam_run(mlp.adam_step))


def _adam_variant(kind):
    """Plausible wrong Adam steps (planted on the CPU only)."""
    def step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        b2 = beta1 if kind == "beta2_is_beta1" else beta2
        m = beta1 * m + (1 - beta1) * g
        v = b2 * v + (1 - b2) * g * g
        e = t - 1 if kind == "bias_exponent_t_minus_1" else t
        mh = m / (1 - beta1 ** max(e, 1)) if kind != "no_bias_correction" else m
        vh = v / (1 - b2 ** max(e, 1)) if kind != "no_bias_correction" else v
        if kind == "bias_exponent_t_minus_1" and t == 1:
            mh, vh = m / (1 - beta1), v / (1 - b2)
        if kind == "eps_inside_sqrt":
            return p - lr * mh / np.sqrt(vh + eps), m, v
        if kind == "v_from_beta1_correction":
            vh = v / (1 - beta1 ** t)
        return p - lr * mh / (np.sqrt(vh) + eps), m, v
    return step


@pytest.mark.parametrize("kind", ["beta2_is_beta1", "bias_exponent_t_minus_1", "no_bias_correction",
                                  "eps_inside_sqrt", "v_from_beta1_correction"])
def test_adam_hand_values_reject_planted_mistakes(kind):
    assert not _adam_ok(_adam_run(_adam_variant(kind))), kind


def _tiny_mlp():
    """A 2-feature network with a few non-zero weights (flat layout W1 [F, 64],
    b1, W2 [64, 64], b2, W3 [64, 2], b3). Hidden units 0-2 of layer 1:
    z0 = xh0 + xh1 - 1, z1 = -xh0 + 0.5, z2 = 2 xh1 - 3; layer 2:
    z0 = h0 - 0.5 h2 + 0.5, z1 = 2 h1 + h2 - 4; outputs
    y0 = h0 + 0.5 h1 + 0.25, y1 = -h0 + 3 h1 - 0.5; every other weight 0."""
    from oracle import mlp
    F, H = 2, mlp.HIDDEN
    W1 = np.zeros((F, H)); b1 = np.zeros(H)
    W1[:, 0] = [1, 1]; b1[0] = -1
    W1[:, 1] = [-1, 0]; b1[1] = 0.5
    W1[:, 2] = [0, 2]; b1[2] = -3
    W2 = np.zeros((H, H)); b2 = np.zeros(H)
    W2[0, 0] = 1; W2[2, 0] = -0.5; b2[0] = 0.5
    W2[1, 1] = 2; W2[2, 1] = 1; b2[1] = -4
    W3 = np.zeros((H, 2)); b3 = np.array([0.25, -0.5])
    W3[0, 0] = 1; W3[1, 0] = 0.5; W3[0, 1] = -1; W3[1, 1] = 3
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    mu, sigma = np.array([1.0, -1.0]), np.array([2.0, 0.5])
    # by hand: x -> xh = ((x0 - 1) / 2, (x1 + 1) / 0.5) -> h1 -> h2 -> y
    #   [3, 0]     -> [1, 2]  -> h1 [2, 0, 1]   -> h2 [2, 0] (z2_1 = -3 cut) -> [2.25, -2.5]
    #   [-1, -0.5] -> [-1, 1] -> h1 [0, 1.5, 0] -> h2 [0.5, 0] (z2_1 = -1)  -> [0.75, -1.0]
    #   [5, 1]     -> [2, 4]  -> h1 [5, 0, 5]   -> h2 [3, 1]                 -> [3.75, -0.5]
    X = np.array([[3.0, 0.0], [-1.0, -0.5], [5.0, 1.0]])
    Y = np.array([[2.25, -2.5], [0.75, -1.0], [3.75, -0.5]])
    return p, X, mu, sigma, Y


def test_mlp_forward_hand_values():
    from oracle import mlp
    p, X, mu, sigma, Y = _tiny_mlp()
    y, _ = mlp.forward(p, X, mu, sigma)
    assert np.allclose(y, Y, rtol=0, atol=1e-12)


def test_mlp_forward_hand_values_reject_planted_mistakes():
    from oracle import mlp
    p, X, mu, sigma, Y = _tiny_mlp()
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, 2)
    relu = lambda z: np.maximum(z, 0)
    variants = {
        "standardise_by_multiplying": lambda x: relu(relu(((x - mu) * sigma) @ W1 + b1) @ W2 + b2) @ W3 + b3,
        "no_standardisation": lambda x: relu(relu(x @ W1 + b1) @ W2 + b2) @ W3 + b3,
        "no_relu_layer1": lambda x: relu((((x - mu) / sigma) @ W1 + b1) @ W2 + b2) @ W3 + b3,
        "no_relu_layer2": lambda x: (relu(((x - mu) / sigma) @ W1 + b1) @ W2 + b2) @ W3 + b3,
        "relu_on_output": lambda x: relu(relu(relu(((x - mu) / sigma) @ W1 + b1) @ W2 + b2) @ W3 + b3),
        "w2_transposed": lambda x: relu(relu(((x - mu) / sigma) @ W1 + b1) @ W2.T + b2) @ W3 + b3,
    }
    for name, f in variants.items():
        assert not np.allclose(f(X), Y, atol=1e-9), name


def test_recall_at_k_hand_case():
    """Per-query |found ∩ truth| / |truth| averaged over queries, ids counted
    once, an empty truth set (no point in range) counting as 1:
    q0 {1,2,3} vs {2,3,4,9} -> 2/4; q1 empty truth -> 1; q2 nothing found of
    {1} -> 0; q3 {7,8} vs {8,7} -> 1; mean 0.625."""
    found = [np.array([1, 2, 2, 3]), np.array([5]), np.array([], np.int64), np.array([7, 8])]
    truth = [np.array([2, 3, 4, 9]), np.array([], np.int64), np.array([1]), np.array([8, 7])]
    assert O.recall_at_k(found, truth) == pytest.approx(0.625, abs=1e-15)
    # planted mistakes: duplicates counted twice (0.6875), empty truth as 0 (0.375)
    dup = np.mean([sum(1 for f in fo if f in set(t.tolist())) / len(t) if len(t) else 1.0
                   for fo, t in zip(found, truth)])
    empty0 = np.mean([len(set(fo.tolist()) & set(t.tolist())) / len(t) if len(t) else 0.0
                      for fo, t in zip(found, truth)])
    assert dup == pytest.approx(0.6875) and empty0 == pytest.approx(0.375)


def test_node_rows_search_equals_level_search(small_index):
    """Searching one node from its own rows (row_base = the node's first rank)
    gives the same answer as searching it inside the whole level: a node's
    edges never leave it."""
    w, idx = small_index
    for i in range(30):
        for p in O.decompose(idx.n, idx.leaf_size, int(w.l[i]), int(w.r[i])):
            if p.kind != "graph":
                continue
            a = O.graph_search(idx, p.depth, p.heap, w.queries[i], 12, p.pl, p.pr)
            rows = slice(p.node_l, p.node_r + 1)
            b = O.graph_search_rows(idx.X[rows], idx.adj[p.depth][rows], idx.entries[p.heap], w.metric,
                                    w.queries[i], 12, p.pl, p.pr, row_base=p.node_l)
            assert a[0].tolist() == b[0].tolist() and np.array_equal(a[1], b[1])


def test_graph_search_expansion_cap_hand_trace():
    """The first hand trace of tests/golden/alg1_traces.json (q = 5.2, entry 0,
    ef = 2, full range) with at most 3 expansions: expanding 0, 1, 2 reaches
    1, 2, 3 (Q = {3, 2}); rank 3 is popped, passes the stop test (Q's worst
    is 2 at 10.24 > 4.84) and the budget ends the search: result [3, 2],
    3 expansions, 4 distance evaluations, one capped search. A cap of 7 or
    more does not change the uncapped trace."""
    g = json.load(open(os.path.join(GOLDEN, "alg1_traces.json")))
    c = g["cases"][0]
    idx = _path_index(g["points_1d"], g["adjacency"], c["entries"], g["metric"])
    cnt = np.zeros(3, np.int64)
    ids, dd = O.graph_search(idx, 0, 0, np.array([c["q"]]), c["ef"], 0, 7, cnt, max_expansions=3)
    assert ids.tolist() == [3, 2] and np.allclose(dd, [4.84, 10.24], atol=1e-12)
    assert cnt.tolist() == [3, 4, 1]
    cnt = np.zeros(3, np.int64)
    ids, _ = O.graph_search(idx, 0, 0, np.array([c["q"]]), c["ef"], 0, 7, cnt, max_expansions=7)
    assert ids.tolist() == c["result_ranks"] and cnt.tolist() == [7, 8, 0]


# ------------------------------ larger fanout (Lemma 4), ESG-1D (Lemma 2), root

def _all_nodes_f(n, leaf, f):
    """Every node of the fanout-f tree as (l, r, depth, heap), breadth first,
    with child bounds l + ceil(j len / f) computed in exact integers."""
    out, frontier, depth = [], [(0, n - 1, 0)], 0
    while frontier:
        nxt = []
        for (l, r, h) in frontier:
            out.append((l, r, depth, h))
            if r - l >= leaf:
                ln = r - l + 1
                for j in range(f):
                    a = l + (j * ln + f - 1) // f
                    b = l + ((j + 1) * ln + f - 1) // f - 1
                    if a <= b:
                        nxt.append((a, b, f * h + 1 + j))
        frontier, depth = nxt, depth + 1
    return out


def _closed_form_f(nodes, leaf, f, lq, rq):
    """Independent statement of the fanout-f choice: along the chain of nodes
    containing the query, the shallowest that is a leaf or holds it with
    f |q| >= |node|; if none, the deepest containing node's children the query
    overlaps (at most two, Lemma 4) each resolved the same way along their own
    chains."""
    def chain(a, b):
        return sorted([nd for nd in nodes if nd[0] <= a and b <= nd[1]], key=lambda t: t[2])

    def accept(nd, a, b):
        return (nd[1] - nd[0] < leaf) or (f * (b - a + 1) >= nd[1] - nd[0] + 1)

    def resolve(a, b):
        for nd in chain(a, b):
            if accept(nd, a, b):
                return ("scan" if nd[1] - nd[0] < leaf else "graph", nd[0], nd[1], a, b, nd[3], nd[2])
        raise AssertionError("unreachable")

    ch = chain(lq, rq)
    for nd in ch:
        if accept(nd, lq, rq):
            return [resolve(lq, rq)]
    deepest = ch[-1]
    kids = [nd for nd in nodes if nd[2] == deepest[2] + 1 and deepest[0] <= nd[0] and nd[1] <= deepest[1]
            and nd[0] <= rq and nd[1] >= lq]
    assert len(kids) <= 2                                             # Lemma 4
    return [resolve(max(lq, nd[0]), min(rq, nd[1])) for nd in sorted(kids)]


@pytest.mark.parametrize("n,leaf,f", [(1, 1, 4), (10, 1, 3), (37, 1, 4), (64, 2, 4), (100, 3, 8),
                                      (130, 1, 16), (90, 5, 5), (257, 16, 16)])
def test_decompose_fanout_matches_closed_form_exhaustive(n, leaf, f):
    nodes = _all_nodes_f(n, leaf, f)
    for lq in range(n):
        for rq in range(lq, n):
            got = [(p.kind, p.node_l, p.node_r, p.pl, p.pr, p.heap, p.depth)
                   for p in O.decompose(n, leaf, lq, rq, f)]
            assert got == _closed_form_f(nodes, leaf, f, lq, rq), (n, leaf, f, lq, rq)


@pytest.mark.parametrize("f", [2, 3, 4, 8, 16])
def test_decompose_fanout_lemma4_invariants(f):
    """At most two pieces that partition the range, each inside its node, and
    every graph piece covers at least 1/f of its node (Lemma 4)."""
    rng = np.random.default_rng(f)
    for n, leaf in [(1000, 16), (4096, 64), (10_000_000, 256)]:
        for _ in range(2000):
            a, b = sorted(rng.integers(0, n, size=2).tolist())
            ps = O.decompose(n, leaf, a, b, f)
            assert 1 <= len(ps) <= 2 and ps[0].pl == a and ps[-1].pr == b
            for x, y in zip(ps, ps[1:]):
                assert y.pl == x.pr + 1
            for p in ps:
                assert p.node_l <= p.pl <= p.pr <= p.node_r
                size = p.node_r - p.node_l + 1
                if p.kind == "graph":
                    assert f * (p.pr - p.pl + 1) >= size and size - 1 >= leaf
                else:
                    assert size - 1 < leaf


def test_fanout2_children_are_algorithm3_halves():
    for l, r in [(0, 0), (0, 1), (3, 10), (5, 1000), (0, 999_999)]:
        kids = O.children(l, r, 2)
        mid = (l + r) // 2
        want = [(l, mid, 0)] + ([(mid + 1, r, 1)] if mid + 1 <= r else [])
        assert kids == want


@pytest.mark.parametrize("n,B", [(1, 2), (2, 2), (7, 2), (100, 2), (100, 3), (1000, 4), (1023, 10), (4096, 16)])
def test_decompose_prefix_exhaustive(n, B):
    """Lemma 2 with base B: the chosen prefix graph contains [0, r] and covers
    more than 1/B of it is covered by the query; the level is the largest i
    with B^i (r + 1) <= n (exact integer powers, a different computation)."""
    sizes = O.prefix_sizes(n, B)
    assert sizes[0] == n and sizes[-1] >= 1 and sizes[-1] // B == 0
    assert all(sizes[i + 1] == n // B ** (i + 1) for i in range(len(sizes) - 1))
    for r in range(n):
        (p,) = O.decompose_prefix(n, B, 0, r)
        i = 0
        while B ** (i + 1) * (r + 1) <= n:
            i += 1
        assert (p.kind, p.node_l, p.node_r, p.pl, p.pr, p.heap, p.depth) == \
            ("graph", 0, n // B ** i - 1, 0, r, i, i)
        size = p.node_r + 1
        assert size >= r + 1 and B * (r + 1) > size            # containment, ratio > 1/B
    with pytest.raises(ValueError):
        O.decompose_prefix(n, B, 1, n - 1) if n > 1 else O.decompose_prefix(n, B, 0, 1)


def test_decompose_root_mode():
    assert O.decompose_root(1000, 16, 5, 7) == [O.Piece("graph", 0, 999, 5, 7, 0, 0)]
    assert O.decompose_root(10, 16, 2, 3) == [O.Piece("scan", 0, 9, 2, 3, 0, 0)]


def _golden_f4():
    g = json.load(open(os.path.join(GOLDEN, "alg3_build_fanout4.json")))
    X = np.array(g["points_1d"], np.float64)[:, None]
    want = np.full((len(g["adjacency"]), len(X), 2 * g["M"]), O.NONE, np.uint32)
    for t, rows in enumerate(g["adjacency"]):
        for i, nb in enumerate(rows):
            want[t, i, :len(nb)] = nb
    return g, X, want


def test_build_fanout4_hand_trace():
    g, X, want = _golden_f4()
    idx = O.build_index(X, None, g["metric"], g["leaf_size"], g["M"], efc=g["efc"],
                        n_entries=g["n_entries"], fanout=g["fanout"])
    assert idx.L == 2 and idx.adj.tolist() == want.tolist()
    assert idx.entries.tolist() == g["entries"]


def test_build_fanout4_hand_trace_rejects_floor_split(tmp_path):
    """Child bounds l + floor(j len / f) instead of the ceiling change the
    nodes of this 10-point tree, and so the graphs."""
    import subprocess
    src = open(os.path.join(os.path.dirname(O.__file__), "esg_oracle.c")).read()
    old = "return l + ((int64_t)j * len + f - 1) / f;"
    assert src.count(old) == 1
    p = tmp_path / "floor.c"
    p.write_text(src.replace(old, "return l + ((int64_t)j * len) / f;"))
    so = tmp_path / "floor.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(p), "-o", str(so), "-lm"])
    g, X, want = _golden_f4()
    adj, ent = _build_with(_load_build_fn(str(so)), X, g["metric"], g["leaf_size"], g["M"], g["efc"],
                           g["n_entries"], fanout=4)
    assert not (np.array_equal(adj, want) and ent.tolist() == g["entries"])


def _check_prefix_golden(build):
    g = json.load(open(os.path.join(GOLDEN, "alg2_build.json")))
    X = np.array(g["points_1d"], np.float64)[:, None]
    ok = True
    for c in g["cases"]:
        idx = build(X, g, c["base"])
        ok &= O.prefix_sizes(len(X), c["base"]) == c["sizes"]
        for i, rows in enumerate(c["levels"]):
            lev = idx.level(i)
            ok &= len(lev) == len(rows)
            for row, nb in zip(lev, rows):
                ok &= row[row != O.NONE].tolist() == nb and bool(np.all(row[len(nb):] == O.NONE))
        ok &= idx.entries.tolist() == c["entries"]
    return ok


def test_build_prefix_hand_trace():
    assert _check_prefix_golden(lambda X, g, B: O.build_prefix_index(
        X, None, g["metric"], g["M"], efc=g["efc"], n_entries=g["n_entries"], base_b=B))


@pytest.mark.parametrize("name,old,new", [
    ("snapshot_one_point_late", "while (lev >= 1 && v + 1 == size[lev]) {", "while (lev >= 1 && v == size[lev]) {"),
    ("no_snapshot", "memcpy(row(&c, lev, i), row(&c, 0, i), sizeof(uint32_t) * (size_t)c.R);", "(void)0;"),
    ("descending_insertion", "insert_point(&c, 0, 0, v);", "insert_point(&c, 0, 0, n - 1 - v);"),
])
def test_build_prefix_hand_trace_rejects_planted_mistakes(tmp_path, name, old, new):
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(O.__file__), "esg_oracle.c")).read()
    assert src.count(old) == 1, name
    p = tmp_path / f"{name}.c"
    p.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(p), "-o", str(so), "-lm"])
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.oracle_build_prefix.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]

    def build(X, g, B):
        sizes = O.prefix_sizes(len(X), B)
        adj = np.empty((sum(sizes), 2 * g["M"]), np.uint32)
        ent = np.empty((len(sizes), g["n_entries"]), np.int32)
        Xc = np.ascontiguousarray(X)
        lib.oracle_build_prefix(Xc.ctypes.data, len(X), 1, 0, B, g["M"], g["efc"], g["n_entries"],
                                len(sizes), adj.ctypes.data, ent.ctypes.data)
        return O.OracleIndex(Xc, np.arange(len(X)), adj, ent, 0, g["M"], g["metric"], "prefix", B)

    assert not _check_prefix_golden(build), name


def test_prefix_search_is_exact_when_ef_covers_the_prefix():
    """A prefix query searched with ef >= the prefix graph's size visits every
    point reachable from the entries: the exact k-NN of those points."""
    w = synthetic.small_mixture(700, 16, 40, n_comp=8, seed=12, M=6)
    idx = O.build_prefix_index(w.base, w.attr, w.metric, w.M, efc=40, n_entries=4, base_b=2)
    for i in range(len(w.queries)):
        r = int(w.r[i])
        ids, dd = O.search(idx, w.queries[i], 0, r, 10, ef=idx.n)
        (p,) = O.decompose_prefix(idx.n, 2, 0, r)
        lev = idx.level(p.depth)
        seen = set(int(e) for e in idx.entries[p.heap] if e >= 0)
        stack = list(seen)
        while stack:
            u = stack.pop()
            for v in lev[u]:
                if v != O.NONE and int(v) not in seen:
                    seen.add(int(v)); stack.append(int(v))
        cand = np.array(sorted(c for c in seen if c <= r), np.int64)
        dist = O.distances(idx.X[cand], w.queries[i], w.metric)
        order = np.lexsort((cand, dist))[:10]
        assert ids.tolist() == cand[order].tolist()
        assert len(seen) >= 0.99 * lev.shape[0]


def test_root_mode_search_is_root_graph_search(small_index):
    w, idx = small_index
    for i in range(10):
        l, r = int(w.l[i]), int(w.r[i])
        a, _ = O.search(idx, w.queries[i], l, r, 10, 16, mode="root")
        b, _ = O.graph_search(idx, 0, 0, w.queries[i], 16, l, r)
        assert a.tolist() == b[:10].tolist()
