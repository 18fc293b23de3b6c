"""GPU parity against the CPU oracle, through the C ABI (ctypes binding).

- decomposition: bit-exact, exhaustive for small trees, all queries of the
  workloads;
- brute force: ids equal to the float64 oracle's wherever the float64 gap
  between neighbours exceeds float32 rounding, distances within 1e-5
  relative, ties ordered by row;
- graph search on a graph built by the oracle (so that no oracle input comes
  from the GPU): recall@k within 0.5 points of the oracle's Algorithm 1 on the
  same graph and ef, nearly all queries identical;
- edge cases: invalid queries, width 1, k above the width, leaf-only ranges.
"""
import numpy as np
import pytest

import oracle as O
import synthetic

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2504_04018_gb300")

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    E.load_library()
    return torch.device("cuda:0")


def _t(a, dev, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=dtype)


# ------------------------------------------------------------ decomposition

def _gpu_pieces(n, leaf, l, r, dev):
    pieces, npieces = E.esg_decompose_batch(n, leaf, _t(l, dev, torch.int64), _t(r, dev, torch.int64))
    torch.cuda.synchronize()
    cols = [c.cpu().numpy() for c in E.unpack_pieces(pieces)]
    return cols, npieces.cpu().numpy()


def _check_pieces(n, leaf, l, r, cols, npieces):
    node_l, node_r, pl, pr, heap, depth, kind = cols
    for i in range(len(l)):
        want = O.decompose(n, leaf, int(l[i]), int(r[i]))
        assert npieces[i] == len(want), (n, leaf, l[i], r[i])
        for s, p in enumerate(want):
            got = (int(node_l[i, s]), int(node_r[i, s]), int(pl[i, s]), int(pr[i, s]),
                   int(heap[i, s]), int(depth[i, s]), int(kind[i, s]))
            exp = (p.node_l, p.node_r, p.pl, p.pr, p.heap, p.depth,
                   E.PIECE_GRAPH if p.kind == "graph" else E.PIECE_SCAN)
            assert got == exp, (n, leaf, l[i], r[i], s)
        for s in range(len(want), 2):
            assert int(kind[i, s]) == 0


@pytest.mark.parametrize("n,leaf", [(1, 1), (7, 1), (100, 3), (1000, 16), (1023, 1)])
def test_decompose_exhaustive(dev, n, leaf):
    ll, rr = np.triu_indices(n)
    cols, npieces = _gpu_pieces(n, leaf, ll, rr, dev)
    _check_pieces(n, leaf, ll, rr, cols, npieces)


@pytest.mark.parametrize("n,leaf", [(300, 64), (600, 256), (1100, 1024)])
def test_decompose_exhaustive_leaf_sweep(dev, n, leaf):
    """Leaf sizes 64, 256 and 1024, every range of a tree a few leaves deep."""
    ll, rr = np.triu_indices(n)
    cols, npieces = _gpu_pieces(n, leaf, ll, rr, dev)
    _check_pieces(n, leaf, ll, rr, cols, npieces)


@pytest.mark.parametrize("n,leaf", [(5_000, 1), (50_000, 64), (1_000_000, 256), (10_000_000, 1024)])
def test_decompose_sampled_leaf_sweep(dev, n, leaf):
    """Sampled ranges (log-uniform widths, uniform left ends) of large trees."""
    rng = np.random.default_rng(n + leaf)
    w = np.maximum(1, np.round(np.exp(rng.uniform(0, np.log(n), 4000)))).astype(np.int64)
    l = (rng.random(4000) * (n - w + 1)).astype(np.int64)
    r = l + w - 1
    cols, npieces = _gpu_pieces(n, leaf, l, r, dev)
    _check_pieces(n, leaf, l, r, cols, npieces)


def test_decompose_invalid_and_workload_ranges(dev):
    l = np.array([5, -1, 0, 3, 999_999, 0])
    r = np.array([4, 3, 1_000_000, 3, 999_999, 999_999])
    cols, npieces = _gpu_pieces(1_000_000, 256, l, r, dev)
    assert npieces.tolist() == [0, 0, 0, 1, 1, 1]
    for mk, n in [(synthetic.tiny, 10_000), (lambda: synthetic.scale(n=1_000_000, nq=10_000, d=8), 1_000_000)]:
        w = mk()
        cols, npieces = _gpu_pieces(n, 256, w.l, w.r, dev)
        _check_pieces(n, 256, w.l, w.r, cols, npieces)


# --------------------------------------------------------------- brute force

def _check_bruteforce(X, Q, l, r, k, metric, ids, dist, count):
    """Returns the largest distance error seen, in units of the plain
    relative bar 1e-5 * scale (above 1 only where the FP32-sum bound is the
    one that holds)."""
    X64 = X.astype(np.float64)
    worst = 0.0
    for i in range(len(Q)):
        li, ri = int(l[i]), int(r[i])
        if not (0 <= li <= ri < len(X)):
            assert count[i] == 0 and np.all(ids[i] == -1)
            continue
        w = ri - li + 1
        gt, gd = O.bruteforce(X64, Q[i].astype(np.float64), li, ri, k + 1, metric)
        c = min(k, w)
        assert count[i] == c
        got = ids[i, :c]
        assert np.all(ids[i, c:] == -1) and np.all(np.isinf(dist[i, c:]))
        assert np.all((got >= li) & (got <= ri)) and len(set(got.tolist())) == c
        # distances of the returned ids, checked against float64
        ref = O.distances(X64[got], Q[i].astype(np.float64), metric)
        scale = np.maximum(np.abs(ref), 1e-2 * np.abs(gd).max() + 1e-30)
        # plus the forward error bound of a d-term FP32 sum, d u sum_j |term_j|
        # (u = 2^-24): an inner product of unit vectors can cancel to far below
        # its terms, so a relative bound alone is too tight there
        q64 = Q[i].astype(np.float64)
        terms = np.abs(X64[got] * q64) if metric == "ip" else (X64[got] - q64) ** 2
        fp32_sum = X.shape[1] * 2.0 ** -24 * terms.sum(axis=1)
        assert np.all(np.abs(dist[i, :c] - ref) <= np.maximum(REL_TOL * scale, fp32_sum))
        worst = max(worst, float(np.max(np.abs(dist[i, :c] - ref) / (REL_TOL * scale))))
        # ids: exact where float64 neighbours are separated beyond rounding
        tol = 4 * REL_TOL * (np.abs(gd).max() + 1e-30)
        kth = gd[c - 1]
        must = set(gt[:c][gd[:c] < kth - tol].tolist())
        assert must <= set(got.tolist())
        assert np.all(ref <= kth + tol)
        gaps = np.diff(gd[:min(c + 1, len(gd))])
        if np.all(gaps > tol):
            assert got.tolist() == gt[:c].tolist()
    return worst


@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("k", [1, 10, 100, 300])
def test_bruteforce_vs_oracle(dev, metric, k):
    w = synthetic.small_mixture(3001, 32, 150, n_comp=8, seed=5, metric=metric,
                                normalise=(metric == "ip"))
    X, Q = w.base, w.queries
    l, r = w.l.copy(), w.r.copy()
    # edge ranges: single point, full, invalid, out of bounds, a ragged tail
    l[:6] = [0, 17, 0, 10, -3, 2950]
    r[:6] = [0, 17, 3000, 9, 5, 3000]
    ids, dist, count = E.esg_bruteforce_filtered_knn(_t(X, dev), _t(Q, dev), _t(l, dev, torch.int64),
                                                     _t(r, dev, torch.int64), k, metric)
    torch.cuda.synchronize()
    worst = _check_bruteforce(X, Q, l, r, k, metric, ids.cpu().numpy(), dist.cpu().numpy(),
                              count.cpu().numpy())
    print(f"bruteforce {metric} k={k}: largest distance error = {worst:.3f} x (1e-5 relative bar)")


def test_bruteforce_ties_by_row(dev):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((50, 16)).astype(np.float32)
    X = np.concatenate([X, X, X])            # every row three times
    Q = rng.standard_normal((20, 16)).astype(np.float32)
    l = np.zeros(20, np.int64)
    r = np.full(20, 149, np.int64)
    ids, dist, count = E.esg_bruteforce_filtered_knn(_t(X, dev), _t(Q, dev), _t(l, dev), _t(r, dev), 9)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy()
    for i in range(20):
        gt, _ = O.bruteforce(X.astype(np.float64), Q[i].astype(np.float64), 0, 149, 9, "l2")
        assert ids[i].tolist() == gt.tolist()
        # ties: the three copies come in row order
        assert ids[i, :3].tolist() == sorted(ids[i, :3].tolist())


def test_bruteforce_uncertified_queries_escalate(dev, monkeypatch):
    """Equal distances leave no gap for the tensor-core certificate: such
    queries run again with a longer candidate list and then through the
    exact SIMT kernel; the answer is still the oracle's (ties by row)."""
    monkeypatch.delenv("ESG_BF_SIMT", raising=False)
    rng = np.random.default_rng(11)
    X = np.repeat(rng.standard_normal((1, 64)).astype(np.float32), 3000, axis=0)
    X[::7] += 0.5                           # some rows farther away
    Q = rng.standard_normal((40, 64)).astype(np.float32)
    l = rng.integers(0, 2000, 40).astype(np.int64)
    r = (l + rng.integers(0, 999, 40)).astype(np.int64)
    ids, dist, count = E.esg_bruteforce_filtered_knn(_t(X, dev), _t(Q, dev), _t(l, dev), _t(r, dev), 10)
    torch.cuda.synchronize()
    ids, count = ids.cpu().numpy(), count.cpu().numpy()
    for i in range(40):
        gt, _ = O.bruteforce(X.astype(np.float64), Q[i].astype(np.float64), int(l[i]), int(r[i]), 10, "l2")
        assert count[i] == len(gt)
        assert ids[i, :count[i]].tolist() == gt.tolist()


# ----------------------------------------------------- search on oracle graph

@pytest.fixture(scope="module")
def tiny_oracle_index():
    w = synthetic.tiny()
    idx = O.build_index(w.base, w.attr, w.metric, w.leaf_size, w.M, efc=200, n_entries=16)
    return w, idx


def _import(idx, w):
    Xr = w.base[idx.perm]
    return E.esg_index_import(Xr, idx.perm, idx.metric, idx.leaf_size, idx.adj, idx.entries)


def _gpu_search(gix, Q, l, r, k, k_max, ef, dev, **kw):
    out = E.esg_search_batch(gix, _t(Q, dev), _t(l, dev, torch.int64), _t(r, dev, torch.int64),
                             None if k is None else _t(k, dev, torch.int32), k_max, ef=ef,
                             want_stats=True, **kw)
    torch.cuda.synchronize()
    return [None if x is None else x.cpu().numpy() for x in out]


@pytest.mark.parametrize("ef", [16, 64, 200])
def test_search_parity_on_oracle_graph(dev, tiny_oracle_index, ef):
    w, idx = tiny_oracle_index
    gix = _import(idx, w)
    k = 10
    ids, dist, count, status, stats = _gpu_search(gix, w.queries, w.l, w.r, None, k, ef, dev)
    inv = np.empty(idx.n, np.int64)
    inv[idx.perm] = np.arange(idx.n)
    found_gpu, found_cpu, truth = [], [], []
    same = 0
    for i in range(len(w.queries)):
        l, r = int(w.l[i]), int(w.r[i])
        ranks = inv[ids[i, :count[i]]]                        # GPU ids are original ids
        assert np.all((ranks >= l) & (ranks <= r))
        assert len(set(ranks.tolist())) == len(ranks)
        assert np.all(np.diff(dist[i, :count[i]]) >= 0)
        cpu, _ = O.search(idx, w.queries[i], l, r, k, ef)
        gt, _ = O.bruteforce(idx.X, w.queries[i], l, r, k, w.metric)
        assert count[i] == min(k, r - l + 1)
        found_gpu.append(ranks); found_cpu.append(cpu); truth.append(gt)
        same += ranks.tolist() == cpu.tolist()
        assert status[i] & ~E.Q_OVERFLOW == 0
    rg, rc = O.recall_at_k(found_gpu, truth), O.recall_at_k(found_cpu, truth)
    assert abs(rg - rc) <= 0.005, (rg, rc)
    assert same >= 0.95 * len(w.queries)


@pytest.mark.parametrize("leaf,metric", [(1, "l2"), (64, "ip"), (256, "l2")])
def test_search_parity_leaf_sweep(dev, leaf, metric):
    """Oracle-built indexes with leaf sizes 1, 64 and 256 (both metrics): the
    GPU's Algorithm 1 matches the oracle's on the same graph and ef."""
    w = synthetic.small_mixture(4000, 32, 300, n_comp=16, seed=71 + leaf, M=8, leaf_size=leaf,
                                metric=metric, normalise=(metric == "ip"))
    idx = O.build_index(w.base, w.attr, w.metric, leaf, 8, efc=100, n_entries=8)
    gix = _import(idx, w)
    k, ef = 10, 32
    ids, dist, count, status, stats = _gpu_search(gix, w.queries, w.l, w.r, None, k, ef, dev)
    inv = np.empty(idx.n, np.int64)
    inv[idx.perm] = np.arange(idx.n)
    found_gpu, found_cpu, truth = [], [], []
    same = 0
    for i in range(len(w.queries)):
        l, r = int(w.l[i]), int(w.r[i])
        ranks = inv[ids[i, :count[i]]]
        assert np.all((ranks >= l) & (ranks <= r)) and len(set(ranks.tolist())) == len(ranks)
        assert count[i] == min(k, r - l + 1)
        cpu, _ = O.search(idx, w.queries[i], l, r, k, ef)
        gt, _ = O.bruteforce(idx.X, w.queries[i], l, r, k, w.metric)
        found_gpu.append(ranks); found_cpu.append(cpu); truth.append(gt)
        same += ranks.tolist() == cpu.tolist()
    rg, rc = O.recall_at_k(found_gpu, truth), O.recall_at_k(found_cpu, truth)
    assert abs(rg - rc) <= 0.005, (rg, rc)
    assert same >= 0.95 * len(w.queries)


def test_search_edge_cases(dev, tiny_oracle_index):
    w, idx = tiny_oracle_index
    gix = _import(idx, w)
    n = idx.n
    Q = np.repeat(w.queries[:1], 9, axis=0)
    l = np.array([5, 0, 0, 100, 42, 0, 9000, 0, -1])
    r = np.array([4, n, n - 1, 100, 50, n - 1, 9255, 255, 7])
    k = np.array([10, 10, 0, 10, 10, 40, 10, 10, 10], np.int32)
    ids, dist, count, status, stats = _gpu_search(gix, Q, l, r, k, 32, 16, dev)
    assert status[0] & E.Q_INVALID and count[0] == 0           # l > r
    assert status[1] & E.Q_INVALID and count[1] == 0           # r >= n
    assert status[2] & E.Q_INVALID and count[2] == 0           # k < 1
    assert count[3] == 1 and ids[3, 0] == idx.perm[100]        # width 1
    assert count[4] == 9                                       # k above the width
    assert status[5] & E.Q_INVALID                              # k > k_max
    assert status[8] & E.Q_INVALID                              # l < 0
    inv = np.empty(n, np.int64)
    inv[idx.perm] = np.arange(n)
    for i in (3, 4):                                           # leaf pieces are exact scans
        gt, gd = O.bruteforce(idx.X, Q[i], int(l[i]), int(r[i]), int(k[i]), w.metric)
        assert inv[ids[i, :count[i]]].tolist() == gt.tolist()
        assert np.allclose(dist[i, :count[i]], gd, rtol=REL_TOL)
    for i in (6, 7):                                           # small graph pieces: valid results
        got = inv[ids[i, :count[i]]]
        assert count[i] == 10 and np.all((got >= l[i]) & (got <= r[i]))
    assert np.all(ids[0] == -1)


def test_search_k_max_and_per_query_k(dev, tiny_oracle_index):
    w, idx = tiny_oracle_index
    gix = _import(idx, w)
    k = np.array([1, 5, 10, 100] * 50, np.int32)
    ids, dist, count, status, stats = _gpu_search(gix, w.queries, w.l, w.r, k, 128, 32, dev)
    for i in range(len(k)):
        c = min(int(k[i]), int(w.r[i] - w.l[i] + 1))
        assert count[i] == c
        assert np.all(ids[i, c:] == -1)


# ------------------------------------------------------------ product build

def test_product_build_invariants_and_recall(dev):
    w = synthetic.tiny()
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=16, metric=w.metric)
    adj, ent, perm = E.esg_index_export(gix)
    assert np.array_equal(perm, O.rerank(w.attr))
    n, R = gix.n, gix.R
    assert gix.L == O.graph_depths(n, w.leaf_size)
    X = w.base[perm].astype(np.float64)
    frontier = [(0, n - 1, 0)]
    for depth in range(gix.L):
        nxt = []
        for (l, r, h) in frontier:
            if r - l < w.leaf_size:
                continue
            rows = adj[depth, l:r + 1]
            valid = rows != 0xFFFFFFFF
            deg = valid.sum(1)
            assert np.all(deg <= R) and np.all(deg >= 1)
            for j in range(R - 1):
                assert np.all(valid[:, j] | ~valid[:, j + 1])
            nb = rows.astype(np.int64)
            self_ids = np.arange(l, r + 1)[:, None]
            assert not np.any(valid & (nb == self_ids))
            assert np.all(~valid | ((nb >= l) & (nb <= r)))
            e = ent[h][ent[h] >= 0]
            assert len(e) > 0 and np.all((e >= l) & (e <= r))
            seen, stack = set(e.tolist()), list(e.tolist())
            while stack:
                u = stack.pop()
                for v in adj[depth, u]:
                    if v != 0xFFFFFFFF and int(v) not in seen:
                        seen.add(int(v)); stack.append(int(v))
            assert len(seen) >= 0.99 * (r - l + 1)
            m = (l + r) // 2
            nxt += [(l, m, 2 * h + 1), (m + 1, r, 2 * h + 2)]
        frontier = nxt
    ids, dist, count, status, stats = _gpu_search(gix, w.queries, w.l, w.r, None, 10, 64, dev)
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    found, truth = [], []
    for i in range(len(w.queries)):
        found.append(inv[ids[i, :count[i]]])
        truth.append(O.bruteforce(X, w.queries[i], int(w.l[i]), int(w.r[i]), 10, w.metric)[0])
    assert O.recall_at_k(found, truth) >= 0.95


@pytest.mark.parametrize("width", [2, 4])
def test_search_width_keeps_recall(dev, tiny_oracle_index, width):
    """Expanding several candidates per iteration changes the visit order
    only: results stay valid and recall does not fall below Algorithm 1's by
    more than 0.5 points at the same ef."""
    w, idx = tiny_oracle_index
    gix = _import(idx, w)
    ids, dist, count, status, stats = _gpu_search(gix, w.queries, w.l, w.r, None, 10, 16, dev,
                                                  width=width)
    inv = np.empty(idx.n, np.int64)
    inv[idx.perm] = np.arange(idx.n)
    found, base, truth = [], [], []
    for i in range(len(w.queries)):
        l, r = int(w.l[i]), int(w.r[i])
        got = inv[ids[i, :count[i]]]
        assert np.all((got >= l) & (got <= r)) and len(set(got.tolist())) == len(got)
        assert count[i] == min(10, r - l + 1)
        found.append(got)
        base.append(O.search(idx, w.queries[i], l, r, 10, 16)[0])
        truth.append(O.bruteforce(idx.X, w.queries[i], l, r, 10, w.metric)[0])
    assert O.recall_at_k(found, truth) >= O.recall_at_k(base, truth) - 0.005


@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("d,k", [(64, 1), (64, 10), (64, 16), (96, 10), (128, 32), (192, 10), (320, 10), (768, 10)])
def test_bruteforce_tensor_core_vs_oracle(dev, metric, d, k, monkeypatch):
    """Shapes that take the tcgen05 path: query tile resident (d <= 192) or
    streamed with the point chunks (d = 320, 768), d padded to a multiple
    of 64, lists of k + 12: split BF16 MMAs, certified FP32 re-rank,
    escalation and SIMT redo of uncertified queries."""
    w = synthetic.small_mixture(5000, d, 300, n_comp=16, seed=17 + d + k, metric=metric,
                                normalise=(metric == "ip"))
    X, Q = w.base, w.queries
    l, r = w.l.copy(), w.r.copy()
    l[:5] = [0, 9, 0, 4990, 100]
    r[:5] = [4999, 9, 3, 4999, 99]       # full, single point, tiny, tail, invalid
    monkeypatch.delenv("ESG_BF_SIMT", raising=False)
    ids, dist, count = E.esg_bruteforce_filtered_knn(_t(X, dev), _t(Q, dev), _t(l, dev, torch.int64),
                                                     _t(r, dev, torch.int64), k, metric)
    torch.cuda.synchronize()
    ids, dist, count = ids.cpu().numpy(), dist.cpu().numpy(), count.cpu().numpy()
    _check_bruteforce(X, Q, l, r, k, metric, ids, dist, count)
    # the SIMT kernel agrees
    monkeypatch.setenv("ESG_BF_SIMT", "1")
    ids2, dist2, count2 = E.esg_bruteforce_filtered_knn(_t(X, dev), _t(Q, dev), _t(l, dev, torch.int64),
                                                        _t(r, dev, torch.int64), k, metric)
    torch.cuda.synchronize()
    assert np.array_equal(count, count2.cpu().numpy())
    fin = np.isfinite(dist)
    assert np.allclose(dist[fin], dist2.cpu().numpy()[fin], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("hash_slots", [1024, 16384])
def test_visited_tables_under_pressure(dev, tiny_oracle_index, hash_slots):
    """ef 800 with the smallest shared visited table (1,024 slots, 768 before
    it counts as full) sends much of a search's visits (about 2,000 per query)
    to the global table, and rows that repeat a neighbour
    id test the de-duplication of both tables (within a lane pair and across
    lanes). On that graph the GPU's Algorithm 1 matches the oracle's, returns
    no id twice, and returns the same results whatever the table size."""
    import dataclasses
    w, idx = tiny_oracle_index
    adj = idx.adj.copy()
    none = np.uint32(0xFFFFFFFF)
    both = (adj[..., 0] != none) & (adj[..., 1] != none)
    adj[..., 1] = np.where(both, adj[..., 0], adj[..., 1])          # lanes 0 and 1 of one pass
    far = (adj[..., 0] != none) & (adj[..., -1] != none)
    adj[..., -1] = np.where(far, adj[..., 0], adj[..., -1])         # v0 of lane 0, v1 of the last lane
    didx = dataclasses.replace(idx, adj=adj)
    gix = E.esg_index_import(w.base[idx.perm], idx.perm, idx.metric, idx.leaf_size, adj, idx.entries)
    k, ef = 10, 800
    ids, dist, count, status, stats = _gpu_search(gix, w.queries, w.l, w.r, None, k, ef, dev,
                                                  params=E.search_params(ef=ef, hash_slots=hash_slots))
    ref = _gpu_search(gix, w.queries, w.l, w.r, None, k, ef, dev,
                      params=E.search_params(ef=ef, hash_slots=16384))
    assert np.array_equal(ids, ref[0]) and np.array_equal(count, ref[2])
    inv = np.empty(idx.n, np.int64)
    inv[idx.perm] = np.arange(idx.n)
    found_gpu, found_cpu, truth = [], [], []
    same = 0
    for i in range(len(w.queries)):
        l, r = int(w.l[i]), int(w.r[i])
        ranks = inv[ids[i, :count[i]]]
        assert np.all((ranks >= l) & (ranks <= r)) and len(set(ranks.tolist())) == len(ranks)
        cpu, _ = O.search(didx, w.queries[i], l, r, k, ef)
        gt, _ = O.bruteforce(idx.X, w.queries[i], l, r, k, w.metric)
        found_gpu.append(ranks); found_cpu.append(cpu); truth.append(gt)
        same += ranks.tolist() == cpu.tolist()
    rg, rc = O.recall_at_k(found_gpu, truth), O.recall_at_k(found_cpu, truth)
    print(f"hash_slots {hash_slots}: recall GPU {rg:.4f} oracle {rc:.4f}, identical {same}/{len(w.queries)}, "
          f"evaluations per query {stats[:, 1].mean():.0f}")
    assert stats[:, 1].mean() > 2 * 768                     # the shared table overflowed
    assert abs(rg - rc) <= 0.005, (rg, rc)
    assert same >= 0.95 * len(w.queries)
