"""Full-size checks on the 10M-point batching workload and the 768-d learned
workload: outputs sampled against the float64 oracle one by one, properties
that hold at any size on every query, recall against the exact GPU brute
force on a query sample."""
import numpy as np
import pytest

import oracle as O
import synthetic

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2504_04018_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def _check_properties(l, r, k, ids, dist, cnt, inv):
    """Every query: count = min(k, width), ids in range and distinct,
    distances ascending."""
    want = np.minimum(k, r - l + 1)
    assert np.array_equal(cnt, want)
    for i in range(len(cnt)):
        c = cnt[i]
        ranks = inv[ids[i, :c]]
        assert ranks.min() >= l[i] and ranks.max() <= r[i]
        assert len(np.unique(ranks)) == c
        assert np.all(np.diff(dist[i, :c]) >= 0)
        assert np.all(ids[i, c:] == -1)


def _gt(Xr_t, q, l, r, kmax, metric, perm):
    gi, gd, gc = E.esg_bruteforce_filtered_knn(Xr_t, _t(q), _t(l), _t(r), kmax, metric)
    torch.cuda.synchronize()
    gi, gd, gc = gi.cpu().numpy(), gd.cpu().numpy(), gc.cpu().numpy()
    return np.where(gi >= 0, perm[np.maximum(gi, 0)], -1), gd, gc, gi


def _recall(ids, cnt, k, gt, gc):
    hits = tot = 0
    for i in range(len(cnt)):
        c = min(int(k[i]), int(gc[i]))
        hits += len(set(ids[i, :min(int(cnt[i]), c)].tolist()) & set(gt[i, :c].tolist()))
        tot += c
    return hits / tot


def _oracle_sample(X, queries, l, r, k, metric, gi, gd, idx):
    """GPU ground truth against the float64 oracle on sampled queries (rows
    of the query's range only, so that wide ranges stay affordable)."""
    for i in idx:
        li, ri = int(l[i]), int(r[i])
        Xs = X[li:ri + 1].astype(np.float64)
        c = min(int(k[i]), ri - li + 1)
        ref, rd = O.bruteforce(Xs, queries[i].astype(np.float64), 0, ri - li, c + 1, metric)
        ref = ref + li
        tol = 4e-5 * (np.abs(rd).max() + 1e-30)
        got = gi[i, :c]
        assert set(ref[:c][rd[:c] < rd[c - 1] - tol].tolist()) <= set(got.tolist())
        exact = O.distances(X[got].astype(np.float64), queries[i].astype(np.float64), metric)
        assert np.allclose(gd[i, :c], exact, rtol=1e-5, atol=1e-6)


def npieces_all(ix, w):
    """Pieces per query from the GPU decomposition (valid ranges all)."""
    _, npieces = E.esg_decompose_batch(ix.n, ix.leaf_size, _t(w.l), _t(w.r))
    torch.cuda.synchronize()
    return npieces.cpu().numpy().astype(np.int64)


@pytest.fixture(scope="module")
def batching_index():
    w = synthetic.batching()
    ix = E.esg_build(w.base, w.attr, M=32, leaf_size=256, n_entries=16, metric="ip", storage="bf16")
    _, _, perm = E.esg_index_export(ix)
    return w, ix, perm


def test_batching_workload(batching_index):
    """10M unit-norm 96-d points, 100,000 queries with widths 0.01%-100% and
    k in {1, 10, 100} in one CUDA-graph launch, launch shape and beam width
    from the autotuner (BF16 traversal, FP32 re-rank)."""
    w, ix, perm = batching_index
    inv = np.empty(len(perm), np.int64)
    inv[perm] = np.arange(len(perm))
    # decomposition: bit-exact on a sample of 20,000 queries
    rng = np.random.default_rng(5)
    sample = rng.choice(len(w.l), 20000, replace=False)
    pieces, npieces = E.esg_decompose_batch(ix.n, ix.leaf_size, _t(w.l[sample]), _t(w.r[sample]))
    torch.cuda.synchronize()
    nl, nr, pl, pr, heap, depth, kind = [c.cpu().numpy() for c in E.unpack_pieces(pieces)]
    npieces = npieces.cpu().numpy()
    for j, i in enumerate(sample):
        want = O.decompose(ix.n, ix.leaf_size, int(w.l[i]), int(w.r[i]))
        assert npieces[j] == len(want)
        for s, p in enumerate(want):
            assert (pl[j, s], pr[j, s], heap[j, s]) == (p.pl, p.pr, p.heap)
    X = w.base[perm]
    Xr = _t(X)
    # autotune on training queries with exact answers
    tq, tl, tr = synthetic.training_queries(w, 2000, 1024, seed=4004)
    tk = np.array([1, 10, 100], np.int32)[np.random.default_rng(4005).integers(0, 3, 2000)]
    tgt, _, tgc, _ = _gt(Xr, tq, tl, tr, 100, "ip", perm)
    base = E.search_params(ef=64, traversal="bf16")
    params, trec, tms = E.esg_autotune(ix, _t(tq), _t(tl), _t(tr), _t(tgt), _t(tgc), k_max=100,
                                       k=_t(tk), target_recall=0.955, base=base)
    print(f"autotuned: ef={params.ef} width={params.width} wpb={params.warps_per_block} "
          f"hash={params.hash_slots} lpr={params.lanes_per_row}, train recall {trec:.4f}")
    # all 100,000 queries in one graph launch
    nq = len(w.l)
    b = E.Batch(ix, max_nq=nq, k_max=100, params=params, use_k=True)
    b.view("queries", (nq, ix.d), torch.float32).copy_(_t(w.queries))
    b.view("l", (nq,), torch.int64).copy_(_t(w.l))
    b.view("r", (nq,), torch.int64).copy_(_t(w.r))
    b.view("k", (nq,), torch.int32).copy_(_t(w.k))
    b.run(nq)
    torch.cuda.synchronize()
    ids = b.view("ids", (nq, 100), torch.int64).cpu().numpy()
    dist = b.view("dist", (nq, 100), torch.float32).cpu().numpy()
    cnt = b.view("count", (nq,), torch.int32).cpu().numpy()
    stats = b.view("stats", (nq, 6), torch.int64).cpu().numpy()
    lat = stats[:, 5]
    assert np.all(lat[cnt > 0] > 0) and np.all(lat < 10**10)   # ns, within the launch
    assert np.array_equal(stats[:, 4], npieces_all(ix, w))
    print(f"batching workload: per-query device latency p50 {np.percentile(lat, 50) / 1e3:.1f} us, "
          f"p99 {np.percentile(lat, 99) / 1e3:.1f} us")
    # the graph replay equals a direct call
    d_ids, _, d_cnt, _, _ = E.esg_search_batch(ix, _t(w.queries[:5000]), _t(w.l[:5000]), _t(w.r[:5000]),
                                               _t(w.k[:5000]), 100, params=params)
    torch.cuda.synchronize()
    assert np.array_equal(d_cnt.cpu().numpy(), cnt[:5000])
    assert np.array_equal(d_ids.cpu().numpy(), ids[:5000])
    _check_properties(w.l, w.r, w.k, ids, dist, cnt, inv)
    # recall on 3,000 held-out queries against the exact GPU ground truth
    ev = rng.choice(nq, 3000, replace=False)
    gt, gd, gc, gi = _gt(Xr, w.queries[ev], w.l[ev], w.r[ev], 100, "ip", perm)
    rec = _recall(ids[ev], cnt[ev], w.k[ev], gt, gc)
    print(f"batching workload: recall {rec:.4f} on 3,000 sampled queries")
    assert rec >= 0.95
    # ground truth against the float64 oracle on 12 sampled queries of width <= 2^20
    small = [j for j in range(len(ev)) if w.r[ev[j]] - w.l[ev[j]] < (1 << 20)][:12]
    _oracle_sample(X, w.queries[ev], w.l[ev], w.r[ev], w.k[ev], "ip", gi, gd, small)


def test_learned_workload():
    """1M anisotropic 768-d unit vectors (power-law spectrum), inner product,
    BF16 storage: the budget predictor is trained on the GPU on traces of
    50,000 training queries and evaluated on 10,000 held-out queries, against
    the fixed-ef search at the same recall."""
    w = synthetic.learned()
    ntr = 50_000
    ix = E.esg_build(w.base, w.attr, M=32, leaf_size=256, n_entries=16, metric="ip", storage="bf16")
    _, _, perm = E.esg_index_export(ix)
    inv = np.empty(len(perm), np.int64)
    inv[perm] = np.arange(len(perm))
    X = w.base[perm]
    Xr = _t(X)
    gt, gd, gc, gi = _gt(Xr, w.queries, w.l, w.r, 10, "ip", perm)
    tr, te = slice(0, ntr), slice(ntr, None)
    rep = E.esg_train_predictor(ix, _t(w.queries[tr]), _t(w.l[tr]), _t(w.r[tr]), _t(gt[tr]), _t(gc[tr]),
                                k_max=10, target_recall=0.955, ef_lo=8, ef_hi=128, traversal="bf16",
                                epochs=40)
    print(f"learned workload: train loss {rep[0]:.4f}, calibration recall {rep[1]:.4f}")
    q, l, r = _t(w.queries[te]), _t(w.l[te]), _t(w.r[te])
    k = np.full(len(w.l[te]), 10)

    def run(**kw):
        ids, dist, cnt, _, stats = E.esg_search_batch(ix, q, l, r, None, 10, traversal="bf16",
                                                      want_stats=True, **kw)
        torch.cuda.synchronize()
        ids, dist, cnt, stats = ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy(), stats.cpu().numpy()
        return ids, dist, cnt, _recall(ids, cnt, k, gt[te], gc[te]), stats[:, 1].mean()

    ids, dist, cnt, rec_l, ev_l = run(ef=128, use_learned=1)
    _check_properties(w.l[te], w.r[te], k, ids, dist, cnt, inv)
    fixed = []
    for ef in (32, 48, 64, 80, 96, 128, 160):
        _, _, _, rec, ev = run(ef=ef)
        fixed.append((ef, rec, ev))
        if rec >= rec_l:
            break
    print(f"learned: recall {rec_l:.4f} at {ev_l:.0f} evals/query; fixed: {fixed}")
    assert rec_l >= 0.95
    # the cheapest fixed beam at the learned recall evaluates more rows
    cheapest = next((ev for ef, rec, ev in fixed if rec >= rec_l), None)
    assert cheapest is not None and ev_l < cheapest
    # ground truth against the float64 oracle on 8 held-out queries
    rng = np.random.default_rng(9)
    idx = rng.choice(np.arange(ntr, len(w.l)), 8, replace=False)
    _oracle_sample(X, w.queries, w.l, w.r, np.full(len(w.l), 10), "ip", gi, gd, idx)
