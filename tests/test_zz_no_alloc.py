"""The allocation-free search entry point (esg_search_batch_noalloc).

It exists for callers that may not allocate device memory while they search
(their GPU memory belongs to another allocator, or the call sits on a path
that must not allocate). It must return what esg_search_batch returns; its
scratch lives in one fixed device array inside the library that every call
reuses, so two calls in a row must both be right (state left behind by the
first call must not leak into the second). Collected last on purpose.
"""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2504_04018_gb300")

pytestmark = pytest.mark.gpu


def _outputs(nq, k_max, dev):
    return (torch.full((nq, k_max), -7, dtype=torch.int64, device=dev),
            torch.full((nq, k_max), -7.0, dtype=torch.float32, device=dev),
            torch.full((nq,), -7, dtype=torch.int32, device=dev),
            torch.full((nq,), -7, dtype=torch.int32, device=dev),
            torch.full((nq, 6), -7, dtype=torch.int64, device=dev))


def test_noalloc_matches_search_batch_twice():
    dev = torch.device("cuda:0")
    w = synthetic.small_mixture(12000, 64, 400, n_comp=24, seed=31, M=12, leaf_size=64)
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=8)
    q = torch.as_tensor(w.queries, device=dev)
    l = torch.as_tensor(w.l, device=dev)
    r = torch.as_tensor(w.r, device=dev)
    k = torch.as_tensor(np.array([1, 5, 10, 20] * 100, np.int32), device=dev)
    params = E.search_params(ef=32)
    ref = E.esg_search_batch(gix, q, l, r, k, 20, params=params, want_stats=True)
    torch.cuda.synchronize()
    ref = [x.cpu().numpy() for x in ref]
    for call in range(2):
        out = _outputs(len(w.queries), 20, dev)
        E.esg_search_batch_noalloc(gix, q, l, r, out, k=k, k_max=20, params=params)
        torch.cuda.synchronize()
        ids, dist, cnt, st, stats = [x.cpu().numpy() for x in out]
        assert np.array_equal(cnt, ref[2]), call
        assert np.array_equal(ids, ref[0]), call
        assert np.array_equal(np.isinf(dist), np.isinf(ref[1])), call
        fin = np.isfinite(ref[1])
        assert np.allclose(dist[fin], ref[1][fin], rtol=1e-6, atol=1e-6)
        assert np.array_equal(st, ref[3]), call
        # counters are deterministic; the last column is a measured latency
        assert np.array_equal(stats[:, :5], ref[4][:, :5]), call
        assert np.all(stats[cnt > 0, 5] > 0), call


def test_noalloc_rejects_batches_beyond_its_scratch():
    dev = torch.device("cuda:0")
    w = synthetic.small_mixture(3000, 16, 8, n_comp=4, seed=32, M=8, leaf_size=64)
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=4)
    nq, k_max = 20000, 1024                         # ~330 MB of per-query scratch
    q = torch.zeros((nq, 16), dtype=torch.float32, device=dev)
    l = torch.zeros(nq, dtype=torch.int64, device=dev)
    r = torch.full((nq,), 10, dtype=torch.int64, device=dev)
    out = _outputs(nq, k_max, dev)
    with pytest.raises(E.EsgError, match="invalid argument"):
        E.esg_search_batch_noalloc(gix, q, l, r, out, k_max=k_max)
    torch.cuda.synchronize()


def _compare(gix, q, l, r, k, k_max, params, dev, calls=2):
    ref = E.esg_search_batch(gix, q, l, r, k, k_max, params=params, want_stats=True)
    torch.cuda.synchronize()
    ref = [x.cpu().numpy() for x in ref]
    for call in range(calls):
        out = _outputs(q.shape[0], k_max, dev)
        E.esg_search_batch_noalloc(gix, q, l, r, out, k=k, k_max=k_max, params=params)
        torch.cuda.synchronize()
        ids, dist, cnt, st, stats = [x.cpu().numpy() for x in out]
        assert np.array_equal(cnt, ref[2]), call
        assert np.array_equal(ids, ref[0]), call
        fin = np.isfinite(ref[1])
        assert np.array_equal(np.isinf(dist), np.isinf(ref[1])), call
        assert np.allclose(dist[fin], ref[1][fin], rtol=1e-6, atol=1e-6)
        assert np.array_equal(st, ref[3]), call
        assert np.array_equal(stats[:, :5], ref[4][:, :5]), call


@pytest.fixture(scope="module")
def bf16_index():
    w = synthetic.small_mixture(20000, 64, 8000, n_comp=32, seed=33, M=12, leaf_size=64)
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=8, storage="bf16")
    return w, gix


def test_noalloc_large_batch_runs_on_a_shrunk_grid(bf16_index):
    """8,000 queries at k_max = 10: the per-warp overflow tables of a full
    persistent grid (every resident warp) exceed the fixed scratch, so the
    entry point halves the grid until they fit; the results must not change."""
    dev = torch.device("cuda:0")
    w, gix = bf16_index
    q, l, r = (torch.as_tensor(a, device=dev) for a in (w.queries, w.l, w.r))
    _compare(gix, q, l, r, None, 10, E.search_params(ef=48), dev)


def test_noalloc_bf16_traversal_and_learned_budget(bf16_index):
    """BF16 traversal rows with the FP32 re-rank, and the learned budget (a
    fixed network: constant log2 ef = 5), whose per-query features and
    budgets also live in the fixed scratch."""
    dev = torch.device("cuda:0")
    w, gix = bf16_index
    q, l, r = (torch.as_tensor(a[:3000], device=dev) for a in (w.queries, w.l, w.r))
    k = torch.as_tensor(np.array([1, 10, 20] * 1000, np.int32), device=dev)
    _compare(gix, q, l, r, k, 20, E.search_params(ef=32, traversal="bf16"), dev)
    nparam, F = E.esg_mlp_num_params(), E.esg_mlp_num_features()
    blob = np.zeros(E.esg_mlp_blob_size(), np.float32)
    blob[nparam - 2] = 5.0                      # b3[0]: log2 ef
    blob[nparam - 1] = 20.0                     # b3[1]: log2 expansion budget (clamped)
    blob[nparam + F:nparam + 2 * F] = 1.0       # feature standard deviations
    E.esg_predictor_set(gix, blob, 8, 64)
    _compare(gix, q, l, r, k, 20, E.search_params(ef=32, traversal="bf16", use_learned=1), dev)


def test_noalloc_checks_buffers_before_the_call(bf16_index):
    dev = torch.device("cuda:0")
    w, gix = bf16_index
    q, l, r = (torch.as_tensor(a[:100], device=dev) for a in (w.queries, w.l, w.r))
    out = list(_outputs(100, 10, dev))
    out[0] = torch.empty((100, 5), dtype=torch.int64, device=dev)          # sized for k_max 5
    with pytest.raises(E.EsgError, match="ids must have shape"):
        E.esg_search_batch_noalloc(gix, q, l, r, tuple(out), k_max=10)
    out = list(_outputs(100, 10, dev))
    out[4] = torch.empty((100, 4), dtype=torch.int64, device=dev)          # stats too narrow
    with pytest.raises(E.EsgError, match="stats must have shape"):
        E.esg_search_batch_noalloc(gix, q, l, r, tuple(out), k_max=10)
    with pytest.raises(E.EsgError, match="queries must be torch.float32"):
        E.esg_search_batch_noalloc(gix, q.double(), l, r, _outputs(100, 10, dev), k_max=10)
    bad = E.search_params(ef=32, warps_per_block=8)                        # rejected in C too
    with pytest.raises(E.EsgError, match="invalid argument"):
        E.esg_search_batch_noalloc(gix, q, l, r, _outputs(100, 10, dev), k_max=10, params=bad)
    bad = E.search_params(ef=32, hash_slots=3000)
    with pytest.raises(E.EsgError, match="invalid argument"):
        E.esg_search_batch_noalloc(gix, q, l, r, _outputs(100, 10, dev), k_max=10, params=bad)
