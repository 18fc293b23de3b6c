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
