"""Low-precision traversal (BF16, FP8-E4M3 with per-row scale) with FP32
re-rank, against the CPU oracle through the C ABI."""
import numpy as np
import pytest

import oracle as O
import synthetic

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2504_04018_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oracle_index():
    w = synthetic.small_mixture(6000, 96, 150, n_comp=32, seed=9, metric="ip", normalise=True,
                                M=16, ef=32, leaf_size=128)
    idx = O.build_index(w.base, w.attr, w.metric, w.leaf_size, w.M, efc=100, n_entries=16)
    return w, idx


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_storage_bits_match_oracle(oracle_index, dtype):
    w, idx = oracle_index
    Xr = w.base[idx.perm]
    gix = E.esg_index_import(Xr, idx.perm, idx.metric, idx.leaf_size, idx.adj, idx.entries,
                             storage=dtype)
    rows, scale = E.esg_index_export_storage(gix, dtype)
    if dtype == "bf16":
        assert np.array_equal(rows, O.bf16_round(Xr))
    else:
        codes, s = O.fp8_quantize_rows(Xr)
        assert np.array_equal(scale, s)
        assert np.array_equal(rows, codes)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_lowprec_search_parity(oracle_index, dtype):
    w, idx = oracle_index
    Xr = w.base[idx.perm]
    gix = E.esg_index_import(Xr, idx.perm, idx.metric, idx.leaf_size, idx.adj, idx.entries,
                             storage=dtype)
    dev = torch.device("cuda:0")
    q = torch.as_tensor(w.queries, device=dev)
    ids, dist, cnt, st, _ = E.esg_search_batch(gix, q, torch.as_tensor(w.l, device=dev),
                                               torch.as_tensor(w.r, device=dev), None, 10, ef=32,
                                               traversal=dtype, rerank=1)
    torch.cuda.synchronize()
    ids, dist, cnt = ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()
    inv = np.empty(idx.n, np.int64)
    inv[idx.perm] = np.arange(idx.n)
    trav = O.traversal_rows(Xr, dtype)
    fg, fc, tr = [], [], []
    for i in range(len(w.queries)):
        l, r = int(w.l[i]), int(w.r[i])
        got = inv[ids[i, :cnt[i]]]
        assert np.all((got >= l) & (got <= r)) and len(set(got.tolist())) == len(got)
        # re-ranked distances are the exact FP32 distances of the returned ids
        ref = O.distances(idx.X[got], w.queries[i], w.metric)
        assert np.allclose(dist[i, :cnt[i]], ref, rtol=1e-5, atol=1e-5)
        cpu, _ = O.search(idx, w.queries[i], l, r, 10, 32, trav_X=trav)
        gt, _ = O.bruteforce(idx.X, w.queries[i], l, r, 10, w.metric)
        fg.append(got); fc.append(cpu); tr.append(gt)
    rg, rc = O.recall_at_k(fg, tr), O.recall_at_k(fc, tr)
    assert abs(rg - rc) <= 0.005, (dtype, rg, rc)
