"""Batched CUDA-graph executor, launch-shape knobs and the autotuner."""
import numpy as np
import pytest

import oracle as O
import synthetic

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2504_04018_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    w = synthetic.small_mixture(8000, 32, 300, n_comp=16, seed=13, M=12, leaf_size=64)
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=8)
    dev = torch.device("cuda:0")
    t = {"q": torch.as_tensor(w.queries, device=dev), "l": torch.as_tensor(w.l, device=dev),
         "r": torch.as_tensor(w.r, device=dev)}
    return w, gix, t


def _search(gix, t, params, k_max=10):
    out = E.esg_search_batch(gix, t["q"], t["l"], t["r"], None, k_max, params=params)
    torch.cuda.synchronize()
    return out[0].cpu().numpy(), out[1].cpu().numpy(), out[2].cpu().numpy()


def test_launch_shape_knobs_do_not_change_results(setup):
    w, gix, t = setup
    ref = _search(gix, t, E.search_params(ef=32))
    for wpb in (1, 2, 4):
        for hs in (1024, 4096, 16384):
            for lpr in (0, 1, 2, 4, 8):
                try:
                    got = _search(gix, t, E.search_params(ef=32, warps_per_block=wpb, hash_slots=hs,
                                                          lanes_per_row=lpr))
                except E.EsgError as e:       # shape that does not fit (shared memory, row split)
                    assert "unsupported" in str(e)
                    continue
                assert np.array_equal(got[0], ref[0]) and np.array_equal(got[2], ref[2])
                assert np.allclose(got[1], ref[1], rtol=1e-6, atol=1e-6)


def test_batch_graph_matches_direct_search(setup):
    w, gix, t = setup
    params = E.search_params(ef=24)
    ref_ids, ref_d, ref_c = _search(gix, t, params)
    b = E.Batch(gix, max_nq=400, k_max=10, params=params)
    nq = len(w.queries)
    for run_nq in (nq, 100, nq):                 # two graphs, one replayed
        b.view("queries", (len(w.queries), w.d), torch.float32)[:run_nq].copy_(t["q"][:run_nq])
        b.view("l", (len(w.queries),), torch.int64)[:run_nq].copy_(t["l"][:run_nq])
        b.view("r", (len(w.queries),), torch.int64)[:run_nq].copy_(t["r"][:run_nq])
        b.run(run_nq)
        torch.cuda.synchronize()
        ids = b.view("ids", (run_nq, 10), torch.int64).cpu().numpy()
        cnt = b.view("count", (run_nq,), torch.int32).cpu().numpy()
        assert np.array_equal(ids, ref_ids[:run_nq])
        assert np.array_equal(cnt, ref_c[:run_nq])
    b.close()


def test_autotune_meets_target(setup):
    w, gix, t = setup
    _, _, perm = E.esg_index_export(gix)
    X = w.base[perm].astype(np.float64)
    gt = np.full((len(w.queries), 10), -1, np.int64)
    gc = np.zeros(len(w.queries), np.int32)
    for i in range(len(w.queries)):
        ids, _ = O.bruteforce(X, w.queries[i], int(w.l[i]), int(w.r[i]), 10, w.metric)
        gt[i, :len(ids)] = perm[ids]
        gc[i] = len(ids)
    dev = torch.device("cuda:0")
    params, rec, ms = E.esg_autotune(gix, t["q"], t["l"], t["r"], torch.as_tensor(gt, device=dev),
                                     torch.as_tensor(gc, device=dev), k_max=10, target_recall=0.97)
    assert rec >= 0.97 and ms > 0
    assert 1 <= params.ef <= 1024 and params.width in (1, 2)
    ids, _, cnt = _search(gix, t, params)
    hits = sum(len(set(ids[i, :cnt[i]].tolist()) & set(gt[i, :gc[i]].tolist())) for i in range(len(gc)))
    assert hits / gc.sum() >= 0.97


def test_budget_classes_do_not_change_results(monkeypatch):
    """With a learned budget whose ef range reaches past the small class
    (ef_hi 128), the queries run in two launches sized for their classes;
    with the split switched off, in one. Results and counters are the same
    for every query whose candidate list did not overflow in either run."""
    import synthetic
    w = synthetic.small_mixture(20000, 32, 600, n_comp=16, seed=41, M=12, leaf_size=64)
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=8)
    nparam, F = E.esg_mlp_num_params(), E.esg_mlp_num_features()
    blob = np.zeros(E.esg_mlp_blob_size(), np.float32)
    # log2 ef = 2 + 0.4 log2 width: beams from about 13 to the cap
    blob[0 * 64 + 0] = 1.0                      # W1[0, 0]: hidden unit 0 reads log2 width
    blob[F * 64 + 64 + 0] = 1.0                 # W2[0, 0]: passed on by layer 2
    blob[F * 64 + 64 + 64 * 64 + 64 + 0] = 0.4  # W3[0, 0]: log2 ef = 2 + 0.4 log2 width
    blob[nparam - 2] = 2.0
    blob[nparam - 1] = 20.0
    blob[nparam:nparam + F] = 0.0
    blob[nparam + F:nparam + 2 * F] = 1.0
    E.esg_predictor_set(gix, blob, 8, 128)
    dev = torch.device("cuda:0")
    q, l, r = (torch.as_tensor(a, device=dev) for a in (w.queries, w.l, w.r))
    k = torch.as_tensor(np.array([1, 10, 100] * 200, np.int32), device=dev)
    p = E.search_params(ef=64, use_learned=1)
    outs = []
    for split in ("64", "0"):
        monkeypatch.setenv("ESG_SMALL_CLASS_EF", split)
        o = E.esg_search_batch(gix, q, l, r, k, 100, params=p, want_stats=True)
        torch.cuda.synchronize()
        outs.append([x.cpu().numpy() for x in o])
    (ia, da, ca, sa, ta), (ib, db, cb, sb, tb) = outs
    ok = ((sa & E.Q_OVERFLOW) == 0) & ((sb & E.Q_OVERFLOW) == 0)
    assert ok.sum() >= 0.9 * len(ok)
    ef_q, _ = E.esg_query_budget(gix, q, l, r, k, 100, ef_fixed=64)
    ef_q = ef_q.cpu().numpy()
    assert np.any(ef_q <= 64) and np.any(ef_q > 64)          # both classes are used
    assert np.array_equal(ia[ok], ib[ok]) and np.array_equal(ca[ok], cb[ok])
    assert np.array_equal(ta[ok, :5], tb[ok, :5])


@pytest.fixture(scope="module")
def lowp_setup():
    w = synthetic.small_mixture(12000, 96, 400, n_comp=16, seed=17, M=12, leaf_size=64)
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=8, storage="bf16")
    E.esg_index_add_storage(gix, "fp8")
    dev = torch.device("cuda:0")
    t = {"q": torch.as_tensor(w.queries, device=dev), "l": torch.as_tensor(w.l, device=dev),
         "r": torch.as_tensor(w.r, device=dev)}
    return w, gix, t


@pytest.mark.parametrize("trav", ["bf16", "fp8"])
def test_register_builds_do_not_change_results(lowp_setup, trav):
    """The 96-register builds (BF16 rows of 3 or 6 vectors per lane, FP8 rows
    of 1 or 3) return what the 128-register builds return; other splits and
    FP32 rows refuse 96 registers."""
    w, gix, t = lowp_setup
    for lpr in (0, 1, 2, 4):
        try:
            ref = _search(gix, t, E.search_params(ef=48, traversal=trav, lanes_per_row=lpr, max_registers=128))
        except E.EsgError as e:
            assert "unsupported" in str(e)
            continue
        for mr in (0, 96):
            try:
                got = _search(gix, t, E.search_params(ef=48, traversal=trav, lanes_per_row=lpr, max_registers=mr))
            except E.EsgError as e:
                assert mr == 96 and "unsupported" in str(e)
                continue
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[2], ref[2])
            assert np.array_equal(got[1], ref[1])
    with pytest.raises(E.EsgError):
        _search(gix, t, E.search_params(ef=48, max_registers=96))     # FP32 rows: no 96-register build
    with pytest.raises(E.EsgError):
        _search(gix, t, E.search_params(ef=48, max_registers=64))


def test_list_and_table_split_per_item(lowp_setup):
    """One batch mixing k = 10 and k = 300 (beam widths 48 and 300): each item
    sizes its candidate list for its own beam and gives the rest of the arena
    to its visited table, so a k = 10 query returns exactly what it returns
    in a batch of k = 10 queries alone (same list capacity, different table
    sizes), whatever the table size asked for."""
    w, gix, t = lowp_setup
    nq = len(w.queries)
    kk = np.where(np.arange(nq) % 3 == 0, 300, 10).astype(np.int32)
    kd = torch.as_tensor(kk, device="cuda:0")
    for hs in (0, 1024, 4096):
        p = E.search_params(ef=48, traversal="bf16", hash_slots=hs)
        ids, dist, cnt = E.esg_search_batch(gix, t["q"], t["l"], t["r"], kd, 300, params=p)[:3]
        torch.cuda.synchronize()
        ids, dist, cnt = ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()
        for k_only in (10, 300):
            sel = np.nonzero(kk == k_only)[0]
            st = torch.as_tensor(sel, device="cuda:0")
            a = E.esg_search_batch(gix, t["q"][st], t["l"][st], t["r"][st], None, k_only, params=p)[:3]
            torch.cuda.synchronize()
            a = [x.cpu().numpy() for x in a]
            assert np.array_equal(a[2], cnt[sel])
            assert np.array_equal(a[0], ids[sel, :k_only])
            assert np.array_equal(a[1], dist[sel, :k_only])
