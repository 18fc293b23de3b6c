"""Learned search budget: the MLP's GPU kernels against the float64 oracle,
the query features against their definition, and the trained predictor
against the plain fixed-ef search it learns from."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as OM
import synthetic

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2504_04018_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rand_problem(seed, B=300):
    rng = np.random.default_rng(seed)
    F = E.esg_mlp_num_features()
    p = (rng.standard_normal(OM.n_params(F)) * 0.2).astype(np.float32)
    X = (rng.standard_normal((B, F)) * 2 + 0.5).astype(np.float32)
    T = rng.standard_normal((B, 2)).astype(np.float32)
    mu = X.mean(0).astype(np.float32)
    sigma = (X.std(0) + 0.3).astype(np.float32)
    return p, X, T, mu, sigma


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def test_param_count():
    assert E.esg_mlp_num_features() == 9
    assert E.esg_mlp_num_params() == OM.n_params(9)


def test_mlp_forward_matches_oracle():
    p, X, T, mu, sigma = _rand_problem(1)
    y = E.esg_mlp_forward(_t(p), _t(X), _t(mu), _t(sigma)).cpu().numpy()
    ref, _ = OM.forward(p, X, mu, sigma)
    assert np.allclose(y, ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("q", [0.5, 0.9])
def test_mlp_gradient_matches_oracle(q):
    p, X, T, mu, sigma = _rand_problem(2)
    loss, g = E.esg_mlp_loss_grad(_t(p), _t(X), _t(T), _t(mu), _t(sigma), q)
    g = g.cpu().numpy()
    ref_loss, ref_g = OM.loss_and_grad(p, X, T, mu, sigma, q)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * np.max(np.abs(ref_g)) + 1e-8


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(3)
    n = OM.n_params(E.esg_mlp_num_features())
    p = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    m = (rng.standard_normal(n) * 0.01).astype(np.float32)
    v = (rng.random(n) * 0.01).astype(np.float32)
    tp, tm, tv = _t(p), _t(m), _t(v)
    E.esg_mlp_adam_step(tp, _t(g), tm, tv, 7, 3e-3)
    rp, rm, rv = OM.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                              v.astype(np.float64), 7, 3e-3)
    # float32 state on the GPU: a few units in the last place of each moment
    assert np.allclose(tm.cpu().numpy(), rm, rtol=1e-5, atol=1e-8)
    assert np.allclose(tv.cpu().numpy(), rv, rtol=1e-5, atol=1e-8)
    assert np.allclose(tp.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)


@pytest.fixture(scope="module")
def learned_setup():
    # 1,024 clusters of ~100 points and a sparse graph (M = 8): fixed beam
    # widths from 10 to 24 span recall 0.91-0.97, so the budget matters
    w = synthetic.small_mixture(100_000, 64, 5000, n_comp=1024, seed=41, M=8, leaf_size=128,
                                fracs=synthetic.log_uniform_fractions(5000, 1e-3, 1.0, 42))
    gix = E.esg_build(w.base, w.attr, M=w.M, leaf_size=w.leaf_size, n_entries=8)
    _, ent, perm = E.esg_index_export(gix)
    X = w.base[perm]
    Xd = _t(X)
    q, l, r = _t(w.queries), _t(w.l), _t(w.r)
    gi, gd, gc = E.esg_bruteforce_filtered_knn(Xd, q, l, r, 10)
    torch.cuda.synchronize()
    gi = gi.cpu().numpy()
    gt = np.where(gi >= 0, perm[np.maximum(gi, 0)], -1)
    return w, gix, X, ent, perm, q, l, r, _t(gt), gc


def test_features_match_definition(learned_setup):
    w, gix, X, ent, perm, q, l, r, gt, gc = learned_setup
    f = E.esg_query_features(gix, q[:200], l[:200], r[:200]).cpu().numpy()
    for i in range(200):
        li, ri = int(w.l[i]), int(w.r[i])
        pcs = O.decompose(gix.n, gix.leaf_size, li, ri)
        assert np.isclose(f[i, 0], np.log2(ri - li + 1), atol=1e-4)
        assert f[i, 1] == len(pcs)
        for s, p in enumerate(pcs):
            assert np.isclose(f[i, 2 + s], np.log2(p.node_r - p.node_l + 1) - np.log2(p.pr - p.pl + 1), atol=1e-4)
        assert f[i, 4] == (1.0 if pcs[0].kind == "graph" else 0.0)
        assert np.isclose(f[i, 5], np.log2(10))
        assert np.isclose(f[i, 7], np.log2(pcs[0].node_r - pcs[0].node_l + 1), atol=1e-4)
        if pcs[0].kind == "graph":
            e = ent[pcs[0].heap]
            e = e[e >= 0]
            dd = O.distances(X[e].astype(np.float64), w.queries[i], w.metric)
            assert np.isclose(f[i, 6], dd.min() / dd.mean(), rtol=1e-4)
            # first-hop top-k gap: k-th smallest minus smallest, over |mean|
            kth = np.sort(dd)[min(10, len(dd)) - 1]
            assert np.isclose(f[i, 8], (kth - dd.min()) / abs(dd.mean()), rtol=1e-3, atol=1e-5)
        else:
            assert f[i, 6] == 1.0 and f[i, 8] == 0.0


def test_trained_predictor_gains_over_fixed_ef(learned_setup):
    """Train on the first 4000 queries (the last fifth of them calibrates the
    margin), then compare on the 1000 unseen queries: the learned budget
    reaches about the target while doing fewer distance evaluations than the
    smallest fixed ef reaching the same recall."""
    w, gix, X, ent, perm, q, l, r, gt, gc = learned_setup
    ntr = 4000
    rep = E.esg_train_predictor(gix, q[:ntr], l[:ntr], r[:ntr], gt[:ntr], gc[:ntr], k_max=10,
                                target_recall=0.95, epochs=80, ef_lo=8, ef_hi=128)
    assert rep[1] >= 0.95
    qt, lt, rt = q[ntr:], l[ntr:], r[ntr:]
    gtt = gt[ntr:].cpu().numpy()
    gct = gc[ntr:].cpu().numpy()

    def run(**kw):
        ids, _, cnt, _, stats = E.esg_search_batch(gix, qt, lt, rt, None, 10, want_stats=True, **kw)
        torch.cuda.synchronize()
        ids, cnt, stats = ids.cpu().numpy(), cnt.cpu().numpy(), stats.cpu().numpy()
        hits = sum(len(set(ids[i, :cnt[i]].tolist()) & set(gtt[i, :gct[i]].tolist())) for i in range(len(cnt)))
        return hits / gct.sum(), stats[:, 1].mean()

    rec_l, ev_l = run(ef=128, use_learned=1)
    assert rec_l >= 0.94
    fixed = [(ef,) + run(ef=ef) for ef in range(10, 65, 2)]
    cheapest = next((ev for ef, rec, ev in fixed if rec >= rec_l), fixed[-1][2])
    print(f"learned: recall {rec_l:.4f}, {ev_l:.0f} evals/query; fixed ef at that recall: "
          f"{cheapest:.0f} evals/query; fixed sweep {fixed}")
    assert ev_l < cheapest


def test_predictor_survives_save_load(learned_setup, tmp_path):
    w, gix, X, ent, perm, q, l, r, gt, gc = learned_setup
    blob, lo, hi = E.esg_predictor_get(gix)
    path = str(tmp_path / "idx.esg")
    E.esg_save(gix, path)
    g2 = E.esg_load(path)
    blob2, lo2, hi2 = E.esg_predictor_get(g2)
    assert np.array_equal(blob, blob2) and (lo, hi) == (lo2, hi2)
    a = E.esg_search_batch(gix, q[:300], l[:300], r[:300], None, 10, ef=128, use_learned=1)[0]
    b = E.esg_search_batch(g2, q[:300], l[:300], r[:300], None, 10, ef=128, use_learned=1)[0]
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_low_precision_rows_survive_save_load(learned_setup, tmp_path):
    """BF16 and FP8 copies added to an index are rebuilt on load, bit for bit."""
    w, gix, X, ent, perm, q, l, r, gt, gc = learned_setup
    for t in ("bf16", "fp8"):
        E.esg_index_add_storage(gix, t)
    path = str(tmp_path / "idx_lp.esg")
    E.esg_save(gix, path)
    g2 = E.esg_load(path)
    for t in ("bf16", "fp8"):
        rows_a, scale_a = E.esg_index_export_storage(gix, t)
        rows_b, scale_b = E.esg_index_export_storage(g2, t)
        assert np.array_equal(rows_a, rows_b)
        if scale_a is not None:
            assert np.array_equal(scale_a, scale_b)
        a = E.esg_search_batch(gix, q[:300], l[:300], r[:300], None, 10, ef=32, traversal=t)[0]
        b = E.esg_search_batch(g2, q[:300], l[:300], r[:300], None, 10, ef=32, traversal=t)[0]
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_constant_predictor_equals_fixed_ef(learned_setup):
    """A network whose output is the constant (log2 32, large) sets every
    query's beam width to 32 and its expansion cap to the default one: the
    learned-budget search must then return exactly what the fixed ef = 32
    search returns (same results, same counters)."""
    w, gix, X, ent, perm, q, l, r, gt, gc = learned_setup
    saved = E.esg_predictor_get(gix)
    try:
        nparam, F = E.esg_mlp_num_params(), E.esg_mlp_num_features()
        blob = np.zeros(E.esg_mlp_blob_size(), np.float32)
        blob[nparam - 2] = 5.0          # b3[0]: log2 ef
        blob[nparam - 1] = 20.0         # b3[1]: log2 expansion budget (clamped to 16 ef + 256)
        blob[nparam + F:nparam + 2 * F] = 1.0   # feature standard deviations
        E.esg_predictor_set(gix, blob, 8, 32)
        a = E.esg_search_batch(gix, q, l, r, None, 10, ef=32, use_learned=1, want_stats=True)
        b = E.esg_search_batch(gix, q, l, r, None, 10, ef=32, want_stats=True)
        torch.cuda.synchronize()
        for x, y in zip(a[:4], b[:4]):
            assert torch.equal(x, y)
        assert torch.equal(a[4][:, :5], b[4][:, :5])
    finally:
        E.esg_predictor_set(gix, *saved)


def test_per_k_class_offsets(learned_setup):
    """Mixed k (1 and 10): one pooled margin leaves the k = 1 class, which the
    pooled recall weighs a tenth of a k = 10 query, below the target; with
    per_k_class each class of k gets its own offset and reaches about the
    target on unseen queries. Without it the offsets stay zero."""
    w, gix, X, ent, perm, q, l, r, gt, gc = learned_setup
    saved = E.esg_predictor_get(gix)
    ks = np.where(np.arange(len(w.l)) % 2 == 0, 1, 10).astype(np.int32)
    kd = _t(ks)
    ntr = 4000
    nparam, F = E.esg_mlp_num_params(), E.esg_mlp_num_features()
    gtt, gct = gt[ntr:].cpu().numpy(), gc[ntr:].cpu().numpy()

    def class_recall():
        ids, _, cnt, _, _ = E.esg_search_batch(gix, q[ntr:], l[ntr:], r[ntr:], kd[ntr:], 10, ef=128,
                                               use_learned=1)
        torch.cuda.synchronize()
        ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy()
        out = {}
        for kk in (1, 10):
            sel = np.nonzero(ks[ntr:] == kk)[0]
            hits = sum(len(set(ids[i, :cnt[i]].tolist()) & set(gtt[i, :min(kk, gct[i])].tolist())) for i in sel)
            out[kk] = hits / sum(min(kk, gct[i]) for i in sel)
        return out

    try:
        for per_class in (0, 1):
            E.esg_train_predictor(gix, q[:ntr], l[:ntr], r[:ntr], gt[:ntr], gc[:ntr], k_max=10, k=kd[:ntr],
                                  target_recall=0.95, epochs=80, ef_lo=8, ef_hi=128, per_k_class=per_class)
            blob, _, _ = E.esg_predictor_get(gix)
            offs = blob[nparam + 2 * F + 2:]
            rec = class_recall()
            print(f"per_k_class={per_class}: offsets {offs[:4]}, recall by k {rec}")
            if per_class:
                assert offs[0] != 0.0 and offs[3] != 0.0
                assert np.all(offs[[1, 2] + list(range(4, len(offs)))] == 0.0)
                assert rec[1] >= 0.93 and rec[10] >= 0.93
            else:
                assert np.all(offs == 0.0)
    finally:
        E.esg_predictor_set(gix, *saved)
