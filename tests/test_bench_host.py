"""Host-side pieces of the benchmark, on the CPU: the recall it reports (the
metric's definition: hits among each query's first min(k, |exact|) exact ids,
summed over queries, over the summed denominators; recall@10 over the
queries with k >= 10) and the float64 checks of its CPU leg."""
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle as O  # noqa: E402


def test_recall_hand_case():
    # query 0: k = 1, exact [5]; found [5] -> 1 of 1
    # query 1: k = 10, exact [0..9]; found 8 of them plus two others -> 8 of 10
    # query 2: k = 100, only 3 points in range (exact [7, 8, 9]); found [9, 7] -> 2 of 3
    # query 3: k = 10, exact [1, 2] (width 2); found [2, 1, 3] with count 2 -> 2 of 2
    k = np.array([1, 10, 100, 10])
    ids = np.full((4, 100), -1, np.int64)
    gt = np.full((4, 100), -1, np.int64)
    gc = np.array([1, 10, 3, 2], np.int32)
    cnt = np.array([1, 10, 2, 2], np.int32)
    ids[0, :1] = [5]; gt[0, :1] = [5]
    ids[1, :10] = [0, 1, 2, 3, 4, 5, 6, 7, 50, 51]; gt[1, :10] = np.arange(10)
    ids[2, :2] = [9, 7]; gt[2, :3] = [7, 8, 9]
    ids[3, :3] = [2, 1, 3]; gt[3, :2] = [1, 2]
    r_all, r10 = bench.recall(ids, cnt, gt, gc, k)
    assert np.isclose(r_all, (1 + 8 + 2 + 2) / (1 + 10 + 3 + 2))
    # recall@10 over k >= 10: q1 8/10, q2 2/3 (min(10, 3)), q3 2/2
    assert np.isclose(r10, (8 + 2 + 2) / (10 + 3 + 2))
    assert not bench.qualifies((r_all, r10))
    assert bench.qualifies((0.95, None)) and bench.qualifies((0.951, 0.95))
    assert not bench.qualifies((0.96, 0.949))
    # a result beyond the query's own k does not count
    ids0 = ids.copy(); cnt0 = cnt.copy()
    ids0[0, :2] = [4, 5]; cnt0[0] = 2
    assert bench.recall(ids0, cnt0, gt, gc, k)[0] < r_all


def test_cpu_leg_checks_catch_wrong_answers():
    rng = np.random.default_rng(3)
    n, d, nq, kk = 400, 16, 12, 5
    attr = rng.permutation(n).astype(np.float64)
    base = rng.standard_normal((n, d)).astype(np.float32)
    queries = rng.standard_normal((nq, d)).astype(np.float32)
    perm = np.argsort(attr, kind="stable")
    Xr = np.ascontiguousarray(base[perm])
    l = rng.integers(0, 200, nq).astype(np.int64)
    r = (l + rng.integers(10, 199, nq)).astype(np.int64)
    w = types.SimpleNamespace(n=n, l=l, r=r, k=np.full(nq, kk), queries=queries, metric="l2")
    gt = np.full((nq, kk), -1, np.int64)
    gc = np.zeros(nq, np.int32)
    dist = np.zeros((nq, kk), np.float32)
    for i in range(nq):
        ranks, dd = O.bruteforce(Xr.astype(np.float64), queries[i].astype(np.float64), int(l[i]), int(r[i]),
                                 kk, "l2")
        gt[i, :len(ranks)] = perm[ranks]          # original ids, as the GPU ground truth gives them
        gc[i] = len(ranks)
        dist[i, :len(ranks)] = dd
    sample = np.arange(nq)
    good = (gt.copy(), dist.copy(), gc.copy())
    bad_d = dist.copy(); bad_d[3, 0] *= 1.01     # one distance off by 1 %
    check, errs = bench.oracle_checks(w, Xr, perm, gt, gc, sample, {"good": good, "bad": (gt, bad_d, gc)},
                                      n_gt=nq)
    assert check["sampled"] == nq and check["identical_id_lists"] == nq
    assert check["max_rel_dist_err"] < 1e-6
    assert errs["good"] < 1e-6 and errs["bad"] > 5e-3
    # a wrong ground truth is seen as such
    gt2 = gt.copy(); gt2[0, :2] = gt2[0, 1::-1]
    check2, _ = bench.oracle_checks(w, Xr, perm, gt2, gc, sample, {}, n_gt=nq)
    assert check2["identical_id_lists"] == nq - 1
