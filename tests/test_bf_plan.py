"""Host work plan of the tensor-core exact search (esg_bruteforce_plan, no GPU
work): the invariants the pipelined kernel relies on, on random workloads and
edge cases, and the balance of the estimated per-CTA cost."""
import numpy as np
import pytest

import synthetic

E = pytest.importorskip("paper_2504_04018_gb300")

TM = TN = 128


def _wbits(l, r):
    w = (r - l + 1).astype(np.int64)
    return np.array([int(x).bit_length() - 1 for x in w], dtype=np.int64)


def _deinterleave(order):
    """Sorted order from the plan's order: rows of full query tiles hold
    sorted position s at row (s mod 4) * 32 + s / 4."""
    out = order.copy()
    s = np.arange(TM)
    for qt in range(len(order) // TM):
        blk = order[qt * TM:(qt + 1) * TM]
        out[qt * TM + s] = blk[(s % 4) * 32 + s // 4]
    return out


def _restart_weight(d):
    nk = -(-d // 64)
    return 6.25 * (2.0 / nk) ** 2


def _cta_costs(l, r, order, tiles, items, cta_first, d):
    """Estimated cost of each CTA's share: tiles + weight per (query, item)
    pair in which the query covers one of the item's tiles."""
    lt, rt = l[order] // TN, r[order] // TN
    wr = _restart_weight(d)
    item_cost = np.empty(len(items))
    for i, (qt, off, cnt, _) in enumerate(items):
        a, b = tiles[off], tiles[off + cnt - 1]
        q = slice(qt * TM, min(len(order), (qt + 1) * TM))
        item_cost[i] = cnt + wr * np.count_nonzero((rt[q] >= a) & (lt[q] <= b))
    return np.array([item_cost[cta_first[c]:cta_first[c + 1]].sum() for c in range(len(cta_first) - 1)])


def check_plan(n, d, l, r, ctas):
    l = np.asarray(l, np.int64)
    r = np.asarray(r, np.int64)
    order, tiles, items, cta_first = E.esg_bruteforce_plan(n, d, l, r, ctas)
    valid = np.flatnonzero((l >= 0) & (l <= r) & (r < n))
    # every valid query once, in (log2 width, l, index) order
    assert sorted(order.tolist()) == valid.tolist()
    srt = _deinterleave(order)
    wb = _wbits(l[valid], r[valid])
    key = {int(q): (int(w), int(l[q]), int(q)) for q, w in zip(valid, wb)}
    keys = [key[int(q)] for q in srt]
    assert keys == sorted(keys)
    nqt = -(-len(order) // TM)
    # the items: consecutive pieces of the covered-tile sequence, in query-tile order
    T = len(tiles)
    if T == 0:
        assert len(items) == 0 and len(cta_first) == 2 and cta_first.tolist() == [0, 0]
        return order, tiles, items, cta_first
    assert items[0, 1] == 0 and np.all(items[:, 2] >= 1)
    assert np.array_equal(items[1:, 1], items[:-1, 1] + items[:-1, 2])
    assert items[-1, 1] + items[-1, 2] == T
    assert np.all(np.diff(items[:, 0]) >= 0) and np.all(items[:, 3] == 0)
    # each query tile's tiles: the sorted union of its queries' covered tiles
    for qt in range(nqt):
        sel = items[items[:, 0] == qt]
        got = np.concatenate([tiles[o:o + c] for _, o, c, _ in sel])
        q = order[qt * TM:(qt + 1) * TM]
        want = sorted(set().union(*[range(l[i] // TN, r[i] // TN + 1) for i in q]))
        assert got.tolist() == want
    # the CTA shares: G = min(ctas, T) contiguous runs of items, each non-empty,
    # with at most one item per query tile
    G = len(cta_first) - 1
    assert G == min(ctas, T)
    assert cta_first[0] == 0 and cta_first[-1] == len(items) and np.all(np.diff(cta_first) >= 1)
    for c in range(G):
        qts = items[cta_first[c]:cta_first[c + 1], 0]
        assert len(np.unique(qts)) == len(qts)
    return order, tiles, items, cta_first


@pytest.mark.parametrize("seed,nq,ctas,d", [(0, 1000, 152, 128), (1, 1300, 37, 768), (2, 129, 152, 64),
                                            (3, 5000, 152, 96)])
def test_plan_invariants_random(seed, nq, ctas, d):
    n = 200_003
    rng = np.random.default_rng(seed)
    fr = 2.0 ** -rng.integers(0, 14, nq)
    l, r = synthetic.ranges_from_fractions(n, fr, seed + 10)
    bad = rng.random(nq) < 0.05                     # some invalid ranges
    l = np.where(bad, r + 1, l)
    check_plan(n, d, l, r, ctas)


def test_plan_edge_cases():
    n = 1000                                         # 8 point tiles, the last one partial
    # no queries, only invalid ones
    assert [len(x) for x in E.esg_bruteforce_plan(n, 128, np.zeros(0), np.zeros(0))] == [0, 0, 0, 2]
    check_plan(n, 128, [5, -1, 10], [4, 3, n], 152)
    # fewer covered tiles than CTAs: one tile per CTA
    _, tiles, _, cta_first = check_plan(n, 128, [0], [n - 1], 152)
    assert len(tiles) == 8 and len(cta_first) == 9
    # one-point ranges at both ends, a partial last query tile of 1
    l = np.array([0, n - 1] * 64 + [17])
    check_plan(n, 128, l, l, 152)
    with pytest.raises(E.EsgError):
        E.esg_bruteforce_plan(n, 128, np.array([0]), np.array([1]), 0)


def test_plan_balances_estimated_cost():
    """Widths 2^-j N (j = 0..10) over 1M points, 10,000 queries: the largest
    estimated share stays within 15 % of the mean and below the largest share
    of an equal split of the covered tiles, under the planner's cost model."""
    n, nq = 1_000_000, 10_000
    fr = 2.0 ** -(np.arange(nq) % 11).astype(np.float64)
    l, r = synthetic.ranges_from_fractions(n, fr, 77)
    for d in (128, 768):
        order, tiles, items, cta_first = check_plan(n, d, l, r, 152)
        cost = _cta_costs(l, r, order, tiles, items, cta_first, d)
        # the same sequence cut into equal tile counts
        T, G = len(tiles), len(cta_first) - 1
        qt_of = np.repeat(items[:, 0], items[:, 2])
        eq_items, eq_first = [], []
        for c in range(G):
            t0, t1 = c * T // G, (c + 1) * T // G
            eq_first.append(len(eq_items))
            t = t0
            while t < t1:
                e = t
                while e < t1 and qt_of[e] == qt_of[t]:
                    e += 1
                eq_items.append((qt_of[t], t, e - t, 0))
                t = e
        eq_first.append(len(eq_items))
        eq = _cta_costs(l, r, order, tiles, np.array(eq_items), np.array(eq_first), d)
        assert cost.max() <= 1.15 * cost.mean(), (d, cost.max() / cost.mean())
        assert cost.max() < eq.max(), (d, cost.max(), eq.max())
