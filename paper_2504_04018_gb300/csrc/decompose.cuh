// The choice of graph pieces for a query range: Algorithm 4's elastic
// subranges on the fanout-f segment tree (Lemmas 3 and 4), the prefix graph
// of the half-bounded index (Lemma 2), or the root graph alone (POST).
#pragma once
#include "esg_internal.cuh"

// Bounds of child j of node [l, r] in a tree of fanout f: first rank
// l + ceil(j len / f) (len = r - l + 1). Child j is [lo(j), lo(j + 1) - 1],
// empty when the node is narrower than f; f = 2 gives [l, mid], [mid + 1, r].
__host__ __device__ inline int64_t esg_child_lo(int64_t l, int64_t len, int32_t f, int64_t j) {
    return l + (j * len + f - 1) / f;
}

// Descend the fanout-f tree over [0, n-1] for the query part [a, b].
// Algorithm 4 applied at each node, in order:
//   1. r - l < leaf_size            -> linear scan piece (leaf);
//   2. [a, b] in [l, r] and f |[a, b]| >= |[l, r]|  -> graph piece
//      (elastic factor >= c = 1/f, tested in integers);
//   3. otherwise continue on the clipped part of each child it overlaps,
//      first child first. Position p of [l, r] lies in child
//      floor(f (p - l) / len).
// A part that is not accepted overlaps at most two children (three would
// cover a whole middle child, at least len / f ranks, and the node would have
// passed test 2), and each part made by a split is a suffix (prefix) of its
// child that fails test 2 only when it fits inside that child's last (first)
// child; so the walk forks at most once and returns at most two pieces
// (Lemma 3 for f = 2, Lemma 4). Returns the piece count, or -1 if more
// would be needed (not reachable for valid input).
__host__ __device__ inline int esg_decompose_tree(int64_t n, int32_t leaf_size, int32_t f, int64_t lq,
                                                  int64_t rq, esg_piece out[2]) {
    int64_t sl[4], sr[4], sa[4], sb[4];
    int32_t sh[4], sd[4];
    int top = 0, cnt = 0;
    sl[0] = 0; sr[0] = n - 1; sa[0] = lq; sb[0] = rq; sh[0] = 0; sd[0] = 0; top = 1;
    while (top > 0) {
        --top;
        const int64_t l = sl[top], r = sr[top], a = sa[top], b = sb[top];
        const int32_t h = sh[top], dep = sd[top];
        int kind = ESG_PIECE_NONE;
        if (r - l < (int64_t)leaf_size) {
            kind = ESG_PIECE_SCAN;
        } else if (l <= a && b <= r && (int64_t)f * (b - a + 1) >= r - l + 1) {
            kind = ESG_PIECE_GRAPH;
        }
        if (kind != ESG_PIECE_NONE) {
            if (cnt >= 2) return -1;
            out[cnt].node_l = l; out[cnt].node_r = r; out[cnt].pl = a; out[cnt].pr = b;
            out[cnt].heap = h; out[cnt].depth = dep; out[cnt].kind = kind; out[cnt].reserved = 0;
            ++cnt;
            continue;
        }
        const int64_t len = r - l + 1;
        const int64_t ja = (int64_t)f * (a - l) / len, jb = (int64_t)f * (b - l) / len;
        if (jb - ja > 1) return -1;
        // push the later child first so that the earlier part is processed first
        for (int64_t j = jb; j >= ja; --j) {
            if (top >= 4) return -1;
            const int64_t cl = esg_child_lo(l, len, f, j), cr = esg_child_lo(l, len, f, j + 1) - 1;
            sl[top] = cl; sr[top] = cr;
            sa[top] = a > cl ? a : cl; sb[top] = b < cr ? b : cr;
            sh[top] = f * h + 1 + (int32_t)j; sd[top] = dep + 1; ++top;
        }
    }
    return cnt;
}

// The pieces of query [lq, rq] under `s`; returns the count (0 for an
// invalid range), or -1 when the tree walk would need more than two.
//   post_root: one piece on the root [0, n-1] (a scan when the tree's root
//              is a leaf);
//   prefix:    valid only for lq = 0: the largest i with n_i = floor(n / B^i)
//              >= rq + 1, graph piece [0, n_i - 1] (level and node i), so that
//              rq + 1 <= n_i < B (rq + 1) (Lemma 2 with base B);
//   tree:      esg_decompose_tree.
__host__ __device__ inline int esg_decompose_one(const DecomposeSpec &s, int64_t lq, int64_t rq,
                                                 esg_piece out[2]) {
    out[0].kind = ESG_PIECE_NONE;
    out[1].kind = ESG_PIECE_NONE;
    if (!(lq >= 0 && lq <= rq && rq <= s.n - 1)) return 0;
    if (s.post_root) {
        const bool leaf = s.layout == ESG_LAYOUT_TREE && s.n - 1 < (int64_t)s.leaf;
        out[0].node_l = 0; out[0].node_r = s.n - 1; out[0].pl = lq; out[0].pr = rq;
        out[0].heap = 0; out[0].depth = 0; out[0].kind = leaf ? ESG_PIECE_SCAN : ESG_PIECE_GRAPH;
        out[0].reserved = 0;
        return 1;
    }
    if (s.layout == ESG_LAYOUT_PREFIX) {
        if (lq != 0) return 0;
        int64_t m = s.n;
        int32_t i = 0;
        while (m / s.fanout >= rq + 1) { m /= s.fanout; ++i; }
        out[0].node_l = 0; out[0].node_r = m - 1; out[0].pl = 0; out[0].pr = rq;
        out[0].heap = i; out[0].depth = i; out[0].kind = ESG_PIECE_GRAPH; out[0].reserved = 0;
        return 1;
    }
    return esg_decompose_tree(s.n, s.leaf, s.fanout, lq, rq, out);
}
