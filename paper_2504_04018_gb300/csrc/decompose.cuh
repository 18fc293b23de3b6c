// Elastic range decomposition (Algorithm 4's choice of subranges, Lemma 3).
#pragma once
#include "esg_internal.cuh"

// Descend the segment tree over [0, n-1] for the query part [a, b].
// Algorithm 4 applied at each node, in order:
//   1. r - l < leaf_size            -> linear scan piece (leaf);
//   2. [a, b] in [l, r] and 2 |[a, b]| >= |[l, r]|  -> graph piece
//      (elastic factor >= c = 1/2, tested in integers);
//   3. otherwise split at mid = floor((l + r) / 2) and continue on the clipped
//      part of each child, left child first.
// Before the first split the query lies inside the node, and each part made
// by a split is a suffix (prefix) of its child that fails step 2 only when it
// fits inside the child's right (left) half; so the walk forks at most once
// and returns at most two pieces (Lemma 3). Returns the piece count, or -1 if
// more than two pieces would be needed (not reachable for valid input).
__host__ __device__ inline int esg_decompose_one(int64_t n, int32_t leaf_size, int64_t lq, int64_t rq,
                                                 esg_piece out[2]) {
    out[0].kind = ESG_PIECE_NONE;
    out[1].kind = ESG_PIECE_NONE;
    if (!(lq >= 0 && lq <= rq && rq <= n - 1)) return 0;
    // explicit stack of pending (node, part); at most 2 live entries
    int64_t sl[4], sr[4], sa[4], sb[4];
    int32_t sh[4], sd[4];
    int top = 0, cnt = 0;
    sl[0] = 0; sr[0] = n - 1; sa[0] = lq; sb[0] = rq; sh[0] = 0; sd[0] = 0; top = 1;
    while (top > 0) {
        --top;
        int64_t l = sl[top], r = sr[top], a = sa[top], b = sb[top];
        int32_t h = sh[top], dep = sd[top];
        int kind = ESG_PIECE_NONE;
        if (r - l < (int64_t)leaf_size) {
            kind = ESG_PIECE_SCAN;
        } else if (l <= a && b <= r && 2 * (b - a + 1) >= r - l + 1) {
            kind = ESG_PIECE_GRAPH;
        }
        if (kind != ESG_PIECE_NONE) {
            if (cnt >= 2) return -1;
            out[cnt].node_l = l; out[cnt].node_r = r; out[cnt].pl = a; out[cnt].pr = b;
            out[cnt].heap = h; out[cnt].depth = dep; out[cnt].kind = kind; out[cnt].reserved = 0;
            ++cnt;
            continue;
        }
        int64_t mid = l + (r - l) / 2;  // == floor((l + r) / 2) for l >= 0
        // push right first so that the left part is processed first
        if (b > mid) {
            if (top >= 4) return -1;
            sl[top] = mid + 1; sr[top] = r; sa[top] = a > mid + 1 ? a : mid + 1; sb[top] = b;
            sh[top] = 2 * h + 2; sd[top] = dep + 1; ++top;
        }
        if (a <= mid) {
            if (top >= 4) return -1;
            sl[top] = l; sr[top] = mid; sa[top] = a; sb[top] = b < mid ? b : mid;
            sh[top] = 2 * h + 1; sd[top] = dep + 1; ++top;
        }
    }
    return cnt;
}
