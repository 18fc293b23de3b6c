/*
 * ESG CPU oracle: graph search (Algorithm 1 with the POST principle), the
 * general-range index build (Algorithm 3, any fanout) and the half-bounded
 * index build (Algorithm 2, any base), in plain single-threaded C with
 * float64 arithmetic.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct reference
 * that the GPU library is checked against. Only tests/, the package smoke
 * entry and the benchmark's CPU-baseline leg may load it. It shares no code
 * with the GPU library.
 *
 * Conventions (same as the Python half of the oracle):
 *  - points are re-ranked so that row i of X holds the point whose attribute
 *    has rank i (Section 1, footnote on re-ranking); all ids here are ranks;
 *  - distances: metric 0 = squared Euclidean sum_j (q_j - x_j)^2,
 *               metric 1 = negative inner product -sum_j q_j x_j;
 *  - every ordering is lexicographic on (distance, rank), so results are
 *    unique even when distances tie;
 *  - a graph level is stored as rows of R uint32 neighbour ranks per point,
 *    unused slots hold 0xFFFFFFFF.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NONE 0xFFFFFFFFu

/* ---------------------------------------------------------------- distance */

static double dist(const double *a, const double *b, int d, int metric) {
    double s = 0.0;
    if (metric == 0) {
        for (int j = 0; j < d; ++j) { double t = a[j] - b[j]; s += t * t; }
        return s;
    }
    for (int j = 0; j < d; ++j) s += a[j] * b[j];
    return -s;
}

/* ------------------------------------------------------------------ heaps */

typedef struct { double d; uint32_t id; } item;

/* a < b in (distance, rank) order */
static int item_less(item a, item b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

/* Binary heap; max_heap = 0 keeps the smallest item on top, 1 the largest. */
typedef struct { item *v; int n, cap, max_heap; } heap;

static int heap_above(const heap *h, item a, item b) {
    return h->max_heap ? item_less(b, a) : item_less(a, b);
}
static void heap_init(heap *h, int cap, int max_heap) {
    h->v = (item *)malloc(sizeof(item) * (size_t)(cap > 0 ? cap : 1));
    h->n = 0; h->cap = cap > 0 ? cap : 1; h->max_heap = max_heap;
}
static void heap_free(heap *h) { free(h->v); h->v = NULL; h->n = h->cap = 0; }
static void heap_push(heap *h, item x) {
    if (h->n == h->cap) { h->cap *= 2; h->v = (item *)realloc(h->v, sizeof(item) * (size_t)h->cap); }
    int i = h->n++;
    h->v[i] = x;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (!heap_above(h, h->v[i], h->v[p])) break;
        item t = h->v[p]; h->v[p] = h->v[i]; h->v[i] = t; i = p;
    }
}
static item heap_pop(heap *h) {
    item top = h->v[0];
    h->v[0] = h->v[--h->n];
    int i = 0;
    for (;;) {
        int a = 2 * i + 1, b = a + 1, m = i;
        if (a < h->n && heap_above(h, h->v[a], h->v[m])) m = a;
        if (b < h->n && heap_above(h, h->v[b], h->v[m])) m = b;
        if (m == i) break;
        item t = h->v[m]; h->v[m] = h->v[i]; h->v[i] = t; i = m;
    }
    return top;
}

static int cmp_item(const void *a, const void *b) {
    item x = *(const item *)a, y = *(const item *)b;
    return item_less(x, y) ? -1 : (item_less(y, x) ? 1 : 0);
}

/* --------------------------------------------------- Algorithm 1 (search) */

/*
 * Graph-Search (Algorithm 1) over one proximity graph, with the POST filter:
 * every reached point may enter the candidate queue P, but only points whose
 * rank lies in [pl, pr] may enter the result queue Q (size bound m = ef).
 *
 * Readings where the listing is underspecified:
 *  - the search starts from a set of entry points (one in the listing);
 *    each goes into P, and into Q when in range;
 *  - a newly reached v goes into P (and, when in range, into Q) only while
 *    |Q| < ef or v is closer than the current worst of Q; otherwise it can
 *    never be returned nor expanded before the stop test fires;
 *  - the stop test (u farther than the worst of Q) applies once |Q| = ef,
 *    so the search runs until P is empty while fewer than ef in-range
 *    points are known;
 *  - Q is trimmed back to ef after each insertion.
 * Passing pl = 0, pr = n - 1 gives the unfiltered search used by the build.
 *
 * max_exp > 0 caps the expansions (a search budget, not part of Algorithm
 * 1): when the stop test has not fired but max_exp expansions were made, the
 * search ends there and counters[2] is incremented; 0 = no cap.
 *
 * Rows: X, adj and visited hold the ranks base, base + 1, ... (rank u is
 * row u - base), so a caller may pass only one node's rows; ids in and out
 * are ranks.
 *
 * visited: caller-provided array of n bytes, all zero on entry; it is left
 * zeroed on return. Returns the number of results written (<= ef) in
 * ascending (distance, rank) order. counters[0] += expansions,
 * counters[1] += distance evaluations (counters holds 3 entries).
 */
static int graph_search(const double *X, int d, int metric, const uint32_t *adj, int R,
                        const uint32_t *entries, int n_entries, const double *q, int ef,
                        uint32_t pl, uint32_t pr, uint8_t *visited, item *out,
                        int64_t *counters, uint32_t base, int64_t max_exp) {
    heap P, Q;
    heap_init(&P, 4 * ef + 16, 0);
    heap_init(&Q, ef + 2, 1);
    int n_vis = 0, vis_cap = 1024;
    uint32_t *vis_list = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)vis_cap);
    int64_t expansions = 0, evals = 0;

    for (int e = 0; e < n_entries; ++e) {
        uint32_t ep = entries[e];
        if (ep == NONE || visited[ep - base]) continue;
        visited[ep - base] = 1;
        if (n_vis == vis_cap) { vis_cap *= 2; vis_list = (uint32_t *)realloc(vis_list, sizeof(uint32_t) * (size_t)vis_cap); }
        vis_list[n_vis++] = ep;
        item it = { dist(q, X + (size_t)(ep - base) * d, d, metric), ep };
        ++evals;
        heap_push(&P, it);
        if (ep >= pl && ep <= pr) {
            heap_push(&Q, it);
            if (Q.n > ef) heap_pop(&Q);
        }
    }
    while (P.n > 0) {
        item u = heap_pop(&P);
        if (Q.n == ef && item_less(Q.v[0], u)) break;      /* u farther than Q.top() */
        if (max_exp > 0 && expansions >= max_exp) {        /* expansion budget spent */
            if (counters) counters[2] += 1;
            break;
        }
        ++expansions;
        const uint32_t *nb = adj + (size_t)(u.id - base) * R;
        for (int j = 0; j < R; ++j) {
            uint32_t v = nb[j];
            if (v == NONE) continue;
            if (visited[v - base]) continue;
            visited[v - base] = 1;
            if (n_vis == vis_cap) { vis_cap *= 2; vis_list = (uint32_t *)realloc(vis_list, sizeof(uint32_t) * (size_t)vis_cap); }
            vis_list[n_vis++] = v;
            item it = { dist(q, X + (size_t)(v - base) * d, d, metric), v };
            ++evals;
            if (Q.n < ef || item_less(it, Q.v[0])) {
                heap_push(&P, it);                           /* P <- P u {v} */
                if (v >= pl && v <= pr) {                    /* POST: out-of-range stays out of Q */
                    heap_push(&Q, it);
                    if (Q.n > ef) heap_pop(&Q);              /* keep the best m = ef */
                }
            }
        }
    }
    int cnt = Q.n;
    for (int i = cnt - 1; i >= 0; --i) out[i] = heap_pop(&Q);
    for (int i = 0; i < n_vis; ++i) visited[vis_list[i] - base] = 0;
    free(vis_list);
    heap_free(&P); heap_free(&Q);
    if (counters) { counters[0] += expansions; counters[1] += evals; }
    return cnt;
}

/* Exported search: one graph, one query; X and adj_level hold the n rows of
 * ranks row_base .. row_base + n - 1 (a whole level with row_base = 0, or
 * one node's rows: its edges never leave it). */
int oracle_graph_search(const double *X, int64_t n, int d, int metric, const uint32_t *adj_level,
                        int R, const uint32_t *entries, int n_entries, const double *q, int ef,
                        int64_t pl, int64_t pr, uint32_t *out_ids, double *out_dist,
                        int64_t *counters, int64_t row_base, int64_t max_exp) {
    uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
    item *out = (item *)malloc(sizeof(item) * (size_t)(ef > 0 ? ef : 1));
    int cnt = graph_search(X, d, metric, adj_level, R, entries, n_entries, q, ef,
                           (uint32_t)pl, (uint32_t)pr, visited, out, counters, (uint32_t)row_base,
                           max_exp);
    for (int i = 0; i < cnt; ++i) { out_ids[i] = out[i].id; out_dist[i] = out[i].d; }
    free(out); free(visited);
    return cnt;
}

/* ----------------------------------------- neighbour selection (occlusion) */

/*
 * Edge occlusion as in HNSW's heuristic neighbour selection: scan the
 * candidates of `base` by increasing distance and keep c unless some already
 * kept s satisfies d(c, s) < d(c, base); stop at `max_keep`.
 * cand must be sorted ascending; returns the number kept (written to keep).
 */
static int select_neighbours(const double *X, int d, int metric, const item *cand, int n_cand,
                             int max_keep, uint32_t *keep) {
    int kept = 0;
    for (int i = 0; i < n_cand && kept < max_keep; ++i) {
        const double *c = X + (size_t)cand[i].id * d;
        int good = 1;
        for (int s = 0; s < kept; ++s) {
            if (dist(c, X + (size_t)keep[s] * d, d, metric) < cand[i].d) { good = 0; break; }
        }
        if (good) keep[kept++] = cand[i].id;
    }
    return kept;
}

/* ------------------------------------------------- Algorithms 2 and 3 build */

typedef struct {
    const double *X; int d, metric, leaf, M, R, efc, E, L, f;
    int64_t n;
    uint32_t *adj;           /* the rows of every level */
    const int64_t *row_off;  /* rank i of level t is row row_off[t] + i of adj */
    int32_t *entries;        /* [graph nodes][E] */
    uint8_t *visited;
    item *buf;               /* scratch, efc + R + 1 items */
} build_ctx;

static uint32_t *row(build_ctx *c, int level, int64_t i) {
    return c->adj + ((size_t)c->row_off[level] + (size_t)i) * (size_t)c->R;
}

static int degree(const uint32_t *r, int R) {
    int k = 0;
    while (k < R && r[k] != NONE) ++k;
    return k;
}

/*
 * Insert point v into the graph of the node [l, r_cur] stored at `depth`
 * (rows l..v-1 already hold the graph of the points inserted so far). The
 * neighbours are found by an unfiltered search (ef = efc) from the node's
 * first point l, selected by occlusion (at most M), and linked both ways;
 * a neighbour whose list is full (R) is re-selected by occlusion over its
 * old list plus v.
 */
static void insert_point(build_ctx *c, int depth, int64_t l, int64_t v) {
    uint32_t *rv = row(c, depth, v);
    for (int j = 0; j < c->R; ++j) rv[j] = NONE;
    if (v == l) return;                                   /* first point: no edges */
    const double *xv = c->X + (size_t)v * c->d;
    uint32_t ep = (uint32_t)l;
    item *W = c->buf;
    int nw = graph_search(c->X, c->d, c->metric, row(c, depth, 0), c->R, &ep, 1, xv, c->efc,
                          0, (uint32_t)(c->n - 1), c->visited, W, NULL, 0, 0);
    uint32_t sel[1024];
    int ns = select_neighbours(c->X, c->d, c->metric, W, nw, c->M, sel);
    for (int s = 0; s < ns; ++s) rv[s] = sel[s];
    for (int s = 0; s < ns; ++s) {
        uint32_t u = sel[s];
        uint32_t *ru = row(c, depth, u);
        int du = degree(ru, c->R);
        if (du < c->R) { ru[du] = (uint32_t)v; continue; }
        const double *xu = c->X + (size_t)u * c->d;
        item *cand = c->buf;                               /* reuse: search results no longer needed */
        for (int j = 0; j < du; ++j) { cand[j].id = ru[j]; cand[j].d = dist(xu, c->X + (size_t)ru[j] * c->d, c->d, c->metric); }
        cand[du].id = (uint32_t)v; cand[du].d = dist(xu, xv, c->d, c->metric);
        qsort(cand, (size_t)du + 1, sizeof(item), cmp_item);
        uint32_t keep[1024];
        int nk = select_neighbours(c->X, c->d, c->metric, cand, du + 1, c->R, keep);
        for (int j = 0; j < c->R; ++j) ru[j] = j < nk ? keep[j] : NONE;
    }
}

/* Query-time entry points of node [l, r]: E ranks evenly spaced over it. */
static void set_entries(build_ctx *c, int64_t h, int64_t l, int64_t r) {
    int64_t n = r - l + 1;
    int E = c->E;
    int32_t *e = c->entries + (size_t)h * (size_t)E;
    for (int i = 0; i < E; ++i) e[i] = -1;
    int cnt = (int)(n < E ? n : E);
    for (int i = 0; i < cnt; ++i) e[i] = (int32_t)(l + (int64_t)i * n / cnt);
}

/* First rank of child j of node [l, r] in a tree of fanout f:
 * l + ceil(j * len / f); child j is [child_lo(j), child_lo(j + 1) - 1], empty
 * when the node has fewer than f points. For f = 2, child 0 is [l, mid]. */
static int64_t child_lo(int64_t l, int64_t r, int f, int j) {
    int64_t len = r - l + 1;
    return l + ((int64_t)j * len + f - 1) / f;
}

/*
 * Build-2D-Index (Algorithm 3) for the node with heap number h covering
 * [l, r] at `depth`, in a tree of fanout f (children of heap node h are
 * f h + 1 + j). Returns 1 when the node got a graph, 0 for a leaf
 * (r - l < leaf: no graph). The graph of [l, r] is a copy of its first
 * child's graph (built from scratch over that child when the child is a leaf)
 * with the remaining points of [l, r] inserted in increasing rank order; the
 * child's stored graph is left untouched (memory snapshot). With f = 2 this
 * is Algorithm 3 as printed; larger f is the extension of Section 4.2.
 */
static int build_node(build_ctx *c, int64_t h, int depth, int64_t l, int64_t r) {
    if (r - l < c->leaf) return 0;
    int first = 0;
    for (int j = 0; j < c->f; ++j) {
        int64_t a = child_lo(l, r, c->f, j), b = child_lo(l, r, c->f, j + 1) - 1;
        if (a > b) continue;
        int g = build_node(c, (int64_t)c->f * h + 1 + j, depth + 1, a, b);
        if (j == 0) first = g;
    }
    int64_t b1 = child_lo(l, r, c->f, 1);
    if (first) {
        for (int64_t i = l; i < b1; ++i)
            memcpy(row(c, depth, i), row(c, depth + 1, i), sizeof(uint32_t) * (size_t)c->R);
    } else {
        for (int64_t i = l; i < b1; ++i) insert_point(c, depth, l, i);
    }
    for (int64_t i = b1; i <= r; ++i) insert_point(c, depth, l, i);
    set_entries(c, h, l, r);
    return 1;
}

static int64_t tree_nodes(int L, int f) {
    int64_t total = 0, w = 1;
    for (int t = 0; t < L; ++t) { total += w; w *= f; }
    return total;
}

/*
 * Exported build of the segment tree (ESG-2D). X: [n, d] float64, rank
 * order. adj: [L][n][R] output (NONE for rows that belong to leaves at a
 * depth). entries: [(f^L - 1) / (f - 1)][E] output (-1 where a node has no
 * graph). L must be the number of depths that contain at least one graph
 * node for this fanout. Returns 0 on success.
 */
int oracle_build(const double *X, int64_t n, int d, int metric, int leaf, int M, int efc, int E,
                 int L, uint32_t *adj, int32_t *entries, int fanout) {
    if (n <= 0 || d <= 0 || M <= 0 || efc <= 0 || E <= 0 || L < 0 || fanout < 2) return 1;
    build_ctx c;
    c.X = X; c.n = n; c.d = d; c.metric = metric; c.leaf = leaf; c.M = M; c.R = 2 * M;
    c.efc = efc; c.E = E; c.L = L; c.f = fanout; c.adj = adj; c.entries = entries;
    if (c.R > 1024 || M > 1024) return 1;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L > 0 ? L : 1));
    for (int t = 0; t < L; ++t) off[t] = (int64_t)t * n;
    c.row_off = off;
    memset(adj, 0xFF, sizeof(uint32_t) * (size_t)L * (size_t)n * (size_t)c.R);
    for (int64_t i = 0; i < tree_nodes(L, fanout) * (int64_t)E; ++i) entries[i] = -1;
    c.visited = (uint8_t *)calloc((size_t)n, 1);
    c.buf = (item *)malloc(sizeof(item) * (size_t)(efc + c.R + 2));
    if (L > 0) build_node(&c, 0, 0, 0, n - 1);
    free(c.visited); free(c.buf); free(off);
    return 0;
}

/*
 * Build-1D-Index (Algorithm 2; base B, the extension of Section 4.1): graphs
 * over the prefixes [0, n_i - 1], n_i = floor(n / B^i), for i = 0..L-1 with
 * every n_i >= 1. The points are inserted into one graph in increasing rank
 * order (Algorithm 2's loop, reading "insert v_i, i in (pre, cur]"), and the
 * graph is copied out (snapshot) each time it holds exactly n_i points.
 * Level i's rows sit at row offset n_0 + ... + n_{i-1} of adj (total rows
 * the sum of the n_i); level 0, the whole graph, is the working graph.
 * Insertion searches start from rank 0. entries: [L][E], E ranks evenly
 * spaced over each prefix. Returns 0 on success.
 */
int oracle_build_prefix(const double *X, int64_t n, int d, int metric, int B, int M, int efc, int E,
                        int L, uint32_t *adj, int32_t *entries) {
    if (n <= 0 || d <= 0 || M <= 0 || efc <= 0 || E <= 0 || L <= 0 || B < 2) return 1;
    build_ctx c;
    c.X = X; c.n = n; c.d = d; c.metric = metric; c.leaf = 0; c.M = M; c.R = 2 * M;
    c.efc = efc; c.E = E; c.L = L; c.f = B; c.adj = adj; c.entries = entries;
    if (c.R > 1024 || M > 1024) return 1;
    int64_t *size = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    int64_t total = 0, m = n;
    for (int i = 0; i < L; ++i) { size[i] = m; off[i] = total; total += m; m /= B; }
    if (size[L - 1] < 1 || m >= 1) { free(size); free(off); return 1; }   /* L must cover every n_i >= 1 */
    c.row_off = off;
    memset(adj, 0xFF, sizeof(uint32_t) * (size_t)total * (size_t)c.R);
    for (int64_t i = 0; i < (int64_t)L * E; ++i) entries[i] = -1;
    c.visited = (uint8_t *)calloc((size_t)n, 1);
    c.buf = (item *)malloc(sizeof(item) * (size_t)(efc + c.R + 2));
    int lev = L - 1;                                  /* next snapshot: the smallest prefix */
    for (int64_t v = 0; v < n; ++v) {
        insert_point(&c, 0, 0, v);
        while (lev >= 1 && v + 1 == size[lev]) {
            for (int64_t i = 0; i < size[lev]; ++i)
                memcpy(row(&c, lev, i), row(&c, 0, i), sizeof(uint32_t) * (size_t)c.R);
            --lev;
        }
    }
    for (int i = 0; i < L; ++i) set_entries(&c, i, 0, size[i] - 1);
    free(c.visited); free(c.buf); free(size); free(off);
    return 0;
}
