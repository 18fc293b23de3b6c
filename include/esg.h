/*
 * esg.h — C ABI of the GB300 (sm_103a) implementation of ESG, elastic graphs
 * for range-filtering approximate k-nearest-neighbour search (RFAKNN),
 * arxiv 2504.04018.
 *
 * Problem (Definitions 1 and 2): points v_0..v_{N-1} in R^d carry a numeric
 * attribute. After re-ranking (Section 1, footnote on re-ranking) the point
 * of rank i is the i-th smallest attribute, so a value range becomes an
 * inclusive rank range [l, r]. A query (q, [l, r], k) asks for the k points
 * with rank in [l, r] closest to q.
 *
 * Method (Section 4.2): a segment tree over ranks holds one proximity graph
 * per node wider than the leaf size (Algorithm 3). A query range is split
 * into at most two elastic subranges (Algorithm 4, Lemma 3): a node is used
 * when it contains the query part and the part covers at least half of it
 * (elastic factor c = 1/2, Definition 3). Each graph piece is answered by a
 * beam search (Algorithm 1) that walks out-of-range points but only admits
 * in-range points to the result queue (the POST principle, Section 2.2);
 * leaf pieces are scanned. The piece results are merged into the top k.
 * The tree may have a larger fanout f with elastic factor 1/f (the extension
 * of Section 4.2, Lemma 4: still at most two pieces). For half-bounded
 * ranges [0, r] the index may instead hold only prefix graphs (ESG-1D,
 * Section 4.1, Algorithm 2, Lemma 2: one piece). A search may also skip the
 * decomposition and answer every query by POST on the root graph (the
 * baseline of Section 3.1).
 *
 * Conventions for every call:
 *  - ranks and ranges are 0-based and inclusive (the paper counts from 1);
 *  - distances: ESG_L2SQ = sum_j (q_j - x_j)^2; ESG_IP = -sum_j q_j x_j;
 *  - results are ordered by (distance, rank); unused result slots hold id -1
 *    and distance +inf;
 *  - "device" pointers are CUDA global memory of the current device, "host"
 *    pointers are ordinary CPU memory; the caller owns every buffer it passes
 *    and the library never frees caller memory;
 *  - asynchronous calls enqueue work on the given stream and return; their
 *    outputs are valid once the stream reaches that point;
 *  - no C++ exception crosses this interface; every call returns an
 *    esg_status and esg_last_error() describes the last failure on the
 *    calling thread.
 */
#ifndef ESG_H
#define ESG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *esg_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    ESG_OK = 0,
    ESG_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter */
    ESG_ERR_OOM = 2,         /* device or host allocation failed */
    ESG_ERR_CUDA = 3,        /* a CUDA runtime call failed (see esg_last_error) */
    ESG_ERR_IO = 4,          /* file could not be read or written */
    ESG_ERR_CORRUPT = 5,     /* file content is not a valid index */
    ESG_ERR_TIMEOUT = 6,     /* a bounded device wait ran out */
    ESG_ERR_UNSUPPORTED = 7  /* valid request this build does not implement */
} esg_status;

typedef enum { ESG_L2SQ = 0, ESG_IP = 1 } esg_metric;

/* Storage type of the vectors used during graph traversal. */
typedef enum { ESG_F32 = 0, ESG_BF16 = 1, ESG_FP8E4M3 = 2 } esg_dtype;

/* Per-query status codes written by esg_search_batch. */
enum {
    ESG_Q_OK = 0,
    ESG_Q_INVALID = 1,   /* l > r, r >= N, l < 0, k < 1 or k > k_max, or l > 0 on a
                            prefix-layout index without post_root: count = 0 */
    ESG_Q_TRUNCATED = 2, /* a beam search hit its expansion cap; results are partial */
    ESG_Q_OVERFLOW = 4   /* the candidate list or visited set overflowed (results valid) */
};

/* Piece kinds of the elastic decomposition. */
enum { ESG_PIECE_NONE = 0, ESG_PIECE_GRAPH = 1, ESG_PIECE_SCAN = 2 };

/*
 * Index layouts.
 *  ESG_LAYOUT_TREE    the segment tree of Algorithm 3 (ESG-2D) with fanout f:
 *                     the children of node [l, r] are [b_j, b_{j+1} - 1],
 *                     b_j = l + ceil(j (r - l + 1) / f), j = 0..f-1 (empty ones
 *                     skipped; f = 2 gives [l, mid], [mid + 1, r]); graph
 *                     levels are the depths that hold a graph node; heap
 *                     numbers: root 0, children of h are f h + 1 + j.
 *  ESG_LAYOUT_PREFIX  the half-bounded index of Algorithm 2 (ESG-1D) with
 *                     base B: graphs over the prefixes [0, n_i - 1],
 *                     n_i = floor(n / B^i), for every i with n_i >= 1; level
 *                     and node number i. Answers ranges [0, r] only (a
 *                     range [l, n - 1] is a prefix of the reversed order:
 *                     build on negated attributes).
 */
typedef enum { ESG_LAYOUT_TREE = 0, ESG_LAYOUT_PREFIX = 1 } esg_layout;

/*
 * One subrange chosen by the decomposition: the graph node [node_l, node_r]
 * (node number `heap`, graph level `depth`, both as in esg_layout) answers
 * the query part [pl, pr]. kind is ESG_PIECE_GRAPH (beam search on the
 * node's graph) or ESG_PIECE_SCAN (linear scan of a leaf).
 */
typedef struct {
    int64_t node_l, node_r, pl, pr;
    int32_t heap, depth, kind, reserved;
} esg_piece;

typedef struct esg_index esg_index; /* opaque; owned by the library */

/*
 * Index build parameters. Defaults: esg_build_params_default().
 *  M                graph degree parameter: an inserted point links to at most
 *                   M neighbours chosen by edge occlusion and a row holds at
 *                   most R = 2M neighbours (Section 5.1 uses M = 16);
 *  leaf_size        l: a tree node with r - l < leaf_size holds no graph and
 *                   is answered by a scan (Algorithms 3 and 4, first test);
 *  n_entries        query entry points per graph node (ranks evenly spaced
 *                   over the node), 1..32;
 *  ef_construction  beam width of the insertion searches (Section 5.1: 200);
 *  batch_div        points inserted concurrently per node and round are at
 *                   most 1/batch_div of the points already in its graph;
 *  fanout           tree fanout f, 2..16 (elastic factor 1/f); for the prefix
 *                   layout the base B, 2..16; 0 = 2;
 *  storage          traversal precision kept on the device besides FP32;
 *  layout           ESG_LAYOUT_TREE (default) or ESG_LAYOUT_PREFIX (the
 *                   leaf size is not used: every prefix has a graph).
 */
typedef struct {
    int32_t M;
    int32_t leaf_size;
    int32_t n_entries;
    int32_t ef_construction;
    int32_t batch_div;
    int32_t fanout;
    esg_metric metric;
    esg_dtype storage;
    esg_layout layout;
    int32_t reserved;
} esg_build_params;

/*
 * Search parameters. Defaults: esg_search_params_default().
 *  ef              beam width m of Algorithm 1 (>= k; raised to k if lower);
 *  max_expansions  cap on expansions per graph piece (0 = 16 * ef + 256);
 *                  reaching it sets ESG_Q_TRUNCATED;
 *  rerank          with BF16/FP8 storage: recompute FP32 distances of the
 *                  final candidates and re-sort (1) or not (0);
 *  use_learned     1 = per-query beam width from the trained predictor
 *                  (falls back to ef when no predictor is trained);
 *  traversal       row type used for traversal distances: ESG_F32, or
 *                  ESG_BF16 / ESG_FP8E4M3 when the index holds that copy
 *                  (FP32 accumulation in every case);
 *  width           candidates expanded per iteration, 1..4. 1 (or 0) is
 *                  Algorithm 1's order (one best candidate at a time); larger
 *                  values expand the `width` best unexpanded candidates
 *                  together (more memory parallelism, slightly different
 *                  visit order);
 *  warps_per_block, hash_slots, lanes_per_row
 *                  launch shape knobs that do not change results: warps per
 *                  CTA (1, 2 or 4), shared visited-table slots of a search
 *                  whose candidate list is the smallest, 256 items (power of
 *                  two, 1024..16384; a search with a wider beam has two fewer
 *                  per list item above 256, at least 1,024) and lanes that
 *                  share one row gather (1..32, a power of two dividing the
 *                  row's 16-byte vectors); 0 = automatic (2,048 slots).
 *                  esg_autotune picks them;
 *  post_root       0 = the elastic decomposition of the index's layout;
 *                  1 = every query is one piece: POST on the root graph alone
 *                  (a scan when the root is a leaf), the baseline the elastic
 *                  graphs improve on (Section 3.1);
 *  max_registers   registers per thread of the search kernel build: 128, or
 *                  96 (five 128-thread blocks per SM: more resident searches;
 *                  built for BF16 rows of 3 or 6 and FP8 rows of 1 or 3
 *                  16-byte vectors per lane, ESG_ERR_UNSUPPORTED otherwise);
 *                  0 = the 96-register build where it exists and shared
 *                  memory lets more searches reside with it. Does not change
 *                  results; esg_autotune picks it.
 */
typedef struct {
    int32_t ef;
    int32_t max_expansions;
    int32_t rerank;
    int32_t use_learned;
    esg_dtype traversal;
    int32_t width;
    int32_t warps_per_block;
    int32_t hash_slots;
    int32_t lanes_per_row;
    int32_t post_root;
    int32_t max_registers;
} esg_search_params;

esg_build_params esg_build_params_default(void);
esg_search_params esg_search_params_default(void);

/*
 * Build an ESG index (Algorithm 3's segment tree of graphs) on the current
 * CUDA device.
 *  vectors  host, [n, d] row-major float32, original order;
 *  attr     host, [n] float64 attribute values, or NULL (attribute = row);
 *           ranks sort by attribute with ties broken by row;
 *  n >= 1, 1 <= d <= 1024 with d % 8 == 0;
 *  out      receives the new index; free it with esg_free.
 * Synchronous: returns when the index is ready. The device copy of the
 * vectors is FP32 (plus BF16 or FP8 if params->storage asks).
 */
esg_status esg_build(const float *vectors, int64_t n, int32_t d, const double *attr,
                     const esg_build_params *params, esg_index **out);

/*
 * Create an index from graphs built elsewhere (for example by a CPU
 * reference build), in the layout the library stores:
 *  vectors  host [n, d] float32 in RANK order (row i = rank i);
 *  perm     host [n] int64: original id of rank i (NULL = identity);
 *  layout, fanout  as in esg_build_params (fanout 2..16);
 *  adj      host uint32 rows of R neighbour ranks, 0xFFFFFFFF padded, R <= 128:
 *           tree: [L, n, R], row i of depth t lists the neighbours of point i
 *           in the graph of the depth-t node containing i; prefix: the
 *           levels' rows one after the other (level i holds ranks
 *           0..n_i - 1), [n_0 + ... + n_{L-1}, R];
 *  entries  host [nodes, n_entries] int32 entry ranks per graph node, -1
 *           padded, n_entries <= 32; nodes = (f^L - 1) / (f - 1) for the
 *           tree, L for the prefix layout.
 * L must equal the number of graph levels of (n, leaf_size, layout, fanout).
 */
esg_status esg_index_import(const float *vectors, const int64_t *perm, int64_t n, int32_t d,
                            esg_metric metric, int32_t leaf_size, esg_layout layout, int32_t fanout,
                            const uint32_t *adj, int32_t L, int32_t R, const int32_t *entries,
                            int32_t n_entries, esg_dtype storage, esg_index **out);

/* Shape of an index: any output pointer may be NULL. */
esg_status esg_index_info(const esg_index *index, int64_t *n, int32_t *d, int32_t *L,
                          int32_t *R, int32_t *n_entries, int32_t *leaf_size,
                          int32_t *metric, int32_t *storage);

/* Layout of an index: layout, fanout (or base), graph nodes (rows of the
 * entries array) and adjacency rows (rows of the adj array, for all levels);
 * any output pointer may be NULL. */
esg_status esg_index_layout(const esg_index *index, int32_t *layout, int32_t *fanout,
                            int64_t *nodes, int64_t *adj_rows);

/*
 * Copy the index's graphs to host buffers of the esg_index_import layout:
 * adj [adj_rows, R] uint32, entries [nodes, n_entries] int32 (see
 * esg_index_layout), perm [n] int64. Any pointer may be NULL to skip it.
 * Synchronous.
 */
esg_status esg_index_export(const esg_index *index, uint32_t *adj, int32_t *entries,
                            int64_t *perm);

/*
 * Copy the rows of ranks row0 .. row0 + nrows - 1 of graph level `level` (a
 * depth of the tree, or prefix graph `level`) to a host buffer
 * adj [nrows, R] uint32, in the esg_index_export layout: for one node
 * [node_l, node_r] of that level, ranks node_l..node_r are the node's whole
 * graph (its edges never leave the node). Lets a caller read one node of a
 * large index without copying every level. Synchronous.
 */
esg_status esg_index_export_rows(const esg_index *index, int32_t level, int64_t row0, int64_t nrows,
                                 uint32_t *adj);

/*
 * Copy the index's low-precision traversal rows of type `dtype` to host
 * buffers (rank order): ESG_BF16: rows = [n, d] uint16 bit patterns;
 * ESG_FP8E4M3: rows = [n, d] uint8 E4M3 codes and scale = [n] float32 per-row
 * scales (x ~= scale * code). ESG_ERR_INVALID_ARG when the index holds no such
 * copy. Synchronous.
 */
esg_status esg_index_export_storage(const esg_index *index, esg_dtype dtype, void *rows,
                                    float *scale);

/*
 * Add a low-precision copy of the rows (ESG_BF16 or ESG_FP8E4M3) to an index
 * so that searches can traverse with it; a copy that exists is kept.
 * Synchronous.
 */
esg_status esg_index_add_storage(esg_index *index, esg_dtype dtype);

void esg_free(esg_index *index);

/*
 * Decomposition of nq query ranges into the pieces a search answers them by,
 * for an index of n points with the given leaf size, layout and fanout:
 *  tree    Algorithm 4's choice of elastic subranges, a node accepted when it
 *          holds the query part and f |part| >= |node| (at most two pieces:
 *          Lemma 3 for f = 2, Lemma 4 for fanout f);
 *  prefix  the prefix graph n_i = floor(n / B^i) with the largest i such that
 *          n_i >= r + 1 (Lemma 2 with base B: contains [0, r], more than 1/B
 *          of it in range); only ranges with l = 0 are valid;
 *  post_root = 1: one piece on the root graph (any valid range).
 *  l, r         device [nq] int64 inclusive rank ranges;
 *  out_pieces   device [nq, 2] esg_piece (unused slot: kind ESG_PIECE_NONE);
 *  out_npieces  device [nq] int32: number of pieces, 0 for an invalid range.
 * Asynchronous on `stream`. Integer-only and exact.
 */
esg_status esg_decompose_batch(int64_t n, int32_t leaf_size, esg_layout layout, int32_t fanout,
                               int32_t post_root, const int64_t *l, const int64_t *r, int64_t nq,
                               esg_piece *out_pieces, int32_t *out_npieces, esg_stream_t stream);

/*
 * Range-filtered approximate k-NN search (Algorithm 4 with Algorithm 1 +
 * POST on each graph piece, exact scan of leaf pieces, merge).
 *  nq          0 .. 2^30 - 1 queries (this bound holds for every batched
 *              search entry point: esg_search_batch_noalloc, max_nq of
 *              esg_batch_create, esg_autotune, esg_train_predictor);
 *  queries     device [nq, d] float32;
 *  l, r        device [nq] int64 inclusive rank ranges;
 *  k           device [nq] int32 per-query k (1..k_max), or NULL for k_max;
 *  k_max       1..1024, row stride of the outputs;
 *  out_ids     device [nq, k_max] int64: original ids (via the re-ranking);
 *  out_dist    device [nq, k_max] float32 distances;
 *  out_count   device [nq] int32: results written, min(k, r - l + 1) when the
 *              graphs reach enough in-range points;
 *  out_status  device [nq] int32 (ESG_Q_* bits) or NULL;
 *  out_stats   device [nq, 6] int64 (expansions, distance evaluations on
 *              traversal rows, out-of-range evaluations, FP32 re-rank rows,
 *              pieces, device latency in ns from the first of the query's
 *              pieces being taken by a warp to the last one finished,
 *              read from %globaltimer; queries run longest estimated
 *              search first, a query's two pieces one after the other)
 *              or NULL.
 * Asynchronous on `stream`; temporary device memory is taken from and
 * returned to the stream-ordered allocator of that stream.
 */
esg_status esg_search_batch(const esg_index *index, const float *queries, int64_t nq,
                            const int64_t *l, const int64_t *r, const int32_t *k, int32_t k_max,
                            const esg_search_params *params, int64_t *out_ids, float *out_dist,
                            int32_t *out_count, int32_t *out_status, int64_t *out_stats,
                            esg_stream_t stream);

/*
 * esg_search_batch without any device allocation (no counterpart in the
 * paper; a deployment aid). For callers that cannot call cudaMalloc or
 * cudaMallocAsync while searching: processes whose GPU memory is owned by
 * another allocator (a framework's caching pool or a fixed budget), and code
 * that must not allocate on a latency-critical path. Same arguments, results
 * and asynchrony as esg_search_batch; the scratch memory comes from one fixed
 * 64 MiB array in device global memory inside this library, which every GPU
 * that loads the library holds until the process exits. Limits: a batch
 * whose scratch cannot fit in 64 MiB is rejected with ESG_ERR_INVALID_ARG
 * (scratch grows with nq * k_max; about 350 bytes per query at k_max = 10
 * plus the visited-set overflow tables, which shrink by running fewer
 * concurrent warps before a batch is refused). The parameters are checked as
 * in esg_search_batch. Each call made outside stream capture looks the
 * array's device address up on the current device (no GPU work); a call on a
 * capturing stream reuses the address found by the last call outside capture
 * on that device, so the first call on each device must come before any
 * stream capture (otherwise ESG_ERR_INVALID_ARG). All calls on a device share
 * the array: calls whose GPU work
 * overlaps in time (different streams, or concurrent host threads) race and
 * corrupt each other's results; serialise them.
 */
esg_status esg_search_batch_noalloc(const esg_index *index, const float *queries, int64_t nq,
                                    const int64_t *l, const int64_t *r, const int32_t *k,
                                    int32_t k_max, const esg_search_params *params,
                                    int64_t *out_ids, float *out_dist, int32_t *out_count,
                                    int32_t *out_status, int64_t *out_stats, esg_stream_t stream);

/*
 * Batched search replayed as one CUDA graph. A batch owns device buffers for
 * up to max_nq queries (inputs: queries [max_nq, d] f32, l, r [max_nq] int64,
 * k [max_nq] int32; outputs as in esg_search_batch, stats [max_nq, 6]) and the
 * search's scratch memory, all allocated at creation. esg_batch_run(nq)
 * replays the whole search (decomposition, item order, persistent beam-search
 * kernel over an atomic queue of (query, piece) items, merge) for the first nq entries
 * with a single cudaGraphLaunch on `stream`; the graph for a given nq is
 * captured on first use (on a private stream) and cached. The k buffer is
 * used only when use_k != 0. Runs on one batch must not overlap.
 */
typedef struct esg_batch esg_batch;
esg_status esg_batch_create(const esg_index *index, int64_t max_nq, int32_t k_max, int32_t use_k,
                            const esg_search_params *params, esg_batch **out);
esg_status esg_batch_buffers(esg_batch *batch, float **queries, int64_t **l, int64_t **r,
                             int32_t **k, int64_t **ids, float **dist, int32_t **count,
                             int32_t **status, int64_t **stats);
esg_status esg_batch_run(esg_batch *batch, int64_t nq, esg_stream_t stream);
void esg_batch_free(esg_batch *batch);

/*
 * Autotuner (library-specific; no counterpart in the paper). Given sample
 * queries with their exact answers (gt_ids device [nq, k_max] original ids,
 * -1 padded; gt_count device [nq]), it chooses the smallest beam width ef
 * (from 8..1024) and search width (1 or 2) whose recall reaches
 * target_recall (hits among each query's first min(k_i, gt_count_i) exact ids,
 * summed, over the sum of min(k_i, gt_count_i); k_i = k[i], or k_max when k
 * is NULL), then the fastest launch shape (warps per block, visited-table
 * slots, lanes per row, registers per thread) by timing with CUDA events (every shape best of
 * three, then the six fastest best of eleven). `base` supplies the other
 * fields (traversal, rerank, ...). Writes the chosen parameters to `out` and,
 * if `report` is not NULL, [recall, milliseconds per search of the sample].
 * With base->use_learned = 1 and a trained predictor, ef is kept (the
 * predictor sets ef per query); widths 1 and 2 are checked against the target
 * and the launch shape is tuned for each that reaches it.
 * Synchronous on `stream`. ESG_ERR_UNSUPPORTED if no setting reaches the target.
 */
esg_status esg_autotune(const esg_index *index, const float *queries, int64_t nq, const int64_t *l,
                        const int64_t *r, const int32_t *k, int32_t k_max, const int64_t *gt_ids,
                        const int32_t *gt_count, float target_recall, const esg_search_params *base,
                        esg_search_params *out, float *report, esg_stream_t stream);

/*
 * Learned search budget (no counterpart in the paper). A small MLP
 * (9 query features -> 64 -> 64 -> 2, ReLU) predicts for each query log2 of
 * the beam width ef and of an expansion budget; the search uses them when
 * esg_search_params.use_learned is 1 and a predictor is trained (otherwise
 * the fixed ef). Features: log2 range width, number of pieces, log2 of each
 * piece's node size over its size, whether the first piece is a graph piece,
 * log2 k, min / mean distance to the first piece's entry points, log2 of the
 * first piece's node size, and the first hop's top-k gap: (min(k, E)-th
 * smallest - smallest entry distance) / |mean entry distance|.
 *
 * esg_train_predictor: traces the plain search (fixed ef over a grid within
 * [ef_lo, ef_hi]) on training queries with exact answers (gt_ids device
 * [nq, k_max] original ids, -1 padded; gt_count device [nq]); labels each
 * query with the smallest ef whose recall (denominator min(k_i, gt_count_i),
 * as in esg_autotune) reaches per_query_recall and the
 * expansions it used; trains the MLP with a pinball loss at `quantile` using
 * the library's GPU forward/backward/Adam kernels (epochs, batch, lr, seed);
 * then calibrates a margin on the last val_fraction of the queries so their
 * pooled recall (hits over all their answers) reaches target_recall; with
 * per_k_class set, also an offset to it for every class of k
 * (floor(log2 k)) with at least 64 of those queries so that the class's own
 * recall reaches target_recall (stricter than the pooled target: the classes
 * of small k, which the pooled recall weighs least, get wider beams).
 * report (may be NULL) receives
 * [final training loss, held-out recall, ef margin (log2), held-out distance
 * evaluations per query]. Synchronous. ESG_ERR_UNSUPPORTED if no margin
 * reaches the target.
 */
typedef struct {
    float target_recall;     /* mean recall@k to reach on held-out queries (0.95) */
    float per_query_recall;  /* label threshold per training query (1.0) */
    float quantile;          /* pinball quantile (0.9) */
    float lr;                /* Adam learning rate (1e-3) */
    float val_fraction;      /* held-out share for calibration (0.2) */
    int32_t epochs;          /* (60) */
    int32_t batch;           /* (1024) */
    int32_t ef_lo, ef_hi;    /* predicted ef range (8, 128) */
    esg_dtype traversal;     /* rows the traced and predicted searches use */
    int32_t per_k_class;     /* 1: each class of k reaches target_recall on its own (0) */
    uint64_t seed;           /* initial weights and minibatch order */
} esg_train_params;

esg_train_params esg_train_params_default(void);
esg_status esg_train_predictor(esg_index *index, const float *queries, int64_t nq, const int64_t *l,
                               const int64_t *r, const int32_t *k, int32_t k_max,
                               const int64_t *gt_ids, const int32_t *gt_count,
                               const esg_train_params *params, float *report, esg_stream_t stream);

/* Trained predictor as a host blob [params, mu[F], sigma[F], margin_ef,
 * margin_expansions, offset[12]] of esg_mlp_blob_size() floats
 * (F = esg_mlp_num_features(); esg_mlp_num_params() + 2 F + 14) with its ef
 * range. A query's predicted log2 ef gets margin_ef plus offset[c], c =
 * floor(log2 k) capped at 11 (zero unless esg_train_predictor calibrated
 * them with per_k_class); its log2 expansion budget gets margin_expansions.
 * set installs one (e.g. a saved one), get reads it back. */
int32_t esg_mlp_blob_size(void);
esg_status esg_predictor_set(esg_index *index, const float *blob, int32_t ef_lo, int32_t ef_hi);
esg_status esg_predictor_get(const esg_index *index, float *blob, int32_t *ef_lo, int32_t *ef_hi);

/* The MLP's own GPU kernels, exposed for checking: parameter count and
 * feature count F; forward y [B, 2] = f(X [B, F]) with standardisation mu,
 * sigma [F]; pinball loss and its gradient [num_params] (deterministic order);
 * one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at step >= 1; and the query
 * features [nq, F]. Device pointers, asynchronous (loss, a host pointer, makes
 * loss_grad synchronous). */
int32_t esg_mlp_num_params(void);
int32_t esg_mlp_num_features(void);
esg_status esg_mlp_forward(const float *params, const float *X, const float *mu, const float *sigma,
                           int64_t B, float *Y, esg_stream_t stream);
esg_status esg_mlp_loss_grad(const float *params, const float *X, const float *T, const float *mu,
                             const float *sigma, int64_t B, float quantile, float *grad, float *loss,
                             esg_stream_t stream);
esg_status esg_mlp_adam_step(float *params, const float *grad, float *m, float *v, int32_t step,
                             float lr, esg_stream_t stream);
esg_status esg_query_features(const esg_index *index, const float *queries, int64_t nq,
                              const int64_t *l, const int64_t *r, const int32_t *k, int32_t k_max,
                              float *features, esg_stream_t stream);

/* The per-query search budget the trained predictor gives, exactly as a
 * search with use_learned = 1 and ef = ef_fixed applies it: ef_out [nq] int32
 * (the beam width of every piece of the query, at least its k) and
 * maxexp_out [nq] int32 (the expansion cap of each piece; 0 = the default
 * cap 16 ef_fixed + 256, used when the network's output is not finite).
 * Device pointers; asynchronous. ESG_ERR_INVALID_ARG without a predictor. */
esg_status esg_query_budget(const esg_index *index, const float *queries, int64_t nq, const int64_t *l,
                            const int64_t *r, const int32_t *k, int32_t k_max, int32_t ef_fixed,
                            int32_t *ef_out, int32_t *maxexp_out, esg_stream_t stream);

/*
 * Exact range-filtered k-NN by brute force (Definitions 1 and 2): for each
 * query the min(k, r - l + 1) rows of `base` with row index in [l, r] closest
 * to q, ordered by (distance, row). Distances are evaluated in float32 in
 * the direct form (sum of squared differences, or the negated dot product).
 *  base      device [n, d] float32 row-major, d % 4 == 0;
 *  queries   device [nq, d] float32;
 *  l, r      device [nq] int64 inclusive row ranges (invalid range: count 0);
 *  k         1..1024;
 *  out_ids   device [nq, k] int64 row indices, out_dist device [nq, k] float32,
 *  out_count device [nq] int32.
 * Asynchronous on `stream`.
 */
esg_status esg_bruteforce_filtered_knn(const float *base, int64_t n, int32_t d, esg_metric metric,
                                       const float *queries, int64_t nq, const int64_t *l,
                                       const int64_t *r, int32_t k, int64_t *out_ids,
                                       float *out_dist, int32_t *out_count, esg_stream_t stream);

/*
 * Host work plan of the tensor-core path of esg_bruteforce_filtered_knn
 * (library-specific, no counterpart in the paper; for inspection and tests,
 * no GPU work). The valid queries (0 <= l <= r < n) are sorted by
 * (floor(log2(r - l + 1)), l, index) and tiled by 128; within each full query
 * tile, sorted position s goes to row (s mod 4) * 32 + s / 4. Each query tile
 * lists the 128-point tiles its ranges cover (ascending); these lists, query
 * tile by query tile, form one sequence of covered tiles, cut into `ctas`
 * contiguous shares (fewer when there are fewer covered tiles) of about equal
 * estimated cost: tiles + 6.25 (2 / ceil(d / 64))^2 per (query, work item)
 * pair in which the query covers one of the item's tiles; a share is split
 * into work items at query-tile boundaries.
 *  n, d       points and dimension of the search (d sets the cost weight);
 *  l, r       host [nq] int64 inclusive ranges;
 *  ctas       CTAs to plan for (the kernel uses one per SM);
 *  sizes      host [4] out: valid queries V, covered tiles T, work items I, CTAs G;
 *  order      host [V] out or NULL: query index at sorted-and-interleaved position;
 *  tiles      host [T] out or NULL: the covered point tiles;
 *  items      host [I, 4] out or NULL: (query tile, first position in tiles,
 *             count, 0), in sequence order;
 *  cta_first  host [G + 1] out or NULL: CTA c runs items [cta_first[c], cta_first[c + 1]).
 * Call with NULL arrays to learn the sizes. ESG_ERR_UNSUPPORTED past 2^31
 * covered tiles.
 */
esg_status esg_bruteforce_plan(int64_t n, int32_t d, const int64_t *l, const int64_t *r, int64_t nq,
                               int32_t ctas, int64_t *sizes, int32_t *order, int32_t *tiles,
                               int32_t *items, int32_t *cta_first);

/*
 * Map attribute value ranges [lo, hi] to inclusive rank ranges [l, r] on the
 * host (binary search over the sorted attributes). A value range holding no
 * point yields l = r + 1. Host pointers, [nq] each.
 */
esg_status esg_attr_to_rank_range(const esg_index *index, const double *lo, const double *hi,
                                  int64_t nq, int64_t *l, int64_t *r);

/* Save / load an index (graphs, vectors, permutation, parameters, the
 * learned predictor) with a versioned header and per-section CRC32. The
 * FP32 rows are stored; the BF16 / FP8 copies the index held are rebuilt on
 * load (quantisation is deterministic). Host path; ESG_ERR_IO when the file
 * cannot be opened or written, ESG_ERR_CORRUPT when the header, a size or a
 * CRC does not match (including files of another format version). */
esg_status esg_save(const esg_index *index, const char *path);
esg_status esg_load(const char *path, esg_index **out);

/*
 * Benchmark timing (library-specific; no counterpart in the paper). While
 * enabled, every esg_search_batch records a CUDA event pair around its beam
 * search kernel on the call's stream and counts the kernels it launches;
 * esg_bruteforce_filtered_knn does the same around its tensor-core kernel.
 * esg_profile_read waits for the recorded events and returns the summed
 * kernel milliseconds, the number of kernels launched and the number of
 * timed kernel launches since the last reset (reset != 0 clears them).
 * Enabling resets the counters. Host pointers; any may be NULL.
 */
esg_status esg_profile_enable(int32_t on);
esg_status esg_profile_read(double *kernel_ms, int64_t *kernel_launches, int64_t *timed_launches,
                            int32_t reset);
/* Tensor-core work issued while profiling was enabled: the FLOPs of the
 * BF16 MMAs the pipelined brute-force kernel issued (three per 128 x 128 x 64
 * block, masked pairs included), for a tensor-pipe roofline. Host pointer,
 * may be NULL; reset != 0 clears the count. */
esg_status esg_profile_tensor_work(double *mma_flops, int32_t reset);

const char *esg_status_str(esg_status s);
const char *esg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ESG_H */
