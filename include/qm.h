/*
 * qm.h -- C ABI of the GB300 community-quality library (libqm.so).
 *
 * Scores community partitions of an unweighted, undirected graph with the
 * metrics of Chen, Liu & Szymanski, "Parallel Toolkit for Measuring the Quality
 * of Network Community Structure" (arXiv 1507.05492):
 *   without ground truth (Sec. II-B): modularity Q (Eq. 8), modularity density
 *     Qds (Eq. 9) and the six measures of Sec. II-B.3;
 *   with ground truth (Sec. II-A): VI (Eq. 1), NMI (Eq. 2), F-measure (Eq. 3),
 *     NVD (Eq. 4), RI (Eq. 5), ARI (Eq. 6), JI (Eq. 7).
 *
 * Conventions shared by every entry point
 *   - Every function returns a qm_status.  No C++ exception crosses the ABI.
 *     On error nothing is written to the caller's output structs, and
 *     qm_last_error() returns a one-line message for the calling thread.
 *   - `where` says whether the label / CSR pointers are host memory (QM_HOST)
 *     or device memory of the current CUDA device (QM_DEVICE).  Result structs
 *     (qm_quality, qm_compare) are always host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is stream-ordered; every call that produces results synchronises that
 *     stream once before it returns, so outputs are valid on return.
 *   - Label arrays are borrowed for the duration of the call only.
 *   - A partition is an int32 label per node with every label in [0, K).  Label
 *     ids with no member are absent communities and are skipped in every sum and
 *     mean.  A label outside [0, K) makes the call return QM_EINVAL.
 *   - Counts are exact int64.  Floating-point results are FP64; every sum of
 *     per-community or per-cell terms is accumulated in 128-bit fixed point, and
 *     the Eq. (9) split penalty's inner sum over neighbouring communities
 *     (sum_j |E_ij|^2 / |c_j|) exactly in 192-bit integers with 128-bit
 *     reciprocals, so a result does not depend on thread scheduling, node order
 *     or pipeline, and is bit-identical whether a partition is scored alone,
 *     inside a batch, or on a graph loaded with QM_REORDER.
 *   - Limits: n_nodes < 2^31, n_arcs <= 2^32 - 2^20.
 *   - Calls on different streams may run concurrently from different threads;
 *     each call takes its own scratch memory from an internal pool.
 *
 * Readings taken where the paper is silent: natural log in VI; d_c = 0 for a
 * one-node community; conductance 0 when 2|E_in| + |E_out| = 0; the partition
 * value of a per-community measure is its unweighted mean over non-empty
 * communities; NMI = 1 when both entropies are 0; ARI = 1 and JI = 1 when their
 * denominators are 0; pairs of nodes are unordered; the Qds split penalty sums
 * over ordered community pairs as Eq. (9) is written.
 */
#ifndef QM_H
#define QM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QM_OK = 0,
    QM_EINVAL = 1,    /* bad argument, label out of range, malformed graph */
    QM_ENOMEM = 2,    /* device or pinned host memory exhausted */
    QM_ECUDA = 3,     /* a CUDA runtime call failed */
    QM_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    QM_EOVERFLOW = 5, /* size beyond the library limits (see above) */
    QM_EBUSY = 6      /* resource temporarily unavailable */
} qm_status;

typedef enum { QM_HOST = 0, QM_DEVICE = 1 } qm_mem;
#define QM_HOST_PTR QM_HOST     /* alternative names of the two memory kinds */
#define QM_DEVICE_PTR QM_DEVICE

/* qm_load_graph flags */
#define QM_VALIDATE 1u /* check symmetry, no self-loops, no repeated arcs, ids in range */
#define QM_REORDER 2u  /* store the graph renumbered for locality (see qm_load_graph) */

/* Label-propagation rounds of the QM_REORDER clustering. */
#define QM_REORDER_ROUNDS 6

/* batched-compare flags */
#define QM_SHARED_TRUTH 1u /* one truth labelling [n] shared by all P candidates */

typedef struct qm_graph qm_graph; /* opaque; owns a device copy of the CSR */

/*
 * qm_load_graph -- copy a symmetric CSR into a library-owned device graph.
 * The paper's graph is unweighted and undirected (Sec. II-B.1); each undirected
 * edge {u,v} must appear as the two arcs (u,v) and (v,u).
 *   row_ptr  int64[n_nodes + 1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = n_arcs
 *   col      int32[n_arcs], neighbour ids in [0, n_nodes)
 *   where    QM_HOST or QM_DEVICE for row_ptr and col
 *   flags    QM_VALIDATE runs a device check of the CSR (untimed set-up work);
 *            QM_REORDER stores the graph renumbered so that nodes of one
 *            cluster are adjacent: QM_REORDER_ROUNDS synchronous
 *            label-propagation rounds on the graph alone (each node takes the
 *            most frequent label of up to 32 evenly spaced neighbours), then
 *            the nodes are renumbered cluster by cluster.  Every call still
 *            takes labels in the caller's node order (they are gathered
 *            through the permutation on the device) and returns the same bits
 *            as without the flag; the gathers of neighbour labels then mostly
 *            hit nearby memory.  Costs one pass per round over the arcs and
 *            4 bytes per node, at load time only; above 2^24 nodes about 4.1
 *            bytes per node more hold the index arrays that bring the
 *            caller's labels into the stored order in two sequential passes
 *            instead of one random gather (see qm_debug_set_perm_buckets).
 *   out      receives the handle; free it with qm_free_graph
 * The arrays are copied: the caller may free them when the call returns.  An
 * unweighted graph with fewer than 2^32 arcs also keeps its upper rows (the
 * arcs (u, v) with v >= u, for tuning algorithm 7): 8 bytes a node and 4 bytes
 * an undirected edge more on the device.
 * Errors: QM_EINVAL (n_nodes < 1, n_arcs odd or 0, bad CSR with QM_VALIDATE),
 * QM_EOVERFLOW, QM_ENOMEM, QM_ECUDA.
 */
qm_status qm_load_graph(const int64_t *row_ptr, const int32_t *col, int64_t n_nodes,
                        int64_t n_arcs, qm_mem where, unsigned flags, void *stream,
                        qm_graph **out);

/*
 * qm_load_graph_weighted -- qm_load_graph for a weighted undirected graph:
 * weight[k] (float32, parallel to col, same memory kind) is the weight of arc
 * k; arcs (u,v) and (v,u) must carry the same weight (checked with
 * QM_VALIDATE).  Every weight must be 0 or in [2^-20, 2^20), so that it is an
 * exact fixed-point integer w * 2^43 and every weight sum is exact; the total
 * weight W must be positive.  qm_score_partition (and the sharded calls) then
 * return Q and Qds in the paper's weighted reading (the note beside Eq. 9):
 *   Q_w   = sum_c [ W_c^in / W - ((2 W_c^in + W_c^out) / (2W))^2 ]
 *   Qds_w = sum_ci [ W_ci^in / W d_ci - ((2 W_ci^in + W_ci^out) / (2W) d_ci)^2
 *                    - sum_{cj != ci} W_ci,cj / (2W) d_ci,cj ]
 * with the densities d_ci and d_ci,cj and the six measures of Sec. II-B.3
 * still counting edges (unweighted).  The batched calls, the one-kernel
 * pipeline and qm_score_partition_noalloc refuse weighted graphs (QM_EINVAL);
 * qm_label_propagation ignores the weights.  QM_REORDER is supported.
 * Costs 4 bytes per arc more on the device.
 * Errors: those of qm_load_graph, and QM_EINVAL for a weight out of range,
 * asymmetric weights or a zero total.
 */
qm_status qm_load_graph_weighted(const int64_t *row_ptr, const int32_t *col, const float *weight, int64_t n_nodes,
                                 int64_t n_arcs, qm_mem where, unsigned flags, void *stream, qm_graph **out);
qm_status qm_free_graph(qm_graph *g);

/* Sizes of a loaded graph; any output pointer may be NULL. */
qm_status qm_graph_info(const qm_graph *g, int64_t *n_nodes, int64_t *n_edges,
                        int64_t *max_degree, size_t *device_bytes);

/* Result of scoring one partition without ground truth (Sec. II-B). */
typedef struct {
    int64_t n_nodes;
    int64_t n_edges;                /* |E| */
    int64_t n_communities_nonempty;
    int64_t intra_edges_total;      /* sum_c |E_c^in| */
    int64_t cut_edges_total;        /* sum_c |E_c^out| / 2 */
    int64_t n_community_pairs;      /* unordered pairs (ci, cj) with |E_ci,cj| > 0 */
    int64_t pair_count_sq_sum;      /* sum over those pairs of |E_ci,cj|^2 */
    double modularity;              /* Q, Eq. (8) */
    double modularity_density;      /* Qds, Eq. (9) */
    double mean_intra_edges;        /* means over non-empty communities, Sec. II-B.3 */
    double mean_intra_density;
    double mean_contraction;
    double mean_inter_edges;
    double mean_expansion;
    double mean_conductance;
} qm_quality;

/* Optional per-community outputs, length K each, memory kind given by `where`
 * of the call; any pointer may be NULL.  Absent communities get zeros. */
typedef struct {
    int64_t *size;          /* |c| */
    int64_t *intra_edges;   /* |E_c^in| */
    int64_t *inter_edges;   /* |E_c^out| */
    double *intra_density;  /* d_c */
    double *contraction;    /* 2|E_c^in| / |c| */
    double *expansion;      /* |E_c^out| / |c| */
    double *conductance;    /* |E_c^out| / (2|E_c^in| + |E_c^out|) */
    double *qds_term;       /* the bracketed term of Eq. (9) for community c */
} qm_percomm;

/*
 * qm_score_partition -- Q, Qds and the six measures of one partition
 * (Eqs. 8-9, Sec. II-B.3; the per-community decomposition of Sec. III-A).
 *   labels  int32[n_nodes], labels in [0, K)
 *   K       number of label ids (>= 1)
 *   out     host struct, written on success
 *   per_comm  NULL or per-community arrays (see qm_percomm)
 * Errors: QM_EINVAL (bad label, K < 1, graph without edges), QM_ENOMEM, QM_ECUDA.
 */
qm_status qm_score_partition(const qm_graph *g, const int32_t *labels, int32_t K, qm_mem where,
                             qm_quality *out, const qm_percomm *per_comm, void *stream);

/* Result of comparing a detected partition with the ground truth (Sec. II-A). */
typedef struct {
    int64_t n_nodes;
    int64_t k_truth;    /* non-empty communities of the ground truth C */
    int64_t k_found;    /* non-empty communities of the detected C' */
    int64_t n_cells;    /* non-zero cells |c n c'| */
    int64_t a11, a10, a01, a00; /* node-pair counts of Sec. II-A.3 */
    int64_t nvd_sum;    /* sum_c max_c' |c n c'| + sum_c' max_c |c n c'| */
    double vi;          /* Eq. (1), natural log */
    double nmi;         /* Eq. (2) */
    double f_measure;   /* Eq. (3), sum over C, max over C' */
    double nvd;         /* Eq. (4) */
    double ri;          /* Eq. (5) */
    double ari;         /* Eq. (6) */
    double ji;          /* Eq. (7) */
} qm_compare;

/*
 * qm_compare_partitions -- Eqs. (1)-(7) from the contingency table of two
 * partitions of the same n_nodes nodes.  truth = C (ground truth), found = C'.
 *   truth  int32[n_nodes] in [0, k_truth); found int32[n_nodes] in [0, k_found)
 * The cells are counted per detected community in shared-memory hash tables
 * (a community with more distinct truth labels than a table holds is split
 * into hash classes sized with room to spare) and the terms of every cell are
 * then formed in parallel.
 * Errors: QM_EINVAL (n_nodes < 2, bad label), QM_ENOMEM, QM_ECUDA, QM_EOVERFLOW
 * (a hash class still overflowed: reported rather than dropped; not expected
 * for any real labelling).
 */
qm_status qm_compare_partitions(const int32_t *truth, const int32_t *found, int64_t n_nodes,
                                int32_t k_truth, int32_t k_found, qm_mem where,
                                qm_compare *out, void *stream);

/*
 * Overlapping communities (covers).  The paper defines its metrics for
 * disjoint communities and leaves overlapping ones to future work (Sec. VI);
 * every formula is written with node sets, and a cover -- a family of node
 * sets in which a node may belong to several communities or to none -- is
 * scored by reading them literally:
 *   |c|          the members of c;
 *   |E_c^in|     edges with both ends in c;
 *   |E_c^out|    edges with exactly one end in c;
 *   |E_ci,cj|    edges {u, v} with u in c_i \ c_j and v in c_j \ c_i;
 *   |c n c'|     nodes in both c and c' (one node may add to several cells);
 *   a11 .. a00   a pair of nodes is together in a cover when the two share a
 *                community.
 * Q, Qds, the six measures and Eqs. (1)-(7) then follow their printed formulas
 * (VI may be negative and F above 1 on covers).  For a cover with exactly one
 * community per node every result equals the partition call's, bit for bit,
 * except cut_edges_total (below).
 *
 * A cover is given node by node: the communities of node u are
 * memb[mptr[u] .. mptr[u+1]), strictly increasing ids in [0, K); mptr is
 * int64[n_nodes + 1] with mptr[0] = 0, memb int32[mptr[n_nodes]] (fewer than
 * 2^31 memberships).  Both arrays live where `where` says.
 *
 * qm_score_cover -- Eqs. (8)-(9) and the Sec. II-B.3 measures of a cover on a
 * loaded graph (any node order; the lists are in the caller's node order).
 * out->cut_edges_total holds the sum over communities of |E_c^out| (an edge
 * may leave several communities; for a partition it is twice the cut edges).
 * Errors: QM_EINVAL (malformed lists, no non-empty community, weighted graph),
 * QM_EOVERFLOW, QM_ENOMEM, QM_ECUDA.
 */
qm_status qm_score_cover(const qm_graph *g, const int64_t *mptr, const int32_t *memb, int32_t K,
                         qm_mem where, qm_quality *out, void *stream);

/*
 * qm_compare_covers -- Eqs. (1)-(7) for two covers of the same n_nodes nodes,
 * truth C = (truth_ptr, truth_memb, k_truth) and detected C' = (found_ptr,
 * found_memb, k_found).  The pair counts follow their definition (pairs
 * sharing a community); the cost beyond the cells grows with the pairs of
 * nodes that both have two or more memberships within one community.
 */
qm_status qm_compare_covers(const int64_t *truth_ptr, const int32_t *truth_memb, int32_t k_truth,
                            const int64_t *found_ptr, const int32_t *found_memb, int32_t k_found,
                            int64_t n_nodes, qm_mem where, qm_compare *out, void *stream);

/*
 * Batched calls.  On graphs of up to 2^21 nodes and 2^24 - 1 arcs the items
 * run the two-phase pipeline of the plain path with every phase spread over
 * all items at once (label histograms and counting sort, far-end gathers,
 * per-community counts with direct or hashed counters, contingency cells, then
 * the FP64 terms of all items), replayed from a captured CUDA graph; the
 * scratch grows with the items (about 11 MB per item of 10^5 nodes and 10^6
 * edges), so large batches run in waves of at most an eighth of free device
 * memory.  Denser graphs of up to 2^21 nodes run one persistent kernel, one
 * block per item.  On larger graphs every item runs the plain full-GPU
 * pipelines one after another, all captured into one CUDA graph launched
 * once, with one copy of all results at the end.  Every way each result is
 * bit-identical to the plain call on that item.
 *
 * qm_score_partitions_batched -- score P partitions of one graph in a single
 * launch.
 *   labels  int32[P][n_nodes] row-major
 *   K       host int32[P], label-id count of each partition
 *   out     host qm_quality[P]
 * Each out[p] is bit-identical to qm_score_partition on partition p.
 */
qm_status qm_score_partitions_batched(const qm_graph *g, const int32_t *labels, int32_t P,
                                      const int32_t *K, qm_mem where, qm_quality *out,
                                      void *stream);

/*
 * qm_compare_partitions_batched -- compare P detected partitions with ground
 * truth in one launch.
 *   truth   int32[n] when flags has QM_SHARED_TRUTH, else int32[P][n]
 *   found   int32[P][n]
 *   k_truth host int32[1] with QM_SHARED_TRUTH, else int32[P]; k_found host int32[P]
 *   out     host qm_compare[P], each bit-identical to qm_compare_partitions
 */
qm_status qm_compare_partitions_batched(const int32_t *truth, const int32_t *found, int64_t n_nodes,
                                        int32_t P, const int32_t *k_truth, const int32_t *k_found,
                                        unsigned flags, qm_mem where, qm_compare *out,
                                        void *stream);

/*
 * qm_evaluate_partitions_batched -- for each of P candidate partitions of one
 * graph, every metric with and without ground truth, in one launch:
 * out_q[p] as qm_score_partition(labels[p]) and out_c[p] as
 * qm_compare_partitions(truth, labels[p]).
 *   truth int32[n] shared by all candidates, k_truth its label-id count
 */
qm_status qm_evaluate_partitions_batched(const qm_graph *g, const int32_t *labels, int32_t P,
                                         const int32_t *K, const int32_t *truth, int32_t k_truth,
                                         qm_mem where, qm_quality *out_q, qm_compare *out_c,
                                         void *stream);

/*
 * qm_score_graphs_batched -- score one partition on each of `count` graphs of
 * possibly different sizes in one persistent launch.
 *   graphs  host array of count graph handles
 *   labels  host array of count pointers, labels[i] = int32[n_nodes of graphs[i]]
 *   K       host int32[count]; out host qm_quality[count]
 */
qm_status qm_score_graphs_batched(const qm_graph *const *graphs, const int32_t *const *labels,
                                  const int32_t *K, int32_t count, qm_mem where, qm_quality *out,
                                  void *stream);

/*
 * qm_workspace_bytes -- device scratch one scoring call of this graph with K
 * label ids needs (with_compare != 0: also a compare against a truth with
 * k_truth ids).  Used for admission control by memory budget.
 */
qm_status qm_workspace_bytes(const qm_graph *g, int32_t K, int32_t with_compare, int32_t k_truth,
                             size_t *bytes);

/* Drop cached scratch buffers and captured CUDA graphs (they are rebuilt on demand). */
qm_status qm_release_cache(void);

/*
 * qm_debug_set_stage_wait -- test hook for the bounded device wait (no
 * counterpart in the paper).  The pair-count kernel stages each long run of
 * packed labels into shared memory with an asynchronous bulk copy and waits for
 * it on an mbarrier for at most `polls` polls (default 2^22); when the wait
 * expires the kernel stops issuing copies, lets the one copy in flight land
 * (a second wait, bounded by the default), sets a status bit and returns, and
 * the call returns QM_ETIMEOUT with the context still usable.  Setting polls to
 * 0 makes every such wait expire at its first check, without withholding any
 * copy, so that a test can drive this path; a negative value restores the
 * default.  Applies to all later calls in the process (captured calls are
 * dropped, as by qm_release_cache).  Only the two-phase scoring pipeline
 * stages copies.
 */
qm_status qm_debug_set_stage_wait(int64_t polls);

/*
 * qm_debug_set_batch_wave -- test hook for the batched calls (no counterpart
 * in the paper).  Large batches of the two-phase batched pipeline run in waves
 * of items sized by free device memory; items > 0 caps every later call's wave
 * at that many items (so that a test can drive the wave loop with a small
 * batch), 0 restores the automatic size.  Results do not depend on it.
 * Errors: QM_EINVAL for items < 0.
 */
qm_status qm_debug_set_batch_wave(int32_t items);

/*
 * qm_debug_set_perm_buckets -- test hook for graphs loaded with QM_REORDER
 * (no counterpart in the paper).  A scoring call on such a graph first brings
 * the caller's labels into the stored order.  On graphs of more than
 * min_nodes nodes (default 2^24) this takes two passes through shared memory,
 * with sequential global reads and writes: labels are grouped per tile of
 * 2^tile_bits caller ids by the window of 2^window_bits new ids they go to,
 * then placed per window; shared memory holds the labels as 3 bytes while
 * K <= 2^24.  By default windows and tiles hold 2^16 ids (tiles of 2^15 or
 * 2^14 where the windows of a larger graph need the room).  Index arrays for
 * this are built at load (4 bytes a node plus two ints per tile and window).
 * Smaller graphs, graphs with more than 8192 windows, and calls whose labels
 * do not fit the shared memory gather the labels directly.  The setting
 * applies to graphs loaded afterwards (so that a test can drive the two
 * passes on a small graph); results do not depend on it.  A negative
 * argument restores its default (for the bits: the automatic choice).
 * Errors: QM_EINVAL for window_bits or tile_bits of 0 or above 16.
 */
qm_status qm_debug_set_perm_buckets(int32_t window_bits, int32_t tile_bits, int64_t min_nodes);

/*
 * Tuning.  qm_autotune times the candidate launch shapes of the scoring and
 * batched kernels on the given inputs and caches the fastest per size bucket
 * (log2 n_nodes, log2 n_arcs, log2 K).  qm_get_tuning reports the shape the
 * next call of that bucket will use: threads per block, shared-memory bytes per
 * block, and the community size above which a whole block (not a warp) scores a
 * community (used by algorithm 0 only).  algorithm selects the scoring pipeline:
 *   0  one kernel visits every community's members and gathers their
 *      neighbours' labels itself;
 *   1  (default) the neighbour labels are first written out in community
 *      order (one streaming pass over the arcs), then a second kernel counts
 *      each community's contiguous segment and a third forms the FP64 terms of
 *      all communities in parallel;
 *   2  as 1, but an arc whose far end is not close to its near end in node-id
 *      order has its label gathered later, through bins by windows of the
 *      node ids, so that those gathers hit one L2-sized window of the label
 *      array at a time (measured slower than 1 on the LFR-style graphs of
 *      10^8 nodes, in either node order; the autotuner tries it above 2^24
 *      nodes);
 *   3  as 2 with every arc binned and about four windows (for tests and
 *      comparisons on small graphs);
 *   4  as 1, with the far-end labels always gathered from a copy packed three
 *      21-bit ids to a 64-bit word (8/3 bytes a node instead of 4, so a larger
 *      share of it stays in L2); algorithm 1 does this on graphs of more than
 *      2^22 nodes.  On a graph loaded with QM_REORDER the gathers first try a
 *      block encoding built per call (per 16 consecutive nodes two labels and
 *      a 16-bit mask, blocks of three or more labels apart: half a byte a
 *      node when the partition follows the stored order, so that it stays in
 *      L2), falling back to the packed copy when too many blocks hold three
 *      or more labels; algorithm 1 does this above 2^26 nodes;
 *   5  as 1, never packed;
 *   6  as 1, but the second kernel sorts each community's segment by label
 *      (a radix sort in shared memory, 8-bit digits) and counts the equal-label
 *      stretches instead of hashing the labels (Eq. (9)'s |E_cj| are those
 *      stretches' lengths); segments longer than a block's sort buffers are
 *      hashed as in 1.  Needs threads * 256 entries of sort buffers per block
 *      (else the shape is refused);
 *   7  as 1, but each undirected edge is gathered once, from its lower node
 *      id, through a copy of the graph's upper rows (arcs to itself and higher
 *      ids) made at load time (unweighted graphs with fewer than 2^32 arcs;
 *      8 bytes a node and 4 an edge): an edge inside c adds to 2|E_c^in|, an
 *      edge to another community puts one entry into the run of the smaller
 *      id, appended to that run's segment from wherever it is found.  Half the
 *      far-end gathers, at the price of scattered appends: faster on graphs in
 *      a random node order whose label array exceeds L2 (the default for
 *      untuned graphs loaded without QM_REORDER above 2^26 nodes), slower on
 *      reordered or smaller graphs.  Sharded calls run 1 instead.
 * Packing needs K <= 2^21; with more label ids the 32-bit labels are gathered.
 * All give bit-identical results.  Weighted graphs take algorithm 1 whatever
 * is set; algorithm 7 needs the upper rows, else it runs as 1.
 */
typedef struct {
    int32_t threads;
    int32_t smem_bytes;
    int32_t big_community;
    int32_t blocks_per_sm;
    int32_t algorithm;
} qm_tuning;

qm_status qm_autotune(const qm_graph *g, const int32_t *labels, int32_t K, qm_mem where,
                      void *stream, qm_tuning *chosen);
qm_status qm_get_tuning(const qm_graph *g, int32_t K, qm_tuning *t);
qm_status qm_set_tuning(const qm_graph *g, int32_t K, const qm_tuning *t);

/*
 * The same for the batched calls (qm_score_partitions_batched,
 * qm_evaluate_partitions_batched), keyed by the batch's largest K.
 * qm_autotune_batched times candidate shapes on the caller's batch, exactly
 * as qm_evaluate_partitions_batched (truth != NULL) or
 * qm_score_partitions_batched (truth == NULL) would run it, and caches the
 * fastest; the batch's results are the same bits for every shape.  The shape
 * sets the threads and shared memory of the per-community counting and cells
 * kernels (a warp's share of the shared memory bounds the runs it counts and
 * the communities it compares; larger ones go to whole blocks); the
 * block/warp community-size split applies to the one-block-per-item kernel
 * only.  The algorithm field is ignored, and the batched kernels take at most
 * 512 threads a block (qm_set_batch_tuning returns QM_EINVAL for more).
 */
qm_status qm_autotune_batched(const qm_graph *g, const int32_t *labels, int32_t P, const int32_t *K,
                              const int32_t *truth, int32_t k_truth, qm_mem where, void *stream,
                              qm_tuning *chosen);
qm_status qm_get_batch_tuning(const qm_graph *g, int32_t K, qm_tuning *t);
qm_status qm_set_batch_tuning(const qm_graph *g, int32_t K, const qm_tuning *t);

/*
 * Sharded scoring -- the paper's decomposition of the no-ground-truth metrics
 * by community (Sec. III-A): community c belongs to shard c mod P, each shard
 * sums the terms of its own communities, and one sum over the shards gives
 * the partition's values (the single reduction of the paper's processes).
 * Each shard needs the whole graph and all labels (neighbours' communities
 * and all community sizes enter the sums).  The partial sums are exact
 * integers, so any split gives the bits of qm_score_partition.
 *
 *   qm_score_partition_part   shard `rank` of `nranks` (1..64) of one call of
 *                             qm_score_partition (same arguments, no
 *                             per-community output); fills *out.
 *   qm_partials_combine       exact sum of `count` partials of the same graph
 *                             and shard count, each shard at most once;
 *                             host-only, touches no GPU.
 *   qm_partial_finalize       the metrics from a partial that covers every
 *                             shard (one small kernel on the current device).
 * Errors: QM_EINVAL (ranks out of range, partials of different graphs or
 * shard counts, a shard repeated or missing), plus those of
 * qm_score_partition.
 */
#define QM_PARTIAL_WORDS 32
typedef struct {
    int64_t n_nodes, n_edges;
    int32_t nranks;                   /* number of shards of the call */
    int32_t flags;                    /* bit 0: a weighted graph's partial */
    uint64_t ranks_mask;              /* shards summed into this partial: bit r = shard r */
    uint64_t words[QM_PARTIAL_WORDS]; /* exact integer sums (opaque) */
} qm_partial;

qm_status qm_score_partition_part(const qm_graph *g, const int32_t *labels, int32_t K, qm_mem where,
                                  int32_t rank, int32_t nranks, qm_partial *out, void *stream);
qm_status qm_partials_combine(const qm_partial *parts, int32_t count, qm_partial *out);
qm_status qm_partial_finalize(const qm_partial *p, qm_quality *out, void *stream);

/*
 * qm_score_partition_noalloc -- qm_score_partition for callers that cannot let
 * a library allocate memory while it runs (no counterpart in the paper).
 *
 * Some hosts hand a plugin no allocator (all GPU memory is budgeted up front),
 * and some latency-critical loops must not pay for the device-wide
 * synchronisation that cudaMalloc / cudaFree can cause.  This call computes the
 * same result as qm_score_partition (bit-identical output) but
 * allocates nothing: its scratch memory is one fixed device array of
 * QM_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library keeps until the process exits, and the result is copied straight
 * into *out.
 *   g       graph loaded with qm_load_graph
 *   labels  device int32[n_nodes], labels in [0, K)
 *   out     host struct, written on success
 * Limits and rules:
 *   - The call runs the one-kernel pipeline (tuning algorithm 0).  Its
 *     workspace must fit the array: about 4 * n_nodes + 36 * K bytes, plus
 *     4 * n_nodes for a graph loaded with QM_REORDER (for example 10,000,000
 *     nodes with 100,000 label ids).  Larger calls return QM_EOVERFLOW with the
 *     required size in qm_last_error().
 *   - labels must be device memory (QM_EINVAL otherwise); no per-community
 *     outputs.
 *   - All calls share the one array, and each call clears what must start at
 *     zero.  Calls whose GPU work overlaps (on different streams, or from
 *     different threads) race on it: issue them one after the other.
 *   - The first call on a device does a one-time set-up on that device (it
 *     resolves the array's device address and the kernels' launch shape); make
 *     that first call before any stream capture begins.
 */
#define QM_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
qm_status qm_score_partition_noalloc(const qm_graph *g, const int32_t *labels, int32_t K,
                                     qm_quality *out, void *stream);

/*
 * qm_label_propagation -- a detected partition C' of the graph by synchronous
 * label propagation (the O(|E|) detector family the paper scores, Sec. I and
 * Sec. IV-C; not SLPA itself).  Labels start as the node ids; in each round
 * every node takes the label found most often among its neighbours (among up
 * to 32 evenly spaced ones: positions floor(i * deg / 32), i < 32, when
 * deg > 32), keeps its own label when that is among the most frequent, and
 * otherwise takes the smallest of the most frequent.  Afterwards the labels
 * present are renumbered in increasing order to [0, K').  Deterministic, and
 * the same for a graph loaded with QM_REORDER.
 *   rounds      number of rounds, 0..1000
 *   labels_out  int32[n_nodes] (host or device memory as `where` says)
 *   k_out       host int32, receives K'
 * Errors: QM_EINVAL, QM_ENOMEM, QM_ECUDA.
 */
qm_status qm_label_propagation(const qm_graph *g, int32_t rounds, int32_t *labels_out, qm_mem where,
                               int32_t *k_out, void *stream);

/* Number of this library's kernel launches issued since load (for accounting). */
int64_t qm_kernel_launches(void);

/*
 * Kernel tracing (per calling thread).  With tracing on, every kernel a call
 * launches is bracketed by CUDA events recorded on the call's stream, and after
 * the call returns qm_trace_read reports each kernel of that call in launch
 * order with its device time (the time between its two events).  A batched
 * call reports its whole graph launch as one entry.  Tracing adds two event
 * records per kernel; it is off by default.
 *   events    caller array of `capacity` entries (may be NULL when capacity is 0)
 *   count     receives the number of kernels of the last traced call
 */
typedef struct {
    char name[28];
    float ms;
} qm_trace_event;

qm_status qm_trace_enable(int32_t on);
qm_status qm_trace_read(qm_trace_event *events, int32_t capacity, int32_t *count);

const char *qm_strerror(qm_status s);
/* Copies the calling thread's last error message into buf (always NUL-terminated). */
qm_status qm_last_error(char *buf, size_t len);
/* The same as qm_last_error (the name the interface plan uses). */
qm_status qm_last_error_detail(char *buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* QM_H */
