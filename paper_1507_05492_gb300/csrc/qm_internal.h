// qm_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qm.h"

namespace qmk {
struct Cell;    // one contingency cell (qm_community.cuh)
struct Rcp;     // 128-bit reciprocal of a community size (qm_device.cuh)
struct RunHdr;  // header of one community's packed run (qm_community.cuh)
}

namespace qm {

// Device copy of a symmetric CSR (library-owned).
struct GraphDev {
    const long long *row_ptr;  // [n + 1]
    const int *col;            // [n_arcs]
    long long n;
    long long n_arcs;
    long long max_degree;
    const int *inv = nullptr;  // loaded with QM_REORDER: new node id -> caller's node id
    const float *wt = nullptr; // weighted graph: [n_arcs] edge weights parallel to col
    // unweighted graphs: the upper rows (arcs (u, v) with v >= u, a self-loop
    // stored as ~u), for gathering each undirected edge once (ALGO_HALF)
    const long long *up_ptr = nullptr;  // [n + 1]
    const int *up_col = nullptr;
    unsigned long long w_lo = 0, w_hi = 0;  // weighted graph: total weight W * 2^43 (128-bit)
};

// Launch shape of the community-major kernels.
struct Shape {
    int threads;        // threads per block (multiple of 32, <= 1024)
    int smem_bytes;     // dynamic shared memory per block
    int big_community;  // communities with more members are scored by a whole block
    int blocks_per_sm;  // resident blocks per SM (filled in from occupancy)
    int algo = 0;       // 0: one-kernel community pass, 1: expand + count (two phases); see ALGO_*
};

// Two-phase pipeline whose phase B sorts each community's run and
// run-length encodes it (k_count_sort) instead of hashing it (k_count);
// gathers as algorithm 1.
constexpr int ALGO_SORT = 6;
// Two-phase pipeline whose phase A gathers each undirected edge once, from its
// lower end, through the graph's upper rows (k_expand_half); otherwise as
// algorithm 1.  Unsharded, unweighted, unbinned calls on graphs that hold the
// upper rows; others run algorithm 1.
constexpr int ALGO_HALF = 7;
// Untuned calls take ALGO_HALF on graphs in their given node order with more
// nodes than this.
constexpr long long HALF_MIN_NODES = 1LL << 26;

// Carving of the dynamic shared memory of a community-major block.
struct SmemPlan {
    int red_off, ctl_off, acc_off, offs_off, rs_off, slot_off, used_off;
    int cap, max_used;        // whole-block table
    int cap_w, max_used_w;    // one warp's table
    int bytes;
};
SmemPlan plan_smem(int threads, int smem_bytes);

// Shared-memory layout of the two-phase count kernel: reduction exchange,
// table control words, two mbarriers, two staging buffers for bulk-copied
// runs, and the counting table (a block table of `cap` slots, or W warp
// slices of cap_w).  Runs of up to `fill` entries (3/4 of the table) are
// staged; warps take runs of up to fill_w.
struct CountPlan {
    int red_off, ctl_off, bar_off, stage_off, slot_off;
    int stage_elems;
    int cap, fill, cap_w, fill_w;
    int ng, cap_g, fill_g;  // ng groups of warps, each with a table of cap_g slots (ng = 1: none)
    int bytes;
};
CountPlan plan_count(int threads, int smem_bytes);

// Device scratch of one plain scoring call (carved from one allocation).
struct ScoreWs {
    int *status;                // [1] bit 0: label out of range
    int *counters;              // [8]
    unsigned long long *gacc;   // [32]
    qm_quality *result;         // [1]
    int *size;                  // [K]
    int *start;                 // [K + 1]
    qmk::Rcp *recip;            // [K] rcp_of(|c|)
    int *cursor;                // [K]
    int *big_list;              // [K]
    int *ovf_list;              // [K]
    int *members;               // [n]
    int *scan_tmp;              // [scan tiles + 1]
    unsigned *aoff;             // two-phase only: [n + 1] arc offsets of member positions
    int *inter;                 // two-phase only: [K] cut arcs of each community (zeroed)
    int *inter_hi;              // two-phase only: [K] packed labels above c of each community (zeroed)
    qmk::RunHdr *hdr_big;       // two-phase only: [K] run headers for whole blocks
    qmk::RunHdr *hdr_small;     // two-phase only: [K] run headers for single warps
    qmk::RunHdr *hdr_long;      // two-phase only: [K] run headers for k_count_long
    qmk::RunHdr *hdr_mid;       // two-phase only: [K] run headers for groups of warps
    int *nbr;                   // two-phase only: [n_arcs] neighbour labels in community order
    unsigned long long *rec;    // two-phase only: [K][6] per-community records
    float *nbrw = nullptr;      // weighted graphs: [n_arcs] weights of the packed cut arcs
    unsigned long long *wl = nullptr;    // weighted graphs: [K][6] intra / cut weight limbs (zeroed)
    unsigned long long *recw = nullptr;  // weighted graphs: [K][4] 256-bit weighted pair sums
    // far-end gathers through destination-window bins (algorithms 2 and 3; qm_binned.cuh)
    unsigned long long *bin_pool = nullptr, *bin_list = nullptr, *bin_sorted = nullptr;
    int *bin_ctr = nullptr;     // [64] counters (zeroed)
    int *bin_seg = nullptr;     // [K]
    long long bin_chunks = 0;   // pool capacity in chunks
    int bin_shift = 0, bin_nbins = 0, bin_near = 0;
    unsigned long long *plab = nullptr;  // packed labels (three 21-bit ids a word), [(n + 2) / 3]
    size_t zero_bytes;          // bytes from `status` that must start at zero
    size_t bytes;               // total bytes carved (the *_ws_bytes size)
};

struct CompareWs {
    int *status;
    int *counters;
    unsigned long long *gacc;
    qm_compare *result;
    int *size_a;                // [ka]
    int *size_b;                // [kb]
    unsigned *rowmax_n;         // [ka]
    unsigned long long *rowmax_r; // [ka]
    int *start;                 // [kb + 1]
    int *cursor;                // [kb]
    int *big_list;              // [kb]
    int *members;               // [n]
    qmk::Cell *cells;  // contingency cells of the counting pass ([n])
    int *scan_tmp;
    double *logt;               // [LOGT_WORDS] log(N / n), then n / N (LOGT_MAX + 1 each)
    size_t zero_bytes;
    size_t bytes;  // total bytes carved (compare_ws_bytes)
};

size_t score_ws_bytes(long long n, int K);
// bin_mode (two-phase pipeline): 0 gathers every label directly; 2 bins the
// arcs whose far end is not close in node-id order, by windows of at least 2^23
// node ids; 3 bins every arc, by about four windows (tests and comparisons).
// Weighted graphs take mode 0.
// pack (two-phase pipeline, direct gathers, K <= 2^21): the far-end gathers
// read a copy of the labels packed three to a 64-bit word.
size_t score2_ws_bytes(long long n, long long n_arcs, int K, bool weighted = false, int bin_mode = 0,
                       bool pack = false);
ScoreWs carve_score2_ws(void *base, long long n, long long n_arcs, int K, bool weighted = false, int bin_mode = 0,
                        bool pack = false);
// The binning mode of a two-phase launch shape on a graph (algorithm 2 or 3
// on an unweighted graph; 0 otherwise).
inline int bin_mode_of(int algo, bool weighted) { return (!weighted && (algo == 2 || algo == 3)) ? algo : 0; }
// Graphs with more nodes than this gather packed labels by default (algorithm
// 1): their label array is well beyond what L2 keeps.
constexpr long long PACK_MIN_NODES = 1LL << 22;
// Whether a two-phase call gathers from the packed copy: algorithm 4 always,
// algorithms 1, ALGO_SORT and ALGO_HALF on graphs above PACK_MIN_NODES;
// unweighted graphs and label ids below 2^21 only.
// Renumbered graphs of more nodes than this gather from the block encoding of
// the labels (qm_expand.cuh) instead of the packed copy (tuning algorithm 4:
// at any size): below it the packed copy mostly stays in L2 already and the
// encoding's pass and decode cost more than they save.
constexpr long long BLOCKS_MIN_NODES = 1LL << 26;
inline bool label_blocks(int algo, long long n) { return algo == 4 || n > BLOCKS_MIN_NODES; }

inline bool packs_labels(int algo, bool weighted, long long n, int K)
{
    return !weighted && K <= (1 << 21) &&
           (algo == 4 || ((algo == 1 || algo == ALGO_SORT || algo == ALGO_HALF) && n > PACK_MIN_NODES));
}
// The autotuner tries the binned gathers on graphs with more nodes than this:
// their label array (4 bytes a node) is beyond what L2 serves at random.
constexpr long long BIN_MIN_NODES = 1LL << 24;
size_t compare_ws_bytes(long long n, int ka, int kb);
ScoreWs carve_score_ws(void *base, long long n, int K);
CompareWs carve_compare_ws(void *base, long long n, int ka, int kb);

// Optional per-community outputs (device pointers).
struct PerCommDev {
    long long *size, *ein, *eout;
    double *dens, *contr, *expn, *cond, *qds;
};

// Optional tracing hook: called with a kernel name right before each launch
// and with nullptr after the last one, on the launching stream.
typedef void (*TraceFn)(const char *name, cudaStream_t s);

// Plain path launchers (stream-ordered, no synchronisation).  Each returns the
// number of kernels it launched, or -1 on a launch error.
int launch_score(const GraphDev &g, const int *labels, int K, const ScoreWs &ws, const Shape &sh,
                 const PerCommDev *pc, int num_sms, cudaStream_t s, TraceFn tr);
int launch_score2(const GraphDev &g, const int *labels, int K, const ScoreWs &ws, const Shape &sh,
                  const PerCommDev *pc, int num_sms, cudaStream_t s, TraceFn tr, int shard_r = 0,
                  int shard_p = 1, bool sizes_ready = false);
// For a renumbered graph: out[j] = labels[inv[j]] and the community sizes into
// ws.size (zeroed), with the label range check of k_hist.  Returns 1 or -1.
int launch_permute_hist(const int *labels, const int *inv, long long n, int *out, int K, const ScoreWs &ws,
                        int num_sms, cudaStream_t s);
// k_score_fin on an accumulator array of GS_COUNT words (a combined set of shard
// partials): status must point at a zero int.  Returns 1 (launches) or -1.
int launch_score_fin(const unsigned long long *gacc, const int *status, long long n, long long E, qm_quality *out,
                     int weighted, cudaStream_t s);
// Load-time checks of a weighted graph's weights (range, and symmetry when
// `full`) and its total weight 2W * 2^43 in three limbs at lim (zeroed by the
// caller); status bit 1: weight out of range, bit 2: asymmetric.
int launch_weight_check(const GraphDev &g, const float *wt, int full, int *status, unsigned long long *lim,
                        int num_sms, cudaStream_t s);
int launch_compare(const int *truth, const int *found, long long n, int ka, int kb,
                   const CompareWs &ws, const Shape &sh, int num_sms, cudaStream_t s, TraceFn tr);
int count_blocks_per_sm(const Shape &sh);
int sort_blocks_per_sm(const Shape &sh);
// Whether k_count_sort can run with this block shape (its warps' buffers fit).
bool sort_shape_ok(int threads, int smem_bytes);

// Generic exclusive scan (qm_kernels.cu) and the graph reorder (qm_reorder.cu).
size_t scan_tmp_elems(long long n);
int scan_offsets(const int *in, int n, int *out, int *tmp, int *counters, const int *status, cudaStream_t s);
int launch_permute_labels(const int *labels, const int *inv, long long n, int P, int *out, int num_sms,
                          cudaStream_t s);
// Bucketed label permutation of a renumbered graph (qm_reorder.cu): built
// once at load, it turns the gather out[j] = labels[inv[j]] into two passes
// with sequential global reads and writes (the random part in shared memory)
// through a scratch array of n ints.  Caller ids are cut into tiles of 2^tb,
// new ids into windows of 2^wb.
constexpr int PB_MAX_BITS = 16;        // 16-bit positions inside tiles and windows
constexpr int PB_MAX_WINDOWS = 8192;   // the build counts windows in shared memory
struct PermBuckets {
    unsigned short *lpos = nullptr;  // [n] caller id -> position in its tile's order (grouped by window)
    unsigned short *dloc = nullptr;  // [n] slot -> new id inside its window
    int *toff = nullptr;             // [ntiles][nw] first slot of each (tile, window) group
    int *tlb = nullptr;              // [ntiles][nw + 1] first tile position of each group
    int wb = 0, tb = 0, nw = 0, ntiles = 0;
    size_t smem_max = 0;             // shared memory a block may take on the graph's device
    size_t bytes = 0;
};
// Device arrays owned by the caller afterwards.  Returns 0, 1 when the sizes
// do not fit the two passes (nothing built), or minus a CUDA error code
// (nothing allocated then).
int build_perm_buckets(const int *inv, long long n, int wb, int tb, int num_sms, cudaStream_t s, PermBuckets *out,
                       int *launches);
void free_perm_buckets(PermBuckets *pb);
// out[j] = labels[inv[j]] by the two passes (tmp: n ints), labels outside
// [0, K) flagged in bit 0 of *status; with `size`, also the community sizes,
// as k_hist.  Returns launches, 0 when K is too large for the passes' shared
// memory (nothing launched: gather the labels instead), or -1.
int launch_permute_buckets(const int *labels, const PermBuckets &pb, long long n, int *tmp, int *out, int *size,
                           int K, int *status, int num_sms, cudaStream_t s,
                           void (*tr)(const char *, cudaStream_t) = nullptr);
// Builds the renumbered CSR (row_ptr, col: new device allocations) and inv
// (new id -> old id) of g from `rounds` label-propagation rounds.  Returns 0,
// or minus a CUDA error code (nothing allocated then).
int reorder_graph(const GraphDev &g, int rounds, int num_sms, cudaStream_t s, long long **row_ptr_out, int **col_out,
                  int **inv_out, int *launches, float **wt_out = nullptr);
// The upper rows of a symmetric CSR (see GraphDev::up_ptr): device arrays
// owned by the caller afterwards.  Needs n_arcs < 2^32.  Returns 0, or minus
// a CUDA error code.
int build_upper_rows(const GraphDev &g, int num_sms, cudaStream_t s, long long **up_ptr_out, int **up_col_out,
                     long long *up_arcs, int *launches);
// qm_label_propagation on the device: `rounds` rounds from the caller's node
// ids, then the labels present are ranked into [0, K'): out (caller order,
// n entries) and hist[n] = K' (device).  lab0, lab1: n ints; hist: n + 1;
// tmp: tmp_elems >= scan_tmp_elems(n + 1) + 64.  Returns launches or -1.
int launch_label_propagation(const GraphDev &g, int rounds, int num_sms, cudaStream_t s, int *lab0, int *lab1,
                             int *hist, int *tmp, size_t tmp_elems, int *out);

// Largest dynamic shared memory a community-major block may request.
constexpr int MAX_DYN_SMEM = 220 * 1024;

// Largest block of the batched kernel (its launch bound: at most 512 threads
// leaves it 128 registers a thread, so that its per-item state stays in
// registers).
constexpr int BATCH_MAX_THREADS = 512;

// Raises the dynamic shared-memory limit of the kernels to MAX_DYN_SMEM (once
// per device, before any launch or capture).
void prepare_kernels();
void prepare_batched_kernel();

// Occupancy of the community-major kernels for a shape.
int score_blocks_per_sm(const Shape &sh);

// Poll limit of k_count's pipelined staging wait for later launches (negative:
// the default).
void set_stage_wait_polls(long long polls);

// ---- batched persistent kernel

// One work item of the batched kernel: score and/or compare one partition.
struct BatchItem {
    const long long *row_ptr;
    const int *col;
    const int *labels;       // partition to score / detected partition
    const int *truth;        // ground truth (compare), or null
    long long n;
    long long n_arcs;
    int K;
    int k_truth;
    int flags;               // 1 = score, 2 = compare
    int pad;
    qm_quality *out_q;       // device result slots
    qm_compare *out_c;
    int *status;             // per-item status word
};

struct BatchScratch {
    int *members;            // [slots][n_max]
    int *size;               // [slots][k_max]
    int *start;              // [slots][k_max + 1]
    int *size_a;             // [slots][kt_max]
    unsigned *rowmax_n;      // [slots][kt_max]
    unsigned long long *rowmax_r; // [slots][kt_max]
    int *big_list;           // [slots][3 k_max]
    qmk::Rcp *recip;           // [slots][k_max]
    long long n_max;
    int k_max, kt_max;
    int slots;
};

size_t batch_scratch_bytes(long long n_max, int k_max, int kt_max, int slots);
BatchScratch carve_batch_scratch(void *base, long long n_max, int k_max, int kt_max, int slots);

int launch_batched(const BatchItem *items_dev, int count, int *queue, const BatchScratch &bs,
                   const Shape &sh, int num_sms, cudaStream_t s, TraceFn tr);
int batched_blocks_per_sm(const Shape &sh);

// ---- used by the allocation-free entry point (qm_noalloc.cu)

// Records the calling thread's error message (read by qm_last_error) and
// returns s.
qm_status set_error(qm_status s, const char *msg);
// Device copy and device id of a loaded graph; QM_EINVAL for a null handle.
qm_status graph_device_view(const qm_graph *g, GraphDev *out, int *device);

// ---- graph validation
int launch_validate(const GraphDev &g, int full, int *status, unsigned long long *max_deg, int num_sms,
                    cudaStream_t s);

}  // namespace qm
