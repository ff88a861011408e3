// qm_batched.h -- the batched pipeline over many candidate partitions.
//
// k_batched (qm_batched.cu) gives every candidate one block, so a launch lasts
// as long as its slowest block and every community is scored by the one-kernel
// pass.  The pipeline declared here runs the two-phase method of the plain path
// over all candidates of a wave at once, each phase spread over the whole GPU:
//   prep    label histograms (with each community's volume) over (candidate,
//           node tile) units, community offsets by one block per candidate,
//           then the counting sort of the nodes by label, which also gives
//           each member position its arc offset (one 64-bit atomic a node);
//   expand  warps over (candidate, 32 member positions) units: far-end label
//           gathers, the packed runs of labels above each community's id;
//   count   warps (small runs) and blocks (the rest) over (candidate,
//           community) units: one integer record per community;
//   cells   the same over the found communities of the candidates compared:
//           contingency cells of Eqs. (1)-(7) into a per-candidate list;
//   fin     one block per candidate: FP64 terms of every community and cell
//           (all lanes busy), the fixed-point sums and the final results.
// The per-community and per-cell device functions are those of the plain path,
// so every result is the same bits as scoring that candidate alone.
#pragma once

#include "qm_internal.h"

namespace qm {

struct BatchUnits {
    // per candidate (slice `it` of each array)
    int *members;                  // [count][n_max] nodes in community order
    unsigned *aoff;                // [count][n_max + 1] arc offset of each member position
    int *start;                    // [count][k_max + 1]
    unsigned long long *cv;        // [count][k_max] (members << 40 | arcs): histogram, then scatter cursors (zeroed)
    qmk::Rcp *recip;               // [count][k_max] rcp_of(|c|)
    int *inter;                    // [count][k_max] cut arcs of each community (zeroed)
    int *inter_hi;                 // [count][k_max] packed run length, labels above c (zeroed)
    unsigned long long *rec;       // [count][k_max][REC_WORDS] count records
    int *nbr;                      // [count][a_max] packed runs
    void *cells;                   // [count][n_max] contingency cells (Cell), compare only
    int *size_a;                   // [count][kt_max] ground-truth sizes (zeroed)
    unsigned *rowmax_n;            // [count][kt_max] (zeroed)
    unsigned long long *rowmax_r;  // [count][kt_max] (zeroed)
    // per wave
    int *tpre;                     // [count + 1] prefix of the candidates' node tiles (BATCH_UNITS_TILE nodes)
    int *cpre;                     // [count + 1] prefix of the candidates' 32-position chunks
    int *kpre;                     // [count + 1] prefix of the candidates' label-id counts
    unsigned long long *big_s;     // [units] (candidate << 32 | community) counted by whole blocks
    unsigned long long *big_c;     // [units] compared by whole blocks
    double *logt;                  // [LOGT_WORDS] log(N / i), then i / N, for N = logt_n
    int *ncells;                   // [count] cells written (zeroed)
    unsigned long long *gcell;     // [count][2] column maxima and cell counts of the comparisons (zeroed)
    int *ctr;                      // [16] list lengths and claim counters (zeroed)
    long long n_max, a_max, logt_n;
    int k_max, kt_max, count;
    void *zero;                    // start of the region that must be zero at launch
    size_t zero_bytes;
    size_t bytes;
};

// Scratch of a wave of `count` candidates: n_max nodes, a_max arcs, k_max
// label ids, kt_max truth ids at most; cells only when some candidate is
// compared.
size_t batch_units_bytes(int count, long long n_max, long long a_max, int k_max, int kt_max, bool cells);
BatchUnits carve_batch_units(void *base, int count, long long n_max, long long a_max, int k_max, int kt_max,
                             bool cells);

// Launches the pipeline (stream-ordered; zero_bytes from `zero` must be zero,
// tpre, cpre and kpre filled, and every item's n_arcs at most
// BATCH_UNITS_MAX_ARCS).  logt_n is the
// node count of the log table (items of another size take the logarithm
// directly).  Returns the number of kernels launched, or -1.
int launch_batch_units(const BatchItem *items_dev, int count, const BatchUnits &b, long long logt_n,
                       const Shape &sh, int num_sms, cudaStream_t s);

// Fills a wave's tables, log(N / i) and i / N for i = 1 .. LOGT_MAX (stream-ordered).
void launch_batch_logt(double *logt, long long N, cudaStream_t s);

// Resident blocks per SM of the count and cells kernels for a launch shape.
int batch_units_blocks_per_sm(const Shape &sh);

// Items the pipeline accepts: runs of at most 2^24 - 1 entries.
constexpr long long BATCH_UNITS_MAX_ARCS = (1LL << 24) - 1;

// Nodes per unit of the histogram and scatter kernels.
constexpr int BATCH_UNITS_TILE = 4096;

}  // namespace qm
