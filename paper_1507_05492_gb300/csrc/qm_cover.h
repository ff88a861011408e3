// qm_cover.h -- overlapping communities (covers): workspace and launchers of
// qm_cover.cu, used by the C ABI in qm_api.cu.
//
// A cover is a family of node sets in which a node may belong to several
// communities or to none, given node by node (the communities of node u are
// memb[mptr[u] .. mptr[u+1]), strictly increasing ids in [0, K)).  The metrics
// read the paper's set formulas literally (|c|, edges inside c, edges leaving
// c, edges leaving c_i and entering c_j, |c n c'|, pairs sharing a community);
// include/qm.h states the reading.
#pragma once

#include "qm_internal.h"

namespace qm {

// One cover, brought to the graph's stored node order with int offsets.
struct CoverSide {
    int *off;    // [n + 1] offsets of each node's list (stored order)
    int *memb;   // [m] community ids
    int *len;    // [n + 1] scratch: list lengths before the scan
    int *size;   // [K] members of each community (zeroed)
    int *cstart; // [K + 1] offsets of each community's member list
    int *cur;    // [K] scatter cursors (zeroed)
    int *cmem;   // [m] members of each community, community by community
    int K;
};

struct CoverWs {
    int *status;               // bit 0: a malformed list or an id out of range; bit 1: too many distinct keys
    int *counters;             // claim counters and scan counters (zeroed)
    unsigned long long *gacc;  // accumulators (GS_* or GC_* words) and the pair corrections (zeroed)
    void *result;              // qm_quality or qm_compare
    CoverSide a, b;            // scoring uses a only
    qmk::Rcp *recip;           // [K] scoring: rcp_of(|c|)
    unsigned *rowmax;          // [ka] comparison: largest cell of each truth community
    unsigned long long *rowbest; // [ka] comparison: largest F ratio of each row (as double bits)
    unsigned *colmax;          // [kb] comparison: largest cell of each found community (zeroed)
    int *scan_tmp;
    size_t zero_bytes;
    size_t bytes;
};

// Scratch of a cover scoring call (n nodes, m memberships, K ids) and of a
// comparison of two covers (ma, mb memberships; ka, kb ids).
size_t cover_score_ws_bytes(long long n, long long m, int K);
CoverWs carve_cover_score_ws(void *base, long long n, long long m, int K);
size_t cover_compare_ws_bytes(long long n, long long ma, int ka, long long mb, int kb);
CoverWs carve_cover_compare_ws(void *base, long long n, long long ma, int ka, long long mb, int kb);

// Launchers (stream-ordered; the workspace's zero_bytes must be zeroed first).
// mptr: int64[n + 1] and memb: int32[m] on the device, in the caller's node
// order; inv: the graph's new id -> caller id map (QM_REORDER) or null.
// Each returns the number of kernels launched, or -1 on a launch error.
int launch_cover_score(const GraphDev &g, const long long *mptr, const int *memb, long long m, int K,
                       const CoverWs &w, int num_sms, cudaStream_t s);
int launch_cover_compare(const long long *aptr, const int *amemb, long long ma, int ka, const long long *bptr,
                         const int *bmemb, long long mb, int kb, long long n, const CoverWs &w, int num_sms,
                         cudaStream_t s);

// Once per device, before any launch or capture.
void prepare_cover_kernels();

}  // namespace qm
