// qm_reorder.cu -- optional locality reorder of a loaded graph (QM_REORDER).
//
// Scoring gathers the label of every arc's far end.  With node ids in random
// order (as in the LFR benchmark graphs of Sec. IV-C, and in many real edge
// lists) those gathers land anywhere in the label array, which at 10^8 nodes
// is three times the L2 cache.  A partition worth scoring follows the graph's
// community structure, so renumbering the nodes cluster by cluster makes most
// of the gathered labels neighbours in memory.  The clusters come from the
// graph alone (a few synchronous label-propagation rounds, never from a
// partition being scored), the renumbering is done once when the graph is
// loaded, and each scoring call gathers its labels through the permutation.
// Every metric is invariant under renumbering and summed exactly, so the
// results are bit-identical with and without the reorder.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "qm_internal.h"
#include "qm_device.cuh"

namespace qm {

using namespace qmk;

// Labels start as the node ids.
__global__ void k_lpa_init(int *lab, long long n)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        lab[u] = (int)u;
}

// One synchronous label-propagation round, one warp per node: the node takes
// the label found most often among (an evenly spaced sample of up to 32 of)
// its neighbours, keeps its own label when that is among the most frequent,
// and otherwise takes the smallest of the tied labels.
__global__ void k_lpa_round(const long long *__restrict__ row_ptr, const int *__restrict__ col, long long n,
                            const int *__restrict__ cur, int *__restrict__ nxt)
{
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const long long rs = __ldg(&row_ptr[u]);
        const long long deg = __ldg(&row_ptr[u + 1]) - rs;
        const int own = __ldg(&cur[u]);
        int lab = -1;
        if (lane < deg) {
            const long long j = deg <= 32 ? lane : (long long)lane * deg / 32;
            lab = __ldg(&cur[__ldg(&col[rs + j])]);
        }
        const unsigned valid = __ballot_sync(0xffffffffu, lab >= 0);
        const unsigned peers = __match_any_sync(0xffffffffu, lab) & valid;
        unsigned long long score = 0ull;
        if (lab >= 0)
            score = ((unsigned long long)__popc(peers) << 33) | ((unsigned long long)(lab == own) << 32) |
                    (unsigned long long)(0xFFFFFFFFu - (unsigned)lab);
        for (int d = 16; d > 0; d >>= 1) score = max(score, __shfl_xor_sync(0xffffffffu, score, d));
        if (lane == 0) nxt[u] = valid ? (int)(0xFFFFFFFFu - (unsigned)(score & 0xFFFFFFFFull)) : own;
    }
}

__global__ void k_count_ids(const int *__restrict__ lab, long long n, int *hist)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        atomicAdd(&hist[lab[u]], 1);
}

// New position of every node: its cluster's offset plus a slot taken in the
// cluster (the order inside a cluster is whatever the atomics give).
__global__ void k_place(const int *__restrict__ lab, long long n, int *cursor, int *inv, int *perm)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&cursor[lab[u]], 1);
        inv[pos] = (int)u;
        perm[u] = pos;
    }
}

__global__ void k_new_degrees(const long long *__restrict__ row_ptr, const int *__restrict__ inv, long long n,
                              int *deg)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int u = inv[j];
        deg[j] = (int)(row_ptr[u + 1] - row_ptr[u]);
    }
}

// 32-bit offsets (sum below 2^32) to the 64-bit row_ptr.
__global__ void k_widen(const unsigned *__restrict__ off, long long n, long long *row_ptr)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += (long long)gridDim.x * blockDim.x)
        row_ptr[j] = (long long)off[j];
}

// Row j of the new CSR is row inv[j] of the old one with every neighbour
// renamed (and its weights, on a weighted graph); one warp per row.
__global__ void k_fill_rows(const long long *__restrict__ row_ptr, const int *__restrict__ col,
                            const int *__restrict__ inv, const int *__restrict__ perm, long long n,
                            const long long *__restrict__ row_ptr2, int *__restrict__ col2,
                            const float *__restrict__ wt, float *__restrict__ wt2)
{
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nw) {
        const int u = __ldg(&inv[j]);
        const long long rs = __ldg(&row_ptr[u]), deg = __ldg(&row_ptr[u + 1]) - rs;
        const long long ws = __ldg(&row_ptr2[j]);
        for (long long e = lane; e < deg; e += 32) {
            col2[ws + e] = __ldg(&perm[__ldg(&col[rs + e])]);
            if (wt) wt2[ws + e] = __ldg(&wt[rs + e]);
        }
    }
}

// out[p][j] = labels[p][inv[j]] for P rows of n labels.
__global__ void k_permute_labels(const int *__restrict__ labels, const int *__restrict__ inv, long long n, int P,
                                 int *__restrict__ out)
{
    const long long total = n * (long long)P;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / n, j = i - p * n;
        out[i] = __ldg(&labels[p * n + __ldg(&inv[j])]);
    }
}

// Label propagation as a detector (qm_label_propagation): labels start as the
// caller's node ids, so a renumbered graph gives the same partition.
__global__ void k_lpa_init_ids(int *lab, const int *__restrict__ inv, long long n)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        lab[u] = inv ? inv[u] : (int)u;
}

// flag[c] = 1 when some node carries label c (c in [0, n)).
__global__ void k_present(int *hist, long long n)
{
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        hist[c] = hist[c] > 0 ? 1 : 0;
}

// out[caller id] = rank of the node's final label among the labels present.
__global__ void k_write_ranks(const int *__restrict__ lab, const int *__restrict__ rank, const int *__restrict__ inv,
                              long long n, int *__restrict__ out)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        out[inv ? inv[j] : j] = rank[lab[j]];
}

static int grid_of(long long work, int threads, int num_sms, int per_sm)
{
    long long g = (work + threads - 1) / threads;
    const long long cap = (long long)num_sms * per_sm;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

int launch_permute_labels(const int *labels, const int *inv, long long n, int P, int *out, int num_sms,
                          cudaStream_t s)
{
    k_permute_labels<<<grid_of(n * (long long)P, 512, num_sms, 8), 512, 0, s>>>(labels, inv, n, P, out);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_label_propagation(const GraphDev &g, int rounds, int num_sms, cudaStream_t s, int *lab0, int *lab1,
                             int *hist, int *tmp, size_t tmp_elems, int *out)
{
    const long long n = g.n;
    const int g1 = grid_of(n, 512, num_sms, 8), gw = grid_of(n * 32, 256, num_sms, 8);
    int L = 0;
    k_lpa_init_ids<<<g1, 512, 0, s>>>(lab0, g.inv, n);
    ++L;
    for (int r = 0; r < rounds; ++r) {
        k_lpa_round<<<gw, 256, 0, s>>>(g.row_ptr, g.col, n, lab0, lab1);
        std::swap(lab0, lab1);
        ++L;
    }
    if (cudaMemsetAsync(hist, 0, (size_t)(n + 1) * 4, s) != cudaSuccess) return -1;
    if (cudaMemsetAsync(tmp, 0, tmp_elems * 4, s) != cudaSuccess) return -1;
    k_count_ids<<<g1, 512, 0, s>>>(lab0, n, hist);
    k_present<<<g1, 512, 0, s>>>(hist, n);
    L += 2;
    int *status = tmp + tmp_elems - 32, *counters = tmp + tmp_elems - 16;
    const int l2 = scan_offsets(hist, (int)n, hist, tmp, counters, status, s);  // hist[n] = number of labels
    if (l2 < 0) return -1;
    L += l2;
    k_write_ranks<<<g1, 512, 0, s>>>(lab0, hist, g.inv, n, out);
    ++L;
    return cudaGetLastError() == cudaSuccess ? L : -1;
}

int reorder_graph(const GraphDev &g, int rounds, int num_sms, cudaStream_t s, long long **row_ptr_out, int **col_out,
                  int **inv_out, int *launches, float **wt_out)
{
    const long long n = g.n;
    int *lab0 = nullptr, *lab1 = nullptr, *hist = nullptr, *perm = nullptr, *inv = nullptr, *tmp = nullptr;
    long long *row2 = nullptr;
    int *col2 = nullptr;
    float *wt2 = nullptr;
    int L = 0;
    auto bad = [&](cudaError_t e) {
        cudaFree(lab0);
        cudaFree(lab1);
        cudaFree(hist);
        cudaFree(perm);
        cudaFree(inv);
        cudaFree(tmp);
        cudaFree(row2);
        cudaFree(col2);
        cudaFree(wt2);
        return e == cudaSuccess ? (int)cudaErrorUnknown : (int)e;
    };
    cudaError_t e = cudaSuccess;
    const size_t tmp_elems = scan_tmp_elems(n + 1) + 64;
    if ((e = cudaMalloc(&lab0, (size_t)n * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&lab1, (size_t)n * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&hist, (size_t)(n + 1) * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&perm, (size_t)n * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&inv, (size_t)n * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&tmp, tmp_elems * 4)) != cudaSuccess) return -bad(e);
    const int g1 = grid_of(n, 512, num_sms, 8), gw = grid_of(n * 32, 256, num_sms, 8);
    k_lpa_init<<<g1, 512, 0, s>>>(lab0, n);
    ++L;
    for (int r = 0; r < rounds; ++r) {
        k_lpa_round<<<gw, 256, 0, s>>>(g.row_ptr, g.col, n, lab0, lab1);
        std::swap(lab0, lab1);
        ++L;
    }
    // cluster offsets: hist -> exclusive scan (in place, n + 1 entries) -> cursor
    if ((e = cudaMemsetAsync(hist, 0, (size_t)(n + 1) * 4, s)) != cudaSuccess) return -bad(e);
    if ((e = cudaMemsetAsync(tmp, 0, tmp_elems * 4, s)) != cudaSuccess) return -bad(e);
    k_count_ids<<<g1, 512, 0, s>>>(lab0, n, hist);
    ++L;
    int *status = tmp + tmp_elems - 32, *counters = tmp + tmp_elems - 16;
    int l2 = scan_offsets(hist, (int)n, hist, tmp, counters, status, s);
    if (l2 < 0) return -bad(cudaGetLastError());
    L += l2;
    k_place<<<g1, 512, 0, s>>>(lab0, n, hist, inv, perm);
    ++L;
    // new row offsets from the degrees in the new order (lab1 is free: reuse it)
    k_new_degrees<<<g1, 512, 0, s>>>(g.row_ptr, inv, n, lab1);
    ++L;
    l2 = scan_offsets(lab1, (int)n, hist, tmp, counters, status, s);
    if (l2 < 0) return -bad(cudaGetLastError());
    L += l2;
    if ((e = cudaMalloc(&row2, (size_t)(n + 1) * 8)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&col2, (size_t)g.n_arcs * 4)) != cudaSuccess) return -bad(e);
    if (g.wt && (e = cudaMalloc(&wt2, (size_t)g.n_arcs * 4)) != cudaSuccess) return -bad(e);
    k_widen<<<g1, 512, 0, s>>>((const unsigned *)hist, n, row2);
    k_fill_rows<<<gw, 256, 0, s>>>(g.row_ptr, g.col, inv, perm, n, row2, col2, g.wt, wt2);
    L += 2;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return -bad(e);
    if ((e = cudaGetLastError()) != cudaSuccess) return -bad(e);
    cudaFree(lab0);
    cudaFree(lab1);
    cudaFree(hist);
    cudaFree(perm);
    cudaFree(tmp);
    *row_ptr_out = row2;
    *col_out = col2;
    *inv_out = inv;
    if (wt_out) *wt_out = wt2;
    if (launches) *launches = L;
    return 0;
}

// ------------------------------------------------------------------ upper rows

// Arcs of node u to itself or to higher ids, one warp per row.
__global__ void k_up_degrees(const long long *__restrict__ row_ptr, const int *__restrict__ col, long long n,
                             int *deg)
{
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const long long rs = __ldg(&row_ptr[u]), re = __ldg(&row_ptr[u + 1]);
        int cnt = 0;
        for (long long e = rs + lane; e < re; e += 32) cnt += __ldg(&col[e]) >= u ? 1 : 0;
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) deg[u] = cnt;
    }
}

// Copies those arcs in row order, a self-loop as ~u; one warp per row.
__global__ void k_up_fill(const long long *__restrict__ row_ptr, const int *__restrict__ col, long long n,
                          const long long *__restrict__ up_ptr, int *__restrict__ up_col)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const long long rs = __ldg(&row_ptr[u]), re = __ldg(&row_ptr[u + 1]);
        long long at = __ldg(&up_ptr[u]);
        for (long long e0 = rs; e0 < re; e0 += 32) {
            const long long e = e0 + lane;
            const int v = e < re ? __ldg(&col[e]) : -1;
            const bool keep = e < re && v >= u;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) up_col[at + __popc(m & lt)] = v == u ? ~v : v;
            at += __popc(m);
        }
    }
}

int build_upper_rows(const GraphDev &g, int num_sms, cudaStream_t s, long long **up_ptr_out, int **up_col_out,
                     long long *up_arcs, int *launches)
{
    const long long n = g.n;
    int *deg = nullptr, *tmp = nullptr;
    long long *up_ptr = nullptr;
    int *up_col = nullptr;
    unsigned *total_h = nullptr;
    auto bad = [&](cudaError_t e) {
        cudaFree(deg);
        cudaFree(tmp);
        cudaFree(up_ptr);
        cudaFree(up_col);
        cudaFreeHost(total_h);
        return e == cudaSuccess ? (int)cudaErrorUnknown : (int)e;
    };
    if (g.n_arcs >= (1LL << 32)) return -bad(cudaErrorInvalidValue);
    cudaError_t e = cudaSuccess;
    int L = 0;
    const size_t tmp_elems = scan_tmp_elems(n + 1) + 64;
    if ((e = cudaMalloc(&deg, (size_t)(n + 1) * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&tmp, tmp_elems * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&up_ptr, (size_t)(n + 1) * 8)) != cudaSuccess) return -bad(e);
    if ((e = cudaMallocHost(&total_h, 16)) != cudaSuccess) return -bad(e);
    if ((e = cudaMemsetAsync(tmp, 0, tmp_elems * 4, s)) != cudaSuccess) return -bad(e);
    const int g1 = grid_of(n, 512, num_sms, 8), gw = grid_of(n * 32, 256, num_sms, 8);
    k_up_degrees<<<gw, 256, 0, s>>>(g.row_ptr, g.col, n, deg);
    ++L;
    int *status = tmp + tmp_elems - 32, *counters = tmp + tmp_elems - 16;
    const int l2 = scan_offsets(deg, (int)n, deg, tmp, counters, status, s);  // deg[n] = total
    if (l2 < 0) return -bad(cudaGetLastError());
    L += l2;
    k_widen<<<g1, 512, 0, s>>>((const unsigned *)deg, n, up_ptr);
    ++L;
    if ((e = cudaMemcpyAsync(total_h, deg + n, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return -bad(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return -bad(e);
    const long long total = (long long)total_h[0];
    if ((e = cudaMalloc(&up_col, (size_t)std::max(total, 1LL) * 4)) != cudaSuccess) return -bad(e);
    k_up_fill<<<gw, 256, 0, s>>>(g.row_ptr, g.col, n, up_ptr, up_col);
    ++L;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return -bad(e);
    if ((e = cudaGetLastError()) != cudaSuccess) return -bad(e);
    cudaFree(deg);
    cudaFree(tmp);
    cudaFreeHost(total_h);
    *up_ptr_out = up_ptr;
    *up_col_out = up_col;
    if (up_arcs) *up_arcs = total;
    if (launches) *launches = L;
    return 0;
}

}  // namespace qm
