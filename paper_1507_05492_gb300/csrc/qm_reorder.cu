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
// loaded, and each scoring call brings its labels into the stored order (a
// gather through the permutation, or on large graphs the two passes through
// shared memory at the end of this file).
// Every metric is invariant under renumbering and summed exactly, so the
// results are bit-identical with and without the reorder.
#include <algorithm>
#include <climits>
#include <cstdint>
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

// ------------------------------------------------------------------ bucketed label permutation

// A scoring call on a renumbered graph first brings the caller's labels into
// the stored order, out[j] = labels[inv[j]].  As one gather that is a random
// 4-byte read per node from an array larger than L2, and each costs DRAM far
// more than 4 bytes.  The buckets built here do it in two passes whose global
// reads and writes are all sequential, the random part in shared memory:
//   pass 1  per tile of 2^tile_bits caller ids: the tile's labels are placed
//           in shared memory grouped by the window of 2^window_bits new ids
//           they are bound for, then each window's group is written to that
//           window's stretch of a scratch array (slots);
//   pass 2  per window: its slots are placed in shared memory at their new
//           ids, and the window is written out in order, the community sizes
//           counted on the way (labels of one cluster are adjacent then).
// Inside a (tile, window) group the order is whatever the build's atomics
// gave; both passes follow the same order, so the result does not depend on it.

constexpr int PB_BUILD_THREADS = 512;
constexpr int PB_THREADS = 1024;

__global__ void k_pb_invert(const int *__restrict__ inv, long long n, int *__restrict__ perm)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        perm[inv[j]] = (int)j;
}

// cnt[w * ntiles + t]: ids of tile t whose new id lies in window w.
__global__ void k_pb_count(const int *__restrict__ perm, long long n, int tb, int wb, int nw, int ntiles, int *cnt)
{
    extern __shared__ int c[];  // [nw]
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < nw; i += blockDim.x) c[i] = 0;
        __syncthreads();
        const long long u0 = (long long)t << tb, u1 = min(n, u0 + (1LL << tb));
        for (long long u = u0 + threadIdx.x; u < u1; u += blockDim.x) atomicAdd(&c[perm[u] >> wb], 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nw; i += blockDim.x) cnt[(long long)i * ntiles + t] = c[i];
        __syncthreads();
    }
}

// From the window-major exclusive prefix `off` (off[nw * ntiles] = n): per
// tile, toff[t][w] = first slot of group (t, w) and tlb[t][w] = its first
// position in the tile's grouped order (tlb[t][nw] = the tile's length).
__global__ void k_pb_tables(const int *__restrict__ off, int nw, int ntiles, int *toff, int *tlb)
{
    __shared__ int wsum[PB_BUILD_THREADS / 32];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (nw + T - 1) / T, w0 = min(nw, tid * per), w1 = min(nw, w0 + per);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int sum = 0;
        for (int w = w0; w < w1; ++w) {
            const long long i = (long long)w * ntiles + t;
            toff[(long long)t * nw + w] = off[i];
            sum += off[i + 1] - off[i];
        }
        int x = sum;  // inclusive scan over the block, chunk by chunk
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int v = lane < T / 32 ? wsum[lane] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += y;
            }
            if (lane < T / 32) wsum[lane] = v;
        }
        __syncthreads();
        int run = x - sum + (wid > 0 ? wsum[wid - 1] : 0);
        for (int w = w0; w < w1; ++w) {
            const long long i = (long long)w * ntiles + t;
            tlb[(long long)t * (nw + 1) + w] = run;
            run += off[i + 1] - off[i];
        }
        if (tid == T - 1) tlb[(long long)t * (nw + 1) + nw] = wsum[T / 32 - 1];
        __syncthreads();
    }
}

// Each caller id's position in its tile's grouped order (lpos) and each
// slot's new id inside its window (dloc); ranks inside a group by atomics.
__global__ void k_pb_place(const int *__restrict__ perm, long long n, int tb, int wb, int nw, int ntiles,
                           const int *__restrict__ toff, const int *__restrict__ tlb, unsigned short *lpos,
                           unsigned short *dloc)
{
    extern __shared__ int cur[];  // [nw]
    const int mask = (1 << wb) - 1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < nw; i += blockDim.x) cur[i] = 0;
        __syncthreads();
        const long long u0 = (long long)t << tb, u1 = min(n, u0 + (1LL << tb));
        for (long long u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const int j = perm[u], w = j >> wb;
            const int r = atomicAdd(&cur[w], 1);
            lpos[u] = (unsigned short)(tlb[(long long)t * (nw + 1) + w] + r);
            dloc[toff[(long long)t * nw + w] + r] = (unsigned short)(j & mask);
        }
        __syncthreads();
    }
}

// Shared memory of the passes with B bytes a label (3 while the labels are
// below 2^24, else 4).
static size_t pb_pass1_smem(int tb, int nw, int B) { return (size_t)B * ((size_t)1 << tb) + (2 * (size_t)nw + 1) * 4; }
static size_t pb_pass2_smem(int wb, int B) { return (size_t)B * ((size_t)1 << wb); }

// Whether the two passes fit with 3-byte labels: shared memory, 16-bit local
// positions, and tables of at most 2^30 entries.
static bool pb_fits(long long n, int wb, int tb, size_t smem_max, int *nw_out, int *ntiles_out)
{
    if (wb < 1 || wb > PB_MAX_BITS || tb < 1 || tb > PB_MAX_BITS) return false;
    const long long nw = (n + (1LL << wb) - 1) >> wb, ntiles = (n + (1LL << tb) - 1) >> tb;
    if (nw > PB_MAX_WINDOWS || nw * ntiles >= (1LL << 30)) return false;
    if (pb_pass1_smem(tb, (int)nw, 3) > smem_max || pb_pass2_smem(wb, 3) > smem_max) return false;
    *nw_out = (int)nw;
    *ntiles_out = (int)ntiles;
    return true;
}

template <int B, bool V4>
__global__ void k_pb_tile(const int *__restrict__ labels, const unsigned short *__restrict__ lpos,
                          const int *__restrict__ toff, const int *__restrict__ tlb, long long n, int tb, int nw,
                          int ntiles, int K, int *__restrict__ tmp, int *status);
template <int B, bool V4>
__global__ void k_pb_window(const int *__restrict__ tmp, const unsigned short *__restrict__ dloc, long long n, int wb,
                            int nw, int *__restrict__ out, int *size, int K);

template <int B, bool V4>
static cudaError_t pb_set_smem_v(size_t smem_max)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_pb_tile<B, V4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pb_window<B, V4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    return e;
}

template <int B>
static cudaError_t pb_set_smem(size_t smem_max)
{
    const cudaError_t e = pb_set_smem_v<B, false>(smem_max);
    return e == cudaSuccess ? pb_set_smem_v<B, true>(smem_max) : e;
}

int build_perm_buckets(const int *inv, long long n, int wb, int tb, int num_sms, cudaStream_t s, PermBuckets *out,
                       int *launches)
{
    int dev = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return -(int)e;
    const size_t smem_max = (size_t)smem_optin;
    int nw = 0, ntiles = 0;
    if (!pb_fits(n, wb, tb, smem_max, &nw, &ntiles)) return 1;
    const long long ncnt = (long long)nw * ntiles;
    int *perm = nullptr, *cnt = nullptr, *tmp = nullptr, *toff = nullptr, *tlb = nullptr;
    unsigned short *lpos = nullptr, *dloc = nullptr;
    auto bad = [&](cudaError_t e) {
        cudaFree(perm);
        cudaFree(cnt);
        cudaFree(tmp);
        cudaFree(toff);
        cudaFree(tlb);
        cudaFree(lpos);
        cudaFree(dloc);
        return e == cudaSuccess ? (int)cudaErrorUnknown : (int)e;
    };
    const size_t tmp_elems = scan_tmp_elems(ncnt + 1) + 64;
    if ((e = cudaMalloc(&perm, (size_t)n * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&cnt, (size_t)(ncnt + 1) * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&tmp, tmp_elems * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&toff, (size_t)ncnt * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&tlb, (size_t)ntiles * (nw + 1) * 4)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&lpos, (size_t)n * 2)) != cudaSuccess) return -bad(e);
    if ((e = cudaMalloc(&dloc, (size_t)n * 2)) != cudaSuccess) return -bad(e);
    if ((e = cudaMemsetAsync(tmp, 0, tmp_elems * 4, s)) != cudaSuccess) return -bad(e);
    if ((e = pb_set_smem<3>(smem_max)) != cudaSuccess || (e = pb_set_smem<4>(smem_max)) != cudaSuccess)
        return -bad(e);
    int L = 0;
    k_pb_invert<<<grid_of(n, 512, num_sms, 8), 512, 0, s>>>(inv, n, perm);
    const int gt = std::min(ntiles, num_sms * 4);
    k_pb_count<<<gt, PB_BUILD_THREADS, (size_t)nw * 4, s>>>(perm, n, tb, wb, nw, ntiles, cnt);
    L += 2;
    int *status = tmp + tmp_elems - 32, *counters = tmp + tmp_elems - 16;
    const int l2 = scan_offsets(cnt, (int)ncnt, cnt, tmp, counters, status, s);
    if (l2 < 0) return -bad(cudaGetLastError());
    L += l2;
    k_pb_tables<<<gt, PB_BUILD_THREADS, 0, s>>>(cnt, nw, ntiles, toff, tlb);
    k_pb_place<<<gt, PB_BUILD_THREADS, (size_t)nw * 4, s>>>(perm, n, tb, wb, nw, ntiles, toff, tlb, lpos, dloc);
    L += 2;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return -bad(e);
    if ((e = cudaGetLastError()) != cudaSuccess) return -bad(e);
    cudaFree(perm);
    cudaFree(cnt);
    cudaFree(tmp);
    out->lpos = lpos;
    out->dloc = dloc;
    out->toff = toff;
    out->tlb = tlb;
    out->wb = wb;
    out->tb = tb;
    out->nw = nw;
    out->ntiles = ntiles;
    out->smem_max = smem_max;
    out->bytes = (size_t)n * 4 + (size_t)ncnt * 4 + (size_t)ntiles * (nw + 1) * 4;
    if (launches) *launches = L;
    return 0;
}

void free_perm_buckets(PermBuckets *pb)
{
    cudaFree(pb->lpos);
    cudaFree(pb->dloc);
    cudaFree(pb->toff);
    cudaFree(pb->tlb);
    *pb = PermBuckets{};
}

constexpr int PB_UNROLL = 4;

// A label in shared memory at position p, B bytes wide (little-endian; with
// B = 3 the labels are known to lie in [0, 2^24)).
template <int B>
__device__ __forceinline__ void pb_put(unsigned char *m, int p, int v)
{
    if (B == 4) {
        ((int *)m)[p] = v;
    } else {
        unsigned char *q = m + 3 * p;
        q[0] = (unsigned char)v;
        q[1] = (unsigned char)(v >> 8);
        q[2] = (unsigned char)(v >> 16);
    }
}

template <int B>
__device__ __forceinline__ int pb_get(const unsigned char *m, int p)
{
    if (B == 4) return ((const int *)m)[p];
    const unsigned char *q = m + 3 * p;
    return (int)q[0] | ((int)q[1] << 8) | ((int)q[2] << 16);
}

// Values v[0 .. len) into shared memory at positions pos[0 .. len), each
// checked against [0, K) (bad).  With V4, v and pos are 16- and 8-byte
// aligned and move four at a time, two groups in flight per thread.
template <int B, bool V4>
__device__ __forceinline__ void pb_stage(const int *__restrict__ v, const unsigned short *__restrict__ pos, int len,
                                         unsigned char *m, int K, bool &bad)
{
    const int T = blockDim.x, tid = threadIdx.x;
    int i = 0;
    if (V4) {
        const int ng = len >> 2;
        for (int g0 = 0; g0 < ng; g0 += 2 * T) {
            int4 x[2];
            ushort4 p[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int g = g0 + q * T + tid;
                if (g < ng) {
                    x[q] = __ldcs((const int4 *)v + g);
                    p[q] = __ldcs((const ushort4 *)pos + g);
                }
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (g0 + q * T + tid < ng) {
                    if ((unsigned)x[q].x >= (unsigned)K || (unsigned)x[q].y >= (unsigned)K ||
                        (unsigned)x[q].z >= (unsigned)K || (unsigned)x[q].w >= (unsigned)K)
                        bad = true;
                    pb_put<B>(m, p[q].x, x[q].x);
                    pb_put<B>(m, p[q].y, x[q].y);
                    pb_put<B>(m, p[q].z, x[q].z);
                    pb_put<B>(m, p[q].w, x[q].w);
                }
        }
        i = ng << 2;
    }
    for (int i0 = i; i0 < len; i0 += T * PB_UNROLL) {
        int x[PB_UNROLL], p[PB_UNROLL];
#pragma unroll
        for (int q = 0; q < PB_UNROLL; ++q) {
            const int k = i0 + q * T + tid;
            p[q] = k < len ? (int)__ldcs(&pos[k]) : -1;
            x[q] = k < len ? __ldcs(&v[k]) : 0;
        }
#pragma unroll
        for (int q = 0; q < PB_UNROLL; ++q)
            if (p[q] >= 0) {
                if ((unsigned)x[q] >= (unsigned)K) bad = true;
                pb_put<B>(m, p[q], x[q]);
            }
    }
}

// Pass 1, one tile per block step: labels into shared memory at their grouped
// positions (checked against [0, K): bit 0 of *status), then every (tile,
// window) group to its slots, a warp per group.
template <int B, bool V4>
__global__ void __launch_bounds__(PB_THREADS, 2) k_pb_tile(const int *__restrict__ labels,
                                                        const unsigned short *__restrict__ lpos,
                                                        const int *__restrict__ toff, const int *__restrict__ tlb,
                                                        long long n, int tb, int nw, int ntiles, int K,
                                                        int *__restrict__ tmp, int *status)
{
    extern __shared__ __align__(16) unsigned char smb[];
    int *lb = (int *)smb, *of = lb + nw + 1;
    unsigned char *sv = (unsigned char *)(of + nw);
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, W = T >> 5;
    bool bad = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long u0 = (long long)t << tb;
        const int len = (int)min(n - u0, 1LL << tb);
        for (int w = tid; w <= nw; w += T) lb[w] = tlb[(long long)t * (nw + 1) + w];
        for (int w = tid; w < nw; w += T) of[w] = toff[(long long)t * nw + w];
        pb_stage<B, V4>(labels + u0, lpos + u0, len, sv, K, bad);
        __syncthreads();
        for (int w = wid; w < nw; w += W) {
            const int b = lb[w], e = lb[w + 1], o = of[w];
            for (int k = b + lane; k < e; k += 32) tmp[o + (k - b)] = pb_get<B>(sv, k);
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, 1);
}

// Pass 2, one window per block step: slots into shared memory at their new
// ids, then the window out in order.  With `size`, the labels are counted as
// k_hist does (pass 1 has checked them).
template <int B, bool V4>
__global__ void __launch_bounds__(PB_THREADS, 2) k_pb_window(const int *__restrict__ tmp,
                                                          const unsigned short *__restrict__ dloc, long long n,
                                                          int wb, int nw, int *__restrict__ out, int *size, int K)
{
    extern __shared__ __align__(16) unsigned char smb[];
    const int T = blockDim.x, tid = threadIdx.x;
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const long long base = (long long)w << wb;
        const int len = (int)min(n - base, 1LL << wb);
        bool unused = false;
        pb_stage<B, V4>(tmp + base, dloc + base, len, smb, INT_MAX, unused);
        __syncthreads();
        for (int i = tid; i - (tid & 31) < len; i += T) {  // warp-uniform trip count
            const bool in = i < len;
            const int l = in ? pb_get<B>(smb, i) : 0;
            if (in) out[base + i] = l;
            if (size) {
                const bool ok = in && (unsigned)l < (unsigned)K;
                const unsigned act = __ballot_sync(0xffffffffu, ok);
                if (ok) {
                    const unsigned peers = __match_any_sync(act, l);
                    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&size[l], __popc(peers));
                }
            }
        }
        __syncthreads();
    }
}

int launch_permute_buckets(const int *labels, const PermBuckets &pb, long long n, int *tmp, int *out, int *size,
                           int K, int *status, int num_sms, cudaStream_t s, void (*tr)(const char *, cudaStream_t))
{
    const bool narrow = K <= (1 << 24);
    const int B = narrow ? 3 : 4;
    const size_t p1 = pb_pass1_smem(pb.tb, pb.nw, B), p2 = pb_pass2_smem(pb.wb, B);
    if (p1 > pb.smem_max || p2 > pb.smem_max) return 0;  // 4-byte labels do not fit: gather them instead
    // resident blocks per SM: two of PB_THREADS at most, and what shared memory allows
    auto per_sm = [](size_t smem) { return (int)std::max<size_t>(1, std::min<size_t>(2, 233472 / (smem + 1024))); };
    const int g1 = std::min(pb.ntiles, num_sms * per_sm(p1)), g2 = std::min(pb.nw, num_sms * per_sm(p2));
    // four at a time where every tile (window) start keeps the 16-byte alignment
    const bool v1 = pb.tb >= 2 && ((uintptr_t)labels & 15) == 0, v2 = pb.wb >= 2;
    auto pass1 = [&](auto kern) {
        kern<<<g1, PB_THREADS, p1, s>>>(labels, pb.lpos, pb.toff, pb.tlb, n, pb.tb, pb.nw, pb.ntiles, K, tmp, status);
    };
    auto pass2 = [&](auto kern) { kern<<<g2, PB_THREADS, p2, s>>>(tmp, pb.dloc, n, pb.wb, pb.nw, out, size, K); };
    if (tr) tr("k_pb_tile", s);
    if (narrow)
        v1 ? pass1(k_pb_tile<3, true>) : pass1(k_pb_tile<3, false>);
    else
        v1 ? pass1(k_pb_tile<4, true>) : pass1(k_pb_tile<4, false>);
    if (tr) tr("k_pb_window", s);
    if (narrow)
        v2 ? pass2(k_pb_window<3, true>) : pass2(k_pb_window<3, false>);
    else
        v2 ? pass2(k_pb_window<4, true>) : pass2(k_pb_window<4, false>);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

}  // namespace qm
