// qm_api.cu -- host runtime behind the C ABI of include/qm.h: graph residency,
// a scratch-memory pool, launch shapes and their autotuner, and the CUDA graphs
// that replay the batched persistent launch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "qm_internal.h"
#include "qm_batched.h"
#include "qm_cover.h"

using namespace qm;

// ------------------------------------------------------------------ errors

static thread_local std::string t_err;
static std::atomic<long long> g_launches{0};

static qm_status fail(qm_status s, const std::string &msg)
{
    t_err = msg;
    return s;
}

static qm_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? QM_ENOMEM : QM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// ------------------------------------------------------------------ tracing

// Per-thread kernel timing.  When enabled, the launchers call trace_mark()
// before each kernel and once after the last one; an event is recorded on the
// launching stream at each mark, so kernel i took event[i+1] - event[i].
struct TraceState {
    bool on = false;
    std::vector<std::string> names;
    std::vector<cudaEvent_t> events;
    size_t used = 0;
    std::vector<std::pair<std::string, float>> last;
};
static thread_local TraceState t_trace;

static void trace_mark(const char *name, cudaStream_t s)
{
    TraceState &t = t_trace;
    if (t.used == t.events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        t.events.push_back(e);
    }
    cudaEventRecord(t.events[t.used], s);
    t.names.resize(t.used + 1);
    t.names[t.used] = name ? name : "";
    ++t.used;
}

static TraceFn trace_begin()
{
    if (!t_trace.on) return nullptr;
    t_trace.used = 0;
    return trace_mark;
}

// After the call's stream synchronisation: turn the marks into durations.
static void trace_collect()
{
    TraceState &t = t_trace;
    if (!t.on) return;
    t.last.clear();
    for (size_t i = 0; i + 1 < t.used; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.events[i], t.events[i + 1]);
        t.last.emplace_back(t.names[i], ms);
    }
    t.used = 0;
}

qm_status qm::set_error(qm_status s, const char *msg)
{
    return fail(s, msg ? msg : "");
}

// ------------------------------------------------------------------ device info

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Also performs the once-per-device kernel set-up (shared-memory limits), so
// every path that launches work calls it first.
static int num_sms_of(int dev)
{
    static std::mutex mu;
    static std::map<int, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    prepare_kernels();
    prepare_batched_kernel();
    prepare_cover_kernels();
    if (prev != dev) cudaSetDevice(prev);
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v < 1) v = 1;
    cache[dev] = v;
    return v;
}

// ------------------------------------------------------------------ memory pool

// Scratch buffers are allocated on first need and reused by later calls; a call
// leases a block exclusively until it returns, so concurrent calls never share
// scratch.
struct PoolBlock {
    void *ptr;
    size_t bytes;
    int device;
    bool pinned;
    bool busy;
};

class Pool {
  public:
    PoolBlock *acquire(size_t bytes, int device, bool pinned)
    {
        std::lock_guard<std::mutex> lk(mu_);
        PoolBlock *best = nullptr;
        for (auto &b : blocks_) {
            if (b->busy || b->device != device || b->pinned != pinned || b->bytes < bytes) continue;
            if (!best || b->bytes < best->bytes) best = b.get();
        }
        if (best) {
            best->busy = true;
            return best;
        }
        const size_t gran = pinned ? 4096 : (1u << 20);
        size_t sz = (bytes + gran - 1) / gran * gran;
        if (sz == 0) sz = gran;
        void *p = nullptr;
        cudaError_t e = pinned ? cudaMallocHost(&p, sz) : cudaMalloc(&p, sz);
        if (e != cudaSuccess) {
            cudaGetLastError();
            trim_locked(device, pinned);
            e = pinned ? cudaMallocHost(&p, sz) : cudaMalloc(&p, sz);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
        }
        blocks_.emplace_back(new PoolBlock{p, sz, device, pinned, true});
        return blocks_.back().get();
    }
    void release(PoolBlock *b)
    {
        if (!b) return;
        std::lock_guard<std::mutex> lk(mu_);
        b->busy = false;
    }
    void trim()
    {
        std::lock_guard<std::mutex> lk(mu_);
        trim_locked(-1, false);
        trim_locked(-1, true);
    }

  private:
    void trim_locked(int device, bool pinned)
    {
        std::vector<std::unique_ptr<PoolBlock>> keep;
        for (auto &b : blocks_) {
            if (!b->busy && b->pinned == pinned && (device < 0 || b->device == device)) {
                int prev = -1;
                cudaGetDevice(&prev);
                if (!pinned) cudaSetDevice(b->device);
                if (pinned) cudaFreeHost(b->ptr); else cudaFree(b->ptr);
                if (!pinned) cudaSetDevice(prev);
                on_free(b.get());
            } else {
                keep.push_back(std::move(b));
            }
        }
        blocks_.swap(keep);
    }
    void on_free(PoolBlock *b);
    std::mutex mu_;
    std::vector<std::unique_ptr<PoolBlock>> blocks_;
};

static Pool g_pool;

struct Lease {
    PoolBlock *b = nullptr;
    Lease() = default;
    explicit Lease(PoolBlock *x) : b(x) {}
    ~Lease() { g_pool.release(b); }
    Lease(const Lease &) = delete;
    Lease &operator=(const Lease &) = delete;
    char *ptr() const { return (char *)b->ptr; }
};

// ------------------------------------------------------------------ batched graph cache

// A captured CUDA graph of one batched launch, valid for the scratch blocks it
// was captured with.  Keyed by (device block, pinned block, shape of the call).
struct GraphKey {
    const void *dev, *pin;
    int count, slots, threads, smem, big;
    long long n_max;
    int k_max, kt_max;
    long long extra = 0;  // two-phase batched graphs: node count of the log table
    bool operator<(const GraphKey &o) const
    {
        return std::tie(dev, pin, count, slots, threads, smem, big, n_max, k_max, kt_max, extra) <
               std::tie(o.dev, o.pin, o.count, o.slots, o.threads, o.smem, o.big, o.n_max, o.k_max, o.kt_max,
                        o.extra);
    }
};

static std::mutex g_graph_mu;
static std::map<GraphKey, cudaGraphExec_t> g_graphs;
static std::atomic<int> g_batch_wave{0};  // qm_debug_set_batch_wave: wave size cap of the batched pipeline

// Renumbered graphs of more than PB_MIN_NODES nodes permute the caller's labels
// in two passes through shared memory (PermBuckets): tiles of 2^16 caller ids
// and windows of 2^16 new ids (up to 4479 windows fit the shared memory of
// pass 1), else tiles of 2^15, then 2^14.  Below that size the label array
// mostly stays in L2 and the plain gather is cheaper.  A test may set the
// sizes (qm_debug_set_perm_buckets; 0 = automatic).
constexpr long long PB_MIN_NODES = 1LL << 24;
static std::atomic<int> g_pb_wb{0};
static std::atomic<int> g_pb_tb{0};
static std::atomic<long long> g_pb_min_nodes{PB_MIN_NODES};

// A captured CUDA graph of one plain scoring call on a small graph (see
// score_impl), valid for the scratch blocks and the graph it was captured with.
struct PlainKey {
    const void *dev, *pin;
    const qm_graph *g;
    int K, threads, smem, big, algo, shard_r, shard_p, partial;
    bool operator<(const PlainKey &o) const
    {
        return std::tie(dev, pin, g, K, threads, smem, big, algo, shard_r, shard_p, partial) <
               std::tie(o.dev, o.pin, o.g, o.K, o.threads, o.smem, o.big, o.algo, o.shard_r, o.shard_p, o.partial);
    }
};
struct PlainGraph {
    cudaGraphExec_t exec;
    int launches;
};
static std::map<PlainKey, PlainGraph> g_plain_graphs;

void Pool::on_free(PoolBlock *b)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        if (it->first.dev == b->ptr || it->first.pin == b->ptr) {
            cudaGraphExecDestroy(it->second);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
    for (auto it = g_plain_graphs.begin(); it != g_plain_graphs.end();) {
        if (it->first.dev == b->ptr || it->first.pin == b->ptr) {
            cudaGraphExecDestroy(it->second.exec);
            it = g_plain_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

// Drops the captured plain-call graphs of a graph that is being freed.
static void drop_plain_graphs(const qm_graph *g)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_plain_graphs.begin(); it != g_plain_graphs.end();) {
        if (it->first.g == g) {
            cudaGraphExecDestroy(it->second.exec);
            it = g_plain_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

// A stream to capture graphs on, one per calling thread and device (captures
// of concurrent calls must not share a stream).
struct CaptureStreams {
    std::map<int, cudaStream_t> by_device;
    ~CaptureStreams()
    {
        for (auto &kv : by_device) cudaStreamDestroy(kv.second);  // errors at process exit are ignored
    }
};

static cudaStream_t capture_stream(int dev)
{
    static thread_local CaptureStreams streams;
    auto it = streams.by_device.find(dev);
    if (it != streams.by_device.end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    streams.by_device[dev] = s;
    return s;
}

// ------------------------------------------------------------------ graph handle

struct qm_graph {
    int device;
    GraphDev d;
    long long *row_ptr;
    int *col;
    int *inv = nullptr;  // QM_REORDER: new node id -> caller's node id (else null)
    float *wt = nullptr; // weighted graph: edge weights parallel to col (else null)
    long long *up_ptr = nullptr;  // unweighted graphs: upper rows (GraphDev::up_ptr)
    int *up_col = nullptr;
    PermBuckets pb;               // QM_REORDER on large graphs: the labels' two-pass permutation
    long long n, n_arcs, max_degree;
    size_t bytes;
    std::mutex mu;
    std::map<int, Shape> tuning;        // plain path, by size bucket
    std::map<int, Shape> tuning_batch;  // batched path, by size bucket
};

qm_status qm::graph_device_view(const qm_graph *g, GraphDev *out, int *device)
{
    if (!g || !out || !device) return QM_EINVAL;
    *out = g->d;
    *device = g->device;
    return QM_OK;
}

static int log2i(long long x)
{
    int r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

static int bucket_of(long long n, long long arcs, long long K)
{
    return (log2i(n) << 16) | (log2i(arcs) << 8) | log2i(K);
}

static Shape default_shape()
{
    Shape s;
    s.threads = 512;
    s.smem_bytes = 96 * 1024;
    s.big_community = 48;
    s.blocks_per_sm = 0;
    s.algo = 1;
    return s;
}

// Batched kernel: one block per item; communities up to 128 members counted by
// single warps (the autotuner's usual choice on 10^5-node graphs).
static Shape default_batch_shape()
{
    Shape s;
    s.threads = 256;
    s.smem_bytes = 96 * 1024;
    s.big_community = 128;
    s.blocks_per_sm = 0;
    s.algo = 0;
    return s;
}

static Shape resolve_plain(Shape s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    num_sms_of(dev);  // kernel set-up before the occupancy query
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, int> occ;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(s.threads, s.smem_bytes, s.algo);
    auto it = occ.find(key);
    if (it == occ.end())
        it = occ.emplace(key, std::max(1, s.algo == ALGO_SORT ? sort_blocks_per_sm(s)
                                          : s.algo            ? count_blocks_per_sm(s)
                                                              : score_blocks_per_sm(s)))
                 .first;
    s.blocks_per_sm = it->second;
    return s;
}

static Shape resolve_batched(Shape s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    num_sms_of(dev);
    static std::mutex mu;
    static std::map<std::tuple<int, int>, int> occ;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(s.threads, s.smem_bytes);
    auto it = occ.find(key);
    if (it == occ.end()) it = occ.emplace(key, std::max(1, batched_blocks_per_sm(s))).first;
    s.blocks_per_sm = it->second;
    return s;
}

static Shape resolve_batch_units(Shape s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    num_sms_of(dev);
    static std::mutex mu;
    static std::map<std::tuple<int, int>, int> occ;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(s.threads, s.smem_bytes);
    auto it = occ.find(key);
    if (it == occ.end()) it = occ.emplace(key, std::max(1, batch_units_blocks_per_sm(s))).first;
    s.blocks_per_sm = it->second;
    return s;
}

static Shape shape_for(qm_graph *g, int K, bool batched)
{
    std::lock_guard<std::mutex> lk(g->mu);
    auto &m = batched ? g->tuning_batch : g->tuning;
    auto it = m.find(bucket_of(g->n, g->n_arcs, K));
    Shape s = it != m.end() ? it->second : (batched ? default_batch_shape() : default_shape());
    if (!batched && g->wt && s.algo != 1) s = default_shape();  // weighted graphs: two-phase pipeline, direct gathers
    // untuned large graphs in their given (unclustered) node order: each edge
    // gathered once pays there (measured at 10^8 nodes; slower at 3.2*10^7,
    // whose packed labels stay in L2, and on reordered graphs)
    if (!batched && it == m.end() && g->up_ptr && !g->inv && g->n > HALF_MIN_NODES) s.algo = ALGO_HALF;
    return batched ? resolve_batched(s) : resolve_plain(s);
}

static bool shape_ok(const qm_tuning *t)
{
    return t && t->threads >= 64 && t->threads <= 1024 && t->threads % 32 == 0 && t->smem_bytes >= 16384 &&
           t->smem_bytes <= MAX_DYN_SMEM && t->big_community >= 1 && (t->algorithm >= 0 && t->algorithm <= ALGO_HALF) &&
           plan_smem(t->threads, t->smem_bytes).max_used_w >= 32 &&
           (t->algorithm != ALGO_SORT || sort_shape_ok(t->threads, t->smem_bytes));
}

extern "C" {

const char *qm_strerror(qm_status s)
{
    switch (s) {
    case QM_OK: return "ok";
    case QM_EINVAL: return "invalid argument";
    case QM_ENOMEM: return "out of memory";
    case QM_ECUDA: return "CUDA error";
    case QM_ETIMEOUT: return "device wait timed out";
    case QM_EOVERFLOW: return "size exceeds library limits";
    case QM_EBUSY: return "busy";
    }
    return "unknown status";
}

qm_status qm_last_error(char *buf, size_t len)
{
    if (!buf || len == 0) return QM_EINVAL;
    std::snprintf(buf, len, "%s", t_err.c_str());
    return QM_OK;
}

qm_status qm_last_error_detail(char *buf, size_t len) { return qm_last_error(buf, len); }

int64_t qm_kernel_launches(void) { return g_launches.load(); }

qm_status qm_trace_enable(int32_t on)
{
    t_trace.on = on != 0;
    t_trace.used = 0;
    t_trace.last.clear();
    return QM_OK;
}

qm_status qm_trace_read(qm_trace_event *events, int32_t capacity, int32_t *count)
{
    if (!count || (capacity > 0 && !events)) return fail(QM_EINVAL, "bad argument");
    const int32_t n = (int32_t)t_trace.last.size();
    *count = n;
    for (int32_t i = 0; i < n && i < capacity; ++i) {
        std::snprintf(events[i].name, sizeof(events[i].name), "%s", t_trace.last[i].first.c_str());
        events[i].ms = t_trace.last[i].second;
    }
    return QM_OK;
}

static qm_status load_impl(const int64_t *row_ptr, const int32_t *col, const float *weight, int64_t n_nodes,
                           int64_t n_arcs, qm_mem where, unsigned flags, void *stream, qm_graph **out)
{
    if (!out || !row_ptr || !col) return fail(QM_EINVAL, "null argument");
    *out = nullptr;
    if (n_nodes < 1) return fail(QM_EINVAL, "n_nodes must be >= 1");
    if (n_nodes >= (1LL << 31)) return fail(QM_EOVERFLOW, "n_nodes must be < 2^31");
    if (n_arcs > (1LL << 32) - (1LL << 20)) return fail(QM_EOVERFLOW, "n_arcs must be <= 2^32 - 2^20");
    if (n_arcs < 2 || (n_arcs & 1)) return fail(QM_EINVAL, "n_arcs must be even and >= 2 (symmetric CSR of a graph with edges)");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    if (where == QM_HOST && (row_ptr[0] != 0 || row_ptr[n_nodes] != n_arcs))
        return fail(QM_EINVAL, "row_ptr must start at 0 and end at n_arcs");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<qm_graph> g(new qm_graph());
    g->device = dev;
    g->n = n_nodes;
    g->n_arcs = n_arcs;
    g->row_ptr = nullptr;
    g->col = nullptr;
    cudaError_t e = cudaMalloc(&g->row_ptr, (size_t)(n_nodes + 1) * 8);
    if (e == cudaErrorMemoryAllocation) {  // cached scratch blocks may hold the memory: free them, retry
        cudaGetLastError();
        g_pool.trim();
        e = cudaMalloc(&g->row_ptr, (size_t)(n_nodes + 1) * 8);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(row_ptr)");
    e = cudaMalloc(&g->col, (size_t)n_arcs * 4);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        g_pool.trim();
        e = cudaMalloc(&g->col, (size_t)n_arcs * 4);
    }
    if (e != cudaSuccess) {
        cudaFree(g->row_ptr);
        return cuda_fail(e, "cudaMalloc(col)");
    }
    auto cleanup = [&]() {
        cudaFree(g->row_ptr);
        cudaFree(g->col);
        cudaFree(g->wt);
    };
    const cudaMemcpyKind kind = where == QM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    e = cudaMemcpyAsync(g->row_ptr, row_ptr, (size_t)(n_nodes + 1) * 8, kind, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->col, col, (size_t)n_arcs * 4, kind, s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMemcpyAsync(graph)");
    }
    g->d.row_ptr = g->row_ptr;
    g->d.col = g->col;
    g->d.n = n_nodes;
    g->d.n_arcs = n_arcs;
    g->d.max_degree = 0;
    Lease ws(g_pool.acquire(256, dev, false));
    Lease pin(g_pool.acquire(256, dev, true));
    if (!ws.b || !pin.b) {
        cleanup();
        return fail(QM_ENOMEM, "scratch allocation failed");
    }
    int *status = (int *)ws.ptr();
    unsigned long long *md = (unsigned long long *)(ws.ptr() + 64);
    e = cudaMemsetAsync(ws.ptr(), 0, 128, s);
    if (e != cudaSuccess || launch_validate(g->d, (flags & QM_VALIDATE) ? 1 : 0, status, md, num_sms_of(dev), s) < 0) {
        cleanup();
        return cuda_fail(e != cudaSuccess ? e : cudaGetLastError(), "graph validation launch");
    }
    g_launches += 1;
    e = cudaMemcpyAsync(pin.ptr(), ws.ptr(), 128, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "graph validation");
    }
    const int st = *(int *)pin.ptr();
    if (st != 0) {
        cleanup();
        return fail(QM_EINVAL, (flags & QM_VALIDATE)
                                   ? "graph is not a valid symmetric simple CSR with sorted rows"
                                   : "row offsets or column ids out of range");
    }
    g->max_degree = (long long)*(unsigned long long *)(pin.ptr() + 64);
    g->d.max_degree = g->max_degree;
    g->bytes = (size_t)(n_nodes + 1) * 8 + (size_t)n_arcs * 4;
    if (weight) {
        e = cudaMalloc(&g->wt, (size_t)n_arcs * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->wt, weight, (size_t)n_arcs * 4, kind, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ws.ptr(), 0, 256, s);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "weights");
        }
        unsigned long long *lim = (unsigned long long *)(ws.ptr() + 128);
        const int LW = launch_weight_check(g->d, g->wt, (flags & QM_VALIDATE) ? 1 : 0, status, lim,
                                           num_sms_of(dev), s);
        e = LW < 0 ? cudaGetLastError() : cudaMemcpyAsync(pin.ptr(), ws.ptr(), 256, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "weight check");
        }
        g_launches += LW;
        const int wst = *(int *)pin.ptr();
        const uint64_t *L = (const uint64_t *)(pin.ptr() + 128);
        const __int128 two_w = (__int128)(int64_t)L[2] * ((__int128)1 << 86) + (__int128)L[1] * ((__int128)1 << 43) +
                               (__int128)L[0];
        const char *why = (wst & 2)   ? "edge weights must be 0 or in [2^-20, 2^20)"
                          : (wst & 4) ? "edge weights must be symmetric (arc (u,v) and arc (v,u) equal)"
                          : two_w <= 0 ? "the total edge weight must be positive"
                          : (two_w & 1) ? "edge weights must be symmetric (odd fixed-point total)"
                                        : nullptr;
        if (why) {
            cleanup();
            return fail(QM_EINVAL, why);
        }
        const unsigned __int128 w_fx = (unsigned __int128)(two_w / 2);
        g->d.wt = g->wt;
        g->d.w_lo = (unsigned long long)w_fx;
        g->d.w_hi = (unsigned long long)(w_fx >> 64);
        g->bytes += (size_t)n_arcs * 4;
    }
    if (flags & QM_REORDER) {
        long long *row2 = nullptr;
        int *col2 = nullptr, *inv = nullptr, L = 0;
        float *wt2 = nullptr;
        int r = reorder_graph(g->d, QM_REORDER_ROUNDS, num_sms_of(dev), s, &row2, &col2, &inv, &L, &wt2);
        if (r == -(int)cudaErrorMemoryAllocation) {  // cached scratch blocks may hold the memory: free them, retry
            cudaGetLastError();
            g_pool.trim();
            r = reorder_graph(g->d, QM_REORDER_ROUNDS, num_sms_of(dev), s, &row2, &col2, &inv, &L, &wt2);
        }
        if (r != 0) {
            cleanup();
            return cuda_fail((cudaError_t)(-r), "graph reorder");
        }
        g_launches += L;
        cudaFree(g->row_ptr);
        cudaFree(g->col);
        g->row_ptr = row2;
        g->col = col2;
        g->inv = inv;
        g->d.row_ptr = row2;
        g->d.col = col2;
        g->d.inv = inv;
        if (g->wt) {
            cudaFree(g->wt);
            g->wt = wt2;
            g->d.wt = wt2;
        }
        g->bytes += (size_t)n_nodes * 4;
        if (n_nodes > g_pb_min_nodes.load()) {
            const int wb0 = g_pb_wb.load(), tb0 = g_pb_tb.load();
            const int shapes[3][2] = {{16, 16}, {16, 15}, {16, 14}};
            int r = 1;
            for (int k = 0; k < 3 && r == 1; ++k) {
                const int wb = wb0 ? wb0 : shapes[k][0], tb = tb0 ? tb0 : shapes[k][1];
                r = build_perm_buckets(inv, n_nodes, wb, tb, num_sms_of(dev), s, &g->pb, &L);
                if (r == -(int)cudaErrorMemoryAllocation) {
                    cudaGetLastError();
                    g_pool.trim();
                    r = build_perm_buckets(inv, n_nodes, wb, tb, num_sms_of(dev), s, &g->pb, &L);
                }
                if (wb0 && tb0) break;
            }
            if (r < 0) {
                cleanup();
                cudaFree(g->inv);
                return cuda_fail((cudaError_t)(-r), "label permutation buckets");
            }
            if (r == 0) {  // (1: the sizes do not fit the two passes; the labels are gathered directly)
                g_launches += L;
                g->bytes += g->pb.bytes;
            }
        }
    }
    if (!weight && n_arcs < (1LL << 32)) {
        // the upper rows, for gathering each undirected edge once (ALGO_HALF)
        long long up_arcs = 0;
        int L = 0;
        int r = build_upper_rows(g->d, num_sms_of(dev), s, &g->up_ptr, &g->up_col, &up_arcs, &L);
        if (r == -(int)cudaErrorMemoryAllocation) {
            cudaGetLastError();
            g_pool.trim();
            r = build_upper_rows(g->d, num_sms_of(dev), s, &g->up_ptr, &g->up_col, &up_arcs, &L);
        }
        if (r != 0) {
            cleanup();
            cudaFree(g->inv);
            free_perm_buckets(&g->pb);
            return cuda_fail((cudaError_t)(-r), "upper rows");
        }
        g_launches += L;
        g->d.up_ptr = g->up_ptr;
        g->d.up_col = g->up_col;
        g->bytes += (size_t)(n_nodes + 1) * 8 + (size_t)up_arcs * 4;
    }
    *out = g.release();
    return QM_OK;
}

qm_status qm_load_graph(const int64_t *row_ptr, const int32_t *col, int64_t n_nodes, int64_t n_arcs,
                        qm_mem where, unsigned flags, void *stream, qm_graph **out)
{
    return load_impl(row_ptr, col, nullptr, n_nodes, n_arcs, where, flags, stream, out);
}

qm_status qm_load_graph_weighted(const int64_t *row_ptr, const int32_t *col, const float *weight, int64_t n_nodes,
                                 int64_t n_arcs, qm_mem where, unsigned flags, void *stream, qm_graph **out)
{
    if (!weight) return fail(QM_EINVAL, "null weights");
    return load_impl(row_ptr, col, weight, n_nodes, n_arcs, where, flags, stream, out);
}

qm_status qm_free_graph(qm_graph *g)
{
    if (!g) return fail(QM_EINVAL, "null graph");
    DeviceGuard dg(g->device);
    drop_plain_graphs(g);
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->inv);
    cudaFree(g->wt);
    cudaFree(g->up_ptr);
    cudaFree(g->up_col);
    free_perm_buckets(&g->pb);
    delete g;
    return QM_OK;
}

qm_status qm_graph_info(const qm_graph *g, int64_t *n_nodes, int64_t *n_edges, int64_t *max_degree,
                        size_t *device_bytes)
{
    if (!g) return fail(QM_EINVAL, "null graph");
    if (n_nodes) *n_nodes = g->n;
    if (n_edges) *n_edges = g->n_arcs / 2;
    if (max_degree) *max_degree = g->max_degree;
    if (device_bytes) *device_bytes = g->bytes;
    return QM_OK;
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

qm_status qm_workspace_bytes(const qm_graph *g, int32_t K, int32_t with_compare, int32_t k_truth, size_t *bytes)
{
    if (!g || !bytes || K < 1 || (with_compare && k_truth < 1)) return fail(QM_EINVAL, "bad argument");
    const bool wt = g->wt != nullptr;
    size_t b = std::max(score_ws_bytes(g->n, K),
                        score2_ws_bytes(g->n, g->n_arcs, K, wt, 0, packs_labels(1, wt, g->n, K))) +
               al256((size_t)g->n * 4);
    if (g->inv) b += al256((size_t)g->n * 4);
    if (g->pb.lpos) b += al256((size_t)g->n * 4);
    if (with_compare) b += compare_ws_bytes(g->n, k_truth, K) + al256((size_t)g->n * 4);
    *bytes = b;
    return QM_OK;
}

// One plain scoring call on an already-leased workspace.
// One scoring call.  A shard (shard_p > 1, two-phase pipeline only) scores the
// communities c with c mod shard_p == shard_r and returns its exact partial
// sums in gacc_out (QM_PARTIAL_WORDS words) instead of a result.
//
// On graphs of up to kPlainGraphMaxN nodes the launch overhead outweighs the
// work, so the call's device work after the label copy (zeroing, kernels,
// read-back) is captured once into a CUDA graph per (scratch blocks, graph,
// K, launch shape) and replayed; the labels go to a fixed place in the
// scratch first.  Calls with per-community output or tracing run directly.
static constexpr long long kPlainGraphMaxN = 1LL << 21;

static qm_status score_impl(qm_graph *g, const int32_t *labels, int32_t K, qm_mem where, qm_quality *out,
                            const qm_percomm *pc, cudaStream_t s, const Shape &sh, int shard_r = 0,
                            int shard_p = 1, uint64_t *gacc_out = nullptr)
{
    const long long n = g->n;
    const bool weighted = g->wt != nullptr;
    const bool graphed = !pc && !t_trace.on && n <= kPlainGraphMaxN;
    const int bmode = bin_mode_of(sh.algo, weighted);
    const bool pack = packs_labels(sh.algo, weighted, n, K);
    size_t need = sh.algo ? score2_ws_bytes(n, g->n_arcs, K, weighted, bmode, pack) : score_ws_bytes(n, K);
    const size_t lab_off = need;
    if (where == QM_HOST || graphed) need += al256((size_t)n * 4);
    const size_t perm_off = need;
    if (g->inv) need += al256((size_t)n * 4);
    const size_t pb_off = need;
    if (g->pb.lpos) need += al256((size_t)n * 4);
    const size_t pc_off = need;
    const bool pc_host = pc && where == QM_HOST;
    if (pc_host) need += al256((size_t)K * 8) * 8;
    Lease ws(g_pool.acquire(need, g->device, false));
    Lease pin(g_pool.acquire(al256(std::max(sizeof(qm_quality), (size_t)QM_PARTIAL_WORDS * 8)) + 256, g->device,
                             true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "scratch allocation failed");
    ScoreWs w = sh.algo ? carve_score2_ws(ws.ptr(), n, g->n_arcs, K, weighted, bmode, pack)
                        : carve_score_ws(ws.ptr(), n, K);
    const int32_t *dl = labels;
    if (where == QM_HOST || graphed) {
        dl = (const int32_t *)(ws.ptr() + lab_off);
        CK(cudaMemcpyAsync((void *)dl, labels, (size_t)n * 4,
                           where == QM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    }
    PerCommDev pcd{};
    void *const *hp = pc ? (void *const *)pc : nullptr;
    const int nsm = num_sms_of(g->device);
    // the call's device work on stream st; returns its kernel launches, or -1
    auto enqueue = [&](cudaStream_t st, TraceFn tr) -> int {
        int L = 0;
        if (cudaMemsetAsync(ws.ptr(), 0, w.zero_bytes, st) != cudaSuccess) return -1;
        const int32_t *src = dl;
        bool sizes_ready = false;
        if (g->inv) {  // the graph is stored renumbered: gather the labels into its order
            int32_t *pl = (int32_t *)(ws.ptr() + perm_off);
            // two passes through shared memory where the graph has them (the two-phase
            // pipeline then takes the community sizes from the second), else one gather
            const int lp = g->pb.lpos ? launch_permute_buckets(dl, g->pb, n, (int *)(ws.ptr() + pb_off), pl,
                                                               sh.algo ? w.size : nullptr, K, w.status, nsm, st, tr)
                                      : 0;
            if (lp < 0) return -1;
            if (lp > 0) {
                sizes_ready = sh.algo != 0;
                L += lp - 1;
            } else if (sh.algo) {  // the two-phase pipeline takes the community sizes from the gather
                if (tr) tr("k_permute_hist", st);
                if (launch_permute_hist(dl, g->inv, n, pl, K, w, nsm, st) < 0) return -1;
                sizes_ready = true;
            } else {
                if (tr) tr("k_permute_labels", st);
                if (launch_permute_labels(dl, g->inv, n, 1, pl, nsm, st) < 0) return -1;
            }
            L += 1;
            src = pl;
        }
        if (pc) {
            void **dp = (void **)&pcd;
            for (int k = 0; k < 8; ++k) {
                if (!hp[k]) { dp[k] = nullptr; continue; }
                dp[k] = pc_host ? (void *)(ws.ptr() + pc_off + al256((size_t)K * 8) * k) : hp[k];
                if (cudaMemsetAsync(dp[k], 0, (size_t)K * 8, st) != cudaSuccess) return -1;
            }
        }
        const int L2 = sh.algo ? launch_score2(g->d, src, K, w, sh, pc ? &pcd : nullptr, nsm, st, tr, shard_r,
                                               shard_p, sizes_ready)
                               : launch_score(g->d, src, K, w, sh, pc ? &pcd : nullptr, nsm, st, tr);
        if (L2 < 0) return -1;
        L += L2;
        if (cudaMemcpyAsync(pin.ptr(), w.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
        const cudaError_t e = gacc_out
            ? cudaMemcpyAsync(pin.ptr() + 256, w.gacc, QM_PARTIAL_WORDS * 8, cudaMemcpyDeviceToHost, st)
            : cudaMemcpyAsync(pin.ptr() + 256, w.result, sizeof(qm_quality), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return -1;
        if (pc_host) {
            void **dp = (void **)&pcd;
            for (int k = 0; k < 8; ++k)
                if (hp[k] && cudaMemcpyAsync(hp[k], dp[k], (size_t)K * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    return -1;
        }
        return L;
    };
    cudaGraphExec_t exec = nullptr;
    int L = -1;
    if (graphed) {
        const PlainKey key{ws.ptr(), pin.ptr(), g, K, sh.threads, sh.smem_bytes, sh.big_community, sh.algo,
                           shard_r, shard_p, gacc_out ? 1 : 0};
        {
            std::lock_guard<std::mutex> lk(g_graph_mu);
            auto it = g_plain_graphs.find(key);
            if (it != g_plain_graphs.end()) {
                exec = it->second.exec;
                L = it->second.launches;
            }
        }
        if (!exec) {
            cudaStream_t cs = capture_stream(g->device);
            cudaGraph_t graph = nullptr;
            int Lc = -1;
            cudaError_t e = cs ? cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) : cudaErrorInvalidValue;
            if (e == cudaSuccess) {
                Lc = enqueue(cs, nullptr);
                e = cudaStreamEndCapture(cs, &graph);
            }
            if (e == cudaSuccess && Lc >= 0 && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
                L = Lc;
                std::lock_guard<std::mutex> lk(g_graph_mu);
                g_plain_graphs[key] = PlainGraph{exec, L};
            } else {
                exec = nullptr;
                cudaGetLastError();  // the call runs without a graph instead
            }
            if (graph) cudaGraphDestroy(graph);
        }
    }
    if (exec) {
        CK(cudaGraphLaunch(exec, s));
        g_launches += L;
    } else {
        L = enqueue(s, trace_begin());
        if (L < 0) return cuda_fail(cudaGetLastError(), "launch_score");
        g_launches += L;
    }
    CK(cudaStreamSynchronize(s));
    trace_collect();
    const int st = *(int *)pin.ptr();
    if (st & 1) return fail(QM_EINVAL, "a label lies outside [0, K)");
    if (st & 2) return fail(QM_EOVERFLOW, "a community borders too many distinct communities");
    if (st & 4) return fail(QM_ETIMEOUT, "a staging copy did not complete within its wait limit");
    if (st) return fail(QM_ECUDA, "device status word set");
    if (gacc_out) std::memcpy(gacc_out, pin.ptr() + 256, QM_PARTIAL_WORDS * 8);
    else std::memcpy(out, pin.ptr() + 256, sizeof(qm_quality));
    return QM_OK;
}

// ---------------------------------------------------------------- sharded scoring

// The accumulator words: 7 sums of three limbs (value = L2 * 2^86 + L1 * 2^43 +
// L0, L0 and L1 unsigned, L2 signed) at words 0..20, 5 unsigned 64-bit
// counters at 21..25, and one more three-limb sum (Q of a weighted graph) at
// 26..28.
static constexpr int PART_TRIPLE_AT[] = {0, 3, 6, 9, 12, 15, 18, 26};
static constexpr int PART_U64_FIRST = 21, PART_U64_COUNT = 5;

static __int128 part_limbs_get(const uint64_t *L)
{
    return (__int128)(int64_t)L[2] * ((__int128)1 << 86) + (__int128)L[1] * ((__int128)1 << 43) + (__int128)L[0];
}

static void part_limbs_put(uint64_t *L, __int128 v)
{
    const unsigned __int128 mask = (((unsigned __int128)1) << 43) - 1;
    const unsigned __int128 u = (unsigned __int128)v;
    L[0] = (uint64_t)(u & mask);
    L[1] = (uint64_t)((u >> 43) & mask);
    L[2] = (uint64_t)(int64_t)(v >> 86);
}

static uint64_t full_mask(int nranks) { return nranks >= 64 ? ~0ull : ((1ull << nranks) - 1ull); }

qm_status qm_score_partition_part(const qm_graph *gc, const int32_t *labels, int32_t K, qm_mem where,
                                  int32_t rank, int32_t nranks, qm_partial *out, void *stream)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !labels || !out) return fail(QM_EINVAL, "null argument");
    if (K < 1) return fail(QM_EINVAL, "K must be >= 1");
    if (nranks < 1 || nranks > 64 || rank < 0 || rank >= nranks)
        return fail(QM_EINVAL, "need 1 <= nranks <= 64 and 0 <= rank < nranks");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    DeviceGuard dg(g->device);
    Shape sh = shape_for(g, K, false);
    if (sh.algo == 0) sh = resolve_plain(default_shape());  // shards run the two-phase pipeline
    std::memset(out, 0, sizeof(*out));
    const qm_status st = score_impl(g, labels, K, where, nullptr, nullptr, (cudaStream_t)stream, sh, rank, nranks,
                                    out->words);
    if (st != QM_OK) return st;
    out->n_nodes = g->n;
    out->n_edges = g->n_arcs / 2;
    out->nranks = nranks;
    out->flags = g->wt ? 1 : 0;
    out->ranks_mask = 1ull << rank;
    return QM_OK;
}

qm_status qm_partials_combine(const qm_partial *parts, int32_t count, qm_partial *out)
{
    if (!parts || !out || count < 1) return fail(QM_EINVAL, "need count >= 1 partials and an output");
    qm_partial r = parts[0];
    for (int t : PART_TRIPLE_AT) part_limbs_put(r.words + t, part_limbs_get(r.words + t));
    for (int i = 1; i < count; ++i) {
        const qm_partial &p = parts[i];
        if (p.n_nodes != r.n_nodes || p.n_edges != r.n_edges || p.nranks != r.nranks || p.flags != r.flags)
            return fail(QM_EINVAL, "partials of different graphs or shard counts");
        if (p.ranks_mask & r.ranks_mask) return fail(QM_EINVAL, "a shard is present twice");
        for (int t : PART_TRIPLE_AT)
            part_limbs_put(r.words + t, part_limbs_get(r.words + t) + part_limbs_get(p.words + t));
        for (int k = 0; k < PART_U64_COUNT; ++k) r.words[PART_U64_FIRST + k] += p.words[PART_U64_FIRST + k];
        r.ranks_mask |= p.ranks_mask;
    }
    *out = r;
    return QM_OK;
}

qm_status qm_partial_finalize(const qm_partial *p, qm_quality *out, void *stream)
{
    if (!p || !out) return fail(QM_EINVAL, "null argument");
    if (p->nranks < 1 || p->nranks > 64 || p->ranks_mask != full_mask(p->nranks))
        return fail(QM_EINVAL, "the partial does not cover every shard");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    Lease ws(g_pool.acquire(1024, dev, false));
    Lease pin(g_pool.acquire(1024, dev, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "scratch allocation failed");
    char *d = ws.ptr();
    std::memcpy(pin.ptr(), p->words, QM_PARTIAL_WORDS * 8);
    CK(cudaMemcpyAsync(d, pin.ptr(), QM_PARTIAL_WORDS * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(d + 256, 0, 16, s));
    if (launch_score_fin((const unsigned long long *)d, (const int *)(d + 256), p->n_nodes, p->n_edges,
                         (qm_quality *)(d + 512), p->flags & 1, s) < 0)
        return cuda_fail(cudaGetLastError(), "finalize launch");
    g_launches += 1;
    CK(cudaMemcpyAsync(pin.ptr() + 512, d + 512, sizeof(qm_quality), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(out, pin.ptr() + 512, sizeof(qm_quality));
    return QM_OK;
}

qm_status qm_score_partition(const qm_graph *gc, const int32_t *labels, int32_t K, qm_mem where, qm_quality *out,
                             const qm_percomm *per_comm, void *stream)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !labels || !out) return fail(QM_EINVAL, "null argument");
    if (K < 1) return fail(QM_EINVAL, "K must be >= 1");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    DeviceGuard dg(g->device);
    return score_impl(g, labels, K, where, out, per_comm, (cudaStream_t)stream, shape_for(g, K, false));
}

qm_status qm_compare_partitions(const int32_t *truth, const int32_t *found, int64_t n, int32_t ka, int32_t kb,
                                qm_mem where, qm_compare *out, void *stream)
{
    if (!truth || !found || !out) return fail(QM_EINVAL, "null argument");
    if (n < 2) return fail(QM_EINVAL, "n_nodes must be >= 2 (no node pairs otherwise)");
    if (n >= (1LL << 31)) return fail(QM_EOVERFLOW, "n_nodes must be < 2^31");
    if (ka < 1 || kb < 1) return fail(QM_EINVAL, "k_truth and k_found must be >= 1");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    size_t need = compare_ws_bytes(n, ka, kb);
    const size_t lab_off = need;
    if (where == QM_HOST) need += 2 * al256((size_t)n * 4);
    Lease ws(g_pool.acquire(need, dev, false));
    Lease pin(g_pool.acquire(512, dev, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "scratch allocation failed");
    CompareWs w = carve_compare_ws(ws.ptr(), n, ka, kb);
    const int32_t *dt = truth, *df = found;
    if (where == QM_HOST) {
        dt = (const int32_t *)(ws.ptr() + lab_off);
        df = (const int32_t *)(ws.ptr() + lab_off + al256((size_t)n * 4));
        CK(cudaMemcpyAsync((void *)dt, truth, (size_t)n * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync((void *)df, found, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemsetAsync(ws.ptr(), 0, w.zero_bytes, s));
    // Comparison runs are the detected communities' member lists (a few hundred
    // entries with few distinct truth labels): small blocks with large warp
    // tables keep almost all of them in warp mode.
    Shape cs = default_shape();
    cs.algo = 0;
    cs.threads = 128;
    cs.smem_bytes = 48 * 1024;
    Shape sh = resolve_plain(cs);
    const int L = launch_compare(dt, df, n, ka, kb, w, sh, num_sms_of(dev), s, trace_begin());
    if (L < 0) return cuda_fail(cudaGetLastError(), "launch_compare");
    g_launches += L;
    CK(cudaMemcpyAsync(pin.ptr(), w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pin.ptr() + 256, w.result, sizeof(qm_compare), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    trace_collect();
    const int st = *(int *)pin.ptr();
    if (st & 1) return fail(QM_EINVAL, "a label lies outside its range");
    if (st & 2) return fail(QM_EOVERFLOW, "a community holds too many distinct communities");
    std::memcpy(out, pin.ptr() + 256, sizeof(qm_compare));
    return QM_OK;
}

// ------------------------------------------------------------------ batched

struct BatchDesc {
    std::vector<BatchItem> items;   // device pointers filled except outputs/status
    long long n_max = 0;
    int k_max = 1, kt_max = 1;
};

// Runs the two-phase batched pipeline (qm_batched.h) over `d.items`, in waves
// that keep the scratch within an eighth of free memory and the unit counts
// within int range.  Labels must already be on the device and every item's arc
// count at most BATCH_UNITS_MAX_ARCS.
static qm_status run_batched_units(int dev, BatchDesc &d, const Shape &sh0, qm_quality *out_q, qm_compare *out_c,
                                   cudaStream_t s)
{
    const int count = (int)d.items.size();
    const int num_sms = num_sms_of(dev);
    Shape sh = resolve_batch_units(sh0);
    long long a_max = 1;
    bool cells = false;
    for (const BatchItem &it : d.items) {
        a_max = std::max(a_max, it.n_arcs);
        cells |= (it.flags & 2) && it.truth;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    auto scratch = [&](int per) { return batch_units_bytes(per, d.n_max, a_max, d.k_max, d.kt_max, cells); };
    int per = count;
    while (per > 1 && ((long long)per * std::max<long long>(d.k_max, (d.n_max + 31) / 32) >= (1LL << 30) ||
                       scratch(per) > free_b / 8))
        per = (per + 1) / 2;
    if (const int cap = g_batch_wave.load(); cap > 0) per = std::min(per, cap);
    const int waves = (count + per - 1) / per;
    const size_t items_b = al256((size_t)count * sizeof(BatchItem));
    const size_t q_b = al256((size_t)count * sizeof(qm_quality));
    const size_t c_b = al256((size_t)count * sizeof(qm_compare));
    const size_t st_b = al256((size_t)count * sizeof(int) + 256);
    const size_t pre_b = al256((size_t)(count + waves) * 3 * sizeof(int));
    const size_t scratch_b = scratch(per);
    Lease ws(g_pool.acquire(items_b + q_b + c_b + st_b + scratch_b, dev, false));
    Lease pin(g_pool.acquire(items_b + q_b + c_b + st_b + pre_b, dev, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "batched scratch allocation failed");
    char *D = ws.ptr(), *H = pin.ptr();
    BatchItem *items_dev = (BatchItem *)D;
    qm_quality *q_dev = (qm_quality *)(D + items_b);
    qm_compare *c_dev = (qm_compare *)(D + items_b + q_b);
    int *st_dev = (int *)(D + items_b + q_b + c_b);
    BatchUnits bu = carve_batch_units(D + items_b + q_b + c_b + st_b, per, d.n_max, a_max, d.k_max, d.kt_max, cells);
    BatchItem *items_h = (BatchItem *)H;
    int *pre_h = (int *)(H + items_b + q_b + c_b + st_b);  // per wave: tpre, cpre, kpre (w1 - w0 + 1 each)
    for (int i = 0; i < count; ++i) {
        items_h[i] = d.items[i];
        items_h[i].out_q = q_dev + i;
        items_h[i].out_c = c_dev + i;
        items_h[i].status = st_dev + i;
    }
    for (int w = 0; w < waves; ++w) {
        const int w0 = w * per, w1 = std::min(count, w0 + per), m = w1 - w0;
        int *tp = pre_h + 3 * (w0 + w), *cp = tp + m + 1, *kp = cp + m + 1;
        tp[0] = cp[0] = kp[0] = 0;
        for (int i = 0; i < m; ++i) {
            const long long n = d.items[w0 + i].n;
            tp[i + 1] = tp[i] + (int)((n + BATCH_UNITS_TILE - 1) / BATCH_UNITS_TILE);
            cp[i + 1] = cp[i] + (int)((n + 31) / 32);
            kp[i + 1] = kp[i] + d.items[w0 + i].K;
        }
    }
    const long long logt_n = count ? d.items[0].n : 0;
    // key: the leases, the wave size, the item bounds and the log table's node
    // count fix everything the graph holds (prefixes and items are copied in at
    // launch)
    GraphKey key{D, H, count, -(2 * per + (cells ? 1 : 0)), sh.threads, sh.smem_bytes, (int)a_max, d.n_max,
                 d.k_max, d.kt_max, logt_n};
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) exec = it->second;
    }
    int L = 0;
    if (!exec) {
        cudaStream_t cs = capture_stream(dev);
        if (!cs) return fail(QM_ECUDA, "no capture stream");
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaMemcpyAsync(items_dev, items_h, (size_t)count * sizeof(BatchItem), cudaMemcpyHostToDevice, cs);
        cudaMemsetAsync(st_dev, 0, (size_t)count * sizeof(int), cs);
        launch_batch_logt(bu.logt, logt_n, cs);
        L = 1;
        for (int w = 0; w < waves && L >= 0; ++w) {
            const int w0 = w * per, w1 = std::min(count, w0 + per), m = w1 - w0;
            const int *tp = pre_h + 3 * (w0 + w);
            cudaMemcpyAsync(bu.tpre, tp, (size_t)(m + 1) * sizeof(int), cudaMemcpyHostToDevice, cs);
            cudaMemcpyAsync(bu.cpre, tp + m + 1, (size_t)(m + 1) * sizeof(int), cudaMemcpyHostToDevice, cs);
            cudaMemcpyAsync(bu.kpre, tp + 2 * (m + 1), (size_t)(m + 1) * sizeof(int), cudaMemcpyHostToDevice, cs);
            cudaMemsetAsync(bu.zero, 0, bu.zero_bytes, cs);
            BatchUnits bw = bu;
            bw.count = m;
            const int l = launch_batch_units(items_dev + w0, m, bw, logt_n, sh, num_sms, cs);
            L = l < 0 ? -1 : L + l;
        }
        cudaMemcpyAsync(H + items_b, D + items_b, q_b + c_b + (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess || L < 0) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e != cudaSuccess ? e : cudaErrorLaunchFailure, "batched graph capture");
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        std::lock_guard<std::mutex> lk(g_graph_mu);
        g_graphs[key] = exec;
    }
    TraceFn tr = trace_begin();
    if (tr) tr("k_bu", s);
    CK(cudaGraphLaunch(exec, s));
    if (tr) tr(nullptr, s);
    g_launches += 1;
    CK(cudaStreamSynchronize(s));
    trace_collect();
    const int *st_h = (const int *)(H + items_b + q_b + c_b);
    for (int i = 0; i < count; ++i) {
        const std::string item = "item " + std::to_string(i);
        if (st_h[i] & 1) return fail(QM_EINVAL, item + ": a label lies outside its range");
        if (st_h[i] & 2) return fail(QM_EOVERFLOW, item + ": a community borders too many communities");
        if (st_h[i]) return fail(QM_ECUDA, item + ": device status " + std::to_string(st_h[i]));
    }
    const qm_quality *qh = (const qm_quality *)(H + items_b);
    const qm_compare *ch = (const qm_compare *)(H + items_b + q_b);
    for (int i = 0; i < count; ++i) {
        if (out_q && (d.items[i].flags & 1)) out_q[i] = qh[i];
        if (out_c && (d.items[i].flags & 2)) out_c[i] = ch[i];
    }
    return QM_OK;
}

// Runs the batched items: the two-phase pipeline when every item's runs fit
// its limits, otherwise the persistent kernel k_batched (one block per item).
// Labels must already be on the device.
static qm_status run_batched(int dev, BatchDesc &d, const Shape &sh0, qm_quality *out_q, qm_compare *out_c,
                             cudaStream_t s, Lease *extra_dev)
{
    {
        bool fits = true;
        for (const BatchItem &it : d.items) fits &= it.n_arcs <= BATCH_UNITS_MAX_ARCS;
        if (fits) return run_batched_units(dev, d, sh0, out_q, out_c, s);
    }
    (void)extra_dev;
    const int count = (int)d.items.size();
    const int num_sms = num_sms_of(dev);
    Shape sh = resolve_batched(sh0);
    int slots = std::min(count, num_sms * sh.blocks_per_sm);
    // bound the per-block scratch to a quarter of free memory
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    while (slots > 1 && batch_scratch_bytes(d.n_max, d.k_max, d.kt_max, slots) > free_b / 4) slots /= 2;
    const size_t items_b = al256((size_t)count * sizeof(BatchItem));
    const size_t q_b = al256((size_t)count * sizeof(qm_quality));
    const size_t c_b = al256((size_t)count * sizeof(qm_compare));
    const size_t st_b = al256((size_t)count * sizeof(int) + 256);
    const size_t scratch_b = batch_scratch_bytes(d.n_max, d.k_max, d.kt_max, slots);
    Lease ws(g_pool.acquire(items_b + q_b + c_b + st_b + scratch_b, dev, false));
    Lease pin(g_pool.acquire(items_b + q_b + c_b + st_b, dev, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "batched scratch allocation failed");
    char *D = ws.ptr(), *H = pin.ptr();
    BatchItem *items_dev = (BatchItem *)D;
    qm_quality *q_dev = (qm_quality *)(D + items_b);
    qm_compare *c_dev = (qm_compare *)(D + items_b + q_b);
    int *st_dev = (int *)(D + items_b + q_b + c_b);          // [count] statuses, then the queue
    int *queue = st_dev + count;
    BatchScratch bs = carve_batch_scratch(D + items_b + q_b + c_b + st_b, d.n_max, d.k_max, d.kt_max, slots);
    BatchItem *items_h = (BatchItem *)H;
    for (int i = 0; i < count; ++i) {
        items_h[i] = d.items[i];
        items_h[i].out_q = q_dev + i;
        items_h[i].out_c = c_dev + i;
        items_h[i].status = st_dev + i;
    }
    GraphKey key{D, H, count, slots, sh.threads, sh.smem_bytes, sh.big_community, d.n_max, d.k_max, d.kt_max};
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) exec = it->second;
    }
    if (!exec) {
        cudaStream_t cs = capture_stream(dev);
        if (!cs) return fail(QM_ECUDA, "no capture stream");
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaMemcpyAsync(items_dev, items_h, (size_t)count * sizeof(BatchItem), cudaMemcpyHostToDevice, cs);
        cudaMemsetAsync(st_dev, 0, (size_t)count * sizeof(int) + 256, cs);
        const int L = launch_batched(items_dev, count, queue, bs, sh, num_sms, cs, nullptr);
        cudaMemcpyAsync(H + items_b, D + items_b, q_b + c_b + (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess || L < 0) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e != cudaSuccess ? e : cudaErrorLaunchFailure, "batched graph capture");
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        std::lock_guard<std::mutex> lk(g_graph_mu);
        g_graphs[key] = exec;
    }
    TraceFn tr = trace_begin();
    if (tr) tr("k_batched", s);
    CK(cudaGraphLaunch(exec, s));
    if (tr) tr(nullptr, s);
    g_launches += 1;
    CK(cudaStreamSynchronize(s));
    trace_collect();
    const int *st_h = (const int *)(H + items_b + q_b + c_b);
    for (int i = 0; i < count; ++i) {
        if (st_h[i] & 1) return fail(QM_EINVAL, "item " + std::to_string(i) + ": a label lies outside its range");
        if (st_h[i] & 2) return fail(QM_EOVERFLOW, "item " + std::to_string(i) + ": a community borders too many communities");
    }
    const qm_quality *qh = (const qm_quality *)(H + items_b);
    const qm_compare *ch = (const qm_compare *)(H + items_b + q_b);
    for (int i = 0; i < count; ++i) {
        if (out_q && (d.items[i].flags & 1)) out_q[i] = qh[i];
        if (out_c && (d.items[i].flags & 2)) out_c[i] = ch[i];
    }
    return QM_OK;
}

// Batched calls on graphs too large for one block per item: every item runs
// the plain full-GPU pipelines (the kernels of qm_score_partition and
// qm_compare_partitions, so the results are the same bits), one after another,
// captured into one CUDA graph that is launched once; the results come back in
// one copy at the end.  Labels (and truths) are device rows in the graph's
// stored order.
static constexpr long long kBatchBlockMaxN = 1LL << 21;

struct LargeItem {
    const int32_t *labels;
    int K;
    const int32_t *truth;
    int kt;
    int flags;  // 1: score, 2: compare with the truth
};

// Launch shape of the comparison pipeline (see qm_compare_partitions).
static Shape compare_shape()
{
    Shape cs = default_shape();
    cs.algo = 0;
    cs.threads = 128;
    cs.smem_bytes = 48 * 1024;
    return resolve_plain(cs);
}

static qm_status run_large_batched(qm_graph *g, int dev, long long n, const std::vector<LargeItem> &items,
                                   qm_quality *out_q, qm_compare *out_c, cudaStream_t s)
{
    const int P = (int)items.size();
    const bool wt = g && g->wt;
    std::vector<Shape> shapes(P);
    size_t sb = 0, cb = 0;
    for (int p = 0; p < P; ++p) {  // shapes and scratch sizes before any capture
        const LargeItem &it = items[p];
        if (it.flags & 1) {
            shapes[p] = shape_for(g, it.K, false);
            const Shape &sh = shapes[p];
            sb = std::max(sb, sh.algo ? score2_ws_bytes(n, g->n_arcs, it.K, wt, bin_mode_of(sh.algo, wt),
                                                        packs_labels(sh.algo, wt, n, it.K))
                                      : score_ws_bytes(n, it.K));
        }
        if (it.flags & 2) cb = std::max(cb, compare_ws_bytes(n, it.kt, it.K));
    }
    const Shape csh = compare_shape();
    const size_t q_b = al256((size_t)P * sizeof(qm_quality)), c_b = al256((size_t)P * sizeof(qm_compare));
    const size_t st_b = al256((size_t)P * 2 * sizeof(int));
    Lease ws(g_pool.acquire(al256(sb) + al256(cb) + q_b + c_b + st_b, dev, false));
    Lease pin(g_pool.acquire(q_b + c_b + st_b, dev, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "batched scratch allocation failed");
    char *S = ws.ptr(), *C = S + al256(sb), *R = C + al256(cb);
    qm_quality *q_dev = (qm_quality *)R;
    qm_compare *c_dev = (qm_compare *)(R + q_b);
    int *st_dev = (int *)(R + q_b + c_b);
    const int nsm = num_sms_of(dev);
    cudaStream_t cs = capture_stream(dev);
    if (!cs) return fail(QM_ECUDA, "no capture stream");
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int L = 0;
    bool ok = cudaMemsetAsync(st_dev, 0, st_b, cs) == cudaSuccess;
    for (int p = 0; p < P && ok; ++p) {
        const LargeItem &it = items[p];
        if (it.flags & 1) {
            const Shape &sh = shapes[p];
            const ScoreWs w = sh.algo ? carve_score2_ws(S, n, g->n_arcs, it.K, wt, bin_mode_of(sh.algo, wt),
                                                        packs_labels(sh.algo, wt, n, it.K))
                                      : carve_score_ws(S, n, it.K);
            ok = cudaMemsetAsync(S, 0, w.zero_bytes, cs) == cudaSuccess;
            const int Li = !ok ? -1
                         : sh.algo ? launch_score2(g->d, it.labels, it.K, w, sh, nullptr, nsm, cs, nullptr)
                                   : launch_score(g->d, it.labels, it.K, w, sh, nullptr, nsm, cs, nullptr);
            ok = Li >= 0 &&
                 cudaMemcpyAsync(q_dev + p, w.result, sizeof(qm_quality), cudaMemcpyDeviceToDevice, cs) == cudaSuccess &&
                 cudaMemcpyAsync(st_dev + 2 * p, w.status, sizeof(int), cudaMemcpyDeviceToDevice, cs) == cudaSuccess;
            L += std::max(Li, 0);
        }
        if (ok && (it.flags & 2)) {
            const CompareWs w = carve_compare_ws(C, n, it.kt, it.K);
            ok = cudaMemsetAsync(C, 0, w.zero_bytes, cs) == cudaSuccess;
            const int Li = ok ? launch_compare(it.truth, it.labels, n, it.kt, it.K, w, csh, nsm, cs, nullptr) : -1;
            ok = Li >= 0 &&
                 cudaMemcpyAsync(c_dev + p, w.result, sizeof(qm_compare), cudaMemcpyDeviceToDevice, cs) == cudaSuccess &&
                 cudaMemcpyAsync(st_dev + 2 * p + 1, w.status, sizeof(int), cudaMemcpyDeviceToDevice, cs) == cudaSuccess;
            L += std::max(Li, 0);
        }
    }
    if (ok) ok = cudaMemcpyAsync(pin.ptr(), R, q_b + c_b + st_b, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && ok) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || !ok) {
        if (exec) cudaGraphExecDestroy(exec);
        return cuda_fail(e != cudaSuccess ? e : cudaErrorLaunchFailure, "batched capture of the plain pipelines");
    }
    TraceFn tr = trace_begin();
    if (tr) tr("batched_plain", s);
    e = cudaGraphLaunch(exec, s);
    if (tr) tr(nullptr, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    g_launches += L;
    trace_collect();
    const char *H = pin.ptr();
    const int *st_h = (const int *)(H + q_b + c_b);
    for (int p = 0; p < P; ++p)
        for (int k = 0; k < 2; ++k) {
            const int v = st_h[2 * p + k];
            if (v & 1) return fail(QM_EINVAL, "item " + std::to_string(p) + ": a label lies outside its range");
            if (v & 2) return fail(QM_EOVERFLOW, "item " + std::to_string(p) + ": a community borders too many communities");
            if (v & 4) return fail(QM_ETIMEOUT, "item " + std::to_string(p) + ": a bounded device wait expired");
            if (v) return fail(QM_ECUDA, "item " + std::to_string(p) + ": device status " + std::to_string(v));
        }
    for (int p = 0; p < P; ++p) {
        if (out_q && (items[p].flags & 1)) out_q[p] = ((const qm_quality *)H)[p];
        if (out_c && (items[p].flags & 2)) out_c[p] = ((const qm_compare *)(H + q_b))[p];
    }
    return QM_OK;
}

// Copies P label rows (and an optional truth) to the device when they are host memory.
static qm_status stage_labels(int dev, const int32_t *labels, size_t n_labels, qm_mem where, cudaStream_t s,
                              Lease &lease, const int32_t **out)
{
    if (where == QM_DEVICE) {
        *out = labels;
        return QM_OK;
    }
    lease.b = g_pool.acquire(n_labels * 4, dev, false);
    if (!lease.b) return fail(QM_ENOMEM, "label staging allocation failed");
    CK(cudaMemcpyAsync(lease.ptr(), labels, n_labels * 4, cudaMemcpyHostToDevice, s));
    *out = (const int32_t *)lease.ptr();
    return QM_OK;
}

static qm_status evaluate_batched(qm_graph *g, const int32_t *labels, int32_t P, const int32_t *K,
                                  const int32_t *truth, int32_t kt, int flags, qm_mem where, qm_quality *out_q,
                                  qm_compare *out_c, cudaStream_t s, const Shape *force = nullptr)
{
    if (!g || !labels || !K || P < 1) return fail(QM_EINVAL, "bad argument");
    if (g->wt) return fail(QM_EINVAL, "weighted graphs are scored by qm_score_partition and the sharded calls");
    if ((flags & 2) && (!truth || kt < 1)) return fail(QM_EINVAL, "truth labels required");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    DeviceGuard dg(g->device);
    BatchDesc d;
    int kmax = 1;
    for (int p = 0; p < P; ++p) {
        if (K[p] < 1) return fail(QM_EINVAL, "K must be >= 1");
        kmax = std::max(kmax, K[p]);
    }
    Lease lab, tru;
    const int32_t *dl = nullptr, *dt = nullptr;
    qm_status st = stage_labels(g->device, labels, (size_t)P * g->n, where, s, lab, &dl);
    if (st != QM_OK) return st;
    if (flags & 2) {
        st = stage_labels(g->device, truth, (size_t)g->n, where, s, tru, &dt);
        if (st != QM_OK) return st;
    }
    Lease plab;
    if (g->inv) {  // renumbered graph: candidates and truth follow its node order
        const size_t rows = (size_t)P + ((flags & 2) ? 1 : 0);
        plab.b = g_pool.acquire(rows * (size_t)g->n * 4, g->device, false);
        if (!plab.b) return fail(QM_ENOMEM, "label permutation allocation failed");
        int32_t *pl = (int32_t *)plab.ptr();
        if (launch_permute_labels(dl, g->inv, g->n, P, pl, num_sms_of(g->device), s) < 0)
            return cuda_fail(cudaGetLastError(), "label permutation");
        dl = pl;
        if (flags & 2) {
            if (launch_permute_labels(dt, g->inv, g->n, 1, pl + (size_t)P * g->n, num_sms_of(g->device), s) < 0)
                return cuda_fail(cudaGetLastError(), "label permutation");
            dt = pl + (size_t)P * g->n;
        }
        g_launches += (flags & 2) ? 2 : 1;
    }
    if (g->n > kBatchBlockMaxN && !force) {  // one block per item would not fill the GPU: plain pipelines
        std::vector<LargeItem> li(P);
        for (int p = 0; p < P; ++p)
            li[p] = LargeItem{dl + (size_t)p * g->n, K[p], (flags & 2) ? dt : nullptr, (flags & 2) ? kt : 0, flags};
        return run_large_batched(g, g->device, g->n, li, out_q, out_c, s);
    }
    d.n_max = g->n;
    d.k_max = kmax;
    d.kt_max = (flags & 2) ? kt : 1;
    d.items.resize(P);
    for (int p = 0; p < P; ++p) {
        BatchItem &it = d.items[p];
        std::memset(&it, 0, sizeof(it));
        it.row_ptr = g->row_ptr;
        it.col = g->col;
        it.labels = dl + (size_t)p * g->n;
        it.truth = (flags & 2) ? dt : nullptr;
        it.n = g->n;
        it.n_arcs = g->n_arcs;
        it.K = K[p];
        it.k_truth = (flags & 2) ? kt : 0;
        it.flags = flags;
    }
    return run_batched(g->device, d, force ? *force : shape_for(g, kmax, true), out_q, out_c, s, nullptr);
}

qm_status qm_score_partitions_batched(const qm_graph *g, const int32_t *labels, int32_t P, const int32_t *K,
                                      qm_mem where, qm_quality *out, void *stream)
{
    if (!out) return fail(QM_EINVAL, "null output");
    return evaluate_batched(const_cast<qm_graph *>(g), labels, P, K, nullptr, 0, 1, where, out, nullptr,
                            (cudaStream_t)stream);
}

qm_status qm_evaluate_partitions_batched(const qm_graph *g, const int32_t *labels, int32_t P, const int32_t *K,
                                         const int32_t *truth, int32_t k_truth, qm_mem where, qm_quality *out_q,
                                         qm_compare *out_c, void *stream)
{
    if (!out_q || !out_c) return fail(QM_EINVAL, "null output");
    return evaluate_batched(const_cast<qm_graph *>(g), labels, P, K, truth, k_truth, 3, where, out_q, out_c,
                            (cudaStream_t)stream);
}

qm_status qm_compare_partitions_batched(const int32_t *truth, const int32_t *found, int64_t n, int32_t P,
                                        const int32_t *k_truth, const int32_t *k_found, unsigned flags,
                                        qm_mem where, qm_compare *out, void *stream)
{
    if (!truth || !found || !k_truth || !k_found || !out || P < 1) return fail(QM_EINVAL, "bad argument");
    if (n < 2) return fail(QM_EINVAL, "n_nodes must be >= 2");
    if (n >= (1LL << 31)) return fail(QM_EOVERFLOW, "n_nodes must be < 2^31");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    const bool shared = (flags & QM_SHARED_TRUTH) != 0;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    Lease lab, tru;
    const int32_t *df = nullptr, *dt = nullptr;
    qm_status st = stage_labels(dev, found, (size_t)P * n, where, s, lab, &df);
    if (st != QM_OK) return st;
    st = stage_labels(dev, truth, (size_t)(shared ? 1 : P) * n, where, s, tru, &dt);
    if (st != QM_OK) return st;
    if (n > kBatchBlockMaxN) {  // one block per item would not fill the GPU: plain pipelines
        std::vector<LargeItem> li(P);
        for (int p = 0; p < P; ++p) {
            const int kt = shared ? k_truth[0] : k_truth[p];
            if (kt < 1 || k_found[p] < 1) return fail(QM_EINVAL, "label-id counts must be >= 1");
            li[p] = LargeItem{df + (size_t)p * n, k_found[p], dt + (shared ? 0 : (size_t)p * n), kt, 2};
        }
        return run_large_batched(nullptr, dev, n, li, nullptr, out, s);
    }
    BatchDesc d;
    d.n_max = n;
    d.items.resize(P);
    for (int p = 0; p < P; ++p) {
        const int kt = shared ? k_truth[0] : k_truth[p];
        if (kt < 1 || k_found[p] < 1) return fail(QM_EINVAL, "label-id counts must be >= 1");
        d.k_max = std::max(d.k_max, k_found[p]);
        d.kt_max = std::max(d.kt_max, kt);
        BatchItem &it = d.items[p];
        std::memset(&it, 0, sizeof(it));
        it.labels = df + (size_t)p * n;
        it.truth = dt + (shared ? 0 : (size_t)p * n);
        it.n = n;
        it.K = k_found[p];
        it.k_truth = kt;
        it.flags = 2;
    }
    return run_batched(dev, d, default_batch_shape(), nullptr, out, s, nullptr);
}

qm_status qm_score_graphs_batched(const qm_graph *const *graphs, const int32_t *const *labels, const int32_t *K,
                                  int32_t count, qm_mem where, qm_quality *out, void *stream)
{
    if (!graphs || !labels || !K || !out || count < 1) return fail(QM_EINVAL, "bad argument");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    const int dev = graphs[0] ? graphs[0]->device : -1;
    BatchDesc d;
    size_t total_labels = 0;
    for (int i = 0; i < count; ++i) {
        if (!graphs[i] || !labels[i] || K[i] < 1) return fail(QM_EINVAL, "bad graph, labels or K");
        if (graphs[i]->wt) return fail(QM_EINVAL, "weighted graphs are scored by qm_score_partition and the sharded calls");
        if (graphs[i]->device != dev) return fail(QM_EINVAL, "all graphs must live on one device");
        d.n_max = std::max(d.n_max, graphs[i]->n);
        d.k_max = std::max(d.k_max, K[i]);
        total_labels += (size_t)graphs[i]->n;
    }
    DeviceGuard dg(dev);
    cudaStream_t s = (cudaStream_t)stream;
    Lease lab;
    std::vector<const int32_t *> dl(count);
    if (where == QM_HOST) {
        lab.b = g_pool.acquire(total_labels * 4 + 256 * (size_t)count, dev, false);
        if (!lab.b) return fail(QM_ENOMEM, "label staging allocation failed");
        size_t off = 0;
        for (int i = 0; i < count; ++i) {
            dl[i] = (const int32_t *)(lab.ptr() + off);
            CK(cudaMemcpyAsync((void *)dl[i], labels[i], (size_t)graphs[i]->n * 4, cudaMemcpyHostToDevice, s));
            off += al256((size_t)graphs[i]->n * 4);
        }
    } else {
        for (int i = 0; i < count; ++i) dl[i] = labels[i];
    }
    size_t perm_total = 0;
    for (int i = 0; i < count; ++i)
        if (graphs[i]->inv) perm_total += al256((size_t)graphs[i]->n * 4);
    Lease plab;
    if (perm_total) {  // renumbered graphs: gather their labels into the graph's node order
        plab.b = g_pool.acquire(perm_total, dev, false);
        if (!plab.b) return fail(QM_ENOMEM, "label permutation allocation failed");
        size_t off = 0;
        for (int i = 0; i < count; ++i) {
            if (!graphs[i]->inv) continue;
            int32_t *pl = (int32_t *)(plab.ptr() + off);
            if (launch_permute_labels(dl[i], graphs[i]->inv, graphs[i]->n, 1, pl, num_sms_of(dev), s) < 0)
                return cuda_fail(cudaGetLastError(), "label permutation");
            g_launches += 1;
            dl[i] = pl;
            off += al256((size_t)graphs[i]->n * 4);
        }
    }
    d.items.resize(count);
    for (int i = 0; i < count; ++i) {
        BatchItem &it = d.items[i];
        std::memset(&it, 0, sizeof(it));
        it.row_ptr = graphs[i]->row_ptr;
        it.col = graphs[i]->col;
        it.labels = dl[i];
        it.n = graphs[i]->n;
        it.n_arcs = graphs[i]->n_arcs;
        it.K = K[i];
        it.flags = 1;
    }
    return run_batched(dev, d, default_batch_shape(), out, nullptr, s, nullptr);
}

qm_status qm_release_cache(void)
{
    g_pool.trim();
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto &kv : g_graphs) cudaGraphExecDestroy(kv.second);
    g_graphs.clear();
    for (auto &kv : g_plain_graphs) cudaGraphExecDestroy(kv.second.exec);
    g_plain_graphs.clear();
    return QM_OK;
}

// ------------------------------------------------------------------ covers (overlapping communities)

// Device copies of a cover's arrays (host arrays are staged; device ones are
// used as they are) and its membership count m = mptr[n].
static qm_status stage_cover(int dev, const int64_t *mptr, const int32_t *memb, long long n, qm_mem where,
                             cudaStream_t s, Lease &lease, const long long **dptr, const int **dmemb, long long *m)
{
    if (where == QM_HOST) {
        *m = mptr[n];
    } else {
        long long v = 0;
        CK(cudaMemcpyAsync(&v, mptr + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *m = v;
    }
    if (*m < 0 || *m >= (1LL << 31)) return fail(QM_EOVERFLOW, "a cover must hold fewer than 2^31 memberships");
    if (where == QM_DEVICE) {
        *dptr = (const long long *)mptr;
        *dmemb = memb;
        return QM_OK;
    }
    const size_t pb = al256(((size_t)n + 1) * 8), mbytes = al256((size_t)std::max(*m, 1LL) * 4);
    lease.b = g_pool.acquire(pb + mbytes, dev, false);
    if (!lease.b) return fail(QM_ENOMEM, "cover staging allocation failed");
    CK(cudaMemcpyAsync(lease.ptr(), mptr, ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, s));
    if (*m > 0) CK(cudaMemcpyAsync(lease.ptr() + pb, memb, (size_t)*m * 4, cudaMemcpyHostToDevice, s));
    *dptr = (const long long *)lease.ptr();
    *dmemb = (const int *)(lease.ptr() + pb);
    return QM_OK;
}

static qm_status cover_status(int st)
{
    if (st & 1) return fail(QM_EINVAL, "a cover's offsets or lists are malformed (lists must be strictly increasing ids in [0, K))");
    if (st & 2) return fail(QM_EOVERFLOW, "a community borders too many distinct communities");
    if (st) return fail(QM_ECUDA, "device status " + std::to_string(st));
    return QM_OK;
}

qm_status qm_score_cover(const qm_graph *gc, const int64_t *mptr, const int32_t *memb, int32_t K, qm_mem where,
                         qm_quality *out, void *stream)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !mptr || !out || (!memb && where == QM_DEVICE)) return fail(QM_EINVAL, "null argument");
    if (K < 1) return fail(QM_EINVAL, "K must be >= 1");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    if (g->wt) return fail(QM_EINVAL, "weighted graphs are scored by qm_score_partition and the sharded calls");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    Lease stage;
    const long long *dptr = nullptr;
    const int *dmemb = nullptr;
    long long m = 0;
    qm_status st = stage_cover(g->device, mptr, memb, g->n, where, s, stage, &dptr, &dmemb, &m);
    if (st != QM_OK) return st;
    Lease ws(g_pool.acquire(cover_score_ws_bytes(g->n, m, K), g->device, false));
    Lease pin(g_pool.acquire(512, g->device, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "scratch allocation failed");
    const CoverWs w = carve_cover_score_ws(ws.ptr(), g->n, m, K);
    CK(cudaMemsetAsync(ws.ptr(), 0, w.zero_bytes, s));
    const int L = launch_cover_score(g->d, dptr, dmemb, m, K, w, num_sms_of(g->device), s);
    if (L < 0) return cuda_fail(cudaGetLastError(), "launch_cover_score");
    g_launches += L;
    CK(cudaMemcpyAsync(pin.ptr(), w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pin.ptr() + 256, w.result, sizeof(qm_quality), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st = cover_status(*(int *)pin.ptr());
    if (st != QM_OK) return st;
    const qm_quality *q = (const qm_quality *)(pin.ptr() + 256);
    if (q->n_communities_nonempty == 0) return fail(QM_EINVAL, "no community of the cover has a member");
    std::memcpy(out, q, sizeof(qm_quality));
    return QM_OK;
}

qm_status qm_compare_covers(const int64_t *truth_ptr, const int32_t *truth_memb, int32_t k_truth,
                            const int64_t *found_ptr, const int32_t *found_memb, int32_t k_found, int64_t n,
                            qm_mem where, qm_compare *out, void *stream)
{
    if (!truth_ptr || !found_ptr || !out) return fail(QM_EINVAL, "null argument");
    if (n < 2) return fail(QM_EINVAL, "n_nodes must be >= 2 (no node pairs otherwise)");
    if (n >= (1LL << 31)) return fail(QM_EOVERFLOW, "n_nodes must be < 2^31");
    if (k_truth < 1 || k_found < 1) return fail(QM_EINVAL, "k_truth and k_found must be >= 1");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    Lease sa, sb;
    const long long *ap = nullptr, *bp = nullptr;
    const int *am = nullptr, *bm = nullptr;
    long long ma = 0, mb = 0;
    qm_status st = stage_cover(dev, truth_ptr, truth_memb, n, where, s, sa, &ap, &am, &ma);
    if (st != QM_OK) return st;
    st = stage_cover(dev, found_ptr, found_memb, n, where, s, sb, &bp, &bm, &mb);
    if (st != QM_OK) return st;
    Lease ws(g_pool.acquire(cover_compare_ws_bytes(n, ma, k_truth, mb, k_found), dev, false));
    Lease pin(g_pool.acquire(512, dev, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "scratch allocation failed");
    const CoverWs w = carve_cover_compare_ws(ws.ptr(), n, ma, k_truth, mb, k_found);
    CK(cudaMemsetAsync(ws.ptr(), 0, w.zero_bytes, s));
    const int L = launch_cover_compare(ap, am, ma, k_truth, bp, bm, mb, k_found, n, w, num_sms_of(dev), s);
    if (L < 0) return cuda_fail(cudaGetLastError(), "launch_cover_compare");
    g_launches += L;
    CK(cudaMemcpyAsync(pin.ptr(), w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pin.ptr() + 256, w.result, sizeof(qm_compare), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st = cover_status(*(int *)pin.ptr());
    if (st != QM_OK) return st;
    std::memcpy(out, pin.ptr() + 256, sizeof(qm_compare));
    return QM_OK;
}

qm_status qm_debug_set_batch_wave(int32_t items)
{
    if (items < 0) return fail(QM_EINVAL, "items must be >= 0");
    g_batch_wave.store(items);
    return QM_OK;
}

qm_status qm_debug_set_perm_buckets(int32_t window_bits, int32_t tile_bits, int64_t min_nodes)
{
    if (window_bits == 0 || window_bits > PB_MAX_BITS || tile_bits == 0 || tile_bits > PB_MAX_BITS)
        return fail(QM_EINVAL, "window_bits and tile_bits must be in [1, 16]");
    g_pb_wb.store(window_bits < 0 ? 0 : window_bits);
    g_pb_tb.store(tile_bits < 0 ? 0 : tile_bits);
    g_pb_min_nodes.store(min_nodes < 0 ? PB_MIN_NODES : (long long)min_nodes);
    return QM_OK;
}

qm_status qm_debug_set_stage_wait(int64_t polls)
{
    qm::set_stage_wait_polls((long long)polls);
    return qm_release_cache();  // captured calls hold the old limit in their kernel arguments
}

// ------------------------------------------------------------------ tuning

qm_status qm_get_tuning(const qm_graph *gc, int32_t K, qm_tuning *t)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !t || K < 1) return fail(QM_EINVAL, "bad argument");
    DeviceGuard dg(g->device);
    const Shape s = shape_for(g, K, false);
    t->threads = s.threads;
    t->smem_bytes = s.smem_bytes;
    t->big_community = s.big_community;
    t->blocks_per_sm = s.blocks_per_sm;
    t->algorithm = s.algo;
    return QM_OK;
}

qm_status qm_set_tuning(const qm_graph *gc, int32_t K, const qm_tuning *t)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || K < 1 || !shape_ok(t)) return fail(QM_EINVAL, "bad tuning");
    Shape s;
    s.threads = t->threads;
    s.smem_bytes = t->smem_bytes;
    s.big_community = t->big_community;
    s.blocks_per_sm = 0;
    s.algo = t->algorithm;
    std::lock_guard<std::mutex> lk(g->mu);
    g->tuning[bucket_of(g->n, g->n_arcs, K)] = s;
    return QM_OK;
}

qm_status qm_label_propagation(const qm_graph *gc, int32_t rounds, int32_t *labels_out, qm_mem where,
                               int32_t *k_out, void *stream)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !labels_out || !k_out) return fail(QM_EINVAL, "null argument");
    if (rounds < 0 || rounds > 1000) return fail(QM_EINVAL, "rounds must be in [0, 1000]");
    if (where != QM_HOST && where != QM_DEVICE) return fail(QM_EINVAL, "bad memory kind");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = g->n;
    const size_t tmp_elems = scan_tmp_elems(n + 1) + 64;
    const size_t b_lab = al256((size_t)n * 4), b_hist = al256((size_t)(n + 1) * 4);
    const size_t need = 2 * b_lab + b_hist + al256(tmp_elems * 4) + (where == QM_HOST ? b_lab : 0);
    Lease ws(g_pool.acquire(need, g->device, false));
    Lease pin(g_pool.acquire(256, g->device, true));
    if (!ws.b || !pin.b) return fail(QM_ENOMEM, "scratch allocation failed");
    char *p = ws.ptr();
    int *lab0 = (int *)p, *lab1 = (int *)(p + b_lab), *hist = (int *)(p + 2 * b_lab);
    int *tmp = (int *)(p + 2 * b_lab + b_hist);
    int *out = where == QM_HOST ? (int *)(p + 2 * b_lab + b_hist + al256(tmp_elems * 4)) : labels_out;
    const int L = launch_label_propagation(g->d, rounds, num_sms_of(g->device), s, lab0, lab1, hist, tmp,
                                           tmp_elems, out);
    if (L < 0) return cuda_fail(cudaGetLastError(), "label propagation launch");
    g_launches += L;
    CK(cudaMemcpyAsync(pin.ptr(), hist + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (where == QM_HOST) CK(cudaMemcpyAsync(labels_out, out, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *k_out = *(int *)pin.ptr();
    return QM_OK;
}

qm_status qm_get_batch_tuning(const qm_graph *gc, int32_t K, qm_tuning *t)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !t || K < 1) return fail(QM_EINVAL, "bad argument");
    DeviceGuard dg(g->device);
    const Shape s = shape_for(g, K, true);
    t->threads = s.threads;
    t->smem_bytes = s.smem_bytes;
    t->big_community = s.big_community;
    t->blocks_per_sm = s.blocks_per_sm;
    t->algorithm = 0;
    return QM_OK;
}

qm_status qm_set_batch_tuning(const qm_graph *gc, int32_t K, const qm_tuning *t)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || K < 1 || !shape_ok(t)) return fail(QM_EINVAL, "bad tuning");
    if (t->threads > BATCH_MAX_THREADS) return fail(QM_EINVAL, "the batched kernel takes at most 512 threads a block");
    Shape s;
    s.threads = t->threads;
    s.smem_bytes = t->smem_bytes;
    s.big_community = t->big_community;
    s.blocks_per_sm = 0;
    s.algo = 0;
    std::lock_guard<std::mutex> lk(g->mu);
    g->tuning_batch[bucket_of(g->n, g->n_arcs, K)] = s;
    return QM_OK;
}

// Times candidate shapes of the batched kernel on the caller's batch (the
// median of 3 launches each, CUDA events on the call's stream) and caches the
// fastest for the batch's size bucket (its largest K).
qm_status qm_autotune_batched(const qm_graph *gc, const int32_t *labels, int32_t P, const int32_t *K,
                              const int32_t *truth, int32_t k_truth, qm_mem where, void *stream,
                              qm_tuning *chosen)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !labels || !K || P < 1) return fail(QM_EINVAL, "bad argument");
    if (g->wt) return fail(QM_EINVAL, "weighted graphs are scored by qm_score_partition and the sharded calls");
    if (truth && k_truth < 1) return fail(QM_EINVAL, "k_truth must be >= 1");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    int kmax = 1;
    for (int p = 0; p < P; ++p) kmax = std::max(kmax, K[p]);
    const int flags = truth ? 3 : 1;
    std::vector<qm_quality> oq(P);
    std::vector<qm_compare> oc(P);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    num_sms_of(g->device);
    float best_ms = 1e30f;
    Shape best = default_shape();
    best.algo = 0;
    // the two-phase pipeline (graphs with at most BATCH_UNITS_MAX_ARCS arcs)
    // has no large-community threshold; the one-block-per-item kernel does
    const bool units = g->n_arcs <= BATCH_UNITS_MAX_ARCS;
    const std::vector<int> smems = units ? std::vector<int>{32 * 1024, 48 * 1024, 64 * 1024, 96 * 1024, 160 * 1024}
                                         : std::vector<int>{64 * 1024, 96 * 1024, 160 * 1024};
    const std::vector<int> bigs = units ? std::vector<int>{128} : std::vector<int>{48, 128, 256};
    for (int th : {256, 512})
        for (int sm : smems)
            for (int bg : bigs) {
                qm_tuning tt{th, sm, bg, 0, 0};
                if (!shape_ok(&tt)) continue;
                Shape sh;
                sh.threads = th;
                sh.smem_bytes = sm;
                sh.big_community = bg;
                sh.blocks_per_sm = 0;
                sh.algo = 0;
                if ((units ? resolve_batch_units(sh) : resolve_batched(sh)).blocks_per_sm < 1) continue;
                float times[3];
                bool ok = true;
                for (int r = 0; r < 3 && ok; ++r) {
                    cudaEventRecord(e0, s);
                    if (evaluate_batched(g, labels, P, K, truth, k_truth, flags, where, oq.data(),
                                         truth ? oc.data() : nullptr, s, &sh) != QM_OK)
                        ok = false;
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&times[r], e0, e1);
                }
                if (!ok) continue;
                std::sort(times, times + 3);
                if (times[1] < best_ms) {
                    best_ms = times[1];
                    best = sh;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g->mu);
        Shape b = best;
        b.blocks_per_sm = 0;
        g->tuning_batch[bucket_of(g->n, g->n_arcs, kmax)] = b;
    }
    if (chosen) {
        const Shape r = units ? resolve_batch_units(best) : resolve_batched(best);
        chosen->threads = r.threads;
        chosen->smem_bytes = r.smem_bytes;
        chosen->big_community = r.big_community;
        chosen->blocks_per_sm = r.blocks_per_sm;
        chosen->algorithm = 0;
    }
    return QM_OK;
}

// Times every candidate shape of the plain path on these inputs (median of 3
// runs each, CUDA events on the call's stream) and caches the fastest.
qm_status qm_autotune(const qm_graph *gc, const int32_t *labels, int32_t K, qm_mem where, void *stream,
                      qm_tuning *chosen)
{
    qm_graph *g = const_cast<qm_graph *>(gc);
    if (!g || !labels || K < 1) return fail(QM_EINVAL, "bad argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    Lease lab;
    const int32_t *dl = nullptr;
    qm_status st = stage_labels(g->device, labels, (size_t)g->n, where, s, lab, &dl);
    if (st != QM_OK) return st;
    const int threads_c[] = {256, 512, 1024};
    const int smem_c[] = {48 * 1024, 96 * 1024, 200 * 1024};
    num_sms_of(g->device);
    const int big_c[] = {24, 48, 96};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    Shape best = default_shape();
    qm_quality q;
    for (int al : {2, 5, 1, ALGO_HALF, ALGO_SORT, 0})
    for (int th : threads_c)
        for (int sm : smem_c)
            for (int bg : big_c) {
                if (al >= 1 && bg != big_c[0]) continue;  // the two-phase path has no size split
                if (al == 0 && g->wt) continue;           // weighted graphs: two-phase pipeline only
                if (al == 2 && (g->wt || g->n <= BIN_MIN_NODES)) continue;  // binning can pay beyond L2 only
                if (al == 5 && (g->wt || !packs_labels(1, false, g->n, K))) continue;  // 1 is 5 there
                if (al == ALGO_SORT && g->wt) continue;   // weighted runs carry weights: hashed only
                if (al == ALGO_HALF && !g->up_ptr) continue;  // no upper rows (weighted or huge graphs)
                Shape sh;
                sh.threads = th;
                sh.smem_bytes = sm;
                sh.big_community = bg;
                sh.blocks_per_sm = 0;
                sh.algo = al;
                qm_tuning tt{th, sm, bg, 0, al};
                if (!shape_ok(&tt)) continue;
                sh = resolve_plain(sh);
                if (sh.blocks_per_sm < 1) continue;
                float times[3];
                bool ok = true;
                for (int r = 0; r < 3 && ok; ++r) {
                    cudaEventRecord(e0, s);
                    if (score_impl(g, dl, K, QM_DEVICE, &q, nullptr, s, sh) != QM_OK) ok = false;
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&times[r], e0, e1);
                }
                if (!ok) continue;
                std::sort(times, times + 3);
                if (times[1] < best_ms) {
                    best_ms = times[1];
                    best = sh;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g->mu);
        Shape b = best;
        b.blocks_per_sm = 0;
        g->tuning[bucket_of(g->n, g->n_arcs, K)] = b;
    }
    if (chosen) {
        chosen->threads = best.threads;
        chosen->smem_bytes = best.smem_bytes;
        chosen->big_community = best.big_community;
        chosen->blocks_per_sm = best.blocks_per_sm;
        chosen->algorithm = best.algo;
    }
    return QM_OK;
}

}  // extern "C"
