// qm_noalloc.cu -- qm_score_partition_noalloc: the plain scoring call without
// any memory allocation.
//
// Some hosts cannot let a library allocate at call time.  An application that
// reserves all of its GPU memory up front and lends a plugin no allocator, or a
// latency-critical loop that must never pay for the device-wide synchronisation
// and the page-table work that cudaMalloc and cudaFree can bring, can still
// score partitions through this entry point.  Its scratch memory is one
// file-scope device array of QM_NOALLOC_SCRATCH_BYTES that every GPU which loads
// the library keeps until the process exits; results are copied straight into
// the caller's struct.  Nothing here calls cudaMalloc, cudaFree, cudaMallocHost
// or any other allocating routine.
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "qm_internal.h"

namespace {

constexpr size_t kScratchBytes = QM_NOALLOC_SCRATCH_BYTES;

// The scratch array.  In host code this name is only a stand-in for the device
// symbol; kernels receive the address that cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char qm_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
    void *scratch = nullptr;  // device address of qm_noalloc_scratch on this device
    int num_sms = 0;
    qm::Shape shape{};
};

std::mutex g_mu;
std::map<int, DeviceSetup> g_setup;

qm_status noalloc_fail(qm_status s, const std::string &m)
{
    return qm::set_error(s, m.c_str());  // reported by qm_last_error()
}

// Once per device, with that device current: resolve the scratch address and
// prepare the kernels' launch shape.  Runs on the first call on the device.
qm_status device_setup(int dev, DeviceSetup *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_setup.find(dev);
    if (it != g_setup.end()) {
        *out = it->second;
        return QM_OK;
    }
    DeviceSetup s;
    cudaError_t e = cudaGetSymbolAddress(&s.scratch, qm_noalloc_scratch);
    if (e != cudaSuccess || !s.scratch) {
        cudaGetLastError();
        return noalloc_fail(QM_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    }
    e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || s.num_sms < 1) {
        cudaGetLastError();
        return noalloc_fail(QM_ECUDA, "cudaDeviceGetAttribute(multiprocessor count) failed");
    }
    qm::prepare_kernels();
    s.shape.threads = 512;
    s.shape.smem_bytes = 96 * 1024;
    s.shape.big_community = 48;
    s.shape.blocks_per_sm = qm::score_blocks_per_sm(s.shape);
    if (s.shape.blocks_per_sm < 1) s.shape.blocks_per_sm = 1;
    if (cudaGetLastError() != cudaSuccess) return noalloc_fail(QM_ECUDA, "kernel set-up failed");
    g_setup[dev] = s;
    *out = s;
    return QM_OK;
}

}  // namespace

extern "C" qm_status qm_score_partition_noalloc(const qm_graph *g, const int32_t *labels, int32_t K,
                                                qm_quality *out, void *stream)
{
    qm::GraphDev gd;
    int dev = -1;
    if (!g || !labels || !out) return noalloc_fail(QM_EINVAL, "null argument");
    if (K < 1) return noalloc_fail(QM_EINVAL, "K must be >= 1");
    if (qm::graph_device_view(g, &gd, &dev) != QM_OK) return noalloc_fail(QM_EINVAL, "bad graph handle");
    if (gd.wt) return noalloc_fail(QM_EINVAL, "weighted graphs are scored by qm_score_partition and the sharded calls");
    const size_t ws_bytes = qm::score_ws_bytes(gd.n, K);
    // a renumbered graph (QM_REORDER) also needs room for the gathered labels
    const size_t need = ws_bytes + (gd.inv ? ((size_t)gd.n * 4 + 255) / 256 * 256 : 0);
    if (need > kScratchBytes)
        return noalloc_fail(QM_EOVERFLOW, "graph and label count need " + std::to_string(need) +
                                              " bytes of scratch; the allocation-free call has " +
                                              std::to_string(kScratchBytes) + " (about 4 n + 36 K bytes fit, 8 n + 36 K for a graph loaded with QM_REORDER)");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    struct Restore {
        int prev, dev;
        ~Restore()
        {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, dev};
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, labels) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return noalloc_fail(QM_EINVAL, "labels must be device memory for the allocation-free call");
    }
    // the kernels read the labels directly: they must live on the graph's GPU
    if (pa.device != dev)
        return noalloc_fail(QM_EINVAL, "labels must be on the graph's GPU (device " + std::to_string(dev) +
                                           ", labels on device " + std::to_string(pa.device) + ")");
    DeviceSetup s;
    qm_status st = device_setup(dev, &s);
    if (st != QM_OK) return st;

    cudaStream_t cs = (cudaStream_t)stream;
    const qm::ScoreWs w = qm::carve_score_ws(s.scratch, gd.n, K);
    // counters, accumulators, status and the histogram must start at zero; the
    // rest of the array is fully written before it is read
    cudaError_t e = cudaMemsetAsync(s.scratch, 0, w.zero_bytes, cs);
    if (e != cudaSuccess) return noalloc_fail(QM_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int32_t *dl = labels;
    if (gd.inv) {
        int32_t *pl = (int32_t *)((char *)s.scratch + ws_bytes);
        if (qm::launch_permute_labels(labels, gd.inv, gd.n, 1, pl, s.num_sms, cs) < 0) {
            e = cudaGetLastError();
            return noalloc_fail(QM_ECUDA, std::string("label permutation: ") + cudaGetErrorString(e));
        }
        dl = pl;
    }
    if (qm::launch_score(gd, dl, K, w, s.shape, nullptr, s.num_sms, cs, nullptr) < 0) {
        e = cudaGetLastError();
        return noalloc_fail(QM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    int status = 0;
    qm_quality result;
    e = cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&result, w.result, sizeof(qm_quality), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return noalloc_fail(QM_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
    if (status & 1) return noalloc_fail(QM_EINVAL, "a label lies outside [0, K)");
    if (status & 2) return noalloc_fail(QM_EOVERFLOW, "a community borders too many distinct communities");
    if (status & 4) return noalloc_fail(QM_ETIMEOUT, "a bounded device wait expired");
    if (status) return noalloc_fail(QM_ECUDA, "device status " + std::to_string(status));
    std::memcpy(out, &result, sizeof(qm_quality));
    return QM_OK;
}
