// pc_batch_run_noalloc: the batched kernel with its scratch in a file-scope
// device array instead of memory from cudaMalloc, for callers that may not
// allocate once they are running.  Nothing here allocates: the device
// address of the array is looked up once per device, the scan table is
// copied into it, and the existing batched launch runs on it.
#include <mutex>

#include "pc_internal.h"

namespace {

constexpr size_t kScratchBytes = sizeof(ScanDesc) * PC_NOALLOC_MAX_SCANS;  // the scan table

// Shared by every call on a device; see the contract in include/pc.h.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call per device; host code must not use the symbol itself).
pc_status scratch_on_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pc_from_cuda(e);
    if (dev < 0 || dev >= kMaxDevices) return PC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return pc_from_cuda(e);
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return PC_OK;
}

}  // namespace

extern "C" pc_status pc_batch_run_noalloc(pc_target t, const pc_scan* scans, int n_scans, int k,
                                          float eps, pc_stream s) {
    if (!scans || n_scans < 1 || n_scans > PC_NOALLOC_MAX_SCANS) return PC_ERR_INVALID_ARG;
    if (!t) return PC_ERR_INVALID_ARG;
    if (!pc_target_is_live(t)) return PC_ERR_DESTROYED;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return PC_ERR_CUDA;
    if (prev != t->device && cudaSetDevice(t->device) != cudaSuccess) return PC_ERR_CUDA;
    struct Restore {
        int dev, was;
        ~Restore() {
            if (dev != was) cudaSetDevice(was);
        }
    } restore{t->device, prev};
    // A pageable host-to-device copy cannot be captured: refuse before any
    // other CUDA call, so a caller's capture is left intact.
    cudaStream_t st = (cudaStream_t)s;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return pc_from_cuda(e);
    if (cs != cudaStreamCaptureStatusNone) return PC_ERR_INVALID_ARG;
    ScanDesc table[PC_NOALLOC_MAX_SCANS];
    BatchShape sh;
    pc_status r = pc_batch_table(t, scans, n_scans, k, eps, table, &sh);
    if (r != PC_OK) return r;
    if (sh.tiles == 0) return PC_OK;

    unsigned char* scratch = nullptr;
    if ((r = scratch_on_current_device(&scratch)) != PC_OK) return r;
    auto* table_dev = reinterpret_cast<ScanDesc*>(scratch);
    e = cudaMemcpyAsync(table_dev, table, sizeof(ScanDesc) * n_scans, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = pc_launch_knn_batch(t, t->g, t->ck, table_dev, n_scans, sh.max_n, sh.tiles, sh.tile, sh.warps, k, eps,
                                sh.any_cov, pc_rho0(t, k), st, sh.host_out);
    return pc_from_cuda(e);
}
