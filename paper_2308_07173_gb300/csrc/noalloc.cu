// pc_batch_run_noalloc: the batched kernel with its scratch in a file-scope
// device array instead of memory from cudaMalloc, for callers that may not
// allocate once they are running.  Nothing here allocates: the device
// address of the array is looked up once per device, the scan table is
// copied into it, and the existing batched launch runs on it.
#include <cmath>
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
    if (!t) return PC_ERR_INVALID_ARG;
    if (!pc_target_is_live(t)) return PC_ERR_DESTROYED;
    if (!scans || n_scans < 1 || n_scans > PC_NOALLOC_MAX_SCANS) return PC_ERR_INVALID_ARG;
    if (k < 1 || k > 64 || !std::isfinite(eps)) return PC_ERR_INVALID_ARG;
    if (t->delta) return PC_ERR_INVALID_ARG;  // appended points: pc_target_compact first
    if ((int64_t)k > t->g.m) return PC_ERR_K_GT_M;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return PC_ERR_CUDA;
    if (prev != t->device && cudaSetDevice(t->device) != cudaSuccess) return PC_ERR_CUDA;
    struct Restore {
        int dev, was;
        ~Restore() {
            if (dev != was) cudaSetDevice(was);
        }
    } restore{t->device, prev};

    bool any_cov = false;
    for (int i = 0; i < n_scans; ++i) {
        const pc_scan& sc = scans[i];
        if (sc.n < 0) return PC_ERR_INVALID_ARG;
        if (sc.n == 0) continue;
        if (!sc.q_dev || !sc.idx_dev || !sc.d2_dev) return PC_ERR_INVALID_ARG;
        if (!pc_is_device_ptr(sc.q_dev) || !pc_is_device_ptr(sc.idx_dev) ||
            !pc_is_device_ptr(sc.d2_dev))
            return PC_ERR_BAD_POINTER;
        if (sc.cov_dev) {
            if (!pc_is_device_ptr(sc.cov_dev)) return PC_ERR_BAD_POINTER;
            any_cov = true;
        }
    }
    const int tile = t->tune.tile < 1 ? 32 : (t->tune.tile > 32 ? 32 : t->tune.tile);
    const int warps = t->tune.warps < 1 ? 4 : (t->tune.warps > 8 ? 8 : t->tune.warps);
    ScanDesc table[PC_NOALLOC_MAX_SCANS];
    int64_t tiles = 0, max_n = 0;
    for (int i = 0; i < n_scans; ++i) {
        table[i].q = scans[i].q_dev;
        table[i].n = scans[i].n;
        table[i].idx = scans[i].idx_dev;
        table[i].d2 = scans[i].d2_dev;
        table[i].cov = scans[i].cov_dev;
        table[i].tile0 = tiles;
        tiles += (scans[i].n + tile - 1) / tile;
        if (scans[i].n > max_n) max_n = scans[i].n;
    }
    if (tiles == 0) return PC_OK;

    unsigned char* scratch = nullptr;
    pc_status r = scratch_on_current_device(&scratch);
    if (r != PC_OK) return r;
    cudaStream_t st = (cudaStream_t)s;
    auto* table_dev = reinterpret_cast<ScanDesc*>(scratch);
    cudaError_t e = cudaMemcpyAsync(table_dev, table, sizeof(ScanDesc) * n_scans,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = pc_launch_knn_batch(t, t->g, t->ck, table_dev, n_scans, max_n, tiles, tile, warps, k, eps, any_cov,
                                pc_rho0(t, k), st);
    return pc_from_cuda(e);
}
