// The C ABI of libpc.so (declared in include/pc.h): argument checks, handle
// lifetime, search-radius calibration, host-buffer entry, status word and
// the batched plan with CUDA-graph replay.  No torch types cross it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "pc_internal.h"

namespace {

std::mutex g_mu;
std::set<const void*> g_live;  // live target and batch handles

bool live(const void* h) {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_live.count(h) != 0;
}
void track(const void* h) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_live.insert(h);
}
void untrack(const void* h) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_live.erase(h);
}

// Device (or managed) memory reachable by kernels; host, pinned and
// unregistered pointers are refused.
bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

pc_status check_target(const pc_target_s* t) {
    if (!t) return PC_ERR_INVALID_ARG;
    if (!live(t)) return PC_ERR_DESTROYED;
    return PC_OK;
}

pc_status check_query_args(const pc_target_s* t, int64_t N, int k) {
    if (k < 1 || k > 64 || N < 0) return PC_ERR_INVALID_ARG;
    if ((int64_t)k > t->g.m + t->delta_m) return PC_ERR_K_GT_M;
    if (N > ((int64_t)1 << 40)) return PC_ERR_INVALID_ARG;
    return PC_OK;
}

void default_tune(pc_tune* tu) {
    tu->tile = 32;
    tu->warps = 4;
    tu->rho_scale = 0.9f;
    tu->order = 0;
    tu->probe = 0;
    tu->slots = 0;
}

pc_status read_and_clear_status(pc_target_s* t, cudaStream_t s) {
    int st = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, t->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return pc_from_cuda(e);
    if (st & pcdev::ST_NONFINITE) return PC_ERR_NONFINITE;
    if (st & pcdev::ST_SEARCH_LIMIT) return PC_ERR_SEARCH_LIMIT;
    if (st & pcdev::ST_BAD_INDEX) return PC_ERR_BAD_INDEX;
    if (st & pcdev::ST_SHORT) return PC_ERR_K_GT_M;
    return PC_OK;
}

// First search radius per k: the 75th percentile of the k-th neighbour
// distance over up to 1024 target points used as queries.  It only sets
// where the widening search starts; results never depend on it.
pc_status calibrate_rho(pc_target_s* t, cudaStream_t s) {
    const int64_t M = t->g.m;
    const int kc = (int)std::min<int64_t>(64, M);
    const int64_t S = std::min<int64_t>(M, 1024);
    const int64_t step = M / S;
    float* q = nullptr;
    int32_t* idx = nullptr;
    float* d2 = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(float) * 3 * S);
    if (e == cudaSuccess) e = cudaMalloc(&idx, sizeof(int32_t) * S * kc);
    if (e == cudaSuccess) e = cudaMalloc(&d2, sizeof(float) * S * kc);
    std::vector<float> hd((size_t)S * kc);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(q, 3 * sizeof(float), t->xyz, sizeof(float4) * step, 3 * sizeof(float),
                              S, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = pc_launch_knn(t, q, S, kc, -1.0f, idx, d2, nullptr, t->g.h, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hd.data(), d2, sizeof(float) * S * kc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (q) cudaFree(q);
    if (idx) cudaFree(idx);
    if (d2) cudaFree(d2);
    if (e != cudaSuccess) return pc_from_cuda(e);
    read_and_clear_status(t, s);  // a capped search here only skips that sample
    cudaMemsetAsync(reinterpret_cast<char*>(t->status) + 32, 0, 32, s);
    cudaStreamSynchronize(s);
    std::vector<float> col;
    for (int kk = 0; kk < 64; ++kk) {
        t->rho_hint[kk] = 0.0f;
        if (kk >= kc) continue;
        col.clear();
        for (int64_t n = 0; n < S; ++n) {
            const float v = hd[(size_t)n * kc + kk];
            if (std::isfinite(v)) col.push_back(std::sqrt(v));
        }
        if (col.empty()) continue;
        const size_t pos = (col.size() * 3) / 4;
        std::nth_element(col.begin(), col.begin() + pos, col.end());
        t->rho_hint[kk] = col[pos];
        // spread of the distances at k = min(kc, 16): a map whose density
        // varies widely (a p90 / p25 above 1.55) gets per-query starting radii
        if (kk == std::min(kc, 16) - 1) {
            std::sort(col.begin(), col.end());
            const float p25 = col[col.size() / 4], p90 = col[(col.size() * 9) / 10];
            t->uneven = p25 > 0.0f && p90 > 1.55f * p25 ? 1 : 0;
        }
    }
    return PC_OK;
}

pc_status ensure_stage(pc_target_s* t, size_t bytes) {
    if (t->stage_bytes >= bytes) return PC_OK;
    if (t->stage) {
        cudaFree(t->stage);
        t->stage = nullptr;
        t->stage_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return pc_from_cuda(e);
    t->stage = p;
    t->stage_bytes = bytes;
    return PC_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// A target (grid + calibration) that is not yet a registered handle.
// Builds a target over xyz.  With `like` (the grid of appended points), the
// cell edge and the starting radii are taken from that target instead of
// the cell-size bisection and the calibration search: both grids are then
// searched with one trial radius, and an append costs one grid build.
static pc_status build_target_internal(const float* xyz, int64_t M, const pc_build_opts& o, cudaStream_t st,
                                       pc_target_s** out, const pc_target_s* like = nullptr) {
    pc_target_s* t = new (std::nothrow) pc_target_s();
    if (!t) return PC_ERR_OOM;
    std::memset(t, 0, sizeof(*t));
    t->magic = PC_MAGIC_LIVE;
    cudaGetDevice(&t->device);
    t->opts = o;
    default_tune(&t->tune);
    pc_build_opts ob = o;
    if (like) ob.cell_size = like->g.h;
    pc_status r = pc_build_grid(xyz, M, ob, st, t);
    if (r == PC_OK) {
        if (like) {
            std::memcpy(t->rho_hint, like->rho_hint, sizeof(t->rho_hint));
            t->uneven = like->uneven;
        }
        else r = calibrate_rho(t, st);
    }
    if (r != PC_OK) {
        cudaStreamSynchronize(st);
        pc_free_grid(t);
        delete t;
        return r;
    }
    *out = t;
    return PC_OK;
}

// The search over the target as it stands: its grid, or its grid and the
// delta grid of appended points searched as one map.
static pc_status launch_search(pc_target_s* t, const float* q, int64_t N, int k, float eps, int32_t* idx,
                               float* d2, float* cov, cudaStream_t st, bool stage = false) {
    if (!t->delta) return pc_from_cuda(pc_launch_knn(t, q, N, k, eps, idx, d2, cov, pc_rho0(t, k), st, stage));
    return pc_from_cuda(pc_launch_knn_union(t, q, N, k, eps, idx, d2, cov, pc_rho0(t, k), st));
}

// The device address of page-locked host memory mapped into the device's
// address space (cudaHostAlloc, cudaHostRegister, torch pin_memory), or
// null for any other pointer.
static void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The address kernels use for p: p itself for device (or managed) memory,
// the device address of mapped page-locked host memory (and *host = true),
// null for anything else.
static void* device_view(const void* p, bool* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return const_cast<void*>(p);
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *host = true;
        return a.devicePointer;
    }
    return nullptr;
}

static void free_delta(pc_target_s* t) {
    if (t->delta) {
        pc_free_grid(t->delta);
        delete t->delta;
        t->delta = nullptr;
    }
    if (t->delta_xyz) cudaFree(t->delta_xyz);
    t->delta_xyz = nullptr;
    t->delta_m = t->delta_cap = 0;
}

pc_status pc_from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PC_OK;
    cudaGetLastError();  // clear a non-sticky error
    if (e == cudaErrorMemoryAllocation) return PC_ERR_OOM;
    return PC_ERR_CUDA;
}

bool pc_target_is_live(const pc_target_s* t) { return t != nullptr && live(t); }

bool pc_is_device_ptr(const void* p) { return is_device_ptr(p); }

float pc_probe_c(const pc_target_s* t) {
    const int p = t->tune.probe;
    return (p == 2 || (p == 0 && t->uneven)) ? 1.6f : 0.0f;
}

float pc_rho0(const pc_target_s* t, int k) {
    float r = (k >= 1 && k <= 64) ? t->rho_hint[k - 1] : 0.0f;
    if (!(r > 0.0f)) r = t->g.h;
    const float sc = t->tune.rho_scale > 0 ? t->tune.rho_scale : 0.9f;
    return r * sc;
}

extern "C" {

void pc_default_build_opts(pc_build_opts* o) {
    if (!o) return;
    o->cell_size = 0.0f;
    o->occupancy = 12.0f;
    o->hash_load = 0.5f;
    o->max_box_cells = 4096;
    o->exhaustive = 1;
}

pc_status pc_build_target(const float* xyz_dev, int64_t M, const pc_build_opts* opts, pc_stream s,
                          pc_target* out) {
    if (!out) return PC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!xyz_dev || M < 1 || M >= ((int64_t)1 << 31)) return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(xyz_dev)) return PC_ERR_BAD_POINTER;
    pc_build_opts o;
    pc_default_build_opts(&o);
    if (opts) o = *opts;
    if (o.occupancy <= 0) o.occupancy = 12.0f;
    if (o.hash_load <= 0 || o.hash_load > 0.9f) o.hash_load = 0.5f;
    if (o.max_box_cells <= 0) o.max_box_cells = 4096;
    pc_target_s* t = nullptr;
    pc_status r = build_target_internal(xyz_dev, M, o, (cudaStream_t)s, &t);
    if (r != PC_OK) return r;
    track(t);
    *out = t;
    return PC_OK;
}

void pc_destroy_target(pc_target t) {
    if (!t || !live(t)) return;
    untrack(t);
    DeviceGuard dg(t->device);
    free_delta(t);
    pc_free_grid(t);
    t->magic = PC_MAGIC_DEAD;
    delete t;
}

pc_status pc_set_tune(pc_target t, const pc_tune* tune) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (!tune) {
        default_tune(&t->tune);
        return PC_OK;
    }
    if (tune->tile > 32 || tune->warps > 8 || !(std::isfinite(tune->rho_scale)) || tune->order < 0 ||
        tune->order > 1 || tune->probe < 0 || tune->probe > 2 || (tune->slots != 0 && tune->slots != 64))
        return PC_ERR_INVALID_ARG;
    t->tune = *tune;
    if (t->tune.tile <= 0) t->tune.tile = 32;
    if (t->tune.warps <= 0) t->tune.warps = 4;
    if (t->tune.rho_scale <= 0) t->tune.rho_scale = 0.9f;
    return PC_OK;
}

pc_status pc_get_info(pc_target t, pc_target_info* info) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (!info) return PC_ERR_INVALID_ARG;
    info->m = t->g.m;
    info->ncells = t->g.ncells;
    info->table_cap = t->table_cap;
    info->cell_size = t->g.h;
    info->origin[0] = t->g.ox;
    info->origin[1] = t->g.oy;
    info->origin[2] = t->g.oz;
    for (int a = 0; a < 3; ++a) info->bbox_max[a] = t->bbox_max[a];
    info->dims[0] = t->g.dimx;
    info->dims[1] = t->g.dimy;
    info->dims[2] = t->g.dimz;
    info->device_bytes = t->device_bytes + (int64_t)t->stage_bytes +
                         (t->delta ? t->delta->device_bytes : 0) + (int64_t)sizeof(float) * 3 * t->delta_cap;
    for (int i = 0; i < 64; ++i) info->rho_hint[i] = t->rho_hint[i];
    info->delta_m = t->delta_m;
    return PC_OK;
}

pc_status pc_knn(pc_target t, const float* q_dev, int64_t N, int k, int32_t* idx_dev,
                 float* d2_dev, pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if ((r = check_query_args(t, N, k)) != PC_OK) return r;
    if (N == 0) return PC_OK;
    if (!q_dev || !idx_dev || !d2_dev) return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(q_dev) || !is_device_ptr(idx_dev) || !is_device_ptr(d2_dev))
        return PC_ERR_BAD_POINTER;
    DeviceGuard dg(t->device);
    return launch_search(t, q_dev, N, k, -1.0f, idx_dev, d2_dev, nullptr, (cudaStream_t)s);
}

pc_status pc_cov(pc_target t, const int32_t* idx_dev, int64_t N, int k, float eps, float* cov_dev,
                 pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (k < 1 || k > 64 || N < 0 || !std::isfinite(eps)) return PC_ERR_INVALID_ARG;
    if (N == 0) return PC_OK;
    if (!idx_dev || !cov_dev) return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(idx_dev) || !is_device_ptr(cov_dev)) return PC_ERR_BAD_POINTER;
    DeviceGuard dg(t->device);
    if (t->delta) return pc_from_cuda(pc_launch_cov_union(t, idx_dev, N, k, eps, cov_dev, (cudaStream_t)s));
    return pc_from_cuda(pc_launch_cov(t, idx_dev, N, k, eps, cov_dev, (cudaStream_t)s));
}

pc_status pc_knn_cov(pc_target t, const float* q_dev, int64_t N, int k, float eps,
                     int32_t* idx_dev, float* d2_dev, float* cov_dev, pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if ((r = check_query_args(t, N, k)) != PC_OK) return r;
    if (!std::isfinite(eps)) return PC_ERR_INVALID_ARG;
    if (N == 0) return PC_OK;
    if (!q_dev || !idx_dev || !d2_dev || !cov_dev) return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(q_dev) || !is_device_ptr(idx_dev) || !is_device_ptr(d2_dev) ||
        !is_device_ptr(cov_dev))
        return PC_ERR_BAD_POINTER;
    DeviceGuard dg(t->device);
    return launch_search(t, q_dev, N, k, eps, idx_dev, d2_dev, cov_dev, (cudaStream_t)s);
}

pc_status pc_knn_cov_host(pc_target t, const float* q_host, int64_t N, int k, float eps,
                          int32_t* idx_host, float* d2_host, float* cov_host, pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if ((r = check_query_args(t, N, k)) != PC_OK) return r;
    if (!std::isfinite(eps)) return PC_ERR_INVALID_ARG;
    if (N == 0) return PC_OK;
    if (!q_host || !idx_host || !d2_host || !cov_host) return PC_ERR_INVALID_ARG;
    DeviceGuard dg(t->device);
    cudaStream_t st = (cudaStream_t)s;
    // Page-locked outputs (k <= 32, no appended points): the search writes
    // them in place, each warp's rows as one block, so the transfer runs
    // during the search; a page-locked q is read in place too.
    void* const mi = (k <= 32 && !t->delta) ? mapped_host(idx_host) : nullptr;
    void* const md = mi ? mapped_host(d2_host) : nullptr;
    void* const mc = md ? mapped_host(cov_host) : nullptr;
    if (mc) {
        const float* q = static_cast<const float*>(mapped_host(q_host));
        if (!q) {
            if ((r = ensure_stage(t, align256(sizeof(float) * 3 * N))) != PC_OK) return r;
            float* qs = static_cast<float*>(t->stage);
            const cudaError_t e = cudaMemcpyAsync(qs, q_host, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return pc_from_cuda(e);
            q = qs;
        }
        r = launch_search(t, q, N, k, eps, static_cast<int32_t*>(mi), static_cast<float*>(md),
                          static_cast<float*>(mc), st, true);
        if (r != PC_OK) return r;
        return read_and_clear_status(t, st);
    }
    const size_t bq = align256(sizeof(float) * 3 * N), bi = align256(sizeof(int32_t) * N * k),
                 bd = align256(sizeof(float) * N * k), bc = align256(sizeof(float) * 6 * N);
    if ((r = ensure_stage(t, bq + bi + bd + bc)) != PC_OK) return r;
    char* base = static_cast<char*>(t->stage);
    float* q = reinterpret_cast<float*>(base);
    int32_t* idx = reinterpret_cast<int32_t*>(base + bq);
    float* d2 = reinterpret_cast<float*>(base + bq + bi);
    float* cov = reinterpret_cast<float*>(base + bq + bi + bd);
    cudaError_t e = cudaMemcpyAsync(q, q_host, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        r = launch_search(t, q, N, k, eps, idx, d2, cov, st);
        if (r != PC_OK) return r;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(idx_host, idx, sizeof(int32_t) * N * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d2_host, d2, sizeof(float) * N * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cov_host, cov, sizeof(float) * 6 * N, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return pc_from_cuda(e);
    return read_and_clear_status(t, st);
}

pc_status pc_sync_status(pc_target t, pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    DeviceGuard dg(t->device);
    return read_and_clear_status(t, (cudaStream_t)s);
}

pc_status pc_get_stats(pc_target t, pc_stream s, pc_stats* out, int reset) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (!out) return PC_ERR_INVALID_ARG;
    DeviceGuard dg(t->device);
    cudaStream_t st = (cudaStream_t)s;
    unsigned long long v[4] = {0, 0, 0, 0};
    char* base = reinterpret_cast<char*>(t->status) + 32;
    cudaError_t e = cudaMemcpyAsync(v, base, sizeof(v), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(base, 0, sizeof(v), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pc_from_cuda(e);
    out->queries = (int64_t)v[0];
    out->warp_search = (int64_t)v[1];
    out->exhaustive = (int64_t)v[2];
    out->candidates = (int64_t)v[3];
    return PC_OK;
}

pc_status pc_batch_plan(pc_target t, const pc_scan* scans, int n_scans, int k, float eps,
                        pc_batch* out) {
    if (!out) return PC_ERR_INVALID_ARG;
    *out = nullptr;
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (!scans || n_scans < 1) return PC_ERR_INVALID_ARG;
    std::vector<ScanDesc> hs(n_scans);
    BatchShape sh;
    if ((r = pc_batch_table(t, scans, n_scans, k, eps, hs.data(), &sh)) != PC_OK) return r;
    DeviceGuard dg(t->device);
    pc_batch_s* b = new (std::nothrow) pc_batch_s();
    if (!b) return PC_ERR_OOM;
    std::memset(b, 0, sizeof(*b));
    b->magic = PC_MAGIC_LIVE;
    b->t = t;
    b->g = t->g;
    b->ck = t->ck;
    b->n_scans = n_scans;
    b->k = k;
    b->eps = eps;
    b->with_cov = sh.any_cov;
    b->host_out = sh.host_out;
    b->tile = sh.tile;
    b->warps = sh.warps;
    b->max_n = sh.max_n;
    b->total_tiles = sh.tiles;
    int64_t queries = 0;
    for (int i = 0; i < n_scans; ++i) queries += scans[i].n;
    b->total_queries = queries;
    cudaError_t e = pc_knn_prepare();
    if (e == cudaSuccess) e = cudaMalloc(&b->scans_dev, sizeof(ScanDesc) * n_scans);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->scans_dev, hs.data(), sizeof(ScanDesc) * n_scans, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (b->scans_dev) cudaFree(b->scans_dev);
        delete b;
        return pc_from_cuda(e);
    }
    track(b);
    *out = b;
    return PC_OK;
}

pc_status pc_batch_run(pc_batch b, pc_stream s) {
    if (!b) return PC_ERR_INVALID_ARG;
    if (!live(b)) return PC_ERR_DESTROYED;
    if (!live(b->t)) return PC_ERR_DESTROYED;
    if (b->t->delta || b->t->g.table != b->g.table) return PC_ERR_INVALID_ARG;  // the target changed since planning
    if (b->total_tiles == 0) return PC_OK;
    DeviceGuard dg(b->t->device);
    cudaStream_t st = (cudaStream_t)s;
    const float rho0 = pc_rho0(b->t, b->k);
    if (st == nullptr)  // the legacy stream cannot be captured: launch directly
        return pc_from_cuda(pc_launch_knn_batch(b->t, b->g, b->ck, b->scans_dev, b->n_scans, b->max_n,
                                                b->total_tiles, b->tile, b->warps, b->k, b->eps, b->with_cov,
                                                rho0, st, b->host_out));
    if (!b->exec || b->captured_on != st) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return pc_from_cuda(e);
        cudaError_t e2 = pc_launch_knn_batch(b->t, b->g, b->ck, b->scans_dev, b->n_scans, b->max_n, b->total_tiles,
                                             b->tile, b->warps, b->k, b->eps, b->with_cov, rho0, st, b->host_out);
        e = cudaStreamEndCapture(st, &b->graph);
        if (e2 != cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            if (b->graph) cudaGraphDestroy(b->graph);
            b->graph = nullptr;
            b->exec = nullptr;
            return pc_from_cuda(e);
        }
        b->captured_on = st;
    }
    return pc_from_cuda(cudaGraphLaunch(b->exec, st));
}

}  // extern "C"

// Checks shared by the batched entries that run on caller-provided scans
// (pc_batch_run_scratch, pc_batch_run_noalloc) and the scan table they
// copy to the device: a live target without appended points, 1 <= k <= 64,
// k <= M, finite eps, every non-empty scan's buffers in device memory.
pc_status pc_batch_table(const pc_target_s* t, const pc_scan* scans, int n_scans, int k, float eps,
                         ScanDesc* table, BatchShape* shape) {
    if (!t) return PC_ERR_INVALID_ARG;
    if (!live(t)) return PC_ERR_DESTROYED;
    if (!scans || n_scans < 1 || k < 1 || k > 64 || !std::isfinite(eps)) return PC_ERR_INVALID_ARG;
    if (t->delta) return PC_ERR_INVALID_ARG;  // appended points: pc_target_compact first
    if ((int64_t)k > t->g.m) return PC_ERR_K_GT_M;
    BatchShape sh;
    sh.tile = std::min(std::max(t->tune.tile, 1), 32);
    sh.warps = std::min(std::max(t->tune.warps, 1), 8);
    sh.tiles = 0;
    sh.max_n = 0;
    sh.any_cov = false;
    sh.host_out = false;
    for (int i = 0; i < n_scans; ++i) {
        const pc_scan& sc = scans[i];
        if (sc.n < 0) return PC_ERR_INVALID_ARG;
        const void* q = sc.q_dev;
        void *idx = sc.idx_dev, *d2 = sc.d2_dev, *cov = sc.cov_dev;
        if (sc.n > 0) {
            if (!sc.q_dev || !sc.idx_dev || !sc.d2_dev) return PC_ERR_INVALID_ARG;
            bool host_q = false;
            q = device_view(sc.q_dev, &host_q);
            idx = device_view(sc.idx_dev, &sh.host_out);
            d2 = device_view(sc.d2_dev, &sh.host_out);
            if (!q || !idx || !d2) return PC_ERR_BAD_POINTER;
            if (sc.cov_dev) {
                if (!(cov = device_view(sc.cov_dev, &sh.host_out))) return PC_ERR_BAD_POINTER;
                sh.any_cov = true;
            }
        }
        table[i].q = static_cast<const float*>(q);
        table[i].n = sc.n;
        table[i].idx = static_cast<int32_t*>(idx);
        table[i].d2 = static_cast<float*>(d2);
        table[i].cov = static_cast<float*>(cov);
        table[i].tile0 = sh.tiles;
        sh.tiles += (sc.n + sh.tile - 1) / sh.tile;
        sh.max_n = std::max<int64_t>(sh.max_n, sc.n);
    }
    *shape = sh;
    return PC_OK;
}

extern "C" {

size_t pc_batch_scratch_bytes(int n_scans) {
    if (n_scans < 1) return 0;
    return sizeof(ScanDesc) * (size_t)n_scans;
}

pc_status pc_batch_run_scratch(pc_target t, const pc_scan* scans, int n_scans, int k, float eps,
                               void* scratch_dev, size_t scratch_bytes, pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (!scans || n_scans < 1) return PC_ERR_INVALID_ARG;
    std::vector<ScanDesc> hs(n_scans);
    BatchShape sh;
    if ((r = pc_batch_table(t, scans, n_scans, k, eps, hs.data(), &sh)) != PC_OK) return r;
    if (!scratch_dev || (reinterpret_cast<uintptr_t>(scratch_dev) & 255u) ||
        scratch_bytes < pc_batch_scratch_bytes(n_scans))
        return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(scratch_dev)) return PC_ERR_BAD_POINTER;
    if (sh.tiles == 0) return PC_OK;
    DeviceGuard dg(t->device);
    cudaStream_t st = (cudaStream_t)s;
    auto* table = static_cast<ScanDesc*>(scratch_dev);
    cudaError_t e = cudaMemcpyAsync(table, hs.data(), sizeof(ScanDesc) * n_scans,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = pc_launch_knn_batch(t, t->g, t->ck, table, n_scans, sh.max_n, sh.tiles, sh.tile, sh.warps, k, eps,
                                sh.any_cov, pc_rho0(t, k), st, sh.host_out);
    return pc_from_cuda(e);
}

void pc_batch_destroy(pc_batch b) {
    if (!b || !live(b)) return;
    untrack(b);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->scans_dev) cudaFree(b->scans_dev);
    b->magic = PC_MAGIC_DEAD;
    delete b;
}

// The cell rule of the grid on the host (same binary32 operations as
// pcdev::cell_of: a subtraction, a product, floor, clamp).
static int host_cell_of(float v, float o, float inv_h) {
    float t = (v - o) * inv_h;
    t = std::floor(t);
    t = std::fmin(std::fmax(t, -1073741824.0f), 1073741824.0f);
    return (int)t;
}

// The window of t->win onto one grid (the main one or the delta's).
static void apply_window(const pc_target_s* t, pcdev::Grid& g, const float* bbox_max) {
    pc_clear_window(g);
    if (!t->has_win) return;
    const pc_window* w = &t->win;
    const float o[3] = {g.ox, g.oy, g.oz};
    const int dim[3] = {g.dimx, g.dimy, g.dimz};
    int lo[3], hi[3], tl[3], th[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = std::max(host_cell_of(w->lo[a], o[a], g.inv_h), 0);
        hi[a] = std::min(host_cell_of(w->hi[a], o[a], g.inv_h), dim[a] - 1);
        // boundary cells whose points can fall outside the box: only where
        // the bound lies inside the grid's bounding box [origin, bbox_max]
        tl[a] = w->lo[a] > o[a] ? lo[a] : -1;
        th[a] = w->hi[a] < bbox_max[a] ? hi[a] : -1;
    }
    g.windowed = 1;
    g.wlx = lo[0];
    g.whx = hi[0];
    g.wly = lo[1];
    g.why = hi[1];
    g.wlz = lo[2];
    g.whz = hi[2];
    g.tlx = tl[0];
    g.thx = th[0];
    g.tly = tl[1];
    g.thy = th[1];
    g.tlz = tl[2];
    g.thz = th[2];
    g.wlox = w->lo[0];
    g.wloy = w->lo[1];
    g.wloz = w->lo[2];
    g.whix = w->hi[0];
    g.whiy = w->hi[1];
    g.whiz = w->hi[2];
}

pc_status pc_set_window(pc_target t, const pc_window* w) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (w)
        for (int a = 0; a < 3; ++a)
            if (std::isnan(w->lo[a]) || std::isnan(w->hi[a]) || !(w->lo[a] <= w->hi[a]))
                return PC_ERR_INVALID_ARG;
    t->has_win = w ? 1 : 0;
    if (w) t->win = *w;
    apply_window(t, t->g, t->bbox_max);
    if (t->delta) apply_window(t, t->delta->g, t->delta->bbox_max);
    return PC_OK;
}

pc_status pc_target_append(pc_target t, const float* xyz_dev, int64_t n, pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (n < 0) return PC_ERR_INVALID_ARG;
    if (n == 0) return PC_OK;
    if (!xyz_dev) return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(xyz_dev)) return PC_ERR_BAD_POINTER;
    const int64_t tot = t->delta_m + n;
    if (t->g.m + tot >= ((int64_t)1 << 31)) return PC_ERR_INVALID_ARG;
    DeviceGuard dg(t->device);
    cudaStream_t st = (cudaStream_t)s;
    if (tot > t->delta_cap) {  // grow the appended-points array (doubling)
        const int64_t cap = std::max<int64_t>(tot, 2 * t->delta_cap);
        float* p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(float) * 3 * cap);
        if (e != cudaSuccess) return pc_from_cuda(e);
        if (t->delta_m > 0)
            e = cudaMemcpyAsync(p, t->delta_xyz, sizeof(float) * 3 * t->delta_m, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFree(p);
            return pc_from_cuda(e);
        }
        if (t->delta_xyz) cudaFree(t->delta_xyz);
        t->delta_xyz = p;
        t->delta_cap = cap;
    }
    cudaError_t e = cudaMemcpyAsync(t->delta_xyz + 3 * t->delta_m, xyz_dev, sizeof(float) * 3 * n,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return pc_from_cuda(e);
    // the delta grid over every appended point (the main grid is untouched)
    pc_target_s* d = nullptr;
    r = build_target_internal(t->delta_xyz, tot, t->opts, st, &d, t);
    if (r != PC_OK) return r;  // e.g. a non-finite point: nothing appended
    d->tune = t->tune;
    d->g.status = t->g.status;  // conditions of the delta search report on the handle
    d->g.stats = t->g.stats;
    if (t->delta) {
        pc_free_grid(t->delta);
        delete t->delta;
    }
    t->delta = d;
    t->delta_m = tot;
    apply_window(t, d->g, d->bbox_max);
    return PC_OK;
}

pc_status pc_target_compact(pc_target t, pc_stream s) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    if (!t->delta) return PC_OK;
    DeviceGuard dg(t->device);
    cudaStream_t st = (cudaStream_t)s;
    const int64_t tot = t->g.m + t->delta_m;
    float* all = nullptr;
    cudaError_t e = cudaMalloc(&all, sizeof(float) * 3 * tot);
    if (e != cudaSuccess) return pc_from_cuda(e);
    e = pc_launch_pack_xyz(t, all, st);
    pc_target_s* n = nullptr;
    if (e == cudaSuccess) r = build_target_internal(all, tot, t->opts, st, &n);
    else r = pc_from_cuda(e);
    cudaStreamSynchronize(st);
    cudaFree(all);
    if (r != PC_OK) return r;
    // the handle keeps its identity and settings; its grid is the new one
    pc_free_grid(t);
    t->g = n->g;
    t->bbox_max[0] = n->bbox_max[0];
    t->bbox_max[1] = n->bbox_max[1];
    t->bbox_max[2] = n->bbox_max[2];
    std::memcpy(t->rho_hint, n->rho_hint, sizeof(t->rho_hint));
    t->table_cap = n->table_cap;
    t->device_bytes = n->device_bytes;
    t->table = n->table;
    t->pts = n->pts;
    t->xyz = n->xyz;
    t->cell_keys = n->cell_keys;
    t->cell_start = n->cell_start;
    t->dstart = n->dstart;
    t->xcut = n->xcut;
    t->status = n->status;
    delete n;  // its buffers now belong to t
    free_delta(t);
    apply_window(t, t->g, t->bbox_max);
    if (t->ck.type != 0) {  // the polynomial/HI origin follows the new bounding box
        t->ck.ox = t->g.ox;
        t->ck.oy = t->g.oy;
        t->ck.oz = t->g.oz;
    }
    return PC_OK;
}

pc_status pc_set_cov_kernel(pc_target t, const pc_cov_kernel* kd) {
    pc_status r = check_target(t);
    if (r != PC_OK) return r;
    CovKernel ck{};
    if (kd && kd->type != PC_KERNEL_NONE) {
        if (kd->type < PC_KERNEL_RBF || kd->type > PC_KERNEL_LAPLACIAN) return PC_ERR_INVALID_ARG;
        if (!std::isfinite(kd->sigma) || !std::isfinite(kd->alpha) || !std::isfinite(kd->c) ||
            !std::isfinite(kd->d))
            return PC_ERR_INVALID_ARG;
        const double sg = kd->sigma;
        ck.type = kd->type;
        switch (kd->type) {
            case PC_KERNEL_RBF:
                if (!(sg >= 0)) return PC_ERR_INVALID_ARG;
                ck.s = (float)sg;
                break;
            case PC_KERNEL_GAUSSIAN:
                if (!(sg > 0)) return PC_ERR_INVALID_ARG;
                ck.s = (float)(1.0 / (2.0 * sg * sg));
                break;
            case PC_KERNEL_LAPLACIAN:
                if (!(sg > 0)) return PC_ERR_INVALID_ARG;
                ck.s = (float)(1.0 / sg);
                break;
            default:
                break;
        }
        ck.alpha = kd->alpha;
        ck.c = kd->c;
        ck.d = kd->d;
        ck.ox = t->g.ox;
        ck.oy = t->g.oy;
        ck.oz = t->g.oz;
    }
    t->ck = ck;
    return PC_OK;
}

size_t pc_gicp_work_bytes(void) { return pc_gicp_work_size(); }

pc_status pc_gicp_linearize(pc_target map, const float* map_cov_dev, const float* src_dev,
                            int64_t n, const float* src_cov_dev, const float* pose_dev,
                            float max_dist, double* out_dev, int32_t* corr_dev, void* work_dev,
                            size_t work_bytes, pc_stream s) {
    pc_status r = check_target(map);
    if (r != PC_OK) return r;
    if (n < 0 || n > ((int64_t)1 << 40) || !(max_dist >= 0.0f)) return PC_ERR_INVALID_ARG;
    if (!out_dev || (reinterpret_cast<uintptr_t>(out_dev) & 7u)) return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(out_dev)) return PC_ERR_BAD_POINTER;
    if (n == 0) {  // nothing to pair: all sums zero (the inputs may be empty tensors)
        DeviceGuard dg(map->device);
        return pc_from_cuda(cudaMemsetAsync(out_dev, 0, PC_GICP_OUT * sizeof(double), (cudaStream_t)s));
    }
    if (!map_cov_dev || !src_dev || !src_cov_dev || !pose_dev || !work_dev) return PC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(out_dev) & 7u) || (reinterpret_cast<uintptr_t>(work_dev) & 255u))
        return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(map_cov_dev) || !is_device_ptr(src_dev) || !is_device_ptr(src_cov_dev) ||
        !is_device_ptr(pose_dev) || !is_device_ptr(out_dev) || !is_device_ptr(work_dev) ||
        (corr_dev && !is_device_ptr(corr_dev)))
        return PC_ERR_BAD_POINTER;
    DeviceGuard dg(map->device);
    const size_t need = pc_gicp_work_size();
    if (need == 0) return PC_ERR_CUDA;
    if (work_bytes < need) return PC_ERR_INVALID_ARG;
    // start radius: the calibrated distance to the nearest other map point
    float r0 = pc_rho0(map, map->g.m >= 2 ? 2 : 1);
    if (!(r0 > 0.0f)) r0 = map->g.h;
    float r0d = r0;
    if (map->delta) {
        r0d = pc_rho0(map->delta, map->delta->g.m >= 2 ? 2 : 1);
        if (!(r0d > 0.0f)) r0d = map->delta->g.h;
    }
    return pc_from_cuda(pc_launch_gicp_linearize(map, map_cov_dev, src_dev, n, src_cov_dev, pose_dev,
                                                 max_dist, out_dev, corr_dev, work_dev, r0, r0d,
                                                 (cudaStream_t)s));
}

pc_status pc_gicp_update(const double* lin_dev, float lambda, float* pose_dev, double* xi_dev,
                         pc_stream s) {
    if (!lin_dev || !pose_dev || !(lambda >= 0.0f)) return PC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(lin_dev) & 7u) || (reinterpret_cast<uintptr_t>(xi_dev) & 7u) ||
        (reinterpret_cast<uintptr_t>(pose_dev) & 3u))
        return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(lin_dev) || !is_device_ptr(pose_dev) || (xi_dev && !is_device_ptr(xi_dev)))
        return PC_ERR_BAD_POINTER;
    return pc_from_cuda(pc_launch_gicp_update(lin_dev, lambda, pose_dev, xi_dev, (cudaStream_t)s));
}

const char* pc_status_string(pc_status st) {
    switch (st) {
        case PC_OK: return "ok";
        case PC_ERR_INVALID_ARG: return "invalid argument";
        case PC_ERR_K_GT_M: return "k larger than the target size";
        case PC_ERR_NONFINITE: return "non-finite coordinate";
        case PC_ERR_OOM: return "device allocation failed";
        case PC_ERR_CUDA: return "CUDA runtime error";
        case PC_ERR_SEARCH_LIMIT: return "search reached max_box_cells (exhaustive scan disabled)";
        case PC_ERR_BAD_POINTER: return "pointer is not device memory";
        case PC_ERR_BAD_INDEX: return "neighbour index outside the target";
        case PC_ERR_DESTROYED: return "handle destroyed or never built";
    }
    return "unknown status";
}

const char* pc_version(void) { return "pc 0.1 sm_103a"; }

}  // extern "C"
