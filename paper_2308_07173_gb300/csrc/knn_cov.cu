// Nearest-points search and neighbourhood covariance on sm_103a CUDA cores
// (Sec. III-C1 "Efficient registration method": the per-point covariances
// C_i of Eq. 19 need every point's k nearest neighbours and the covariance
// of that neighbourhood -- the step the paper moves from CPU to GPU).
//
// Exactness rests on one fact, certified_tau: for a box of cells around q,
// every target point outside the box has a binary32 d2 above a computable
// tau, so any radius t with t^2 <= tau that holds >= k points holds the k
// nearest.  Two searches use it:
//
// * Lane path (k <= 32; lane_tile) -- one query per lane of a 32-query
//   tile.  Pass 1 walks the rows of the box (occupancy bitmap + rank, one
//   contiguous point range per row) and counts points under eight trial
//   radii; the smallest radius holding >= k (and <= the survivor cap)
//   wins, a failing lane retries with the radii scaled, and pass 2
//   collects the winners' positions in shared memory.  A register odd-even
//   merge sort network sorts 32-bit keys (d2 bits with a slot tag), an exact fix-up
//   orders equal buckets by (d2, index), and the covariance reads the k
//   neighbours from the cell-sorted copy in rank order.
// * Warp path (k > 32, and the lane path's leftovers; knn_search) -- one
//   query per warp: the cells of a radius-driven box are looked up in the
//   voxel hash one per lane, candidates arrive 32 at a time as coalesced
//   float4 loads, survivors of the certified filter are merged into a
//   register top-k by bitonic shuffles, and the radius widens until k are
//   certified; past max_box_cells an exact scan over all occupied cells
//   (or PC_ERR_SEARCH_LIMIT) ends it.
//
// The covariance is a two-pass binary32 mean/centred sum shifted by the
// nearest neighbour; for eps >= 0 a binary32 Jacobi eigen-solve gives the
// normal n and C' = I - (1-eps) n n^T.  Nothing here changes a result bit
// with the tile, launch shape, radii, tile order or batching.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "knn_kernels.cuh"

// ---------------------------------------------------------------- host side
namespace {

// Opt every search kernel (both window variants) into large dynamic shared
// memory, once per device (outside any stream capture: the first launch or
// plan does it).
std::mutex g_attr_mu;
unsigned g_attr_done = 0u;
cudaError_t ensure_attrs() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned bit = 1u << (dev & 31);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (g_attr_done & bit) return cudaSuccess;
    if ((e = allow_all_smem<false>()) != cudaSuccess) return e;
    if ((e = pc_knn_win_attrs()) != cudaSuccess) return e;
    if ((e = pc_knn_union_attrs()) != cudaSuccess) return e;
    if ((e = pc_knn_union_win_attrs()) != cudaSuccess) return e;
    g_attr_done |= bit;
    return cudaSuccess;
}

int clamp_tile(int t) { return t <= 0 ? 32 : (t > 32 ? 32 : t); }

// The search mode for k on this target: its tune may ask for 64 survivor
// slots (mode 1) for every k <= 32.
int target_mode(const pc_target_s* t, int k) {
    const int m = search_mode(k);
    return (m == 0 && t->tune.slots == 64) ? 1 : m;
}
int clamp_warps(int w) { return w <= 0 ? 4 : (w > 8 ? 8 : w); }

// Calls f(kernel) with the search kernel for (mode, with_cov, windowed).
template <bool BATCH, typename F>
cudaError_t with_kernel(int mode, bool with_cov, bool windowed, F&& f, bool stage = false) {
    void* kern = windowed ? pc_knn_kernel_win(mode, with_cov, BATCH, stage)
                          : knn_kernel<false>(mode, with_cov, BATCH, stage);
    return f(kern);
}

}  // namespace

cudaError_t pc_launch_knn(const pc_target_s* t, const float* q, int64_t N, int k, float eps,
                          int32_t* idx, float* d2, float* cov, float rho0, cudaStream_t s, bool stage) {
    if (N == 0) return cudaSuccess;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    const int tile = clamp_tile(t->tune.tile);
    const int warps = clamp_warps(t->tune.warps);
    // the covariance (plain, or weighted by the target's kernel descriptor)
    // is fused into the search
    const bool with_cov = cov != nullptr;
    const int mode = target_mode(t, k);
    stage = stage && mode < 2 && with_cov;  // the warp path writes its rows directly
    TileArgs a{k, eps, t->tune.rho_scale > 0 ? t->tune.rho_scale : 0.9f, t->tune.order == 0 ? 1 : 0, t->ck,
               pc_probe_c(t)};
    const size_t smem = (size_t)warps * warp_bytes(mode, stage, k);
    const int64_t tiles = (N + tile - 1) / tile;
    const int64_t blocks = (tiles + warps - 1) / warps;
    Grid g = t->g;
    float* covp = with_cov ? cov : nullptr;
    void* args[] = {&g, (void*)&q, (void*)&N, (void*)&tile, &a, &rho0, &idx, &d2, &covp};
    return with_kernel<false>(
        mode, with_cov, g.windowed != 0,
        [&](void* kern) { return cudaLaunchKernel(kern, dim3((unsigned)blocks), dim3(warps * 32), args, smem, s); },
        stage);
}

// The union search (a target with appended points): the same launch shape
// as pc_launch_knn over the main grid and the delta grid together.
cudaError_t pc_launch_knn_union(const pc_target_s* t, const float* q, int64_t N, int k, float eps,
                                int32_t* idx, float* d2, float* cov, float rho0, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    const int tile = clamp_tile(t->tune.tile);
    const int warps = clamp_warps(t->tune.warps);
    const bool with_cov = cov != nullptr;
    const int mode = target_mode(t, k);
    TileArgs a{k, eps, t->tune.rho_scale > 0 ? t->tune.rho_scale : 0.9f, t->tune.order == 0 ? 1 : 0, t->ck,
               pc_probe_c(t)};
    const size_t smem = (size_t)warps * warp_smem_bytes(mode);
    const int64_t tiles = (N + tile - 1) / tile;
    const int64_t blocks = (tiles + warps - 1) / warps;
    Grid g = t->g;
    Grid dg = t->delta->g;
    float* covp = with_cov ? cov : nullptr;
    void* args[] = {&g, &dg, (void*)&q, (void*)&N, (void*)&tile, &a, &rho0, &idx, &d2, &covp};
    void* kern = g.windowed ? pc_knn_union_kernel_win(mode, with_cov) : pc_knn_union_kernel(mode, with_cov);
    return cudaLaunchKernel(kern, dim3((unsigned)blocks), dim3(warps * 32), args, smem, s);
}

cudaError_t pc_knn_prepare() { return ensure_attrs(); }

cudaError_t pc_launch_cov(const pc_target_s* t, const int32_t* idx, int64_t N, int k, float eps,
                          float* cov, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int threads = 128;
    const int64_t blocks = (N + threads - 1) / threads;
    k_cov<<<(unsigned)blocks, threads, 0, s>>>(t->g, idx, N, k, eps, cov);
    return cudaGetLastError();
}

cudaError_t pc_launch_knn_batch(const pc_target_s* t, const Grid& gv, const CovKernel& ck,
                                const ScanDesc* scans_dev, int nscans, int64_t max_n,
                                int64_t total_tiles, int tile, int warps, int k, float eps,
                                bool with_cov, float rho0, cudaStream_t s, bool stage) {
    if (total_tiles == 0) return cudaSuccess;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    TileArgs a{k, eps, t->tune.rho_scale > 0 ? t->tune.rho_scale : 0.9f, t->tune.order == 0 ? 1 : 0, ck,
               pc_probe_c(t)};
    const int64_t blocks = (total_tiles + warps - 1) / warps;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    const int mode = target_mode(t, k);
    stage = stage && mode < 2;  // the warp path writes its rows directly
    const size_t smem = (size_t)warps * warp_bytes(mode, stage, k);
    Grid g = gv;
    void* args[] = {&g, (void*)&scans_dev, &nscans, &total_tiles, &tile, &a, &rho0};
    return with_kernel<true>(
        mode, with_cov, g.windowed != 0,
        [&](void* kern) { return cudaLaunchKernel(kern, dim3((unsigned)blocks), dim3(warps * 32), args, smem, s); },
        stage);
}
