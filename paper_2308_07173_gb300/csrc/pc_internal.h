// Host-side definitions shared by the library's translation units.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pc.h"
#include "pc_device.cuh"

constexpr uint32_t PC_MAGIC_LIVE = 0x70637467u;  // "pctg"
constexpr uint32_t PC_MAGIC_DEAD = 0xdeadbeefu;

// Kernel-descriptor weights of the covariance (pc_set_cov_kernel), as the
// device sees them: s = sigma (RBF), 1 / (2 sigma^2) (Gaussian) or
// 1 / sigma (Laplacian); o = the target's bounding-box minimum.
struct CovKernel {
    int type;
    float s, alpha, c, d;
    float ox, oy, oz;
};

// One scan of a batched launch, as the batched kernel reads it from the scan table.
struct ScanDesc {
    const float* q;
    int64_t n;
    int32_t* idx;
    float* d2;
    float* cov;     // may be null: no covariance for this scan
    int64_t tile0;  // first work item of this scan
};

struct pc_target_s {
    uint32_t magic;
    int device;
    pcdev::Grid g;        // kernel view; the pointers below back it
    pc_build_opts opts;
    pc_tune tune;
    float bbox_max[3];
    float rho_hint[64];
    int uneven;  // the calibration's k-th-neighbour distances spread widely (p90 / p25 > 1.55)
    int64_t table_cap;
    int64_t device_bytes;
    // owned device memory
    uint4* table;
    float4* pts;
    float4* xyz;
    unsigned long long* cell_keys;
    uint32_t* cell_start;
    uint32_t* dstart;
    uint2* xcut;  // sub-cell cut of the row index (Grid::xcut), or null
    int* status;  // 64 bytes: status word, then 4 u64 statistics counters at +32
    // staging for pc_knn_cov_host, grown on demand
    void* stage;
    size_t stage_bytes;
    CovKernel ck;  // covariance weights (type 0: none)
    // incremental updates (pc_target_append): the appended points, f32
    // [delta_m, 3] in append order, and a grid over them; their indices
    // follow the main map's (M + position)
    pc_target_s* delta;
    float* delta_xyz;
    int64_t delta_m, delta_cap;
    // the window of pc_set_window, kept to re-apply to a rebuilt delta grid
    pc_window win;
    int has_win;
};

struct pc_batch_s {
    uint32_t magic;
    pc_target_s* t;
    pcdev::Grid g;  // the target's view when planned (window included)
    CovKernel ck;   // and its covariance weights
    int64_t max_n;  // largest scan
    int n_scans;
    int k;
    float eps;
    bool with_cov;
    bool host_out;  // outputs in mapped host memory: the staged kernel
    int tile;
    int warps;
    int64_t total_tiles;
    int64_t total_queries;
    ScanDesc* scans_dev;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaStream_t captured_on;
};

// The whole grid as the search window (no point tests).
inline void pc_clear_window(pcdev::Grid& g) {
    g.windowed = 0;
    g.wlx = 0;
    g.whx = g.dimx - 1;
    g.wly = 0;
    g.why = g.dimy - 1;
    g.wlz = 0;
    g.whz = g.dimz - 1;
    g.tlx = g.thx = g.tly = g.thy = g.tlz = g.thz = -1;
    g.wlox = g.wloy = g.wloz = -INFINITY;
    g.whix = g.whiy = g.whiz = INFINITY;
}

// grid_build.cu
pc_status pc_build_grid(const float* xyz, int64_t M, const pc_build_opts& o, cudaStream_t s,
                        pc_target_s* t);
void pc_free_grid(pc_target_s* t);
size_t pc_sort_temp_words(int64_t n);
cudaError_t pc_radix_sort_pairs(unsigned long long** keys, uint32_t** vals, unsigned long long* keys_alt,
                                uint32_t* vals_alt, int64_t n, int nbits, uint32_t* temp, cudaStream_t s);
size_t pc_scan_temp_words(int64_t n);
cudaError_t pc_scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                              uint32_t* temp, cudaStream_t s);

// knn_window.cu: the window variant of the search kernels
void* pc_knn_kernel_win(int mode, bool with_cov, bool batch, bool stage = false);
cudaError_t pc_knn_win_attrs();

// knn_cov.cu.  stage: the outputs are host-mapped memory; each warp stages
// its tile's rows in shared memory and writes them as whole blocks (lane
// path with covariance; the warp path, k > 32, writes its rows directly).
cudaError_t pc_launch_knn(const pc_target_s* t, const float* q, int64_t N, int k, float eps,
                          int32_t* idx, float* d2, float* cov, float rho0, cudaStream_t s, bool stage = false);
cudaError_t pc_launch_knn_union(const pc_target_s* t, const float* q, int64_t N, int k, float eps,
                                int32_t* idx, float* d2, float* cov, float rho0, cudaStream_t s);
// Opts the search kernels into large shared memory on the current device
// (once; call outside any stream capture).
cudaError_t pc_knn_prepare();
cudaError_t pc_launch_cov(const pc_target_s* t, const int32_t* idx, int64_t N, int k, float eps,
                          float* cov, cudaStream_t s);
cudaError_t pc_launch_knn_batch(const pc_target_s* t, const pcdev::Grid& g, const CovKernel& ck,
                                const ScanDesc* scans_dev, int nscans, int64_t max_n,
                                int64_t total_tiles, int tile, int warps, int k, float eps,
                                bool with_cov, float rho0, cudaStream_t s, bool stage = false);

// gicp.cu
size_t pc_gicp_work_size();
cudaError_t pc_launch_gicp_linearize(const pc_target_s* t, const float* map_cov, const float* src,
                                     int64_t n, const float* src_cov, const float* pose,
                                     float max_dist, double* out, int32_t* corr, void* work,
                                     float r0, float r0d, cudaStream_t s);
cudaError_t pc_launch_gicp_update(const double* lin, float lambda, float* pose, double* xi,
                                  cudaStream_t s);

// knn_union.cu / knn_union_win.cu: the search kernels over the main grid
// plus the delta grid (whole-map and window variants)
void* pc_knn_union_kernel(int mode, bool with_cov);
cudaError_t pc_knn_union_attrs();
void* pc_knn_union_kernel_win(int mode, bool with_cov);
cudaError_t pc_knn_union_win_attrs();

// delta.cu: covariances and packing over the main grid plus the delta grid
cudaError_t pc_launch_cov_union(const pc_target_s* t, const int32_t* idx, int64_t N, int k, float eps,
                                float* cov, cudaStream_t s);
cudaError_t pc_launch_pack_xyz(const pc_target_s* t, float* out, cudaStream_t s);

// pc_api.cu
float pc_rho0(const pc_target_s* t, int k);
// The probe constant of the lane path's per-query starting radius (0: off).
float pc_probe_c(const pc_target_s* t);
// Launch shape of a batched call over caller-provided scans.
struct BatchShape {
    int64_t tiles;  // work items (tiles of `tile` queries) over all scans; 0: nothing to do
    int64_t max_n;  // largest scan
    int tile, warps;
    bool any_cov;   // some scan asks for covariances
    bool host_out;  // some output is mapped page-locked host memory (staged block writes)
};
// Argument checks and scan table shared by pc_batch_plan,
// pc_batch_run_scratch and pc_batch_run_noalloc; fills table[0, n_scans)
// with the addresses kernels use (mapped host memory translated).
pc_status pc_batch_table(const pc_target_s* t, const pc_scan* scans, int n_scans, int k, float eps,
                         ScanDesc* table, BatchShape* shape);
pc_status pc_from_cuda(cudaError_t e);
bool pc_target_is_live(const pc_target_s* t);
bool pc_is_device_ptr(const void* p);
