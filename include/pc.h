/*
 * pc.h -- C ABI of the GB300 nearest-points + covariance library (libpc.so).
 *
 * The operation is the data-parallel step of GICP-style scan registration
 * (Sec. III-C1 "Efficient registration method", Eq. 18-20): every point is
 * modelled as a Gaussian N(p_i, C_i), and C_i is estimated from the point's
 * k nearest neighbours in a target cloud or map.  The paper names "finding
 * corresponding points and computing covariance" as the CPU bottleneck and
 * moves both to the GPU (Sec. III-C1, Fig. 5; Sec. IV-E1); the map side is
 * held in a "GPU-hash data structure" (Sec. III-C3 "Scan match for
 * correction").
 *
 * Conventions shared by every call:
 *  - Points are float32 [n,3] row-major (x, y, z), contiguous.
 *  - Indices are 0-based positions in the caller's target array.
 *  - idx is int32 [N,k], d2 is float32 [N,k], both ascending by the key
 *    (d2, index): ties go to the lower index.  d2 is the binary32 value
 *    fmaf(dz,dz, fmaf(dy,dy, dx*dx)), dx = q.x - p.x, bit-exact.
 *  - cov is float32 [N,6] = (xx, xy, xz, yy, yz, zz) of
 *    C = (1/k) sum_j (p_j - mu)(p_j - mu)^T over the k neighbours; with
 *    eps >= 0 it is the plane-regularised V diag(1,1,eps) V^T, V the
 *    eigenvectors of C ordered by decreasing eigenvalue, i.e.
 *    I - (1-eps) n n^T with n the unit normal (smallest eigenvalue).
 *  - "_dev" pointers are device memory (cudaMalloc / torch CUDA tensors);
 *    the caller owns them.  A host or unregistered pointer where device
 *    memory is required returns PC_ERR_BAD_POINTER.  The batched entries
 *    (pc_scan) also take page-locked host memory mapped into the device's
 *    address space, and pc_knn_cov_host uses such buffers in place.
 *  - Every call except pc_build_target and pc_knn_cov_host is asynchronous
 *    on the given stream (a cudaStream_t cast to void*; NULL = the legacy
 *    default stream).  Argument errors are returned synchronously and
 *    nothing is launched.  Conditions found on the device (a non-finite
 *    query, a search past the configured limit, an out-of-range index given
 *    to pc_cov) set bits in the target's status word: the affected rows get
 *    idx = -1, d2 = +inf, cov = NaN, and pc_sync_status reports them.
 *  - No call throws, traps or aborts.
 *  - One GPU; a target handle is bound to the device that was current when
 *    it was built.
 */
#ifndef PC_H
#define PC_H

#include <stdint.h>

#if defined(__GNUC__)
#define PC_API __attribute__((visibility("default")))
#else
#define PC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pc_target_s *pc_target; /* opaque, library-owned */
typedef struct pc_batch_s *pc_batch;   /* opaque, library-owned */
typedef void *pc_stream;               /* cudaStream_t */

typedef enum {
    PC_OK = 0,
    PC_ERR_INVALID_ARG = 1,  /* k < 1, k > 64, N < 0, M < 1, M >= 2^31, NULL with N > 0 */
    PC_ERR_K_GT_M = 2,       /* k larger than the target size */
    PC_ERR_NONFINITE = 3,    /* NaN/inf in the target (build) or a query (status) */
    PC_ERR_OOM = 4,          /* device allocation failed */
    PC_ERR_CUDA = 5,         /* any other CUDA runtime error */
    PC_ERR_SEARCH_LIMIT = 6, /* widening search hit max_box_cells with exhaustive = 0 */
    PC_ERR_BAD_POINTER = 7,  /* host / unregistered pointer where device memory is required */
    PC_ERR_BAD_INDEX = 8,    /* pc_cov got an index outside [0, M) */
    PC_ERR_DESTROYED = 9     /* handle already destroyed */
} pc_status;

/* Target-build options (Sec. III-C3: the map is held in a GPU hash). */
typedef struct {
    float cell_size;   /* > 0: voxel edge h in the caller's units; <= 0: chosen so the
                          mean points per occupied cell is about `occupancy` */
    float occupancy;   /* target mean points per occupied cell for the automatic h; <= 0: 12 */
    float hash_load;   /* open-addressing load factor in (0, 0.9]; <= 0: 0.5 */
    int max_box_cells; /* the radius-widening search stops growing its cell box here; <= 0: 4096 */
    int exhaustive;    /* past max_box_cells: 1 = exact scan of every occupied cell,
                          0 = mark the row and report PC_ERR_SEARCH_LIMIT */
} pc_build_opts;

/* Launch shape of the search kernel.  None of these changes any result. */
typedef struct {
    int tile;          /* queries per warp work item (one per lane for k <= 32), 1..32;
                          <= 0: 32 */
    int warps;         /* warps per block, 1..8; <= 0: 4 */
    float rho_scale;   /* scales the target's calibrated k-th-neighbour radius that the
                          search starts from (k <= 32: trial radii 0.75..1.46 x it);
                          <= 0: 0.9 */
    int order;         /* 0: issue query tiles last-first (a ring-by-ring LiDAR scan ends
                          with its slowest, farthest rings); 1: first-first */
    int probe;         /* where each query's trial radii start (k <= 32): 0 auto (1 on a
                          map whose calibration saw an even density, else 2); 1 the
                          calibrated radius for every query; 2 a per-query radius from
                          the point count of the 27 cells around it */
    int slots;         /* survivor slots per query of the lane path (its k tile): 0 by
                          k (32 for k <= 24, 64 for 25..32); 64 for every k <= 32 */
} pc_tune;

/* What the built target looks like (for reporting and tuning). */
typedef struct {
    int64_t m;          /* target points */
    int64_t ncells;     /* occupied cells */
    int64_t table_cap;  /* hash slots */
    float cell_size;    /* h */
    float origin[3];    /* grid origin = bbox minimum */
    float bbox_max[3];
    int dims[3];        /* cells per axis */
    int64_t device_bytes; /* device memory held by the handle */
    float rho_hint[64]; /* calibrated first search radius for k = 1..64 (0 if k > M) */
    int64_t delta_m;    /* points appended by pc_target_append and not yet compacted
                           (m counts the main grid only) */
} pc_target_info;

/* Counters kept by the search kernels since the last reset (one atomic per
 * warp work item; they never change a result). */
typedef struct {
    int64_t queries;     /* queries answered */
    int64_t warp_search; /* of those, answered by the warp-cooperative search
                            (k > 32, or k <= 32 queries the lane path handed over) */
    int64_t exhaustive;  /* searches that ended in the exhaustive cell scan */
    int64_t candidates;  /* target points whose distance the lane path computed
                            (its counting and collecting passes together) */
} pc_stats;

/* One scan of a batch, caller-owned: device memory, or page-locked host
 * memory mapped into the device's address space (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory).  When any scan's idx, d2 or cov is
 * such host memory, the batch runs the staged kernel: each warp writes its
 * tile's rows as whole blocks, so the results reach host memory during the
 * search with no copy (for k <= 32; the warp path, k > 32, writes its rows
 * directly).  Results are identical either way.  Any other pointer returns
 * PC_ERR_BAD_POINTER. */
typedef struct {
    const float *q_dev; /* [n,3] */
    int64_t n;
    int32_t *idx_dev;   /* [n,k] */
    float *d2_dev;      /* [n,k] */
    float *cov_dev;     /* [n,6], may be NULL to skip the covariance */
} pc_scan;

/* Fills *o with the defaults listed above. */
PC_API void pc_default_build_opts(pc_build_opts *o);

/* Builds the device-resident voxel-hash grid over the target xyz_dev[M,3]
 * (Sec. III-C3 "GPU-hash data structure"): finite check and bounding box,
 * cell keys, an LSD radix sort of (key, index), the occupied-cell table in an
 * open-addressing hash, and cell-ordered float4 copies of the points.  The
 * library copies the points; xyz_dev may be freed afterwards.  Synchronises
 * `s` (it reads sizes back).  opts may be NULL (defaults).  Errors:
 * PC_ERR_INVALID_ARG (M < 1 or M >= 2^31, NULL pointers), PC_ERR_BAD_POINTER,
 * PC_ERR_NONFINITE (any NaN/inf coordinate; no handle is made), PC_ERR_OOM,
 * PC_ERR_CUDA.  On success *out owns device memory until pc_destroy_target. */
PC_API pc_status pc_build_target(const float *xyz_dev, int64_t M, const pc_build_opts *opts,
                          pc_stream s, pc_target *out);

/* Frees the handle.  NULL is a no-op.  Work still queued on a stream that
 * uses the handle must have finished (synchronise first). */
PC_API void pc_destroy_target(pc_target t);

/* Sets the launch shape for later calls on t (NULL restores defaults). */
PC_API pc_status pc_set_tune(pc_target t, const pc_tune *tune);

PC_API pc_status pc_get_info(pc_target t, pc_target_info *info);

/* k nearest target points of each query q_dev[N,3] (Sec. III-C1: "finding
 * corresponding points"): idx_dev[N,k], d2_dev[N,k] as described above.
 * 1 <= k <= 64 and k <= M, N >= 0 (N = 0 is a no-op). */
PC_API pc_status pc_knn(pc_target t, const float *q_dev, int64_t N, int k, int32_t *idx_dev,
                 float *d2_dev, pc_stream s);

/* Covariance of each neighbourhood row idx_dev[N,k] over the target
 * (Sec. III-C1: C_i of Eq. 19 "computing covariance"): cov_dev[N,6].  eps < 0
 * returns the raw C; eps >= 0 the plane-regularised form.  An index outside
 * [0, M) gives a NaN row and PC_ERR_BAD_INDEX in the status word. */
PC_API pc_status pc_cov(pc_target t, const int32_t *idx_dev, int64_t N, int k, float eps,
                 float *cov_dev, pc_stream s);

/* An axis-aligned box of the map's coordinates; +-inf bounds are allowed. */
typedef struct {
    float lo[3];
    float hi[3];
} pc_window;

/* Sliding-window submap (Sec. III-C3: scan matching uses the points of a
 * window M_i of the unified map M^W, selected per pose through the GPU hash
 * structure): restricts every later search on this target -- pc_knn,
 * pc_knn_cov, pc_knn_cov_host, the batched forms and pc_gicp_linearize -- to
 * the map points p with lo <= p <= hi componentwise, without rebuilding the
 * grid.  NULL restores the whole map.  Results are exactly those of the same
 * search over the submap, with indices into the whole map (ties still go to
 * the lower index).  Search boxes are clipped to the window's cells and
 * only the window's boundary cells test their points, so the cost follows
 * the window, not the map.  A query whose window holds fewer than k points
 * gets idx -1 / d2 +inf / cov NaN and PC_ERR_K_GT_M in the status word (with
 * exhaustive = 0 it may report PC_ERR_SEARCH_LIMIT instead).  pc_cov is not
 * affected (it takes the neighbours as given).  The window is copied into
 * each launch when it is issued; a batch plan keeps the window that was set
 * when pc_batch_plan was called.  Host-only: no device work, no
 * synchronisation.  Errors: PC_ERR_INVALID_ARG for a NaN bound or lo > hi
 * on an axis; the handle errors of pc_knn. */
PC_API pc_status pc_set_window(pc_target t, const pc_window *w);

/* Kernel descriptors of Table I (Sec. III-C1: the covariance is computed
 * "using the kernel descriptors"). */
typedef enum {
    PC_KERNEL_NONE = 0,       /* plain covariance */
    PC_KERNEL_RBF = 1,        /* exp(-|x - y|^2 sigma) */
    PC_KERNEL_GAUSSIAN = 2,   /* exp(-|x - y|^2 / (2 sigma^2)) */
    PC_KERNEL_POLYNOMIAL = 3, /* (alpha <x', y'> + c)^d */
    PC_KERNEL_HI = 4,         /* sum_i min(x'_i, y'_i) / sum_i x'_i */
    PC_KERNEL_LAPLACIAN = 5   /* exp(-|x - y| / sigma) */
} pc_kernel_type;

typedef struct {
    int type; /* pc_kernel_type */
    float sigma, alpha, c, d;
} pc_cov_kernel;

/* Weights the covariance of every later fused search on this target --
 * pc_knn_cov, pc_knn_cov_host and the batched forms -- by a kernel
 * descriptor: for query x = q and its neighbours y = p_j, w_j = K(x, y_j),
 * W = sum w_j, mu = sum w_j p_j / W, C = sum w_j (p_j - mu)(p_j - mu)^T / W,
 * then the plane regularisation for eps >= 0 as before.  Polynomial and HI
 * use coordinates relative to the target's bounding-box minimum (x' = x - o,
 * y' = y - o).  The paper names the kernels but not how they enter the
 * covariance; this weighted form is the reading.  Per query the weights and
 * moments are binary32 (two passes shifted by the nearest neighbour).  A row
 * whose total weight is not positive and finite (a polynomial can make it
 * so) is NaN.  The neighbours are unchanged: the search runs as without a
 * kernel, and the weighted covariance is formed in the same launch, in the
 * search's epilogue, from the neighbours it has just found.  NULL or type
 * PC_KERNEL_NONE restores the plain covariance.  pc_cov is not affected (it
 * has no query points).  A batch plan keeps the kernel set when it was
 * planned.  Host-only.  Errors: PC_ERR_INVALID_ARG for an unknown type, a
 * non-finite parameter, sigma < 0 (RBF) or sigma <= 0 (Gaussian,
 * Laplacian); the handle errors of pc_knn. */
PC_API pc_status pc_set_cov_kernel(pc_target t, const pc_cov_kernel *kd);

/* Incremental map update (the map grows while it is used, Sec. III-C3's
 * unified map): appends n points (device f32 [n,3]) to the target without
 * rebuilding its grid.  They get the indices M + (their position among all
 * appended points), and every later search -- pc_knn, pc_knn_cov,
 * pc_knn_cov_host, pc_cov, pc_gicp_linearize -- answers over the whole
 * union exactly: one launch searches the main grid and a small grid over
 * the appended points together (each query's boxes on both grids, filtered
 * by the smaller of their certified radii), so results equal a target
 * built from all the points at once (idx and d2 bit for bit; the
 * covariance to its rounding).  The delta grid is rebuilt from all appended points at
 * each call (O(appended) work; the main grid is never touched).  Windows and
 * covariance kernels apply to both.  The batched forms refuse a target with
 * appended points (PC_ERR_INVALID_ARG): compact it first.  Synchronous with
 * respect to `s` (it builds a grid); allocates.  Errors: PC_ERR_NONFINITE
 * (nothing is appended), PC_ERR_INVALID_ARG (n < 0, M + appended >= 2^31),
 * PC_ERR_BAD_POINTER, PC_ERR_OOM. */
PC_API pc_status pc_target_append(pc_target t, const float *xyz_dev, int64_t n, pc_stream s);

/* Folds the appended points into a new main grid over all M + appended
 * points (same indices, same handle, window and settings kept) and drops the
 * delta.  A no-op without appended points.  Batch plans made before it must
 * be made again (pc_batch_run refuses them). */
PC_API pc_status pc_target_compact(pc_target t, pc_stream s);

/* pc_knn and pc_cov fused in one launch; identical results to the two calls. */
PC_API pc_status pc_knn_cov(pc_target t, const float *q_dev, int64_t N, int k, float eps,
                     int32_t *idx_dev, float *d2_dev, float *cov_dev, pc_stream s);

/* pc_knn_cov from HOST buffers (pinned or pageable), synchronising `s`
 * before returning; results identical to pc_knn_cov.  When idx, d2 and cov
 * are all page-locked and mapped into the device's address space
 * (cudaHostAlloc, cudaHostRegister, torch pin_memory), k <= 32 and the
 * target has no appended points, the search writes them in place: each
 * warp stages its tile's rows in shared memory and writes them as whole
 * lines, so the transfer runs during the search; a page-locked q is then
 * also read in place.  Otherwise q is copied in and idx/d2/cov copied out
 * through device staging buffers kept in the handle and grown on demand
 * (PC_ERR_OOM if that fails).  Device-side conditions are returned
 * directly (no separate pc_sync_status needed); rows are written as by
 * pc_knn_cov even then. */
PC_API pc_status pc_knn_cov_host(pc_target t, const float *q_host, int64_t N, int k, float eps,
                          int32_t *idx_host, float *d2_host, float *cov_host, pc_stream s);

/* Synchronises `s` and copies the target's counters to *out; reset != 0
 * zeroes them afterwards. */
PC_API pc_status pc_get_stats(pc_target t, pc_stream s, pc_stats *out, int reset);

/* Synchronises `s`, returns and clears the target's status word: PC_OK, or
 * the first of PC_ERR_NONFINITE, PC_ERR_SEARCH_LIMIT, PC_ERR_BAD_INDEX,
 * PC_ERR_K_GT_M (a search window held fewer than k points) raised since the
 * last call, or PC_ERR_CUDA if the stream reported an error. */
PC_API pc_status pc_sync_status(pc_target t, pc_stream s);

/* Batched form: many scans against one target in ONE launch, one warp per
 * (scan, tile) item of the scans' prefix-summed tile table, replayed as a
 * CUDA graph.  pc_batch_plan copies the scan table to the device; the
 * pointers in `scans` must stay valid while the plan is used.  All scans
 * share k and eps.  Results are bit-identical to pc_knn_cov on each scan
 * alone. */
PC_API pc_status pc_batch_plan(pc_target t, const pc_scan *scans, int n_scans, int k, float eps,
                        pc_batch *out);
/* Runs the plan on `s`.  The first run on a stream captures the launch in a
 * CUDA graph; later runs replay it. */
PC_API pc_status pc_batch_run(pc_batch b, pc_stream s);
PC_API void pc_batch_destroy(pc_batch b);

/* Bytes of device scratch pc_batch_run_scratch needs for n_scans scans. */
PC_API size_t pc_batch_scratch_bytes(int n_scans);

/* The batched form (same kernel and results as pc_batch_run) with scratch
 * the caller owns: scratch_dev is device memory of at least
 * pc_batch_scratch_bytes(n_scans) bytes, 256-byte aligned, used for the scan
 * table.  No allocation and no graph.  Calls with
 * distinct scratch may run concurrently on different streams and overlap on
 * the device -- the continuous-batching server launches each step this way.
 * Asynchronous on `s`; the scan table is copied from `scans` before the call
 * returns.  Errors: those of pc_batch_plan, PC_ERR_INVALID_ARG for a NULL,
 * misaligned or too small scratch. */
PC_API pc_status pc_batch_run_scratch(pc_target t, const pc_scan *scans, int n_scans, int k,
                                      float eps, void *scratch_dev, size_t scratch_bytes,
                                      pc_stream s);

/* Largest n_scans that pc_batch_run_noalloc accepts. */
#define PC_NOALLOC_MAX_SCANS 256

/* The batched search + covariance of pc_batch_plan/pc_batch_run in one call
 * that allocates no memory at all.  The paper has no counterpart; this entry
 * is for callers that may not allocate device memory once they are running:
 * a real-time estimation loop that reserves its GPU memory at start-up and
 * must not stall later (cudaMalloc and cudaFree can synchronise the whole
 * device), or an application that hands out every device buffer from its
 * own pool.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Its scratch -- the scan table -- lives in
 * one file-scope device array sized for PC_NOALLOC_MAX_SCANS scans (about
 * 12 KB), which every GPU that loads the library keeps until the process
 * exits.  The caller still passes the target, and the inputs and outputs in
 * `scans` (as for pc_batch_plan).
 *  - n_scans < 1 or > PC_NOALLOC_MAX_SCANS returns PC_ERR_INVALID_ARG and
 *    launches nothing; other argument errors are those of pc_batch_plan.
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current).
 *  - It cannot be captured into a CUDA graph: the scan table is copied from
 *    the caller's pageable host memory, which stream capture does not
 *    allow.  On a stream that is capturing it returns PC_ERR_INVALID_ARG
 *    and enqueues nothing, so the capture stays valid.  (pc_batch_plan and
 *    pc_batch_run are the capturable batched form.)
 *  - Every call on a device uses the same array and it keeps the last
 *    call's scan table: calls that overlap on the GPU -- on two streams, or from two host
 *    threads -- race and corrupt each other's results.  Serialise them.
 *  - Asynchronous on `s` apart from the table copy: the table is copied
 *    from the caller's host array before the call returns, so that array
 *    may be reused at once, but a copy from pageable memory may make the
 *    host wait for work already queued on `s`.
 *  - Results are identical to pc_knn_cov on each scan alone (idx, d2 and
 *    cov bit for bit); a scan with n = 0 is skipped and one with cov_dev =
 *    NULL gets no covariances. */
PC_API pc_status pc_batch_run_noalloc(pc_target t, const pc_scan *scans, int n_scans, int k,
                                      float eps, pc_stream s);

/* ---- GICP registration on top of the search (Sec. III-C1, Eq. 18-20) ---- */

/* Number of doubles pc_gicp_linearize writes to out_dev. */
#define PC_GICP_OUT 29

/* Bytes of device workspace pc_gicp_linearize needs on the current device
 * (a ticket counter and one partial-sum row per resident block; ~80 KB on
 * a 152-SM GPU); 0 if no device is usable. */
PC_API size_t pc_gicp_work_bytes(void);

/* One Gauss-Newton linearisation of scan-to-map GICP (Sec. III-C1: the
 * transformation error d_i of Eq. 18, its covariance of Eq. 19 and the
 * objective of Eq. 20), with the map the target `map` was built from.
 *
 *  map_cov_dev  f32 [M,6] packed (xx xy xz yy yz zz) covariance C_q of every
 *               map point, in the caller's map order (e.g. pc_knn_cov of the
 *               map against itself).
 *  src_dev      f32 [n,3] source scan points p; src_cov_dev f32 [n,6] their
 *               covariances C_p (pc_knn_cov of the scan against a target
 *               built from the scan).
 *  pose_dev     f32 [12] device-resident pose: R row-major (9) then t (3).
 *  max_dist     correspondence distance: a source point pairs with its
 *               exact nearest map point q (pinned binary32 d2, ties to the
 *               lower index) when d2 <= fl(max_dist^2); +inf pairs all.
 *  out_dev      f64 [29]: H upper triangle row by row (21), b (6), E, the
 *               number of pairs summed, where with p' = R p + t (binary32,
 *               fmaf(R_a2,p_z, fmaf(R_a1,p_y, fmaf(R_a0,p_x, t_a)))),
 *               d = q - p', Omega = (C_q + R C_p R^T)^-1 and
 *               J = [[p']_x, -I] (left perturbation T <- exp(xi^) T,
 *               xi = (omega, v)):  H = sum J^T Omega J,
 *               b = sum J^T Omega d,  E = sum d^T Omega d.  A pair whose
 *               combined covariance is not positive definite (binary32
 *               determinant <= 0) is matched but not summed.  Per pair the
 *               terms are binary32; the sums are binary64 in a fixed
 *               order, so the same call repeats bit for bit.
 *  corr_dev     optional i32 [n]: the map index of each pair, -1 for a
 *               point with no map point within max_dist or a non-finite p'.
 *  work_dev     device workspace of at least pc_gicp_work_bytes() bytes,
 *               256-byte aligned, owned by the caller; calls that share it
 *               must not overlap on the GPU.
 * Asynchronous on `s`; allocates nothing.  Errors: PC_ERR_INVALID_ARG for
 * n < 0, a NaN or negative max_dist, a NULL, misaligned or too small
 * argument; PC_ERR_BAD_POINTER for host pointers; a destroyed or foreign
 * handle as for pc_knn.  A non-finite p' sets PC_ERR_NONFINITE, a search
 * that passed max_box_cells with exhaustive = 0 PC_ERR_SEARCH_LIMIT in the
 * status word (pc_sync_status); such points do not pair. */
PC_API pc_status pc_gicp_linearize(pc_target map, const float *map_cov_dev, const float *src_dev,
                                   int64_t n, const float *src_cov_dev, const float *pose_dev,
                                   float max_dist, double *out_dev, int32_t *corr_dev,
                                   void *work_dev, size_t work_bytes, pc_stream s);

/* The Gauss-Newton (lambda = 0) or Levenberg-Marquardt (lambda > 0) step
 * after pc_gicp_linearize, on the device: solves (H + lambda I) xi = -b by
 * Cholesky in binary64 from lin_dev (the 29 doubles above) and moves the
 * pose in place, R <- Exp(omega) R, t <- Exp(omega) t + v (Rodrigues).
 * xi_dev (optional, f64 [6]) receives xi, or NaNs when H + lambda I is not
 * positive definite (the pose is then left unchanged).  One single-thread
 * launch on `s`, so linearise + update iterations queue (or graph-capture)
 * with no host round trip.  PC_ERR_INVALID_ARG for NULL lin/pose or a
 * negative or NaN lambda, PC_ERR_BAD_POINTER for host pointers. */
PC_API pc_status pc_gicp_update(const double *lin_dev, float lambda, float *pose_dev,
                                double *xi_dev, pc_stream s);

/* ---- Wall detection (Sec. III-D, Eq. 24-30) ---- */

typedef struct pc_wall_s *pc_wall; /* opaque, library-owned */

typedef struct {
    float voxel;      /* voxel edge of the voxel filter, m (default 0.2) */
    float cell2d;     /* edge of the 2-D voting cells, m (default 0.2) */
    int min_votes;    /* a 2-D cell holding more voxels than this is a vertical
                         feature; the rest is ground (default 2) */
    float tol;        /* Euclidean clustering distance, m (default 0.45) */
    int min_cluster;  /* smallest cluster (voxels) that can be the wall (10) */
    float max_range;  /* |x|, |y| kept, m (default 128) */
    float max_height; /* |z| kept, m (default 16) */
} pc_wall_opts;

typedef struct {
    int64_t n_voxels;   /* voxels after the voxel filter */
    int64_t n_vertical; /* of those, vertical features */
    int64_t wall_label; /* the wall cluster's label (its smallest voxel index), -1: none */
    int64_t wall_count; /* voxels in the wall cluster */
    float wall_length;  /* its extent along x, m */
    double beta[3];     /* y = beta0 + beta1 x + beta2 x^2 over the wall (Eq. 28); NaN if none */
    double d_w;         /* beta0: the wall's lateral offset at the vehicle origin (Eq. 29) */
} pc_wall_result;

PC_API void pc_wall_default_opts(pc_wall_opts *o);

/* A detector for scans of up to max_points points (vehicle body frame: x
 * forward, y left, z up).  Allocates every device buffer once (about
 * 150 B per point); pc_wall_detect allocates nothing.  Errors:
 * PC_ERR_INVALID_ARG (max_points < 1 or >= 2^31, non-positive or non-finite
 * sizes, a key range over 63 bits), PC_ERR_OOM. */
PC_API pc_status pc_wall_create(int64_t max_points, const pc_wall_opts *o, pc_wall *out);

/* One scan, asynchronous on `s` (pts_dev: f32 [n,3] device memory, n <=
 * max_points):
 *  1. voxel filter: voxel (i,j,k) = floor(fl(p * fl(1/voxel))); points that
 *     are not finite or whose voxel lies outside the configured range are
 *     dropped; voxels are numbered in ascending key order; each voxelised
 *     point is the centroid of its points (binary64 sum in input order,
 *     rounded to binary32);
 *  2. 2-D voting: each voxel votes for the cell floor(fl(c * fl(1/cell2d)))
 *     of its centroid's x, y (a hash table, Eq. 25); voxels in cells with more
 *     than min_votes votes are vertical features, the rest ground;
 *  3. Euclidean clustering of the vertical voxels: linked when the pinned
 *     binary32 squared distance of their centroids is <= fl(tol^2);
 *     clusters are connected components labelled by their smallest voxel
 *     index (Eq. 26);
 *  4. the wall: the longest cluster (fl(max x - min x)) of >= min_cluster
 *     voxels on the right (fl(min y + max y) < 0), ties to the smaller
 *     label (Eq. 27);
 *  5. y = b0 + b1 x + b2 x^2 by least squares over the wall's centroids in
 *     binary64 (Eq. 28), d_w = b0 (Eq. 29); b1, b2 shape the wall-following
 *     path of Eq. 30.
 * Voxels, flags and labels are deterministic; the fit repeats bit for bit.
 * Errors: PC_ERR_INVALID_ARG (bad handle, n < 0 or > max_points, NULL
 * points), PC_ERR_BAD_POINTER (host points). */
PC_API pc_status pc_wall_detect(pc_wall w, const float *pts_dev, int64_t n, pc_stream s);

/* Synchronises `s` and reads the last detection: the summary, and (each
 * optional) per voxel the centroid (f32 [n_voxels,3]), vertical flag (i32)
 * and cluster label (i32, -1 for ground) into host arrays of at least
 * n_voxels rows.  Returns PC_ERR_SEARCH_LIMIT if an internal iteration cap
 * was reached (a hash table or a union-find chase; not expected). */
PC_API pc_status pc_wall_get(pc_wall w, pc_stream s, pc_wall_result *res, float *centroids_host,
                             int32_t *vertical_host, int32_t *labels_host);

PC_API void pc_wall_destroy(pc_wall w);

PC_API const char *pc_status_string(pc_status st);

/* Library version string, e.g. "pc 0.1 sm_103a". */
PC_API const char *pc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PC_H */
