// GICP linearisation on the GPU (Sec. III-C1, Eq. 18-20): one Gauss-Newton
// step of scan-to-map registration on top of the voxel-hash grid.
//
// For every source point p (binary32, [n,3]) and the pose T = (R, t):
//   p' = R p + t      binary32, fmaf(R_a2, p_z, fmaf(R_a1, p_y, fmaf(R_a0, p_x, t_a)))
//   q  = the nearest map point of p' under (d2, index), d2 the pinned
//        binary32 distance -- exact, found by a lane-per-point box search
//        that widens until the certified radius covers either a point or
//        max_dist (nothing further away can pair)
//   the pair counts when d2 <= fl(max_dist^2) and S = C_q + R C_p R^T has a
//   positive determinant; then with d = q - p', Omega = S^-1 and
//   J = [ [p']_x , -I ] (left perturbation T <- exp(xi^) T, xi = (omega, v)):
//     H += J^T Omega J,   b += J^T Omega d,   E += d^T Omega d.
//
// Per pair the arithmetic is binary32 (Omega by adjugate / determinant);
// the 29 sums (H upper triangle, b, E, pair count) are added over a warp in
// binary32 by a reduce-scatter (five halving exchanges, after which lane j
// holds the warp total of sum j: 31 shuffles where one butterfly per sum
// takes 145), over warps, blocks and the grid in binary64, always in the
// same order, so a launch is bit-reproducible.  The last block to finish adds the
// block partials (a ticket counter in the caller's workspace).
//
// A second kernel solves (H + lambda I) xi = -b in binary64 (Cholesky) and
// moves the device-resident pose: R <- Exp(omega) R, t <- Exp(omega) t + v,
// so a whole registration runs on one stream without host round trips.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "pc_device.cuh"
#include "pc_internal.h"
#include "pc_search.cuh"

using namespace pcdev;

namespace {

typedef unsigned long long u64;

constexpr int GICP_THREADS = 256;
constexpr int GICP_VALS = 29;         // H upper triangle (21), b (6), E, pairs
constexpr int GICP_STRIDE = 32;       // doubles per block partial (256 B)
constexpr size_t GICP_HEAD = 256;     // ticket counter, padded

// eta of certified_tau for the (unclamped) box [l, h] around p.
__device__ __forceinline__ float box_eta(const Grid& g, float px, float py, float pz, int lx, int hx,
                                         int ly, int hy, int lz, int hz) {
    const int cm = max(max(max(abs(lx), abs(hx + 1)), max(abs(ly), abs(hy + 1))),
                       max(abs(lz), abs(hz + 1)));
    const float pm = fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz)));
    return 0x1p-20f * (g.coord_scale + pm + (float)cm * g.h);
}

// Exact nearest map point of p among those with d2 <= max_d2: its position
// in pts (or -1) and its d2.  A box of half-width r is searched for points
// with d2 <= T = min(tau, max_d2); every point outside the box has d2 >
// tau, so a hit is the global nearest, and no hit with tau >= max_d2 means
// nothing lies within max_d2.  Otherwise r doubles.  A box beyond
// max_box_cells ends in a linear scan of the whole map (exhaustive) or in
// `limited` with no pair.
__device__ int nearest_within(const Grid& g, float px, float py, float pz, float max_d2, float r,
                              float& bd2, bool& limited) {
    for (int attempt = 0; attempt < 48; ++attempt) {
        const int ulx = cell_of(__fsub_rn(px, r), g.ox, g.inv_h);
        const int uhx = cell_of(__fadd_rn(px, r), g.ox, g.inv_h);
        const int uly = cell_of(__fsub_rn(py, r), g.oy, g.inv_h);
        const int uhy = cell_of(__fadd_rn(py, r), g.oy, g.inv_h);
        const int ulz = cell_of(__fsub_rn(pz, r), g.oz, g.inv_h);
        const int uhz = cell_of(__fadd_rn(pz, r), g.oz, g.inv_h);
        const float tau = certified_tau(g, px, py, pz, ulx, uhx, uly, uhy, ulz, uhz);
        const int lx = max(ulx, g.wlx), hx = min(uhx, g.whx);
        const int ly = max(uly, g.wly), hy = min(uhy, g.why);
        const int lz = max(ulz, g.wlz), hz = min(uhz, g.whz);
        const int64_t ncl = (int64_t)max(hx - lx + 1, 0) * max(hy - ly + 1, 0) * max(hz - lz + 1, 0);
        if (ncl > (int64_t)g.max_box_cells) break;
        if (tau >= 0.0f) {
            const float T = fminf(tau, max_d2);
            u64 best = EMPTY_KEY;
            uint32_t bpos = 0u;
            if (ncl > 0) {
                const float eta = box_eta(g, px, py, pz, ulx, uhx, uly, uhy, ulz, uhz);
                auto visit = [&](uint32_t pos, const float4 q) {
                    const float d = sqdist_pinned(px, py, pz, q.x, q.y, q.z);
                    const u64 key = ((u64)__float_as_uint(d) << 32) | (u64)__float_as_uint(q.w);
                    if (d <= T && key < best) {
                        best = key;
                        bpos = pos;
                    }
                };
                if (g.dstart) for_rows(g, px, py, pz, lx, hx, ly, hy, lz, hz, eta, T, visit);
                else for_box_points(g, px, py, pz, lx, hx, ly, hy, lz, hz, eta, T, visit);
            }
            if (best != EMPTY_KEY) {
                bd2 = __uint_as_float((uint32_t)(best >> 32));
                return (int)bpos;
            }
            if (tau >= max_d2) return -1;
        }
        r = fminf(r * 2.0f, 1e30f);
    }
    if (!g.exhaustive) {
        limited = true;
        return -1;
    }
    atomicAdd(&g.stats[2], 1ull);
    u64 best = EMPTY_KEY;
    uint32_t bpos = 0u;
    for (int64_t i = 0; i < g.m; ++i) {
        const float4 q = __ldg(&g.pts[i]);
        if (g.windowed && !in_window(g, q)) continue;
        const float d = sqdist_pinned(px, py, pz, q.x, q.y, q.z);
        const u64 key = ((u64)__float_as_uint(d) << 32) | (u64)__float_as_uint(q.w);
        if (d <= max_d2 && key < best) {
            best = key;
            bpos = (uint32_t)i;
        }
    }
    if (best == EMPTY_KEY) return -1;
    bd2 = __uint_as_float((uint32_t)(best >> 32));
    return (int)bpos;
}

// One pair's 29 terms in binary32 (all zero when S is not positive
// definite by its binary32 determinant); returns whether it counted.
__device__ __forceinline__ bool pair_terms(const float* R, float px, float py, float pz, float4 q,
                                           const float* __restrict__ cq, const float* __restrict__ cp,
                                           float (&v)[32]) {
    // S = C_q + R C_p R^T (symmetric; C packed xx xy xz yy yz zz)
    const float Cp[3][3] = {{cp[0], cp[1], cp[2]}, {cp[1], cp[3], cp[4]}, {cp[2], cp[4], cp[5]}};
    float M[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            M[a][c] = fmaf(R[3 * a + 2], Cp[2][c], fmaf(R[3 * a + 1], Cp[1][c], R[3 * a] * Cp[0][c]));
    float S[6];
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ic[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const int a = ia[j], c = ic[j];
        S[j] = cq[j] + fmaf(M[a][2], R[3 * c + 2], fmaf(M[a][1], R[3 * c + 1], M[a][0] * R[3 * c]));
    }
    const float s00 = S[0], s01 = S[1], s02 = S[2], s11 = S[3], s12 = S[4], s22 = S[5];
    const float a00 = fmaf(s11, s22, -s12 * s12);
    const float a01 = fmaf(s02, s12, -s01 * s22);
    const float a02 = fmaf(s01, s12, -s02 * s11);
    const float a11 = fmaf(s00, s22, -s02 * s02);
    const float a12 = fmaf(s02, s01, -s00 * s12);
    const float a22 = fmaf(s00, s11, -s01 * s01);
    const float det = fmaf(s00, a00, fmaf(s01, a01, s02 * a02));
    if (!(det > 0.0f) || !isfinite(det)) return false;
    const float inv = 1.0f / det;
    const float O[3][3] = {{a00 * inv, a01 * inv, a02 * inv},
                           {a01 * inv, a11 * inv, a12 * inv},
                           {a02 * inv, a12 * inv, a22 * inv}};
    const float d[3] = {q.x - px, q.y - py, q.z - pz};
    float Od[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Od[a] = fmaf(O[a][2], d[2], fmaf(O[a][1], d[1], O[a][0] * d[0]));
    // A = Omega [p']_x, column by column
    float A[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        A[a][0] = fmaf(pz, O[a][1], -py * O[a][2]);
        A[a][1] = fmaf(px, O[a][2], -pz * O[a][0]);
        A[a][2] = fmaf(py, O[a][0], -px * O[a][1]);
    }
    // H_ww = [p']_x^T A, H_wv = [p']_x Omega = -A^T, H_vv = Omega
    float Hw[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Hw[0][c] = fmaf(pz, A[1][c], -py * A[2][c]);
        Hw[1][c] = fmaf(px, A[2][c], -pz * A[0][c]);
        Hw[2][c] = fmaf(py, A[0][c], -px * A[1][c]);
    }
    int w = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
            float h;
            if (r < 3 && c < 3) h = Hw[r][c];
            else if (r < 3) h = -A[c - 3][r];
            else h = O[r - 3][c - 3];
            v[w++] = h;
        }
    // b_w = [p']_x^T Omega d = Od x p',  b_v = -Omega d
    v[21] = fmaf(Od[1], pz, -Od[2] * py);
    v[22] = fmaf(Od[2], px, -Od[0] * pz);
    v[23] = fmaf(Od[0], py, -Od[1] * px);
    v[24] = -Od[0];
    v[25] = -Od[1];
    v[26] = -Od[2];
    v[27] = fmaf(d[2], Od[2], fmaf(d[1], Od[1], d[0] * Od[0]));
    v[28] = 1.0f;
    return true;
}

__global__ void __launch_bounds__(GICP_THREADS) k_gicp_linearize(
    Grid g, Grid dg, int has_delta, float r0d, const float* __restrict__ map_cov, const float* __restrict__ src,
    int64_t n, const float* __restrict__ src_cov, const float* __restrict__ pose, float max_d2, float r0,
    double* __restrict__ out, int32_t* __restrict__ corr, unsigned char* __restrict__ work) {
    __shared__ double red[GICP_THREADS / 32][GICP_STRIDE];
    __shared__ unsigned ticket;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float R[9], t[3];
#pragma unroll
    for (int j = 0; j < 9; ++j) R[j] = __ldg(pose + j);
#pragma unroll
    for (int j = 0; j < 3; ++j) t[j] = __ldg(pose + 9 + j);
    double acc = 0.0;  // lane v keeps the running sum of value v
    const int64_t stride = (int64_t)gridDim.x * GICP_THREADS;
    for (int64_t base = (int64_t)blockIdx.x * GICP_THREADS + warp * 32; base < n; base += stride) {
        const int64_t i = base + lane;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.0f;
        if (i < n) {
            const float sx = __ldg(src + 3 * i), sy = __ldg(src + 3 * i + 1), sz = __ldg(src + 3 * i + 2);
            const float px = __fmaf_rn(R[2], sz, __fmaf_rn(R[1], sy, __fmaf_rn(R[0], sx, t[0])));
            const float py = __fmaf_rn(R[5], sz, __fmaf_rn(R[4], sy, __fmaf_rn(R[3], sx, t[1])));
            const float pz = __fmaf_rn(R[8], sz, __fmaf_rn(R[7], sy, __fmaf_rn(R[6], sx, t[2])));
            int32_t pair = -1;
            if (isfinite(px) && isfinite(py) && isfinite(pz)) {
                float bd2 = INFINITY;
                bool limited = false;
                const int pos = nearest_within(g, px, py, pz, max_d2, r0, bd2, limited);
                float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (pos >= 0) {
                    q = __ldg(&g.pts[pos]);
                    pair = (int32_t)__float_as_uint(q.w);
                }
                if (has_delta) {  // appended points: the nearer of the two (main index on ties)
                    float bd2d = INFINITY;
                    const int posd = nearest_within(dg, px, py, pz, max_d2, r0d, bd2d, limited);
                    if (posd >= 0 && (pos < 0 || __float_as_uint(bd2d) < __float_as_uint(bd2))) {
                        q = __ldg(&dg.pts[posd]);
                        pair = (int32_t)(g.m + (int64_t)__float_as_uint(q.w));
                    }
                }
                if (limited) atomicOr(g.status, ST_SEARCH_LIMIT);
                if (pair >= 0) pair_terms(R, px, py, pz, q, map_cov + 6 * (int64_t)pair, src_cov + 6 * i, v);
            } else {
                atomicOr(g.status, ST_NONFINITE);
            }
            if (corr) corr[i] = pair;
        }
        // Reduce-scatter across the warp: at each halving step a lane keeps
        // half of its values (by its lane bit) and adds the partner's copy
        // of them; after five steps lane j holds the warp total of value j.
#pragma unroll
        for (int half = 16; half > 0; half >>= 1) {
            const bool upper = (lane & half) != 0;
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const float send = upper ? v[j] : v[j + half];
                const float keep = upper ? v[j + half] : v[j];
                v[j] = keep + __shfl_xor_sync(FULL, send, half);
            }
        }
        if (lane < GICP_VALS) acc += (double)v[0];
    }
    red[warp][lane] = acc;
    __syncthreads();
    double* part = reinterpret_cast<double*>(work + GICP_HEAD);
    if (threadIdx.x < GICP_VALS) {
        double s = 0.0;
        for (int w = 0; w < GICP_THREADS / 32; ++w) s += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * GICP_STRIDE + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(reinterpret_cast<unsigned*>(work), 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    // last block: add the block partials in block order, 8 interleaved
    // groups then the groups in order (a fixed order for a fixed grid)
    __threadfence();
    const int v = lane, grp = warp;
    double s = 0.0;
    if (v < GICP_VALS)
        for (unsigned b = grp; b < gridDim.x; b += GICP_THREADS / 32)
            s += __ldcg(&part[(size_t)b * GICP_STRIDE + v]);
    __syncthreads();
    red[grp][v] = s;
    __syncthreads();
    if (threadIdx.x < GICP_VALS) {
        double tot = 0.0;
        for (int w = 0; w < GICP_THREADS / 32; ++w) tot += red[w][threadIdx.x];
        out[threadIdx.x] = tot;
    }
    if (threadIdx.x == 0) *reinterpret_cast<unsigned*>(work) = 0u;
}

// (H + lambda I) xi = -b by Cholesky in binary64, then the pose update.
// Writes xi (6) to xi_out when given; a matrix that is not positive
// definite leaves the pose alone and writes NaN to xi.
__global__ void k_gicp_update(const double* __restrict__ lin, float lambda, float* __restrict__ pose,
                              double* __restrict__ xi_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double A[6][6], x[6];
    int w = 0;
    for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) {
            A[r][c] = lin[w];
            A[c][r] = lin[w];
            ++w;
        }
    for (int r = 0; r < 6; ++r) {
        A[r][r] += (double)lambda;
        x[r] = -lin[21 + r];
    }
    bool ok = true;
    // A = L L^T, L in the lower triangle of A
    for (int j = 0; j < 6 && ok; ++j) {
        double dsum = A[j][j];
        for (int k = 0; k < j; ++k) dsum -= A[j][k] * A[j][k];
        if (!(dsum > 0.0)) {
            ok = false;
            break;
        }
        const double ljj = sqrt(dsum);
        A[j][j] = ljj;
        for (int i = j + 1; i < 6; ++i) {
            double s = A[i][j];
            for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
            A[i][j] = s / ljj;
        }
    }
    if (ok) {
        for (int i = 0; i < 6; ++i) {  // L y = -b
            double s = x[i];
            for (int k = 0; k < i; ++k) s -= A[i][k] * x[k];
            x[i] = s / A[i][i];
        }
        for (int i = 5; i >= 0; --i) {  // L^T xi = y
            double s = x[i];
            for (int k = i + 1; k < 6; ++k) s -= A[k][i] * x[k];
            x[i] = s / A[i][i];
        }
    }
    if (xi_out)
        for (int i = 0; i < 6; ++i) xi_out[i] = ok ? x[i] : NAN;
    if (!ok) return;
    // Exp(omega) by the Rodrigues formula: I + a [w]_x + c [w]_x^2 with
    // a = sin(th)/th, c = (1 - cos(th))/th^2 (series for small th)
    const double wx = x[0], wy = x[1], wz = x[2];
    const double th2 = wx * wx + wy * wy + wz * wz;
    double a, c;
    if (th2 < 1e-12) {
        a = 1.0 - th2 / 6.0;
        c = 0.5 - th2 / 24.0;
    } else {
        const double th = sqrt(th2);
        a = sin(th) / th;
        c = (1.0 - cos(th)) / th2;
    }
    const double K[3][3] = {{0, -wz, wy}, {wz, 0, -wx}, {-wy, wx, 0}};
    double E[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double k2 = 0.0;
            for (int m = 0; m < 3; ++m) k2 += K[i][m] * K[m][j];
            E[i][j] = (i == j ? 1.0 : 0.0) + a * K[i][j] + c * k2;
        }
    double Rn[3][3], tn[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m) s += E[i][m] * (double)pose[3 * m + j];
            Rn[i][j] = s;
        }
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += E[i][m] * (double)pose[9 + m];
        tn[i] = s + x[3 + i];
    }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) pose[3 * i + j] = (float)Rn[i][j];
        pose[9 + i] = (float)tn[i];
    }
}

std::mutex g_blocks_mu;
int g_blocks[64] = {0};

// Resident blocks of the linearisation kernel on the current device.
int gicp_max_blocks() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lk(g_blocks_mu);
    if (g_blocks[dev] > 0) return g_blocks[dev];
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gicp_linearize, GICP_THREADS, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    g_blocks[dev] = sms * per_sm;
    return g_blocks[dev];
}

}  // namespace

size_t pc_gicp_work_size() {
    const int b = gicp_max_blocks();
    return b > 0 ? GICP_HEAD + (size_t)b * GICP_STRIDE * sizeof(double) : 0;
}

cudaError_t pc_launch_gicp_linearize(const pc_target_s* t, const float* map_cov, const float* src,
                                     int64_t n, const float* src_cov, const float* pose,
                                     float max_dist, double* out, int32_t* corr, void* work,
                                     float r0, float r0d, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(out, 0, GICP_VALS * sizeof(double), s);
    const int maxb = gicp_max_blocks();
    if (maxb < 1) return cudaErrorInvalidDevice;
    const int64_t need = (n + GICP_THREADS - 1) / GICP_THREADS;
    const int blocks = (int)(need < maxb ? need : maxb);
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const float max_d2 = max_dist * max_dist;
    const Grid dg = t->delta ? t->delta->g : t->g;
    k_gicp_linearize<<<blocks, GICP_THREADS, 0, s>>>(t->g, dg, t->delta ? 1 : 0, r0d, map_cov, src, n, src_cov,
                                                     pose, max_d2, r0, out, corr,
                                                     static_cast<unsigned char*>(work));
    return cudaGetLastError();
}

cudaError_t pc_launch_gicp_update(const double* lin, float lambda, float* pose, double* xi,
                                  cudaStream_t s) {
    k_gicp_update<<<1, 32, 0, s>>>(lin, lambda, pose, xi);
    return cudaGetLastError();
}
