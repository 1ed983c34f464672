// Searches over a map that grew by pc_target_append: the main grid (points
// 0 .. M-1) and a small delta grid over the appended points (M .. M+Md-1).
//
// The main grid is searched by the usual kernels.  Then one thread per query
// starts from that exact row and visits the delta points that can still
// enter it: those strictly closer than the row's k-th neighbour (a delta
// index M + j is larger than every main index, so on equal d2 the main
// point keeps its place).  The visit covers a box of the delta grid whose
// certified radius reaches that distance, so nothing closer is missed; each
// closer point is inserted into the sorted row.  A row with fewer than k
// main neighbours visits the whole delta grid.  Delta points far from a
// query are never touched, whatever their number.  The covariance of the
// final row, plain or kernel-weighted, reads each neighbour from the grid
// that owns it, in rank order.
#include "cov_weighted.cuh"

namespace {

constexpr int MAXK = 64;

struct Src {
    const float4* main_xyz;
    const float4* delta_xyz;
    int64_t m;
    __device__ __forceinline__ float4 at(int32_t gi) const {
        return gi < m ? __ldg(&main_xyz[gi]) : __ldg(&delta_xyz[gi - m]);
    }
};

// main results in idx_a/d2_a (width ka; may alias the output when ka == k)
__global__ void k_merge_delta(Src src, Grid dg, const float* __restrict__ q, int64_t N, int k, int ka,
                              const int32_t* idx_a, const float* d2_a, int32_t* idx, float* d2,
                              float* __restrict__ cov, float eps, CovKernel ck) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    typedef unsigned long long u64;
    u64 L[MAXK];
    for (int r = 0; r < k; ++r) {
        const int32_t i = r < ka ? idx_a[n * ka + r] : -1;
        L[r] = i >= 0 ? (((u64)__float_as_uint(d2_a[n * ka + r]) << 32) | (u64)(uint32_t)i) : EMPTY_KEY;
    }
    const float qx = __ldg(q + 3 * n), qy = __ldg(q + 3 * n + 1), qz = __ldg(q + 3 * n + 2);
    if (isfinite(qx) && isfinite(qy) && isfinite(qz)) {
        const float T = L[k - 1] == EMPTY_KEY ? INFINITY : __uint_as_float((uint32_t)(L[k - 1] >> 32));
        // the box of the delta grid: certified to hold every point with d2 < T
        int lx = dg.wlx, hx = dg.whx, ly = dg.wly, hy = dg.why, lz = dg.wlz, hz = dg.whz;
        float eta = 0x1p-20f * (dg.coord_scale + fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz))) +
                                (float)(max(dg.dimx, max(dg.dimy, dg.dimz)) + 2) * dg.h);
        bool whole = !(T < 1e30f);
        if (!whole) {
            float Rb = __fadd_ru(__fmul_ru(sqrtf(T), 1.0f + 0x1p-20f), 2.0f * eta);
            bool ok = false;
            for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
                const int ulx = cell_of(__fsub_rn(qx, Rb), dg.ox, dg.inv_h), uhx = cell_of(__fadd_rn(qx, Rb), dg.ox, dg.inv_h);
                const int uly = cell_of(__fsub_rn(qy, Rb), dg.oy, dg.inv_h), uhy = cell_of(__fadd_rn(qy, Rb), dg.oy, dg.inv_h);
                const int ulz = cell_of(__fsub_rn(qz, Rb), dg.oz, dg.inv_h), uhz = cell_of(__fadd_rn(qz, Rb), dg.oz, dg.inv_h);
                if (certified_tau(dg, qx, qy, qz, ulx, uhx, uly, uhy, ulz, uhz) >= T) {
                    ok = true;
                    lx = max(ulx, dg.wlx); hx = min(uhx, dg.whx);
                    ly = max(uly, dg.wly); hy = min(uhy, dg.why);
                    lz = max(ulz, dg.wlz); hz = min(uhz, dg.whz);
                    const int cm = max(max(max(abs(ulx), abs(uhx + 1)), max(abs(uly), abs(uhy + 1))),
                                       max(abs(ulz), abs(uhz + 1)));
                    eta = 0x1p-20f * (dg.coord_scale + fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz))) +
                                      (float)cm * dg.h);
                } else {
                    Rb = __fmul_ru(Rb, 1.01f) + eta;
                }
            }
            whole = !ok;
        }
        const float tmax = T;
        auto offer = [&](uint32_t, const float4 p) {
            const float d = sqdist_pinned(qx, qy, qz, p.x, p.y, p.z);
            const u64 key = ((u64)__float_as_uint(d) << 32) | (u64)(uint32_t)(src.m + (int64_t)__float_as_uint(p.w));
            if (!(key < L[k - 1])) return;
            int r = k - 1;
            while (r > 0 && key < L[r - 1]) {
                L[r] = L[r - 1];
                --r;
            }
            L[r] = key;
        };
        if (whole) {
            // no bound: every occupied cell of the delta grid inside its window
            const u64 mx = (1ull << dg.bx) - 1ull, my = (1ull << dg.by) - 1ull;
            for (int64_t u = 0; u < dg.ncells; ++u) {
                const u64 key = dg.cell_keys[u];
                const int cx = (int)(key & mx), cy = (int)((key >> dg.bx) & my), cz = (int)(key >> (dg.bx + dg.by));
                if (cx < dg.wlx || cx > dg.whx || cy < dg.wly || cy > dg.why || cz < dg.wlz || cz > dg.whz) continue;
                const bool test = dg.windowed && (cx == dg.tlx || cx == dg.thx || cy == dg.tly || cy == dg.thy ||
                                                  cz == dg.tlz || cz == dg.thz);
                for (uint32_t i = dg.cell_start[u]; i < dg.cell_start[u + 1]; ++i)
                    offer(i, window_cut<true>(dg, test, __ldg(&dg.pts[i])));
            }
        } else if (lx <= hx && ly <= hy && lz <= hz) {
            if (dg.occ) for_rows<true>(dg, qx, qy, qz, lx, hx, ly, hy, lz, hz, eta, tmax, offer);
            else for_box_points<true>(dg, qx, qy, qz, lx, hx, ly, hy, lz, hz, eta, tmax, offer);
        }
    }
    int32_t oi[MAXK];
    bool full = true;
    for (int r = 0; r < k; ++r) {
        const bool v = L[r] != EMPTY_KEY;
        full = full && v;
        oi[r] = v ? (int32_t)(uint32_t)L[r] : -1;
        idx[n * k + r] = oi[r];
        d2[n * k + r] = v ? __uint_as_float((uint32_t)(L[r] >> 32)) : INFINITY;
    }
    if (!cov) return;
    float* out = cov + 6 * n;
    if (!full) {
        nan_row(out);
        return;
    }
    auto get = [&](int j) { return src.at(oi[j]); };
    if (ck.type == 0) cov_core(get, k, eps, out);
    else weighted_core(get, ck, qx, qy, qz, k, eps, out);
}

// pc_cov over the union: neighbour rows are global indices
__global__ void k_cov_union(Src src, const int32_t* __restrict__ idx, int64_t N, int k, int64_t mtot, float eps,
                            float* __restrict__ cov, int* status) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int32_t* nb = idx + n * k;
    bool oob = false;
    for (int j = 0; j < k; ++j) oob |= nb[j] < 0 || (int64_t)nb[j] >= mtot;
    if (oob) {
        atomicOr(status, ST_BAD_INDEX);
        nan_row(cov + 6 * n);
        return;
    }
    cov_core([&](int j) { return src.at(nb[j]); }, k, eps, cov + 6 * n);
}

// the main map (caller order) then the appended points, as f32 [M+Md, 3]
__global__ void k_pack_xyz(const float4* __restrict__ main_xyz, int64_t m, const float* __restrict__ delta,
                           int64_t md, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m + md) return;
    if (i < m) {
        const float4 p = main_xyz[i];
        out[3 * i] = p.x;
        out[3 * i + 1] = p.y;
        out[3 * i + 2] = p.z;
    } else {
        out[3 * i] = delta[3 * (i - m)];
        out[3 * i + 1] = delta[3 * (i - m) + 1];
        out[3 * i + 2] = delta[3 * (i - m) + 2];
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t pc_union_temp_bytes(const pc_target_s* t, int64_t N, int k) {
    const int ka = (int)std::min<int64_t>(k, t->g.m);
    if (ka == k) return 0;
    return align256(sizeof(int32_t) * N * ka) + align256(sizeof(float) * N * ka);
}

cudaError_t pc_launch_knn_union(const pc_target_s* t, const float* q, int64_t N, int k, float eps,
                                int32_t* idx, float* d2, float* cov, void* temp, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int ka = (int)std::min<int64_t>(k, t->g.m);
    int32_t* ia = idx;
    float* da = d2;
    if (ka != k) {  // a main grid with fewer than k points: its rows go to the staging area
        char* base = static_cast<char*>(temp);
        ia = reinterpret_cast<int32_t*>(base);
        da = reinterpret_cast<float*>(base + align256(sizeof(int32_t) * N * ka));
    }
    cudaError_t e = pc_launch_knn(t, q, N, ka, -1.0f, ia, da, nullptr, pc_rho0(t, ka), s);
    if (e != cudaSuccess) return e;
    Src src{t->g.xyz, t->delta->g.xyz, t->g.m};
    const int threads = 128;
    k_merge_delta<<<(unsigned)((N + threads - 1) / threads), threads, 0, s>>>(src, t->delta->g, q, N, k, ka, ia, da,
                                                                             idx, d2, cov, eps, t->ck);
    return cudaGetLastError();
}

cudaError_t pc_launch_cov_union(const pc_target_s* t, const int32_t* idx, int64_t N, int k, float eps,
                                float* cov, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    Src src{t->g.xyz, t->delta->g.xyz, t->g.m};
    const int threads = 128;
    k_cov_union<<<(unsigned)((N + threads - 1) / threads), threads, 0, s>>>(src, idx, N, k, t->g.m + t->delta_m,
                                                                           eps, cov, t->g.status);
    return cudaGetLastError();
}

cudaError_t pc_launch_pack_xyz(const pc_target_s* t, float* out, cudaStream_t s) {
    const int64_t tot = t->g.m + t->delta_m;
    if (tot == 0) return cudaSuccess;
    const int threads = 256;
    k_pack_xyz<<<(unsigned)((tot + threads - 1) / threads), threads, 0, s>>>(t->g.xyz, t->g.m, t->delta_xyz,
                                                                            t->delta_m, out);
    return cudaGetLastError();
}
