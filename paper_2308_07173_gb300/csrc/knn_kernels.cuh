// The search and covariance kernels, shared by knn_cov.cu (whole-map
// searches) and knn_window.cu (searches restricted to a window, WIN = true):
// each translation unit instantiates one window variant, so the whole-map
// kernels carry no window code and the two compile in parallel.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <utility>

#include "pc_device.cuh"
#include "pc_internal.h"
#include "pc_search.cuh"

using namespace pcdev;

namespace {

typedef unsigned long long u64;

__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }
__device__ __forceinline__ u64 umax64(u64 a, u64 b) { return a < b ? b : a; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Bitonic sort of one key per lane into DESCENDING lane order.
__device__ __forceinline__ u64 sort32_desc(u64 x, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            u64 y = __shfl_xor_sync(FULL, x, stride);
            bool desc_block = (lane & size) == 0;  // all lanes at size 32
            bool lower = (lane & stride) == 0;
            x = (lower == desc_block) ? umax64(x, y) : umin64(x, y);
        }
    }
    return x;
}

// Bitonic merge of a bitonic lane sequence into ASCENDING lane order.
__device__ __forceinline__ u64 merge32_asc(u64 x, int lane) {
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        u64 y = __shfl_xor_sync(FULL, x, stride);
        x = ((lane & stride) == 0) ? umin64(x, y) : umax64(x, y);
    }
    return x;
}

template <int SLOTS>
struct SearchState {
    u64 L[SLOTS];  // lane l: rank l (slot 0) and rank 32 + l (slot 1)
    u64 kth;       // warp-uniform: the rank k-1 key, EMPTY_KEY until k exist
    int npend;     // warp-uniform: survivors staged in shared memory
};

template <int SLOTS>
__device__ __forceinline__ void state_reset(SearchState<SLOTS>& S) {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) S.L[s] = EMPTY_KEY;
    S.kth = EMPTY_KEY;
    S.npend = 0;
}

template <int SLOTS>
__device__ __forceinline__ u64 topk_rank(const SearchState<SLOTS>& S, int r) {
    u64 v = (SLOTS == 2 && r >= 32) ? S.L[SLOTS - 1] : S.L[0];
    return __shfl_sync(FULL, v, r & 31);
}

// Merge 32 staged keys (one per lane, any order) into the sorted top list.
// A ascending + B descending -> min(A, B) is bitonic and holds the smallest
// |A| of A u B; for two slots the 64-list [L0, min(L1, c)] is bitonic.
template <int SLOTS>
__device__ __forceinline__ void topk_merge(SearchState<SLOTS>& S, u64 c, int k, int lane) {
    c = sort32_desc(c, lane);
    if (SLOTS == 1) {
        S.L[0] = merge32_asc(umin64(S.L[0], c), lane);
    } else {
        u64 b = umin64(S.L[SLOTS - 1], c);
        u64 lo = umin64(S.L[0], b), hi = umax64(S.L[0], b);
        S.L[0] = merge32_asc(lo, lane);
        S.L[SLOTS - 1] = merge32_asc(hi, lane);
    }
    S.kth = topk_rank(S, k - 1);
}

template <int SLOTS>
__device__ __forceinline__ void offer(SearchState<SLOTS>& S, bool pass, u64 key, u64* pend, int k,
                                      int lane) {
    unsigned m = __ballot_sync(FULL, pass);
    if (m == 0u) return;
    if (pass) pend[S.npend + __popc(m & lanemask_lt())] = key;
    S.npend += __popc(m);
    __syncwarp();
    if (S.npend >= 32) {
        topk_merge(S, pend[lane], k, lane);
        __syncwarp();
        const int rest = S.npend - 32;
        if (lane < rest) pend[lane] = pend[32 + lane];
        __syncwarp();
        S.npend = rest;
    }
}

template <int SLOTS>
__device__ __forceinline__ void flush(SearchState<SLOTS>& S, u64* pend, int k, int lane) {
    if (S.npend > 0) {
        u64 c = lane < S.npend ? pend[lane] : EMPTY_KEY;
        topk_merge(S, c, k, lane);
        S.npend = 0;
    }
    __syncwarp();
}

// One pass over up to 32 point ranges (one per lane): every point becomes a
// candidate, 32 per step, each lane finding its owning range by a binary
// search over the warp's exclusive prefix of counts.  Keys carry the point's
// index plus ibase (the appended-points grid numbers its points after the
// main grid's).
template <int SLOTS>
__device__ __forceinline__ void scan_ranges(const Grid& g, float qx, float qy, float qz,
                                            uint32_t start, uint32_t cnt, float tau,
                                            SearchState<SLOTS>& S, u64* pend, int k, int lane,
                                            uint32_t ibase) {
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t excl = incl - cnt;
    for (uint32_t cb = 0; cb < total; cb += 32) {
        const uint32_t t = cb + lane;
        int j = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            uint32_t e = __shfl_sync(FULL, excl, j + s);
            if (e <= t) j += s;
        }
        const uint32_t st = __shfl_sync(FULL, start, j);
        const uint32_t ej = __shfl_sync(FULL, excl, j);
        bool pass = false;
        u64 key = EMPTY_KEY;
        if (t < total) {
            const float4 p = __ldg(&g.pts[st + (t - ej)]);
            const float d2 = sqdist_pinned(qx, qy, qz, p.x, p.y, p.z);
            key = ((u64)__float_as_uint(d2) << 32) | (u64)(__float_as_uint(p.w) + ibase);
            pass = (d2 <= tau) && (key < S.kth) && (!g.windowed || in_window(g, p));
        }
        offer(S, pass, key, pend, k, lane);
    }
}

// Lower bound on the binary32 d2 from q to any point of cell (cx, cy, cz);
// same margin argument as certified_tau.
__device__ __forceinline__ float cell_lower_bound2(const Grid& g, float qx, float qy, float qz,
                                                   int cx, int cy, int cz) {
    float qm = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
    int cm = max(cx, max(cy, cz)) + 1;
    float eta = 0x1p-20f * (g.coord_scale + qm + (float)cm * g.h);
    float s = 0.0f;
    {
        float lo = g.ox + (float)cx * g.h, hi = g.ox + (float)(cx + 1) * g.h;
        float d = fmaxf(fmaxf(lo - qx, qx - hi), 0.0f) - eta;
        if (d > 0.0f) s = s + d * d;
    }
    {
        float lo = g.oy + (float)cy * g.h, hi = g.oy + (float)(cy + 1) * g.h;
        float d = fmaxf(fmaxf(lo - qy, qy - hi), 0.0f) - eta;
        if (d > 0.0f) s = s + d * d;
    }
    {
        float lo = g.oz + (float)cz * g.h, hi = g.oz + (float)(cz + 1) * g.h;
        float d = fmaxf(fmaxf(lo - qz, qz - hi), 0.0f) - eta;
        if (d > 0.0f) s = s + d * d;
    }
    return s * (1.0f - 0x1p-20f);
}

template <int SLOTS>
__device__ void scan_box(const Grid& g, float qx, float qy, float qz, int lx, int ly, int lz,
                         int ex, int ey, int ez, float tau, SearchState<SLOTS>& S, u64* pend,
                         int k, int lane, uint32_t ibase) {
    const int ncl = ex * ey * ez;
    for (int base = 0; base < ncl; base += 32) {
        const int c = base + lane;
        uint32_t start = 0u, cnt = 0u;
        if (c < ncl) {
            const int cx = lx + c % ex;
            const int r = c / ex;
            const int cy = ly + r % ey;
            const int cz = lz + r / ey;
            const uint2 v = lookup_cell(g, pack_key(cx, cy, cz, g.bx, g.by));
            start = v.x;
            cnt = v.y;
        }
        scan_ranges(g, qx, qy, qz, start, cnt, tau, S, pend, k, lane, ibase);
    }
}

template <int SLOTS>
__device__ void scan_all_cells(const Grid& g, float qx, float qy, float qz, SearchState<SLOTS>& S,
                               u64* pend, int k, int lane, uint32_t ibase) {
    const u64 mx = (1ull << g.bx) - 1ull, my = (1ull << g.by) - 1ull;
    for (int64_t ub = 0; ub < g.ncells; ub += 32) {
        const int64_t u = ub + lane;
        uint32_t start = 0u, cnt = 0u;
        if (u < g.ncells) {
            const u64 key = g.cell_keys[u];
            const int cx = (int)(key & mx), cy = (int)((key >> g.bx) & my),
                      cz = (int)(key >> (g.bx + g.by));
            const float lb2 = cell_lower_bound2(g, qx, qy, qz, cx, cy, cz);
            const float kd = S.kth == EMPTY_KEY ? INFINITY : __uint_as_float((uint32_t)(S.kth >> 32));
            const bool win = cx >= g.wlx && cx <= g.whx && cy >= g.wly && cy <= g.why &&
                             cz >= g.wlz && cz <= g.whz;
            if (win && lb2 <= kd) {
                start = g.cell_start[u];
                cnt = g.cell_start[u + 1] - start;
            }
        }
        scan_ranges(g, qx, qy, qz, start, cnt, INFINITY, S, pend, k, lane, ibase);
    }
}

// The cell box of radius rho around q on one grid, clamped to its window
// range (the whole grid when no window is set), and the certified tau of
// the unclamped box.
struct WarpBox {
    int lx, ly, lz;
    int ex, ey, ez;
    int64_t ncl;
    float tau;
};

__device__ __forceinline__ WarpBox warp_box(const Grid& g, float qx, float qy, float qz, float rho) {
    const int lx = cell_of(__fsub_rn(qx, rho), g.ox, g.inv_h);
    const int hx = cell_of(__fadd_rn(qx, rho), g.ox, g.inv_h);
    const int ly = cell_of(__fsub_rn(qy, rho), g.oy, g.inv_h);
    const int hy = cell_of(__fadd_rn(qy, rho), g.oy, g.inv_h);
    const int lz = cell_of(__fsub_rn(qz, rho), g.oz, g.inv_h);
    const int hz = cell_of(__fadd_rn(qz, rho), g.oz, g.inv_h);
    WarpBox b;
    b.tau = certified_tau(g, qx, qy, qz, lx, hx, ly, hy, lz, hz);
    b.lx = max(lx, g.wlx);
    b.ly = max(ly, g.wly);
    b.lz = max(lz, g.wlz);
    b.ex = max(min(hx, g.whx) - b.lx + 1, 0);
    b.ey = max(min(hy, g.why) - b.ly + 1, 0);
    b.ez = max(min(hz, g.whz) - b.lz + 1, 0);
    b.ncl = (int64_t)b.ex * b.ey * b.ez;
    return b;
}

// Exact k nearest neighbours of one query (warp-uniform control flow).
// Returns SEARCH_OK, SEARCH_LIMIT (max_box_cells reached with exhaustive =
// 0) or SEARCH_SHORT (the exhaustive scan found fewer than k points: the
// window holds fewer than k).  With DEL the search runs over the union of
// g and the appended-points grid dg, whose point j is g.m + j: every
// attempt scans both grids' boxes of the same radius, filtered by the
// smaller of their two certified taus (a point of either grid outside its
// box lies beyond both), and the exhaustive scan covers both grids.
constexpr int SEARCH_OK = 0, SEARCH_LIMIT = 1, SEARCH_SHORT = 2;
template <int SLOTS, bool DEL>
__device__ int knn_search(const Grid& g, const Grid& dg, float qx, float qy, float qz, int k, float& rho,
                          SearchState<SLOTS>& S, u64* pend, int lane) {
    for (int attempt = 0; attempt < 40; ++attempt) {
        const WarpBox b = warp_box(g, qx, qy, qz, rho);
        WarpBox d = b;
        float tau = b.tau;
        if (DEL) {
            d = warp_box(dg, qx, qy, qz, rho);
            tau = fminf(tau, d.tau);
            if (d.ncl > (int64_t)dg.max_box_cells) break;
        }
        if (b.ncl > (int64_t)g.max_box_cells) break;
        state_reset(S);
        if (b.ncl > 0) scan_box(g, qx, qy, qz, b.lx, b.ly, b.lz, b.ex, b.ey, b.ez, tau, S, pend, k, lane, 0u);
        if (DEL && d.ncl > 0)
            scan_box(dg, qx, qy, qz, d.lx, d.ly, d.lz, d.ex, d.ey, d.ez, tau, S, pend, k, lane, (uint32_t)g.m);
        flush(S, pend, k, lane);
        if (S.kth != EMPTY_KEY) return SEARCH_OK;
        int found = 0;
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) found += __popc(__ballot_sync(FULL, S.L[s] != EMPTY_KEY));
        float f = 1.3f * sqrtf((float)k / (float)max(found, 1));
        f = fminf(fmaxf(f, 1.5f), 4.0f);
        rho = fminf(fmaxf(rho, 1e-3f * g.h) * f, 1e30f);
    }
    if (!g.exhaustive) return SEARCH_LIMIT;
    if (lane == 0) atomicAdd(&g.stats[2], 1ull);
    state_reset(S);
    scan_all_cells(g, qx, qy, qz, S, pend, k, lane, 0u);
    if (DEL) scan_all_cells(dg, qx, qy, qz, S, pend, k, lane, (uint32_t)g.m);
    flush(S, pend, k, lane);
    return S.kth != EMPTY_KEY ? SEARCH_OK : SEARCH_SHORT;
}

// ---------------------------------------------------------------- covariance

// Unit null vector of the symmetric 3x3 matrix with rows r0, r1, r2 (of
// rank 2 up to rounding): the cross product of two rows is orthogonal to
// both, and of the three pairs the one with the largest cross product is
// the best conditioned.  A zero matrix gives e_z.
__host__ __device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

__host__ __device__ __forceinline__ float3 null_vector(float3 r0, float3 r1, float3 r2) {
    const float3 c01 = cross3(r0, r1), c02 = cross3(r0, r2), c12 = cross3(r1, r2);
    const float d01 = dot3(c01, c01), d02 = dot3(c02, c02), d12 = dot3(c12, c12);
    float3 c = c01;
    float d = d01;
    if (d02 > d) { c = c02; d = d02; }
    if (d12 > d) { c = c12; d = d12; }
    if (!(d > 0.0f)) return make_float3(0.0f, 0.0f, 1.0f);
    const float inv = 1.0f / sqrtf(d);
    return make_float3(c.x * inv, c.y * inv, c.z * inv);
}

// Unit eigenvector of the smallest eigenvalue of a symmetric 3x3 matrix A,
// in closed form, binary32.  The matrix is first scaled by an exact power
// of two; a zero matrix gives e_z.
//
// Eigenvalues by the trigonometric form (Smith 1961): with m = tr(A)/3,
// B = A - m I, p = sqrt(tr(B^2)/6) and r = det(B)/(2 p^3) in [-1, 1],
// phi = acos(r)/3, the eigenvalues are m + 2p cos(phi + 2 pi j/3),
// j = 0 (largest), 1 (smallest), 2.  Which one is computed decides the
// accuracy (the hybrid of Kopp 2008, "Efficient numerical diagonalization
// of hermitian 3x3 matrices"):
// * r < 0: the middle eigenvalue is nearer the largest, so the smallest is
//   the isolated one (lambda2 - lambda3 >= (lambda1 - lambda3)/2) and its
//   value has a bounded derivative in r.  The normal is the null vector of
//   A - lambda3 I.
// * r >= 0: the two smallest are the close pair; the largest is isolated
//   and accurate, its eigenvector e1 is the null vector of A - lambda1 I,
//   and the normal is the smaller eigenvector of A restricted to the plane
//   orthogonal to e1 (a 2x2 problem solved by one Jacobi rotation, exact
//   for any separation of the pair, a repeated pair included).
// Either way the normal's error is ~ u ||A|| / (lambda2 - lambda3), the
// perturbation bound itself, as for an iterative solver.
__host__ __device__ float3 min_eigvec(float a00, float a01, float a02, float a11, float a12, float a22) {
    const float amax = fmaxf(fmaxf(fabsf(a00), fabsf(a11)),
                             fmaxf(fabsf(a22), fmaxf(fmaxf(fabsf(a01), fabsf(a02)), fabsf(a12))));
    if (!(amax > 0.0f) || !isfinite(amax)) return make_float3(0.0f, 0.0f, 1.0f);
    int e;
    frexpf(amax, &e);
    const float sc = ldexpf(1.0f, -e);
    a00 *= sc; a01 *= sc; a02 *= sc; a11 *= sc; a12 *= sc; a22 *= sc;
    const float m = (a00 + a11 + a22) / 3.0f;
    const float b00 = a00 - m, b11 = a11 - m, b22 = a22 - m;
    const float p2 = (b00 * b00 + b11 * b11 + b22 * b22 + 2.0f * (a01 * a01 + a02 * a02 + a12 * a12)) / 6.0f;
    if (!(p2 > 0.0f)) return make_float3(0.0f, 0.0f, 1.0f);  // A = m I: every direction
    const float p = sqrtf(p2);
    const float det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) + a02 * (a01 * a12 - b11 * a02);
    const float r = fminf(fmaxf(det / (2.0f * p2 * p), -1.0f), 1.0f);
    const float phi = acosf(r) / 3.0f;
    if (r < 0.0f) {
        const float l3 = m + 2.0f * p * cosf(phi + 2.09439510f);
        return null_vector(make_float3(a00 - l3, a01, a02), make_float3(a01, a11 - l3, a12),
                           make_float3(a02, a12, a22 - l3));
    }
    const float l1 = m + 2.0f * p * cosf(phi);
    const float3 e1 = null_vector(make_float3(a00 - l1, a01, a02), make_float3(a01, a11 - l1, a12),
                                  make_float3(a02, a12, a22 - l1));
    // orthonormal u, v spanning the plane orthogonal to e1
    const float ax = fabsf(e1.x), ay = fabsf(e1.y), az = fabsf(e1.z);
    const float3 w = (ax <= ay && ax <= az) ? make_float3(1.0f, 0.0f, 0.0f)
                   : (ay <= az ? make_float3(0.0f, 1.0f, 0.0f) : make_float3(0.0f, 0.0f, 1.0f));
    float3 u = cross3(e1, w);
    const float iu = 1.0f / sqrtf(dot3(u, u));
    u = make_float3(u.x * iu, u.y * iu, u.z * iu);
    const float3 v = cross3(e1, u);
    const float3 Au = make_float3(a00 * u.x + a01 * u.y + a02 * u.z, a01 * u.x + a11 * u.y + a12 * u.z,
                                  a02 * u.x + a12 * u.y + a22 * u.z);
    const float3 Av = make_float3(a00 * v.x + a01 * v.y + a02 * v.z, a01 * v.x + a11 * v.y + a12 * v.z,
                                  a02 * v.x + a12 * v.y + a22 * v.z);
    const float suu = dot3(u, Au), suv = dot3(v, Au), svv = dot3(v, Av);
    // the rotation (c, s) that diagonalises [[suu, suv], [suv, svv]] (the
    // smaller root t of t^2 + 2 t theta - 1 = 0, Golub & Van Loan sec. 8.5):
    // eigenvector (c, -s) for suu - t suv, (s, c) for svv + t suv
    float c = 1.0f, sn = 0.0f, lu = suu, lv = svv;
    if (suv != 0.0f) {
        const float theta = (svv - suu) / (2.0f * suv);
        const float at = fabsf(theta);
        const float t = at > 1e18f ? 0.5f / theta : copysignf(1.0f, theta) / (at + sqrtf(theta * theta + 1.0f));
        c = 1.0f / sqrtf(t * t + 1.0f);
        sn = t * c;
        lu = suu - t * suv;
        lv = svv + t * suv;
    }
    const float x = lu <= lv ? c : sn, y = lu <= lv ? -sn : c;
    const float3 nv = make_float3(x * u.x + y * v.x, x * u.y + y * v.y, x * u.z + y * v.z);
    const float in = 1.0f / sqrtf(dot3(nv, nv));
    return make_float3(nv.x * in, nv.y * in, nv.z * in);
}

// Covariance of one neighbourhood (Sec. III-C1, C_i of Eq. 19) from its
// points in rank order, get(j) for j = 0..k-1.  Two passes in binary32,
// both shifted by the first (nearest) neighbour p0 so the sums stay small:
// mean m of (p_j - p0), then the centred moments of (p_j - p0) - m, divided
// by k.  Built with --fmad=false, so every + and * below is rounded once;
// every caller runs this same code on the same values, so the fused kernel
// and pc_cov agree bit for bit.
// The six packed entries of one covariance row: three 8-byte stores when
// the row is 8-byte aligned (every row of an aligned [N,6] array is).
__device__ __forceinline__ void store6(float* out, float a, float b, float c, float d, float e, float f) {
    if ((reinterpret_cast<uintptr_t>(out) & 7) == 0) {
        float2* o2 = reinterpret_cast<float2*>(out);
        o2[0] = make_float2(a, b);
        o2[1] = make_float2(c, d);
        o2[2] = make_float2(e, f);
    } else {
        out[0] = a; out[1] = b; out[2] = c; out[3] = d; out[4] = e; out[5] = f;
    }
}

// The end of every plain covariance: centred sums / k, then, for eps >= 0,
// the plane regularisation C' = I - (1 - eps) n n^T; stored packed.
__device__ __forceinline__ void cov_finish(float cxx, float cxy, float cxz, float cyy, float cyz, float czz,
                                           float fk, float eps, float* out) {
    cxx = cxx / fk; cxy = cxy / fk; cxz = cxz / fk;
    cyy = cyy / fk; cyz = cyz / fk; czz = czz / fk;
    if (eps < 0.0f) {
        store6(out, cxx, cxy, cxz, cyy, cyz, czz);
        return;
    }
    const float3 n = min_eigvec(cxx, cxy, cxz, cyy, cyz, czz);
    const float f = 1.0f - eps;
    store6(out, 1.0f - f * n.x * n.x, -f * n.x * n.y, -f * n.x * n.z, 1.0f - f * n.y * n.y, -f * n.y * n.z,
           1.0f - f * n.z * n.z);
}

template <typename G>
__device__ __forceinline__ void cov_core(G&& get, int k, float eps, float* out) {
    const float4 p0 = get(0);
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int j = 0; j < k; ++j) {
        const float4 p = get(j);
        sx = sx + (p.x - p0.x);
        sy = sy + (p.y - p0.y);
        sz = sz + (p.z - p0.z);
    }
    const float fk = (float)k;
    const float mx = sx / fk, my = sy / fk, mz = sz / fk;
    float cxx = 0.0f, cxy = 0.0f, cxz = 0.0f, cyy = 0.0f, cyz = 0.0f, czz = 0.0f;
    for (int j = 0; j < k; ++j) {
        const float4 p = get(j);
        const float dx = (p.x - p0.x) - mx;
        const float dy = (p.y - p0.y) - my;
        const float dz = (p.z - p0.z) - mz;
        cxx = __fmaf_rn(dx, dx, cxx);
        cxy = __fmaf_rn(dx, dy, cxy);
        cxz = __fmaf_rn(dx, dz, cxz);
        cyy = __fmaf_rn(dy, dy, cyy);
        cyz = __fmaf_rn(dy, dz, cyz);
        czz = __fmaf_rn(dz, dz, czz);
    }
    cov_finish(cxx, cxy, cxz, cyy, cyz, czz, fk, eps, out);
}

__device__ __forceinline__ void nan_row(float* out) {
    const float nan = __int_as_float(0x7fc00000);
    for (int e = 0; e < 6; ++e) out[e] = nan;
}

// Covariance of the neighbourhood row nb[0], nb[st], ..., nb[(k-1) st]
// (caller indices, read from the caller-order copy).  `check`: validate
// every index (pc_cov); otherwise a leading -1 marks an unanswered row.
__device__ void cov_row(const Grid& g, const int32_t* nb, int st, int k, float eps, float* out,
                        bool check) {
    bool bad = nb[0] < 0;
    if (check) {
        bool oob = false;
        for (int j = 0; j < k; ++j) oob |= (nb[j * st] < 0) || ((int64_t)nb[j * st] >= g.m);
        if (oob) atomicOr(g.status, ST_BAD_INDEX);
        bad = oob;
    }
    if (bad) {
        nan_row(out);
        return;
    }
    cov_core([&](int j) { return __ldg(&g.xyz[nb[j * st]]); }, k, eps, out);
}

// Positions in the lane lists: a main-grid position, or an appended-points
// grid position with DTAG set (both grids hold fewer than 2^31 points).
constexpr uint32_t DTAG = 0x80000000u;

template <bool DEL>
__device__ __forceinline__ float4 pt_at(const Grid& g, const Grid& dg, uint32_t tp) {
    if (!DEL) return __ldg(&g.pts[tp]);
    const float4* base = (tp & DTAG) ? dg.pts : g.pts;
    return __ldg(&base[tp & ~DTAG]);
}

// Index of the point at tagged position tp in the union numbering: main
// points keep their index, appended point j is g.m + j.
template <bool DEL>
__device__ __forceinline__ uint32_t union_index(const Grid& g, uint32_t tp, float4 p) {
    const uint32_t i = __float_as_uint(p.w);
    return (DEL && (tp & DTAG)) ? (uint32_t)g.m + i : i;
}

// cov_row over the union numbering (a leading -1 marks an unanswered row).
template <bool DEL>
__device__ void cov_row_union(const Grid& g, const Grid& dg, const int32_t* nb, int k, float eps, float* out) {
    if (!DEL) {
        cov_row(g, nb, 1, k, eps, out, false);
        return;
    }
    if (nb[0] < 0) {
        nan_row(out);
        return;
    }
    cov_core([&](int j) {
        const int64_t i = nb[j];
        return i < g.m ? __ldg(&g.xyz[i]) : __ldg(&dg.xyz[i - g.m]);
    }, k, eps, out);
}

// Kernel-descriptor weighted covariance of one neighbourhood (Sec. III-C1:
// the covariance is computed "using the kernel descriptors" of Table I).
// For query x = q and its k neighbours y_j in rank order:
//   w_j = K(x, y_j),  W = sum w_j,
//   mu = sum w_j y_j / W,  C = sum w_j (y_j - mu)(y_j - mu)^T / W,
// then, for eps >= 0, C' = I - (1 - eps) n n^T with n the smallest-eigenvalue
// eigenvector (the same Jacobi solver as the plain covariance).  Binary32,
// two passes shifted by the nearest neighbour y_0 like the plain form.  A row
// whose W is not positive and finite is NaN.  The search kernels call it in
// place of cov_core when a descriptor is set, reading the neighbours from the
// cell-sorted copy they already hold in cache.
__device__ __forceinline__ float kd_weight(const CovKernel& ck, float qx, float qy, float qz, float4 p) {
    const float dx = qx - p.x, dy = qy - p.y, dz = qz - p.z;
    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
    switch (ck.type) {
        case 1:  // RBF
        case 2:  // Gaussian (s = 1 / (2 sigma^2))
            return expf(-r2 * ck.s);
        case 3: {  // Polynomial on coordinates relative to the bounding-box minimum
            const float ax = qx - ck.ox, ay = qy - ck.oy, az = qz - ck.oz;
            const float bx = p.x - ck.ox, by = p.y - ck.oy, bz = p.z - ck.oz;
            const float dot = __fmaf_rn(az, bz, __fmaf_rn(ay, by, ax * bx));
            return powf(__fmaf_rn(ck.alpha, dot, ck.c), ck.d);
        }
        case 4: {  // histogram intersection, same relative coordinates
            const float ax = qx - ck.ox, ay = qy - ck.oy, az = qz - ck.oz;
            const float bx = p.x - ck.ox, by = p.y - ck.oy, bz = p.z - ck.oz;
            return (fminf(ax, bx) + fminf(ay, by) + fminf(az, bz)) / (ax + ay + az);
        }
        case 5:  // Laplacian (s = 1 / sigma)
            return expf(-sqrtf(r2) * ck.s);
    }
    return 1.0f;
}

template <typename G>
__device__ void weighted_core(G&& get, const CovKernel& ck, float qx, float qy, float qz, int k, float eps,
                              float* out) {
    if (!isfinite(qx) || !isfinite(qy) || !isfinite(qz)) {
        nan_row(out);
        return;
    }
    const float4 p0 = get(0);
    float W = 0.0f, sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int j = 0; j < k; ++j) {
        const float4 p = get(j);
        const float w = kd_weight(ck, qx, qy, qz, p);
        W = W + w;
        sx = __fmaf_rn(w, p.x - p0.x, sx);
        sy = __fmaf_rn(w, p.y - p0.y, sy);
        sz = __fmaf_rn(w, p.z - p0.z, sz);
    }
    if (!(W > 0.0f) || !isfinite(W)) {
        nan_row(out);
        return;
    }
    const float mx = sx / W, my = sy / W, mz = sz / W;
    float cxx = 0.0f, cxy = 0.0f, cxz = 0.0f, cyy = 0.0f, cyz = 0.0f, czz = 0.0f;
    for (int j = 0; j < k; ++j) {
        const float4 p = get(j);
        const float w = kd_weight(ck, qx, qy, qz, p);
        const float dx = (p.x - p0.x) - mx, dy = (p.y - p0.y) - my, dz = (p.z - p0.z) - mz;
        const float wx = w * dx, wy = w * dy;
        cxx = __fmaf_rn(wx, dx, cxx);
        cxy = __fmaf_rn(wx, dy, cxy);
        cxz = __fmaf_rn(wx, dz, cxz);
        cyy = __fmaf_rn(wy, dy, cyy);
        cyz = __fmaf_rn(wy, dz, cyz);
        czz = __fmaf_rn(w * dz, dz, czz);
    }
    cxx = cxx / W; cxy = cxy / W; cxz = cxz / W;
    cyy = cyy / W; cyz = cyz / W; czz = czz / W;
    if (eps < 0.0f) {
        out[0] = cxx; out[1] = cxy; out[2] = cxz; out[3] = cyy; out[4] = cyz; out[5] = czz;
        return;
    }
    const float3 n = min_eigvec(cxx, cxy, cxz, cyy, cyz, czz);
    const float f = 1.0f - eps;
    out[0] = 1.0f - f * n.x * n.x;
    out[1] = -f * n.x * n.y;
    out[2] = -f * n.x * n.z;
    out[3] = 1.0f - f * n.y * n.y;
    out[4] = -f * n.y * n.z;
    out[5] = 1.0f - f * n.z * n.z;
}

// ---------------------------------------------------------------- tiles
struct TileArgs {
    int k;
    float eps;
    float rho_scale;
    int last_first;  // issue tiles from the end of the query array
    CovKernel ck;    // kernel-descriptor weights; type 0: the plain covariance
    float probe_c;   // > 0: each lane estimates its own starting radius (probe_radius)
};

// The covariance of a written row (caller or union indices; a leading -1
// marks an unanswered row), plain or weighted by the descriptor in a.
template <bool DEL>
__device__ void cov_row_any(const Grid& g, const Grid& dg, const int32_t* nb, int k, const TileArgs& a, float qx,
                            float qy, float qz, float* out) {
    if (a.ck.type == 0) {
        cov_row_union<DEL>(g, dg, nb, k, a.eps, out);
        return;
    }
    if (nb[0] < 0) {
        nan_row(out);
        return;
    }
    weighted_core([&](int j) {
        const int64_t i = nb[j];
        return (!DEL || i < g.m) ? __ldg(&g.xyz[i]) : __ldg(&dg.xyz[i - g.m]);
    }, a.ck, qx, qy, qz, k, a.eps, out);
}

// Per-warp shared memory: 64 staged survivor keys of the warp-cooperative
// search, then the lane path's survivor lists: 32 slots x 32 lanes of
// positions into pts ([slot][lane], so a slot is one 128-byte row).
// Search modes: 0 = lane path with room for 32 survivors (k <= 24),
// 1 = lane path with room for 64 (k <= 32), 2 = warp path only (k > 32).
__host__ __device__ __forceinline__ int lane_cap(int mode) { return mode == 0 ? 32 : mode == 1 ? 64 : 0; }
__host__ __device__ __forceinline__ int search_mode(int k) { return k <= 24 ? 0 : (k <= 32 ? 1 : 2); }
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int mode) {
    return 64 * sizeof(u64) + (size_t)lane_cap(mode) * 32 * sizeof(uint32_t);
}
// Staging area of a warp whose outputs go to host memory: the tile's idx
// rows, d2 rows and covariance rows, each laid out as in the output arrays.
__host__ __device__ __forceinline__ size_t stage_bytes(int k) { return (size_t)32 * (2 * k + 6) * sizeof(float); }
__host__ __device__ __forceinline__ size_t warp_bytes(int mode, bool stage, int k) {
    return warp_smem_bytes(mode) + (stage ? stage_bytes(k) : 0);
}

// Copies n words from shared memory to global (or host-mapped) memory with
// the whole warp: 16-byte vectors when both ends allow it, so each store
// instruction writes 512 contiguous bytes.
__device__ __forceinline__ void warp_copy_out(uint32_t* __restrict__ dst, const uint32_t* src, int n, int lane) {
    int done = 0;
    if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
        const int n4 = n >> 2;
        for (int i = lane; i < n4; i += 32)
            reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
        done = n4 << 2;
    }
    for (int i = done + lane; i < n; i += 32) dst[i] = src[i];
}

__device__ __forceinline__ void cas32(uint32_t& a, uint32_t& b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Batcher's odd-even merge sort over the first NN registers, ascending:
// merges sorted runs of length p into runs of 2p; within a merge, elements
// k apart are compared, k halving from p, and only pairs inside the same
// run of 2p.  The comparator list is computed at compile time and expanded
// as a parameter pack, so every register index is a constant (NN = 32: 191
// comparators, where a bitonic network takes 240).  For NN not a power of
// two the list is the next power of two's less every comparator that
// reaches past NN: with the registers from NN on holding the largest key,
// such a comparator never moves anything, so what remains sorts NN keys.
template <int NN>
struct OemNet {
    struct Table {
        int a[NN * NN], b[NN * NN];
        int n;
    };
    __host__ __device__ static constexpr Table make() {
        Table t{};
        t.n = 0;
        for (int p = 1; p < NN; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < NN; j += 2 * k)
                    for (int i = 0; i < k && i + j + k < NN; ++i)
                        if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                            t.a[t.n] = i + j;
                            t.b[t.n] = i + j + k;
                            ++t.n;
                        }
        return t;
    }
};

template <int NN, int CAP, int... Cs>
__device__ __forceinline__ void oem_apply(uint32_t (&K)[CAP], std::integer_sequence<int, Cs...>) {
    (cas32(K[std::integral_constant<int, OemNet<NN>::make().a[Cs]>::value],
           K[std::integral_constant<int, OemNet<NN>::make().b[Cs]>::value]),
     ...);
}

template <int NN, int CAP>
__device__ __forceinline__ void sort_regs(uint32_t (&K)[CAP]) {
    oem_apply<NN>(K, std::make_integer_sequence<int, OemNet<NN>::make().n>{});
}

// Trial radii of the lane path, as multiples of the starting radius: a
// geometric ladder from 0.75 to 1.46.  With 32 survivor slots (k <= 24) the
// ladder has eight steps of ratio 1.1, so the count at the chosen radius is
// at most ~1.2x the smallest count that reaches k on a surface and seldom
// overflows the slots; with 64 slots four steps of ratio ~1.22 leave room
// for the ~1.5x overshoot, and counting four radii instead of eight makes
// the first pass cheaper (k = 32: 0.148 -> 0.132 ms on the C2 scan).
template <int CAP>
struct Ladder {
    static constexpr int N = CAP == 32 ? 8 : 4;
    __device__ static __forceinline__ float mul(int j) {
        if (CAP == 32)
            return j == 0 ? 0.75f : j == 1 ? 0.83f : j == 2 ? 0.91f : j == 3 ? 1.0f
                 : j == 4 ? 1.1f : j == 5 ? 1.21f : j == 6 ? 1.33f : 1.46f;
        return j == 0 ? 0.8f : j == 1 ? 1.0f : j == 2 ? 1.22f : 1.46f;
    }
};

// (d2, index) key of the survivor in a lane's slot, recomputed from pts.
template <bool DEL>
__device__ __forceinline__ u64 slot_key(const Grid& g, const Grid& dg, const uint32_t* posl, int slot,
                                        int lane, float qx, float qy, float qz) {
    const uint32_t tp = posl[slot * 32 + lane];
    const float4 p = pt_at<DEL>(g, dg, tp);
    const float d = sqdist_pinned(qx, qy, qz, p.x, p.y, p.z);
    return ((u64)__float_as_uint(d) << 32) | (u64)union_index<DEL>(g, tp, p);
}

// A lane's own starting radius where the map's density is uneven: the
// points of the 27 cells around q (counted through the row index, no point
// is read) set a surface density n / (9 h^2), and the radius of a disc
// holding k points at that density, c h sqrt(k / n), is where the trial
// radii start; at most 3 h (and 3 h when the block is empty).  Only the
// search's speed depends on it.
template <bool WIN>
__device__ __forceinline__ float probe_radius(const Grid& g, float qx, float qy, float qz, int k, float c) {
    const int cx = cell_of(qx, g.ox, g.inv_h), cy = cell_of(qy, g.oy, g.inv_h), cz = cell_of(qz, g.oz, g.inv_h);
    const int x0 = max(cx - 1, WIN ? g.wlx : 0), x1 = min(cx + 1, WIN ? g.whx : g.dimx - 1);
    const int y0 = max(cy - 1, WIN ? g.wly : 0), y1 = min(cy + 1, WIN ? g.why : g.dimy - 1);
    const int z0 = max(cz - 1, WIN ? g.wlz : 0), z1 = min(cz + 1, WIN ? g.whz : g.dimz - 1);
    uint32_t n = 0;
    if (g.dstart && x0 <= x1)
        for (int z = z0; z <= z1; ++z)
            for (int y = y0; y <= y1; ++y) n += row_range(g, y, z, x0, x1).y;
    const float cap = 3.0f * g.h;
    return n > 0 ? fminf(c * g.h * sqrtf((float)k / (float)n), cap) : cap;
}

// k <= 32: one query per lane.  Pass 1 counts, for each trial radius
// r_j = m_j rho0, the target points with d2 <= t_j = min(r_j^2, tau), tau
// certified for the box around the largest radius; the smallest t_j that
// holds >= k points (and at most CAP) is exact by the same argument as the
// warp search: every point with d2 <= t_j lies in the box, so the k
// smallest of those are the k smallest overall.  Pass 2 collects their
// positions in the lane's shared-memory list.  They are ordered by a
// register odd-even merge sort network on 32-bit keys (d2 bits << 1, low five
// bits replaced by the slot), which orders d2 to within 16 ulps; any run of
// neighbours left in the same 16-ulp bucket is then put in exact (d2,
// index) order by bubble passes on the full keys.  Lanes whose query needs
// a wider radius, more than 32 survivors or a bigger box are finished by
// the warp-cooperative search, one query at a time.
//
// With DEL the search covers the union of the main grid g and the grid dg of
// appended points (point j of dg is g.m + j): both grids' boxes of the trial
// radius are counted and collected in the same passes, filtered by the
// smaller of their certified taus, and list entries from dg carry DTAG.
//
// With STG the outputs are page-locked host memory: each lane writes its
// idx/d2 row and covariance into the warp's staging area `stg` (laid out as
// the output arrays), and the warp copies each array's block of the tile out
// in 16-byte vectors, so host memory receives whole lines instead of the
// lanes' scattered 16-byte pieces.
template <int CAP, bool COV, bool WIN, bool DEL, bool STG>
__device__ void lane_tile(const Grid& g, const Grid& dg, const float* __restrict__ q, int64_t n0, int cnt,
                          const TileArgs& a, float rho0, int32_t* __restrict__ idx,
                          float* __restrict__ d2, float* __restrict__ cov, u64* pend,
                          uint32_t* posl, uint32_t* stg, int lane) {
    constexpr int NRAD = Ladder<CAP>::N;
    auto rad_mul = [](int jj) { return Ladder<CAP>::mul(jj); };
    const int k = a.k;
    const bool active = lane < cnt;
    const int64_t n = n0 + lane;
    // With STG the rows go to the warp's staging area (laid out as in the
    // output arrays) and are copied out as one block per tile.
    int32_t* const si = reinterpret_cast<int32_t*>(stg);
    float* const sd = reinterpret_cast<float*>(stg + 32 * k);
    float* const sc = reinterpret_cast<float*>(stg + 64 * k);
    float qx = 0.0f, qy = 0.0f, qz = 0.0f;
    if (active) {
        qx = __ldg(q + 3 * n);
        qy = __ldg(q + 3 * n + 1);
        qz = __ldg(q + 3 * n + 2);
    }
    const bool finite = active && isfinite(qx) && isfinite(qy) && isfinite(qz);
    bool fallback = false;
    int m = 0;
    float thr = -1.0f;
    uint32_t visits = 0;  // candidate points whose distance this lane computed
    int lx = 0, hx = -1, ly = 0, hy = -1, lz = 0, hz = -1;
    float eta = 0.0f;
    int dlx = 0, dhx = -1, dly = 0, dhy = -1, dlz = 0, dhz = -1;
    float deta = 0.0f;
    // Up to three lane-parallel attempts: a lane whose largest trial radius
    // held fewer than k points retries with the radii x1.8.  A lane whose
    // count jumped from below k at one radius to above CAP at the next (a
    // wall entering the ball between two rungs) retries with thresholds
    // spaced evenly in d2 between those two radii, where a surface's count
    // grows evenly; one whose smallest radius held more than CAP retries
    // with the radii x0.7.  Only lanes that still fail go to the warp
    // search, whose latency (tens of microseconds for one query) would
    // otherwise set the end of the launch.
    float rho = finite && a.probe_c > 0.0f ? probe_radius<WIN>(g, qx, qy, qz, a.k, a.probe_c) : rho0;
    float rlo2 = 0.0f, rhi2 = -1.0f;  // the interval to subdivide (squared radii), rhi2 > 0
    bool todo = finite;
    for (int attempt = 0; attempt < 3 && __any_sync(FULL, todo); ++attempt) {
        if (todo) {
            todo = false;
            const bool refine = rhi2 > 0.0f;
            const float rmax = refine ? sqrtf(rhi2) : rho * rad_mul(NRAD - 1);
            const int ulx = cell_of(__fsub_rn(qx, rmax), g.ox, g.inv_h);
            const int uhx = cell_of(__fadd_rn(qx, rmax), g.ox, g.inv_h);
            const int uly = cell_of(__fsub_rn(qy, rmax), g.oy, g.inv_h);
            const int uhy = cell_of(__fadd_rn(qy, rmax), g.oy, g.inv_h);
            const int ulz = cell_of(__fsub_rn(qz, rmax), g.oz, g.inv_h);
            const int uhz = cell_of(__fadd_rn(qz, rmax), g.oz, g.inv_h);
            float tau = certified_tau(g, qx, qy, qz, ulx, uhx, uly, uhy, ulz, uhz);
            const float qm = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
            {
                const int cm = max(max(max(abs(ulx), abs(uhx + 1)), max(abs(uly), abs(uhy + 1))),
                                   max(abs(ulz), abs(uhz + 1)));
                eta = 0x1p-20f * (g.coord_scale + qm + (float)cm * g.h);
            }
            lx = max(ulx, WIN ? g.wlx : 0); hx = min(uhx, WIN ? g.whx : g.dimx - 1);
            ly = max(uly, WIN ? g.wly : 0); hy = min(uhy, WIN ? g.why : g.dimy - 1);
            lz = max(ulz, WIN ? g.wlz : 0); hz = min(uhz, WIN ? g.whz : g.dimz - 1);
            const int64_t ncl = (int64_t)max(hx - lx + 1, 0) * max(hy - ly + 1, 0) * max(hz - lz + 1, 0);
            const int64_t nrows = (int64_t)max(hy - ly + 1, 0) * max(hz - lz + 1, 0);
            bool big = ncl > 4096 || nrows > 256 || (!g.dstart && ncl > 256);
            if (DEL) {
                const int vlx = cell_of(__fsub_rn(qx, rmax), dg.ox, dg.inv_h);
                const int vhx = cell_of(__fadd_rn(qx, rmax), dg.ox, dg.inv_h);
                const int vly = cell_of(__fsub_rn(qy, rmax), dg.oy, dg.inv_h);
                const int vhy = cell_of(__fadd_rn(qy, rmax), dg.oy, dg.inv_h);
                const int vlz = cell_of(__fsub_rn(qz, rmax), dg.oz, dg.inv_h);
                const int vhz = cell_of(__fadd_rn(qz, rmax), dg.oz, dg.inv_h);
                tau = fminf(tau, certified_tau(dg, qx, qy, qz, vlx, vhx, vly, vhy, vlz, vhz));
                const int cm = max(max(max(abs(vlx), abs(vhx + 1)), max(abs(vly), abs(vhy + 1))),
                                   max(abs(vlz), abs(vhz + 1)));
                deta = 0x1p-20f * (dg.coord_scale + qm + (float)cm * dg.h);
                dlx = max(vlx, WIN ? dg.wlx : 0); dhx = min(vhx, WIN ? dg.whx : dg.dimx - 1);
                dly = max(vly, WIN ? dg.wly : 0); dhy = min(vhy, WIN ? dg.why : dg.dimy - 1);
                dlz = max(vlz, WIN ? dg.wlz : 0); dhz = min(vhz, WIN ? dg.whz : dg.dimz - 1);
                const int64_t dncl =
                    (int64_t)max(dhx - dlx + 1, 0) * max(dhy - dly + 1, 0) * max(dhz - dlz + 1, 0);
                const int64_t dnrows = (int64_t)max(dhy - dly + 1, 0) * max(dhz - dlz + 1, 0);
                big = big || dncl > 4096 || dnrows > 256 || (!dg.dstart && dncl > 256);
            }
            fallback = false;
            if (tau < 0.0f || big) {
                fallback = true;
            } else {
                float t[NRAD];
                int c[NRAD];
#pragma unroll
                for (int j = 0; j < NRAD; ++j) {
                    const float r = rho * rad_mul(j);
                    const float tr = refine ? rlo2 + (rhi2 - rlo2) * ((float)(j + 1) / (float)NRAD) : r * r;
                    t[j] = fminf(tr, tau);
                    c[j] = 0;
                }
                auto count = [&](uint32_t, const float4 p) {
                    const float d = sqdist_pinned(qx, qy, qz, p.x, p.y, p.z);
                    ++visits;
#pragma unroll
                    for (int j = 0; j < NRAD; ++j) c[j] += d <= t[j] ? 1 : 0;
                };
                if (g.dstart) for_rows<WIN>(g, qx, qy, qz, lx, hx, ly, hy, lz, hz, eta, t[NRAD - 1], count);
                else for_box_points<WIN>(g, qx, qy, qz, lx, hx, ly, hy, lz, hz, eta, t[NRAD - 1], count);
                if (DEL) {
                    if (dg.dstart)
                        for_rows<WIN>(dg, qx, qy, qz, dlx, dhx, dly, dhy, dlz, dhz, deta, t[NRAD - 1], count);
                    else
                        for_box_points<WIN>(dg, qx, qy, qz, dlx, dhx, dly, dhy, dlz, dhz, deta, t[NRAD - 1],
                                            count);
                }
                int js = -1;
#pragma unroll
                for (int j = NRAD - 1; j >= 0; --j)
                    if (c[j] >= k) js = j;
                int cj = 0;
                float tj = -1.0f, tl = -1.0f;
#pragma unroll
                for (int j = 0; j < NRAD; ++j) {
                    if (j == js) { cj = c[j]; tj = t[j]; }
                    if (j + 1 == js) tl = t[j];
                }
                if (js < 0 || cj > CAP) {
                    fallback = true;
                    // too few within the certified radii: widen (a wider box also
                    // certifies further); too many: subdivide the jump or narrow
                    const bool widen = js < 0;
                    todo = true;
                    if (!widen && js > 0 && !refine) {
                        rlo2 = tl;
                        rhi2 = tj;
                    } else {
                        rho = widen ? rho * 1.8f : rho * 0.7f;
                        rhi2 = -1.0f;
                    }
                } else {
                    m = cj;
                    thr = tj;
                }
            }
        }
    }
    if (m > 0) {
        int w = 0;
        auto collect = [&](uint32_t pos, const float4 p) {
            const float d = sqdist_pinned(qx, qy, qz, p.x, p.y, p.z);
            ++visits;
            if (d <= thr && w < CAP) {
                posl[w * 32 + lane] = pos;
                ++w;
            }
        };
        if (g.dstart) for_rows<WIN>(g, qx, qy, qz, lx, hx, ly, hy, lz, hz, eta, thr, collect);
        else for_box_points<WIN>(g, qx, qy, qz, lx, hx, ly, hy, lz, hz, eta, thr, collect);
        if (DEL) {
            auto collect_d = [&](uint32_t pos, const float4 p) { collect(pos | DTAG, p); };
            if (dg.dstart) for_rows<WIN>(dg, qx, qy, qz, dlx, dhx, dly, dhy, dlz, dhz, deta, thr, collect_d);
            else for_box_points<WIN>(dg, qx, qy, qz, dlx, dhx, dly, dhy, dlz, dhz, deta, thr, collect_d);
        }
    }
    __syncwarp();
    uint32_t K[CAP];
#pragma unroll
    for (int s = 0; s < CAP; ++s) {
        uint32_t key = 0xffffffffu;
        if (s < m) {
            const float4 p = pt_at<DEL>(g, dg, posl[s * 32 + lane]);
            const float d = sqdist_pinned(qx, qy, qz, p.x, p.y, p.z);
            key = ((__float_as_uint(d) << 1) & ~(uint32_t)(CAP - 1)) | (uint32_t)s;
        }
        K[s] = key;
    }
    const unsigned mmax = __reduce_max_sync(FULL, (unsigned)m);
    if (mmax <= 16u) sort_regs<16>(K);
    else if (CAP == 32 || mmax <= 32u) sort_regs<32>(K);
    else sort_regs<CAP>(K);
    bool amb = false;
#pragma unroll
    for (int r = 0; r + 1 < CAP; ++r) amb |= (r + 1 < m) && ((K[r] ^ K[r + 1]) < (uint32_t)CAP);
    for (int pass = 0; amb && pass < CAP; ++pass) {
        bool swapped = false;
#pragma unroll
        for (int r = 0; r + 1 < CAP; ++r) {
            if (r + 1 < m && ((K[r] ^ K[r + 1]) < (uint32_t)CAP)) {
                const u64 ka = slot_key<DEL>(g, dg, posl, (int)(K[r] & (CAP - 1)), lane, qx, qy, qz);
                const u64 kb = slot_key<DEL>(g, dg, posl, (int)(K[r + 1] & (CAP - 1)), lane, qx, qy, qz);
                if (kb < ka) {
                    const uint32_t tmp = K[r];
                    K[r] = K[r + 1];
                    K[r + 1] = tmp;
                    swapped = true;
                }
            }
        }
        amb = swapped;
    }
    if (m > 0) {
        int32_t* const irow = STG ? si + lane * k : idx + n * k;
        float* const drow = STG ? sd + lane * k : d2 + n * k;
        // rank-ordered positions, rewritten in place into the list's first k slots
        uint32_t P[32];
#pragma unroll
        for (int r = 0; r < 32; ++r)
            if (r < k) P[r] = posl[(K[r] & (CAP - 1)) * 32 + lane];
        // Each lane writes its own row, so every store instruction touches
        // 32 rows; a row of 4j (2j) entries on a 16- (8-) byte aligned base is
        // whole vectors, which takes a quarter (half) of the instructions.
        const uintptr_t ab = STG ? reinterpret_cast<uintptr_t>(stg)
                                 : reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(d2);
        const int vw = ((k & 3) == 0 && (ab & 15) == 0) ? 4 : (((k & 1) == 0 && (ab & 7) == 0) ? 2 : 1);
        auto entry = [&](int r, int& iv, float& dv) {
            posl[r * 32 + lane] = P[r];
            const float4 p = pt_at<DEL>(g, dg, P[r]);
            iv = (int)union_index<DEL>(g, P[r], p);
            dv = sqdist_pinned(qx, qy, qz, p.x, p.y, p.z);
        };
        if (vw == 4) {
#pragma unroll
            for (int r = 0; r < 32; r += 4)
                if (r < k) {
                    int4 iv;
                    float4 dv;
                    entry(r, iv.x, dv.x);
                    entry(r + 1, iv.y, dv.y);
                    entry(r + 2, iv.z, dv.z);
                    entry(r + 3, iv.w, dv.w);
                    *reinterpret_cast<int4*>(irow + r) = iv;
                    *reinterpret_cast<float4*>(drow + r) = dv;
                }
        } else if (vw == 2) {
#pragma unroll
            for (int r = 0; r < 32; r += 2)
                if (r < k) {
                    int2 iv;
                    float2 dv;
                    entry(r, iv.x, dv.x);
                    entry(r + 1, iv.y, dv.y);
                    *reinterpret_cast<int2*>(irow + r) = iv;
                    *reinterpret_cast<float2*>(drow + r) = dv;
                }
        } else {
#pragma unroll
            for (int r = 0; r < 32; ++r)
                if (r < k) {
                    int iv;
                    float dv;
                    entry(r, iv, dv);
                    irow[r] = iv;
                    drow[r] = dv;
                }
        }
    } else if (active && !finite) {
        int32_t* const irow = STG ? si + lane * k : idx + n * k;
        float* const drow = STG ? sd + lane * k : d2 + n * k;
        for (int r = 0; r < k; ++r) {
            irow[r] = -1;
            drow[r] = INFINITY;
        }
        atomicOr(g.status, ST_NONFINITE);
    }
    unsigned fb = __ballot_sync(FULL, fallback);
    const unsigned nvis = __reduce_add_sync(FULL, visits);
    if (lane == 0) {
        atomicAdd(&g.stats[0], (unsigned long long)cnt);
        if (fb) atomicAdd(&g.stats[1], (unsigned long long)__popc(fb));
        if (nvis) atomicAdd(&g.stats[3], (unsigned long long)nvis);
    }
    while (fb) {
        const int f = __ffs(fb) - 1;
        fb &= fb - 1u;
        const float fx = __shfl_sync(FULL, qx, f), fy = __shfl_sync(FULL, qy, f),
                    fz = __shfl_sync(FULL, qz, f);
        float rho = rho0 * rad_mul(NRAD - 1);
        SearchState<1> S;
        state_reset(S);
        const int sr = knn_search<1, DEL>(g, dg, fx, fy, fz, k, rho, S, pend, lane);
        const bool ok = sr == SEARCH_OK;
        if (!ok && lane == 0) atomicOr(g.status, sr == SEARCH_SHORT ? ST_SHORT : ST_SEARCH_LIMIT);
        const int64_t nf = n0 + f;
        if (lane < k) {
            int32_t* const fi = STG ? si + f * k : idx + nf * k;
            float* const fd = STG ? sd + f * k : d2 + nf * k;
            fi[lane] = ok ? (int32_t)(uint32_t)S.L[0] : -1;
            fd[lane] = ok ? __uint_as_float((uint32_t)(S.L[0] >> 32)) : INFINITY;
        }
    }
    if (STG) {
        __syncwarp();  // the staged rows of every lane, then one block per array
        warp_copy_out(reinterpret_cast<uint32_t*>(idx + n0 * k), stg, cnt * k, lane);
        warp_copy_out(reinterpret_cast<uint32_t*>(d2 + n0 * k), stg + 32 * k, cnt * k, lane);
    }
    if (COV && cov != nullptr) {
        __syncwarp();  // orders the idx rows written by other lanes
        float* const crow = STG ? sc + 6 * lane : cov + 6 * n;
        if (m > 0) {  // neighbours straight from the cell-sorted copy, in rank order
            auto get = [&](int j) { return pt_at<DEL>(g, dg, posl[j * 32 + lane]); };
            if (a.ck.type != 0) weighted_core(get, a.ck, qx, qy, qz, k, a.eps, crow);
            else cov_core(get, k, a.eps, crow);
        } else if (active) {
            cov_row_any<DEL>(g, dg, STG ? si + lane * k : idx + n * k, k, a, qx, qy, qz, crow);
        }
        if (STG) {
            __syncwarp();
            warp_copy_out(reinterpret_cast<uint32_t*>(cov + 6 * n0), stg + 64 * k, cnt * 6, lane);
        }
    }
    __syncwarp();
}

// k > 32: the warp-cooperative search for each query of the tile in turn.
template <bool COV, bool DEL>
__device__ void warp_tile(const Grid& g, const Grid& dg, const float* __restrict__ q, int64_t n0, int cnt,
                          const TileArgs& a, float rho0, int32_t* __restrict__ idx,
                          float* __restrict__ d2, float* __restrict__ cov, u64* pend,
                          int lane) {
    const int k = a.k;
    float rho = rho0;
    if (lane == 0) {
        atomicAdd(&g.stats[0], (unsigned long long)cnt);
        atomicAdd(&g.stats[1], (unsigned long long)cnt);
    }
    for (int i = 0; i < cnt; ++i) {
        const int64_t n = n0 + i;
        const float qx = __ldg(q + 3 * n), qy = __ldg(q + 3 * n + 1), qz = __ldg(q + 3 * n + 2);
        const bool finite = isfinite(qx) && isfinite(qy) && isfinite(qz);
        SearchState<2> S;
        state_reset(S);
        int sr = SEARCH_LIMIT;
        if (finite) sr = knn_search<2, DEL>(g, dg, qx, qy, qz, k, rho, S, pend, lane);
        const bool ok = finite && sr == SEARCH_OK;
        if (!ok && lane == 0)
            atomicOr(g.status, !finite ? ST_NONFINITE : sr == SEARCH_SHORT ? ST_SHORT : ST_SEARCH_LIMIT);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int r = s * 32 + lane;
            if (r < k) {
                const u64 key = S.L[s];
                const int32_t oi = ok ? (int32_t)(uint32_t)key : -1;
                idx[n * k + r] = oi;
                d2[n * k + r] = ok ? __uint_as_float((uint32_t)(key >> 32)) : INFINITY;
            }
        }
        if (ok) {
            const float dk = __uint_as_float((uint32_t)(S.kth >> 32));
            rho = fminf(fmaxf(sqrtf(dk) * 1.15f, 1e-2f * g.h), 1e30f);
        }
    }
    if (COV && cov != nullptr) {
        __syncwarp();
        if (lane < cnt) {
            const int64_t nl = n0 + lane;
            cov_row_any<DEL>(g, dg, idx + nl * k, k, a, __ldg(q + 3 * nl), __ldg(q + 3 * nl + 1),
                             __ldg(q + 3 * nl + 2), cov + 6 * nl);
        }
        __syncwarp();
    }
}

template <int MODE, bool COV, bool WIN, bool DEL = false, bool STG = false>
__device__ __forceinline__ void process_tile(const Grid& g, const Grid& dg, const float* __restrict__ q, int64_t n0,
                                             int cnt, const TileArgs& a, float rho0,
                                             int32_t* __restrict__ idx, float* __restrict__ d2,
                                             float* __restrict__ cov, unsigned char* wsmem,
                                             int lane) {
    u64* pend = reinterpret_cast<u64*>(wsmem);
    uint32_t* posl = reinterpret_cast<uint32_t*>(wsmem + 64 * sizeof(u64));
    uint32_t* stg = STG ? reinterpret_cast<uint32_t*>(wsmem + warp_smem_bytes(MODE)) : nullptr;
    if (MODE == 0)
        lane_tile<32, COV, WIN, DEL, STG>(g, dg, q, n0, cnt, a, rho0, idx, d2, cov, pend, posl, stg, lane);
    else if (MODE == 1)
        lane_tile<64, COV, WIN, DEL, STG>(g, dg, q, n0, cnt, a, rho0, idx, d2, cov, pend, posl, stg, lane);
    else
        warp_tile<COV, DEL>(g, dg, q, n0, cnt, a, rho0, idx, d2, cov, pend, lane);
}

template <int MODE, bool COV, bool WIN, bool STG = false>
__global__ void __launch_bounds__(256, 2) k_knn(Grid g, const float* __restrict__ q, int64_t N,
                                             int tile, TileArgs a, float rho0,
                                             int32_t* __restrict__ idx, float* __restrict__ d2,
                                             float* __restrict__ cov) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    // Tiles are issued last-first.  A spinning LiDAR scan stored ring by ring
    // with rising elevation ends with its farthest, sparsest points, whose
    // tiles cost the most; starting them first lets the cheap near-range
    // tiles fill the end of the launch.  (The order never changes a result.)
    const int64_t tiles = (N + tile - 1) / tile;
    const int64_t w = (int64_t)blockIdx.x * nwarps + warp;
    if (w >= tiles) return;
    const int64_t t = a.last_first ? tiles - 1 - w : w;
    const int64_t n0 = t * tile;
    const int cnt = (int)min((int64_t)tile, N - n0);
    process_tile<MODE, COV, WIN, false, STG>(g, g, q, n0, cnt, a, rho0, idx, d2, cov,
                                             smem + (size_t)warp * warp_bytes(MODE, STG, a.k), lane);
}

// Batched form: one warp per (scan, tile) item of the scans' prefix-summed
// tile table, found by a binary search over the table, items issued
// last-first as in k_knn (the last scan's farthest tiles start first).  A
// plain grid rather than a persistent loop over a device work counter: the
// hardware block scheduler balances the load as well, and without the loop
// state the kernel keeps k_knn's registers (a persistent version spilled at
// the 128-register cap and ran 23 % slower than one launch over the same
// queries concatenated).
// At most 96 registers in the lane path with up to 32 survivors, which it
// fits without spilling (left free, the compiler takes 111); the 64-survivor
// and warp paths keep up to 128.
template <int MODE, bool COV, bool WIN, bool STG = false>
__global__ void __maxnreg__(MODE == 0 ? 96 : 128) k_knn_batch(Grid g, const ScanDesc* __restrict__ scans,
                                                   int nscans, int64_t total_tiles, int tile,
                                                   TileArgs a, float rho0) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * nwarps + warp;
    if (w >= total_tiles) return;
    const int64_t item = a.last_first ? total_tiles - 1 - w : w;
    int lo = 0, hi = nscans - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (scans[mid].tile0 <= item) lo = mid; else hi = mid - 1;
    }
    const ScanDesc sd = scans[lo];
    const int64_t n0 = (item - sd.tile0) * tile;
    const int cnt = (int)min((int64_t)tile, sd.n - n0);
    process_tile<MODE, COV, WIN, false, STG>(g, g, sd.q, n0, cnt, a, rho0, sd.idx, sd.d2, sd.cov,
                                             smem + (size_t)warp * warp_bytes(MODE, STG, a.k), lane);
}

// Search over a map grown by appended points: the main grid g and the
// appended-points grid dg as one map (indices of dg's points follow g's).
// Same tiling and tile order as k_knn.
template <int MODE, bool COV, bool WIN>
__global__ void __launch_bounds__(256, 2) k_knn_union(Grid g, Grid dg, const float* __restrict__ q, int64_t N,
                                                   int tile, TileArgs a, float rho0,
                                                   int32_t* __restrict__ idx, float* __restrict__ d2,
                                                   float* __restrict__ cov) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int64_t tiles = (N + tile - 1) / tile;
    const int64_t w = (int64_t)blockIdx.x * nwarps + warp;
    if (w >= tiles) return;
    const int64_t t = a.last_first ? tiles - 1 - w : w;
    const int64_t n0 = t * tile;
    const int cnt = (int)min((int64_t)tile, N - n0);
    process_tile<MODE, COV, WIN, true>(g, dg, q, n0, cnt, a, rho0, idx, d2, cov,
                                       smem + (size_t)warp * warp_smem_bytes(MODE), lane);
}

__global__ void k_cov(Grid g, const int32_t* __restrict__ idx, int64_t N, int k, float eps,
                      float* __restrict__ cov) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    cov_row(g, idx + n * k, 1, k, eps, cov + 6 * n, true);
}

template <typename K>
cudaError_t allow_smem(K kern) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// The search kernel for (mode, covariance, batched) of this window variant.
template <bool WIN>
void* knn_kernel(int mode, bool with_cov, bool batch, bool stage = false) {
    // outputs in host memory: the staged lane-path kernels
    if (stage && mode < 2) {
        if (batch && with_cov)
            return mode == 0 ? (void*)k_knn_batch<0, true, WIN, true> : (void*)k_knn_batch<1, true, WIN, true>;
        if (batch)
            return mode == 0 ? (void*)k_knn_batch<0, false, WIN, true> : (void*)k_knn_batch<1, false, WIN, true>;
        if (with_cov) return mode == 0 ? (void*)k_knn<0, true, WIN, true> : (void*)k_knn<1, true, WIN, true>;
    }
#define PC_PICK(M, C) (batch ? (void*)k_knn_batch<M, C, WIN> : (void*)k_knn<M, C, WIN>)
    switch (mode * 2 + (with_cov ? 1 : 0)) {
        case 0: return PC_PICK(0, false);
        case 1: return PC_PICK(0, true);
        case 2: return PC_PICK(1, false);
        case 3: return PC_PICK(1, true);
        case 4: return PC_PICK(2, false);
        default: return PC_PICK(2, true);
    }
#undef PC_PICK
}

// The union search kernel for (mode, covariance) of this window variant.
template <bool WIN>
void* knn_union_kernel(int mode, bool with_cov) {
    switch (mode * 2 + (with_cov ? 1 : 0)) {
        case 0: return (void*)k_knn_union<0, false, WIN>;
        case 1: return (void*)k_knn_union<0, true, WIN>;
        case 2: return (void*)k_knn_union<1, false, WIN>;
        case 3: return (void*)k_knn_union<1, true, WIN>;
        case 4: return (void*)k_knn_union<2, false, WIN>;
        default: return (void*)k_knn_union<2, true, WIN>;
    }
}

template <bool WIN>
cudaError_t allow_union_smem() {
    cudaError_t e = cudaSuccess;
    for (int mode = 0; mode < 3; ++mode)
        for (int c = 0; c < 2; ++c)
            if ((e = allow_smem(knn_union_kernel<WIN>(mode, c != 0))) != cudaSuccess) return e;
    return cudaSuccess;
}

// Opts every search kernel of this window variant into large dynamic
// shared memory.
template <bool WIN>
cudaError_t allow_all_smem() {
    cudaError_t e = cudaSuccess;
    for (int mode = 0; mode < 3; ++mode)
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                if ((e = allow_smem(knn_kernel<WIN>(mode, c != 0, b != 0))) != cudaSuccess) return e;
    for (int mode = 0; mode < 2; ++mode)
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                if ((e = allow_smem(knn_kernel<WIN>(mode, c != 0, b != 0, true))) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace

