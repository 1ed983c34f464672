// Box searches over the voxel-hash grid shared by the kNN kernels and the
// GICP linearisation: the certified radius of a cell box, and visits of the
// points in a box (row by row through the row index, or cell by cell
// through the hash).
#pragma once

#include "pc_device.cuh"

namespace pcdev {

// A point outside the window is handed to the visitor with x = +inf, so its
// d2 is +inf and every threshold rejects it (a select, not a branch inside
// the visit loop: a skip there doubled the loop's time).  The visits call it
// only on rows and cells of the window's boundary; WIN = false compiles to
// nothing.
template <bool WIN>
__device__ __forceinline__ float4 window_cut(const Grid& g, bool test, float4 p) {
    if (WIN && test && !in_window(g, p)) p.x = INFINITY;
    return p;
}

// Distance from q to the nearer face of the cell slab [lo, hi] on one axis.
__device__ __forceinline__ float slab_gap(float q, float o, int lo, int hi, float h) {
    const float flo = o + (float)lo * h;
    const float fhi = o + (float)(hi + 1) * h;
    return fminf(q - flo, fhi - q);
}

// tau such that EVERY target point outside the cell box [l, h] has a binary32
// d2 strictly greater than tau (or -1 if nothing can be certified).
//
// A point in a cell c' < l on some axis has fl(fl(p-o)*inv_h) < l, so
// p < o + l*h*(1 + 3.01u) with u = 2^-24; symmetrically for c' > h.  The
// face positions and the gap are computed with a few more roundings.  All
// together the true distance to any outside point is at least
// gap - 8u*(|o| + |q| + |c|*h), where the margin eta below is twice that.
// The binary32 d2 of a point at true distance D is >= D^2 (1 - 5u), so
// tau = Rs^2 (1 - 2^-20) with Rs = gap - eta is strictly below it.  For
// Rs < 2^-60 nothing is certified (products could be subnormal).
__device__ __forceinline__ float certified_tau(const Grid& g, float qx, float qy, float qz, int lx,
                                               int hx, int ly, int hy, int lz, int hz) {
    float R = fminf(slab_gap(qx, g.ox, lx, hx, g.h),
                    fminf(slab_gap(qy, g.oy, ly, hy, g.h), slab_gap(qz, g.oz, lz, hz, g.h)));
    int cm = max(max(max(abs(lx), abs(hx + 1)), max(abs(ly), abs(hy + 1))),
                 max(abs(lz), abs(hz + 1)));
    float qm = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
    float eta = 0x1p-20f * (g.coord_scale + qm + (float)cm * g.h);
    float Rs = R - eta;
    if (!(Rs > 0x1p-60f)) return -1.0f;
    return (Rs * Rs) * (1.0f - 0x1p-20f);
}

// Visit every point of the cell box [l, h] (clamped to the grid) whose
// cell can hold a point within sqrt(tmax) of q, as f(position, point).
// Rows along x are pruned by a conservative lower bound (the eta margin of
// certified_tau); each surviving cell is a hash lookup.
template <bool WIN = true, typename F>
__device__ __forceinline__ void for_box_points(const Grid& g, float qx, float qy, float qz, int lx,
                                               int hx, int ly, int hy, int lz, int hz, float eta,
                                               float tmax, F&& f) {
    for (int cz = lz; cz <= hz; ++cz) {
        const bool wz = WIN && g.windowed && (cz == g.tlz || cz == g.thz);
        const float zl = g.oz + (float)cz * g.h, zh = g.oz + (float)(cz + 1) * g.h;
        const float gz = fmaxf(fmaxf(zl - qz, qz - zh), 0.0f) - eta;
        const float gz2 = gz > 0.0f ? gz * gz : 0.0f;
        for (int cy = ly; cy <= hy; ++cy) {
            const float yl = g.oy + (float)cy * g.h, yh = g.oy + (float)(cy + 1) * g.h;
            const float gy = fmaxf(fmaxf(yl - qy, qy - yh), 0.0f) - eta;
            const float gyz2 = gz2 + (gy > 0.0f ? gy * gy : 0.0f);
            if (gyz2 * (1.0f - 0x1p-20f) > tmax) continue;
            const bool wyz = wz || (WIN && g.windowed && (cy == g.tly || cy == g.thy));
            for (int cx = lx; cx <= hx; ++cx) {
                const float xl = g.ox + (float)cx * g.h, xh = g.ox + (float)(cx + 1) * g.h;
                const float gx = fmaxf(fmaxf(xl - qx, qx - xh), 0.0f) - eta;
                const float lb2 = gyz2 + (gx > 0.0f ? gx * gx : 0.0f);
                if (lb2 * (1.0f - 0x1p-20f) > tmax) continue;
                const bool test = wyz || (WIN && g.windowed && (cx == g.tlx || cx == g.thx));
                const uint2 r = lookup_cell(g, pack_key(cx, cy, cz, g.bx, g.by));
                if (WIN && test) {
                    for (uint32_t i = 0; i < r.y; ++i) f(r.x + i, window_cut<WIN>(g, true, __ldg(&g.pts[r.x + i])));
                } else {
                    for (uint32_t i = 0; i < r.y; ++i) f(r.x + i, __ldg(&g.pts[r.x + i]));
                }
            }
        }
    }
}

// The part of row (cy, cz) that can hold a point within sqrt(tmax) of q, as
// a range of pts through the row index: the row is skipped when the lower
// bound of dy^2 + dz^2 exceeds tmax, else narrowed along x to half-width
// sqrt(tmax (1 + 2^-18) - that bound) widened by eta (the cell rule's
// rounding).  A point outside the range has a binary32 d2 above tmax.
__device__ __forceinline__ uint2 row_part(const Grid& g, float qx, float qy, float qz, int cy,
                                          int cz, int lx, int hx, float eta, float tmax, float tx) {
    const float zl = g.oz + (float)cz * g.h, zh = g.oz + (float)(cz + 1) * g.h;
    const float gz = fmaxf(fmaxf(zl - qz, qz - zh), 0.0f) - eta;
    const float yl = g.oy + (float)cy * g.h, yh = g.oy + (float)(cy + 1) * g.h;
    const float gy = fmaxf(fmaxf(yl - qy, qy - yh), 0.0f) - eta;
    const float gyz2 = (gz > 0.0f ? gz * gz : 0.0f) + (gy > 0.0f ? gy * gy : 0.0f);
    if (gyz2 * (1.0f - 0x1p-20f) > tmax) return make_uint2(0u, 0u);
    const float xw = sqrtf(fmaxf(tx - gyz2, 0.0f)) + eta;
    const float ul = cell_coord(__fsub_rn(qx, xw), g.ox, g.inv_h);
    const float uh = cell_coord(__fadd_rn(qx, xw), g.ox, g.inv_h);
    const int c0 = cell_of(__fsub_rn(qx, xw), g.ox, g.inv_h);
    const int c1 = cell_of(__fadd_rn(qx, xw), g.ox, g.inv_h);
    const int x0 = max(lx, c0);
    const int x1 = min(hx, c1);
    if (x0 > x1) return make_uint2(0u, 0u);
    if (!g.xcut) return row_range(g, cy, cz, x0, x1);
    // Inside the end cells, sub-bins wholly beyond qx -+ xw: their points
    // have u(p) < u(qx - xw) (or > u(qx + xw)), so p lies beyond the same
    // bound that excludes the cells before x0 and after x1.
    return row_range_cut(g, cy, cz, x0, x1, x0 == c0 ? sub_bin(ul) : 0, x1 == c1 ? sub_bin(uh) : 7);
}

// Same visit as for_box_points through the row index: every row of the box
// is one contiguous range of pts.  Rows are resolved two at a time so their
// index loads overlap.  An empty box (a query beyond the grid or the window
// on some axis) visits nothing: the row walk below assumes ly <= hy, and a
// row index outside [0, dimy) would address the wrong row of the bitmap.
template <bool WIN = true, typename F>
__device__ __forceinline__ void for_rows(const Grid& g, float qx, float qy, float qz, int lx, int hx,
                                         int ly, int hy, int lz, int hz, float eta, float tmax,
                                         F&& f) {
    if (lx > hx || ly > hy) return;
    const float tx = tmax * (1.0f + 0x1p-18f);
    // the window's boundary cells along x are in every row of the box
    const bool wx = WIN && g.windowed && (lx == g.tlx || hx == g.thx);
    int cy = ly, cz = lz;
    while (cz <= hz) {
        const int cy2 = cy < hy ? cy + 1 : ly;
        const int cz2 = cy < hy ? cz : cz + 1;
        const uint2 ra = row_part(g, qx, qy, qz, cy, cz, lx, hx, eta, tmax, tx);
        const uint2 rb = cz2 <= hz ? row_part(g, qx, qy, qz, cy2, cz2, lx, hx, eta, tmax, tx)
                                   : make_uint2(0u, 0u);
        // a row on a boundary cell of the window tests its points (never in
        // the whole-map variant, WIN = false)
        const bool ta = WIN && (wx || cy == g.tly || cy == g.thy || cz == g.tlz || cz == g.thz);
        const bool tb = WIN && (wx || cy2 == g.tly || cy2 == g.thy || cz2 == g.tlz || cz2 == g.thz);
        // The window test runs only on the rows that need it: the choice of
        // loop is made once per row, so untested rows run the plain loop (a
        // select inside one shared loop cost ~25 % of the window search).
        if (WIN && ta) {
            for (uint32_t i = 0; i < ra.y; ++i) f(ra.x + i, window_cut<WIN>(g, true, __ldg(&g.pts[ra.x + i])));
        } else {
            for (uint32_t i = 0; i < ra.y; ++i) f(ra.x + i, __ldg(&g.pts[ra.x + i]));
        }
        if (WIN && tb) {
            for (uint32_t i = 0; i < rb.y; ++i) f(rb.x + i, window_cut<WIN>(g, true, __ldg(&g.pts[rb.x + i])));
        } else {
            for (uint32_t i = 0; i < rb.y; ++i) f(rb.x + i, __ldg(&g.pts[rb.x + i]));
        }
        cy = cy2 < hy ? cy2 + 1 : ly;
        cz = cy2 < hy ? cz2 : cz2 + 1;
    }
}

}  // namespace pcdev
