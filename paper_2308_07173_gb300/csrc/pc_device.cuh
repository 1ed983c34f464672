// Device-side definitions shared by the grid build and the search kernels:
// the voxel-hash grid layout, the cell-coordinate rule and the hash probe.
//
// The grid is the "GPU-hash data structure" over the target of Sec. III-C3:
// every target point p lands in the cell
//     c_a = floor( fl( fl(p_a - o_a) * inv_h ) ),  a in {x, y, z}
// (o = bounding-box minimum, inv_h = fl(1/h)); queries use the same rule, so
// the rounding error of the rule is the same on both sides and the search
// can bound it (see certified_radius2 in knn_cov.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pcdev {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long EMPTY_KEY = ~0ull;

// status-word bits (one int per target handle)
constexpr int ST_NONFINITE = 1;
constexpr int ST_SEARCH_LIMIT = 2;
constexpr int ST_BAD_INDEX = 4;
constexpr int ST_SHORT = 8;  // fewer than k target points in the window

// Read-only view of a built target, passed by value to every search kernel.
struct Grid {
    float ox, oy, oz;       // origin = bbox minimum
    float h, inv_h;         // cell edge and fl(1/h)
    int dimx, dimy, dimz;   // occupied range of cell coordinates is [0, dim)
    int bx, by;             // key = cx | cy << bx | cz << (bx + by)
    int log2cap;            // hash capacity = 1 << log2cap
    int max_box_cells;
    int exhaustive;
    float coord_scale;      // max |coordinate| over origin and bbox corners
    int64_t m;              // target points
    int64_t ncells;         // occupied cells
    const uint4* table;     // slot = {key lo, key hi, start, count}
    const float4* pts;      // cell-sorted: (x, y, z, bits of the original index)
    const float4* xyz;      // caller order: (x, y, z, 0)
    const unsigned long long* cell_keys;  // occupied cell keys, ascending [ncells]
    const uint32_t* cell_start;           // [ncells + 1] into pts
    // Row index (null when the grid is too large for it): dstart[L] is the
    // position in pts of the first point of the occupied cells with linear
    // index >= L, L = cx + dimx (cy + dimy cz) in [0, dimx dimy dimz].
    // Occupied cells are ordered by L, so a run of cells along x is one
    // contiguous range of pts, read with one pair of loads.
    const uint32_t* dstart;
    // Sub-cell cut of the row index (null when not built): points inside a
    // cell are ordered by their eighth of the cell along x (the sub-bin, see
    // sub_bin), and xcut[L] packs, for b = 1..8, the number of the cell's
    // points in sub-bins below b into byte b - 1 (byte 7 = the cell's count).
    // A cell of 255 points or more has the all-zero word: no cut.
    const uint2* xcut;
    int* status;
    unsigned long long* stats;  // [0] queries, [1] warp-search fallbacks, [2] exhaustive scans,
                                // [3] lane-path candidate points
    // Search window (pc_set_window): only target points p with
    // wlo <= p <= whi (componentwise) are searched.  [wl, wh] is the range of
    // cells that can hold them (the whole grid when windowed == 0); a point
    // in a cell strictly inside that range is inside the box (the cell rule
    // is monotone), so only the range's boundary cells can hold points
    // outside it -- and only where the bound lies inside the target's
    // bounding box.  tl/th are those cells (-1 where no point can be cut).
    int windowed;
    int wlx, whx, wly, why, wlz, whz;
    int tlx, thx, tly, thy, tlz, thz;
    float wlox, wloy, wloz, whix, whiy, whiz;
};

__device__ __forceinline__ bool in_window(const Grid& g, float4 p) {
    return p.x >= g.wlox && p.x <= g.whix && p.y >= g.wloy && p.y <= g.whiy && p.z >= g.wloz &&
           p.z <= g.whiz;
}

// The cell coordinate before rounding down: fl(fl(v - o) * inv_h).  It is
// monotone in v, so u(p) < u(v) implies p < v.
__device__ __forceinline__ float cell_coord(float v, float o, float inv_h) {
    return __fmul_rn(__fsub_rn(v, o), inv_h);
}

__device__ __forceinline__ int cell_of(float v, float o, float inv_h) {
    float t = cell_coord(v, o, inv_h);
    t = floorf(t);
    t = fminf(fmaxf(t, -1073741824.0f), 1073741824.0f);
    return (int)t;
}

// The eighth of its cell a cell coordinate u falls in: floor(8 (u - floor u)),
// 0..7 (u - floor u and the product by 8 are exact).
__device__ __forceinline__ int sub_bin(float u) {
    return (int)floorf(__fmul_rn(__fsub_rn(u, floorf(u)), 8.0f));
}

__device__ __forceinline__ unsigned long long pack_key(int cx, int cy, int cz, int bx, int by) {
    return (unsigned long long)(unsigned)cx | ((unsigned long long)(unsigned)cy << bx) |
           ((unsigned long long)(unsigned)cz << (bx + by));
}

__device__ __forceinline__ uint32_t hash_slot(unsigned long long key, int log2cap) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - log2cap));
}

// (start, count) of an occupied cell, (0, 0) for an empty one.  Linear
// probing; the table always has empty slots (load <= 0.9), and the probe
// count is capped at the capacity anyway.
__device__ __forceinline__ uint2 lookup_cell(const Grid& g, unsigned long long key) {
    const uint32_t mask = (1u << g.log2cap) - 1u;
    uint32_t slot = hash_slot(key, g.log2cap);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint4 e = __ldg(&g.table[slot]);
        unsigned long long k = (unsigned long long)e.x | ((unsigned long long)e.y << 32);
        if (k == key) return make_uint2(e.z, e.w);
        if (k == EMPTY_KEY) break;
        slot = (slot + 1u) & mask;
    }
    return make_uint2(0u, 0u);
}

// Points of the occupied cells x0..x1 (x0 <= x1) of row (cy, cz) as one
// range (start, count) of pts, through the row index.
__device__ __forceinline__ uint2 row_range(const Grid& g, int cy, int cz, int x0, int x1) {
    const int64_t base = (int64_t)g.dimx * ((int64_t)cy + (int64_t)g.dimy * cz);
    const uint32_t s = __ldg(&g.dstart[base + x0]);
    return make_uint2(s, __ldg(&g.dstart[base + x1 + 1]) - s);
}

// Byte b - 1 of a sub-cell cut word: the cell's points in sub-bins below b.
__device__ __forceinline__ uint32_t cut_below(uint2 w, int b) {
    const unsigned long long v = ((unsigned long long)w.y << 32) | w.x;
    return (uint32_t)(v >> (8 * (b - 1))) & 255u;
}

// row_range without the points of cell x0 in sub-bins below b0 and those of
// cell x1 in sub-bins above b1 (b0 = 0 and b1 = 7 cut nothing), through the
// sub-cell cut; the loads of both tables are independent.
__device__ __forceinline__ uint2 row_range_cut(const Grid& g, int cy, int cz, int x0, int x1, int b0, int b1) {
    const int64_t base = (int64_t)g.dimx * ((int64_t)cy + (int64_t)g.dimy * cz);
    const uint32_t s = __ldg(&g.dstart[base + x0]);
    const uint32_t e = __ldg(&g.dstart[base + x1 + 1]);
    const uint2 w0 = __ldg(&g.xcut[base + x0]);
    const uint2 w1 = __ldg(&g.xcut[base + x1]);
    const uint32_t skip = b0 > 0 ? cut_below(w0, b0) : 0u;
    const uint32_t drop = cut_below(w1, 8) - cut_below(w1, b1 + 1);
    const uint32_t n = e - s;  // >= skip + drop by construction; clamped all the same
    return skip + drop <= n ? make_uint2(s + skip, n - skip - drop) : make_uint2(s, n);
}

// The pinned binary32 squared distance: fmaf(dz,dz, fmaf(dy,dy, dx*dx)).
__device__ __forceinline__ float sqdist_pinned(float qx, float qy, float qz, float px, float py,
                                               float pz) {
    float dx = __fsub_rn(qx, px);
    float dy = __fsub_rn(qy, py);
    float dz = __fsub_rn(qz, pz);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

}  // namespace pcdev
