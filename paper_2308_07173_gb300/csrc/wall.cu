// Wall detection for resilient navigation (Sec. III-D, Eq. 24-30): a
// voxel filter, ground removal by 2-D hash voting, Euclidean clustering of
// the vertical voxels, the wall as the longest right-side cluster and its
// quadratic fit -- all on the device, on buffers sized once when the
// detector is created.
//
//  1. voxel key of every point (binary32 floor(p * fl(1/v)) per axis, fields
//     offset into [0, 2^b - 2]; dropped points get the all-ones key), stable
//     LSD radix sort of (key, index), run starts by a flag scan; each voxel's
//     centroid is summed in binary64 in index order, divided by the count and
//     rounded to binary32;
//  2. each voxel votes for the 2-D cell of its centroid in an open-addressing
//     hash (integer counts, so the result is order-free); a voxel is
//     vertical when its cell holds more than min_votes voxels;
//  3. vertical voxels are linked when their pinned binary32 d2 <= fl(tol^2):
//     a hash of cells of edge tol (1 + 2^-10) keeps per-cell linked lists, and
//     a lock-free union-find (every voxel first under its smallest linked
//     neighbour, a dozen rounds of pointer jumping, then unions that hook the
//     larger root under the smaller, with path halving) gives every
//     component its smallest voxel index as label;
//  4. per cluster: count and the extremes of x and y (ordered-integer
//     atomics); the wall is the cluster of >= min_cluster voxels with
//     fl(min y + max y) < 0 and the largest fl(max x - min x), ties to the
//     smaller label;
//  5. y = b0 + b1 x + b2 x^2 by least squares over the wall's centroids: the
//     sums of the normal equations in binary64 over a fixed grid in a fixed
//     order (block partials added by the last block), solved by Gaussian
//     elimination with partial pivoting; d_w = b0.
// Every bounded loop (probes, list walks, root chases) carries an iteration
// cap; running out sets an error bit in the result instead of spinning.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "pc_internal.h"

namespace {

typedef unsigned long long u64;
constexpr u64 INVALID_KEY = ~0ull;
constexpr int WALL_ERR_LIMIT = 1;

__device__ __forceinline__ unsigned f2ord(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ uint32_t hslot(u64 key, int log2cap) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - log2cap));
}

// Insert-or-find in an open-addressing table of keys; returns the slot or
// -1 when the table is full (cannot happen: capacity >= 2 x entries).
__device__ int hash_insert(u64* keys, int log2cap, u64 key) {
    const uint32_t mask = (1u << log2cap) - 1u;
    uint32_t s = hslot(key, log2cap);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const u64 prev = atomicCAS(&keys[s], INVALID_KEY, key);
        if (prev == INVALID_KEY || prev == key) return (int)s;
        s = (s + 1u) & mask;
    }
    return -1;
}

__device__ int hash_find(const u64* keys, int log2cap, u64 key) {
    const uint32_t mask = (1u << log2cap) - 1u;
    uint32_t s = hslot(key, log2cap);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const u64 k = keys[s];
        if (k == key) return (int)s;
        if (k == INVALID_KEY) return -1;
        s = (s + 1u) & mask;
    }
    return -1;
}

__device__ __forceinline__ float sqdist3(float4 a, float4 b) {
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

struct WallParams {
    float inv_v, inv_g, inv_c;  // voxel, vote cell, cluster cell
    int bxy, bz;
    long long oxy, oz;
    int min_votes, min_cluster;
    float tol2;
    int log2cap;  // both hash tables
};

// 1. voxel keys
__global__ void k_wall_keys(const float* __restrict__ pts, int64_t n, WallParams P, u64* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    u64 key = INVALID_KEY;
    if (isfinite(x) && isfinite(y) && isfinite(z)) {
        const float fi = floorf(__fmul_rn(x, P.inv_v)), fj = floorf(__fmul_rn(y, P.inv_v)),
                    fk = floorf(__fmul_rn(z, P.inv_v));
        const float lo = -(float)P.oxy, hi = (float)(P.oxy - 2), loz = -(float)P.oz, hiz = (float)(P.oz - 2);
        if (fi >= lo && fi <= hi && fj >= lo && fj <= hi && fk >= loz && fk <= hiz) {
            const u64 ci = (u64)((long long)fi + P.oxy), cj = (u64)((long long)fj + P.oxy),
                      ck = (u64)((long long)fk + P.oz);
            key = ci | (cj << P.bxy) | (ck << (2 * P.bxy));
        }
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

__global__ void k_wall_flags(const u64* __restrict__ keys, int64_t n, uint32_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u64 k = keys[i];
    flags[i] = (k != INVALID_KEY && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

// run starts; starts[nv] = the first dropped position (or n)
__global__ void k_wall_starts(const u64* __restrict__ keys, const uint32_t* __restrict__ flags,
                              const uint32_t* __restrict__ rank, int64_t n, uint32_t* __restrict__ starts,
                              const uint32_t* __restrict__ nv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flags[i]) starts[rank[i]] = (uint32_t)i;
    const bool valid = keys[i] != INVALID_KEY;
    const bool next_invalid = (i + 1 == n) || keys[i + 1] == INVALID_KEY;
    if (valid && next_invalid) starts[*nv] = (uint32_t)(i + 1);
    if (i == 0 && !valid) starts[0] = 0u;  // nothing valid: nv = 0
}

__global__ void k_wall_centroid(const float* __restrict__ pts, const uint32_t* __restrict__ vals,
                                const uint32_t* __restrict__ starts, const uint32_t* __restrict__ nvp,
                                float4* __restrict__ cent) {
    const uint32_t nv = *nvp;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const uint32_t a = starts[v], b = starts[v + 1];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (uint32_t s = a; s < b; ++s) {
            const uint32_t i = vals[s];
            sx += (double)pts[3 * (size_t)i];
            sy += (double)pts[3 * (size_t)i + 1];
            sz += (double)pts[3 * (size_t)i + 2];
        }
        const double c = (double)(b - a);
        cent[v] = make_float4((float)(sx / c), (float)(sy / c), (float)(sz / c), 0.0f);
    }
}

__device__ __forceinline__ u64 vote_key(float4 c, float inv_g) {
    const long long u = (long long)floorf(__fmul_rn(c.x, inv_g)), w = (long long)floorf(__fmul_rn(c.y, inv_g));
    return ((u64)(u + (1ll << 31)) << 32) | (u64)(w + (1ll << 31));
}

__device__ __forceinline__ u64 cluster_key(float4 c, float inv_c) {
    const long long a = (long long)floorf(__fmul_rn(c.x, inv_c)) + (1ll << 20);
    const long long b = (long long)floorf(__fmul_rn(c.y, inv_c)) + (1ll << 20);
    const long long d = (long long)floorf(__fmul_rn(c.z, inv_c)) + (1ll << 20);
    return ((u64)a & 0x1fffffull) | (((u64)b & 0x1fffffull) << 21) | (((u64)d & 0x1fffffull) << 42);
}

// 2. votes
__global__ void k_wall_vote(const float4* __restrict__ cent, const uint32_t* __restrict__ nvp, WallParams P,
                            u64* __restrict__ vkeys, uint32_t* __restrict__ vcount, int* err) {
    const uint32_t nv = *nvp;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const int s = hash_insert(vkeys, P.log2cap, vote_key(cent[v], P.inv_g));
        if (s < 0) atomicOr(err, WALL_ERR_LIMIT);
        else atomicAdd(&vcount[s], 1u);
    }
}

// vertical flags, and the cluster-cell lists of the vertical voxels
__global__ void k_wall_vertical(const float4* __restrict__ cent, const uint32_t* __restrict__ nvp,
                                WallParams P, const u64* __restrict__ vkeys,
                                const uint32_t* __restrict__ vcount, int* __restrict__ vertical,
                                int* __restrict__ parent, u64* __restrict__ ckeys, int* __restrict__ head,
                                int* __restrict__ next, unsigned* __restrict__ nvert, int* err) {
    const uint32_t nv = *nvp;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const int s = hash_find(vkeys, P.log2cap, vote_key(cent[v], P.inv_g));
        const bool vert = s >= 0 && (int)vcount[s] > P.min_votes;
        vertical[v] = vert ? 1 : 0;
        parent[v] = (int)v;
        next[v] = -1;
        if (!vert) continue;
        atomicAdd(nvert, 1u);
        const int cs = hash_insert(ckeys, P.log2cap, cluster_key(cent[v], P.inv_c));
        if (cs < 0) {
            atomicOr(err, WALL_ERR_LIMIT);
            continue;
        }
        next[v] = atomicExch(&head[cs], (int)v);
    }
}

// Root of a: parents only ever point to smaller indices (roots point to
// themselves), so a node may be re-pointed to its grandparent at any time
// (path halving) without losing its root -- a write that races with another
// only writes an ancestor.  The chase is capped at `cap` steps.
__device__ int uf_find(int* parent, int a, uint32_t cap, int* err) {
    volatile int* par = parent;
    int p = par[a];
    for (uint32_t it = 0; it <= cap; ++it) {
        const int gp = par[p];
        if (gp == p) return p;
        par[a] = gp;
        a = p;
        p = gp;
    }
    atomicOr(err, WALL_ERR_LIMIT);
    return p;
}

__device__ void uf_union(int* parent, int a, int b, uint32_t cap, int* err) {
    for (uint32_t it = 0; it <= cap; ++it) {
        a = uf_find(parent, a, cap, err);
        b = uf_find(parent, b, cap, err);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        // hook the larger root a under the smaller b
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
    atomicOr(err, WALL_ERR_LIMIT);
}

// Visits the vertical voxels linked to v (d2 <= tol^2) with smaller index
// that lie in neighbour cell `c` (0..26) of v's cluster cell.
template <typename F>
__device__ __forceinline__ void for_links_in_cell(const float4* __restrict__ cent, uint32_t v, uint32_t nv,
                                                  int c, const WallParams& P, const u64* __restrict__ ckeys,
                                                  const int* __restrict__ head, const int* __restrict__ next,
                                                  F&& f) {
    const float4 cv = cent[v];
    const u64 k0 = cluster_key(cv, P.inv_c);
    const long long a0 = (long long)(k0 & 0x1fffffull), b0 = (long long)((k0 >> 21) & 0x1fffffull),
                    d0 = (long long)(k0 >> 42);
    const int dx = c % 3 - 1, dy = (c / 3) % 3 - 1, dz = c / 9 - 1;
    const u64 key = ((u64)(a0 + dx) & 0x1fffffull) | (((u64)(b0 + dy) & 0x1fffffull) << 21) |
                    (((u64)(d0 + dz) & 0x1fffffull) << 42);
    const int s = hash_find(ckeys, P.log2cap, key);
    if (s < 0) return;
    int j = head[s];
    for (uint32_t it = 0; j >= 0 && it <= nv; ++it) {
        if ((uint32_t)j < v && sqdist3(cv, cent[j]) <= P.tol2) f(j);
        j = next[j];
    }
}

// 3a. every vertical voxel starts under its smallest linked neighbour (a
// valid forest: parents are smaller members of the same component), so the
// unions that follow mostly find their ends already joined.  One warp per
// voxel, one lane per neighbouring cell: the 27 list walks run side by side.
__global__ void k_wall_link_init(const float4* __restrict__ cent, const uint32_t* __restrict__ nvp, WallParams P,
                                 const int* __restrict__ vertical, const u64* __restrict__ ckeys,
                                 const int* __restrict__ head, const int* __restrict__ next, int* parent) {
    const uint32_t nv = *nvp;
    const int lane = threadIdx.x & 31;
    const uint32_t wpb = blockDim.x >> 5;
    for (uint32_t v = blockIdx.x * wpb + (threadIdx.x >> 5); v < nv; v += gridDim.x * wpb) {
        if (!vertical[v]) continue;  // warp-uniform
        int m = (int)v;
        if (lane < 27) for_links_in_cell(cent, v, nv, lane, P, ckeys, head, next, [&](int j) { m = j < m ? j : m; });
        for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) parent[v] = m;
    }
}

// 3b. one round of pointer jumping: every vertical voxel moves up to its
// grandparent (the init forest has chains as long as a wall; a dozen rounds
// flatten them, so the unions below chase short paths)
__global__ void k_wall_jump(const uint32_t* __restrict__ nvp, const int* __restrict__ vertical, int* parent) {
    const uint32_t nv = *nvp;
    volatile int* par = parent;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        if (!vertical[v]) continue;
        const int p = par[v];
        const int gp = par[p];
        if (gp != p) par[v] = gp;
    }
}
constexpr int JUMP_ROUNDS = 12;

// 3. links between vertical voxels in the 27 neighbouring cluster cells:
// one warp per voxel, one lane per cell; pairs already under one parent are
// joined, the rest go through the union-find
__global__ void k_wall_union(const float4* __restrict__ cent, const uint32_t* __restrict__ nvp, WallParams P,
                             const int* __restrict__ vertical, const u64* __restrict__ ckeys,
                             const int* __restrict__ head, const int* __restrict__ next, int* parent, int* err) {
    const uint32_t nv = *nvp;
    const int lane = threadIdx.x & 31;
    const uint32_t wpb = blockDim.x >> 5;
    for (uint32_t v = blockIdx.x * wpb + (threadIdx.x >> 5); v < nv; v += gridDim.x * wpb) {
        if (!vertical[v]) continue;  // warp-uniform
        if (lane >= 27) continue;
        const int pv = __ldcg(&parent[v]);
        for_links_in_cell(cent, v, nv, lane, P, ckeys, head, next, [&](int j) {
            if (__ldcg(&parent[j]) != pv) uf_union(parent, (int)v, j, nv, err);
        });
    }
}

// labels and per-cluster extremes
__global__ void k_wall_label(const float4* __restrict__ cent, const uint32_t* __restrict__ nvp,
                             const int* __restrict__ vertical, int* parent,
                             int* __restrict__ label, unsigned* __restrict__ cmin_x, unsigned* __restrict__ cmax_x,
                             unsigned* __restrict__ cmin_y, unsigned* __restrict__ cmax_y,
                             unsigned* __restrict__ ccount, int* err) {
    const uint32_t nv = *nvp;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        if (!vertical[v]) {
            label[v] = -1;
            continue;
        }
        const int L = uf_find(parent, (int)v, nv, err);
        label[v] = L;
        const float4 c = cent[v];
        atomicMin(&cmin_x[L], f2ord(c.x));
        atomicMax(&cmax_x[L], f2ord(c.x));
        atomicMin(&cmin_y[L], f2ord(c.y));
        atomicMax(&cmax_y[L], f2ord(c.y));
        atomicAdd(&ccount[L], 1u);
    }
}

struct WallOut {
    long long n_voxels, n_vertical, wall_label, wall_count;
    float wall_length;
    int err;
    double beta[3];
};

// 4. the wall: max over clusters of (ordered length << 32) | (2^32 - 1 -
// label), i.e. the longest, then the smaller label
__global__ void k_wall_pick(const uint32_t* __restrict__ nvp, WallParams P, const unsigned* __restrict__ cmin_x,
                            const unsigned* __restrict__ cmax_x, const unsigned* __restrict__ cmin_y,
                            const unsigned* __restrict__ cmax_y, const unsigned* __restrict__ ccount,
                            u64* __restrict__ pick) {
    const uint32_t nv = *nvp;
    u64 best = 0ull;
    for (uint32_t L = blockIdx.x * blockDim.x + threadIdx.x; L < nv; L += gridDim.x * blockDim.x) {
        const unsigned cnt = ccount[L];
        if (cnt == 0u || (int)cnt < P.min_cluster) continue;
        if (!(__fadd_rn(ord2f(cmin_y[L]), ord2f(cmax_y[L])) < 0.0f)) continue;
        const float len = __fsub_rn(ord2f(cmax_x[L]), ord2f(cmin_x[L]));
        const u64 key = ((u64)f2ord(len) << 32) | (u64)(0xffffffffu - L);
        best = best > key ? best : key;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const u64 other = __shfl_xor_sync(0xffffffffu, best, o);
        best = best > other ? best : other;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(pick, best);
}

// 5. the fit: FIT_BLOCKS blocks of FIT_NT threads, a fixed voxel-to-thread
// map, binary64 sums of n, x, x^2, x^3, x^4, y, xy, x^2 y reduced over the
// warp and the block in a fixed order; the last block to finish adds the
// block partials in block order and solves the normal equations.
constexpr int FIT_NT = 256, FIT_BLOCKS = 64, FIT_VALS = 8;
__global__ void __launch_bounds__(FIT_NT) k_wall_fit(const float4* __restrict__ cent,
                                                     const uint32_t* __restrict__ nvp,
                                                     const int* __restrict__ label,
                                                     const unsigned* __restrict__ ccount,
                                                     const unsigned* __restrict__ nvert,
                                                     const int* __restrict__ err, const u64* __restrict__ pick,
                                                     double* __restrict__ partial, unsigned* __restrict__ ticket,
                                                     WallOut* out) {
    __shared__ double red[FIT_NT / 32][FIT_VALS];
    __shared__ unsigned last;
    const uint32_t nv = *nvp;
    const u64 b = *pick;
    const long long wl = b == 0ull ? -1ll : (long long)(0xffffffffu - (uint32_t)(b & 0xffffffffull));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[FIT_VALS] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (wl >= 0)
        for (uint32_t v = blockIdx.x * FIT_NT + threadIdx.x; v < nv; v += FIT_BLOCKS * FIT_NT) {
            if (label[v] != (int)wl) continue;
            const double x = (double)cent[v].x, y = (double)cent[v].y;
            const double x2 = x * x;
            acc[0] += 1.0;
            acc[1] += x;
            acc[2] += x2;
            acc[3] += x2 * x;
            acc[4] += x2 * x2;
            acc[5] += y;
            acc[6] += x * y;
            acc[7] += x2 * y;
        }
#pragma unroll
    for (int j = 0; j < FIT_VALS; ++j) {
        double a = acc[j];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) red[warp][j] = a;
    }
    __syncthreads();
    if (threadIdx.x < FIT_VALS) {
        double t = 0.0;
        for (int w = 0; w < FIT_NT / 32; ++w) t += red[w][threadIdx.x];
        partial[blockIdx.x * FIT_VALS + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == FIT_BLOCKS - 1 ? 1u : 0u;
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double S[FIT_VALS];
    for (int j = 0; j < FIT_VALS; ++j) {
        S[j] = 0.0;
        for (int bk = 0; bk < FIT_BLOCKS; ++bk) S[j] += __ldcg(&partial[bk * FIT_VALS + j]);
    }
    *ticket = 0u;
    out->n_voxels = nv;
    out->n_vertical = *nvert;
    out->wall_label = wl;
    out->wall_count = wl >= 0 ? (long long)ccount[wl] : 0;
    out->wall_length = b == 0ull ? 0.0f : ord2f((unsigned)(b >> 32));
    out->err = *err;
    out->beta[0] = out->beta[1] = out->beta[2] = NAN;
    if (wl < 0) return;
    double M[3][4] = {{S[0], S[1], S[2], S[5]}, {S[1], S[2], S[3], S[6]}, {S[2], S[3], S[4], S[7]}};
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int a = c + 1; a < 3; ++a)
            if (fabs(M[a][c]) > fabs(M[piv][c])) piv = a;
        if (!(fabs(M[piv][c]) > 0.0)) return;
        for (int bb = 0; bb < 4; ++bb) {
            const double t = M[c][bb];
            M[c][bb] = M[piv][bb];
            M[piv][bb] = t;
        }
        for (int a = 0; a < 3; ++a) {
            if (a == c) continue;
            const double f = M[a][c] / M[c][c];
            for (int bb = c; bb < 4; ++bb) M[a][bb] -= f * M[c][bb];
        }
    }
    for (int a = 0; a < 3; ++a) out->beta[a] = M[a][3] / M[a][a];
}

int bits_to_hold(long long n) {
    int b = 1;
    while ((1ll << b) < n) ++b;
    return b;
}

}  // namespace

struct pc_wall_s {
    uint32_t magic;
    int device;
    int64_t cap;  // max points
    pc_wall_opts opts;
    WallParams P;
    size_t sort_words, scan_words;
    void* mem;  // one allocation, carved below
    u64 *keys, *keys_alt, *vkeys, *ckeys;
    uint32_t *vals, *vals_alt, *flags, *rank, *starts, *sort_tmp, *scan_tmp, *nv, *vcount;
    float4* cent;
    int *vertical, *parent, *label, *head, *next, *err;
    unsigned *cmin_x, *cmax_x, *cmin_y, *cmax_y, *ccount, *nvert;
    WallOut* out;
    u64* pick;
    double* partial;
    unsigned* ticket;
    uint32_t* sorted_vals;  // where the sort left the indices
};

namespace {
constexpr uint32_t WALL_MAGIC = 0x77616c6cu;  // "wall"

bool wall_live(const pc_wall_s* w) { return w && w->magic == WALL_MAGIC; }

unsigned blocks_for(int64_t n, int nt) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + nt - 1) / nt, 65535)); }
}  // namespace

extern "C" {

void pc_wall_default_opts(pc_wall_opts* o) {
    if (!o) return;
    o->voxel = 0.2f;
    o->cell2d = 0.2f;
    o->min_votes = 2;
    o->tol = 0.45f;
    o->min_cluster = 10;
    o->max_range = 128.0f;
    o->max_height = 16.0f;
}

pc_status pc_wall_create(int64_t max_points, const pc_wall_opts* opts, pc_wall* out) {
    if (!out) return PC_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_points < 1 || max_points >= ((int64_t)1 << 31)) return PC_ERR_INVALID_ARG;
    pc_wall_opts o;
    pc_wall_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.voxel > 0) || !(o.cell2d > 0) || !(o.tol > 0) || !(o.max_range > 0) || !(o.max_height > 0) ||
        o.min_votes < 0 || o.min_cluster < 0 || !std::isfinite(o.voxel) || !std::isfinite(o.cell2d) ||
        !std::isfinite(o.tol) || !std::isfinite(o.max_range) || !std::isfinite(o.max_height))
        return PC_ERR_INVALID_ARG;
    WallParams P{};
    P.inv_v = 1.0f / o.voxel;
    P.inv_g = 1.0f / o.cell2d;
    P.inv_c = 1.0f / (o.tol * (1.0f + 0x1p-10f));
    const long long rxy = (long long)std::ceil(o.max_range / o.voxel) + 1;
    const long long rz = (long long)std::ceil(o.max_height / o.voxel) + 1;
    P.bxy = bits_to_hold(2 * rxy);
    P.bz = bits_to_hold(2 * rz);
    if (2 * P.bxy + P.bz > 63) return PC_ERR_INVALID_ARG;
    P.oxy = 1ll << (P.bxy - 1);
    P.oz = 1ll << (P.bz - 1);
    P.min_votes = o.min_votes;
    P.min_cluster = o.min_cluster;
    P.tol2 = o.tol * o.tol;
    int lc = 1;
    while ((1ll << lc) < 2 * max_points) ++lc;
    P.log2cap = lc;
    const int64_t N = max_points, C = 1ll << lc;
    pc_wall_s* w = new (std::nothrow) pc_wall_s();
    if (!w) return PC_ERR_OOM;
    std::memset(w, 0, sizeof(*w));
    cudaGetDevice(&w->device);
    w->cap = N;
    w->opts = o;
    w->P = P;
    w->sort_words = pc_sort_temp_words(N);
    w->scan_words = pc_scan_temp_words(N);
    // carve one allocation (every part 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o2 = off;
        off += (bytes + 255) & ~(size_t)255;
        return o2;
    };
    const size_t o_keys = take(8 * N), o_keys_alt = take(8 * N), o_vkeys = take(8 * C), o_ckeys = take(8 * C);
    const size_t o_vals = take(4 * N), o_vals_alt = take(4 * N), o_flags = take(4 * N), o_rank = take(4 * N),
                 o_starts = take(4 * (N + 1)), o_sort = take(4 * w->sort_words), o_scan = take(4 * w->scan_words),
                 o_nv = take(4), o_vcount = take(4 * C);
    const size_t o_cent = take(16 * N);
    const size_t o_vert = take(4 * N), o_par = take(4 * N), o_label = take(4 * N), o_head = take(4 * C),
                 o_next = take(4 * N), o_err = take(4);
    const size_t o_cminx = take(4 * N), o_cmaxx = take(4 * N), o_cminy = take(4 * N), o_cmaxy = take(4 * N),
                 o_ccount = take(4 * N), o_nvert = take(4), o_out = take(sizeof(WallOut)), o_pick = take(8),
                 o_partial = take(sizeof(double) * FIT_BLOCKS * FIT_VALS), o_ticket = take(4);
    cudaError_t e = cudaMalloc(&w->mem, off);
    if (e != cudaSuccess) {
        delete w;
        return pc_from_cuda(e);
    }
    char* b = static_cast<char*>(w->mem);
    w->keys = reinterpret_cast<u64*>(b + o_keys);
    w->keys_alt = reinterpret_cast<u64*>(b + o_keys_alt);
    w->vkeys = reinterpret_cast<u64*>(b + o_vkeys);
    w->ckeys = reinterpret_cast<u64*>(b + o_ckeys);
    w->vals = reinterpret_cast<uint32_t*>(b + o_vals);
    w->vals_alt = reinterpret_cast<uint32_t*>(b + o_vals_alt);
    w->flags = reinterpret_cast<uint32_t*>(b + o_flags);
    w->rank = reinterpret_cast<uint32_t*>(b + o_rank);
    w->starts = reinterpret_cast<uint32_t*>(b + o_starts);
    w->sort_tmp = reinterpret_cast<uint32_t*>(b + o_sort);
    w->scan_tmp = reinterpret_cast<uint32_t*>(b + o_scan);
    w->nv = reinterpret_cast<uint32_t*>(b + o_nv);
    w->vcount = reinterpret_cast<uint32_t*>(b + o_vcount);
    w->cent = reinterpret_cast<float4*>(b + o_cent);
    w->vertical = reinterpret_cast<int*>(b + o_vert);
    w->parent = reinterpret_cast<int*>(b + o_par);
    w->label = reinterpret_cast<int*>(b + o_label);
    w->head = reinterpret_cast<int*>(b + o_head);
    w->next = reinterpret_cast<int*>(b + o_next);
    w->err = reinterpret_cast<int*>(b + o_err);
    w->cmin_x = reinterpret_cast<unsigned*>(b + o_cminx);
    w->cmax_x = reinterpret_cast<unsigned*>(b + o_cmaxx);
    w->cmin_y = reinterpret_cast<unsigned*>(b + o_cminy);
    w->cmax_y = reinterpret_cast<unsigned*>(b + o_cmaxy);
    w->ccount = reinterpret_cast<unsigned*>(b + o_ccount);
    w->nvert = reinterpret_cast<unsigned*>(b + o_nvert);
    w->out = reinterpret_cast<WallOut*>(b + o_out);
    w->pick = reinterpret_cast<u64*>(b + o_pick);
    w->partial = reinterpret_cast<double*>(b + o_partial);
    w->ticket = reinterpret_cast<unsigned*>(b + o_ticket);
    w->magic = WALL_MAGIC;
    *out = w;
    return PC_OK;
}

pc_status pc_wall_detect(pc_wall w, const float* pts_dev, int64_t n, pc_stream s) {
    if (!wall_live(w)) return PC_ERR_INVALID_ARG;
    if (n < 0 || n > w->cap) return PC_ERR_INVALID_ARG;
    if (n > 0 && !pts_dev) return PC_ERR_INVALID_ARG;
    if (n > 0 && !pc_is_device_ptr(pts_dev)) return PC_ERR_BAD_POINTER;
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != w->device) cudaSetDevice(w->device);
    cudaStream_t st = (cudaStream_t)s;
    const WallParams P = w->P;
    const int64_t C = 1ll << P.log2cap;
    const int NT = 256;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
        return e == cudaSuccess;
    };
    ok(cudaMemsetAsync(w->vkeys, 0xff, 8 * C, st));
    ok(cudaMemsetAsync(w->ckeys, 0xff, 8 * C, st));
    ok(cudaMemsetAsync(w->vcount, 0, 4 * C, st));
    ok(cudaMemsetAsync(w->head, 0xff, 4 * C, st));
    ok(cudaMemsetAsync(w->err, 0, 4, st));
    ok(cudaMemsetAsync(w->nvert, 0, 4, st));
    ok(cudaMemsetAsync(w->nv, 0, 4, st));
    ok(cudaMemsetAsync(w->cmin_x, 0xff, 4 * w->cap, st));
    ok(cudaMemsetAsync(w->cmin_y, 0xff, 4 * w->cap, st));
    ok(cudaMemsetAsync(w->cmax_x, 0, 4 * w->cap, st));
    ok(cudaMemsetAsync(w->cmax_y, 0, 4 * w->cap, st));
    ok(cudaMemsetAsync(w->ccount, 0, 4 * w->cap, st));
    ok(cudaMemsetAsync(w->starts, 0, 4, st));
    ok(cudaMemsetAsync(w->pick, 0, 8, st));
    ok(cudaMemsetAsync(w->ticket, 0, 4, st));
    if (n > 0) {
        const unsigned gb = (unsigned)((n + NT - 1) / NT);
        k_wall_keys<<<gb, NT, 0, st>>>(pts_dev, n, P, w->keys, w->vals);
        ok(cudaGetLastError());
        // dropped points carry all ones in every sorted bit and sort last
        u64* k = w->keys;
        uint32_t* v = w->vals;
        ok(pc_radix_sort_pairs(&k, &v, w->keys_alt, w->vals_alt, n, 2 * P.bxy + P.bz, w->sort_tmp, st));
        w->sorted_vals = v;
        k_wall_flags<<<gb, NT, 0, st>>>(k, n, w->flags);
        ok(cudaGetLastError());
        ok(pc_scan_exclusive(w->flags, w->rank, n, w->nv, w->scan_tmp, st));
        k_wall_starts<<<gb, NT, 0, st>>>(k, w->flags, w->rank, n, w->starts, w->nv);
        ok(cudaGetLastError());
        const unsigned vb = blocks_for(n, NT);
        k_wall_centroid<<<vb, NT, 0, st>>>(pts_dev, v, w->starts, w->nv, w->cent);
        k_wall_vote<<<vb, NT, 0, st>>>(w->cent, w->nv, P, w->vkeys, w->vcount, w->err);
        k_wall_vertical<<<vb, NT, 0, st>>>(w->cent, w->nv, P, w->vkeys, w->vcount, w->vertical, w->parent,
                                          w->ckeys, w->head, w->next, w->nvert, w->err);
        // one warp per voxel for the list walks
        const unsigned wb = blocks_for(n * 32, NT);
        k_wall_link_init<<<wb, NT, 0, st>>>(w->cent, w->nv, P, w->vertical, w->ckeys, w->head, w->next,
                                           w->parent);
        for (int r = 0; r < JUMP_ROUNDS; ++r) k_wall_jump<<<vb, NT, 0, st>>>(w->nv, w->vertical, w->parent);
        k_wall_union<<<wb, NT, 0, st>>>(w->cent, w->nv, P, w->vertical, w->ckeys, w->head, w->next, w->parent,
                                       w->err);
        k_wall_label<<<vb, NT, 0, st>>>(w->cent, w->nv, w->vertical, w->parent, w->label, w->cmin_x, w->cmax_x,
                                       w->cmin_y, w->cmax_y, w->ccount, w->err);
        ok(cudaGetLastError());
    }
    k_wall_pick<<<blocks_for(std::max<int64_t>(n, 1), NT), NT, 0, st>>>(w->nv, P, w->cmin_x, w->cmax_x, w->cmin_y,
                                                                        w->cmax_y, w->ccount, w->pick);
    k_wall_fit<<<FIT_BLOCKS, FIT_NT, 0, st>>>(w->cent, w->nv, w->label, w->ccount, w->nvert, w->err, w->pick,
                                              w->partial, w->ticket, w->out);
    ok(cudaGetLastError());
    if (prev >= 0 && prev != w->device) cudaSetDevice(prev);
    return pc_from_cuda(e);
}

pc_status pc_wall_get(pc_wall w, pc_stream s, pc_wall_result* res, float* centroids_host, int32_t* vertical_host,
                      int32_t* labels_host) {
    if (!wall_live(w) || !res) return PC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)s;
    WallOut o;
    cudaError_t e = cudaMemcpyAsync(&o, w->out, sizeof(o), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pc_from_cuda(e);
    res->n_voxels = o.n_voxels;
    res->n_vertical = o.n_vertical;
    res->wall_label = o.wall_label;
    res->wall_count = o.wall_count;
    res->wall_length = o.wall_length;
    for (int a = 0; a < 3; ++a) res->beta[a] = o.beta[a];
    res->d_w = o.beta[0];
    const int64_t nv = o.n_voxels;
    if (nv > 0 && centroids_host) {
        // float4 on the device, xyz on the host
        float4* tmp = new (std::nothrow) float4[nv];
        if (!tmp) return PC_ERR_OOM;
        e = cudaMemcpyAsync(tmp, w->cent, sizeof(float4) * nv, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (int64_t i = 0; e == cudaSuccess && i < nv; ++i) {
            centroids_host[3 * i] = tmp[i].x;
            centroids_host[3 * i + 1] = tmp[i].y;
            centroids_host[3 * i + 2] = tmp[i].z;
        }
        delete[] tmp;
    }
    if (e == cudaSuccess && nv > 0 && vertical_host)
        e = cudaMemcpyAsync(vertical_host, w->vertical, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && nv > 0 && labels_host)
        e = cudaMemcpyAsync(labels_host, w->label, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pc_from_cuda(e);
    return o.err ? PC_ERR_SEARCH_LIMIT : PC_OK;
}

void pc_wall_destroy(pc_wall w) {
    if (!wall_live(w)) return;
    w->magic = 0;
    if (w->mem) cudaFree(w->mem);
    delete w;
}

}  // extern "C"
