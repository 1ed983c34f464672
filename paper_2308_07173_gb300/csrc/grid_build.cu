// Target build: the device-resident voxel-hash grid over the map
// (Sec. III-C3 "Scan match for correction": the map is queried through a
// "GPU-hash data structure").
//
//   1. finite check + bounding box            (k_bbox)
//   2. cell edge h: given, or the h whose mean points per occupied cell is
//      the requested occupancy, found by bisection on a device hash-set
//      count of occupied cells                (k_count_cells)
//   3. cell key per point, packed cx | cy << bx | cz << (bx+by)  (k_keys)
//   4. stable LSD radix sort of (key, index), 8-bit digits, only the key
//      bits in use                            (k_rs_*)
//   5. run boundaries -> occupied cells (key, start)  (k_flags, scan, k_cells)
//   6. open-addressing hash key -> (start, count), linear probing
//                                             (k_hash_insert)
//   7. float4 copies: cell order with the original index in .w, and the
//      caller's order for the covariance gathers  (k_gather)
//
// The build synchronises its stream a few times to read sizes back; it is a
// one-off per map and off the per-scan path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pc_internal.h"

using namespace pcdev;

namespace {

typedef unsigned long long u64;

// order-preserving float <-> uint32 map for atomic min/max
__host__ __device__ __forceinline__ unsigned f2ord(float f) {
#ifdef __CUDA_ARCH__
    unsigned u = __float_as_uint(f);
#else
    unsigned u;
    std::memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ord2f(unsigned o) {
    unsigned u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void k_bbox_init(unsigned* bb) {
    if (threadIdx.x < 3) bb[threadIdx.x] = 0xffffffffu;
    else if (threadIdx.x < 6) bb[threadIdx.x] = 0u;
}

__global__ void k_bbox(const float* __restrict__ xyz, int64_t M, unsigned* bb, int* status) {
    unsigned mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = xyz[3 * i + a];
            if (!isfinite(v)) {
                bad = true;
            } else {
                const unsigned u = f2ord(v);
                mn[a] = min(mn[a], u);
                mx[a] = max(mx[a], u);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], __shfl_xor_sync(FULL, mn[a], o));
            mx[a] = max(mx[a], __shfl_xor_sync(FULL, mx[a], o));
        }
    const bool any_bad = __any_sync(FULL, bad);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bb[a], mn[a]);
            atomicMax(&bb[3 + a], mx[a]);
        }
        if (any_bad) atomicOr(status, ST_NONFINITE);
    }
}

// number of occupied cells for a trial h (21-bit packing; h >= extent/2^20)
__global__ void k_count_cells(const float* __restrict__ xyz, int64_t M, float ox, float oy,
                              float oz, float inv_h, u64* set, int log2cap,
                              unsigned long long* counter) {
    const uint32_t mask = (1u << log2cap) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const int cx = min(max(cell_of(xyz[3 * i], ox, inv_h), 0), (1 << 21) - 1);
        const int cy = min(max(cell_of(xyz[3 * i + 1], oy, inv_h), 0), (1 << 21) - 1);
        const int cz = min(max(cell_of(xyz[3 * i + 2], oz, inv_h), 0), (1 << 21) - 1);
        const u64 key = pack_key(cx, cy, cz, 21, 21);
        uint32_t slot = hash_slot(key, log2cap);
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const u64 prev = atomicCAS(&set[slot], EMPTY_KEY, key);
            if (prev == EMPTY_KEY) {
                atomicAdd(counter, 1ull);
                break;
            }
            if (prev == key) break;
            slot = (slot + 1u) & mask;
        }
    }
}

__global__ void k_dims(float mxx, float mxy, float mxz, float ox, float oy, float oz, float inv_h,
                       int* dims) {
    dims[0] = cell_of(mxx, ox, inv_h) + 1;
    dims[1] = cell_of(mxy, oy, inv_h) + 1;
    dims[2] = cell_of(mxz, oz, inv_h) + 1;
}

// Sort key of each point: its cell key, followed (sub = 3) by its sub-bin
// along x, so that a cell's points end up ordered by sub-bin.
__global__ void k_keys(const float* __restrict__ xyz, int64_t M, float ox, float oy, float oz,
                       float inv_h, int bx, int by, int sub, u64* __restrict__ keys,
                       uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int cx = cell_of(xyz[3 * i], ox, inv_h);
    const int cy = cell_of(xyz[3 * i + 1], oy, inv_h);
    const int cz = cell_of(xyz[3 * i + 2], oz, inv_h);
    const u64 key = pack_key(cx, cy, cz, bx, by);
    keys[i] = sub ? (key << 3) | (u64)sub_bin(cell_coord(xyz[3 * i], ox, inv_h)) : key;
    vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------- scans
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total, uint32_t* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const uint32_t pre = warp ? sh[warp - 1] : 0u;
    *total = sh[NT / 32 - 1];
    __syncthreads();
    return pre + x - v;
}

constexpr int SC_NT = 1024, SC_IPT = 4, SC_TILE = SC_NT * SC_IPT;

__global__ void __launch_bounds__(SC_NT) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                       uint32_t* bsum) {
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_IPT;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SC_IPT; ++j)
        if (base + j < n) s += in[base + j];
    uint32_t tot;
    block_excl_scan<SC_NT>(s, &tot, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SC_NT) k_scan_top(uint32_t* bsum, int nb, uint32_t* total) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += SC_NT) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan<SC_NT>(v, &tot, sh);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(SC_NT) k_scan_down(const uint32_t* __restrict__ in,
                                                     uint32_t* __restrict__ out, int64_t n,
                                                     const uint32_t* __restrict__ bsum) {
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_IPT;
    uint32_t v[SC_IPT];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SC_IPT; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        s += v[j];
    }
    uint32_t tot;
    uint32_t run = bsum[blockIdx.x] + block_excl_scan<SC_NT>(s, &tot, sh);
#pragma unroll
    for (int j = 0; j < SC_IPT; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_NT = 256, RS_IPT = 16, RS_TILE = RS_NT * RS_IPT, RS_WARPS = RS_NT / 32;
constexpr int RS_ROUNDS = RS_TILE / RS_WARPS / 32;  // 16 rounds of 32 per warp

__global__ void __launch_bounds__(RS_NT) k_rs_hist(const u64* __restrict__ keys, int64_t n,
                                                   int shift, uint32_t* counts, int nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int j = 0; j < RS_IPT; ++j) {
        const int64_t i = base + (int64_t)j * RS_NT + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(SC_NT) k_rs_scan_digits(uint32_t* counts, int nb,
                                                          uint32_t* totals) {
    __shared__ uint32_t sh[32];
    uint32_t* row = counts + (int64_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += SC_NT) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? row[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan<SC_NT>(v, &tot, sh);
        if (i < nb) row[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Stable scatter: inside a block each warp ranks its 16 rounds of 32 items in
// order (match.any groups equal digits; the lowest lane of a group bumps the
// warp's running digit count), then warps are offset in warp order.
__global__ void __launch_bounds__(RS_NT) k_rs_scatter(const u64* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      u64* __restrict__ kout,
                                                      uint32_t* __restrict__ vout, int64_t n,
                                                      int shift, const uint32_t* __restrict__ counts,
                                                      int nb, const uint32_t* __restrict__ totals) {
    __shared__ uint32_t wh[RS_WARPS][256];
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t sh[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        uint32_t tot;
        dbase[tid] = block_excl_scan<RS_NT>(totals[tid], &tot, sh);
    }
    for (int d = tid; d < RS_WARPS * 256; d += RS_NT) (&wh[0][0])[d] = 0u;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (RS_ROUNDS * 32);
    u64 key[RS_ROUNDS];
    uint32_t val[RS_ROUNDS], rank[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0ull;
        val[r] = valid ? vin[i] : 0u;
        const unsigned d = valid ? ((unsigned)(key[r] >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(FULL, d);
        const unsigned lt = __popc(peers & lanemask_lt());
        const uint32_t b0 = valid ? wh[warp][d] : 0u;
        __syncwarp();
        if (valid && lt == 0u) wh[warp][d] = b0 + __popc(peers);
        __syncwarp();
        rank[r] = b0 + lt;
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = wh[w][tid];
            wh[w][tid] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            const unsigned d = (unsigned)(key[r] >> shift) & 255u;
            const uint32_t pos = dbase[d] + counts[(int64_t)d * nb + blockIdx.x] + wh[warp][d] + rank[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ---------------------------------------------------------------- cells
__global__ void k_flags(const u64* __restrict__ keys, int64_t n, int sub, uint32_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (i == 0 || (keys[i] >> sub) != (keys[i - 1] >> sub)) ? 1u : 0u;
}

__global__ void k_cells(const u64* __restrict__ keys, const uint32_t* __restrict__ flags,
                        const uint32_t* __restrict__ ord, int64_t n, int sub, u64* __restrict__ cell_keys,
                        uint32_t* __restrict__ cell_start, uint32_t U) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flags[i]) {
        cell_keys[ord[i]] = keys[i] >> sub;
        cell_start[ord[i]] = (uint32_t)i;
    }
    if (i == 0) cell_start[U] = (uint32_t)n;
}

__global__ void k_hash_insert(const u64* __restrict__ cell_keys,
                              const uint32_t* __restrict__ cell_start, int64_t U, uint4* table,
                              int log2cap) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    const u64 key = cell_keys[u];
    const uint32_t start = cell_start[u], cnt = cell_start[u + 1] - start;
    const uint32_t mask = (1u << log2cap) - 1u;
    uint32_t slot = hash_slot(key, log2cap);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const u64 prev = atomicCAS(reinterpret_cast<u64*>(&table[slot]), EMPTY_KEY, key);
        if (prev == EMPTY_KEY) {
            table[slot].z = start;
            table[slot].w = cnt;
            return;
        }
        slot = (slot + 1u) & mask;
    }
}

__global__ void k_occ_set(const u64* __restrict__ cell_keys, int64_t U, int bx, int by, int dimx,
                          int dimy, uint32_t* occ) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    const u64 key = cell_keys[u];
    const int64_t cx = (int64_t)(key & ((1ull << bx) - 1ull));
    const int64_t cy = (int64_t)((key >> bx) & ((1ull << by) - 1ull));
    const int64_t cz = (int64_t)(key >> (bx + by));
    const int64_t L = cx + (int64_t)dimx * (cy + (int64_t)dimy * cz);
    atomicOr(&occ[L >> 5], 1u << (uint32_t)(L & 31));
}

// Dense starts from the row index: for every linear cell index L of the
// grid (and L = ngrid), the rank u of the first occupied cell at or after
// L, read through the bitmap and the word ranks, gives dstart[L] =
// cell_start[u].
__global__ void k_dstart(const uint32_t* __restrict__ occ, const uint32_t* __restrict__ rank,
                         const uint32_t* __restrict__ cell_start, int64_t ngrid, uint32_t ncells,
                         uint32_t* __restrict__ dstart) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L > ngrid) return;
    uint32_t u = ncells;
    if (L < ngrid) {
        const int64_t w = L >> 5;
        u = rank[w] + (uint32_t)__popc(occ[w] & ((1u << (uint32_t)(L & 31)) - 1u));
    }
    dstart[L] = cell_start[u];
}

// Sub-cell cut words (pc_device.cuh, Grid::xcut) from the sorted keys (cell
// key << 3 | sub-bin): each run of equal sub-bins in a cell writes the
// counts below the sub-bins it starts, the cell's last point those above
// its own.  Cells of 255 points or more keep the zero word (no cut).
__global__ void k_xcut(const u64* __restrict__ keys, int64_t n, int bx, int by, int dimx, int dimy,
                       const uint32_t* __restrict__ dstart, unsigned char* __restrict__ xcut) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u64 key = keys[i] >> 3;
    const int sb = (int)(keys[i] & 7u);
    const int64_t cx = (int64_t)(key & ((1ull << bx) - 1));
    const int64_t cy = (int64_t)((key >> bx) & ((1ull << by) - 1));
    const int64_t cz = (int64_t)(key >> (bx + by));
    const int64_t L = cx + (int64_t)dimx * (cy + (int64_t)dimy * cz);
    const uint32_t s = dstart[L], cnt = dstart[L + 1] - s;
    if (cnt >= 255u) return;
    const uint32_t r = (uint32_t)i - s;  // rank in the cell
    const int prev = r > 0 ? (int)(keys[i - 1] & 7u) : -1;
    for (int b = prev + 1; b <= sb; ++b)
        if (b >= 1) xcut[8 * L + (b - 1)] = (unsigned char)r;
    if (r + 1 == cnt)
        for (int b = sb + 1; b <= 8; ++b) xcut[8 * L + (b - 1)] = (unsigned char)cnt;
}

__global__ void k_popc(const uint32_t* __restrict__ occ, int64_t nw, uint32_t* __restrict__ out) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) out[w] = (uint32_t)__popc(occ[w]);
}

__global__ void k_gather(const float* __restrict__ xyz, const uint32_t* __restrict__ vals,
                         int64_t n, float4* __restrict__ pts, float4* __restrict__ xyz4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t o = vals[i];
    const float x = xyz[3 * (int64_t)o], y = xyz[3 * (int64_t)o + 1], z = xyz[3 * (int64_t)o + 2];
    pts[i] = make_float4(x, y, z, __uint_as_float(o));
    xyz4[o] = make_float4(x, y, z, 0.0f);
}

// ---------------------------------------------------------------- host helpers
struct Scratch {
    std::vector<void*> bufs;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T* alloc(size_t count) {
        void* p = nullptr;
        if (err != cudaSuccess) return nullptr;
        err = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (err != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Scratch() {
        for (void* p : bufs) cudaFree(p);
    }
};

int bits_for(int dim) {  // bits to hold 0..dim-1, at least 1
    int b = 1;
    while ((1ll << b) < (long long)dim) ++b;
    return b;
}

unsigned grid_for(int64_t n, int nt) { return (unsigned)std::max<int64_t>(1, (n + nt - 1) / nt); }

cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                           Scratch& sc, cudaStream_t s) {
    const int nb = (int)((n + SC_TILE - 1) / SC_TILE);
    uint32_t* bsum = sc.alloc<uint32_t>(nb);
    if (!bsum) return sc.err;
    k_scan_reduce<<<nb, SC_NT, 0, s>>>(in, n, bsum);
    k_scan_top<<<1, SC_NT, 0, s>>>(bsum, nb, total_dev);
    k_scan_down<<<nb, SC_NT, 0, s>>>(in, out, n, bsum);
    return cudaGetLastError();
}

cudaError_t radix_sort(u64*& keys, uint32_t*& vals, u64* keys_alt, uint32_t* vals_alt, int64_t n,
                       int nbits, Scratch& sc, cudaStream_t s) {
    const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
    uint32_t* counts = sc.alloc<uint32_t>((size_t)256 * nb);
    uint32_t* totals = sc.alloc<uint32_t>(256);
    if (!counts || !totals) return sc.err;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_rs_hist<<<nb, RS_NT, 0, s>>>(keys, n, shift, counts, nb);
        k_rs_scan_digits<<<256, SC_NT, 0, s>>>(counts, nb, totals);
        k_rs_scatter<<<nb, RS_NT, 0, s>>>(keys, vals, keys_alt, vals_alt, n, shift, counts, nb,
                                          totals);
        std::swap(keys, keys_alt);
        std::swap(vals, vals_alt);
    }
    return cudaGetLastError();
}

}  // namespace

// Sort and scan on caller buffers (used by the wall detector, which sizes
// everything once at creation).
size_t pc_sort_temp_words(int64_t n) {
    const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    return (size_t)256 * (size_t)std::max<int64_t>(nb, 1) + 256;
}

cudaError_t pc_radix_sort_pairs(u64** keys, uint32_t** vals, u64* keys_alt, uint32_t* vals_alt,
                                int64_t n, int nbits, uint32_t* temp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
    uint32_t* counts = temp;
    uint32_t* totals = temp + (size_t)256 * nb;
    u64* k = *keys;
    uint32_t* v = *vals;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_rs_hist<<<nb, RS_NT, 0, s>>>(k, n, shift, counts, nb);
        k_rs_scan_digits<<<256, SC_NT, 0, s>>>(counts, nb, totals);
        k_rs_scatter<<<nb, RS_NT, 0, s>>>(k, v, keys_alt, vals_alt, n, shift, counts, nb, totals);
        std::swap(k, keys_alt);
        std::swap(v, vals_alt);
    }
    *keys = k;
    *vals = v;
    return cudaGetLastError();
}

size_t pc_scan_temp_words(int64_t n) {
    return (size_t)std::max<int64_t>((n + SC_TILE - 1) / SC_TILE, 1);
}

cudaError_t pc_scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                              uint32_t* temp, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
    const int nb = (int)((n + SC_TILE - 1) / SC_TILE);
    k_scan_reduce<<<nb, SC_NT, 0, s>>>(in, n, temp);
    k_scan_top<<<1, SC_NT, 0, s>>>(temp, nb, total_dev);
    k_scan_down<<<nb, SC_NT, 0, s>>>(in, out, n, temp);
    return cudaGetLastError();
}

namespace {

// occupied cells for trial h
cudaError_t count_cells(const float* xyz, int64_t M, const float o[3], float h, u64* set,
                        int log2cap, unsigned long long* counter, cudaStream_t s,
                        unsigned long long* out) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(set, 0xff, sizeof(u64) << log2cap, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    const float inv_h = 1.0f / h;
    k_count_cells<<<grid_for(M, 256), 256, 0, s>>>(xyz, M, o[0], o[1], o[2], inv_h, set, log2cap,
                                                   counter);
    if ((e = cudaMemcpyAsync(out, counter, sizeof(*out), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

}  // namespace

void pc_free_grid(pc_target_s* t) {
    void* ps[] = {t->table, t->pts, t->xyz, t->cell_keys, t->cell_start, t->status, t->stage,
                  t->dstart, t->xcut};
    for (void* p : ps)
        if (p) cudaFree(p);
    t->table = nullptr;
    t->pts = t->xyz = nullptr;
    t->cell_keys = nullptr;
    t->cell_start = nullptr;
    t->status = nullptr;
    t->dstart = nullptr;
    t->xcut = nullptr;
    t->stage = nullptr;
    t->stage_bytes = 0;
}

#define PC_TRY(expr)                                     \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) return pc_from_cuda(_e);  \
    } while (0)

pc_status pc_build_grid(const float* xyz, int64_t M, const pc_build_opts& opts, cudaStream_t s,
                        pc_target_s* t) {
    Scratch sc;
    // persistent small buffers first
    // status word + statistics counters (64 bytes)
    PC_TRY(cudaMalloc(&t->status, 64));
    PC_TRY(cudaMemsetAsync(t->status, 0, 64, s));

    // 1. bbox + finite check
    unsigned* bb = sc.alloc<unsigned>(8);
    if (!bb) return pc_from_cuda(sc.err);
    k_bbox_init<<<1, 32, 0, s>>>(bb);
    {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned blocks = (unsigned)std::min<int64_t>(grid_for(M, 256), (int64_t)sms * 8);
        k_bbox<<<blocks, 256, 0, s>>>(xyz, M, bb, t->status);
    }
    PC_TRY(cudaGetLastError());
    unsigned hb[6];
    int hstatus = 0;
    PC_TRY(cudaMemcpyAsync(hb, bb, sizeof(hb), cudaMemcpyDeviceToHost, s));
    PC_TRY(cudaMemcpyAsync(&hstatus, t->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    PC_TRY(cudaStreamSynchronize(s));
    if (hstatus & ST_NONFINITE) return PC_ERR_NONFINITE;
    float o[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        o[a] = ord2f(hb[a]);
        mx[a] = ord2f(hb[3 + a]);
        t->bbox_max[a] = mx[a];
    }
    float ext = 0.0f, scale = 0.0f;
    for (int a = 0; a < 3; ++a) {
        ext = std::max(ext, mx[a] - o[a]);
        scale = std::max(scale, std::max(std::fabs(o[a]), std::fabs(mx[a])));
    }

    // 2. cell edge
    const float h_floor = ext > 0.0f ? ext / 1048576.0f * 1.001f : 0.0f;  // dims <= 2^20 + 1
    float h = opts.cell_size;
    if (!(h > 0.0f) || !std::isfinite(h)) {
        if (ext == 0.0f) {
            h = 1.0f;
        } else {
            int log2cap = 10;
            while ((1ll << log2cap) < 2 * M) ++log2cap;
            u64* set = sc.alloc<u64>((size_t)1 << log2cap);
            unsigned long long* counter = sc.alloc<unsigned long long>(1);
            if (!set || !counter) return pc_from_cuda(sc.err);
            const double target = opts.occupancy > 0 ? opts.occupancy : 12.0;
            double lo = h_floor, hi = (double)ext * 1.001;
            unsigned long long U = 0;
            PC_TRY(count_cells(xyz, M, o, (float)hi, set, log2cap, counter, s, &U));
            if ((double)M / (double)std::max(U, 1ull) >= target) {
                for (int it = 0; it < 14; ++it) {
                    const double mid = std::sqrt(lo * hi);
                    PC_TRY(count_cells(xyz, M, o, (float)mid, set, log2cap, counter, s, &U));
                    if ((double)M / (double)std::max(U, 1ull) < target) lo = mid; else hi = mid;
                }
            }
            h = (float)hi;
        }
    }
    h = std::max(h, h_floor);
    const float inv_h = 1.0f / h;

    // dims with the device rule
    int* dims_dev = sc.alloc<int>(4);
    if (!dims_dev) return pc_from_cuda(sc.err);
    k_dims<<<1, 1, 0, s>>>(mx[0], mx[1], mx[2], o[0], o[1], o[2], inv_h, dims_dev);
    int dims[3];
    PC_TRY(cudaMemcpyAsync(dims, dims_dev, sizeof(dims), cudaMemcpyDeviceToHost, s));
    PC_TRY(cudaStreamSynchronize(s));
    const int bx = bits_for(dims[0]), by = bits_for(dims[1]), bz = bits_for(dims[2]);
    if (bx > 21 || by > 21 || bz > 21) return PC_ERR_INVALID_ARG;
    // The row index (dense cell starts) is built when it costs at most eight
    // times the points' copy, else searches visit cells through the hash;
    // with it, the sub-cell cut (8 bytes a grid cell) when that costs at
    // most eight times the copy.
    const int64_t ngrid = (int64_t)dims[0] * dims[1] * dims[2];
    const bool dense = ngrid < ((int64_t)1 << 31) && (ngrid + 1) * 4 <= 8 * 16 * M;
    const int sub = (dense && bx + by + bz + 3 <= 64 && 8 * ngrid <= 8 * 16 * M) ? 3 : 0;

    // 3-4. keys and sort
    u64* keys = sc.alloc<u64>(M);
    u64* keys_alt = sc.alloc<u64>(M);
    uint32_t* vals = sc.alloc<uint32_t>(M);
    uint32_t* vals_alt = sc.alloc<uint32_t>(M);
    if (!keys || !keys_alt || !vals || !vals_alt) return pc_from_cuda(sc.err);
    k_keys<<<grid_for(M, 256), 256, 0, s>>>(xyz, M, o[0], o[1], o[2], inv_h, bx, by, sub, keys, vals);
    PC_TRY(cudaGetLastError());
    PC_TRY(radix_sort(keys, vals, keys_alt, vals_alt, M, bx + by + bz + sub, sc, s));

    // 5. occupied cells
    uint32_t* flags = sc.alloc<uint32_t>(M);
    uint32_t* ord = sc.alloc<uint32_t>(M);
    uint32_t* total_dev = sc.alloc<uint32_t>(1);
    if (!flags || !ord || !total_dev) return pc_from_cuda(sc.err);
    k_flags<<<grid_for(M, 256), 256, 0, s>>>(keys, M, sub, flags);
    PC_TRY(scan_exclusive(flags, ord, M, total_dev, sc, s));
    uint32_t U = 0;
    PC_TRY(cudaMemcpyAsync(&U, total_dev, sizeof(U), cudaMemcpyDeviceToHost, s));
    PC_TRY(cudaStreamSynchronize(s));
    PC_TRY(cudaMalloc(&t->cell_keys, sizeof(u64) * std::max<uint32_t>(U, 1)));
    PC_TRY(cudaMalloc(&t->cell_start, sizeof(uint32_t) * ((size_t)U + 1)));
    k_cells<<<grid_for(M, 256), 256, 0, s>>>(keys, flags, ord, M, sub, t->cell_keys, t->cell_start, U);
    PC_TRY(cudaGetLastError());

    // 6. hash table
    const double load = (opts.hash_load > 0 && opts.hash_load <= 0.9) ? opts.hash_load : 0.5;
    int log2cap = 1;
    while ((double)(1ll << log2cap) * load < (double)U) ++log2cap;
    t->table_cap = 1ll << log2cap;
    PC_TRY(cudaMalloc(&t->table, sizeof(uint4) * (size_t)t->table_cap));
    PC_TRY(cudaMemsetAsync(t->table, 0xff, sizeof(uint4) * (size_t)t->table_cap, s));
    k_hash_insert<<<grid_for(U, 256), 256, 0, s>>>(t->cell_keys, t->cell_start, U, t->table,
                                                    log2cap);
    PC_TRY(cudaGetLastError());

    // 6b. row index: dense cell starts over the grid, built through an
    // occupancy bitmap and per-word ranks in scratch memory
    int64_t dense_words = 0;
    if (dense) {
        const int64_t nwords = (ngrid + 31) / 32;
        uint32_t* occ = sc.alloc<uint32_t>(nwords);
        uint32_t* rank = sc.alloc<uint32_t>(nwords);
        uint32_t* pop = sc.alloc<uint32_t>(nwords);
        uint32_t* tot2 = sc.alloc<uint32_t>(1);
        if (!occ || !rank || !pop || !tot2) return pc_from_cuda(sc.err);
        PC_TRY(cudaMemsetAsync(occ, 0, sizeof(uint32_t) * (size_t)nwords, s));
        k_occ_set<<<grid_for(U, 256), 256, 0, s>>>(t->cell_keys, U, bx, by, dims[0], dims[1], occ);
        k_popc<<<grid_for(nwords, 256), 256, 0, s>>>(occ, nwords, pop);
        PC_TRY(cudaGetLastError());
        PC_TRY(scan_exclusive(pop, rank, nwords, tot2, sc, s));
        PC_TRY(cudaMalloc(&t->dstart, sizeof(uint32_t) * (size_t)(ngrid + 1)));
        k_dstart<<<grid_for(ngrid + 1, 256), 256, 0, s>>>(occ, rank, t->cell_start, ngrid, U, t->dstart);
        PC_TRY(cudaGetLastError());
        dense_words = ngrid + 1;
        if (sub) {  // 6c. sub-cell cut
            PC_TRY(cudaMalloc(&t->xcut, sizeof(uint2) * (size_t)ngrid));
            PC_TRY(cudaMemsetAsync(t->xcut, 0, sizeof(uint2) * (size_t)ngrid, s));
            k_xcut<<<grid_for(M, 256), 256, 0, s>>>(keys, M, bx, by, dims[0], dims[1], t->dstart,
                                                      reinterpret_cast<unsigned char*>(t->xcut));
            PC_TRY(cudaGetLastError());
            dense_words += 2 * ngrid;
        }
    }

    // 7. float4 copies
    PC_TRY(cudaMalloc(&t->pts, sizeof(float4) * (size_t)M));
    PC_TRY(cudaMalloc(&t->xyz, sizeof(float4) * (size_t)M));
    k_gather<<<grid_for(M, 256), 256, 0, s>>>(xyz, vals, M, t->pts, t->xyz);
    PC_TRY(cudaGetLastError());
    PC_TRY(cudaStreamSynchronize(s));

    Grid& g = t->g;
    g.ox = o[0];
    g.oy = o[1];
    g.oz = o[2];
    g.h = h;
    g.inv_h = inv_h;
    g.dimx = dims[0];
    g.dimy = dims[1];
    g.dimz = dims[2];
    g.bx = bx;
    g.by = by;
    g.log2cap = log2cap;
    g.max_box_cells = opts.max_box_cells > 0 ? opts.max_box_cells : 4096;
    g.exhaustive = opts.exhaustive ? 1 : 0;
    g.coord_scale = scale;
    g.m = M;
    g.ncells = U;
    g.table = t->table;
    g.pts = t->pts;
    g.xyz = t->xyz;
    g.cell_keys = t->cell_keys;
    g.cell_start = t->cell_start;
    g.dstart = t->dstart;
    g.xcut = t->xcut;
    g.status = t->status;
    g.stats = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(t->status) + 32);
    pc_clear_window(g);
    t->device_bytes = (int64_t)(sizeof(uint4) * t->table_cap + 2 * sizeof(float4) * M +
                                sizeof(u64) * U + sizeof(uint32_t) * (U + 1) + 64 +
                                sizeof(uint32_t) * dense_words);
    return PC_OK;
}
