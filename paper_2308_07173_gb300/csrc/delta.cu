// pc_cov and packing over a map that grew by pc_target_append: the main
// grid (points 0 .. M-1) and the delta grid over the appended points
// (M .. M+Md-1).  The search itself, with its fused covariance, runs in the
// union kernels (knn_union.cu), which visit both grids in one pass; here
// each neighbour of a row is read from the grid that owns it, in rank order.
#include "knn_kernels.cuh"

namespace {

struct Src {
    const float4* main_xyz;
    const float4* delta_xyz;
    int64_t m;
    __device__ __forceinline__ float4 at(int32_t gi) const {
        return gi < m ? __ldg(&main_xyz[gi]) : __ldg(&delta_xyz[gi - m]);
    }
};

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

}  // namespace

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
