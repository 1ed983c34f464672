// Neighbourhood covariance weighted by a kernel descriptor (Sec. III-C1:
// the covariance is computed "using the kernel descriptors" of Table I).
//
// For query x = q and its k neighbours y_j (rows of idx, in rank order):
//   w_j = K(x, y_j),  W = sum w_j,
//   mu = sum w_j y_j / W,  C = sum w_j (y_j - mu)(y_j - mu)^T / W,
// then, for eps >= 0, C' = I - (1 - eps) n n^T with n the smallest-eigenvalue
// eigenvector (the same Jacobi solver as the plain covariance).  Binary32,
// two passes shifted by the nearest neighbour y_0 like the plain form.  A
// row that failed its search (idx -1) or whose W is not positive and finite
// is NaN.  One thread per query; the neighbours come from the caller-order
// float4 copy of the target.
#include "cov_weighted.cuh"

namespace {

__device__ void weighted_row(const Grid& g, const CovKernel& ck, float qx, float qy, float qz,
                             const int32_t* __restrict__ nb, int k, float eps, float* out) {
    if (nb[0] < 0) {
        nan_row(out);
        return;
    }
    weighted_core([&](int j) { return __ldg(&g.xyz[nb[j]]); }, ck, qx, qy, qz, k, eps, out);
}

__global__ void k_cov_weighted(Grid g, CovKernel ck, const float* __restrict__ q,
                               const int32_t* __restrict__ idx, int64_t N, int k, float eps,
                               float* __restrict__ cov) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    weighted_row(g, ck, __ldg(q + 3 * n), __ldg(q + 3 * n + 1), __ldg(q + 3 * n + 2), idx + n * k, k, eps,
                 cov + 6 * n);
}

// Batched: blockIdx.y strides over the scans of the table, blockIdx.x over
// a scan's queries; scans without a covariance output are skipped.
__global__ void k_cov_weighted_batch(Grid g, CovKernel ck, const ScanDesc* __restrict__ scans,
                                     int nscans, int k, float eps) {
    for (int sidx = blockIdx.y; sidx < nscans; sidx += gridDim.y) {
        const ScanDesc sd = scans[sidx];
        if (sd.cov == nullptr) continue;
        for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < sd.n;
             n += (int64_t)gridDim.x * blockDim.x)
            weighted_row(g, ck, __ldg(sd.q + 3 * n), __ldg(sd.q + 3 * n + 1), __ldg(sd.q + 3 * n + 2),
                         sd.idx + n * k, k, eps, sd.cov + 6 * n);
    }
}

}  // namespace

cudaError_t pc_launch_cov_weighted(const Grid& g, const CovKernel& ck, const float* q,
                                   const int32_t* idx, int64_t N, int k, float eps, float* cov,
                                   cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int threads = 128;
    const int64_t blocks = (N + threads - 1) / threads;
    k_cov_weighted<<<(unsigned)blocks, threads, 0, s>>>(g, ck, q, idx, N, k, eps, cov);
    return cudaGetLastError();
}

cudaError_t pc_launch_cov_weighted_batch(const Grid& g, const CovKernel& ck, const ScanDesc* scans_dev,
                                         int nscans, int64_t max_n, int k, float eps, cudaStream_t s) {
    if (nscans < 1 || max_n < 1) return cudaSuccess;
    const int threads = 128;
    const int64_t bx = std::min<int64_t>((max_n + threads - 1) / threads, 65535);
    const int by = std::min(nscans, 65535);
    k_cov_weighted_batch<<<dim3((unsigned)bx, (unsigned)by), threads, 0, s>>>(g, ck, scans_dev, nscans, k,
                                                                            eps);
    return cudaGetLastError();
}
