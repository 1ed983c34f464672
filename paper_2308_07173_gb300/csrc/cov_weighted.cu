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
#include "knn_kernels.cuh"

namespace {

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

__device__ void weighted_row(const Grid& g, const CovKernel& ck, float qx, float qy, float qz,
                             const int32_t* __restrict__ nb, int k, float eps, float* out) {
    if (nb[0] < 0 || !isfinite(qx) || !isfinite(qy) || !isfinite(qz)) {
        nan_row(out);
        return;
    }
    const float4 p0 = __ldg(&g.xyz[nb[0]]);
    float W = 0.0f, sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int j = 0; j < k; ++j) {
        const float4 p = __ldg(&g.xyz[nb[j]]);
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
        const float4 p = __ldg(&g.xyz[nb[j]]);
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
