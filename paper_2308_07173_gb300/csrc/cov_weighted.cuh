// Kernel-descriptor weighted covariance of one neighbourhood (Sec. III-C1,
// Table I), shared by the single-grid pass (cov_weighted.cu) and the
// main + delta merge (delta.cu).  `get(j)` returns neighbour j in rank order.
#pragma once

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

}  // namespace
