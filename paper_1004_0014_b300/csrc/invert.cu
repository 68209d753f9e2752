// Whole-grid inversion of the pull-back DVF (Section 2.3 with ref. 13).
//
// The push-forward field y satisfies u + y(u) + x(u + y(u)) = u at every voxel
// centre u, where x = mean + sum_k u_k w_k is interpolated trilinearly and
// clamped to the grid edge. Chen et al.'s fixed point y <- -x(u + y) updates
// each voxel from its own previous value only, so the sweeps of the whole
// field collapse into one pass in which every thread iterates its voxel to
// convergence: the field is read from L1/L2 around the voxel instead of being
// streamed through HBM once per sweep.
//
// Two kernels:
//   k_dvf_idx  x = mean + U w in voxel units (x/dx, y/dy, z/dz, 0), one
//              float4 per voxel: HBM-bound, 12 + 12K bytes read (float32
//              storage) and 16 written per voxel;
//   k_invert   the per-voxel fixed point on that field: 8 float4 taps per
//              step, then 12 bytes of y (mm) written per voxel.
// Iterates are kept as displacements in voxel units (cell = u + floor(d),
// fraction = d - floor(d)), so their precision is that of the displacement,
// not of the absolute index.
#include "internal.h"

namespace pr {
namespace {

constexpr int kInvThreads = 256;

template <int K, typename TS>
__global__ void __launch_bounds__(kInvThreads) k_dvf_idx(const float* __restrict__ mean, const TS* __restrict__ U,
                                                         const double* __restrict__ w_dev, VolDev vd, int vec_ok,
                                                         float4* __restrict__ X) {
    const long long n = vd.n;
    const long long v0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 4;
    if (v0 >= n) return;
    float w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = (float)w_dev[k];
    float d[3][4];
    const bool full = vec_ok && v0 + 3 < n;
    if (full) {
#pragma unroll
        for (int c = 0; c < 3; ++c) ld4(mean + c * n + v0, d[c]);
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float u[4];
                ld4(U + (3LL * k + c) * n + v0, u);
#pragma unroll
                for (int e = 0; e < 4; ++e) d[c][e] = __fmaf_rn(u[e], w[k], d[c][e]);
            }
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long v = v0 + e < n ? v0 + e : n - 1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float x = __ldg(mean + c * n + v);
#pragma unroll
                for (int k = 0; k < K; ++k) x = __fmaf_rn(ld_val(U + (3LL * k + c) * n + v), w[k], x);
                d[c][e] = x;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (v0 + e < n) X[v0 + e] = make_float4(d[0][e] * vd.inv_dx, d[1][e] * vd.inv_dy, d[2][e] * vd.inv_dz, 0.0f);
}

// Cell and fraction on one axis of the point u + d (voxel units), clamped to
// the grid edge: a point below 0 uses cell 0 with fraction 0, a point at or
// above n - 1 uses cell n - 2 with fraction 1 (cell 0, fraction 0 when n = 1).
__device__ __forceinline__ int edge_cell(int u, float d, int n, float& t) {
    const float fl = floorf(d);
    t = d - fl;
    const int c = u + (int)fminf(fmaxf(fl, -1.0e6f), 1.0e6f);
    if (c < 0) {
        t = 0.0f;
        return 0;
    }
    if (c >= n - 1) {
        t = n > 1 ? 1.0f : 0.0f;
        return max(n - 2, 0);
    }
    return c;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

__global__ void __launch_bounds__(kInvThreads) k_invert(const float4* __restrict__ X, VolDev vd, float tol2,
                                                        int max_iter, float* __restrict__ y,
                                                        unsigned int* __restrict__ stats) {
    const int n = (int)vd.n;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    int steps = 0;
    bool converged = true;
    if (v < n) {
        const int jk = v / vd.nx;
        const int i = v - jk * vd.nx, j = jk % vd.ny, k = jk / vd.ny;
        const float sp[3] = {vd.dx, vd.dy, vd.dz};
        // first sweep from y = 0: x at the node itself
        const float4 x0 = __ldg(X + v);
        float d[3] = {-x0.x, -x0.y, -x0.z};
        float s2 = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) s2 = __fmaf_rn(d[c] * sp[c], d[c] * sp[c], s2);
        steps = 1;
        converged = s2 < tol2;
        while (!converged && steps < max_iter) {
            float tx, ty, tz;
            const int cx = edge_cell(i, d[0], vd.nx, tx), cy = edge_cell(j, d[1], vd.ny, ty),
                      cz = edge_cell(k, d[2], vd.nz, tz);
            const int cx1 = min(cx + 1, vd.nx - 1), cy1 = min(cy + 1, vd.ny - 1), cz1 = min(cz + 1, vd.nz - 1);
            const int r00 = (cz * vd.ny + cy) * vd.nx, r10 = (cz * vd.ny + cy1) * vd.nx;
            const int r01 = (cz1 * vd.ny + cy) * vd.nx, r11 = (cz1 * vd.ny + cy1) * vd.nx;
            const float4 a000 = __ldg(X + r00 + cx), a100 = __ldg(X + r00 + cx1);
            const float4 a010 = __ldg(X + r10 + cx), a110 = __ldg(X + r10 + cx1);
            const float4 a001 = __ldg(X + r01 + cx), a101 = __ldg(X + r01 + cx1);
            const float4 a011 = __ldg(X + r11 + cx), a111 = __ldg(X + r11 + cx1);
            float xi[3];
            xi[0] = lerpf(lerpf(lerpf(a000.x, a100.x, tx), lerpf(a010.x, a110.x, tx), ty),
                          lerpf(lerpf(a001.x, a101.x, tx), lerpf(a011.x, a111.x, tx), ty), tz);
            xi[1] = lerpf(lerpf(lerpf(a000.y, a100.y, tx), lerpf(a010.y, a110.y, tx), ty),
                          lerpf(lerpf(a001.y, a101.y, tx), lerpf(a011.y, a111.y, tx), ty), tz);
            xi[2] = lerpf(lerpf(lerpf(a000.z, a100.z, tx), lerpf(a010.z, a110.z, tx), ty),
                          lerpf(lerpf(a001.z, a101.z, tx), lerpf(a011.z, a111.z, tx), ty), tz);
            s2 = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float step = (-xi[c] - d[c]) * sp[c];
                s2 = __fmaf_rn(step, step, s2);
                d[c] = -xi[c];
            }
            ++steps;
            converged = s2 < tol2;
        }
        y[v] = d[0] * vd.dx;
        y[n + v] = d[1] * vd.dy;
        y[2LL * n + v] = d[2] * vd.dz;
    }
    // deterministic statistics: the largest step count and the number of
    // voxels whose last update was not below tol
    int m = steps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const unsigned int open = __popc(__ballot_sync(0xffffffffu, v < n && !converged));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(stats, (unsigned int)m);
        if (open) atomicAdd(stats + 1, open);
    }
}

template <typename TS>
cudaError_t dvf_idx_k(Launcher& L, const ModelDev& m, const TS* U, const double* w_dev, float4* X) {
    const long long threads = (m.vd.n + 3) / 4;
    const dim3 grid((unsigned)((threads + kInvThreads - 1) / kInvThreads));
    const int vec_ok = m.vd.n % 4 == 0;
    switch (m.K) {
        case 1: return L(k_dvf_idx<1, TS>, grid, dim3(kInvThreads), 0, m.mean, U, w_dev, m.vd, vec_ok, X);
        case 2: return L(k_dvf_idx<2, TS>, grid, dim3(kInvThreads), 0, m.mean, U, w_dev, m.vd, vec_ok, X);
        case 3: return L(k_dvf_idx<3, TS>, grid, dim3(kInvThreads), 0, m.mean, U, w_dev, m.vd, vec_ok, X);
        case 4: return L(k_dvf_idx<4, TS>, grid, dim3(kInvThreads), 0, m.mean, U, w_dev, m.vd, vec_ok, X);
        case 5: return L(k_dvf_idx<5, TS>, grid, dim3(kInvThreads), 0, m.mean, U, w_dev, m.vd, vec_ok, X);
        case 6: return L(k_dvf_idx<6, TS>, grid, dim3(kInvThreads), 0, m.mean, U, w_dev, m.vd, vec_ok, X);
        case 7: return L(k_dvf_idx<7, TS>, grid, dim3(kInvThreads), 0, m.mean, U, w_dev, m.vd, vec_ok, X);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_invert(Launcher& L, const ModelDev& m, const double* w_dev, float4* X, double tol, int max_iter,
                          float* y, unsigned int* stats) {
    if (m.vd.n <= 0 || m.vd.n >= 0x7fffffffLL || max_iter < 1) return cudaErrorInvalidValue;
    cudaError_t e = m.storage == 1
                        ? dvf_idx_k(L, m, static_cast<const __nv_bfloat16*>(m.U), w_dev, X)
                        : dvf_idx_k(L, m, static_cast<const float*>(m.U), w_dev, X);
    if (e != cudaSuccess) return e;
    const float tol2 = (float)(tol * tol);
    const dim3 grid((unsigned)((m.vd.n + kInvThreads - 1) / kInvThreads));
    return L(k_invert, grid, dim3(kInvThreads), 0, X, m.vd, tol2, max_iter, y, stats);
}

}  // namespace pr
