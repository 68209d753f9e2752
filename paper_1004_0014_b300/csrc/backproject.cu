// G3: the transpose P^T of the projector by a voxel-driven gather (no atomics).
//
// P's samples are anchored at the source, so the samples that touch voxel v
// (those within one voxel of it on every axis, where its trilinear hat weight
// is nonzero) can be listed from v alone: project the corners of v's support
// box onto the detector, visit every pixel of that footprint, intersect the
// pixel's ray with the box, and enumerate the samples inside. Each sample
// uses the projector's own ray_dir_index / sample_pos, so both operators see
// the same points and the pair is an exact transpose up to FP32 summation
// order.
//
// With h given, the per-voxel value g(v) = (P^T r)(v) is contracted with
// h_k(v) on the fly (the gradient formula after Eq. 4: dJ/dw_k = 2 sum_v
// g(v) h_k(v), or the vector-Jacobian product without the 2) and g is never
// stored; block partials are reduced in FP64 in a fixed order.
#include "internal.h"

namespace pr {
namespace {

constexpr int kBpThreads = 128;

__device__ __forceinline__ void footprint(const RayGeom& g, float px, float py, float pz, float& umin,
                                          float& umax, float& vmin, float& vmax) {
    float rx = px - g.src[0], ry = py - g.src[1], rz = pz - g.src[2];
    float depth = rx * g.ehat[0] + ry * g.ehat[1] + rz * g.ehat[2];
    float lam = g.sdd / depth;
    float u = lam * (rx * g.pu[0] + ry * g.pu[1] + rz * g.pu[2]) + g.cu;
    float v = lam * (rx * g.pv[0] + ry * g.pv[1] + rz * g.pv[2]) + g.cv;
    umin = fminf(umin, u);
    umax = fmaxf(umax, u);
    vmin = fminf(vmin, v);
    vmax = fmaxf(vmax, v);
}

template <int K>
__global__ void __launch_bounds__(kBpThreads)
k_backproject(const RayGeom* __restrict__ rgp, VolDev vd, const float* __restrict__ r, float* __restrict__ g_out,
              const float* __restrict__ h, double* partials, unsigned int* counter, double* out) {
    const RayGeom g = *rgp;
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float acc = 0.0f;
    if (v < vd.n) {
        long long jk = v / vd.nx;
        int i = (int)(v - jk * vd.nx), j = (int)(jk % vd.ny), k = (int)(jk / vd.ny);
        // Support box of voxel v in world coordinates and its detector footprint.
        float cx = g.origin[0] + i * g.sp[0], cy = g.origin[1] + j * g.sp[1], cz = g.origin[2] + k * g.sp[2];
        float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            footprint(g, cx + ((c & 1) ? g.sp[0] : -g.sp[0]), cy + ((c & 2) ? g.sp[1] : -g.sp[1]),
                      cz + ((c & 4) ? g.sp[2] : -g.sp[2]), umin, umax, vmin, vmax);
        umin = fmaxf(umin, -1.0f);
        vmin = fmaxf(vmin, -1.0f);
        umax = fminf(umax, (float)g.nu);
        vmax = fminf(vmax, (float)g.nv);
        int u0 = max(0, (int)ceilf(umin)), u1 = min(g.nu - 1, (int)floorf(umax));
        int w0 = max(0, (int)ceilf(vmin)), w1 = min(g.nv - 1, (int)floorf(vmax));
        const float lo[3] = {(float)(i - 1), (float)(j - 1), (float)(k - 1)};
        const float hi[3] = {(float)(i + 1), (float)(j + 1), (float)(k + 1)};
        const float fi = (float)i, fj = (float)j, fk = (float)k;
        for (int iv = w0; iv <= w1; ++iv) {
            for (int iu = u0; iu <= u1; ++iu) {
                float b[3], t0, t1;
                ray_dir_index(g, iu, iv, b);
                if (!ray_box(g.a, b, lo, hi, t0, t1)) continue;
                int s0 = (int)fminf(fmaxf(ceilf(t0 / g.ds - 0.5f), 0.0f), 1.0e7f);
                int s1 = (int)fminf(floorf(t1 / g.ds - 0.5f), 1.0e7f);
                float wsum = 0.0f;
                for (int s = s0; s <= s1; ++s) {
                    float q[3];
                    sample_pos(g, b, s, q);
                    float wx = 1.0f - fabsf(q[0] - fi), wy = 1.0f - fabsf(q[1] - fj), wz = 1.0f - fabsf(q[2] - fk);
                    if (wx > 0.0f && wy > 0.0f && wz > 0.0f) wsum = __fmaf_rn(wx * wy, wz, wsum);
                }
                acc = __fmaf_rn(wsum, __ldg(r + (long long)iv * g.nu + iu), acc);
            }
        }
        acc *= g.ds;
        if (g_out) g_out[v] = acc;
    }
    if constexpr (K > 0) {
        double d[K];
#pragma unroll
        for (int m = 0; m < K; ++m) d[m] = 0.0;
        if (v < vd.n)
#pragma unroll
            for (int m = 0; m < K; ++m) d[m] = (double)acc * (double)__ldg(h + m * vd.n + v);
        block_sum<K>(d);
        if (!publish_partials<K>(d, partials, blockIdx.x, gridDim.x, counter)) return;
        double tot[K];
        total_partials<K>(partials, gridDim.x, tot);
        if (threadIdx.x == 0) {
            *counter = 0;
            for (int m = 0; m < K; ++m) out[m] = tot[m];
        }
    }
}

}  // namespace

int backproject_blocks(const VolDev& vd) { return (int)((vd.n + kBpThreads - 1) / kBpThreads); }

cudaError_t launch_backproject(Launcher& L, const VolDev& vd, const RayGeom* rg, const float* r, float* g_flat,
                               const float* h, int K, double* partials, unsigned int* counter, double* out) {
    dim3 grid((unsigned)backproject_blocks(vd));
    dim3 block(kBpThreads);
    if (!h) K = 0;
    switch (K) {
        case 0: return L(k_backproject<0>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
        case 1: return L(k_backproject<1>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
        case 2: return L(k_backproject<2>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
        case 3: return L(k_backproject<3>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
        case 4: return L(k_backproject<4>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
        case 5: return L(k_backproject<5>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
        case 6: return L(k_backproject<6>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
        case 7: return L(k_backproject<7>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pr
