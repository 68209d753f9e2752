// G3: the transpose P^T of the projector by a voxel-driven gather (no atomics).
//
// P's samples are anchored at the source, so the samples that touch voxel v
// (those within one voxel of it on every axis, where its trilinear hat weight
// is nonzero) can be listed from v alone: project the corners of v's support
// box onto the detector, visit every pixel of that footprint, intersect the
// pixel's ray with the box, and enumerate the samples inside. Each sample
// uses the projector's own ray_dir_index / ray_lattice, so both operators see
// the same points and the pair is an exact transpose up to FP32 summation
// order.
//
// With h given, the per-voxel value g(v) = (P^T r)(v) is contracted with
// h_k(v) on the fly (the gradient formula after Eq. 4: dJ/dw_k = 2 sum_v
// g(v) h_k(v), or the vector-Jacobian product without the 2) and g is never
// stored; block partials are reduced in FP64 in a fixed order.
//
// Fixed gantry angle (Section 5: fluoroscopy keeps P the same for every
// frame): the weight of each footprint pixel, sum over its samples of the
// hat product, depends on the geometry alone. A table of these weights
// (footprint rectangle per voxel, weights slot-major: slot s of voxel v at
// s * N + v, so a warp reads consecutive voxels) is built once per angle;
// with it the transpose is a gather of stored weights against r, in the same
// pixel order and with the same multiply-adds as the on-the-fly form, so the
// two give bitwise-equal results.
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

// Footprint rectangle [u0, u1] x [w0, w1] of voxel (i, j, k): the detector
// pixels whose rays can cross the voxel's support box (v - spacing, v + spacing).
__device__ __forceinline__ void voxel_footprint(const RayGeom& g, int i, int j, int k, int& u0, int& u1, int& w0,
                                                int& w1) {
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
    u0 = max(0, (int)ceilf(umin)), u1 = min(g.nu - 1, (int)floorf(umax));
    w0 = max(0, (int)ceilf(vmin)), w1 = min(g.nv - 1, (int)floorf(vmax));
}

// Weight of pixel (iu, iv) for voxel (i, j, k): the sum over the ray's samples
// inside the voxel's support of the trilinear hat product (0 if it misses).
__device__ __forceinline__ float pixel_weight(const RayGeom& g, int i, int j, int k, int iu, int iv) {
    const float lo[3] = {(float)(i - 1), (float)(j - 1), (float)(k - 1)};
    const float hi[3] = {(float)(i + 1), (float)(j + 1), (float)(k + 1)};
    // voxel centres in the lattice's cell-origin coordinates (q - 1/2): the
    // hat weights 1 - |q - i| below are then formed exactly as the
    // projector's corner weights, from the same lattice values
    const float fi = (float)i - 0.5f, fj = (float)j - 0.5f, fk = (float)k - 0.5f;
    float b[3], t0, t1;
    ray_dir_index(g, iu, iv, b);
    if (!ray_box(g.a, b, lo, hi, t0, t1)) return 0.0f;
    int s0 = (int)fminf(fmaxf(ceilf(t0 / g.ds - 0.5f), 0.0f), 1.0e7f);
    int s1 = (int)fminf(floorf(t1 / g.ds - 0.5f), 1.0e7f);
    RayLattice L;
    ray_lattice(g, b, L);
    float wsum = 0.0f;
    for (int s = s0; s <= s1; ++s) {
        float q[3];
        lattice_point(L, (float)s, q);
        float wx = 1.0f - fabsf(q[0] - fi), wy = 1.0f - fabsf(q[1] - fj), wz = 1.0f - fabsf(q[2] - fk);
        if (wx > 0.0f && wy > 0.0f && wz > 0.0f) wsum = __fmaf_rn(wx * wy, wz, wsum);
    }
    return wsum;
}

template <int K>
__global__ void __launch_bounds__(kBpThreads)
k_backproject(const RayGeom* __restrict__ rgp, VolDev vd, const float* __restrict__ r, float* __restrict__ g_out,
              const float* __restrict__ h, double* partials, unsigned int* counter, double* out, BpTable tab) {
    const RayGeom g = *rgp;
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float acc = 0.0f;
    // Contracted with h and not stored: a voxel whose h_k are all zero (air,
    // away from the warped image's edges) adds nothing, so its footprint is
    // not visited.
    bool needed = v < vd.n;
    if constexpr (K > 0) {
        if (needed && !g_out) {
            bool any = false;
#pragma unroll
            for (int m = 0; m < K; ++m) any = any || __ldg(h + m * vd.n + v) != 0.0f;
            needed = any;
        }
    }
    if (needed) {
        long long jk = v / vd.nx;
        int i = (int)(v - jk * vd.nx), j = (int)(jk % vd.ny), k = (int)(jk / vd.ny);
        if (tab.w) {  // fixed angle: stored weights, same pixel order and multiply-adds
            const short4 fp = __ldg(tab.rect + v);
            int slot = 0;
            for (int iv = fp.y; iv < fp.y + fp.w; ++iv)
                for (int iu = fp.x; iu < fp.x + fp.z; ++iu, ++slot)
                    acc = __fmaf_rn(__ldg(tab.w + (long long)slot * vd.n + v), __ldg(r + (long long)iv * g.nu + iu),
                                    acc);
        } else {
            int u0, u1, w0, w1;
            voxel_footprint(g, i, j, k, u0, u1, w0, w1);
            for (int iv = w0; iv <= w1; ++iv)
                for (int iu = u0; iu <= u1; ++iu)
                    acc = __fmaf_rn(pixel_weight(g, i, j, k, iu, iv), __ldg(r + (long long)iv * g.nu + iu), acc);
        }
        acc *= g.ds;
    }
    if (g_out && v < vd.n) g_out[v] = acc;
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

// Fixed-angle table, pass 1: each voxel's footprint rectangle, and the largest
// footprint (slots) over the grid.
__global__ void __launch_bounds__(kBpThreads) k_bp_rect(const RayGeom* __restrict__ rgp, VolDev vd, short4* rect,
                                                         unsigned int* max_slots) {
    const RayGeom g = *rgp;
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned int sz = 0;
    if (v < vd.n) {
        long long jk = v / vd.nx;
        int i = (int)(v - jk * vd.nx), j = (int)(jk % vd.ny), k = (int)(jk / vd.ny);
        int u0, u1, w0, w1;
        voxel_footprint(g, i, j, k, u0, u1, w0, w1);
        const int nu = max(0, u1 - u0 + 1), nv = max(0, w1 - w0 + 1);
        rect[v] = make_short4((short)u0, (short)w0, (short)nu, (short)nv);
        sz = (unsigned int)(nu * nv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sz = max(sz, __shfl_xor_sync(0xffffffffu, sz, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_slots, sz);
}

// Pass 2: the weights, slot-major.
__global__ void __launch_bounds__(kBpThreads) k_bp_fill(const RayGeom* __restrict__ rgp, VolDev vd,
                                                         const short4* __restrict__ rect, float* w) {
    const RayGeom g = *rgp;
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= vd.n) return;
    long long jk = v / vd.nx;
    int i = (int)(v - jk * vd.nx), j = (int)(jk % vd.ny), k = (int)(jk / vd.ny);
    const short4 fp = rect[v];
    int slot = 0;
    for (int iv = fp.y; iv < fp.y + fp.w; ++iv)
        for (int iu = fp.x; iu < fp.x + fp.z; ++iu, ++slot) w[(long long)slot * vd.n + v] = pixel_weight(g, i, j, k, iu, iv);
}

}  // namespace

cudaError_t launch_bp_rect(Launcher& L, const VolDev& vd, const RayGeom* rg, short4* rect, unsigned int* max_slots) {
    return L(k_bp_rect, dim3((unsigned)((vd.n + kBpThreads - 1) / kBpThreads)), dim3(kBpThreads), 0, rg, vd, rect,
             max_slots);
}

cudaError_t launch_bp_fill(Launcher& L, const VolDev& vd, const RayGeom* rg, const short4* rect, float* w) {
    return L(k_bp_fill, dim3((unsigned)((vd.n + kBpThreads - 1) / kBpThreads)), dim3(kBpThreads), 0, rg, vd, rect, w);
}

int backproject_blocks(const VolDev& vd) { return (int)((vd.n + kBpThreads - 1) / kBpThreads); }

cudaError_t launch_backproject(Launcher& L, const VolDev& vd, const RayGeom* rg, const float* r, float* g_flat,
                               const float* h, int K, double* partials, unsigned int* counter, double* out,
                               BpTable tab) {
    dim3 grid((unsigned)backproject_blocks(vd));
    dim3 block(kBpThreads);
    if (!h) K = 0;
    switch (K) {
        case 0: return L(k_backproject<0>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
        case 1: return L(k_backproject<1>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
        case 2: return L(k_backproject<2>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
        case 3: return L(k_backproject<3>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
        case 4: return L(k_backproject<4>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
        case 5: return L(k_backproject<5>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
        case 6: return L(k_backproject<6>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
        case 7: return L(k_backproject<7>, grid, block, 0, rg, vd, r, g_flat, h, partials, counter, out, tab);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pr
