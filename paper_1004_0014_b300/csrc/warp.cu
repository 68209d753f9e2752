// G1: fused DVF synthesis and trilinear warp (Eq. 1, Section 2.2).
//
// One thread handles two consecutive voxels of the flat grid. It reads the
// mean DVF (3 planes) and the K eigenvector fields (3K planes) with 8-byte
// vector loads (4-byte for bfloat16 storage), forms x = mean + sum_k u_k w_k,
// pulls back to q = v + x / spacing, and evaluates the zero-padded trilinear
// interpolant of f0 at q from the padded reference volume. On gradient points
// it also forms the exact derivative of the interpolant and h_k = (df/dx) . u_k
// with the eigenvector values already in registers. The pass is HBM-bound:
// 12 + 12K bytes of field reads per voxel (float32) against 4 bytes of f
// (+4K of h) written; the f0 taps hit L1/L2.
//
// For the padded outputs that only the projector reads, a chunk of 512
// voxels that all lie outside the support box of the warped volume at w (the
// displacement bound around the nonzero voxels of f0) gets its zeros written
// without any field read: the result is the same volume, and the field stream
// shrinks to the chunks that meet the box. Those modes run resident blocks
// that take the decisions for all their chunks at once, then stream.
//
// Two voxels per thread (not four) keep the registers at 48-51 for K <= 3,
// so five 256-thread blocks share an SM: the f0 taps wait on the pull-back
// point, and more resident warps hide that wait (measured 78 -> 64 us per
// paper-scale pass, K = 3).
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "internal.h"

namespace pr {
namespace {

constexpr int kWarpThreads = 256;
constexpr int kWarpVox = 2;                          // voxels per thread
constexpr int kWarpChunk = kWarpVox * kWarpThreads;  // voxels per block and step
constexpr int kWarpMaxChunks = 128;                  // chunks per block (support-restricted modes)

// The two consecutive values at p (8-byte aligned float32, 4-byte aligned
// bfloat16), as floats.
__device__ __forceinline__ void ld2(const float* p, float (&v)[2]) {
    float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x;
    v[1] = t.y;
}
__device__ __forceinline__ void ld2(const __nv_bfloat16* p, float (&v)[2]) {
    unsigned int t = __ldg(reinterpret_cast<const unsigned int*>(p));
    float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&t));
    v[0] = a.x;
    v[1] = a.y;
}

template <typename TS>
struct WarpArgs {
    const TS* f0p;
    const float* mean;
    const TS* U;
    const double* w;
    VolDev vd;
    float* out_pad;  // kWarpFH: interleaved (nch floats per voxel); kWarpFPad: planar
    float* f_flat;
    float* h_flat;
    const Support* sup;  // padded modes: skip the field reads outside the support box (nullable)
    const int* dirty;    // with sup: box of the blocks that may still hold nonzeros (nullable, see k_warp)
    int vec_ok;      // N % 2 == 0: planes are aligned for the two-voxel vector loads
};

// Whether any voxel of the flat range [vb, ve] lies in the inclusive box
// (lo x, y, z, hi x, y, z): the range's rows are tested one by one. 32-bit
// index arithmetic: a model's padded grid has fewer than 2^29 voxels.
__device__ __forceinline__ bool range_in_box(const VolDev& vd, int vb, int ve, const int* box) {
    const int nx = vd.nx, ny = vd.ny;
    const int r0 = vb / nx, r1 = ve / nx;
    int j = r0 % ny, kz = r0 / ny;
    for (int r = r0; r <= r1; ++r) {
        if (j >= box[1] && j <= box[4] && kz >= box[2] && kz <= box[5]) {
            const int row = r * nx;
            const int ia = max(vb, row) - row, ib = min(ve, row + nx - 1) - row;
            if (ib >= box[0] && ia <= box[3]) return true;
        }
        if (++j == ny) {
            j = 0;
            ++kz;
        }
    }
    return false;
}

// Whether the solver volume of this model type is the packed float32 f +
// float16 h record (bfloat16 storage, K = 4 or 5; see fh_layout).
template <int K, typename TS>
__host__ __device__ constexpr bool half_h() {
    return std::is_same<TS, __nv_bfloat16>::value && (K == 4 || K == 5);
}

__device__ __forceinline__ float pack_half2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return __uint_as_float(*reinterpret_cast<const unsigned int*>(&h));
}

// Zeros for the voxels v0, v0 + 1 (those below n) in the padded output layout.
template <int K, int MODE, typename TS>
__device__ __forceinline__ void zero_pair(const WarpArgs<TS>& A, long long v0) {
    constexpr int kNch = half_h<K, TS>() ? 4 : (K <= 3 ? 4 : (K <= 5 ? 6 : 8));
    const VolDev& vd = A.vd;
    const int jk = (int)v0 / vd.nx;
    int i = (int)v0 - jk * vd.nx, j = jk % vd.ny, kz = jk / vd.ny;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (v0 + e < vd.n) {
            const int pidx = ((kz + 1) * vd.nyp + (j + 1)) * vd.nxp + (i + 1);
            if (MODE == kWarpFH) {
                if (kNch == 6) {
                    reinterpret_cast<float4*>(A.out_pad)[pidx] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    reinterpret_cast<float2*>(A.out_pad + 4 * vd.np)[pidx] = make_float2(0.0f, 0.0f);
                } else {
                    float4* dst = reinterpret_cast<float4*>(A.out_pad + (long long)pidx * kNch);
#pragma unroll
                    for (int c4 = 0; c4 < kNch / 4; ++c4) dst[c4] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
            } else {
                A.out_pad[pidx] = 0.0f;
            }
        }
        if (++i == vd.nx) {
            i = 0;
            if (++j == vd.ny) {
                j = 0;
                ++kz;
            }
        }
    }
}

__device__ __forceinline__ float lerp(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

// DVF synthesis, pull-back warp and (kH) h_k for the two consecutive voxels
// v0, v0 + 1 whose mean (mx) and eigenvector (u) values are already in registers.
template <int K, int MODE, typename TS>
__device__ __forceinline__ void warp_pair(const WarpArgs<TS>& A, long long v0, const float (&w)[K],
                                      const float (&mx)[3][2], const float (&u)[K][3][2]) {
    constexpr bool kH = (MODE == kWarpFH || MODE == kWarpFlatFH);
    constexpr int kNch = K <= 3 ? 4 : (K <= 5 ? 6 : 8);
    const VolDev& vd = A.vd;
    const long long n = vd.n;
    // 32-bit index arithmetic: a model's padded grid has fewer than 2^29 voxels
    const int jk = (int)v0 / vd.nx;
    int i = (int)v0 - jk * vd.nx;
    int j = jk % vd.ny;
    int kz = jk / vd.ny;
    const int plane = vd.nxp * vd.nyp;

#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (v0 + e < n) {
            float d0 = mx[0][e], d1 = mx[1][e], d2 = mx[2][e];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                d0 = __fmaf_rn(u[k][0][e], w[k], d0);
                d1 = __fmaf_rn(u[k][1][e], w[k], d1);
                d2 = __fmaf_rn(u[k][2][e], w[k], d2);
            }
            // Pull-back point q = v + x / spacing, split as the integer voxel
            // index plus the small displacement: cell = v + floor(x/dx) and the
            // fraction x/dx - floor(x/dx) keep the displacement's precision
            // instead of that of the full index.
            float ux = d0 * vd.inv_dx, uy = d1 * vd.inv_dy, uz = d2 * vd.inv_dz;
            float fux = floorf(ux), fuy = floorf(uy), fuz = floorf(uz);
            float tx = ux - fux, ty = uy - fuy, tz = uz - fuz;
            float val = 0.0f;
            float gx = 0.0f, gy = 0.0f, gz = 0.0f;
            // inside the interpolant's support (-1, n) on every axis; the bounds on
            // fu keep the int conversion in range for any displacement
            const bool in_x = fux > -1.0e6f && fux < 1.0e6f, in_y = fuy > -1.0e6f && fuy < 1.0e6f,
                       in_z = fuz > -1.0e6f && fuz < 1.0e6f;
            int cx = in_x ? i + (int)fux : -2, cy = in_y ? j + (int)fuy : -2, cz = in_z ? kz + (int)fuz : -2;
            if ((cx > -1 || (cx == -1 && tx > 0.0f)) && cx < vd.nx && (cy > -1 || (cy == -1 && ty > 0.0f)) &&
                cy < vd.ny && (cz > -1 || (cz == -1 && tz > 0.0f)) && cz < vd.nz) {
                const int base = ((cz + 1) * vd.nyp + (cy + 1)) * vd.nxp + (cx + 1);
                const TS* c0 = A.f0p + base;
                float c000 = ld_val(c0), c100 = ld_val(c0 + 1);
                float c010 = ld_val(c0 + vd.nxp), c110 = ld_val(c0 + vd.nxp + 1);
                float c001 = ld_val(c0 + plane), c101 = ld_val(c0 + plane + 1);
                float c011 = ld_val(c0 + plane + vd.nxp), c111 = ld_val(c0 + plane + vd.nxp + 1);
                float x00 = lerp(c000, c100, tx), x10 = lerp(c010, c110, tx);
                float x01 = lerp(c001, c101, tx), x11 = lerp(c011, c111, tx);
                float y0 = lerp(x00, x10, ty), y1 = lerp(x01, x11, ty);
                val = lerp(y0, y1, tz);
                if (kH) {
                    float e00 = c100 - c000, e10 = c110 - c010, e01 = c101 - c001, e11 = c111 - c011;
                    gx = lerp(lerp(e00, e10, ty), lerp(e01, e11, ty), tz) * vd.inv_dx;
                    gy = lerp(x10 - x00, x11 - x01, tz) * vd.inv_dy;
                    gz = (y1 - y0) * vd.inv_dz;
                }
            }
            float h[K];
#pragma unroll
            for (int k = 0; k < K; ++k)
                h[k] = kH ? __fmaf_rn(gz, u[k][2][e], __fmaf_rn(gy, u[k][1][e], gx * u[k][0][e])) : 0.0f;

            const int pidx = ((kz + 1) * vd.nyp + (j + 1)) * vd.nxp + (i + 1);
            if (MODE == kWarpFH && half_h<K, TS>()) {
                reinterpret_cast<float4*>(A.out_pad)[pidx] =
                    make_float4(val, pack_half2(h[0], h[1 % K]), pack_half2(h[2 % K], h[3 % K]),
                                pack_half2(K == 5 ? h[4 % K] : 0.0f, 0.0f));
            } else if (MODE == kWarpFH) {
                float o[kNch];
                o[0] = val;
#pragma unroll
                for (int c = 1; c < kNch; ++c) o[c] = (c - 1 < K) ? h[c - 1 < K ? c - 1 : 0] : 0.0f;
                if (kNch == 6) {
                    reinterpret_cast<float4*>(A.out_pad)[pidx] = make_float4(o[0], o[1], o[2], o[3]);
                    reinterpret_cast<float2*>(A.out_pad + 4 * vd.np)[pidx] = make_float2(o[4], o[5 < kNch ? 5 : 0]);
                } else {
                    float4* dst = reinterpret_cast<float4*>(A.out_pad + (long long)pidx * kNch);
#pragma unroll
                    for (int c4 = 0; c4 < kNch / 4; ++c4)
                        dst[c4] = make_float4(o[4 * c4], o[4 * c4 + 1], o[4 * c4 + 2], o[4 * c4 + 3]);
                }
            } else if (MODE == kWarpFPad) {
                A.out_pad[pidx] = val;
            } else {
                if (A.f_flat) A.f_flat[v0 + e] = val;
                if (kH && A.h_flat)
#pragma unroll
                    for (int k = 0; k < K; ++k) A.h_flat[k * n + v0 + e] = h[k];
            }
        }
        // next voxel of the flat order
        if (++i == vd.nx) {
            i = 0;
            if (++j == vd.ny) {
                j = 0;
                ++kz;
            }
        }
    }
}

// Resident 256-thread blocks per SM the register cap aims at (measured on the
// paper-scale pass): K <= 3 five (four for bfloat16, whose conversions spill at
// five); K = 4, 5 three (for bfloat16, whose fields take half the registers,
// five at K = 4 and four at K = 5); K = 6, 7 two.
template <int K, typename TS>
constexpr int warp_min_blocks() {
    constexpr bool f32 = std::is_same<TS, float>::value;
    return K <= 3 ? (f32 ? 5 : 4) : (K <= 5 ? (f32 ? 3 : (K == 4 ? 5 : 4)) : 2);
}

// Fields of the two voxels v0, v0 + 1 (v0 < n), then the warp and h (warp_pair).
template <int K, int MODE, typename TS>
__device__ __forceinline__ void eval_pair(const WarpArgs<TS>& A, long long v0) {
    const long long n = A.vd.n;
    float w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = (float)A.w[k];

    // Fields of the two voxels: mean (3) and eigenvectors (3K).
    float mx[3][2];
    float u[K][3][2];
    const bool full = A.vec_ok && (v0 + 1 < n);
    if (full) {
#pragma unroll
        for (int c = 0; c < 3; ++c) ld2(A.mean + c * n + v0, mx[c]);
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) ld2(A.U + (3LL * k + c) * n + v0, u[k][c]);
    } else {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            long long v = v0 + e < n ? v0 + e : n - 1;
#pragma unroll
            for (int c = 0; c < 3; ++c) mx[c][e] = __ldg(A.mean + c * n + v);
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) u[k][c][e] = ld_val(A.U + (3LL * k + c) * n + v);
        }
    }
    warp_pair<K, MODE, TS>(A, v0, w, mx, u);
}

template <int K, int MODE, typename TS>
__global__ void __launch_bounds__(kWarpThreads, warp_min_blocks<K, TS>()) k_warp(WarpArgs<TS> A) {
    const VolDev& vd = A.vd;
    const long long n = vd.n;

    if ((MODE == kWarpFH || MODE == kWarpFPad) && A.sup) {
        // Resident blocks: block b takes the 512-voxel chunks b, b + G, ...
        // (G blocks). A chunk that meets the support box at w is evaluated; one
        // that does not writes zeros and reads no field, unless it also misses
        // the dirty box (A.dirty: every chunk that may still hold a nonzero
        // from an earlier pass meets it), so that it holds zeros already and
        // is left alone. The decisions of all of a block's chunks are taken
        // at its start, one thread per chunk, so a block waits for them once.
        __shared__ unsigned char action[kWarpMaxChunks];  // 0: already zero, 1: write zeros, 2: evaluate
        const long long nchunks = (n + kWarpChunk - 1) / kWarpChunk;
        const int mine = (int)((nchunks - blockIdx.x + gridDim.x - 1) / gridDim.x);
        if ((int)threadIdx.x < mine) {
            const long long chunk = blockIdx.x + (long long)threadIdx.x * gridDim.x;
            int old[6];
            if (A.dirty)
                for (int c = 0; c < 6; ++c) old[c] = __ldcg(A.dirty + c);
            int lo[3], hi[3];
            warp_box(A.sup, vd, A.w, K, lo, hi);
            const int box[6] = {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]};
            const int vb = (int)(chunk * kWarpChunk);
            const int ve = (int)(min((long long)vb + kWarpChunk, n) - 1);
            action[threadIdx.x] =
                range_in_box(vd, vb, ve, box) ? 2 : (!A.dirty || range_in_box(vd, vb, ve, old) ? 1 : 0);
        }
        __syncthreads();
        for (int i = 0; i < mine; ++i) {
            const long long v0 = (blockIdx.x + (long long)i * gridDim.x) * kWarpChunk + threadIdx.x * kWarpVox;
            const int act = action[i];
            if (v0 >= n || act == 0) continue;
            if (act == 2)
                eval_pair<K, MODE, TS>(A, v0);
            else
                zero_pair<K, MODE, TS>(A, v0);
        }
        return;
    }
    const long long v0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * kWarpVox;
    if (v0 >= n) return;
    eval_pair<K, MODE, TS>(A, v0);
}

__global__ void k_warp_box(VolDev vd, const double* __restrict__ w, int K, const Support* __restrict__ sup, int grow,
                           int* box) {
    int lo[3], hi[3];
    warp_box(sup, vd, w, K, lo, hi, grow);
    for (int c = 0; c < 3; ++c) box[c] = lo[c], box[3 + c] = hi[c];
}

// Blocks of k_warp<K, MODE, TS> resident on the current device at once
// (computed once per device; concurrent callers compute the same value).
template <int K, int MODE, typename TS>
int resident_blocks() {
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_warp<K, MODE, TS>, kWarpThreads, 0);
        v = sms * (per > 0 ? per : 1);
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <int K, typename TS>
cudaError_t dispatch_mode(Launcher& L, const ModelDev& m, const double* w, int mode, float* out_pad,
                          float* f_flat, float* h_flat, const Support* sup, const int* dirty) {
    WarpArgs<TS> A;
    A.f0p = static_cast<const TS*>(m.f0p);
    A.mean = m.mean;
    A.U = static_cast<const TS*>(m.U);
    A.w = w;
    A.vd = m.vd;
    A.out_pad = out_pad;
    A.f_flat = f_flat;
    A.h_flat = h_flat;
    A.sup = (mode == kWarpFH || mode == kWarpFPad) ? sup : nullptr;
    A.dirty = A.sup ? dirty : nullptr;
    A.vec_ok = (m.vd.n % kWarpVox == 0) ? 1 : 0;
    long long threads = (m.vd.n + kWarpVox - 1) / kWarpVox;
    dim3 grid((unsigned)((threads + kWarpThreads - 1) / kWarpThreads));
    if (A.sup) {  // resident blocks over the chunks (at most kWarpMaxChunks each)
        const long long nchunks = (m.vd.n + kWarpChunk - 1) / kWarpChunk;
        long long g = mode == kWarpFH ? resident_blocks<K, kWarpFH, TS>() : resident_blocks<K, kWarpFPad, TS>();
        if (g <= 0) return cudaErrorInvalidDevice;
        g = std::max(g, (nchunks + kWarpMaxChunks - 1) / kWarpMaxChunks);
        grid = dim3((unsigned)std::min(g, nchunks));
    }
    switch (mode) {
        case kWarpFH: return L(k_warp<K, kWarpFH, TS>, grid, dim3(kWarpThreads), 0, A);
        case kWarpFPad: return L(k_warp<K, kWarpFPad, TS>, grid, dim3(kWarpThreads), 0, A);
        case kWarpFlatF: return L(k_warp<K, kWarpFlatF, TS>, grid, dim3(kWarpThreads), 0, A);
        case kWarpFlatFH: return L(k_warp<K, kWarpFlatFH, TS>, grid, dim3(kWarpThreads), 0, A);
    }
    return cudaErrorInvalidValue;
}

template <typename TS>
cudaError_t dispatch_k(Launcher& L, const ModelDev& m, const double* w, int mode, float* out_pad,
                       float* f_flat, float* h_flat, const Support* sup, const int* dirty) {
    switch (m.K) {
        case 1: return dispatch_mode<1, TS>(L, m, w, mode, out_pad, f_flat, h_flat, sup, dirty);
        case 2: return dispatch_mode<2, TS>(L, m, w, mode, out_pad, f_flat, h_flat, sup, dirty);
        case 3: return dispatch_mode<3, TS>(L, m, w, mode, out_pad, f_flat, h_flat, sup, dirty);
        case 4: return dispatch_mode<4, TS>(L, m, w, mode, out_pad, f_flat, h_flat, sup, dirty);
        case 5: return dispatch_mode<5, TS>(L, m, w, mode, out_pad, f_flat, h_flat, sup, dirty);
        case 6: return dispatch_mode<6, TS>(L, m, w, mode, out_pad, f_flat, h_flat, sup, dirty);
        case 7: return dispatch_mode<7, TS>(L, m, w, mode, out_pad, f_flat, h_flat, sup, dirty);
    }
    return cudaErrorInvalidValue;
}

__global__ void __launch_bounds__(256) k_pad(VolDev vd, const float* __restrict__ src, float* __restrict__ dst) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= vd.n) return;
    long long jk = v / vd.nx;
    int i = (int)(v - jk * vd.nx), j = (int)(jk % vd.ny), k = (int)(jk / vd.ny);
    dst[((long long)(k + 1) * vd.nyp + (j + 1)) * vd.nxp + (i + 1)] = __ldg(src + v);
}

__global__ void __launch_bounds__(256) k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                                                 long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

}  // namespace

cudaError_t launch_to_bf16(Launcher& L, const float* src, __nv_bfloat16* dst, long long n) {
    dim3 grid((unsigned)((n + 255) / 256));
    return L(k_to_bf16, grid, dim3(256), 0, src, dst, n);
}

cudaError_t launch_warp(Launcher& L, const ModelDev& m, const double* w_dev, int mode, float* out_pad,
                        float* f_flat, float* h_flat, const Support* sup, const int* dirty) {
    if (m.storage == 1) return dispatch_k<__nv_bfloat16>(L, m, w_dev, mode, out_pad, f_flat, h_flat, sup, dirty);
    return dispatch_k<float>(L, m, w_dev, mode, out_pad, f_flat, h_flat, sup, dirty);
}

cudaError_t launch_warp_box(Launcher& L, const ModelDev& m, const double* w_dev, const Support* sup, int grow,
                            int* box_dev) {
    return L(k_warp_box, dim3(1), dim3(1), 0, m.vd, w_dev, m.K, sup, grow, box_dev);
}

cudaError_t launch_pad(Launcher& L, const VolDev& vd, const float* src, float* dst_pad) {
    dim3 grid((unsigned)((vd.n + 255) / 256));
    return L(k_pad, grid, dim3(256), 0, vd, src, dst_pad);
}

}  // namespace pr
