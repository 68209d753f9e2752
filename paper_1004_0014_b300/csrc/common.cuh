// Shared device-side definitions of the pcarecon CUDA library: grid and ray
// geometry, the on-device solver state, sample-position arithmetic shared by
// the projector and its gather transpose, deterministic block reductions and
// a launcher that either launches on a stream or records a CUDA-graph node.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace pr {

constexpr int kMaxK = 7;
constexpr int kMaxMom = 12;  // doubles per block partial row of the reductions
constexpr int kProjMom = 24; // doubles per block partial row of the projector's moments (3 + 3 x 7)

// Voxel grid of a model. Device volumes are stored with a one-voxel zero border
// ("padded"): element (i, j, k), -1 <= i <= nx, sits at
// ((k + 1) * nyp + (j + 1)) * nxp + (i + 1), so every trilinear tap of a point
// clamped into the index box [-1, n] is in bounds and the border supplies the
// zero value of the interpolant outside the grid.
struct VolDev {
    int nx, ny, nz;
    int nxp, nyp, nzp;  // n + 2
    float dx, dy, dz;
    float inv_dx, inv_dy, inv_dz;
    long long n;   // voxels
    long long np;  // padded voxels
};

// Ray geometry of one gantry angle, in float. Directions are built per pixel as
// d00 + iu * eu + iv * ev (world mm, from the source to the pixel centre),
// normalised, then scaled to index units by inv_sp; `a` is the source in
// index coordinates ((S - origin) / spacing).
struct RayGeom {
    float a[3];
    float d00[3];
    float eu[3];
    float ev[3];
    float inv_sp[3];
    float nmax[3];  // nx, ny, nz as float: the interpolant's support is (-1, n)
    float ds;       // sample step, mm
    int nu, nv;
    // For voxel footprints (gather transpose): a world point P lands on the
    // continuous pixel coordinate (lam (P - S).pu + cu, lam (P - S).pv + cv) with
    // lam = sdd / ((P - S).ehat).
    float src[3];     // source, world mm
    float ehat[3];    // unit central-ray direction
    float pu[3], pv[3];  // eu / |eu|^2, ev / |ev|^2
    float cu, cv;     // (nu - 1) / 2, (nv - 1) / 2
    float sdd;
    float origin[3];  // world position of voxel (0, 0, 0)
    float sp[3];      // voxel spacing, mm
    int tile_u;       // detector columns of the split projector's warp tile: 4 (4 x 8) or 2 (2 x 16)
};

// Where a model's warped volume can be nonzero (computed once at load). The
// warped f and h at voxel v are nonzero only if the pull-back point v + x(v)
// lies within one cell of a nonzero voxel of f0, so |v_c - u_c| < 1 + |x_c|/dx_c
// for some nonzero f0 voxel u, and |x_c| <= max|mean_c| + sum_k |w_k| max|u_kc|.
// A ray sample can be nonzero only one cell further out. Samples outside that
// box are exact zeros, so clipping rays to it changes no sum.
struct Support {
    int lo[3], hi[3];                  // index box of the nonzero f0 voxels (lo > hi: f0 == 0)
    unsigned int mean_max[3];          // bits of max |mean_c| (non-negative floats order as uints)
    unsigned int u_max[kMaxK][3];      // bits of max |u_kc|
};

// Sample box (index space) of a ray march over the warped volume at
// coefficients w; returns false when the volume is zero everywhere.
// margin (nullable) receives the largest per-axis reach 2 + d_c (voxels): a
// sample whose cell is farther than that from every nonzero f0 voxel is 0.
__device__ __forceinline__ bool support_box(const Support& s, const VolDev& vd, const double* w, int K,
                                            float lo[3], float hi[3], float* margin = nullptr) {
    const float inv[3] = {vd.inv_dx, vd.inv_dy, vd.inv_dz};
    const float n[3] = {(float)vd.nx, (float)vd.ny, (float)vd.nz};
    bool any = true;
    float reach = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float d = __uint_as_float(s.mean_max[c]);
        for (int k = 0; k < K; ++k) d += (float)fabs(w[k]) * __uint_as_float(s.u_max[k][c]);
        d = d * inv[c] * 1.01f + 0.01f;  // margin for float rounding of x and of the bounds
        lo[c] = fmaxf(-1.0f, (float)s.lo[c] - 2.0f - d);
        hi[c] = fminf(n[c], (float)s.hi[c] + 2.0f + d);
        reach = fmaxf(reach, 2.0f + d);
        any = any && (s.lo[c] <= s.hi[c]) && (lo[c] < hi[c]);
    }
    if (margin) *margin = reach;
    return any;
}

// Voxel box that may hold nonzero f or h at coefficients w. The pull-back
// point of voxel v lies within |x_c| / dx_c <= d_c voxels of v, and f, h are
// nonzero only where it is less than one cell from a nonzero f0 voxel, i.e.
// for v_c in (lo_c - 1 - d_c, hi_c + 1 + d_c). support_box returns the
// projector's sample box, one voxel wider on each side; that box, rounded
// outward and widened by `grow` voxels, is returned, so every voxel outside it
// is an exact zero. Without a support record: the whole grid.
__device__ __forceinline__ void warp_box(const Support* sup, const VolDev& vd, const double* w, int K, int lo[3],
                                         int hi[3], int grow = 0) {
    const int n[3] = {vd.nx, vd.ny, vd.nz};
    if (!sup) {
        for (int c = 0; c < 3; ++c) lo[c] = 0, hi[c] = n[c] - 1;
        return;
    }
    float flo[3], fhi[3];
    const bool any = support_box(*sup, vd, w, K, flo, fhi);
    for (int c = 0; c < 3; ++c) {
        // flo, fhi lie in [-1, n] (NaN coefficients give the whole grid)
        lo[c] = any ? max((int)floorf(flo[c]) - grow, 0) : 1;
        hi[c] = any ? min((int)ceilf(fhi[c]) + grow, n[c] - 1) : 0;
    }
}

// Solver phases handled by the controller in the last block of a reduction.
enum Phase : int {
    kPhaseNone = 0,   // plain projection, no reduction
    kPhaseInit = 1,   // first projection at w0: (a, b) by Eq. 4
    kPhaseTrial = 2,  // line-search trial: Armijo test, then Eq. 4 on acceptance
};

// Per-solve parameters (written by the host before each solve).
struct SolveParams {
    RayGeom rg;
    double w0[8];
    double c1, beta, grad_tol, step0, tumor_tol, step_growth, step_growth_bt;
    int max_iters, max_bt, tumor_max_iter, K;
    int cold_start;  // 1: start from w0; 0: from the state's last accepted w
    int warm_step;   // 1: a warm start also takes the state's next step
    int predict;     // 1: a warm start extrapolates w linearly from the last two solves
    int step_model;  // 1: curvature-informed first trial and quadratic backtracking
    int tlog_cap;    // bytes of tlog
    unsigned char* tlog;  // per-trial choices of this solve (nullable), see log_trial
};

// On-device state of one solve (FP64 scalars; Section 2.2's alternation).
struct SolveState {
    SolveParams prm;
    double w[8];   // accepted coefficients
    double wt[8];  // coefficients being evaluated (trial)
    double g[8];   // dJ/dw at (w, a, b)
    double a, b, J, Jt, mu, mu_prev, gnorm, gnorm0;
    double sy, syy, R;
    int iter, bt, trials, total_bt, stop, accepted, pad1_, running;
    double tumor[3];
    int tumor_steps, pad_;
    long long cum_solves, cum_trials, cum_iters, cum_lsf;  // since the model was loaded
    double mu_next;  // first trial step of the next iteration or warm-started solve (0 = none)
    double w_prev[8];  // final w of the solve before the last one (for the predictor)
    int history;       // warm-started solves in a row with a known final w (0, 1, >= 2)
    // Voxel box (lo x, y, z, hi x, y, z) that every 512-voxel chunk of the
    // model's (f, h) volume holding a nonzero meets; all zeros (a one-voxel
    // box) is valid for the all-zero volume of a freshly loaded model. Written
    // by the controller after each solver pass, read by the next warp pass.
    int fh_box[6];
};

// ---------------------------------------------------------------------------
// Sample positions: one definition for the projector and its transpose, so the
// two see bitwise-identical points.
// ---------------------------------------------------------------------------

// Unit direction of the ray to pixel (iu, iv), in index units per mm.
__device__ __forceinline__ void ray_dir_index(const RayGeom& g, int iu, int iv, float b[3]) {
    float fu = (float)iu, fv = (float)iv;
    float d0 = __fmaf_rn(fv, g.ev[0], __fmaf_rn(fu, g.eu[0], g.d00[0]));
    float d1 = __fmaf_rn(fv, g.ev[1], __fmaf_rn(fu, g.eu[1], g.d00[1]));
    float d2 = __fmaf_rn(fv, g.ev[2], __fmaf_rn(fu, g.eu[2], g.d00[2]));
    float inv = rsqrtf(__fmaf_rn(d0, d0, __fmaf_rn(d1, d1, __fmul_rn(d2, d2))));
    b[0] = __fmul_rn(__fmul_rn(d0, inv), g.inv_sp[0]);
    b[1] = __fmul_rn(__fmul_rn(d1, inv), g.inv_sp[1]);
    b[2] = __fmul_rn(__fmul_rn(d2, inv), g.inv_sp[2]);
}

// Sample lattice of one ray: sample s (at distance (s + 1/2) ds from the
// source) lies at index position q_s = o + s d + 1/2, with the step d = ds b
// and o = a + (ds / 2) b - 1/2, each rounded once per ray. The projector works
// in cell-origin coordinates q_s - 1/2 = o + s d (one multiply-add per axis
// and sample; the nearest integer of q_s - 1/2 is the lower corner of the
// trilinear cell of q_s), and the transpose evaluates the same values.
struct RayLattice {
    float o[3];  // q_0 - 1/2
    float d[3];  // step between samples, index units
};

__device__ __forceinline__ void ray_lattice(const RayGeom& g, const float b[3], RayLattice& L) {
    const float hs = 0.5f * g.ds;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        L.d[c] = __fmul_rn(g.ds, b[c]);
        L.o[c] = __fsub_rn(__fmaf_rn(hs, b[c], g.a[c]), 0.5f);
    }
}

// q_s - 1/2 for sample index sf (an integer held as a float, |sf| < 2^24).
__device__ __forceinline__ void lattice_point(const RayLattice& L, float sf, float qm[3]) {
    qm[0] = __fmaf_rn(sf, L.d[0], L.o[0]);
    qm[1] = __fmaf_rn(sf, L.d[1], L.o[1]);
    qm[2] = __fmaf_rn(sf, L.d[2], L.o[2]);
}

// Index-space position q_s of sample s (adding 1/2 back is exact for
// |q| < 2^22, i.e. anywhere near a grid).
__device__ __forceinline__ void sample_pos(const RayLattice& L, int s, float q[3]) {
    lattice_point(L, (float)s, q);
    q[0] = __fadd_rn(q[0], 0.5f);
    q[1] = __fadd_rn(q[1], 0.5f);
    q[2] = __fadd_rn(q[2], 0.5f);
}

// Ray parameter interval (mm) inside the index box [lo_c, hi_c] per axis.
// Returns false when the ray misses it.
__device__ __forceinline__ bool ray_box(const float a[3], const float b[3], const float lo[3],
                                        const float hi[3], float& t0, float& t1) {
    t0 = 0.0f;
    t1 = 3.0e38f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (b[c] != 0.0f) {
            float inv = 1.0f / b[c];
            float ta = (lo[c] - a[c]) * inv, tb = (hi[c] - a[c]) * inv;
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (!(a[c] > lo[c] && a[c] < hi[c])) {
            return false;
        }
    }
    return t1 > t0;
}

// ---------------------------------------------------------------------------
// Deterministic reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV doubles over the block (blockDim.x a multiple of 32, <= 1024) in a
// fixed order; thread 0 gets the totals in v.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[32][NV];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int m = 0; m < NV; ++m) v[m] = warp_sum(v[m]);
    if (lane == 0)
#pragma unroll
        for (int m = 0; m < NV; ++m) sh[wid][m] = v[m];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            double x = lane < nw ? sh[lane][m] : 0.0;
            v[m] = warp_sum(x);
        }
    }
    __syncthreads();
}

// Float-float (unevaluated hi + lo) arithmetic for exact-enough sums without
// the FP64 pipe, which is narrow on B300: a product of two floats is exactly
// hi + lo (TwoProduct with an FMA), and TwoSum keeps the rounding error of
// each addition, so a warp's sum of 32 such terms keeps ~48 bits.
__device__ __forceinline__ void ff_prod(float a, float b, float& hi, float& lo) {
    hi = __fmul_rn(a, b);
    lo = __fmaf_rn(a, b, -hi);
}

__device__ __forceinline__ void ff_add(float& hi, float& lo, float bhi, float blo) {
    float s = __fadd_rn(hi, bhi);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bhi, bb));
    e = __fadd_rn(e, __fadd_rn(lo, blo));
    float t = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(t, s));
    hi = t;
}

// Recursive-halving warp sums of NV values (NV <= 32), P = NV rounded up to a
// power of two. At each of log2(P) exchange levels (lane strides 16, 8, ...)
// every lane gives half of its remaining values to its partner and adds the
// partner's copy of the half it keeps; plain butterfly levels over the
// remaining strides then finish the sums. Each lane ends with one total: that
// of value `idx` (the return value; idx >= NV is padding), the same in the
// 32 / P lanes lane / (32 / P) == idx. P - 1 + log2(32 / P) additions per
// lane instead of 5 NV, and the sums come out spread over the lanes, so their
// stores go out in parallel. The order of every addition is fixed by lane.
template <int NV>
struct Halving {
    static_assert(NV >= 1 && NV <= 32, "1..32 values");
    static constexpr int P = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32;
    static constexpr int kSpan = 32 / P;  // lanes holding the same total
};

template <int NV>
__device__ __forceinline__ int warp_halving_sum(const double (&v)[NV], double& out) {
    constexpr int P = Halving<NV>::P;
    const int lane = threadIdx.x & 31;
    double x[P];
#pragma unroll
    for (int i = 0; i < P; ++i) x[i] = i < NV ? v[i < NV ? i : 0] : 0.0;
    int idx = 0;
#pragma unroll
    for (int lev = 0; (P >> lev) > 1; ++lev) {
        const int half = P >> (lev + 1), s = 16 >> lev;
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double give = up ? x[i] : x[half + i], keep = up ? x[half + i] : x[i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, give, s);
        }
        idx += up ? half : 0;
    }
#pragma unroll
    for (int s = Halving<NV>::kSpan >> 1; s >= 1; s >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], s);
    out = x[0];
    return idx;
}

// The same for float-float values (hi, lo); lane / (32 / P) == idx holds it.
template <int NV>
__device__ __forceinline__ int warp_halving_sum_ff(const float (&hi)[NV], const float (&lo)[NV], float& oh, float& ol) {
    constexpr int P = Halving<NV>::P;
    const int lane = threadIdx.x & 31;
    float h[P], l[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        h[i] = i < NV ? hi[i < NV ? i : 0] : 0.0f;
        l[i] = i < NV ? lo[i < NV ? i : 0] : 0.0f;
    }
    int idx = 0;
#pragma unroll
    for (int lev = 0; (P >> lev) > 1; ++lev) {
        const int half = P >> (lev + 1), s = 16 >> lev;
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float gh = up ? h[i] : h[half + i], gl = up ? l[i] : l[half + i];
            float kh = up ? h[half + i] : h[i], kl = up ? l[half + i] : l[i];
            ff_add(kh, kl, __shfl_xor_sync(0xffffffffu, gh, s), __shfl_xor_sync(0xffffffffu, gl, s));
            h[i] = kh;
            l[i] = kl;
        }
        idx += up ? half : 0;
    }
#pragma unroll
    for (int s = Halving<NV>::kSpan >> 1; s >= 1; s >>= 1)
        ff_add(h[0], l[0], __shfl_xor_sync(0xffffffffu, h[0], s), __shfl_xor_sync(0xffffffffu, l[0], s));
    oh = h[0];
    ol = l[0];
    return idx;
}

// Block sum of NV float-float values in a fixed order: float-float within
// each warp, FP64 across the warps; thread 0 gets the totals in out.
template <int NV>
__device__ __forceinline__ void block_sum_ff(float (&hi)[NV], float (&lo)[NV], double (&out)[NV]) {
    __shared__ double sh[32][NV];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            float bh = __shfl_down_sync(0xffffffffu, hi[m], o), bl = __shfl_down_sync(0xffffffffu, lo[m], o);
            ff_add(hi[m], lo[m], bh, bl);
        }
    if (lane == 0)
#pragma unroll
        for (int m = 0; m < NV; ++m) sh[wid][m] = (double)hi[m] + (double)lo[m];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            double x = lane < nw ? sh[lane][m] : 0.0;
            out[m] = warp_sum(x);
        }
    }
    __syncthreads();
}

// Write this block's NV partial sums (thread 0 holds them), then report whether
// this block is the last of `nblocks` to finish. The last block may then read
// every row with ldcg and must reset *counter to 0.
template <int NV, int STRIDE = kMaxMom>
__device__ __forceinline__ bool publish_partials(const double (&v)[NV], double* partials, int block,
                                                 int nblocks, unsigned int* counter) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int m = 0; m < NV; ++m) partials[(size_t)block * STRIDE + m] = v[m];
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

// In the last block: total of NV partial rows over nblocks, fixed order.
template <int NV, int STRIDE = kMaxMom>
__device__ __forceinline__ void total_partials(const double* partials, int nblocks, double (&tot)[NV]) {
#pragma unroll
    for (int m = 0; m < NV; ++m) tot[m] = 0.0;
    for (int r = threadIdx.x; r < nblocks; r += blockDim.x)
#pragma unroll
        for (int m = 0; m < NV; ++m) tot[m] += __ldcg(partials + (size_t)r * STRIDE + m);
    block_sum<NV>(tot);
}

__device__ __forceinline__ void set_loop(SolveState* st, int run, cudaGraphConditionalHandle h,
                                         int use_graph) {
    st->running = run;
    if (use_graph) cudaGraphSetConditional(h, run ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Storage types
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ld_val(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, float (&v)[4]) {
    uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&t.x);
    __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&t.y);
    float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

}  // namespace pr

// ---------------------------------------------------------------------------
// Host: launch on a stream, or append a kernel node to a graph chain.
// ---------------------------------------------------------------------------
namespace pr {

struct Launcher {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t last{};
    bool has_last = false;
    int count = 0;  // kernels launched or recorded
    // Graph mode: the next kernel node depends on `last` through a
    // programmatic edge from its launch-completion port (it may start once
    // every block of `last` has started; it must execute griddepcontrol.wait
    // before it reads what `last` writes). Cleared by that node.
    bool programmatic_next = false;

    template <typename... KArgs, typename... Args>
    cudaError_t operator()(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                           Args&&... args) {
        ++count;
        if (!graph) return launch(kern, grid, block, smem, static_cast<KArgs>(args)...);
        return node(kern, grid, block, smem, static_cast<KArgs>(args)...);
    }

    // cudaLaunchKernel reports this launch's own error; the process-wide
    // last-error state (which may hold an unrelated earlier error of the
    // caller's) is neither read nor cleared.
    template <typename... KArgs>
    cudaError_t launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, KArgs... args) {
        void* ptrs[sizeof...(KArgs) + 1] = {(void*)&args...};
        return cudaLaunchKernel((const void*)kern, grid, block, ptrs, smem, stream);
    }

    template <typename... KArgs>
    cudaError_t node(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, KArgs... args) {
        void* ptrs[] = {(void*)&args...};
        cudaKernelNodeParams p = {};
        p.func = (void*)kern;
        p.gridDim = grid;
        p.blockDim = block;
        p.sharedMemBytes = (unsigned)smem;
        p.kernelParams = ptrs;
        p.extra = nullptr;
        cudaGraphNode_t n;
        cudaError_t e;
        if (programmatic_next && has_last) {
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeKernel;
            np.kernel.func = p.func;
            np.kernel.gridDim = grid;
            np.kernel.blockDim = block;
            np.kernel.sharedMemBytes = (unsigned)smem;
            np.kernel.kernelParams = ptrs;
            cudaGraphEdgeData ed = {};
            ed.from_port = cudaGraphKernelNodePortLaunchCompletion;
            ed.type = cudaGraphDependencyTypeProgrammatic;
            e = cudaGraphAddNode(&n, graph, &last, &ed, 1, &np);
        } else {
            e = cudaGraphAddKernelNode(&n, graph, has_last ? &last : nullptr, has_last ? 1 : 0, &p);
        }
        programmatic_next = false;
        if (e == cudaSuccess) {
            last = n;
            has_last = true;
        }
        return e;
    }
};

}  // namespace pr
