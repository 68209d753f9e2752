// G2: cone-beam ray-march projector (Eq. 2's projection matrix P) with the
// fused residual/moment epilogue, and the on-device controller of Section
// 2.2's alternation: Eq. 4 for (a, b), Armijo's rule for the step of Eq. 3,
// and the stopping rule. Also the y-moment / initialisation kernel, the
// cost-gradient kernel of the step-level call, and the Section 2.3 tumor
// fixed point.
//
// Projector layout: one thread per ray; a warp of the solver pass owns a
// 4 x 8 patch of detector pixels (4 along u, 8 along v), or 2 x 16 within 30
// degrees of a diagonal of the volume's x-y axes, so the 32 samples a warp
// takes at one step lie within about one voxel of each other and the eight
// trilinear taps of the warp hit a handful of cache lines. A tall patch keeps
// the warp's rays in few (x, y) columns of the volume: each corner load then
// touches fewer cache lines (4 x 8 is 4-8% faster than 8 x 4 at every angle
// but 0, where it is equal; 2 x 16 is 3-6% faster again from 15 to 75
// degrees and slower near the axes). All lanes of a warp march the union of their sample
// ranges; a point outside the interpolant's support is clamped onto the zero
// border of the padded volume and adds exactly zero, so the loop has no
// divergent exits. The solver pass (k_project_split) splits each warp's range
// into parts taken from a work queue; the single-channel pass (k_project) gives
// a block of 256 threads a 32 x 8 tile.
#include <cuda_fp16.h>
#include <math.h>

#include "internal.h"

#include <algorithm>
#include <atomic>
#include <utility>
#include <vector>

namespace pr {
namespace {

constexpr int kTileU = 32, kTileV = 8, kProjThreads = kTileU * kTileV;
constexpr int kReduceThreads = 256;
constexpr int kReduceBlocks = 296;  // 2 per SM on a 148-SM B300
constexpr int kMaxSamples = 1 << 22;  // samples per ray, far above any real geometry
constexpr double kModelMinDecrease = 1e-6;  // see controller_project

// ---------------------------------------------------------------------------
// Controller pieces (one thread of the warp that completes a pass; FP64)
// ---------------------------------------------------------------------------

// Eq. 4: (a, b) = (Y^T Y)^-1 Y^T p with Y = [y, 1].
__device__ bool fit_ab(const SolveState* st, double sp, double spy, double* a, double* b) {
    double det = st->syy * st->R - st->sy * st->sy;
    if (!(det > 1e-12 * st->syy * st->R)) return false;
    *a = (st->R * spy - st->sy * sp) / det;
    *b = (st->syy * sp - st->sy * spy) / det;
    return isfinite(*a) && isfinite(*b);
}

// The largest power of two not above x (x > 0): steps stay exact power-of-two
// multiples, so FP32 rounding of a cost can change a step only across a
// power-of-two boundary.
__device__ double pow2_floor(double x) {
    int e;
    frexp(x, &e);  // x = m 2^e, 0.5 <= m < 1
    return ldexp(1.0, e - 1);
}

__device__ void next_trial(SolveState* st, int K) {
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
        if (k < K) st->wt[k] = st->w[k] - st->mu * st->g[k];
}

// ---------------------------------------------------------------------------
// Solve initialisation: y moments, finiteness of y, reset of the state.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kReduceThreads)
k_begin(const float* __restrict__ y, int R, SolveState* st, double* partials, unsigned int* counter) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        float yv = y[r];
        if (isfinite(yv)) {
            v[0] += yv;
            v[1] += (double)yv * yv;
        } else {
            v[2] += 1.0;
        }
    }
    block_sum<3>(v);
    if (!publish_partials<3>(v, partials, blockIdx.x, gridDim.x, counter)) return;
    double tot[3];
    total_partials<3>(partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
        *counter = 0;
        const int K = st->prm.K;
        st->sy = tot[0];
        st->syy = tot[1];
        st->R = (double)R;
        // Starting point: w0 (cold start), the last solve's w (warm start), or,
        // with prediction and two earlier solves, the linear extrapolation
        // 2 w(j-1) - w(j-2) from their final w.
        const bool cold = st->prm.cold_start != 0;
        const bool predict = !cold && st->prm.predict && st->history >= 2;
        for (int k = 0; k < kMaxK; ++k) {
            double last = st->w[k];
            double w0 = k < K ? (cold ? st->prm.w0[k] : (predict ? 2.0 * last - st->w_prev[k] : last)) : 0.0;
            st->w_prev[k] = cold ? 0.0 : last;
            st->w[k] = w0;
            st->wt[k] = w0;
            st->g[k] = 0.0;
        }
        st->history = cold ? 1 : min(st->history + 1, 2);
        st->a = 1.0;
        st->b = 0.0;
        st->J = st->Jt = 0.0;
        st->mu = st->mu_prev = 0.0;
        st->gnorm = st->gnorm0 = 0.0;
        st->iter = st->bt = st->trials = st->total_bt = 0;
        st->stop = tot[2] > 0.0 ? 4 : 0;  // PR_STOP_NONFINITE
        st->accepted = 0;
        st->running = 1;
        st->cum_solves += 1;
        if (st->prm.cold_start || !st->prm.warm_step) st->mu_next = 0.0;
    }
}

// ---------------------------------------------------------------------------
// G2 projector
// ---------------------------------------------------------------------------

// Trilinear accumulation of one sample into acc[0..NCH) (1 or 8 channels).
template <int NCH>
__device__ __forceinline__ void accumulate(const float* __restrict__ vol, const VolDev& vd, const float q[3],
                                           float (&acc)[NCH], float& comp);

// Compensated (Kahan) addition: the f channel's ray sum is the projection in
// the cost J, and its float rounding over ~600 samples would otherwise be
// the largest error in J (large enough to decide line-search tests near
// convergence); the h channels only feed the gradient direction.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
    float y = __fsub_rn(x, comp);
    float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// Cell of a sample: integer corner index i (clamped to [-1, n-1]) and the
// fraction t in [0, 1]. A point outside the support (-1, n) lands on the zero
// border with t saturated to 0 or 1, so it contributes exactly zero.
__device__ __forceinline__ int cell(float q, int n, float& t) {
    int i = min(max(__float2int_rd(q), -1), n - 1);
    t = __saturatef(q - (float)i);
    return i;
}

// Brick-level trace of a ray's sample range. Level k of the brick holding a
// point means every nonzero f0 voxel is at least 4 (k - 1) voxels away from it
// (Chebyshev), and the warped f and every h_k at a sample can be nonzero only
// within `margin` (support_box) of a nonzero f0 voxel. So from each end of
// [s_lo, s_hi] the samples with 4 (k - 1) > margin are skipped, advancing by as
// many samples as the slack allows (a sample moves at most ds max|b_c| voxels).
// Only exact zeros are skipped; at most kTraceSteps look-ups per end.
constexpr int kTraceSteps = 32;

__device__ __forceinline__ float brick_slack(const RayLattice& L, int s, const SupportRef& sr) {
    float q[3];
    sample_pos(L, s, q);
    const int bx = min(max((int)floorf(q[0] * 0.25f), 0), sr.bn[0] - 1);
    const int by = min(max((int)floorf(q[1] * 0.25f), 0), sr.bn[1] - 1);
    const int bz = min(max((int)floorf(q[2] * 0.25f), 0), sr.bn[2] - 1);
    const int k = __ldg(sr.lev + (bz * sr.bn[1] + by) * sr.bn[0] + bx);
    return 4.0f * (float)(k - 1);
}

__device__ __forceinline__ void trace_range(const RayLattice& L, const SupportRef& sr, float margin, int& s_lo,
                                            int& s_hi) {
    if (!sr.lev || s_lo > s_hi) return;
    const float step = fmaxf(fabsf(L.d[0]), fmaxf(fabsf(L.d[1]), fabsf(L.d[2])));
    if (!(step > 1.0e-6f)) return;
    for (int it = 0; it < kTraceSteps && s_lo <= s_hi; ++it) {
        const float slack = brick_slack(L, s_lo, sr) - margin;
        if (!(slack > 0.0f)) break;
        s_lo += max(1, (int)fminf(slack / step, 1.0e6f));
    }
    for (int it = 0; it < kTraceSteps && s_lo <= s_hi; ++it) {
        const float slack = brick_slack(L, s_hi, sr) - margin;
        if (!(slack > 0.0f)) break;
        s_hi -= max(1, (int)fminf(slack / step, 1.0e6f));
    }
}

// Cells by rounding: for |x| < 2^22, the float sum x + 1.5 * 2^23 holds the
// nearest integer of x in its low mantissa bits, and subtracting the constant
// again gives that integer as a float, exactly. In cell-origin coordinates
// x = q - 1/2 the nearest integer is the lower corner i0 of q's trilinear cell
// and t = x - i0 is in [-1/2, 1/2], so the corner weights are 1/2 - t and
// 1/2 + t, all without a float/int conversion. (At an exact integer q either
// neighbouring cell may be taken; the interpolated value is the same.)
constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
constexpr int kRoundBits = 0x4B400000; // its bit pattern

// The two float16 values packed in a float's bits, as floats (low half first).
__device__ __forceinline__ float2 unpack_half2(float x) {
    const unsigned int u = __float_as_uint(x);
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

// Sample accumulation that keeps the eight corners of the last trilinear cell
// in registers: consecutive samples 1 mm apart often fall in the same 2-2.5 mm
// cell, and then a lane that stays in its cell does not touch L1 for that
// sample. NCH = 4: one float4 (f, h_1..h_3) per corner; NCH = 6: a float4 and a
// float2 (h_4, h_5) per corner. Index arithmetic is 32-bit (volumes below
// 2^29 padded voxels).
//
// kClamp = false requires every sample to lie inside the index box
// (-1, n) of its axis: its cell is then within the padded volume. With kClamp
// the corner is clamped to [-1, n - 1] and the weights saturated, so a point
// anywhere lands on the zero border and adds exactly zero.
template <int NCH, bool HH = false>
struct CellCache {
    unsigned int base = 0xffffffffu;
    float c[8][NCH];     // corners: index = dx + 2 dy + 4 dz
    float comp = 0.0f;   // running compensation of acc[0]

    // bias: the padded index of the corner whose rounded coordinates have the
    // bit patterns of kRound, i.e. (1 - kRoundBits) (plane + row + 1) mod 2^32
    template <bool kClamp>
    __device__ __forceinline__ void sample(const float* __restrict__ vol, const VolDev& vd, unsigned int bias,
                                           const float qm[3], float (&acc)[NCH]) {
        float w0[3], w1[3];
        unsigned int bits[3];
        const int n[3] = {vd.nx, vd.ny, vd.nz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float m = __fadd_rn(qm[a], kRound);
            int bb = __float_as_int(m);
            float r;
            if (kClamp) {
                bb = min(max(bb, kRoundBits - 1), kRoundBits + n[a] - 1);
                r = __fsub_rn(__int_as_float(bb), kRound);
            } else {
                r = __fsub_rn(m, kRound);
            }
            const float t = __fsub_rn(qm[a], r);
            w1[a] = kClamp ? __saturatef(__fadd_rn(t, 0.5f)) : __fadd_rn(t, 0.5f);
            w0[a] = kClamp ? __saturatef(__fsub_rn(0.5f, t)) : __fsub_rn(0.5f, t);
            bits[a] = (unsigned int)bb;
        }
        const unsigned int plane = (unsigned int)(vd.nxp * vd.nyp);
        const unsigned int b = bits[2] * plane + bits[1] * (unsigned int)vd.nxp + bits[0] + bias;
        if (b != base) {
            base = b;
            const unsigned int off[4] = {0u, (unsigned int)vd.nxp, plane, plane + (unsigned int)vd.nxp};
            const float4* v4 = reinterpret_cast<const float4*>(vol);
            if constexpr (HH) {
                // one 16-byte record per corner: f, then float16 pairs (h1, h2), (h3, h4), (h5, 0)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 a = __ldg(v4 + b + off[k >> 1] + (k & 1));
                    const float2 p = unpack_half2(a.y), q = unpack_half2(a.z), r = unpack_half2(a.w);
                    c[k][0] = a.x, c[k][1] = p.x, c[k][2] = p.y, c[k][3] = q.x, c[k][4] = q.y, c[k][5] = r.x;
                }
            } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 a0 = __ldg(v4 + b + off[k]), a1 = __ldg(v4 + b + off[k] + 1);
                c[2 * k][0] = a0.x, c[2 * k][1] = a0.y, c[2 * k][2] = a0.z, c[2 * k][3] = a0.w;
                c[2 * k + 1][0] = a1.x, c[2 * k + 1][1] = a1.y, c[2 * k + 1][2] = a1.z, c[2 * k + 1][3] = a1.w;
            }
            }
            if constexpr (NCH == 6 && !HH) {
                const float2* v2 = reinterpret_cast<const float2*>(vol + 4 * vd.np);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float2 e0 = __ldg(v2 + b + off[k]), e1 = __ldg(v2 + b + off[k] + 1);
                    c[2 * k][4] = e0.x, c[2 * k][5] = e0.y;
                    c[2 * k + 1][4] = e1.x, c[2 * k + 1][5] = e1.y;
                }
            }
        }
        const float wyz[4] = {__fmul_rn(w0[1], w0[2]), __fmul_rn(w1[1], w0[2]), __fmul_rn(w0[1], w1[2]),
                              __fmul_rn(w1[1], w1[2])};
        float s0 = 0.0f;  // this sample's f value, added to the ray sum with compensation
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float a = __fmul_rn(wyz[k], w0[0]), e = __fmul_rn(wyz[k], w1[0]);
            s0 = __fmaf_rn(e, c[2 * k + 1][0], __fmaf_rn(a, c[2 * k][0], s0));
#pragma unroll
            for (int ch = 1; ch < NCH; ++ch)
                acc[ch] = __fmaf_rn(e, c[2 * k + 1][ch], __fmaf_rn(a, c[2 * k][ch], acc[ch]));
        }
        kahan_add(acc[0], comp, s0);
    }
};

__device__ __forceinline__ unsigned int cell_bias(const VolDev& vd) {
    return (1u - (unsigned int)kRoundBits) * (unsigned int)(vd.nxp * vd.nyp + vd.nxp + 1);
}

template <int NCH>
__device__ __forceinline__ void accumulate(const float* __restrict__ vol, const VolDev& vd, const float q[3],
                                           float (&acc)[NCH], float& comp) {
    float tx, ty, tz;
    int ix = cell(q[0], vd.nx, tx), iy = cell(q[1], vd.ny, ty), iz = cell(q[2], vd.nz, tz);
    int b = ((iz + 1) * vd.nyp + (iy + 1)) * vd.nxp + (ix + 1);
    const int plane = vd.nxp * vd.nyp;
    const int off[4] = {0, vd.nxp, plane, plane + vd.nxp};
    float wy0 = 1.0f - ty, wz0 = 1.0f - tz;
    const float wyz[4] = {wy0 * wz0, ty * wz0, wy0 * tz, ty * tz};
    float s0 = 0.0f;  // this sample's f value
    if (NCH == 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float* p = vol + b + off[k];
            float a0 = __ldg(p), a1 = __ldg(p + 1);
            s0 = __fmaf_rn(wyz[k], __fmaf_rn(tx, a1 - a0, a0), s0);
        }
    } else {
        constexpr int NV4 = NCH / 4;
        const float4* v4 = reinterpret_cast<const float4*>(vol);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4* p = v4 + (size_t)(b + off[k]) * NV4;
            float w0 = wyz[k] * (1.0f - tx), w1 = wyz[k] * tx;
#pragma unroll
            for (int h = 0; h < NV4; ++h) {
                float4 a0 = __ldg(p + h), a1 = __ldg(p + NV4 + h);
                if (h == 0)
                    s0 = __fmaf_rn(w1, a1.x, __fmaf_rn(w0, a0.x, s0));
                else
                    acc[4 * h + 0] = __fmaf_rn(w1, a1.x, __fmaf_rn(w0, a0.x, acc[4 * h + 0]));
                acc[4 * h + 1] = __fmaf_rn(w1, a1.y, __fmaf_rn(w0, a0.y, acc[4 * h + 1]));
                acc[4 * h + 2] = __fmaf_rn(w1, a1.z, __fmaf_rn(w0, a0.z, acc[4 * h + 2]));
                acc[4 * h + 3] = __fmaf_rn(w1, a1.w, __fmaf_rn(w0, a0.w, acc[4 * h + 3]));
            }
        }
    }
    kahan_add(acc[0], comp, s0);
}

struct ProjArgs {
    const float* vol;
    VolDev vd;
    const RayGeom* rg;
    const int* order;  // tile permutation (nullable): long rays first, so the last wave is short
    int nu, nv, K;
    int ntu;           // tiles along u
    float* p;
    float* q;
    const float* y;
    SolveState* st;
    double* partials;
    unsigned int* counter;
    int phase;
    cudaGraphConditionalHandle h;
    int use_graph;
    SupportRef sup;
};

// Moments of one projection pass, summed in FP64 over rays (products of two
// floats are exact in FP64): [0] sum p^2, [1] sum p y, [2] sum p,
// [3 + k] sum p q_k, [3 + KM + k] sum y q_k, [3 + 2 KM + k] sum q_k, with
// KM = 3 or 7 the channel capacity. From them J and dJ/dw follow for any
// (a, b) without another pass over the detector:
//   J(a, b)   = Spp - 2a Spy - 2b Sp + a^2 Syy + 2ab Sy + b^2 R        (Eq. 2)
//   g_k(a, b) = 2 (Spq_k - a Syq_k - b Sq_k)      (gradient after Eq. 4,
//               forward form: 2 sum_rays r (P h_k), r = p - a y - b)
template <int KM>
__device__ double cost_at(const SolveState* st, const double* m, double a, double b) {
    return m[0] - 2.0 * a * m[1] - 2.0 * b * m[2] + a * a * st->syy + 2.0 * a * b * st->sy + b * b * st->R;
}

// Cost and gradient at the state's (a, b) from the moments, then the stopping
// rule (Section 2.2) and, if the solve goes on, the first trial of the next
// step. One thread of the warp that completes the pass.
// The floating-point choices of line-search trial st->trials (1-based), one
// byte: bit 7 accepted, bit 6 stop (a rejected trial: the predicted decrease
// was unresolvable; an accepted one: the gradient test was met after it),
// bits 0-5 e + 32, where 2^e is the factor that scales mu next (0 when the
// factors are fixed, step_model 0). Kept so that a checker can follow the
// same path in FP64 and tell a rounding tie from a wrong branch.
__device__ void log_trial(SolveState* st, bool ok, bool stop, int e) {
    const int i = st->trials - 1;
    if (st->prm.tlog && i >= 0 && i < st->prm.tlog_cap)
        st->prm.tlog[i] = (unsigned char)((ok ? 0x80 : 0) | (stop ? 0x40 : 0) | ((e + 32) & 0x3f));
}

template <int KM>
__device__ void finish_point(SolveState* st, const double* m, int K, cudaGraphConditionalHandle h,
                             int use_graph) {
    const double a = st->a, b = st->b;
    st->J = cost_at<KM>(st, m, a, b);
    double gn2 = 0.0;
    for (int k = 0; k < kMaxK; ++k) {
        double gk = k < K ? 2.0 * (m[3 + k] - a * m[3 + KM + k] - b * m[3 + 2 * KM + k]) : 0.0;
        st->g[k] = gk;
        gn2 += gk * gk;
    }
    double gn = sqrt(gn2);
    st->gnorm = gn;
    if (st->iter == 0) st->gnorm0 = gn;
    if (st->stop != 0) {
        set_loop(st, 0, h, use_graph);
        return;
    }
    if (!isfinite(st->J) || !isfinite(gn)) {
        st->stop = 4;
        set_loop(st, 0, h, use_graph);
        return;
    }
    if (gn <= st->prm.grad_tol * st->gnorm0 || gn == 0.0) {
        st->stop = 1;  // PR_STOP_GRAD_TOL
        const int i = st->trials - 1;  // the accepted trial before this point, if any
        if (st->accepted && st->prm.tlog && i >= 0 && i < st->prm.tlog_cap) st->prm.tlog[i] |= 0x40;
        set_loop(st, 0, h, use_graph);
        return;
    }
    if (st->iter >= st->prm.max_iters) {
        st->stop = 2;  // PR_STOP_MAX_ITERS
        set_loop(st, 0, h, use_graph);
        return;
    }
    // after an accepted step (this solve or, warm-started, the previous frame's
    // last) the next step; otherwise a first trial that moves w by step0 mm
    st->mu = st->mu_next > 0.0 ? st->mu_next : st->prm.step0 / gn;
    st->bt = 0;
    next_trial(st, K);
    set_loop(st, 1, h, use_graph);
}

template <int KM>
__device__ void controller_project(SolveState* st, const double* m, int phase, cudaGraphConditionalHandle h,
                                   int use_graph, const Support* sup, const VolDev& vd) {
    const int K = st->prm.K;
    double a, b;
    // The (f, h) volume of this pass holds nonzeros only in blocks that meet
    // the warp's support box at wt; recorded one voxel wider (the warp forms
    // the same box in another kernel, where rounding may differ by an ulp)
    // so that the next warp pass can leave the other blocks alone.
    {
        int lo[3], hi[3];
        warp_box(sup, vd, st->wt, K, lo, hi, 1);
        for (int c = 0; c < 3; ++c) st->fh_box[c] = lo[c], st->fh_box[3 + c] = hi[c];
    }
    if (phase == kPhaseInit) {
        // Eq. 4 at the starting w, then the cost and gradient there
        if (st->stop == 0 && !fit_ab(st, m[2], m[1], &a, &b)) st->stop = 5;  // singular fit
        if (st->stop == 0) {
            st->a = a;
            st->b = b;
        }
        finish_point<KM>(st, m, K, h, use_graph);
        return;
    }
    // kPhaseTrial: Armijo's sufficient-decrease test at fixed (a, b) (Section 2.2).
    if (st->stop != 0) {
        set_loop(st, 0, h, use_graph);
        return;
    }
    st->trials += 1;
    st->cum_trials += 1;
    if (st->trials > (st->prm.max_iters + 1) * (st->prm.max_bt + 1) + 1) {
        st->stop = 6;  // internal guard: more trials than the options allow
        set_loop(st, 0, h, use_graph);
        return;
    }
    double Jt = cost_at<KM>(st, m, st->a, st->b);
    st->Jt = Jt;
    const double mu = st->mu, gn2 = st->gnorm * st->gnorm;
    // curvature of J along -g from this trial: J(mu) ~ J - mu |g|^2 + (curv/2) mu^2
    const double curv = 2.0 * (Jt - st->J + mu * gn2) / (mu * mu);
    // The quadratic model is used only where this step's predicted decrease
    // mu |g|^2 is resolvable in the cost (above kModelMinDecrease x J): a step
    // too small to change the cost would otherwise read as high curvature and
    // shrink the next step further and further.
    const bool model = st->prm.step_model == 1 && curv > 0.0 && isfinite(curv) &&
                       mu * gn2 > kModelMinDecrease * fabs(st->J);
    bool ok = isfinite(Jt) && Jt <= st->J - st->prm.c1 * mu * gn2;
    if (ok) {
        for (int k = 0; k < kMaxK; ++k)
            if (k < K) st->w[k] = st->wt[k];
        st->mu_prev = mu;
        // next first trial: the quadratic model's minimiser, at most
        // step_growth x mu; without the model, grow after a first-try
        // acceptance and keep after backtracking
        if (st->prm.step_model == 1) {
            // an accepted step is at most halved: near convergence the curvature
            // of a cost difference is mostly rounding
            const double f = pow2_floor(fmax(model ? fmin(st->prm.step_growth, gn2 / curv / mu) : st->prm.step_growth,
                                             0.5));
            st->mu_next = mu * f;
            log_trial(st, true, false, ilogb(f));
        } else {
            st->mu_next = (st->bt == 0 ? st->prm.step_growth : st->prm.step_growth_bt) * mu;
            log_trial(st, true, false, 0);
        }
        st->iter += 1;
        st->cum_iters += 1;
        st->accepted = 1;
        if (fit_ab(st, m[2], m[1], &a, &b)) {  // step 2, Eq. 4
            st->a = a;
            st->b = b;
        } else {
            st->stop = 5;
        }
        finish_point<KM>(st, m, K, h, use_graph);
        return;
    }
    st->accepted = 0;
    st->bt += 1;
    st->total_bt += 1;
    if (st->prm.step_model == 1 && !(mu * gn2 > kModelMinDecrease * fabs(st->J))) {
        // Even this step's predicted decrease is below what the cost resolves,
        // and a smaller one only less: the gradient is sufficiently small
        // (Section 2.2's stop) at the cost's resolution. w keeps its last
        // accepted value; the next frame starts from this step.
        log_trial(st, false, true, 0);
        st->stop = 7;  // PR_STOP_RESOLVED
        st->mu_next = mu;
        set_loop(st, 0, h, use_graph);
        return;
    }
    // backtrack: to the quadratic model's minimiser as a power-of-two fraction
    // of mu within [1/16, beta], or by beta
    double f = st->prm.beta;
    if (st->prm.step_model == 1) f = pow2_floor(model ? fmin(st->prm.beta, fmax(1.0 / 16.0, gn2 / curv / mu)) : st->prm.beta);
    log_trial(st, false, false, st->prm.step_model == 1 ? ilogb(f) : 0);
    if (st->bt > st->prm.max_bt) {
        st->stop = 3;  // PR_STOP_LINESEARCH_FAILED: w keeps its last accepted value
        st->cum_lsf += 1;
        st->mu_next = 0.0;  // the collapsed step says nothing about the next frame
        set_loop(st, 0, h, use_graph);
        return;
    }
    st->mu = mu * f;
    next_trial(st, K);
}

// Four 256-thread blocks per SM for the (f, h) volume (at most 64 registers):
// the march is issue-bound and needs the resident warps to hide L1 latency.
template <int NCH>
__global__ void __launch_bounds__(kProjThreads, NCH == 4 ? 4 : 1) k_project(ProjArgs A) {
    const RayGeom g = *A.rg;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int tile = A.order ? __ldg(A.order + blockIdx.x) : (int)blockIdx.x;
    if (tile < 0 || tile >= (int)gridDim.x) tile = blockIdx.x;  // a permutation never trips this
    const int tu = tile % A.ntu, tv = tile / A.ntu;
    const int iu = tu * kTileU + (wid & 3) * 8 + (lane & 7);
    const int iv = tv * kTileV + (wid >> 2) * 4 + (lane >> 3);
    const bool valid = iu < A.nu && iv < A.nv;

    float b[3];
    ray_dir_index(g, valid ? iu : 0, valid ? iv : 0, b);
    RayLattice L;
    ray_lattice(g, b, L);
    float lo[3] = {-1.0f, -1.0f, -1.0f}, hi[3] = {g.nmax[0], g.nmax[1], g.nmax[2]};
    bool nonzero = true;
    float margin = 0.0f;
    if (A.sup.sup && A.sup.w) nonzero = support_box(*A.sup.sup, A.vd, A.sup.w, A.sup.K, lo, hi, &margin);
    float t0, t1;
    int s_lo = 0x7fffffff, s_hi = -1;
    if (valid && nonzero && ray_box(g.a, b, lo, hi, t0, t1)) {
        // t0, t1 are bounded by the box; the clamps only keep the int
        // conversion and the loop counter far from overflow.
        s_lo = (int)fminf(fmaxf(ceilf(t0 / g.ds - 0.5f), 0.0f), (float)kMaxSamples);
        s_hi = (int)fminf(floorf(t1 / g.ds - 0.5f), (float)kMaxSamples);
        if (A.sup.w) trace_range(L, A.sup, margin, s_lo, s_hi);
        if (s_lo > s_hi) s_lo = 0x7fffffff, s_hi = -1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s_lo = min(s_lo, __shfl_xor_sync(0xffffffffu, s_lo, o));
        s_hi = max(s_hi, __shfl_xor_sync(0xffffffffu, s_hi, o));
    }
    float acc[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) acc[c] = 0.0f;
    if constexpr (NCH == 4) {
        CellCache<4> cache;
        const unsigned int bias = cell_bias(A.vd);
        for (int s = s_lo; s <= s_hi; ++s) {
            float qm[3];
            lattice_point(L, (float)s, qm);
            cache.template sample<true>(A.vol, A.vd, bias, qm, acc);
        }
    } else {
        float comp = 0.0f;
        for (int s = s_lo; s <= s_hi; ++s) {
            float q[3];
            sample_pos(L, s, q);
            accumulate<NCH>(A.vol, A.vd, q, acc, comp);
        }
    }

    const int R = A.nu * A.nv;
    const int r = iv * A.nu + iu;
    float pv = acc[0] * g.ds;
    if (valid) {
        A.p[r] = pv;
        if (NCH > 1 && A.q)
            for (int k = 0; k < A.K; ++k) A.q[(long long)k * R + r] = acc[1 + (k < NCH - 1 ? k : 0)] * g.ds;
    }
    if (A.phase == kPhaseNone) return;

    // Epilogue: this pass's moments (FP64; see cost_at), block sums, and the
    // controller in the last block to finish (single-channel pass).
    // Products of two floats are exact as float-float pairs, and the sums run
    // in float-float within a warp and in FP64 across warps and blocks.
    constexpr int KM = NCH == 8 ? 7 : 3;
    constexpr int NV = 3 + 3 * KM;
    float mh[NV], ml[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) mh[i] = ml[i] = 0.0f;
    if (valid) {
        const float yv = A.y[r];
        ff_prod(pv, pv, mh[0], ml[0]);
        ff_prod(pv, yv, mh[1], ml[1]);
        mh[2] = pv;
        if constexpr (NCH > 1) {
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                if (k < A.K) {
                    const float qv = acc[1 + k] * g.ds;
                    ff_prod(pv, qv, mh[3 + k], ml[3 + k]);
                    ff_prod(yv, qv, mh[3 + KM + k], ml[3 + KM + k]);
                    mh[3 + 2 * KM + k] = qv;
                }
            }
        }
    }
    double m[NV];
    block_sum_ff<NV>(mh, ml, m);
    const int nblocks = gridDim.x;
    if (!publish_partials<NV, kProjMom>(m, A.partials, tile, nblocks, A.counter)) return;
    double tot[NV];
    total_partials<NV, kProjMom>(A.partials, nblocks, tot);
    if (threadIdx.x == 0) {
        *A.counter = 0;
        controller_project<KM>(A.st, tot, A.phase, A.h, A.use_graph, A.sup.sup, A.vd);
    }
}

// ---------------------------------------------------------------------------
// Solver-pass projector with split rays and a dynamic work queue
// ---------------------------------------------------------------------------
//
// The 4/8-channel pass has 1.3 rays per resident thread at paper scale, and
// its run time was the time of the longest 32x8 tile: the last wave left SMs
// idle and blocks held their slots while waiting for their slowest warp. Here
// the unit of work is a quarter of the sample range of a 32-ray warp tile.
// Warps take items from a global counter, longest tiles first (the parts of
// a tile one after another), so the busy time evens out at the scale of a
// quarter of a ray. Each part's sums go to scratch; the warp that finishes a
// tile's last part adds the parts in a fixed order, writes p and q and the
// tile's moments; fixed groups of 64 tiles and then the groups are summed in
// tile order by whichever warp completes them, and the warp that completes
// the last group runs the controller. Every sum is taken in an order fixed
// by tile and part index, never by timing, so results are deterministic.
// No warp ever waits for another.
constexpr int kParts = 4;        // sample-range parts per warp tile
// A march runs without clamps when its end samples lie this far (index units)
// inside the box where every cell is within the padded volume: far above the
// rounding of a sample position, so every sample between them is inside too.
constexpr float kInsideMargin = 1.0f / 64.0f;
constexpr int kGroupTiles = 64;  // tiles per fixed-order moment group
constexpr int kSplitThreads = 256;

// Warp tiles of tu x (32 / tu) detector pixels covering nu x nv.
__host__ __device__ __forceinline__ int split_tiles_of(int nu, int nv, int tu) {
    return ((nu + tu - 1) / tu) * ((nv + 32 / tu - 1) / (32 / tu));
}

struct SplitArgs {
    const float* vol;
    VolDev vd;
    const RayGeom* rg;
    const int* order;  // warp-tile permutations of both shapes, longest rays first (nullable)
    int nu, nv, K;
    int ntiles, ngroups;  // of the shape with more tiles: the scratch layout (split_tiles)
    float* p;
    float* q;
    const float* y;
    SolveState* st;
    float* part;        // [tile][kParts][NCH + 1][32]: channel sums and the f compensation
    double* tile_mom;   // [tile][kProjMom]
    double* group_mom;  // [group][kProjMom]
    unsigned int* ctr;  // [0] queue, [1] warps done, [2] groups done, [4 + g] group g, [4 + ngroups + t] tile t
    int phase;
    cudaGraphConditionalHandle h;
    int use_graph;
    SupportRef sup;
};

// The warp that completed a tile group: sums the group's tile moments in tile
// order and, if it also completed the last group, the group sums in group
// order, then runs the controller. Out of line and apart from finish_tile:
// only one warp per group runs it, so its code and registers stay out of the
// per-tile path.
template <int NCH>
__device__ __noinline__ void finish_group(const SplitArgs& A, int group, int ntiles, int ngroups) {
    constexpr int KM = NCH == 8 ? 7 : (NCH == 6 ? 5 : 3);
    constexpr int NV = 3 + 3 * KM;
    const int lane = threadIdx.x & 31;
    const int gsize = min(kGroupTiles, ntiles - group * kGroupTiles);
    unsigned int prev = 0;
    __threadfence();
    if (lane == 0) A.ctr[4 + group] = 0;
    double gm[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) gm[m] = 0.0;
    for (int t = lane; t < gsize; t += 32)
#pragma unroll
        for (int m = 0; m < NV; ++m) gm[m] += __ldcg(A.tile_mom + (size_t)(group * kGroupTiles + t) * kProjMom + m);
    {
        double gs;
        const int idx = warp_halving_sum<NV>(gm, gs);
        if (lane % Halving<NV>::kSpan == 0 && idx < NV) A.group_mom[(size_t)group * kProjMom + idx] = gs;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) prev = atomicAdd(A.ctr + 2, 1u);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != (unsigned int)ngroups - 1) return;

    // ---- this warp completed the last group: totals in group order, controller ----
    __threadfence();
    double tot[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) tot[m] = 0.0;
    for (int gg = lane; gg < ngroups; gg += 32)
#pragma unroll
        for (int m = 0; m < NV; ++m) tot[m] += __ldcg(A.group_mom + (size_t)gg * kProjMom + m);
    {
        double ts;
        warp_halving_sum<NV>(tot, ts);
        // gather the totals into lane 0 (total m sits in lane m * kSpan)
#pragma unroll
        for (int m = 0; m < NV; ++m) tot[m] = __shfl_sync(0xffffffffu, ts, m * Halving<NV>::kSpan);
    }
    if (lane == 0) {
        A.ctr[2] = 0;
        controller_project<KM>(A.st, tot, A.phase, A.h, A.use_graph, A.sup.sup, A.vd);
    }
}

// The warp that completed a tile: adds its parts in part order, writes p and
// q, and (solver phases) forms the tile's moments and carries the fixed-order
// group and total sums. Kept out of line so that its registers do not weigh on
// the sample loop.
template <int NCH>
__device__ __noinline__ void finish_tile(const SplitArgs& A, int tile, int iu, int iv, bool valid, float ds, int ntiles,
                                         int ngroups) {
    constexpr int KM = NCH == 8 ? 7 : (NCH == 6 ? 5 : 3);
    constexpr int NV = 3 + 3 * KM;
    const int lane = threadIdx.x & 31;
    unsigned int* tile_ctr = A.ctr + 4 + A.ngroups;
    unsigned int prev = 0;
    // ---- this warp completed the tile: parts in fixed order ----
    __threadfence();
    if (lane == 0) tile_ctr[tile] = 0;
    const float* src = A.part + (size_t)tile * kParts * (NCH + 1) * 32 + lane;
    float fs = 0.0f, hs[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) hs[c] = 0.0f;
#pragma unroll
    for (int pp = 0; pp < kParts; ++pp) {
        const float* sp = src + (size_t)pp * (NCH + 1) * 32;
        fs = __fadd_rn(fs, __fsub_rn(__ldcg(sp), __ldcg(sp + NCH * 32)));
#pragma unroll
        for (int c = 1; c < NCH; ++c) hs[c] = __fadd_rn(hs[c], __ldcg(sp + c * 32));
    }
    const int R = A.nu * A.nv;
    const int r = iv * A.nu + iu;
    const float pv = fs * ds;
    if (valid) {
        A.p[r] = pv;
        if (A.q)
            for (int k = 0; k < A.K; ++k) A.q[(long long)k * R + r] = hs[1 + (k < NCH - 1 ? k : 0)] * ds;
    }
    if (A.phase == kPhaseNone) return;

    // tile moments (see cost_at): exact float-float products, float-float warp
    // sums by recursive halving (each moment's total ends in its own lanes)
    float mh[NV], ml[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) mh[i] = ml[i] = 0.0f;
    if (valid) {
        const float yv = A.y[r];
        ff_prod(pv, pv, mh[0], ml[0]);
        ff_prod(pv, yv, mh[1], ml[1]);
        mh[2] = pv;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if (k < A.K) {
                const float qv = hs[1 + k] * ds;
                ff_prod(pv, qv, mh[3 + k], ml[3 + k]);
                ff_prod(yv, qv, mh[3 + KM + k], ml[3 + KM + k]);
                mh[3 + 2 * KM + k] = qv;
            }
        }
    }
    {
        float th, tl;
        const int idx = warp_halving_sum_ff<NV>(mh, ml, th, tl);
        if (lane % Halving<NV>::kSpan == 0 && idx < NV)
            A.tile_mom[(size_t)tile * kProjMom + idx] = (double)th + (double)tl;
    }
    __threadfence();
    __syncwarp();
    const int group = tile / kGroupTiles;
    if (lane == 0) prev = atomicAdd(A.ctr + 4 + group, 1u);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev == (unsigned int)min(kGroupTiles, ntiles - group * kGroupTiles) - 1)
        finish_group<NCH>(A, group, ntiles, ngroups);
}

template <int NCH, bool HH = false>
__global__ void __launch_bounds__(kSplitThreads, NCH == 4 ? 4 : 2) k_project_split(SplitArgs A) {
    const RayGeom g = *A.rg;
    const int lane = threadIdx.x & 31;
    // This angle's warp tile, tu x (32 / tu) pixels (4 x 8 or 2 x 16): its
    // tile counts live in shared memory and are read once per work item, so
    // they hold no registers across the sample loop.
    __shared__ int shape[5];  // tu, tiles along u, tiles, tile groups, offset of its order
    if (threadIdx.x == 0) {
        const int tu = g.tile_u == 2 ? 2 : 4, nt = split_tiles_of(A.nu, A.nv, tu);
        shape[0] = tu;
        shape[1] = (A.nu + tu - 1) / tu;
        shape[2] = nt;
        shape[3] = (nt + kGroupTiles - 1) / kGroupTiles;
        shape[4] = tu == 2 ? split_tiles_of(A.nu, A.nv, 4) : 0;
    }
    __syncthreads();
    const volatile int* vshape = shape;
    unsigned int* tile_ctr = A.ctr + 4 + A.ngroups;  // the layout's (largest) group count

    float lo[3] = {-1.0f, -1.0f, -1.0f}, hi[3] = {g.nmax[0], g.nmax[1], g.nmax[2]};
    bool nonzero = true;
    float margin = 0.0f;
    if (A.sup.sup && A.sup.w) nonzero = support_box(*A.sup.sup, A.vd, A.sup.w, A.sup.K, lo, hi, &margin);
    bool volume_ready = false;

    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(A.ctr, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int ntiles = vshape[2];
        if (item >= (unsigned int)ntiles * kParts) break;
        const int slot = (int)(item / kParts), part = (int)(item - (unsigned int)slot * kParts);
        int tile = A.order ? __ldg(A.order + vshape[4] + slot) : slot;
        if (tile < 0 || tile >= ntiles) tile = slot;  // a permutation never trips this
        const int tu = vshape[0], ntu = vshape[1];
        const int iu = (tile % ntu) * tu + (lane & (tu - 1)), iv = (tile / ntu) * (32 / tu) + (lane / tu);
        const bool valid = iu < A.nu && iv < A.nv;

        float b[3];
        ray_dir_index(g, valid ? iu : 0, valid ? iv : 0, b);
        RayLattice L;
        ray_lattice(g, b, L);
        float t0, t1;
        int s_lo = 0x7fffffff, s_hi = -1;
        if (valid && nonzero && ray_box(g.a, b, lo, hi, t0, t1)) {
            s_lo = (int)fminf(fmaxf(ceilf(t0 / g.ds - 0.5f), 0.0f), (float)kMaxSamples);
            s_hi = (int)fminf(floorf(t1 / g.ds - 0.5f), (float)kMaxSamples);
            if (A.sup.w) trace_range(L, A.sup, margin, s_lo, s_hi);
            if (s_lo > s_hi) s_lo = 0x7fffffff, s_hi = -1;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s_lo = min(s_lo, __shfl_xor_sync(0xffffffffu, s_lo, o));
            s_hi = max(s_hi, __shfl_xor_sync(0xffffffffu, s_hi, o));
        }
        float acc[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) acc[c] = 0.0f;
        float comp = 0.0f;
        if (!volume_ready) {
            // Launched behind the warp kernel with a programmatic edge, this
            // grid may start while the warp's last blocks still write the
            // volume: the ray set-up above reads only w, the geometry and
            // the support, and the samples wait here for the warp grid to
            // complete with its writes visible (a no-op after an ordinary
            // dependency).
            asm volatile("griddepcontrol.wait;" ::: "memory");
            volume_ready = true;
        }
        if (s_hi >= s_lo) {
            const int Ls = s_hi - s_lo + 1;
            const int s_a = s_lo + (Ls * part) / kParts, s_e = s_lo + (Ls * (part + 1)) / kParts;
            if constexpr (NCH == 4 || NCH == 6) {
                // Every lane marches the warp's range [s_a, s_e); where all of
                // those samples of all 32 rays lie inside the grid (checked at
                // both ends: the samples of a ray lie on a segment) the cells
                // need no clamps. Otherwise (rays grazing a face of the grid,
                // a ragged detector edge) the clamped march runs.
                bool inside = true;
                if (s_e > s_a) {
                    float q0[3], q1[3];
                    lattice_point(L, (float)s_a, q0);
                    lattice_point(L, (float)(s_e - 1), q1);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float top = g.nmax[c] - 0.5f - kInsideMargin, bot = -1.5f + kInsideMargin;
                        inside = inside && q0[c] >= bot && q0[c] <= top && q1[c] >= bot && q1[c] <= top;
                    }
                }
                const unsigned int bias = cell_bias(A.vd);
                CellCache<NCH, HH> cache;
                if (__all_sync(0xffffffffu, inside)) {
                    for (float sf = (float)s_a, se = (float)s_e; sf < se; sf += 1.0f) {
                        float qm[3];
                        lattice_point(L, sf, qm);
                        cache.template sample<false>(A.vol, A.vd, bias, qm, acc);
                    }
                } else {
                    for (float sf = (float)s_a, se = (float)s_e; sf < se; sf += 1.0f) {
                        float qm[3];
                        lattice_point(L, sf, qm);
                        cache.template sample<true>(A.vol, A.vd, bias, qm, acc);
                    }
                }
                comp = cache.comp;
            } else {
                for (int s = s_a; s < s_e; ++s) {
                    float q[3];
                    sample_pos(L, s, q);
                    accumulate<NCH>(A.vol, A.vd, q, acc, comp);
                }
            }
        }
        // publish this part, then count it
        float* dst = A.part + ((size_t)tile * kParts + part) * (NCH + 1) * 32 + lane;
#pragma unroll
        for (int c = 0; c < NCH; ++c) dst[c * 32] = acc[c];
        dst[NCH * 32] = comp;
        __threadfence();
        __syncwarp();
        unsigned int prev = 0;
        if (lane == 0) prev = atomicAdd(tile_ctr + tile, 1u);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev != kParts - 1) continue;

        finish_tile<NCH>(A, tile, iu, iv, valid, g.ds, vshape[2], vshape[3]);
    }
    // The last warp to leave resets the queue for the next launch (no warp of
    // this launch reads it again).
    if (lane == 0) {
        const unsigned int total = gridDim.x * (blockDim.x >> 5);
        if (atomicAdd(A.ctr + 1, 1u) == total - 1) {
            A.ctr[0] = 0;
            A.ctr[1] = 0;
        }
    }
}

// Cost and gradient at explicit (a, b) (ab_dev[0..1]) for the step-level entry.
__global__ void __launch_bounds__(kReduceThreads)
k_cost_grad(const float* __restrict__ p, const float* __restrict__ q, const float* __restrict__ y, int R, int K,
            const double* ab, double* partials, unsigned int* counter, double* out) {
    const double a = ab[0], b = ab[1];
    // FP64 residual (it cancels), FP32 products per thread, FP64 sums
    float vf[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) vf[m] = 0.0f;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        float res = (float)((double)p[r] - fma(a, (double)y[r], b));
        vf[0] = __fmaf_rn(res, res, vf[0]);
        if (q)
#pragma unroll
            for (int k = 0; k < kMaxK; ++k)
                if (k < K) vf[1 + k] = __fmaf_rn(res, q[(long long)k * R + r], vf[1 + k]);
    }
    double v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = vf[m];
    block_sum<8>(v);
    if (!publish_partials<8>(v, partials, blockIdx.x, gridDim.x, counter)) return;
    double tot[8];
    total_partials<8>(partials, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    *counter = 0;
    out[0] = tot[0];
    for (int k = 0; k < K; ++k) out[1 + k] = 2.0 * tot[1 + k];
}

// ---------------------------------------------------------------------------
// Section 2.3: tumor position by the fixed-point inversion of the pull-back
// DVF (Chen et al.), evaluated at the single point c0: p <- c0 - x(p), with x
// = mean + U w trilinearly interpolated and clamped to the grid edge. FP64.
// ---------------------------------------------------------------------------
// One warp: lanes 0..23 each take one (corner, component) pair of the eight
// trilinear corners and three DVF components, so a fixed-point step costs one
// round of loads instead of 24 dependent ones. Lane 0's sums are broadcast,
// so every lane follows the same iterate.
template <typename TS>
__global__ void k_tumor(const float* mean, const TS* U, VolDev vd, int K, const double* w, double c0x,
                        double c0y, double c0z, double tol, int max_iter, const SolveParams* prm,
                        double* xyz, int* steps) {
    if (blockIdx.x != 0) return;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    if (prm) {  // per-solve options of an on-device solve
        tol = prm->tumor_tol;
        max_iter = prm->tumor_max_iter;
    }
    double wl[kMaxK];
    for (int k = 0; k < kMaxK; ++k) wl[k] = k < K ? w[k] : 0.0;
    const double c0[3] = {c0x, c0y, c0z};
    const double sp[3] = {(double)vd.dx, (double)vd.dy, (double)vd.dz};
    const int nn[3] = {vd.nx, vd.ny, vd.nz};
    const int corner = lane / 3, comp = lane % 3;
    double cur[3] = {c0x, c0y, c0z};
    int it = 0;
    while (it < max_iter) {
        // cell and fractions of the current point (clamped to the grid edge)
        int i0[3];
        double t[3];
        for (int c = 0; c < 3; ++c) {
            double o = -0.5 * (nn[c] - 1) * sp[c];
            double q = fmin(fmax((cur[c] - o) / sp[c], 0.0), (double)(nn[c] - 1));
            int i = max(0, min((int)floor(q), nn[c] - 2));
            i0[c] = i;
            t[c] = q - i;
        }
        double contrib = 0.0;
        if (lane < 24) {
            int cx = corner & 1, cy = (corner >> 1) & 1, cz = corner >> 2;
            int i = i0[0] + cx, j = i0[1] + cy, k = i0[2] + cz;
            if (i < vd.nx && j < vd.ny && k < vd.nz) {
                long long e = (long long)comp * vd.n + ((long long)k * vd.ny + j) * vd.nx + i;
                double xv = mean[e];
                for (int m = 0; m < K; ++m) xv += (double)ld_val(U + 3LL * m * vd.n + e) * wl[m];
                double wt = (cx ? t[0] : 1.0 - t[0]) * (cy ? t[1] : 1.0 - t[1]) * (cz ? t[2] : 1.0 - t[2]);
                contrib = wt * xv;
            }
        }
        double x[3];
        for (int c = 0; c < 3; ++c) {
            double v = (lane < 24 && comp == c) ? contrib : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            x[c] = __shfl_sync(0xffffffffu, v, 0);
        }
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            double nx = c0[c] - x[c];
            d2 += (nx - cur[c]) * (nx - cur[c]);
            cur[c] = nx;
        }
        ++it;
        if (sqrt(d2) < tol) break;
    }
    if (lane == 0) {
        xyz[0] = cur[0];
        xyz[1] = cur[1];
        xyz[2] = cur[2];
        *steps = it;
    }
}

// r = p - a y - b (ab[0] = a, ab[1] = b), the residual of Eq. 2.
__global__ void __launch_bounds__(256) k_residual(const float* __restrict__ p, const float* __restrict__ y, int R,
                                                  const double* ab, float* __restrict__ r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R) r[i] = (float)((double)p[i] - ab[0] * (double)y[i] - ab[1]);
}

}  // namespace

cudaError_t launch_residual(Launcher& L, const float* p, const float* y, int R, const double* ab_dev, float* r) {
    return L(k_residual, dim3((R + 255) / 256), dim3(256), 0, p, y, R, ab_dev, r);
}

int project_blocks(int nu, int nv) { return ((nu + kTileU - 1) / kTileU) * ((nv + kTileV - 1) / kTileV); }

void project_tile_order(int nu, int nv, int* order) {
    // Detector tiles sorted by the distance of their centre from the detector
    // centre: central rays cross the most volume, so they start first and the
    // last, partial wave of blocks holds the short edge tiles.
    const int ntu = (nu + kTileU - 1) / kTileU, ntv = (nv + kTileV - 1) / kTileV, n = ntu * ntv;
    const double cu = 0.5 * nu, cv = 0.5 * nv;
    struct Key { double d; int t; };
    Key* keys = new Key[n];
    for (int t = 0; t < n; ++t) {
        double u = ((t % ntu) + 0.5) * kTileU - cu, v = ((t / ntu) + 0.5) * kTileV - cv;
        keys[t] = {u * u + v * v, t};
    }
    // insertion sort on a stable key (small n; deterministic)
    for (int i = 1; i < n; ++i) {
        Key k = keys[i];
        int j = i - 1;
        while (j >= 0 && (keys[j].d > k.d || (keys[j].d == k.d && keys[j].t > k.t))) {
            keys[j + 1] = keys[j];
            --j;
        }
        keys[j + 1] = k;
    }
    for (int t = 0; t < n; ++t) order[t] = keys[t].t;
    delete[] keys;
}
int reduce_blocks() { return kReduceBlocks; }

cudaError_t launch_begin(Launcher& L, const float* y, int R, SolveState* st, double* partials,
                         unsigned int* counter) {
    return L(k_begin, dim3(kReduceBlocks), dim3(kReduceThreads), 0, y, R, st, partials, counter);
}

int split_tiles(int nu, int nv) { return max(split_tiles_of(nu, nv, 4), split_tiles_of(nu, nv, 2)); }
int split_groups(int nu, int nv) { return (split_tiles(nu, nv) + kGroupTiles - 1) / kGroupTiles; }
size_t split_part_floats(int nu, int nv, int nch) { return (size_t)split_tiles(nu, nv) * kParts * (nch + 1) * 32; }
size_t split_counters(int nu, int nv) { return 4 + (size_t)split_groups(nu, nv) + (size_t)split_tiles(nu, nv); }
int split_order_ints(int nu, int nv) { return split_tiles_of(nu, nv, 4) + split_tiles_of(nu, nv, 2); }

void project_warp_tile_order(int nu, int nv, int* order) {
    // For each tile shape (4 x 8, then 2 x 16): the warp tiles sorted by the
    // distance of their centre from the detector centre (long central rays
    // first); ties by tile index.
    const double cu = 0.5 * nu, cv = 0.5 * nv;
    for (int tu : {4, 2}) {
        const int tv = 32 / tu, ntu = (nu + tu - 1) / tu, n = split_tiles_of(nu, nv, tu);
        std::vector<std::pair<double, int>> keys((size_t)n);
        for (int t = 0; t < n; ++t) {
            double u = ((t % ntu) + 0.5) * tu - cu, v = ((t / ntu) + 0.5) * tv - cv;
            keys[(size_t)t] = {u * u + v * v, t};
        }
        std::sort(keys.begin(), keys.end());
        for (int t = 0; t < n; ++t) order[t] = keys[(size_t)t].second;
        order += n;
    }
}

namespace {
// Resident blocks of the split projector on this device (computed once per device).
int split_grid(int nch) {
    // per device and channel count; several host threads may ask at once (the
    // serving worker and callers), and any of them may fill an entry: they all
    // compute the same value
    static std::atomic<int> cached[4][64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::atomic<int>& c = cached[nch == kFhHalf6 ? 3 : (nch == 8 ? 2 : (nch == 6 ? 1 : 0))][dev];
    int v = c.load(std::memory_order_relaxed);
    if (v == 0) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (nch == kFhHalf6)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_project_split<6, true>, kSplitThreads, 0);
        else if (nch == 8)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_project_split<8>, kSplitThreads, 0);
        else if (nch == 6)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_project_split<6>, kSplitThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_project_split<4>, kSplitThreads, 0);
        v = sms * (per > 0 ? per : 1);
        c.store(v, std::memory_order_relaxed);
    }
    return v;
}
}  // namespace

cudaError_t launch_project(Launcher& L, const VolDev& vd, const float* vol_pad, int nch, int K,
                           const RayGeom* rg, const int* order, int nu, int nv, float* p, float* q,
                           const float* y, SolveState* st, double* partials, unsigned int* counter,
                           int phase, cudaGraphConditionalHandle h, int use_graph, SupportRef sup,
                           const SplitScratch* ss) {
    if (nch >= 4 && ss && ss->ctr) {
        const int ntiles = split_tiles(nu, nv), ngroups = split_groups(nu, nv);
        SplitArgs S{vol_pad, vd, rg, ss->order, nu, nv, K, ntiles, ngroups, p, q, y, st,
                    ss->part, ss->tile_mom, ss->group_mom, ss->ctr, phase, h, use_graph, sup};
        const int blocks = split_grid(nch);
        if (blocks <= 0) return cudaErrorInvalidDevice;
        const int need = (ntiles * kParts + kSplitThreads / 32 - 1) / (kSplitThreads / 32);
        const dim3 grid((unsigned)(need < blocks ? need : blocks));
        if (nch == kFhHalf6) return L(k_project_split<6, true>, grid, dim3(kSplitThreads), 0, S);
        if (nch == 8) return L(k_project_split<8>, grid, dim3(kSplitThreads), 0, S);
        if (nch == 6) return L(k_project_split<6>, grid, dim3(kSplitThreads), 0, S);
        if (nch == 4) return L(k_project_split<4>, grid, dim3(kSplitThreads), 0, S);
        return cudaErrorInvalidValue;
    }
    const int ntu = (nu + kTileU - 1) / kTileU, ntv = (nv + kTileV - 1) / kTileV;
    ProjArgs A{vol_pad, vd, rg, order, nu, nv, K, ntu, p, q, y, st, partials, counter, phase, h, use_graph, sup};
    dim3 grid(ntu * ntv);
    switch (nch) {
        case 1: return L(k_project<1>, grid, dim3(kProjThreads), 0, A);
        case 4: return L(k_project<4>, grid, dim3(kProjThreads), 0, A);
        case 8: return L(k_project<8>, grid, dim3(kProjThreads), 0, A);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cost_grad(Launcher& L, const float* p, const float* q, const float* y, int R, int K,
                             const double* ab_dev, double* partials, unsigned int* counter, double* out) {
    return L(k_cost_grad, dim3(kReduceBlocks), dim3(kReduceThreads), 0, p, q, y, R, K, ab_dev, partials,
             counter, out);
}

cudaError_t launch_tumor(Launcher& L, const ModelDev& m, const double* w_dev, double tol, int max_iter,
                         const SolveParams* prm, double* xyz_out, int* steps_out) {
    if (m.storage == 1)
        return L(k_tumor<__nv_bfloat16>, dim3(1), dim3(32), 0, m.mean,
                 static_cast<const __nv_bfloat16*>(m.U), m.vd, m.K, w_dev, m.c0[0], m.c0[1], m.c0[2], tol,
                 max_iter, prm, xyz_out, steps_out);
    return L(k_tumor<float>, dim3(1), dim3(32), 0, m.mean, static_cast<const float*>(m.U), m.vd, m.K, w_dev,
             m.c0[0], m.c0[1], m.c0[2], tol, max_iter, prm, xyz_out, steps_out);
}

// ---------------------------------------------------------------------------
// Support of a model (once at load)
// ---------------------------------------------------------------------------
namespace {

__global__ void k_support_init(Support* s) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int c = 0; c < 3; ++c) {
            s->lo[c] = 0x7fffffff;
            s->hi[c] = -0x7fffffff;
            s->mean_max[c] = 0u;
            for (int k = 0; k < kMaxK; ++k) s->u_max[k][c] = 0u;
        }
    }
}

__global__ void __launch_bounds__(256) k_brick_occ(VolDev vd, const float* __restrict__ f0, unsigned char* occ, int bnx,
                                                    int bny) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < vd.n; v += (long long)gridDim.x * blockDim.x) {
        if (f0[v] != 0.0f) {
            long long jk = v / vd.nx;
            const int i = (int)(v - jk * vd.nx), j = (int)(jk % vd.ny), k = (int)(jk / vd.ny);
            occ[((k >> 2) * bny + (j >> 2)) * bnx + (i >> 2)] = 1;
        }
    }
}

// One thread per ray: the projector's own clipping (support box, then the
// brick trace), summed as 64-bit counts.
__global__ void __launch_bounds__(256) k_count_samples(VolDev vd, const RayGeom* __restrict__ rgp, int nu, int nv,
                                                       SupportRef sr, unsigned long long* count) {
    const RayGeom g = *rgp;
    float lo[3] = {-1.0f, -1.0f, -1.0f}, hi[3] = {g.nmax[0], g.nmax[1], g.nmax[2]};
    float margin = 0.0f;
    bool nonzero = true;
    if (sr.sup && sr.w) nonzero = support_box(*sr.sup, vd, sr.w, sr.K, lo, hi, &margin);
    unsigned long long c = 0;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nu * nv && nonzero) {
        float b[3], t0, t1;
        ray_dir_index(g, r % nu, r / nu, b);
        RayLattice L;
        ray_lattice(g, b, L);
        if (ray_box(g.a, b, lo, hi, t0, t1)) {
            int s_lo = (int)fminf(fmaxf(ceilf(t0 / g.ds - 0.5f), 0.0f), (float)kMaxSamples);
            int s_hi = (int)fminf(floorf(t1 / g.ds - 0.5f), (float)kMaxSamples);
            if (sr.w) trace_range(L, sr, margin, s_lo, s_hi);
            if (s_hi >= s_lo) c = (unsigned long long)(s_hi - s_lo + 1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void __launch_bounds__(256) k_support_box(VolDev vd, const float* __restrict__ f0, Support* s) {
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < vd.n;
         v += (long long)gridDim.x * blockDim.x) {
        if (f0[v] != 0.0f) {
            long long jk = v / vd.nx;
            int idx[3] = {(int)(v - jk * vd.nx), (int)(jk % vd.ny), (int)(jk / vd.ny)};
            for (int c = 0; c < 3; ++c) {
                lo[c] = min(lo[c], idx[c]);
                hi[c] = max(hi[c], idx[c]);
            }
        }
    }
    for (int c = 0; c < 3; ++c) {
        int a = __reduce_min_sync(0xffffffffu, lo[c]), b = __reduce_max_sync(0xffffffffu, hi[c]);
        if ((threadIdx.x & 31) == 0 && a <= b) {
            atomicMin(&s->lo[c], a);
            atomicMax(&s->hi[c], b);
        }
    }
}

__global__ void __launch_bounds__(256) k_maxabs(const float* __restrict__ x, long long n, unsigned int* out) {
    unsigned int m = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float a = fabsf(x[i]);
        if (!(a <= 3.0e38f)) a = 3.0e38f;  // non-finite: the bound becomes huge, the box the whole grid
        m = max(m, __float_as_uint(a));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace

cudaError_t launch_brick_occ(Launcher& L, const VolDev& vd, const float* f0, unsigned char* occ) {
    const int bnx = (vd.nx + 3) / 4, bny = (vd.ny + 3) / 4;
    return L(k_brick_occ, dim3(148 * 8), dim3(256), 0, vd, f0, occ, bnx, bny);
}

cudaError_t launch_count_samples(Launcher& L, const VolDev& vd, const RayGeom* rg, int nu, int nv, SupportRef sup,
                                 unsigned long long* count) {
    return L(k_count_samples, dim3((unsigned)((nu * nv + 255) / 256)), dim3(256), 0, vd, rg, nu, nv, sup, count);
}

cudaError_t launch_support_init(Launcher& L, Support* sup) { return L(k_support_init, dim3(1), dim3(32), 0, sup); }

cudaError_t launch_support_box(Launcher& L, const VolDev& vd, const float* f0, Support* sup) {
    return L(k_support_box, dim3(1184), dim3(256), 0, vd, f0, sup);
}

cudaError_t launch_maxabs(Launcher& L, const float* x, long long n, unsigned int* out) {
    return L(k_maxabs, dim3(1184), dim3(256), 0, x, n, out);
}

}  // namespace pr
