// Internal interface between the C-ABI runtime (runtime.cu) and the kernel
// translation units (warp.cu, project.cu, backproject.cu).
#pragma once

#include "common.cuh"

namespace pr {

// Device buffers of one loaded model (all owned by the runtime).
struct ModelDev {
    VolDev vd;
    int K;
    int storage;       // 0 = float32, 1 = bfloat16 (f0 and U)
    const void* f0p;   // padded reference volume
    const float* mean; // [3][N]
    const void* U;     // [K][3][N]
    double c0[3];      // tumor reference position (mm)
};

// Output selection of the warp kernel (Section 2.2's f and h_k = (df/dx) . u_k).
enum WarpMode : int {
    kWarpFH = 0,      // f and h interleaved into the padded solver volume
    kWarpFPad = 1,    // f only, padded planar (for projection)
    kWarpFlatF = 2,   // f only, unpadded [N]
    kWarpFlatFH = 3,  // f [N] (nullable) and h [K][N] (nullable), unpadded
};

// Channels per voxel of the solver volume: f, h_1..h_K, rounded up to 4, 6 or 8.
// 4 and 8: interleaved float4 per voxel (one or two). 6 (K = 4, 5): a float4
// array of (f, h_1, h_2, h_3) over the padded grid, then a float2 array of
// (h_4, h_5), so that every corner is one 16-byte and one 8-byte aligned load.
inline int fh_channels(int K) { return K <= 3 ? 4 : (K <= 5 ? 6 : 8); }

// Layout code of the solver volume: fh_channels(K) as above, or kFhHalf6 for a
// model stored in bfloat16 with K = 4 or 5, whose (f, h_1..h_5) are one 16-byte
// record per voxel: f as float32, then (h_1, h_2), (h_3, h_4) and (h_5, 0) as
// float16 pairs (the ray sums of every channel still run in float32).
constexpr int kFhHalf6 = 16;
inline int fh_layout(int K, int storage) { return (storage == 1 && (K == 4 || K == 5)) ? kFhHalf6 : fh_channels(K); }
inline int fh_floats(int layout) { return layout == kFhHalf6 ? 4 : layout; }   // stored floats per voxel
inline int fh_logical(int layout) { return layout == kFhHalf6 ? 6 : layout; }  // channels the projector sums

// G1: x = mean + U w (Eq. 1), f(v) = F0(v + x(v)), h_k(v) (Section 2.2).
// w_dev: K doubles in device memory. sup (device, nullable; padded modes
// only): the model's support record; voxels outside the support box at w_dev
// are exact zeros and are written as zeros without reading their fields.
// dirty (device, 6 ints, nullable; with sup): a box that every 512-voxel
// chunk of out_pad holding a nonzero meets; chunks that miss both it and the
// support box are not written. The caller keeps it valid after the pass (the
// solve's controller records the pass's box; other callers use
// launch_warp_box).
cudaError_t launch_warp(Launcher& L, const ModelDev& m, const double* w_dev, int mode, float* out_pad,
                        float* f_flat, float* h_flat, const Support* sup = nullptr, const int* dirty = nullptr);

// Voxel box [lo, hi] (per axis, clamped to the grid; empty when lo > hi) that
// the support-restricted warp evaluates at coefficients w_dev, widened by
// `grow` voxels, written as six ints (lo x, y, z, hi x, y, z) to box_dev.
// sup == nullptr gives the whole grid.
cudaError_t launch_warp_box(Launcher& L, const ModelDev& m, const double* w_dev, const Support* sup, int grow,
                            int* box_dev);

// Round float32 to bfloat16 (round-to-nearest-even), n elements.
cudaError_t launch_to_bf16(Launcher& L, const float* src, __nv_bfloat16* dst, long long n);

// Copy an unpadded volume into a padded one (border must already be zero).
cudaError_t launch_pad(Launcher& L, const VolDev& vd, const float* src, float* dst_pad);

// y moments and solve initialisation (first kernel of a solve).
cudaError_t launch_begin(Launcher& L, const float* y, int R, SolveState* st, double* partials,
                         unsigned int* counter);

// G2: cone-beam projection of a padded volume with `nch` channels per voxel
// (1 = planar f, 4 or 8 = interleaved f, h). rg: device RayGeom. p: [R];
// q: [K][R] (channels 1..K, nullable). For phase != kPhaseNone, y, st,
// partials and counter drive the fused reduction and the controller.
// Optional clipping of the ray march to the support of a model's warped
// volume: sup (device) and the coefficients w (device, K doubles) it was warped at.
// lev (nullable): per 4^3-voxel brick of the grid (bn[0] x bn[1] x bn[2], x
// fastest) the Chebyshev distance in bricks to the nearest brick holding a
// nonzero f0 voxel (0: the brick holds one; capped at 255), so that rays skip
// the samples at either end that lie too far from the body to be nonzero.
struct SupportRef {
    const Support* sup = nullptr;
    const double* w = nullptr;
    int K = 0;
    const unsigned char* lev = nullptr;
    int bn[3] = {0, 0, 0};
};

// Brick occupancy of an unpadded f0 (device, float32): occ[brick] = 1 where the
// brick holds a nonzero voxel (occ zeroed by the caller; bricks of 4^3 voxels).
cudaError_t launch_brick_occ(Launcher& L, const VolDev& vd, const float* f0, unsigned char* occ);

// Exact per-ray sample count of the solver-pass projector (after the support box
// and the brick-level trace) at coefficients w (device doubles) into *count
// (device, zeroed by the caller).
cudaError_t launch_count_samples(Launcher& L, const VolDev& vd, const RayGeom* rg, int nu, int nv, SupportRef sup,
                                 unsigned long long* count);

// Scratch of the split-ray solver-pass projector (one per model; see
// k_project_split): warp-tile order, per-part sums, tile and group moments,
// and counters that must be zero before the first launch (each launch leaves
// them zero).
struct SplitScratch {
    const int* order = nullptr;   // split_order_ints ints (project_warp_tile_order)
    float* part = nullptr;        // split_part_floats floats
    double* tile_mom = nullptr;   // split_tiles x kProjMom doubles
    double* group_mom = nullptr;  // split_groups x kProjMom doubles
    unsigned int* ctr = nullptr;  // split_counters uints, zeroed once
};
// Scratch sizes of the split projector: tiles and tile groups of the warp
// tile shape (4 x 8 or 2 x 16 pixels, RayGeom::tile_u) with more tiles.
int split_tiles(int nu, int nv);
int split_groups(int nu, int nv);
size_t split_part_floats(int nu, int nv, int nch);
size_t split_counters(int nu, int nv);
int split_order_ints(int nu, int nv);
// Host: the launch order of the 4 x 8 warp tiles, centre first, followed by
// that of the 2 x 16 tiles (split_order_ints ints).
void project_warp_tile_order(int nu, int nv, int* order);

// order: device permutation of the detector tiles (nullable), see project_tile_order.
// With nch 4 or 8 and ss given, the split-ray kernel runs (its own tile order
// and scratch from ss; `order`, `partials` and `counter` unused).
cudaError_t launch_project(Launcher& L, const VolDev& vd, const float* vol_pad, int nch, int K,
                           const RayGeom* rg, const int* order, int nu, int nv, float* p, float* q,
                           const float* y, SolveState* st, double* partials, unsigned int* counter,
                           int phase, cudaGraphConditionalHandle h, int use_graph, SupportRef sup = {},
                           const SplitScratch* ss = nullptr);

// Support of f0 and the largest |mean_c|, |u_kc| into sup (device); f0, mean, U
// float32 unpadded (U may be one plane at a time: plane index k*3 + c).
cudaError_t launch_support_init(Launcher& L, Support* sup);
cudaError_t launch_support_box(Launcher& L, const VolDev& vd, const float* f0, Support* sup);
cudaError_t launch_maxabs(Launcher& L, const float* x, long long n, unsigned int* out);

// Host: the projector's tile launch order for an nu x nv detector (project_blocks ints).
void project_tile_order(int nu, int nv, int* order);

// Generic cost / gradient for explicit (w, a, b) from stored p, q: out[0] = J,
// out[1 + k] = 2 sum r q_k.
cudaError_t launch_cost_grad(Launcher& L, const float* p, const float* q, const float* y, int R, int K,
                             const double* ab_dev, double* partials, unsigned int* counter,
                             double* out);

// Section 2.3 tumor fixed point at w (device doubles) into xyz_out / steps_out.
// prm (nullable): take tol and max_iter from these per-solve parameters instead.
cudaError_t launch_tumor(Launcher& L, const ModelDev& m, const double* w_dev, double tol, int max_iter,
                         const SolveParams* prm, double* xyz_out, int* steps_out);

// Section 2.3 with ref. 13 on the whole grid: push-forward field y [3][N] (mm,
// device) of x = mean + U w (w_dev: K device doubles). X: scratch of N float4.
// stats (device, 2 uints, zeroed by the caller): [0] the largest per-voxel step
// count, [1] voxels whose last update was not below tol (mm).
cudaError_t launch_invert(Launcher& L, const ModelDev& m, const double* w_dev, float4* X, double tol, int max_iter,
                          float* y, unsigned int* stats);

// r = p - a y - b with (a, b) = ab_dev[0..1].
cudaError_t launch_residual(Launcher& L, const float* p, const float* y, int R, const double* ab_dev, float* r);

// Fixed-angle table of the transpose (see backproject.cu): per voxel its
// footprint rectangle (u0, w0, width, height), and the pixel weights slot-major
// (slot s of voxel v at w[s * N + v]). Null w: weights computed on the fly.
struct BpTable {
    const short4* rect = nullptr;
    const float* w = nullptr;
};

// P^T by voxel-driven gather. With h (K planes, unpadded) given, the per-voxel
// values are never stored: out[k] = sum_v (P^T r)(v) h_k(v) (and g_flat may be
// null); otherwise g_flat [N] receives P^T r. With tab.w, the weights come from
// a table built for rg's angle (bitwise the same result).
cudaError_t launch_backproject(Launcher& L, const VolDev& vd, const RayGeom* rg, const float* r,
                               float* g_flat, const float* h, int K, double* partials,
                               unsigned int* counter, double* out, BpTable tab = {});

// Fixed-angle table: rect [N] and the largest footprint into *max_slots (device,
// zeroed by the caller), then the weights (max_slots x N floats).
cudaError_t launch_bp_rect(Launcher& L, const VolDev& vd, const RayGeom* rg, short4* rect, unsigned int* max_slots);
cudaError_t launch_bp_fill(Launcher& L, const VolDev& vd, const RayGeom* rg, const short4* rect, float* w);

// Record msg as the calling thread's pr_last_error() text; returns code.
int set_last_error(int code, const char* msg);

// Number of blocks the reductions use (size of the partials buffer rows).
int project_blocks(int nu, int nv);
int reduce_blocks();
int backproject_blocks(const VolDev& vd);

}  // namespace pr
