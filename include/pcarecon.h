/*
 * pcarecon: single-projection volumetric reconstruction with a PCA lung-motion
 * model, and 3D tumor localisation, on one B300 GPU (sm_103a).
 *
 * Method: Li, Jia, Lewis, Gu, Folkerts, Men, Jiang, "Real-time volumetric image
 * reconstruction and 3D tumor localization based on a single x-ray projection
 * image for lung cancer radiotherapy". Given a patient's reference volume f0, a
 * mean DVF and K PCA eigenvector fields (Section 2.1, Eq. 1), one measured
 * cone-beam projection y and its gantry angle, the library minimises
 *     J(w, a, b) = || P f(x, f0) - a y - b 1 ||^2,  x = mean + U w     (Eq. 2)
 * by alternating a gradient step on w with Armijo's line search (Eq. 3) and
 * the exact (a, b) of Eq. 4, then locates the tumor through the inverted
 * pull-back DVF (Section 2.3). Every step runs in this library's CUDA kernels.
 *
 * Conventions (all entry points):
 *   - Volumes are [nz][ny][nx] float32, x fastest. Voxel (i,j,k) is at
 *     origin + (i,j,k)*spacing (mm), origin = -(n-1)/2*spacing: the isocentre is
 *     the volume centre. x lateral (patient right = -x), y anterior-posterior
 *     (+y posterior), z superior-inferior (+z cranial).
 *   - Vector fields are planar [3][nz][ny][nx] (mm, component 0 = x);
 *     eigenvectors are [K][3][nz][ny][nx]. DVFs are pull-back fields: the
 *     image at v is f0 trilinearly interpolated at v + x(v) (zero outside the
 *     grid).
 *   - Gantry angle th (rad): source (SAD sin th, -SAD cos th, 0); detector
 *     centre at distance SDD from the source along (-sin th, cos th, 0); detector
 *     axes u = (cos th, sin th, 0), v = (0, 0, 1); pixel (iu, iv) centre at
 *     (iu - (nu-1)/2) du, (iv - (nv-1)/2) dv; projections are [nv][nu] float32.
 *   - Projector P: for each pixel, ds * sum over s >= 0 of the trilinear
 *     interpolant at S + (s + 1/2) ds d (d = unit direction to the pixel
 *     centre): ray samples are anchored at the source, so P^T is enumerable
 *     per voxel.
 *   - Every call returns an int status: 0 = PR_OK, < 0 = error (then
 *     pr_last_error() gives a message for the calling thread). No exception or
 *     CUDA error crosses the boundary. A CUDA fault inside a call is reported
 *     as PR_ECUDA; the context must then be destroyed.
 *   - Pointers marked "host" are host memory, "device" are device memory of
 *     the context's GPU; `location` arguments say which (PR_HOST/PR_DEVICE).
 *     The library never keeps a caller pointer after a call returns: inputs
 *     are copied, outputs are written before return (synchronous calls) or
 *     before the context stream reaches the end of the enqueued work
 *     (*_async calls).
 *   - All device work runs on the context's stream (the one given to
 *     pr_create, else one the library creates). A context is not thread-safe:
 *     one host thread at a time.
 */
#ifndef PCARECON_H
#define PCARECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PR_OK 0
#define PR_EINVAL (-1)      /* bad argument (null pointer, size, shape, value) */
#define PR_ENOMEM (-2)      /* device or pinned host allocation failed */
#define PR_EADMIT (-3)      /* the model does not fit the context's HBM budget */
#define PR_ECUDA (-4)       /* a CUDA runtime call or kernel failed */
#define PR_ETIMEOUT (-5)    /* a bounded wait ran out */
#define PR_ENOMODEL (-6)    /* unknown or released model id */
#define PR_EUNSUPPORTED (-7)
#define PR_QUEUED 1         /* pr_load_model with the admission queue on: the model does not fit
                               the HBM budget now and waits for admission (not an error) */

/* ---- why a solve stopped (pr_result.stop_reason) ---- */
#define PR_STOP_GRAD_TOL 1          /* |grad J| <= grad_tol * |grad J at start| */
#define PR_STOP_MAX_ITERS 2         /* max_iters accepted steps (Section 2.2's iteration cap) */
#define PR_STOP_LINESEARCH_FAILED 3 /* Armijo found no step within max_backtracks; w kept */
#define PR_STOP_NONFINITE 4         /* non-finite projection or measurement; w kept */
#define PR_STOP_SINGULAR_FIT 5      /* Y^T Y of Eq. 4 is singular (constant y); w kept */
#define PR_STOP_GUARD 6             /* internal trial bound reached (should not happen) */
#define PR_STOP_RESOLVED 7          /* step_model 1: a rejected trial's predicted decrease
                                       mu |grad J|^2 was already <= 1e-6 J, so no step can
                                       lower J by a resolvable amount; w kept */

#define PR_MAX_K 7 /* most PCA modes per model */

enum { PR_HOST = 0, PR_DEVICE = 1 };
enum { PR_F32 = 0, PR_BF16 = 1 }; /* storage of f0 and U on the device */
enum { PR_LOOP_GRAPH = 0, PR_LOOP_HOST = 1 };

typedef struct pr_ctx pr_ctx;

typedef struct {
    int nx, ny, nz;     /* voxels */
    double dx, dy, dz;  /* spacing, mm */
} pr_volume_desc;

typedef struct {
    double sad, sdd; /* source-isocentre and source-detector distances, mm */
    int nu, nv;      /* detector pixels */
    double du, dv;   /* pixel pitch, mm */
    double ds;       /* ray sample step, mm; <= 0 selects half the smallest voxel spacing */
} pr_geometry;

/* Solver options (Section 2.2). The paper names Armijo's rule and a stop on a
 * small gradient or an iteration cap; the constants are this library's
 * defaults (pr_default_opts). */
typedef struct {
    int max_iters;       /* accepted steps; default 10 */
    double grad_tol;     /* relative gradient-norm stop; default 1e-6 */
    double c1;           /* Armijo sufficient-decrease constant; default 1e-4 */
    double beta;         /* backtracking factor; default 0.5 */
    int max_backtracks;  /* default 8 */
    double step0_mm;     /* first trial step moves w by this many mm; default 1 */
    int cold_start;      /* 1: start from w0 with a first trial step of step0_mm;
                            0: start from the model's last accepted w and step */
    double w0[PR_MAX_K];
    int loop_mode;       /* PR_LOOP_GRAPH (on-device loop in a CUDA graph) or PR_LOOP_HOST */
    double tumor_tol;    /* fixed-point stop, mm; default 1e-6 */
    int tumor_max_iter;  /* default 100 */
    double step_growth;    /* cap of the next first trial: step_growth x the accepted step
                              (step_model 0: used after a first-try acceptance); default 2 */
    double step_growth_bt; /* step_model 0: next first trial = step_growth_bt x an accepted
                              step that needed backtracking; default 1 */
    int warm_step;         /* 1: a warm-started solve also starts from the model's next
                              step (unless the last solve's line search failed); default 1 */
    int predict;           /* 1: a warm-started solve starts from 2 w(j-1) - w(j-2), the
                              linear prediction from the last two solves' final w
                              (Section 5's predicted coefficients); default 0 */
    int step_model;        /* 1: each trial measures the curvature of J along -g; a rejected
                              trial backtracks to the quadratic model's minimiser and the next
                              first trial is that minimiser (within [1/2, step_growth] x mu),
                              both rounded down to a power-of-two multiple of mu
                              (backtracking within [1/16, beta] x mu); the model is used only
                              where mu |g|^2 > 1e-6 J, elsewhere beta / step_growth apply;
                              0: backtrack by beta, growth factors only; default 1 */
} pr_solve_opts;

typedef struct {
    int K;
    double w[PR_MAX_K];     /* PCA coefficients (Eq. 1) */
    double a, b;            /* intensity fit (Eq. 4) */
    double J;               /* cost at (w, a, b) (Eq. 2) */
    double grad[PR_MAX_K];  /* dJ/dw at (w, a, b) */
    double grad_norm, grad_norm0;
    int iters;              /* accepted steps */
    int trials;             /* cost evaluations in line searches */
    int backtracks;
    int stop_reason;        /* PR_STOP_* */
    double tumor_xyz[3];    /* mm, Section 2.3 */
    int tumor_steps;
    double mu;              /* first trial step of the next warm-started solve (0 = none:
                               it moves w by step0_mm) */
} pr_result;

/* Library version string (static storage). */
const char* pr_version(void);

/* Message for the last failed call on this host thread (static storage per thread). */
const char* pr_last_error(void);

/* Fill *o with the defaults listed in pr_solve_opts. */
void pr_default_opts(pr_solve_opts* o);

/* Create a context on CUDA device `device`. `stream` is a cudaStream_t to run
 * on, or NULL to let the library create one. `hbm_budget_bytes` caps the
 * device memory of all loaded models (0 = 80% of the device memory free at
 * creation). Ownership of *out passes to the caller; release with pr_destroy. */
int pr_create(pr_ctx** out, int device, void* stream, size_t hbm_budget_bytes);

/* Free every model and buffer of the context; waits for its stream first. */
void pr_destroy(pr_ctx* ctx);

/* Section 2.1, Eq. 1: load one patient's motion model and scan geometry.
 * f0 [nz][ny][nx] reference volume (1/mm), mean_dvf [3][nz][ny][nx] (mm),
 * U [K][3][nz][ny][nx] eigenvector fields, 1 <= K <= PR_MAX_K, all float32 at
 * `location`. `storage` selects the device copy of f0 and U (PR_F32 or
 * PR_BF16, round-to-nearest-even; the mean stays float32). With PR_BF16 and
 * K = 4 or 5 the solver's intermediate derivative images h_k are also held
 * as float16 beside a float32 f (their ray sums and every reduction stay
 * float32/float64). tumor_ref_xyz is the
 * tumor centre in the reference image (mm), used by Section 2.3. The data are
 * copied into resident, immutable device buffers; the model's warm-start w is
 * set to 0. Returns PR_EADMIT if the model would exceed the HBM budget.
 * *model_id receives a handle. */
int pr_load_model(pr_ctx* ctx, const pr_volume_desc* vol, const pr_geometry* geom, int location,
                  const float* f0, const float* mean_dvf, const float* U, int K, int storage,
                  const double tumor_ref_xyz[3], int* model_id);

/* Release a model and its device buffers (or drop it from the admission
 * queue). Released memory admits waiting models in FIFO order (see
 * pr_set_admission_queue); their upload runs inside this call. */
int pr_release_model(pr_ctx* ctx, int model_id);

/* HBM admission queue (no counterpart in the paper; the serving use of
 * Section 4's real-time setting). Off by default: pr_load_model then fails
 * with PR_EADMIT when a model does not fit the context's budget. With
 * enable != 0, such a model (and every model loaded after it while any
 * waits) is instead queued: pr_load_model copies its inputs to host memory
 * owned by the library, assigns *model_id and returns PR_QUEUED. The model is
 * admitted (uploaded, made resident) as soon as releases free enough budget
 * for it, in loading order. Frames may be submitted for a waiting model: they
 * stay queued until it is admitted. Synchronous calls on a waiting model fail
 * with PR_ENOMODEL. A model larger than the whole budget still fails with
 * PR_EADMIT. */
int pr_set_admission_queue(pr_ctx* ctx, int enable);

enum { PR_MODEL_RESIDENT = 0, PR_MODEL_WAITING = 1 };

/* *status = PR_MODEL_RESIDENT or PR_MODEL_WAITING (admission queue).
 * Errors: PR_EINVAL, PR_ENOMODEL. */
int pr_model_status(pr_ctx* ctx, int model_id, int* status);

/* Device bytes held by a model (data, workspace, graph buffers). */
int pr_model_footprint(pr_ctx* ctx, int model_id, size_t* bytes);

/* Section 2.2 + 2.3: reconstruct from one projection y [nv][nu] (float32 at
 * y_location) at gantry angle `angle_rad`. opts NULL = defaults. Warm start:
 * unless opts->cold_start, w starts at the model's last accepted w, and the
 * final w becomes the next warm start (the paper initialises each frame from
 * the previous one, Section 4). volume_out (nullable, host) receives the
 * reconstructed image f [nz][ny][nx]. Synchronous. Errors: PR_EINVAL,
 * PR_ENOMODEL, PR_ECUDA. A solve that stops on a failed line search or a
 * non-finite value still returns PR_OK with out->stop_reason telling why. */
int pr_reconstruct(pr_ctx* ctx, int model_id, const float* y, int y_location, double angle_rad,
                   const pr_solve_opts* opts, pr_result* out, float* volume_out);

/* Several solves (Sections 2.2 and 2.3 each) in one CUDA graph launch, with
 * no host round trip between them: solve i reconstructs y[i] (host,
 * [nv][nu] float32 in the geometry of model model_ids[i]) at angles[i], as
 * pr_reconstruct would. Solves of one model run in the order given, each
 * warm-starting from the one before; solves of different models are
 * independent and run concurrently on the GPU. opts (nullable = defaults)
 * apply to every solve; the host loop mode is not allowed. out[i] receives
 * solve i's result. The instantiated graph is kept for the next call with the
 * same sequence of model ids (only the staged frames and parameters change);
 * a model release discards it. 1 <= n <= 4096. Synchronous; not while
 * serving. Errors: PR_EINVAL, PR_ENOMODEL, PR_ENOMEM, PR_ECUDA. */
int pr_reconstruct_batch(pr_ctx* ctx, int n, const int* model_ids, const float* const* y,
                         const double* angles, const pr_solve_opts* opts, pr_result* out);

/* As pr_reconstruct with a device-resident y, but only enqueues the solve on
 * the context stream and returns. y_dev is read by the enqueued work, so it
 * must stay valid and unchanged until pr_fetch_result returns. Fetch the
 * result with pr_fetch_result. */
int pr_reconstruct_async(pr_ctx* ctx, int model_id, const float* y_dev, double angle_rad,
                         const pr_solve_opts* opts);

/* Wait for the model's last enqueued solve and copy its result to *out. */
int pr_fetch_result(pr_ctx* ctx, int model_id, pr_result* out);

/* ---- serving: continuous submission of frames from many patients ----
 *
 * Requests are admitted into `slots` concurrent solve slots (one CUDA stream
 * each) as soon as a slot frees up and no earlier frame of the same model is
 * still in flight; different models' solves then overlap on the GPU, and each
 * model's frames run in submission order, each warm-started from the previous
 * (Section 4). Models are admitted to the device by pr_load_model's HBM
 * budget check (PR_EADMIT, or the admission queue of pr_set_admission_queue)
 * and can be loaded and released while serving. When serving stops, frames
 * of models still waiting for admission stay queued (a restart drops them). The
 * serving worker is a host thread of the context; while it runs, the
 * synchronous calls (pr_reconstruct, pr_warp, ...) must not be used on a
 * model that has submitted frames outstanding. */
typedef struct {
    uint64_t tag;       /* the caller's tag from pr_submit */
    int model_id;
    int status;         /* PR_OK or the error of this solve */
    pr_result result;
    double queue_ms;    /* submit to dispatch into a slot (host clock) */
    double gpu_ms;      /* slot mode: the solve's device time on its slot stream (CUDA events);
                           tick-batched mode: launch of its tick to its result (host clock) */
    double latency_ms;  /* submit to completion (host clock) */
} pr_served;

/* Start the serving worker with `slots` (1..64) concurrent solve streams
 * (after pr_serve_stop this restarts it; results not yet polled are dropped). */
int pr_serve_start(pr_ctx* ctx, int slots);

/* Start the serving worker in tick-batched mode: each tick gathers, in
 * submission order, the oldest pending frame of each resident model that has
 * no frame in flight (at most tick_frames of them; 0 = no limit) and runs
 * them all with ONE graph launch. The graph holds every resident
 * model's whole solve (Sections 2.2 and 2.3) as a branch behind a
 * conditional IF node; a first kernel switches on the branches of the models
 * the tick took, and the solves of those branches run concurrently on the
 * GPU. The graph is built once per set of resident models (again after a
 * load, release or admission) and only the staged frames and flags change
 * between ticks. `lanes` (1..8) ticks may be in flight at once, each on its
 * own stream and never sharing a model, so frames arriving during a tick are
 * taken by the next free lane. Each branch's last kernel writes its final
 * state into mapped host memory and raises a per-branch flag, so a frame's
 * result is taken as soon as its own solve finishes, and its model's next
 * frame can join another lane's tick while the rest of this tick runs.
 * Results are polled as in slot mode; each model's frames run in submission
 * order, each warm-started from the previous, and give the same results as
 * solved alone.
 * Errors: PR_EINVAL (lanes or tick_frames out of range, serving already
 * started), PR_ECUDA. */
int pr_serve_start_batched(pr_ctx* ctx, int lanes, int tick_frames);

/* Queue one frame: y [nv][nu] float32 (host, copied before return), gantry
 * angle, options (NULL = defaults; the host loop mode is not allowed), and a
 * tag returned with the result. Errors: PR_EINVAL, PR_ENOMODEL, PR_ECUDA
 * (an earlier device error of the worker). */
int pr_submit(pr_ctx* ctx, int model_id, const float* y, double angle_rad, const pr_solve_opts* opts,
              uint64_t tag);

/* Take one finished frame: waits up to timeout_ms (0 = do not wait, < 0 =
 * wait indefinitely while frames are outstanding). PR_OK with *out filled,
 * PR_ETIMEOUT if none finished in time, PR_EINVAL if nothing is outstanding. */
int pr_poll(pr_ctx* ctx, int timeout_ms, pr_served* out);

/* Wait for every submitted frame to finish (results stay pollable) and stop
 * the worker. */
int pr_serve_stop(pr_ctx* ctx);

/* Read / overwrite a model's warm-start coefficients (K doubles, host).
 * pr_set_state also forgets the warm-start step (the next solve's first
 * trial moves w by step0_mm) and the history used by `predict`. */
int pr_get_state(pr_ctx* ctx, int model_id, double* w);
int pr_set_state(pr_ctx* ctx, int model_id, const double* w);

/* Eq. 1 + Section 2.2 warp at coefficients w (K doubles, host):
 * f_dev [nz][ny][nx] (device, nullable) receives f(v) = f0(v + x(v));
 * h_dev [K][nz][ny][nx] (device, nullable) receives h_k = (df/dx) . u_k, the
 * exact derivative of the trilinear interpolant. Synchronous. */
int pr_warp(pr_ctx* ctx, int model_id, const double* w, float* f_dev, float* h_dev);

/* Eq. 2's projection matrix P applied to a caller volume f_dev [nz][ny][nx]
 * (device) on the grid `vol`, with geometry `geom` at `angle_rad`: p_dev
 * [nv][nu] (device). Synchronous. */
int pr_project(pr_ctx* ctx, const pr_volume_desc* vol, const pr_geometry* geom, double angle_rad,
               const float* f_dev, float* p_dev);

/* P^T (the transpose of pr_project, needed by the gradient formula after
 * Eq. 4) applied to r_dev [nv][nu] (device) by a voxel-driven gather:
 * g_dev [nz][ny][nx] (device). Synchronous. */
int pr_backproject(pr_ctx* ctx, const pr_volume_desc* vol, const pr_geometry* geom,
                   double angle_rad, const float* r_dev, float* g_dev);

/* Forward model for autograd: p_dev [nv][nu] (device) = P f(mean + U w), w
 * K doubles (host). Synchronous. */
int pr_forward(pr_ctx* ctx, int model_id, const double* w, double angle_rad, float* p_dev);

/* Vector-Jacobian product of pr_forward: grad_w[k] = sum over pixels of
 * grad_p * d p / d w_k = sum over voxels of (P^T grad_p)(v) h_k(v), computed
 * with the gather adjoint (the per-voxel P^T is never stored). grad_p_dev
 * [nv][nu] (device), grad_w K doubles (host). Synchronous. */
int pr_vjp(pr_ctx* ctx, int model_id, const double* w, double angle_rad, const float* grad_p_dev,
           double* grad_w);

/* One cost/gradient evaluation, the per-step quantity of Section 2.2: for
 * coefficients w and intensity terms (a, b), with y_dev [nv][nu] (device):
 * *J = ||P f - a y - b||^2 and grad[k] = dJ/dw_k = 2 sum_v (P^T r)(v) h_k(v),
 * r = P f - a y - b. mode 0 computes it in forward mode (sum over pixels of
 * 2 r (P h_k), the same number), mode 1 with the gather adjoint. p_dev
 * (device, nullable) receives P f. Synchronous. */
int pr_cost_grad(pr_ctx* ctx, int model_id, const float* y_dev, double angle_rad, const double* w,
                 double a, double b, int mode, double* J, double* grad, float* p_dev);

/* Section 2.3: tumor position for coefficients w (host, K doubles): the
 * fixed point p = c0 - x(p) of the pull-back DVF x = mean + U w (trilinear,
 * clamped to the grid edge), from p = c0, stopping when a step is below tol mm
 * or after max_iter steps. xyz (host) receives p, *steps the step count. */
int pr_tumor(pr_ctx* ctx, int model_id, const double* w, double tol, int max_iter, double* xyz,
             int* steps);

/* The line-search choices of the model's last solve, one byte per trial (no
 * counterpart in the paper; for checking a solve against a reference that
 * may break a rounding tie the other way): bit 7 the trial was accepted,
 * bit 6 it ended the solve (a rejected trial whose predicted decrease was
 * unresolvable, or an accepted one after which the gradient test was met),
 * bits 0-5 e + 32 with 2^e the factor that scaled the step next (0 when
 * step_model is 0). Copies min(trials, cap, 1024) bytes to out (host) and
 * sets *n to the number of trials. Synchronous. Errors: PR_EINVAL,
 * PR_ENOMODEL, PR_ECUDA. */
int pr_trial_log(pr_ctx* ctx, int model_id, unsigned char* out, int cap, int* n);

/* Measurement (no counterpart in the paper): the number of ray samples the
 * solver-pass projector evaluates for the model at angle_rad and coefficients
 * w (K doubles, host), summed over rays: each ray's samples inside the warped
 * volume's support box, less those at either end that the brick levels show
 * to be exactly zero. Synchronous. Errors: PR_EINVAL, PR_ENOMODEL, PR_ECUDA. */
int pr_count_samples(pr_ctx* ctx, int model_id, double angle_rad, const double* w, long long* count);

/* Measurement (no counterpart in the paper): the voxel box the solver's warp
 * pass (Eq. 1 and the pull-back of Section 2.2) evaluates at coefficients w
 * (K doubles, host): box[0..2] = lowest x, y, z voxel index, box[3..5] =
 * highest, clamped to the grid (empty when box[c] > box[3 + c]). Voxels
 * outside it lie farther than the displacement bound from every nonzero f0
 * voxel and are exact zeros: a chunk of the pass (512 consecutive voxels of
 * the flat grid) none of whose voxels is in the box writes its zeros without
 * reading a field, or is left alone where no earlier pass can have left a
 * nonzero in it. Synchronous. Errors: PR_EINVAL, PR_ENOMODEL, PR_ECUDA. */
int pr_warp_box(pr_ctx* ctx, int model_id, const double* w, int box[6]);

/* Section 5's fixed-angle geometry (fluoroscopy: the gantry does not move,
 * so P is the same matrix for every frame). Builds the model's table of the
 * transpose at angle_rad: for each voxel its detector footprint and the weight
 * of every footprint pixel (the sum of the trilinear hat over the pixel's ray
 * samples), about (footprint pixels) x N floats. pr_vjp and pr_cost_grad mode
 * 1 at exactly this angle then gather the stored weights instead of
 * recomputing them, with bitwise-identical results; other angles compute as
 * before. A NaN angle drops the table. The table counts against the HBM
 * budget (PR_EADMIT if it does not fit); *table_bytes (nullable) receives its
 * size. Synchronous. Errors: PR_EINVAL (infinite angle, detector wider than
 * 32767), PR_ENOMODEL, PR_EADMIT, PR_ENOMEM, PR_ECUDA. */
int pr_fix_angle(pr_ctx* ctx, int model_id, double angle_rad, size_t* table_bytes);

/* Section 2.3 with ref. 13 over the whole grid: the push-forward DVF y, the
 * inverse of the model's pull-back field x = mean + U w (w: K doubles, host),
 * i.e. u + y(u) + x(u + y(u)) = u at every voxel centre u, x interpolated
 * trilinearly with clamp to the grid edge. Chen et al.'s fixed point
 * y <- -x(u + y) from y = 0 is iterated at each voxel until its update is
 * below tol mm (Euclidean) or after max_iter (1..100000) updates. y_dev
 * [3][nz][ny][nx] float32 mm (device, caller-owned). max_steps (nullable)
 * receives the largest per-voxel update count, unconverged (nullable) the
 * number of voxels whose last update was not below tol. The model's solver
 * volume buffer is used as scratch (not while the model has frames in a
 * serving slot). Synchronous. Errors: PR_EINVAL (null w or y_dev, tol < 0,
 * max_iter out of range, a grid of 2^31 voxels or more), PR_ENOMODEL,
 * PR_ECUDA. */
int pr_invert_dvf(pr_ctx* ctx, int model_id, const double* w, double tol, int max_iter, float* y_dev,
                  int* max_steps, long long* unconverged);

/* ---- allocation-free cost and gradient (no counterpart in the paper) ----
 *
 * For callers that cannot allocate device memory while they run: a real-time
 * guidance loop that reserves all of its memory at start-up (a cudaMalloc can
 * synchronise the device and stall a frame), an application whose device
 * memory belongs to another allocator, or code where allocating is not
 * allowed at all. It computes, from projections the caller already has,
 *   out_dev[0]   = the cost: the sum over pixels of (p - a y - b)^2
 *   out_dev[1+k] = its derivative with respect to PCA coefficient k: twice
 *                  the sum over pixels of (p - a y - b) q_k, where q_k is the
 *                  projection of the image's derivative along mode k
 * with p_dev [R], q_dev [K][R], y_dev [R] float32 and out_dev [1 + K] double
 * (entries of out_dev past 1 + K are not touched),
 * all device memory of `device`, enqueued on `stream` (a cudaStream_t; NULL =
 * the legacy default stream) without a host synchronisation. It needs no
 * pr_ctx and allocates nothing: its scratch (block sums, a completion counter
 * and the outputs, 49,552 bytes) is one fixed array in the library that every
 * GPU which loads the library holds until the process exits. Limits: 1 <= K <=
 * PR_MAX_K (the array holds 1 + 7 sums per block), R >= 1; larger K is
 * rejected with PR_EINVAL. The first call on a device looks up that array's
 * device address (one-time set-up); make that first call before any stream
 * capture. All calls on a device share the array: calls whose work can
 * overlap on the GPU (different streams without ordering) race and give
 * wrong results; calls on one stream are safe. Errors: PR_EINVAL, PR_ECUDA,
 * with pr_last_error(). */
int pr_cost_grad_static(int device, void* stream, const float* p_dev, const float* q_dev, const float* y_dev,
                        int R, int K, double a, double b, double* out_dev);

/* ---- measurement (no counterpart in the paper; used by benchmarks) ---- */

/* Kernels pr_time_kernel can time. */
enum {
    PR_KERNEL_WARP_FH = 0,      /* fused DVF synthesis + warp writing f and h (solver pass) */
    PR_KERNEL_PROJECT_FH = 1,   /* ray-march projection of (f, h_1..h_K) (solver pass) */
    PR_KERNEL_REGRAD = 2,       /* residual, cost and gradient over the detector (pr_cost_grad) */
    PR_KERNEL_BACKPROJECT = 3,  /* gather transpose contracted with h (adjoint gradient; the
                                   fixed-angle table when pr_fix_angle built one at this angle) */
    PR_KERNEL_WARP_F = 4,       /* warp writing f only */
    PR_KERNEL_PROJECT_F = 5,    /* ray-march projection of f only */
    PR_KERNEL_INVERT = 6,       /* whole-grid DVF inversion (pr_invert_dvf, tol 1e-5 mm, 64 steps) */
    PR_KERNEL_PROJECT_FH_TRIAL = 7 /* the solver pass as a line-search trial runs it: projection with
                                      the moments and the controller (on a copy of the solve state) */
};

/* Launch kernel `which` `iters` times back to back on the context stream
 * at the model's current warm-start w and gantry angle `angle_rad`, and
 * return the mean device time per launch in *avg_ms (CUDA events recorded on
 * that stream). Overwrites the model's scratch buffers, not its warm start. */
int pr_time_kernel(pr_ctx* ctx, int model_id, int which, double angle_rad, int iters, double* avg_ms);

typedef struct {
    long long solves;   /* solves enqueued on this model since it was loaded */
    long long trials;   /* line-search trials run by those solves */
    long long kernels;  /* CUDA kernels those solves launched */
    long long iters;    /* accepted steps of those solves */
    long long line_search_failures;  /* those solves that stopped on a failed line search */
} pr_stats;

/* Cumulative counters of a model (waits for its enqueued work). */
int pr_model_stats(pr_ctx* ctx, int model_id, pr_stats* out);

/* Bytes one pr_reconstruct with a host y moves host-to-device (y and the
 * per-solve parameters) and device-to-host (the result record). */
int pr_io_bytes(pr_ctx* ctx, int model_id, size_t* h2d, size_t* d2h);

#ifdef __cplusplus
}
#endif

#endif /* PCARECON_H */
