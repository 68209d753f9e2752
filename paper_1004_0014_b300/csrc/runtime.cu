// C-ABI runtime of pcarecon: contexts, resident patient models with HBM
// admission, the per-model CUDA graph that runs Section 2.2's whole
// alternation on the device (a conditional WHILE node whose body is warp ->
// project, with the moments, the Armijo and stopping decisions taken in FP64
// by the projector's last finishing warp), batched solves in one graph, the
// serving worker, the host-driven loop used as the plain baseline, fixed-angle
// transpose tables, and the step-level entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "pcarecon.h"

using namespace pr;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(PR_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                             \
    } while (0)

struct Model {
    int id = 0;
    pr_volume_desc vol{};
    pr_geometry geom{};
    int K = 0, storage = 0, nch = 4;
    ModelDev md{};
    int R = 0;
    // device buffers
    void* f0p = nullptr;
    float* mean = nullptr;
    void* U = nullptr;
    float* fh = nullptr;    // padded, nch floats per voxel
    float* fpad = nullptr;  // padded planar f
    float* p = nullptr;     // [R]
    float* q = nullptr;     // [K][R]
    float* y = nullptr;     // [R]
    float* r = nullptr;     // [R]
    float* flat = nullptr;  // [N] scratch
    float* hbuf = nullptr;  // [K][N] scratch (adjoint paths, allocated on first use)
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    SolveState* st = nullptr;
    double* wdev = nullptr;   // 8 doubles: coefficients of step-level calls
    double* out = nullptr;    // 16 doubles: reduction outputs; [8..9] = (a, b)
    RayGeom* rg = nullptr;    // geometry of step-level calls
    int* steps = nullptr;
    int* order = nullptr;           // projector tile order
    int* order_w = nullptr;         // split projector's warp-tile order
    unsigned char* tlog = nullptr;  // per-trial choices of the last solve (kTrialLog bytes)
    // fixed-angle transpose table (pr_fix_angle); bt_bytes counted in `bytes`
    bool fixed = false;
    double fixed_angle = 0.0;
    short4* bt_rect = nullptr;
    float* bt_w = nullptr;
    size_t bt_bytes = 0;
    SplitScratch ss;                // split projector's scratch (order_w, parts, moments, counters)
    Support* sup = nullptr;         // where the warped volume can be nonzero
    unsigned char* lev = nullptr;   // brick levels of f0 (see SupportRef)
    int bn[3] = {0, 0, 0};
    SolveState* st_host = nullptr;  // pinned
    size_t bytes = 0;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle hloop = 0;
    int launches_per_solve_min = 0;
};

}  // namespace

int pr::set_last_error(int code, const char* msg) { return fail(code, "%s", msg); }

namespace {

// Serving: requests wait in a FIFO; a worker thread moves each into a free slot
// (its own CUDA stream) as soon as one frees up and no earlier frame of the
// same patient is still in flight, so different patients' solves overlap on
// the GPU while each patient's frames stay in order for the warm start.
struct ServeRequest {
    int model = 0;
    uint64_t tag = 0;
    double angle = 0.0;
    pr_solve_opts opts{};
    std::vector<float> y;
    std::chrono::steady_clock::time_point t_submit;
};

struct ServeSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    SolveState* host_state = nullptr;  // pinned
    float* y_pinned = nullptr;         // pinned staging of the frame's y (y_cap floats)
    size_t y_cap = 0;
    bool busy = false;
    ServeRequest req;
    std::chrono::steady_clock::time_point t_dispatch;
};

struct Batch;  // pr_reconstruct_batch's graph and staging (defined with it)

// Tick-batched serving: a lane is one CUDA graph over every resident model,
// each model's whole solve behind a conditional IF node whose flag a first
// kernel sets from the tick's staged `active` array. A tick stages the
// frames it takes (at most one per model), launches the graph once and copies
// the models' final states back; lanes run on their own streams and never
// share a model (a model with a frame in flight is not taken).
struct TickLane {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long epoch = -1;          // model-set epoch the graph was built for
    std::map<int, int> pos;        // model id -> branch index
    std::vector<size_t> y_off;     // branch -> offset of its frame in the staging (floats)
    int cap = 0;                   // branches the staging holds
    size_t y_cap = 0;              // floats of frame staging
    int* active = nullptr;         // device: branch flags
    cudaGraphConditionalHandle* handles = nullptr;  // device: the IF nodes' handles
    SolveParams* prm = nullptr;    // device: per-branch parameters
    float* y = nullptr;            // device: frames
    SolveState* res = nullptr;     // device: final states
    int* active_h = nullptr;       // pinned mirrors
    SolveParams* prm_h = nullptr;
    float* y_h = nullptr;
    // Results, written by each branch's last kernel straight into mapped
    // pinned host memory, then the branch's flag is set to the tick's
    // sequence number: the worker retires each frame as its branch finishes.
    SolveState* res_h = nullptr;   // mapped pinned (res: its device address)
    int* flag_h = nullptr;         // mapped pinned (flag: its device address)
    int* flag = nullptr;
    int seq = 0;                   // sequence number of the last tick (flags start at 0)
    bool busy = false;
    std::vector<ServeRequest> reqs;  // the frames of the tick in flight
    std::vector<char> retired;       // per frame: result already taken
    std::chrono::steady_clock::time_point t_dispatch;
};

struct Serve {
    std::thread worker;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeRequest> pending;
    std::deque<pr_served> done;
    std::vector<ServeSlot> slots;  // slot mode
    std::vector<TickLane> lanes;   // tick-batched mode
    int tick_frames = 0;           // most frames per tick (0 = every dispatchable frame)
    std::set<int> in_flight;  // models with a dispatched solve
    long long outstanding = 0;  // submitted and not yet polled into `done`
    bool stop = false;
    int error = 0;
    std::string error_msg;
};

// A model that did not fit the HBM budget when loaded with the admission
// queue on: its inputs (host copies) wait in FIFO order until released
// memory lets it in.
struct Waiting {
    int id = 0;
    pr_volume_desc vol{};
    pr_geometry geom{};
    int K = 0, storage = 0;
    double c0[3] = {0, 0, 0};
    std::vector<float> f0, mean, U;
    size_t need = 0;
};

}  // namespace

struct pr_ctx {
    int device = 0;
    std::mutex mu;           // models map and serving state (the worker thread reads both)
    Serve* serve = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, used = 0;
    int next_id = 1;
    std::map<int, Model*> models;
    long long model_epoch = 0;      // changes whenever a model is admitted or released
    bool admit_queue = false;       // over-budget models wait instead of failing
    std::deque<Waiting*> waiting;   // admission queue, FIFO
    float* pad = nullptr;  // scratch for pr_project
    size_t pad_cap = 0;
    RayGeom* rg = nullptr;
    Batch* batch = nullptr;  // graph and staging of pr_reconstruct_batch
};

namespace {

size_t pad_voxels(const pr_volume_desc& v) { return (size_t)(v.nx + 2) * (v.ny + 2) * (v.nz + 2); }

// Padded volumes are indexed with 32-bit arithmetic in the projector.
bool vol_ok(const pr_volume_desc* v) {
    return v && v->nx >= 1 && v->ny >= 1 && v->nz >= 1 && v->dx > 0 && v->dy > 0 && v->dz > 0 &&
           (double)(v->nx + 2) * (v->ny + 2) * (v->nz + 2) < 536870912.0 && isfinite(v->dx) && isfinite(v->dy) && isfinite(v->dz);
}

bool geom_ok(const pr_geometry* g) {
    return g && g->nu >= 1 && g->nv >= 1 && g->du > 0 && g->dv > 0 && g->sad > 0 && g->sdd > g->sad &&
           (double)g->nu * g->nv < 2.0e9 && isfinite(g->sad) && isfinite(g->sdd) && isfinite(g->du) &&
           isfinite(g->dv) && isfinite(g->ds);
}

double resolved_ds(const pr_volume_desc& v, const pr_geometry& g) {
    return g.ds > 0 ? g.ds : 0.5 * fmin(v.dx, fmin(v.dy, v.dz));
}

VolDev make_vd(const pr_volume_desc& v) {
    VolDev d;
    d.nx = v.nx;
    d.ny = v.ny;
    d.nz = v.nz;
    d.nxp = v.nx + 2;
    d.nyp = v.ny + 2;
    d.nzp = v.nz + 2;
    d.dx = (float)v.dx;
    d.dy = (float)v.dy;
    d.dz = (float)v.dz;
    d.inv_dx = (float)(1.0 / v.dx);
    d.inv_dy = (float)(1.0 / v.dy);
    d.inv_dz = (float)(1.0 / v.dz);
    d.n = (long long)v.nx * v.ny * v.nz;
    d.np = (long long)pad_voxels(v);
    return d;
}

// Ray geometry of gantry angle th (computed in FP64, stored in FP32).
RayGeom make_rg(const pr_volume_desc& v, const pr_geometry& g, double th) {
    RayGeom r;
    double st = sin(th), ct = cos(th);
    double S[3] = {g.sad * st, -g.sad * ct, 0.0};
    double eh[3] = {-st, ct, 0.0}, uh[3] = {ct, st, 0.0}, vh[3] = {0.0, 0.0, 1.0};
    double sp[3] = {v.dx, v.dy, v.dz};
    int n[3] = {v.nx, v.ny, v.nz};
    double cu = 0.5 * (g.nu - 1), cv = 0.5 * (g.nv - 1);
    for (int c = 0; c < 3; ++c) {
        double o = -0.5 * (n[c] - 1) * sp[c];
        r.a[c] = (float)((S[c] - o) / sp[c]);
        r.eu[c] = (float)(g.du * uh[c]);
        r.ev[c] = (float)(g.dv * vh[c]);
        r.d00[c] = (float)(g.sdd * eh[c] - cu * g.du * uh[c] - cv * g.dv * vh[c]);
        r.inv_sp[c] = (float)(1.0 / sp[c]);
        r.nmax[c] = (float)n[c];
        r.src[c] = (float)S[c];
        r.ehat[c] = (float)eh[c];
        r.pu[c] = (float)(uh[c] / g.du);
        r.pv[c] = (float)(vh[c] / g.dv);
        r.origin[c] = (float)o;
        r.sp[c] = (float)sp[c];
    }
    r.ds = (float)resolved_ds(v, g);
    r.nu = g.nu;
    r.nv = g.nv;
    r.cu = (float)cu;
    r.cv = (float)cv;
    r.sdd = (float)g.sdd;
    // Warp tile of the split projector: within 15 degrees of a volume axis the
    // detector's u direction runs along one axis and 4 x 8 pixels are fastest;
    // nearer the diagonals 2 x 16 keeps a warp's rays in fewer (x, y) columns
    // (measured crossover at paper scale).
    r.tile_u = fmin(fabs(st), fabs(ct)) < 0.2588190451 ? 4 : 2;
    return r;
}

// Brick levels of f0 (already in m->flat, unpadded): occupancy on the device,
// then a multi-source breadth-first search over the 26 neighbours on the host
// (level = Chebyshev distance in bricks to an occupied brick, capped at 255).
cudaError_t make_brick_levels(Launcher& L, Model* m, cudaStream_t s) {
    const size_t nb = (size_t)m->bn[0] * m->bn[1] * m->bn[2];
    cudaError_t e = cudaMemsetAsync(m->lev, 0, nb, s);
    if (!e) e = launch_brick_occ(L, m->md.vd, m->flat, m->lev);
    std::vector<unsigned char> lev(nb);
    if (!e) e = cudaMemcpyAsync(lev.data(), m->lev, nb, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return e;
    std::vector<int> q;
    q.reserve(nb);
    for (size_t b = 0; b < nb; ++b) {
        if (lev[b]) {
            lev[b] = 0;
            q.push_back((int)b);
        } else {
            lev[b] = 255;
        }
    }
    const int bx = m->bn[0], by = m->bn[1], bz = m->bn[2];
    for (size_t h = 0; h < q.size(); ++h) {
        const int b = q[h], x = b % bx, y = (b / bx) % by, z = b / (bx * by);
        const int next = lev[(size_t)b] + 1;
        if (next >= 255) continue;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int X = x + dx, Y = y + dy, Z = z + dz;
                    if (X < 0 || Y < 0 || Z < 0 || X >= bx || Y >= by || Z >= bz) continue;
                    const size_t nbi = ((size_t)Z * by + Y) * bx + X;
                    if (lev[nbi] > next) {
                        lev[nbi] = (unsigned char)next;
                        q.push_back((int)nbi);
                    }
                }
    }
    e = cudaMemcpyAsync(m->lev, lev.data(), nb, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);  // lev (host) lives until the copy is done
    return e;
}

// The projector's support description of model m at coefficients w (device).
SupportRef sref(const Model* m, const double* w) {
    SupportRef r;
    r.sup = m->sup;
    r.w = w;
    r.K = m->K;
    r.lev = m->lev;
    for (int c = 0; c < 3; ++c) r.bn[c] = m->bn[c];
    return r;
}

Model* find(pr_ctx* c, int id) {
    auto it = c->models.find(id);
    return it == c->models.end() ? nullptr : it->second;
}

template <typename T>
cudaError_t dalloc(T** p, size_t bytes, size_t* total) {
    *total += bytes;
    return cudaMalloc((void**)p, bytes);
}

void free_model(Model* m) {
    if (!m) return;
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->graph) cudaGraphDestroy(m->graph);
    void* bufs[] = {m->f0p, m->mean, m->U, m->fh, m->fpad, m->p, m->q, m->y, m->r, m->flat, m->hbuf,
                    m->partials, m->counter, m->st, m->wdev, m->out, m->rg, m->steps, m->order, m->sup,
                    m->order_w, m->ss.part, m->ss.tile_mom, m->ss.group_mom, m->ss.ctr, m->tlog,
                    m->bt_rect, m->bt_w, m->lev};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (m->st_host) cudaFreeHost(m->st_host);
    delete m;
}

// Scratch rows for block partials: the largest grid among the reductions.
size_t partial_rows(const pr_geometry& g, const VolDev& vd) {
    size_t a = project_blocks(g.nu, g.nv), b = reduce_blocks(), c = backproject_blocks(vd);
    size_t r = a > b ? a : b;
    return r > c ? r : c;
}

// Doubles of the block-partial buffer: the reductions' rows and the
// projector's wider moment rows.
size_t partial_doubles(const pr_geometry& g, const VolDev& vd) {
    size_t a = partial_rows(g, vd) * kMaxMom, b = (size_t)project_blocks(g.nu, g.nv) * kProjMom;
    return a > b ? a : b;
}

// Device bytes pr_load_model allocates for a model (the admission check uses
// this before allocating; the gradient-adjoint scratch of K x N floats is
// allocated on first use and added to the footprint then).
constexpr int kTrialLog = 1024;  // bytes of the per-solve trial log

size_t model_bytes(const pr_volume_desc& v, const pr_geometry& g, int K, int storage) {
    VolDev vd = make_vd(v);
    size_t n = (size_t)vd.n, np = (size_t)vd.np, R = (size_t)g.nu * g.nv;
    size_t ts = storage == PR_BF16 ? 2 : 4;
    const int layout = fh_layout(K, storage);
    size_t nch = (size_t)fh_logical(layout);
    return np * ts + 3 * n * 4 + 3 * (size_t)K * n * ts + np * (size_t)fh_floats(layout) * 4 + np * 4 + R * 4 + R * K * 4 + R * 4 +
           R * 4 + n * 4 + partial_doubles(g, vd) * 8 + 64 + sizeof(SolveState) + 64 + 128 +
           sizeof(RayGeom) + 16 + (size_t)project_blocks(g.nu, g.nv) * sizeof(int) + sizeof(Support) +
           (size_t)split_order_ints(g.nu, g.nv) * sizeof(int) + split_part_floats(g.nu, g.nv, (int)nch) * 4 +
           ((size_t)split_tiles(g.nu, g.nv) + split_groups(g.nu, g.nv)) * kProjMom * 8 +
           split_counters(g.nu, g.nv) * 4 + kTrialLog +
           (size_t)((v.nx + 3) / 4) * ((v.ny + 3) / 4) * ((v.nz + 3) / 4);
}

SolveParams make_params(const Model* m, double angle, const pr_solve_opts* o) {
    SolveParams prm;
    memset(&prm, 0, sizeof prm);
    prm.rg = make_rg(m->vol, m->geom, angle);
    for (int k = 0; k < 8; ++k) prm.w0[k] = (k < m->K && o->cold_start) ? o->w0[k] : 0.0;
    prm.c1 = o->c1;
    prm.beta = o->beta;
    prm.grad_tol = o->grad_tol;
    prm.step0 = o->step0_mm;
    prm.step_growth = o->step_growth;
    prm.step_growth_bt = o->step_growth_bt;
    prm.warm_step = o->warm_step ? 1 : 0;
    prm.predict = o->predict ? 1 : 0;
    prm.step_model = o->step_model;
    prm.tumor_tol = o->tumor_tol;
    prm.max_iters = o->max_iters;
    prm.max_bt = o->max_backtracks;
    prm.tumor_max_iter = o->tumor_max_iter;
    prm.K = m->K;
    prm.cold_start = o->cold_start ? 1 : 0;
    prm.tlog = m->tlog;
    prm.tlog_cap = kTrialLog;
    return prm;
}

int write_params(pr_ctx* c, Model* m, double angle, const pr_solve_opts* o, cudaStream_t stream) {
    SolveParams prm = make_params(m, angle, o);
    // Pageable source: the copy is staged before cudaMemcpyAsync returns, so
    // back-to-back asynchronous solves cannot see a later solve's parameters.
    CK(cudaMemcpyAsync(&m->st->prm, &prm, sizeof prm, cudaMemcpyHostToDevice, stream));
    return PR_OK;
}

bool opts_ok(const pr_solve_opts* o) {
    return o->max_iters >= 0 && o->max_iters <= 100000 && o->max_backtracks >= 0 && o->max_backtracks <= 200 &&
           o->beta > 0 && o->beta < 1 && o->c1 >= 0 && o->c1 < 1 && o->step0_mm > 0 && o->grad_tol >= 0 &&
           o->tumor_max_iter >= 0 && o->tumor_max_iter <= 100000 && o->tumor_tol >= 0 &&
           o->step_growth > 0 && o->step_growth <= 100 && o->step_growth_bt > 0 && o->step_growth_bt <= 100 &&
           (o->step_model == 0 || o->step_model == 1) &&
           (o->loop_mode == PR_LOOP_GRAPH || o->loop_mode == PR_LOOP_HOST);
}

// Section 2.2's loop as a CUDA graph: prologue (y moments; f and h at w0;
// projection, whose last finishing warp fits Eq. 4 and forms the cost and
// gradient), a WHILE node whose body is one line-search trial (warp, then
// projection with the Armijo test, Eq. 4, cost, gradient and stopping rule in
// the warp that completes it), and the Section 2.3 tumor kernel.
int build_graph(pr_ctx* c, Model* m) {
    CK(cudaGraphCreate(&m->graph, 0));
    CK(cudaGraphConditionalHandleCreate(&m->hloop, m->graph, 1, cudaGraphCondAssignDefault));
    Launcher L;
    L.graph = m->graph;
    SolveState* st = m->st;
    CK(launch_begin(L, m->y, m->R, st, m->partials, m->counter));
    CK(launch_warp(L, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
    L.programmatic_next = true;  // the projector waits for the warp before sampling
    CK(launch_project(L, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y, st,
                      m->partials, m->counter, kPhaseInit, m->hloop, 1, sref(m, st->wt), &m->ss));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = m->hloop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond;
    CK(cudaGraphAddNode(&cond, m->graph, &L.last, nullptr, 1, &cp));
    Launcher B;
    B.graph = cp.conditional.phGraph_out[0];
    CK(launch_warp(B, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
    B.programmatic_next = true;  // the projector waits for the warp before sampling
    CK(launch_project(B, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y, st,
                      m->partials, m->counter, kPhaseTrial, m->hloop, 1, sref(m, st->wt), &m->ss));
    L.last = cond;
    CK(launch_tumor(L, m->md, st->w, 0.0, 0, &st->prm, st->tumor, &st->tumor_steps));
    CK(cudaGraphInstantiate(&m->exec, m->graph, 0));
    return PR_OK;
}

// The same alternation driven from the host: one device-to-host read of the
// loop flag per line-search trial (the plain baseline).
int host_loop(pr_ctx* c, Model* m, int opt_max_iters, int opt_max_bt) {
    Launcher L;
    L.stream = c->stream;
    SolveState* st = m->st;
    CK(launch_begin(L, m->y, m->R, st, m->partials, m->counter));
    CK(launch_warp(L, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
    CK(launch_project(L, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y, st,
                      m->partials, m->counter, kPhaseInit, 0, 0, sref(m, st->wt), &m->ss));
    long long guard = 0, bound = (long long)(opt_max_iters + 1) * (opt_max_bt + 1) + 2;
    for (;;) {
        CK(cudaMemcpyAsync(&m->st_host->running, &st->running, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (!m->st_host->running) break;
        if (++guard > bound) return fail(PR_ETIMEOUT, "host loop exceeded its trial bound");
        CK(launch_warp(L, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
        CK(launch_project(L, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y,
                          st, m->partials, m->counter, kPhaseTrial, 0, 0, sref(m, st->wt), &m->ss));
        }
    CK(launch_tumor(L, m->md, st->w, 0.0, 0, &st->prm, st->tumor, &st->tumor_steps));
    return PR_OK;
}

void fill_result(const Model* m, const SolveState& s, pr_result* out) {
    memset(out, 0, sizeof *out);
    out->K = m->K;
    for (int k = 0; k < m->K; ++k) {
        out->w[k] = s.w[k];
        out->grad[k] = s.g[k];
    }
    out->a = s.a;
    out->b = s.b;
    out->J = s.J;
    out->grad_norm = s.gnorm;
    out->grad_norm0 = s.gnorm0;
    out->iters = s.iter;
    out->trials = s.trials;
    out->backtracks = s.total_bt;
    out->stop_reason = s.stop;
    for (int c = 0; c < 3; ++c) out->tumor_xyz[c] = s.tumor[c];
    out->tumor_steps = s.tumor_steps;
    out->mu = s.mu_next;
}

int enqueue_solve(pr_ctx* c, Model* m, double angle, const pr_solve_opts* opts) {
    pr_solve_opts o;
    if (opts)
        o = *opts;
    else
        pr_default_opts(&o);
    if (!opts_ok(&o)) return fail(PR_EINVAL, "invalid solve options");
    if (!isfinite(angle)) return fail(PR_EINVAL, "angle is not finite");
    int rc = write_params(c, m, angle, &o, c->stream);
    if (rc) return rc;
    if (o.loop_mode == PR_LOOP_HOST) return host_loop(c, m, o.max_iters, o.max_backtracks);
    if (!m->exec) {
        rc = build_graph(c, m);
        if (rc) return rc;
    }
    CK(cudaGraphLaunch(m->exec, c->stream));
    return PR_OK;
}

// The fixed-angle transpose table of m if it was built for exactly this angle.
BpTable bp_table(const Model* m, double angle) {
    BpTable t;
    if (m->fixed && m->bt_w && angle == m->fixed_angle) {
        t.rect = m->bt_rect;
        t.w = m->bt_w;
    }
    return t;
}

void drop_bp_table(pr_ctx* c, Model* m) {
    if (m->bt_rect) cudaFree(m->bt_rect);
    if (m->bt_w) cudaFree(m->bt_w);
    m->bt_rect = nullptr;
    m->bt_w = nullptr;
    m->fixed = false;
    std::lock_guard<std::mutex> lock(c->mu);
    m->bytes -= m->bt_bytes;
    c->used -= m->bt_bytes;
    m->bt_bytes = 0;
}

// The adjoint's h scratch (K x N floats), allocated on first use and charged
// to the model and the context like the rest of the model.
int ensure_hbuf(pr_ctx* c, Model* m) {
    if (m->hbuf) return PR_OK;
    const size_t bytes = (size_t)m->K * m->md.vd.n * 4;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        if (c->used + bytes > c->budget)
            return fail(PR_EADMIT, "adjoint scratch of %zu bytes exceeds the HBM budget", bytes);
        c->used += bytes;
    }
    if (cudaMalloc(&m->hbuf, bytes) != cudaSuccess) {
        cudaGetLastError();
        m->hbuf = nullptr;
        std::lock_guard<std::mutex> lock(c->mu);
        c->used -= bytes;
        return fail(PR_ENOMEM, "adjoint scratch of %zu bytes: allocation failed", bytes);
    }
    std::lock_guard<std::mutex> lock(c->mu);
    m->bytes += bytes;
    return PR_OK;
}

int set_w(pr_ctx* c, Model* m, const double* w) {
    double buf[8] = {0};
    for (int k = 0; k < m->K; ++k) {
        if (!isfinite(w[k])) return fail(PR_EINVAL, "w[%d] is not finite", k);
        buf[k] = w[k];
    }
    CK(cudaMemcpyAsync(m->wdev, buf, sizeof buf, cudaMemcpyHostToDevice, c->stream));
    return PR_OK;
}

int set_rg(pr_ctx* c, RayGeom* dst, const pr_volume_desc& v, const pr_geometry& g, double angle) {
    if (!isfinite(angle)) return fail(PR_EINVAL, "angle is not finite");
    RayGeom rg = make_rg(v, g, angle);
    CK(cudaMemcpyAsync(dst, &rg, sizeof rg, cudaMemcpyHostToDevice, c->stream));
    return PR_OK;
}

#define TRY(x)                 \
    do {                       \
        int rc_ = (x);         \
        if (rc_) return rc_;   \
    } while (0)

#define GET_MODEL(c, id, m)                                                    \
    if (!(c)) return fail(PR_EINVAL, "null context");                          \
    Model* m = find((c), (id));                                                \
    if (!m) return fail(PR_ENOMODEL, "unknown model id %d", (int)(id));        \
    CK(cudaSetDevice((c)->device))

double ms_between(std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Worker: retire finished slots, then fill free slots with the oldest request
// whose model has nothing in flight. Runs until stopped and idle.
// ---------------------------------------------------------------------------
// Batched solves in one graph (pr_reconstruct_batch)
// ---------------------------------------------------------------------------
// One CUDA graph holds every solve of a batch. A solve is a chain of nodes:
// copy its y and parameters from the batch's staging arrays into the model,
// the solve's kernels with a conditional WHILE of its own, the tumor, and a
// copy of the final state into the batch's result array. Solves of one model
// are chained in batch order (each warm-starts from the one before); solves
// of different models are independent branches that the GPU runs
// concurrently. The instantiated graph is kept while the batch's model
// sequence repeats; only the staged data change between launches.
struct Batch {
    std::vector<int> key;  // model ids in batch order
    std::vector<size_t> y_off;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float* y = nullptr;  // staged frames (device)
    size_t y_cap = 0;
    SolveParams* prm = nullptr;  // staged parameters (device)
    SolveState* res = nullptr;   // final states (device)
    SolveState* res_host = nullptr;  // pinned
    int cap = 0;
};

void batch_drop_graph(Batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->key.clear();
}

void batch_free(pr_ctx* c) {
    Batch* b = c->batch;
    if (!b) return;
    batch_drop_graph(b);
    if (b->y) cudaFree(b->y);
    if (b->prm) cudaFree(b->prm);
    if (b->res) cudaFree(b->res);
    if (b->res_host) cudaFreeHost(b->res_host);
    delete b;
    c->batch = nullptr;
}

int add_solve_nodes(cudaGraph_t g, Model* m, const cudaGraphNode_t* dep, const float* y_src, const SolveParams* prm_src,
                    SolveState* res_dst, cudaGraphNode_t* last) {
    SolveState* st = m->st;
    cudaGraphNode_t ny, np, nr;
    CK(cudaGraphAddMemcpyNode1D(&ny, g, dep, dep ? 1 : 0, m->y, y_src, (size_t)m->R * 4, cudaMemcpyDeviceToDevice));
    CK(cudaGraphAddMemcpyNode1D(&np, g, &ny, 1, &st->prm, prm_src, sizeof(SolveParams), cudaMemcpyDeviceToDevice));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    Launcher L;
    L.graph = g;
    L.last = np;
    L.has_last = true;
    CK(launch_begin(L, m->y, m->R, st, m->partials, m->counter));
    CK(launch_warp(L, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
    L.programmatic_next = true;  // the projector waits for the warp before sampling
    CK(launch_project(L, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y, st,
                      m->partials, m->counter, kPhaseInit, h, 1, sref(m, st->wt), &m->ss));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond;
    CK(cudaGraphAddNode(&cond, g, &L.last, nullptr, 1, &cp));
    Launcher B;
    B.graph = cp.conditional.phGraph_out[0];
    CK(launch_warp(B, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
    B.programmatic_next = true;  // the projector waits for the warp before sampling
    CK(launch_project(B, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y, st,
                      m->partials, m->counter, kPhaseTrial, h, 1, sref(m, st->wt), &m->ss));
    L.last = cond;
    CK(launch_tumor(L, m->md, st->w, 0.0, 0, &st->prm, st->tumor, &st->tumor_steps));
    CK(cudaGraphAddMemcpyNode1D(&nr, g, &L.last, 1, res_dst, st, sizeof(SolveState), cudaMemcpyDeviceToDevice));
    *last = nr;
    return PR_OK;
}

int build_batch_graph(Batch* b, const std::vector<Model*>& ms) {
    batch_drop_graph(b);
    CK(cudaGraphCreate(&b->graph, 0));
    std::map<const Model*, cudaGraphNode_t> tail;
    for (size_t i = 0; i < ms.size(); ++i) {
        auto it = tail.find(ms[i]);
        cudaGraphNode_t last;
        TRY(add_solve_nodes(b->graph, ms[i], it == tail.end() ? nullptr : &it->second, b->y + b->y_off[i], b->prm + i,
                            b->res + i, &last));
        tail[ms[i]] = last;
    }
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return PR_OK;
}

// ---------------------------------------------------------------------------
// Tick-batched serving lanes
// ---------------------------------------------------------------------------

// Sets each branch's IF flag from the tick's staged flags.
__global__ void k_tick_set(const int* __restrict__ active, const cudaGraphConditionalHandle* __restrict__ h, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cudaGraphSetConditional(h[i], active[i] ? 1u : 0u);
}

// Word copy (the branch's staging -> model transfers inside the graph).
__global__ void k_copy_words(const unsigned int* __restrict__ src, unsigned int* __restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// A branch's last kernel (one block): its final state into host memory, then,
// once every thread's stores are visible to the host, the branch's flag set to
// the tick's sequence number (its entry of the staged flags).
__global__ void k_publish(const unsigned int* __restrict__ st, unsigned int* res, size_t n, volatile int* flag,
                          const int* __restrict__ seq) {
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) res[i] = st[i];
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) *flag = *seq;
}

constexpr int kMaxLaneModels = 1024;

void lane_free_graph(TickLane& ln) {
    if (ln.exec) cudaGraphExecDestroy(ln.exec);
    if (ln.graph) cudaGraphDestroy(ln.graph);
    ln.exec = nullptr;
    ln.graph = nullptr;
    ln.epoch = -1;
}

void lane_free(TickLane& ln) {
    lane_free_graph(ln);
    void* dev[] = {ln.active, ln.handles, ln.prm, ln.y};
    for (void* d : dev)
        if (d) cudaFree(d);
    void* host[] = {ln.active_h, ln.prm_h, ln.y_h, ln.res_h, ln.flag_h};
    for (void* h : host)
        if (h) cudaFreeHost(h);
    ln.active = nullptr, ln.handles = nullptr, ln.prm = nullptr, ln.y = nullptr, ln.res = nullptr;
    ln.active_h = nullptr, ln.prm_h = nullptr, ln.y_h = nullptr, ln.res_h = nullptr, ln.flag_h = nullptr;
    ln.flag = nullptr;
    ln.cap = 0, ln.y_cap = 0;
}

// One branch: frame and parameters from the staging into the model, the
// whole solve (Section 2.2 with its own WHILE node, then Section 2.3), the
// final state into the staging.
int add_tick_branch(cudaGraph_t body, Model* m, const float* y_src, const SolveParams* prm_src, SolveState* res_dst,
                    int* flag, const int* seq) {
    SolveState* st = m->st;
    Launcher L;
    L.graph = body;
    CK(L(k_copy_words, dim3(48), dim3(256), 0, reinterpret_cast<const unsigned int*>(y_src),
         reinterpret_cast<unsigned int*>(m->y), (size_t)m->R));
    CK(L(k_copy_words, dim3(1), dim3(256), 0, reinterpret_cast<const unsigned int*>(prm_src),
         reinterpret_cast<unsigned int*>(&st->prm), sizeof(SolveParams) / 4));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, body, 1, cudaGraphCondAssignDefault));
    CK(launch_begin(L, m->y, m->R, st, m->partials, m->counter));
    CK(launch_warp(L, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
    L.programmatic_next = true;  // the projector waits for the warp before sampling
    CK(launch_project(L, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y, st,
                      m->partials, m->counter, kPhaseInit, h, 1, sref(m, st->wt), &m->ss));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond;
    CK(cudaGraphAddNode(&cond, body, &L.last, nullptr, 1, &cp));
    Launcher B;
    B.graph = cp.conditional.phGraph_out[0];
    CK(launch_warp(B, m->md, st->wt, kWarpFH, m->fh, nullptr, nullptr, m->sup, st->fh_box));
    B.programmatic_next = true;  // the projector waits for the warp before sampling
    CK(launch_project(B, m->md.vd, m->fh, m->nch, m->K, &st->prm.rg, m->order, m->geom.nu, m->geom.nv, m->p, m->q, m->y, st,
                      m->partials, m->counter, kPhaseTrial, h, 1, sref(m, st->wt), &m->ss));
    L.last = cond;
    CK(launch_tumor(L, m->md, st->w, 0.0, 0, &st->prm, st->tumor, &st->tumor_steps));
    CK(L(k_publish, dim3(1), dim3(128), 0, reinterpret_cast<const unsigned int*>(st),
         reinterpret_cast<unsigned int*>(res_dst), sizeof(SolveState) / 4, (volatile int*)flag, seq));
    return PR_OK;
}

// (Re)build a lane's graph over the resident models `ms` (id order), growing
// its staging as needed. Called with the context lock held, so no model can
// be released meanwhile.
int build_lane(TickLane& ln, const std::vector<Model*>& ms, long long epoch) {
    lane_free_graph(ln);
    const int n = (int)ms.size();
    if (n > kMaxLaneModels) return fail(PR_EUNSUPPORTED, "more than %d models in a serving lane", kMaxLaneModels);
    std::vector<size_t> off((size_t)n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        off[(size_t)i] = total;
        total += ((size_t)ms[(size_t)i]->R + 3) / 4 * 4;
    }
    if (ln.cap < n || ln.y_cap < total) {
        const int cap = std::max(n, 1);
        const size_t ycap = std::max<size_t>(total, 4);
        void* dev[] = {ln.active, ln.handles, ln.prm, ln.y};
        for (void* d : dev)
            if (d) cudaFree(d);
        void* host[] = {ln.active_h, ln.prm_h, ln.y_h, ln.res_h, ln.flag_h};
        for (void* h : host)
            if (h) cudaFreeHost(h);
        ln.active = nullptr, ln.handles = nullptr, ln.prm = nullptr, ln.y = nullptr, ln.res = nullptr;
        ln.active_h = nullptr, ln.prm_h = nullptr, ln.y_h = nullptr, ln.res_h = nullptr, ln.flag_h = nullptr;
        ln.flag = nullptr, ln.seq = 0;
        ln.cap = 0, ln.y_cap = 0;
        cudaError_t e = cudaMalloc(&ln.active, (size_t)cap * sizeof(int));
        if (!e) e = cudaMalloc(&ln.handles, (size_t)cap * sizeof(cudaGraphConditionalHandle));
        if (!e) e = cudaMalloc(&ln.prm, (size_t)cap * sizeof(SolveParams));
        if (!e) e = cudaMalloc(&ln.y, ycap * 4);
        if (!e) e = cudaHostAlloc((void**)&ln.active_h, (size_t)cap * sizeof(int), cudaHostAllocDefault);
        if (!e) e = cudaHostAlloc((void**)&ln.prm_h, (size_t)cap * sizeof(SolveParams), cudaHostAllocDefault);
        if (!e) e = cudaHostAlloc((void**)&ln.y_h, ycap * 4, cudaHostAllocDefault);
        if (!e) e = cudaHostAlloc((void**)&ln.res_h, (size_t)cap * sizeof(SolveState), cudaHostAllocMapped);
        if (!e) e = cudaHostAlloc((void**)&ln.flag_h, (size_t)cap * sizeof(int), cudaHostAllocMapped);
        if (!e) e = cudaHostGetDevicePointer((void**)&ln.res, ln.res_h, 0);
        if (!e) e = cudaHostGetDevicePointer((void**)&ln.flag, ln.flag_h, 0);
        if (!e) memset(ln.flag_h, 0, (size_t)cap * sizeof(int));
        if (e) {
            cudaGetLastError();
            return fail(PR_ENOMEM, "serving lane staging: %s", cudaGetErrorString(e));
        }
        ln.cap = cap;
        ln.y_cap = ycap;
    }
    CK(cudaGraphCreate(&ln.graph, 0));
    std::vector<cudaGraphConditionalHandle> hs((size_t)n);
    for (int i = 0; i < n; ++i) CK(cudaGraphConditionalHandleCreate(&hs[(size_t)i], ln.graph, 0, cudaGraphCondAssignDefault));
    if (n > 0)
        CK(cudaMemcpy(ln.handles, hs.data(), (size_t)n * sizeof(cudaGraphConditionalHandle), cudaMemcpyHostToDevice));
    Launcher L;
    L.graph = ln.graph;
    CK(L(k_tick_set, dim3(1), dim3((unsigned)std::max(32, (n + 31) / 32 * 32)), 0, (const int*)ln.active,
         (const cudaGraphConditionalHandle*)ln.handles, n));
    const cudaGraphNode_t root = L.last;
    ln.pos.clear();
    for (int i = 0; i < n; ++i) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hs[(size_t)i];
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, ln.graph, &root, nullptr, 1, &cp));
        TRY(add_tick_branch(cp.conditional.phGraph_out[0], ms[(size_t)i], ln.y + off[(size_t)i], ln.prm + i, ln.res + i,
                            ln.flag + i, ln.active + i));
        ln.pos[ms[(size_t)i]->id] = i;
    }
    CK(cudaGraphInstantiate(&ln.exec, ln.graph, 0));
    ln.y_off = off;
    ln.epoch = epoch;
    return PR_OK;
}

// Stage one tick's frames into the lane and launch it (lock not held; the
// chosen models have frames in flight, so they stay resident).
cudaError_t launch_tick(TickLane& ln, const std::vector<std::pair<Model*, const ServeRequest*>>& work) {
    const int n = (int)ln.y_off.size();
    memset(ln.active_h, 0, (size_t)n * sizeof(int));
    ln.seq = ln.seq == 0x7fffffff ? 1 : ln.seq + 1;
    cudaError_t e = cudaEventRecord(ln.start, ln.stream);
    for (const auto& wr : work) {
        Model* m = wr.first;
        const ServeRequest* r = wr.second;
        const int i = ln.pos.at(m->id);
        ln.active_h[i] = ln.seq;  // switches the branch on; its result flag will carry this value
        ln.prm_h[i] = make_params(m, r->angle, &r->opts);
        memcpy(ln.y_h + ln.y_off[(size_t)i], r->y.data(), (size_t)m->R * 4);
        if (!e) e = cudaMemcpyAsync(ln.y + ln.y_off[(size_t)i], ln.y_h + ln.y_off[(size_t)i], (size_t)m->R * 4,
                                    cudaMemcpyHostToDevice, ln.stream);
    }
    if (!e) e = cudaMemcpyAsync(ln.prm, ln.prm_h, (size_t)n * sizeof(SolveParams), cudaMemcpyHostToDevice, ln.stream);
    if (!e) e = cudaMemcpyAsync(ln.active, ln.active_h, (size_t)n * sizeof(int), cudaMemcpyHostToDevice, ln.stream);
    if (!e) e = cudaGraphLaunch(ln.exec, ln.stream);
    if (!e) e = cudaEventRecord(ln.done, ln.stream);
    return e;
}

// Worker of the tick-batched mode: retire finished ticks, then give every
// free lane the oldest pending frame of each resident model that has nothing
// in flight, as one launch.
void serve_loop_ticks(pr_ctx* c) {
    cudaSetDevice(c->device);
    Serve* sv = c->serve;
    std::unique_lock<std::mutex> lock(c->mu);
    for (;;) {
        bool busy = false, progressed = false;
        for (TickLane& ln : sv->lanes) {
            if (!ln.busy) continue;
            // frames whose branch has published its result: retire them now,
            // so that their models can take part in the next free lane's tick
            const auto now = std::chrono::steady_clock::now();
            for (size_t k = 0; k < ln.reqs.size(); ++k) {
                if (ln.retired[k]) continue;
                const ServeRequest& r = ln.reqs[k];
                const int i = ln.pos.at(r.model);
                if (reinterpret_cast<volatile int*>(ln.flag_h)[i] != ln.seq) continue;
                std::atomic_thread_fence(std::memory_order_acquire);
                SolveState st_copy;
                memcpy(&st_copy, (const void*)(ln.res_h + i), sizeof st_copy);
                pr_served out;
                memset(&out, 0, sizeof out);
                out.tag = r.tag;
                out.model_id = r.model;
                Model* m = find(c, r.model);
                if (m) fill_result(m, st_copy, &out.result);
                out.queue_ms = ms_between(r.t_submit, ln.t_dispatch);
                out.gpu_ms = ms_between(ln.t_dispatch, now);
                out.latency_ms = ms_between(r.t_submit, now);
                sv->in_flight.erase(r.model);
                sv->done.push_back(out);
                ln.retired[k] = 1;
                progressed = true;
            }
            if (progressed) sv->cv_done.notify_all();
            cudaError_t q = cudaEventQuery(ln.done);
            if (q == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            // the tick is over: its branches' flags, written before the graph
            // completed, are all visible now; anything not retired failed
            std::atomic_thread_fence(std::memory_order_acquire);
            const auto end = std::chrono::steady_clock::now();
            for (size_t k = 0; k < ln.reqs.size(); ++k) {
                if (ln.retired[k]) continue;
                const ServeRequest& r = ln.reqs[k];
                const int i = ln.pos.at(r.model);
                pr_served out;
                memset(&out, 0, sizeof out);
                out.tag = r.tag;
                out.model_id = r.model;
                Model* m = find(c, r.model);
                if (q == cudaSuccess && m && reinterpret_cast<volatile int*>(ln.flag_h)[i] == ln.seq) {
                    SolveState st_copy;
                    memcpy(&st_copy, (const void*)(ln.res_h + i), sizeof st_copy);
                    fill_result(m, st_copy, &out.result);
                    out.queue_ms = ms_between(r.t_submit, ln.t_dispatch);
                    out.gpu_ms = ms_between(ln.t_dispatch, end);
                    out.latency_ms = ms_between(r.t_submit, end);
                } else {
                    out.status = PR_ECUDA;
                    sv->error = PR_ECUDA;
                    sv->error_msg = q != cudaSuccess ? std::string("served tick failed: ") + cudaGetErrorString(q)
                                                     : std::string("a served branch finished without its result");
                }
                sv->in_flight.erase(r.model);
                sv->done.push_back(out);
            }
            ln.reqs.clear();
            ln.retired.clear();
            ln.busy = false;
            sv->cv_done.notify_all();
            progressed = true;
        }
        bool dispatchable = false;
        for (TickLane& ln : sv->lanes) {
            if (ln.busy || sv->error) continue;
            std::vector<ServeRequest> chosen;
            std::set<int> taken;
            for (auto it = sv->pending.begin(); it != sv->pending.end();) {
                if (sv->tick_frames > 0 && (int)chosen.size() >= sv->tick_frames) break;
                if (!sv->in_flight.count(it->model) && !taken.count(it->model) && find(c, it->model)) {
                    taken.insert(it->model);
                    chosen.push_back(std::move(*it));
                    it = sv->pending.erase(it);
                } else {
                    ++it;
                }
            }
            if (chosen.empty()) break;
            dispatchable = true;
            int rc = PR_OK;
            if (ln.epoch != c->model_epoch) {
                std::vector<Model*> ms;
                for (auto& kv : c->models) ms.push_back(kv.second);
                rc = build_lane(ln, ms, c->model_epoch);
            }
            std::vector<std::pair<Model*, const ServeRequest*>> work;
            for (const ServeRequest& r : chosen) {
                work.push_back({find(c, r.model), &r});
                sv->in_flight.insert(r.model);
            }
            ln.busy = true;
            ln.t_dispatch = std::chrono::steady_clock::now();
            cudaError_t e = rc ? cudaErrorUnknown : cudaSuccess;
            if (!e) {
                lock.unlock();
                e = launch_tick(ln, work);
                lock.lock();
            }
            if (e) {
                ln.busy = false;
                sv->error = PR_ECUDA;
                sv->error_msg = rc ? std::string("serving lane build failed: ") + g_err
                                   : std::string("tick dispatch failed: ") + cudaGetErrorString(e);
                for (const ServeRequest& r : chosen) {
                    sv->in_flight.erase(r.model);
                    pr_served out;
                    memset(&out, 0, sizeof out);
                    out.tag = r.tag;
                    out.model_id = r.model;
                    out.status = PR_ECUDA;
                    sv->done.push_back(out);
                }
                sv->cv_done.notify_all();
                continue;
            }
            for (ServeRequest& r : chosen) {
                r.y.clear();
                r.y.shrink_to_fit();
            }
            ln.retired.assign(chosen.size(), 0);
            ln.reqs = std::move(chosen);
            busy = true;
            progressed = true;
        }
        // Stop once idle; frames of models still waiting for admission stay
        // queued, and after an error nothing more is dispatched.
        if (sv->stop && !busy && !dispatchable) {
            bool any = false;
            for (const ServeRequest& r : sv->pending) any = any || find(c, r.model) != nullptr;
            if (!any || sv->error) break;
        }
        if (busy && !progressed) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        } else if (!busy && !progressed) {
            sv->cv_work.wait_for(lock, std::chrono::milliseconds(50));
        }
    }
}

void serve_loop(pr_ctx* c) {
    cudaSetDevice(c->device);
    Serve* sv = c->serve;
    std::unique_lock<std::mutex> lock(c->mu);
    for (;;) {
        bool busy = false, progressed = false;
        for (ServeSlot& sl : sv->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            pr_served out;
            memset(&out, 0, sizeof out);
            out.tag = sl.req.tag;
            out.model_id = sl.req.model;
            Model* m = find(c, sl.req.model);
            if (q != cudaSuccess) {
                out.status = PR_ECUDA;
                sv->error = PR_ECUDA;
                sv->error_msg = std::string("served solve failed: ") + cudaGetErrorString(q);
            } else if (m) {
                fill_result(m, *sl.host_state, &out.result);
                float g = 0.0f;
                cudaEventElapsedTime(&g, sl.start, sl.done);
                out.gpu_ms = g;
            }
            auto now = std::chrono::steady_clock::now();
            out.queue_ms = ms_between(sl.req.t_submit, sl.t_dispatch);
            out.latency_ms = ms_between(sl.req.t_submit, now);
            sv->in_flight.erase(sl.req.model);
            sl.busy = false;
            sl.req.y.clear();
            sv->done.push_back(out);
            sv->cv_done.notify_all();
            progressed = true;
        }
        for (ServeSlot& sl : sv->slots) {
            if (sl.busy || sv->error) continue;
            auto it = sv->pending.begin();
            while (it != sv->pending.end() && (sv->in_flight.count(it->model) || !find(c, it->model))) ++it;
            if (it == sv->pending.end()) break;
            Model* m = find(c, it->model);
            if (m && !m->exec && build_graph(c, m) != PR_OK) m = nullptr;  // admitted while serving
            sl.req = std::move(*it);
            sv->pending.erase(it);
            sl.t_dispatch = std::chrono::steady_clock::now();
            // The slot and the patient are claimed; the CUDA calls run without the
            // lock so that submitters and pollers are never held behind them (the
            // model cannot be released while it has a frame in flight).
            sl.busy = true;
            sv->in_flight.insert(sl.req.model);
            lock.unlock();
            cudaError_t e = cudaSuccess;
            if (!m) {
                e = cudaErrorInvalidValue;
            } else {
                const size_t R = (size_t)m->R;
                if (sl.y_cap < R) {
                    if (sl.y_pinned) cudaFreeHost(sl.y_pinned);
                    sl.y_pinned = nullptr;
                    sl.y_cap = 0;
                    e = cudaHostAlloc((void**)&sl.y_pinned, R * 4, cudaHostAllocDefault);
                    if (!e) sl.y_cap = R;
                }
                if (!e) {
                    memcpy(sl.y_pinned, sl.req.y.data(), R * 4);
                    e = cudaEventRecord(sl.start, sl.stream);
                }
                if (!e) e = cudaMemcpyAsync(m->y, sl.y_pinned, R * 4, cudaMemcpyHostToDevice, sl.stream);
                if (!e && write_params(c, m, sl.req.angle, &sl.req.opts, sl.stream) != PR_OK) e = cudaErrorUnknown;
                if (!e) e = cudaGraphLaunch(m->exec, sl.stream);
                if (!e) e = cudaMemcpyAsync(sl.host_state, m->st, sizeof(SolveState), cudaMemcpyDeviceToHost, sl.stream);
                if (!e) e = cudaEventRecord(sl.done, sl.stream);
            }
            lock.lock();
            if (e) {
                sl.busy = false;
                sv->in_flight.erase(sl.req.model);
                sv->error = PR_ECUDA;
                sv->error_msg = std::string("dispatch failed: ") + cudaGetErrorString(e);
                pr_served out;
                memset(&out, 0, sizeof out);
                out.tag = sl.req.tag;
                out.model_id = sl.req.model;
                out.status = PR_ECUDA;
                sv->done.push_back(out);
                sv->cv_done.notify_all();
                continue;
            }
            sl.req.y.clear();
            sl.req.y.shrink_to_fit();
            busy = true;
            progressed = true;
        }
        if (sv->stop && !busy) {
            // stop once idle; frames of models still waiting for admission stay
            // queued, and after an error nothing more is dispatched
            bool any = false;
            for (const ServeRequest& r : sv->pending) any = any || find(c, r.model) != nullptr;
            if (!any || sv->error) break;
        }
        if (busy && !progressed) {
            // a solve is running: poll its event again shortly
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        } else if (!busy && !progressed) {
            sv->cv_work.wait_for(lock, std::chrono::milliseconds(50));
        }
    }
}

int serve_stop(pr_ctx* c) {
    if (!c->serve) return PR_OK;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        c->serve->stop = true;
    }
    c->serve->cv_work.notify_all();
    if (c->serve->worker.joinable()) c->serve->worker.join();
    return PR_OK;
}

void serve_free(pr_ctx* c) {
    if (!c->serve) return;
    serve_stop(c);
    for (ServeSlot& sl : c->serve->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.start) cudaEventDestroy(sl.start);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.host_state) cudaFreeHost(sl.host_state);
        if (sl.y_pinned) cudaFreeHost(sl.y_pinned);
    }
    for (TickLane& ln : c->serve->lanes) {
        if (ln.stream) cudaStreamSynchronize(ln.stream);
        lane_free(ln);
        if (ln.start) cudaEventDestroy(ln.start);
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.stream) cudaStreamDestroy(ln.stream);
    }
    delete c->serve;
    c->serve = nullptr;
}

}  // namespace

extern "C" {

const char* pr_version(void) { return "pcarecon 0.1 (sm_103a)"; }

const char* pr_last_error(void) { return g_err.c_str(); }

void pr_default_opts(pr_solve_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->max_iters = 10;
    o->grad_tol = 1e-6;
    o->c1 = 1e-4;
    o->beta = 0.5;
    o->max_backtracks = 8;
    o->step0_mm = 1.0;
    o->cold_start = 0;
    o->loop_mode = PR_LOOP_GRAPH;
    o->tumor_tol = 1e-6;
    o->tumor_max_iter = 100;
    o->step_growth = 2.0;
    o->step_growth_bt = 1.0;
    o->warm_step = 1;
    o->step_model = 1;
}

int pr_create(pr_ctx** out, int device, void* stream, size_t hbm_budget_bytes) {
    if (!out) return fail(PR_EINVAL, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(PR_EINVAL, "device %d out of range (%d devices)", device, ndev);
    CK(cudaSetDevice(device));
    pr_ctx* c = new pr_ctx;
    c->device = device;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(PR_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)fr);
    if (cudaMalloc((void**)&c->rg, sizeof(RayGeom)) != cudaSuccess) {
        pr_destroy(c);
        return fail(PR_ENOMEM, "cudaMalloc failed");
    }
    *out = c;
    return PR_OK;
}

void pr_destroy(pr_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    serve_free(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    batch_free(c);
    for (auto& kv : c->models) free_model(kv.second);
    c->models.clear();
    for (Waiting* w : c->waiting) delete w;
    c->waiting.clear();
    if (c->pad) cudaFree(c->pad);
    if (c->rg) cudaFree(c->rg);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

namespace {

// Allocate, upload and register a model under `id` (0 = a new id).
int load_resident(pr_ctx* c, const pr_volume_desc* vol, const pr_geometry* geom, int location, const float* f0,
                  const float* mean_dvf, const float* U, int K, int storage, const double tumor_ref_xyz[3], int id,
                  int* model_id) {
    Model* m = new Model;
    m->vol = *vol;
    m->geom = *geom;
    m->geom.ds = resolved_ds(*vol, *geom);
    m->K = K;
    m->storage = storage;
    m->nch = fh_layout(K, storage);
    m->R = geom->nu * geom->nv;
    VolDev vd = make_vd(*vol);
    size_t n = (size_t)vd.n, np = (size_t)vd.np, R = (size_t)m->R;
    size_t ts = storage == PR_BF16 ? 2 : 4;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = dalloc(p, bytes, &m->bytes);
    };
    A(&m->f0p, np * ts);
    A(&m->mean, 3 * n * 4);
    A(&m->U, 3 * (size_t)K * n * ts);
    A(&m->fh, np * fh_floats(m->nch) * 4);
    A(&m->fpad, np * 4);
    A(&m->p, R * 4);
    A(&m->q, R * K * 4);
    A(&m->y, R * 4);
    A(&m->r, R * 4);
    A(&m->flat, n * 4);
    m->md.vd = vd;
    A(&m->partials, partial_doubles(m->geom, m->md.vd) * 8);
    A(&m->counter, 64);
    A(&m->st, sizeof(SolveState));
    A(&m->wdev, 8 * 8);
    A(&m->out, 16 * 8);
    A(&m->rg, sizeof(RayGeom));
    A(&m->steps, 16);
    A(&m->order, (size_t)project_blocks(geom->nu, geom->nv) * sizeof(int));
    A(&m->sup, sizeof(Support));
    A(&m->order_w, (size_t)split_order_ints(geom->nu, geom->nv) * sizeof(int));
    A(&m->ss.part, split_part_floats(geom->nu, geom->nv, fh_logical(m->nch)) * 4);
    A(&m->ss.tile_mom, (size_t)split_tiles(geom->nu, geom->nv) * kProjMom * 8);
    A(&m->ss.group_mom, (size_t)split_groups(geom->nu, geom->nv) * kProjMom * 8);
    A(&m->ss.ctr, split_counters(geom->nu, geom->nv) * 4);
    m->ss.order = m->order_w;
    A(&m->tlog, kTrialLog);
    m->bn[0] = (vol->nx + 3) / 4, m->bn[1] = (vol->ny + 3) / 4, m->bn[2] = (vol->nz + 3) / 4;
    A(&m->lev, (size_t)m->bn[0] * m->bn[1] * m->bn[2]);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&m->st_host, sizeof(SolveState), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        free_model(m);
        cudaGetLastError();
        return fail(PR_ENOMEM, "device allocation failed: %s", cudaGetErrorString(e));
    }
    m->md.K = K;
    m->md.storage = storage;
    m->md.f0p = m->f0p;
    m->md.mean = m->mean;
    m->md.U = m->U;
    for (int i = 0; i < 3; ++i) m->md.c0[i] = tumor_ref_xyz[i];

    // Upload: float32 staging on the device, then conversion / padding kernels.
    int rc = PR_OK;
    cudaMemcpyKind kind = location == PR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaStream_t s = c->stream;
    std::vector<int> order_host((size_t)project_blocks(geom->nu, geom->nv));  // lives until the sync below
    std::vector<int> order_w_host((size_t)split_order_ints(geom->nu, geom->nv));
    do {
        if ((e = cudaMemsetAsync(m->f0p, 0, np * ts, s))) break;
        if ((e = cudaMemsetAsync(m->fh, 0, np * fh_floats(m->nch) * 4, s))) break;
        if ((e = cudaMemsetAsync(m->fpad, 0, np * 4, s))) break;
        if ((e = cudaMemsetAsync(m->partials, 0, partial_doubles(m->geom, m->md.vd) * 8, s))) break;
        if ((e = cudaMemsetAsync(m->counter, 0, 64, s))) break;
        if ((e = cudaMemsetAsync(m->st, 0, sizeof(SolveState), s))) break;
        if ((e = cudaMemcpyAsync(m->mean, mean_dvf, 3 * n * 4, kind, s))) break;
        if ((e = cudaMemsetAsync(m->ss.ctr, 0, split_counters(geom->nu, geom->nv) * 4, s))) break;
        project_warp_tile_order(geom->nu, geom->nv, order_w_host.data());
        if ((e = cudaMemcpyAsync(m->order_w, order_w_host.data(), order_w_host.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, s)))
            break;
        project_tile_order(geom->nu, geom->nv, order_host.data());
        if ((e = cudaMemcpyAsync(m->order, order_host.data(), order_host.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, s)))
            break;
        // f0 -> padded float32 (fpad as staging), then to storage type.
        if ((e = cudaMemcpyAsync(m->flat, f0, n * 4, kind, s))) break;
        Launcher L;
        L.stream = s;
        if ((e = launch_support_init(L, m->sup))) break;
        if ((e = launch_support_box(L, vd, m->flat, m->sup))) break;
        if ((e = make_brick_levels(L, m, s))) break;
        for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = launch_maxabs(L, m->mean + (size_t)c * n, (long long)n, &m->sup->mean_max[c]);
        if (e) break;
        if ((e = launch_pad(L, vd, m->flat, m->fpad))) break;
        if (storage == PR_F32) {
            if ((e = cudaMemcpyAsync(m->f0p, m->fpad, np * 4, cudaMemcpyDeviceToDevice, s))) break;
            if ((e = cudaMemcpyAsync(m->U, U, 3 * (size_t)K * n * 4, kind, s))) break;
            for (int pl = 0; pl < 3 * K && e == cudaSuccess; ++pl)
                e = launch_maxabs(L, (const float*)m->U + (size_t)pl * n, (long long)n, &m->sup->u_max[pl / 3][pl % 3]);
            if (e) break;
        } else {
            if ((e = launch_to_bf16(L, m->fpad, (__nv_bfloat16*)m->f0p, np))) break;
            // U converted plane by plane through the float32 scratch
            for (int pl = 0; pl < 3 * K && e == cudaSuccess; ++pl) {
                if ((e = cudaMemcpyAsync(m->flat, U + (size_t)pl * n, n * 4, kind, s))) break;
                if ((e = launch_maxabs(L, m->flat, (long long)n, &m->sup->u_max[pl / 3][pl % 3]))) break;
                e = launch_to_bf16(L, m->flat, (__nv_bfloat16*)m->U + (size_t)pl * n, n);
            }
            if (e) break;
        }
        if ((e = cudaMemsetAsync(m->fpad, 0, np * 4, s))) break;
        e = cudaStreamSynchronize(s);
    } while (0);
    if (e != cudaSuccess) {
        rc = fail(PR_ECUDA, "model upload failed: %s", cudaGetErrorString(e));
        free_model(m);
        return rc;
    }
    {
        std::lock_guard<std::mutex> lock(c->mu);
        m->id = id ? id : c->next_id++;
        c->used += m->bytes;
        c->models[m->id] = m;
        c->model_epoch += 1;
        *model_id = m->id;
    }
    if (c->serve) c->serve->cv_work.notify_all();  // its queued frames can now run
    return PR_OK;
}

// Admit waiting models in FIFO order while the budget has room for the one
// at the front (called after memory was released).
int admit_waiting(pr_ctx* c) {
    for (;;) {
        Waiting* w = nullptr;
        {
            std::lock_guard<std::mutex> lock(c->mu);
            if (c->waiting.empty() || c->used + c->waiting.front()->need > c->budget) return PR_OK;
            w = c->waiting.front();
        }
        int got = 0;
        int rc = load_resident(c, &w->vol, &w->geom, PR_HOST, w->f0.data(), w->mean.data(), w->U.data(), w->K,
                               w->storage, w->c0, w->id, &got);
        if (rc) return rc;  // stays at the front of the queue
        {
            std::lock_guard<std::mutex> lock(c->mu);
            c->waiting.pop_front();
        }
        delete w;
    }
}

Waiting* find_waiting(pr_ctx* c, int id) {
    for (Waiting* w : c->waiting)
        if (w->id == id) return w;
    return nullptr;
}

}  // namespace

extern "C" {

int pr_load_model(pr_ctx* c, const pr_volume_desc* vol, const pr_geometry* geom, int location, const float* f0,
                  const float* mean_dvf, const float* U, int K, int storage, const double tumor_ref_xyz[3],
                  int* model_id) {
    if (!c || !model_id) return fail(PR_EINVAL, "null context or model_id");
    if (!vol_ok(vol)) return fail(PR_EINVAL, "invalid volume descriptor");
    if (!geom_ok(geom)) return fail(PR_EINVAL, "invalid geometry");
    if (K < 1 || K > PR_MAX_K) return fail(PR_EINVAL, "K=%d outside 1..%d", K, PR_MAX_K);
    if (storage != PR_F32 && storage != PR_BF16) return fail(PR_EINVAL, "unknown storage %d", storage);
    if (location != PR_HOST && location != PR_DEVICE) return fail(PR_EINVAL, "unknown location %d", location);
    if (!f0 || !mean_dvf || !U || !tumor_ref_xyz) return fail(PR_EINVAL, "null input array");
    CK(cudaSetDevice(c->device));
    size_t need = model_bytes(*vol, *geom, K, storage);
    size_t used_now;
    bool queue;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        used_now = c->used;
        queue = c->admit_queue;
        // behind models already waiting, in arrival order
        if (queue && !c->waiting.empty()) used_now = c->budget;
    }
    if (used_now + need <= c->budget)
        return load_resident(c, vol, geom, location, f0, mean_dvf, U, K, storage, tumor_ref_xyz, 0, model_id);
    if (!queue || need > c->budget)
        return fail(PR_EADMIT, "model needs %zu bytes, %zu of %zu budget in use", need, used_now, c->budget);
    // admission queue: keep host copies of the inputs until memory frees up
    Waiting* w = new Waiting;
    w->vol = *vol;
    w->geom = *geom;
    w->K = K;
    w->storage = storage;
    w->need = need;
    for (int i = 0; i < 3; ++i) w->c0[i] = tumor_ref_xyz[i];
    const size_t n = (size_t)vol->nx * vol->ny * vol->nz;
    w->f0.resize(n);
    w->mean.resize(3 * n);
    w->U.resize(3 * (size_t)K * n);
    const cudaMemcpyKind kind = location == PR_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpy(w->f0.data(), f0, n * 4, kind);
    if (!e) e = cudaMemcpy(w->mean.data(), mean_dvf, 3 * n * 4, kind);
    if (!e) e = cudaMemcpy(w->U.data(), U, 3 * (size_t)K * n * 4, kind);
    if (e) {
        delete w;
        return fail(PR_ECUDA, "copying the waiting model's inputs failed: %s", cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lock(c->mu);
        w->id = c->next_id++;
        c->waiting.push_back(w);
        *model_id = w->id;
    }
    fail(PR_QUEUED, "model %d needs %zu bytes and waits for admission", *model_id, need);
    return PR_QUEUED;
}

int pr_set_admission_queue(pr_ctx* c, int enable) {
    if (!c) return fail(PR_EINVAL, "null context");
    std::lock_guard<std::mutex> lock(c->mu);
    c->admit_queue = enable != 0;
    return PR_OK;
}

int pr_model_status(pr_ctx* c, int id, int* status) {
    if (!c || !status) return fail(PR_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(c->mu);
    if (find(c, id)) {
        *status = PR_MODEL_RESIDENT;
        return PR_OK;
    }
    for (size_t i = 0; i < c->waiting.size(); ++i)
        if (c->waiting[i]->id == id) {
            *status = PR_MODEL_WAITING;
            return PR_OK;
        }
    return fail(PR_ENOMODEL, "unknown model id %d", id);
}

int pr_release_model(pr_ctx* c, int id) {
    if (!c) return fail(PR_EINVAL, "null context");
    {
        std::lock_guard<std::mutex> lock(c->mu);
        Waiting* w = find_waiting(c, id);
        if (w) {
            if (c->serve)
                for (const ServeRequest& r : c->serve->pending)
                    if (r.model == id) return fail(PR_EINVAL, "model %d has served frames outstanding", id);
            c->waiting.erase(std::find(c->waiting.begin(), c->waiting.end(), w));
            delete w;
            return PR_OK;
        }
    }
    GET_MODEL(c, id, m);
    CK(cudaStreamSynchronize(c->stream));
    {
        std::lock_guard<std::mutex> lock(c->mu);
        if (c->serve) {
            bool queued = c->serve->in_flight.count(id) > 0;
            for (const ServeRequest& r : c->serve->pending) queued = queued || r.model == id;
            if (queued) return fail(PR_EINVAL, "model %d has served frames outstanding", id);
        }
        c->used -= m->bytes;
        c->models.erase(id);
        c->model_epoch += 1;
    }
    if (c->batch && std::find(c->batch->key.begin(), c->batch->key.end(), id) != c->batch->key.end())
        batch_drop_graph(c->batch);  // its nodes point into this model's buffers
    free_model(m);
    return admit_waiting(c);
}

int pr_model_footprint(pr_ctx* c, int id, size_t* bytes) {
    GET_MODEL(c, id, m);
    if (!bytes) return fail(PR_EINVAL, "null output");
    *bytes = m->bytes;
    return PR_OK;
}

int pr_reconstruct_async(pr_ctx* c, int id, const float* y_dev, double angle, const pr_solve_opts* opts) {
    GET_MODEL(c, id, m);
    if (!y_dev) return fail(PR_EINVAL, "null y");
    if (opts && opts->loop_mode == PR_LOOP_HOST) return fail(PR_EINVAL, "host loop is synchronous; use pr_reconstruct");
    CK(cudaMemcpyAsync(m->y, y_dev, (size_t)m->R * 4, cudaMemcpyDeviceToDevice, c->stream));
    return enqueue_solve(c, m, angle, opts);
}

int pr_trial_log(pr_ctx* c, int id, unsigned char* out, int cap, int* n) {
    GET_MODEL(c, id, m);
    if (!out || !n || cap < 0) return fail(PR_EINVAL, "null argument or negative cap");
    int trials = 0;
    CK(cudaMemcpyAsync(&trials, &m->st->trials, sizeof trials, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int k = std::min(std::min(trials, cap), kTrialLog);
    if (k > 0) CK(cudaMemcpy(out, m->tlog, (size_t)k, cudaMemcpyDeviceToHost));
    *n = trials;
    return PR_OK;
}

int pr_fetch_result(pr_ctx* c, int id, pr_result* out) {
    GET_MODEL(c, id, m);
    if (!out) return fail(PR_EINVAL, "null result");
    CK(cudaMemcpyAsync(m->st_host, m->st, sizeof(SolveState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    fill_result(m, *m->st_host, out);
    return PR_OK;
}

int pr_reconstruct(pr_ctx* c, int id, const float* y, int y_location, double angle, const pr_solve_opts* opts,
                   pr_result* out, float* volume_out) {
    GET_MODEL(c, id, m);
    if (!y || !out) return fail(PR_EINVAL, "null y or result");
    if (y_location != PR_HOST && y_location != PR_DEVICE) return fail(PR_EINVAL, "unknown y location");
    CK(cudaMemcpyAsync(m->y, y, (size_t)m->R * 4,
                       y_location == PR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    TRY(enqueue_solve(c, m, angle, opts));
    if (volume_out) {
        Launcher L;
        L.stream = c->stream;
        CK(launch_warp(L, m->md, m->st->w, kWarpFlatF, nullptr, m->flat, nullptr));
        CK(cudaMemcpyAsync(volume_out, m->flat, (size_t)m->md.vd.n * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    return pr_fetch_result(c, id, out);
}

int pr_reconstruct_batch(pr_ctx* c, int n, const int* model_ids, const float* const* y, const double* angles,
                         const pr_solve_opts* opts, pr_result* out) {
    if (!c || !model_ids || !y || !angles || !out) return fail(PR_EINVAL, "null argument");
    if (n < 1 || n > 4096) return fail(PR_EINVAL, "batch size %d outside 1..4096", n);
    if (c->serve && !c->serve->stop) return fail(PR_EINVAL, "stop serving before a batch");
    pr_solve_opts o;
    if (opts)
        o = *opts;
    else
        pr_default_opts(&o);
    if (!opts_ok(&o) || o.loop_mode != PR_LOOP_GRAPH) return fail(PR_EINVAL, "invalid solve options for a batch");
    std::vector<Model*> ms((size_t)n);
    std::vector<size_t> off((size_t)n);
    size_t total = 0;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        for (int i = 0; i < n; ++i) {
            Model* m = find(c, model_ids[i]);
            if (!m) return fail(PR_ENOMODEL, "no model %d", model_ids[i]);
            if (!y[i]) return fail(PR_EINVAL, "null y[%d]", i);
            if (!isfinite(angles[i])) return fail(PR_EINVAL, "angle %d is not finite", i);
            ms[(size_t)i] = m;
            off[(size_t)i] = total;
            total += ((size_t)m->R + 3) / 4 * 4;  // 16-byte aligned slices
        }
    }
    CK(cudaSetDevice(c->device));
    if (!c->batch) c->batch = new Batch;
    Batch* b = c->batch;
    if (b->y_cap < total || b->cap < n) {  // grow the staging; graphs bake its addresses
        batch_drop_graph(b);
        if (b->y) cudaFree(b->y);
        if (b->prm) cudaFree(b->prm);
        if (b->res) cudaFree(b->res);
        if (b->res_host) cudaFreeHost(b->res_host);
        b->y = nullptr, b->prm = nullptr, b->res = nullptr, b->res_host = nullptr, b->y_cap = 0, b->cap = 0;
        cudaError_t e = cudaMalloc(&b->y, total * 4);
        if (!e) e = cudaMalloc(&b->prm, (size_t)n * sizeof(SolveParams));
        if (!e) e = cudaMalloc(&b->res, (size_t)n * sizeof(SolveState));
        if (!e) e = cudaHostAlloc((void**)&b->res_host, (size_t)n * sizeof(SolveState), cudaHostAllocDefault);
        if (e) {
            batch_free(c);
            cudaGetLastError();
            return fail(PR_ENOMEM, "batch staging: %s", cudaGetErrorString(e));
        }
        b->y_cap = total;
        b->cap = n;
    }
    std::vector<int> key(model_ids, model_ids + n);
    if (!b->exec || key != b->key || off != b->y_off) {
        b->y_off = off;
        int rc = build_batch_graph(b, ms);
        if (rc) {
            batch_drop_graph(b);
            return rc;
        }
        b->key = key;
    }
    std::vector<SolveParams> prm((size_t)n);
    for (int i = 0; i < n; ++i) {
        Model* m = ms[(size_t)i];
        prm[(size_t)i] = make_params(m, angles[i], &o);
        CK(cudaMemcpyAsync(b->y + off[(size_t)i], y[i], (size_t)m->R * 4, cudaMemcpyHostToDevice, c->stream));
    }
    CK(cudaMemcpyAsync(b->prm, prm.data(), (size_t)n * sizeof(SolveParams), cudaMemcpyHostToDevice, c->stream));
    CK(cudaGraphLaunch(b->exec, c->stream));
    CK(cudaMemcpyAsync(b->res_host, b->res, (size_t)n * sizeof(SolveState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < n; ++i) fill_result(ms[(size_t)i], b->res_host[i], &out[i]);
    return PR_OK;
}

int pr_get_state(pr_ctx* c, int id, double* w) {
    GET_MODEL(c, id, m);
    if (!w) return fail(PR_EINVAL, "null w");
    double buf[8];
    CK(cudaMemcpyAsync(buf, m->st->w, sizeof buf, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < m->K; ++k) w[k] = buf[k];
    return PR_OK;
}

int pr_set_state(pr_ctx* c, int id, const double* w) {
    GET_MODEL(c, id, m);
    if (!w) return fail(PR_EINVAL, "null w");
    double buf[8] = {0};
    for (int k = 0; k < m->K; ++k) {
        if (!isfinite(w[k])) return fail(PR_EINVAL, "w[%d] is not finite", k);
        buf[k] = w[k];
    }
    CK(cudaMemcpyAsync(m->st->w, buf, sizeof buf, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(&m->st->mu_next, 0, sizeof(double), c->stream));
    CK(cudaMemsetAsync(&m->st->history, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PR_OK;
}

int pr_warp(pr_ctx* c, int id, const double* w, float* f_dev, float* h_dev) {
    GET_MODEL(c, id, m);
    if (!w) return fail(PR_EINVAL, "null w");
    TRY(set_w(c, m, w));
    Launcher L;
    L.stream = c->stream;
    CK(launch_warp(L, m->md, m->wdev, h_dev ? kWarpFlatFH : kWarpFlatF, nullptr, f_dev, h_dev));
    CK(cudaStreamSynchronize(c->stream));
    return PR_OK;
}

int pr_project(pr_ctx* c, const pr_volume_desc* vol, const pr_geometry* geom, double angle, const float* f_dev,
               float* p_dev) {
    if (!c) return fail(PR_EINVAL, "null context");
    if (!vol_ok(vol) || !geom_ok(geom)) return fail(PR_EINVAL, "invalid volume or geometry");
    if (!f_dev || !p_dev) return fail(PR_EINVAL, "null volume or projection");
    CK(cudaSetDevice(c->device));
    size_t np = pad_voxels(*vol);
    if (np > c->pad_cap) {
        if (c->pad) cudaFree(c->pad);
        c->pad = nullptr;
        c->pad_cap = 0;
        CK(cudaMalloc((void**)&c->pad, np * 4));
        c->pad_cap = np;
    }
    TRY(set_rg(c, c->rg, *vol, *geom, angle));
    VolDev vd = make_vd(*vol);
    Launcher L;
    L.stream = c->stream;
    CK(cudaMemsetAsync(c->pad, 0, np * 4, c->stream));
    CK(launch_pad(L, vd, f_dev, c->pad));
    CK(launch_project(L, vd, c->pad, 1, 0, c->rg, nullptr, geom->nu, geom->nv, p_dev, nullptr, nullptr, nullptr, nullptr,
                      nullptr, kPhaseNone, 0, 0));
    CK(cudaStreamSynchronize(c->stream));
    return PR_OK;
}

int pr_backproject(pr_ctx* c, const pr_volume_desc* vol, const pr_geometry* geom, double angle, const float* r_dev,
                   float* g_dev) {
    if (!c) return fail(PR_EINVAL, "null context");
    if (!vol_ok(vol) || !geom_ok(geom)) return fail(PR_EINVAL, "invalid volume or geometry");
    if (!r_dev || !g_dev) return fail(PR_EINVAL, "null residual or output");
    CK(cudaSetDevice(c->device));
    TRY(set_rg(c, c->rg, *vol, *geom, angle));
    VolDev vd = make_vd(*vol);
    Launcher L;
    L.stream = c->stream;
    CK(launch_backproject(L, vd, c->rg, r_dev, g_dev, nullptr, 0, nullptr, nullptr, nullptr));
    CK(cudaStreamSynchronize(c->stream));
    return PR_OK;
}

int pr_forward(pr_ctx* c, int id, const double* w, double angle, float* p_dev) {
    GET_MODEL(c, id, m);
    if (!w || !p_dev) return fail(PR_EINVAL, "null w or projection");
    TRY(set_w(c, m, w));
    TRY(set_rg(c, m->rg, m->vol, m->geom, angle));
    Launcher L;
    L.stream = c->stream;
    CK(launch_warp(L, m->md, m->wdev, kWarpFPad, m->fpad, nullptr, nullptr, m->sup));
    CK(launch_project(L, m->md.vd, m->fpad, 1, 0, m->rg, m->order, m->geom.nu, m->geom.nv, p_dev, nullptr, nullptr, nullptr,
                      nullptr, nullptr, kPhaseNone, 0, 0, sref(m, m->wdev)));
    CK(cudaStreamSynchronize(c->stream));
    return PR_OK;
}

int pr_count_samples(pr_ctx* c, int id, double angle, const double* w, long long* count) {
    GET_MODEL(c, id, m);
    if (!w || !count) return fail(PR_EINVAL, "null argument");
    TRY(set_w(c, m, w));
    TRY(set_rg(c, m->rg, m->vol, m->geom, angle));
    Launcher L;
    L.stream = c->stream;
    unsigned long long* dev = reinterpret_cast<unsigned long long*>(m->partials);
    unsigned long long host = 0;
    CK(cudaMemsetAsync(dev, 0, sizeof host, c->stream));
    CK(launch_count_samples(L, m->md.vd, m->rg, m->geom.nu, m->geom.nv, sref(m, m->wdev), dev));
    CK(cudaMemcpyAsync(&host, dev, sizeof host, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = (long long)host;
    return PR_OK;
}

int pr_warp_box(pr_ctx* c, int id, const double* w, int box[6]) {
    GET_MODEL(c, id, m);
    if (!w || !box) return fail(PR_EINVAL, "null argument");
    TRY(set_w(c, m, w));
    Launcher L;
    L.stream = c->stream;
    int* dev = reinterpret_cast<int*>(m->partials);
    CK(launch_warp_box(L, m->md, m->wdev, m->sup, 0, dev));
    CK(cudaMemcpyAsync(box, dev, 6 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PR_OK;
}

int pr_fix_angle(pr_ctx* c, int id, double angle, size_t* table_bytes) {
    GET_MODEL(c, id, m);
    CK(cudaStreamSynchronize(c->stream));
    drop_bp_table(c, m);
    if (table_bytes) *table_bytes = 0;
    if (isnan(angle)) return PR_OK;  // NaN: back to weights computed per call
    if (!isfinite(angle)) return fail(PR_EINVAL, "angle is not finite");
    if (m->geom.nu > 32767 || m->geom.nv > 32767) return fail(PR_EINVAL, "detector too wide for the table");
    const VolDev& vd = m->md.vd;
    TRY(set_rg(c, m->rg, m->vol, m->geom, angle));
    Launcher L;
    L.stream = c->stream;
    short4* rect = nullptr;
    CK(cudaMalloc(&rect, (size_t)vd.n * sizeof(short4)));
    unsigned int* slots_dev = reinterpret_cast<unsigned int*>(m->partials);
    unsigned int slots = 0;
    cudaError_t e = cudaMemsetAsync(slots_dev, 0, sizeof(unsigned int), c->stream);
    if (!e) e = launch_bp_rect(L, vd, m->rg, rect, slots_dev);
    if (!e) e = cudaMemcpyAsync(&slots, slots_dev, sizeof slots, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
        cudaFree(rect);
        return fail(PR_ECUDA, "fixed-angle footprints: %s", cudaGetErrorString(e));
    }
    const size_t need = (size_t)vd.n * sizeof(short4) + (size_t)slots * vd.n * sizeof(float);
    {
        std::lock_guard<std::mutex> lock(c->mu);
        if (c->used + need > c->budget) {
            cudaFree(rect);
            return fail(PR_EADMIT, "fixed-angle table of %zu bytes exceeds the HBM budget", need);
        }
    }
    float* w = nullptr;
    if (slots > 0 && cudaMalloc(&w, (size_t)slots * vd.n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(rect);
        return fail(PR_ENOMEM, "fixed-angle table of %zu bytes: allocation failed", need);
    }
    if (slots > 0) e = launch_bp_fill(L, vd, m->rg, rect, w);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
        cudaFree(rect);
        if (w) cudaFree(w);
        return fail(PR_ECUDA, "fixed-angle weights: %s", cudaGetErrorString(e));
    }
    m->bt_rect = rect;
    m->bt_w = w;
    m->fixed = w != nullptr;
    m->fixed_angle = angle;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        m->bt_bytes = need;
        m->bytes += need;
        c->used += need;
    }
    if (table_bytes) *table_bytes = need;
    return PR_OK;
}

int pr_vjp(pr_ctx* c, int id, const double* w, double angle, const float* grad_p_dev, double* grad_w) {
    GET_MODEL(c, id, m);
    if (!w || !grad_p_dev || !grad_w) return fail(PR_EINVAL, "null argument");
    TRY(ensure_hbuf(c, m));
    TRY(set_w(c, m, w));
    TRY(set_rg(c, m->rg, m->vol, m->geom, angle));
    Launcher L;
    L.stream = c->stream;
    CK(launch_warp(L, m->md, m->wdev, kWarpFlatFH, nullptr, nullptr, m->hbuf));
    CK(launch_backproject(L, m->md.vd, m->rg, grad_p_dev, nullptr, m->hbuf, m->K, m->partials, m->counter, m->out,
                          bp_table(m, angle)));
    double buf[8];
    CK(cudaMemcpyAsync(buf, m->out, sizeof(double) * m->K, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < m->K; ++k) grad_w[k] = buf[k];
    return PR_OK;
}

int pr_cost_grad(pr_ctx* c, int id, const float* y_dev, double angle, const double* w, double a, double b, int mode,
                 double* J, double* grad, float* p_dev) {
    GET_MODEL(c, id, m);
    if (!y_dev || !w || !J || !grad) return fail(PR_EINVAL, "null argument");
    if (mode != 0 && mode != 1) return fail(PR_EINVAL, "mode must be 0 (forward) or 1 (adjoint)");
    if (!isfinite(a) || !isfinite(b)) return fail(PR_EINVAL, "a, b must be finite");
    TRY(set_w(c, m, w));
    TRY(set_rg(c, m->rg, m->vol, m->geom, angle));
    double ab[2] = {a, b};
    CK(cudaMemcpyAsync(m->out + 8, ab, sizeof ab, cudaMemcpyHostToDevice, c->stream));
    Launcher L;
    L.stream = c->stream;
    const int nu = m->geom.nu, nv = m->geom.nv;
    double res[8] = {0};
    if (mode == 0) {
        CK(launch_warp(L, m->md, m->wdev, kWarpFH, m->fh, nullptr, nullptr, m->sup, m->st->fh_box));
        CK(launch_warp_box(L, m->md, m->wdev, m->sup, 1, m->st->fh_box));  // what the volume now holds
        CK(launch_project(L, m->md.vd, m->fh, m->nch, m->K, m->rg, m->order, nu, nv, m->p, m->q, nullptr, nullptr, nullptr,
                          nullptr, kPhaseNone, 0, 0, sref(m, m->wdev), &m->ss));
        CK(launch_cost_grad(L, m->p, m->q, y_dev, m->R, m->K, m->out + 8, m->partials, m->counter, m->out));
        CK(cudaMemcpyAsync(res, m->out, sizeof(double) * (1 + m->K), cudaMemcpyDeviceToHost, c->stream));
    } else {
        TRY(ensure_hbuf(c, m));
        CK(launch_warp(L, m->md, m->wdev, kWarpFPad, m->fpad, nullptr, nullptr, m->sup));
        CK(launch_warp(L, m->md, m->wdev, kWarpFlatFH, nullptr, nullptr, m->hbuf));
        CK(launch_project(L, m->md.vd, m->fpad, 1, 0, m->rg, m->order, nu, nv, m->p, nullptr, nullptr, nullptr, nullptr,
                          nullptr, kPhaseNone, 0, 0, sref(m, m->wdev)));
        CK(launch_cost_grad(L, m->p, nullptr, y_dev, m->R, 0, m->out + 8, m->partials, m->counter, m->out));
        CK(launch_residual(L, m->p, y_dev, m->R, m->out + 8, m->r));
        CK(cudaMemcpyAsync(res, m->out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(launch_backproject(L, m->md.vd, m->rg, m->r, nullptr, m->hbuf, m->K, m->partials, m->counter,
                              m->out + 1, bp_table(m, angle)));
        CK(cudaMemcpyAsync(res + 1, m->out + 1, sizeof(double) * m->K, cudaMemcpyDeviceToHost, c->stream));
    }
    if (p_dev) CK(cudaMemcpyAsync(p_dev, m->p, (size_t)m->R * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *J = res[0];
    for (int k = 0; k < m->K; ++k) grad[k] = mode == 0 ? res[1 + k] : 2.0 * res[1 + k];
    return PR_OK;
}

int pr_tumor(pr_ctx* c, int id, const double* w, double tol, int max_iter, double* xyz, int* steps) {
    GET_MODEL(c, id, m);
    if (!w || !xyz) return fail(PR_EINVAL, "null argument");
    if (!(tol >= 0) || max_iter < 0) return fail(PR_EINVAL, "invalid tol or max_iter");
    TRY(set_w(c, m, w));
    Launcher L;
    L.stream = c->stream;
    CK(launch_tumor(L, m->md, m->wdev, tol, max_iter, nullptr, m->out, m->steps));
    double buf[3];
    int st = 0;
    CK(cudaMemcpyAsync(buf, m->out, sizeof buf, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&st, m->steps, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 3; ++i) xyz[i] = buf[i];
    if (steps) *steps = st;
    return PR_OK;
}

int pr_invert_dvf(pr_ctx* c, int id, const double* w, double tol, int max_iter, float* y_dev, int* max_steps,
                  long long* unconverged) {
    GET_MODEL(c, id, m);
    if (!w || !y_dev) return fail(PR_EINVAL, "null argument");
    if (!(tol >= 0) || !std::isfinite(tol) || max_iter < 1 || max_iter > 100000)
        return fail(PR_EINVAL, "invalid tol or max_iter");
    if (m->vol.nx * (long long)m->vol.ny * m->vol.nz >= 0x7fffffffLL) return fail(PR_EINVAL, "grid too large");
    TRY(set_w(c, m, w));
    Launcher L;
    L.stream = c->stream;
    unsigned int* stats = reinterpret_cast<unsigned int*>(m->partials);
    CK(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned int), c->stream));
    CK(launch_invert(L, m->md, m->wdev, reinterpret_cast<float4*>(m->fh), tol, max_iter, y_dev, stats));
    // the scratch field overwrote the solver volume's zero border
    CK(cudaMemsetAsync(m->fh, 0, (size_t)m->md.vd.np * fh_floats(m->nch) * 4, c->stream));
    unsigned int st[2] = {0, 0};
    CK(cudaMemcpyAsync(st, stats, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (max_steps) *max_steps = (int)st[0];
    if (unconverged) *unconverged = (long long)st[1];
    return PR_OK;
}

int pr_time_kernel(pr_ctx* c, int id, int which, double angle, int iters, double* avg_ms) {
    GET_MODEL(c, id, m);
    if (!avg_ms || iters < 1 || iters > 100000) return fail(PR_EINVAL, "invalid iters or output");
    if (which < PR_KERNEL_WARP_FH || which > PR_KERNEL_PROJECT_FH_TRIAL) return fail(PR_EINVAL, "unknown kernel %d", which);
    if (which == PR_KERNEL_INVERT && m->vol.nx * (long long)m->vol.ny * m->vol.nz >= 0x7fffffffLL)
        return fail(PR_EINVAL, "grid too large");
    TRY(set_rg(c, m->rg, m->vol, m->geom, angle));
    if (which == PR_KERNEL_BACKPROJECT) TRY(ensure_hbuf(c, m));
    Launcher L;
    L.stream = c->stream;
    const int nu = m->geom.nu, nv = m->geom.nv;
    double ab[2] = {1.0, 0.0};
    CK(cudaMemcpyAsync(m->out + 8, ab, sizeof ab, cudaMemcpyHostToDevice, c->stream));
    // Inputs the timed kernel reads: f/h at the warm-start w, p and q.
    CK(launch_warp(L, m->md, m->st->w, kWarpFH, m->fh, nullptr, nullptr, m->sup, m->st->fh_box));
    CK(launch_warp_box(L, m->md, m->st->w, m->sup, 1, m->st->fh_box));  // what the volume now holds
    CK(launch_warp(L, m->md, m->st->w, kWarpFPad, m->fpad, nullptr, nullptr, m->sup));
    if (which == PR_KERNEL_BACKPROJECT) CK(launch_warp(L, m->md, m->st->w, kWarpFlatFH, nullptr, nullptr, m->hbuf));
    CK(launch_project(L, m->md.vd, m->fh, m->nch, m->K, m->rg, m->order, nu, nv, m->p, m->q, nullptr, nullptr, nullptr, nullptr,
                      kPhaseNone, 0, 0, sref(m, m->st->w), &m->ss));
    float* ytmp = nullptr;  // output of the timed inversion (3N floats, freed below)
    if (which == PR_KERNEL_INVERT) CK(cudaMalloc(&ytmp, (size_t)3 * m->md.vd.n * sizeof(float)));
    SolveState* sst = nullptr;  // copy of the solve state the timed trial passes update (freed below)
    if (which == PR_KERNEL_PROJECT_FH_TRIAL) {
        CK(cudaMalloc(&sst, sizeof(SolveState)));
        CK(cudaMemcpyAsync(sst, m->st, sizeof(SolveState), cudaMemcpyDeviceToDevice, c->stream));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
    for (int i = 0; i < iters && err == cudaSuccess; ++i) {
        switch (which) {
            case PR_KERNEL_WARP_FH:  // as in a solve: the blocks outside both boxes are left alone
                err = launch_warp(L, m->md, m->st->w, kWarpFH, m->fh, nullptr, nullptr, m->sup, m->st->fh_box);
                break;
            case PR_KERNEL_PROJECT_FH:
                err = launch_project(L, m->md.vd, m->fh, m->nch, m->K, m->rg, m->order, nu, nv, m->p, m->q, nullptr, nullptr,
                                     nullptr, nullptr, kPhaseNone, 0, 0, sref(m, m->st->w), &m->ss);
                break;
            case PR_KERNEL_REGRAD:
                err = launch_cost_grad(L, m->p, m->q, m->p, m->R, m->K, m->out + 8, m->partials, m->counter, m->out);
                break;
            case PR_KERNEL_BACKPROJECT:
                err = launch_backproject(L, m->md.vd, m->rg, m->p, nullptr, m->hbuf, m->K, m->partials, m->counter,
                                         m->out, bp_table(m, angle));
                break;
            case PR_KERNEL_WARP_F: err = launch_warp(L, m->md, m->st->w, kWarpFPad, m->fpad, nullptr, nullptr, m->sup); break;
            case PR_KERNEL_PROJECT_F:
                err = launch_project(L, m->md.vd, m->fpad, 1, 0, m->rg, m->order, nu, nv, m->r, nullptr, nullptr, nullptr,
                                     nullptr, nullptr, kPhaseNone, 0, 0, sref(m, m->st->w));
                break;
            case PR_KERNEL_INVERT:
                err = launch_invert(L, m->md, m->st->w, reinterpret_cast<float4*>(m->fh), 1e-5, 64, ytmp,
                                    reinterpret_cast<unsigned int*>(m->partials));
                break;
            case PR_KERNEL_PROJECT_FH_TRIAL:
                err = launch_project(L, m->md.vd, m->fh, m->nch, m->K, m->rg, m->order, nu, nv, m->p, m->q, m->y, sst,
                                     m->partials, m->counter, kPhaseTrial, 0, 0, sref(m, m->st->w), &m->ss);
                break;
        }
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (which == PR_KERNEL_INVERT && err == cudaSuccess)  // restore the zero border (the field was scratch)
        err = cudaMemsetAsync(m->fh, 0, (size_t)m->md.vd.np * fh_floats(m->nch) * 4, c->stream);
    if (ytmp || sst) {
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        if (ytmp) cudaFree(ytmp);
        if (sst) cudaFree(sst);
        if (err == cudaSuccess) err = e2;
    }
    CK(err);
    *avg_ms = (double)ms / iters;
    return PR_OK;
}

int pr_model_stats(pr_ctx* c, int id, pr_stats* out) {
    GET_MODEL(c, id, m);
    if (!out) return fail(PR_EINVAL, "null output");
    CK(cudaMemcpyAsync(m->st_host, m->st, sizeof(SolveState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out->solves = m->st_host->cum_solves;
    out->trials = m->st_host->cum_trials;
    // per solve: begin, warp, project, tumor; per trial: warp, project (the
    // body of the loop)
    out->kernels = 4 * out->solves + 2 * out->trials;
    out->iters = m->st_host->cum_iters;
    out->line_search_failures = m->st_host->cum_lsf;
    return PR_OK;
}

int pr_io_bytes(pr_ctx* c, int id, size_t* h2d, size_t* d2h) {
    GET_MODEL(c, id, m);
    if (!h2d || !d2h) return fail(PR_EINVAL, "null output");
    *h2d = (size_t)m->R * 4 + sizeof(SolveParams);
    *d2h = sizeof(SolveState);
    return PR_OK;
}

int pr_serve_start(pr_ctx* c, int slots) {
    if (!c) return fail(PR_EINVAL, "null context");
    if (slots < 1 || slots > 64) return fail(PR_EINVAL, "slots must be 1..64");
    if (c->serve && !c->serve->stop) return fail(PR_EINVAL, "serving already started");
    if (c->serve) serve_free(c);  // restart after pr_serve_stop: untaken results are dropped
    CK(cudaSetDevice(c->device));
    Serve* sv = new Serve;
    sv->slots.resize(slots);
    for (ServeSlot& sl : sv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (!e) e = cudaEventCreate(&sl.start);
        if (!e) e = cudaEventCreate(&sl.done);
        if (!e) e = cudaHostAlloc((void**)&sl.host_state, sizeof(SolveState), cudaHostAllocDefault);
        if (e) {
            c->serve = sv;
            serve_free(c);
            return fail(PR_ECUDA, "serving set-up failed: %s", cudaGetErrorString(e));
        }
    }
    c->serve = sv;
    sv->worker = std::thread(serve_loop, c);
    return PR_OK;
}

int pr_serve_start_batched(pr_ctx* c, int lanes, int tick_frames) {
    if (!c) return fail(PR_EINVAL, "null context");
    if (lanes < 1 || lanes > 8) return fail(PR_EINVAL, "lanes must be 1..8");
    if (tick_frames < 0) return fail(PR_EINVAL, "tick_frames must be >= 0");
    if (c->serve && !c->serve->stop) return fail(PR_EINVAL, "serving already started");
    CK(cudaSetDevice(c->device));
    if (c->serve) serve_free(c);  // restart after pr_serve_stop: untaken results are dropped
    Serve* sv = new Serve;
    sv->tick_frames = tick_frames;
    sv->lanes.resize(lanes);
    for (TickLane& ln : sv->lanes) {
        cudaError_t e = cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking);
        if (!e) e = cudaEventCreate(&ln.start);
        if (!e) e = cudaEventCreate(&ln.done);
        if (e) {
            c->serve = sv;
            serve_free(c);
            return fail(PR_ECUDA, "serving set-up failed: %s", cudaGetErrorString(e));
        }
    }
    c->serve = sv;
    sv->worker = std::thread(serve_loop_ticks, c);
    return PR_OK;
}

int pr_submit(pr_ctx* c, int id, const float* y, double angle, const pr_solve_opts* opts, uint64_t tag) {
    if (!c) return fail(PR_EINVAL, "null context");
    Model* m = nullptr;
    int R = 0;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        m = find(c, id);
        Waiting* w = m ? nullptr : find_waiting(c, id);
        if (!m && !w) return fail(PR_ENOMODEL, "unknown model id %d", id);
        R = m ? m->R : w->geom.nu * w->geom.nv;
    }
    CK(cudaSetDevice(c->device));
    if (!c->serve) return fail(PR_EINVAL, "serving not started (pr_serve_start)");
    if (!y) return fail(PR_EINVAL, "null y");
    pr_solve_opts o;
    if (opts)
        o = *opts;
    else
        pr_default_opts(&o);
    if (!opts_ok(&o) || o.loop_mode != PR_LOOP_GRAPH) return fail(PR_EINVAL, "invalid solve options for serving");
    if (!isfinite(angle)) return fail(PR_EINVAL, "angle is not finite");
    if (m && c->serve->slots.size() && !m->exec) TRY(build_graph(c, m));
    ServeRequest r;
    r.model = id;
    r.tag = tag;
    r.angle = angle;
    r.opts = o;
    r.y.assign(y, y + R);
    r.t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lock(c->mu);
        if (c->serve->error) return fail(c->serve->error, "%s", c->serve->error_msg.c_str());
        c->serve->pending.push_back(std::move(r));
        c->serve->outstanding += 1;
    }
    c->serve->cv_work.notify_all();
    return PR_OK;
}

int pr_poll(pr_ctx* c, int timeout_ms, pr_served* out) {
    if (!c || !out) return fail(PR_EINVAL, "null argument");
    if (!c->serve) return fail(PR_EINVAL, "serving not started (pr_serve_start)");
    std::unique_lock<std::mutex> lock(c->mu);
    Serve* sv = c->serve;
    if (sv->done.empty() && sv->outstanding == 0) return fail(PR_EINVAL, "no frames outstanding");
    auto ready = [&] { return !sv->done.empty(); };
    if (timeout_ms < 0)
        sv->cv_done.wait(lock, ready);
    else if (timeout_ms > 0)
        sv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready);
    if (sv->done.empty()) return fail(PR_ETIMEOUT, "no frame finished within %d ms", timeout_ms);
    *out = sv->done.front();
    sv->done.pop_front();
    sv->outstanding -= 1;
    return out->status == PR_OK ? PR_OK : fail(out->status, "%s", sv->error_msg.c_str());
}

int pr_serve_stop(pr_ctx* c) {
    if (!c) return fail(PR_EINVAL, "null context");
    if (!c->serve) return fail(PR_EINVAL, "serving not started");
    serve_stop(c);
    // the worker is gone; results stay pollable, so keep the structure but
    // allow a restart only after the remaining results are taken
    return c->serve->error ? fail(c->serve->error, "%s", c->serve->error_msg.c_str()) : PR_OK;
}

}  // extern "C"
