/*
 * FP64 CPU oracle for single-projection PCA reconstruction (Li et al.,
 * "Real-time volumetric image reconstruction and 3D tumor localization based
 * on a single x-ray projection image for lung cancer radiotherapy").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA library is checked against. Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it. It shares no code with the
 * CUDA path.
 *
 * Every routine is a straight loop in double precision:
 *   or_dvf          Eq. 1 / the constraint of Eq. 2: x = mean + sum_k u_k w_k
 *   or_warp         Section 2.2: f(v) = f0 trilinearly interpolated at v + x(v)
 *   or_warp_jac     Section 2.2: h_k(v) = (df/dx)(v) . u_k(v), the exact
 *                   derivative of the trilinear interpolant
 *   or_project      Eq. 2: the projection matrix P (cone-beam ray sums)
 *   or_backproject  the gradient formula after Eq. 4: P^T, the transpose of P
 *   or_tumor        Section 2.3: tumor position through the inverted pull-back
 *                   DVF, by the fixed-point inversion of Chen et al. (ref. 13)
 *   or_invert       Section 2.3 with ref. 13 over the whole grid: the
 *                   push-forward DVF, the inverse of the pull-back field
 *
 * Readings where the paper is silent (each also used by the CUDA path):
 *   - grid: voxel (i,j,k) at origin + (i,j,k)*spacing, origin = -(n-1)/2*spacing;
 *     arrays [nz][ny][nx], fields planar [3][nz][ny][nx], U [K][3][nz][ny][nx];
 *   - the interpolant of a volume is trilinear with zero value outside the grid;
 *     the cell of q is floor(q) (an integer q uses the cell [q, q+1]);
 *   - source S = (SAD sin th, -SAD cos th, 0), detector centre
 *     S + SDD (-sin th, cos th, 0), detector axes u = (cos th, sin th, 0),
 *     v = (0, 0, 1), pixel (iu, iv) centre at (iu - (nu-1)/2) du along u and
 *     (iv - (nv-1)/2) dv along v, detector arrays [nv][nu];
 *   - P f for a ray = ds * sum over s >= 0 of F(S + (s + 1/2) ds d), d the unit
 *     direction to the pixel centre: samples anchored at the source;
 *   - tumor inversion uses the DVF interpolated trilinearly with clamp-to-edge.
 *
 * Built plain (liboracle.so, one thread) for every check. The same source
 * built with OpenMP (liboracle_omp.so) serves only to time the method on all
 * host cores: the loops whose iterations write disjoint outputs (DVF, warp,
 * Jacobian, projection) run in parallel and give bitwise the same results;
 * the transpose, a scatter, accumulates into one buffer per thread that are
 * then added in thread order (the same sums in another order).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the loops below may use (1 in the plain build). */
int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
} or_vol;

typedef struct {
    double sad, sdd;
    int nu, nv;
    double du, dv, ds;
} or_geom;

static size_t vox(const or_vol* v, int i, int j, int k) {
    return ((size_t)k * v->ny + j) * v->nx + i;
}

static void origin(const or_vol* v, double o[3]) {
    o[0] = -0.5 * (v->nx - 1) * v->dx;
    o[1] = -0.5 * (v->ny - 1) * v->dy;
    o[2] = -0.5 * (v->nz - 1) * v->dz;
}

/* Value of volume f at grid index (i,j,k); zero outside the grid. */
static double at(const or_vol* v, const double* f, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= v->nx || j >= v->ny || k >= v->nz) return 0.0;
    return f[vox(v, i, j, k)];
}

/*
 * Trilinear interpolant of f (zero outside the grid) at continuous index q,
 * and, if grad != NULL, its exact partial derivatives with respect to q:
 * dF/dqx = sum over the y,z corner pairs of (wy wz) * (c[1][.][.] - c[0][.][.]).
 */
static double trilinear(const or_vol* v, const double* f, const double q[3], double grad[3]) {
    int i0 = (int)floor(q[0]), j0 = (int)floor(q[1]), k0 = (int)floor(q[2]);
    double tx = q[0] - i0, ty = q[1] - j0, tz = q[2] - k0;
    double c[2][2][2];
    for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1)
            for (int c0 = 0; c0 < 2; ++c0) c[c2][c1][c0] = at(v, f, i0 + c0, j0 + c1, k0 + c2);
    double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
    double val = 0.0;
    for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1)
            for (int c0 = 0; c0 < 2; ++c0) val += wx[c0] * wy[c1] * wz[c2] * c[c2][c1][c0];
    if (grad) {
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                gx += wy[a] * wz[b] * (c[b][a][1] - c[b][a][0]);
                gy += wx[a] * wz[b] * (c[b][1][a] - c[b][0][a]);
                gz += wx[a] * wy[b] * (c[1][b][a] - c[0][b][a]);
            }
        grad[0] = gx;
        grad[1] = gy;
        grad[2] = gz;
    }
    return val;
}

/* Eq. 1 with the constraint of Eq. 2: x = mean + U w, planar [3][N]. */
void or_dvf(const or_vol* v, const double* mean, const double* U, int K, const double* w,
            double* x) {
    size_t n3 = 3 * (size_t)v->nx * v->ny * v->nz;
#pragma omp parallel for schedule(static)
    for (size_t e = 0; e < n3; ++e) {
        double s = mean[e];
        for (int k = 0; k < K; ++k) s += U[(size_t)k * n3 + e] * w[k];
        x[e] = s;
    }
}

/* Continuous index of the pull-back point v + x(v) of voxel (i,j,k). */
static void pullback_index(const or_vol* v, const double* x, int i, int j, int k, double q[3]) {
    size_t n = (size_t)v->nx * v->ny * v->nz, e = vox(v, i, j, k);
    q[0] = i + x[e] / v->dx;
    q[1] = j + x[n + e] / v->dy;
    q[2] = k + x[2 * n + e] / v->dz;
}

/* Section 2.2: the reconstructed image f(v) = F0(v + x(v)), by trilinear interpolation. */
void or_warp(const or_vol* v, const double* f0, const double* x, double* f) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < v->nz; ++k)
        for (int j = 0; j < v->ny; ++j)
            for (int i = 0; i < v->nx; ++i) {
                double q[3];
                pullback_index(v, x, i, j, k, q);
                f[vox(v, i, j, k)] = trilinear(v, f0, q, NULL);
            }
}

/*
 * Section 2.2 (df/dx consistent with the interpolation) and the gradient
 * formula after Eq. 4 (U^T df/dx): h_k(v) = sum_c dF0/dq_c(q(v)) / spacing_c * U[k][c][v],
 * h planar [K][N].
 */
void or_warp_jac(const or_vol* v, const double* f0, const double* x, const double* U, int K,
                 double* h) {
    size_t n = (size_t)v->nx * v->ny * v->nz;
    double sp[3] = {v->dx, v->dy, v->dz};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < v->nz; ++k)
        for (int j = 0; j < v->ny; ++j)
            for (int i = 0; i < v->nx; ++i) {
                double q[3], g[3];
                size_t e = vox(v, i, j, k);
                pullback_index(v, x, i, j, k, q);
                trilinear(v, f0, q, g);
                for (int m = 0; m < K; ++m) {
                    double s = 0.0;
                    for (int c = 0; c < 3; ++c) s += g[c] / sp[c] * U[((size_t)m * 3 + c) * n + e];
                    h[(size_t)m * n + e] = s;
                }
            }
}

/* Source position and unit direction of the ray to pixel (iu, iv) at gantry angle th. */
void or_ray(const or_geom* g, double th, int iu, int iv, double src[3], double dir[3]) {
    double st = sin(th), ct = cos(th);
    double su = (iu - 0.5 * (g->nu - 1)) * g->du, sv = (iv - 0.5 * (g->nv - 1)) * g->dv;
    src[0] = g->sad * st;
    src[1] = -g->sad * ct;
    src[2] = 0.0;
    double pix[3] = {src[0] - g->sdd * st + su * ct, src[1] + g->sdd * ct + su * st, sv};
    double d[3] = {pix[0] - src[0], pix[1] - src[1], pix[2] - src[2]};
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int c = 0; c < 3; ++c) dir[c] = d[c] / len;
}

/*
 * Range of sample numbers s whose points can have a nonzero interpolant:
 * the ray parameter interval inside the index box [-2, n+1] per axis (the
 * interpolant is zero outside (-1, n); the extra index of margin only adds
 * zero-valued samples). Returns 0 when the ray misses the box.
 */
static int sample_range(const or_vol* v, const or_geom* g, const double src[3], const double dir[3],
                        long* s_lo, long* s_hi) {
    double o[3], sp[3] = {v->dx, v->dy, v->dz};
    int nn[3] = {v->nx, v->ny, v->nz};
    origin(v, o);
    double t0 = 0.0, t1 = 1e300;
    for (int c = 0; c < 3; ++c) {
        double lo = o[c] + (-2.0) * sp[c], hi = o[c] + (nn[c] + 1.0) * sp[c];
        if (dir[c] == 0.0) {
            if (src[c] <= lo || src[c] >= hi) return 0;
            continue;
        }
        double ta = (lo - src[c]) / dir[c], tb = (hi - src[c]) / dir[c];
        if (ta > tb) {
            double t = ta;
            ta = tb;
            tb = t;
        }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t1 <= t0) return 0;
    long a = (long)floor(t0 / g->ds - 0.5), b = (long)ceil(t1 / g->ds - 0.5);
    if (a < 0) a = 0;
    if (b < a) return 0;
    *s_lo = a;
    *s_hi = b;
    return 1;
}

static void sample_index(const or_vol* v, const double src[3], const double dir[3], double t,
                         double q[3]) {
    double o[3], sp[3] = {v->dx, v->dy, v->dz};
    origin(v, o);
    for (int c = 0; c < 3; ++c) q[c] = (src[c] + t * dir[c] - o[c]) / sp[c];
}

/* Eq. 2: p = P f, one line integral (source-anchored sample sum) per pixel, p [nv][nu]. */
void or_project(const or_vol* v, const or_geom* g, double th, const double* f, double* p) {
#pragma omp parallel for schedule(dynamic)
    for (int iv = 0; iv < g->nv; ++iv)
        for (int iu = 0; iu < g->nu; ++iu) {
            double src[3], dir[3], acc = 0.0;
            long s0, s1;
            or_ray(g, th, iu, iv, src, dir);
            if (sample_range(v, g, src, dir, &s0, &s1))
                for (long s = s0; s <= s1; ++s) {
                    double q[3];
                    sample_index(v, src, dir, (s + 0.5) * g->ds, q);
                    acc += trilinear(v, f, q, NULL);
                }
            p[(size_t)iv * g->nu + iu] = g->ds * acc;
        }
}

/*
 * The transpose P^T of or_project: every sample of every ray spreads
 * ds * r(ray) over the eight grid points of its cell with the same trilinear
 * weights (points outside the grid are dropped, as their values are zero in P).
 */
/* One detector row of or_backproject, added into out. */
static void backproject_row(const or_vol* v, const or_geom* g, double th, const double* r, int iv, double* out) {
    for (int iu = 0; iu < g->nu; ++iu) {
        double src[3], dir[3];
        long s0, s1;
        double val = g->ds * r[(size_t)iv * g->nu + iu];
        or_ray(g, th, iu, iv, src, dir);
        if (!sample_range(v, g, src, dir, &s0, &s1)) continue;
        for (long s = s0; s <= s1; ++s) {
            double q[3];
            sample_index(v, src, dir, (s + 0.5) * g->ds, q);
            int i0 = (int)floor(q[0]), j0 = (int)floor(q[1]), k0 = (int)floor(q[2]);
            double tx = q[0] - i0, ty = q[1] - j0, tz = q[2] - k0;
            double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
            for (int c2 = 0; c2 < 2; ++c2)
                for (int c1 = 0; c1 < 2; ++c1)
                    for (int c0 = 0; c0 < 2; ++c0) {
                        int i = i0 + c0, j = j0 + c1, k = k0 + c2;
                        if (i < 0 || j < 0 || k < 0 || i >= v->nx || j >= v->ny || k >= v->nz) continue;
                        out[vox(v, i, j, k)] += wx[c0] * wy[c1] * wz[c2] * val;
                    }
        }
    }
}

void or_backproject(const or_vol* v, const or_geom* g, double th, const double* r, double* out) {
    size_t n = (size_t)v->nx * v->ny * v->nz;
    memset(out, 0, n * sizeof(double));
#ifdef _OPENMP
    int nt = omp_get_max_threads();
    double* priv = nt > 1 ? (double*)calloc((size_t)nt * n, sizeof(double)) : NULL;
    if (priv) {
#pragma omp parallel
        {
            double* mine = priv + (size_t)omp_get_thread_num() * n;
#pragma omp for schedule(dynamic)
            for (int iv = 0; iv < g->nv; ++iv) backproject_row(v, g, th, r, iv, mine);
        }
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < n; ++e)
            for (int t = 0; t < nt; ++t) out[e] += priv[(size_t)t * n + e];
        free(priv);
        return;
    }
#endif
    for (int iv = 0; iv < g->nv; ++iv) backproject_row(v, g, th, r, iv, out);
}

/* DVF x = mean + U w interpolated trilinearly at world point p, clamped to the grid edge. */
static void dvf_at(const or_vol* v, const double* mean, const double* U, int K, const double* w,
                   const double p[3], double out[3]) {
    double o[3], sp[3] = {v->dx, v->dy, v->dz};
    int nn[3] = {v->nx, v->ny, v->nz};
    int i0[3];
    double t[3];
    size_t n = (size_t)v->nx * v->ny * v->nz;
    origin(v, o);
    for (int c = 0; c < 3; ++c) {
        double q = (p[c] - o[c]) / sp[c];
        if (q < 0.0) q = 0.0;
        if (q > nn[c] - 1) q = nn[c] - 1;
        i0[c] = (int)floor(q);
        if (i0[c] > nn[c] - 2) i0[c] = nn[c] - 2;
        if (i0[c] < 0) i0[c] = 0;
        t[c] = q - i0[c];
    }
    for (int comp = 0; comp < 3; ++comp) {
        double acc = 0.0;
        for (int c2 = 0; c2 < 2; ++c2)
            for (int c1 = 0; c1 < 2; ++c1)
                for (int c0 = 0; c0 < 2; ++c0) {
                    int i = i0[0] + c0, j = i0[1] + c1, k = i0[2] + c2;
                    if (i >= v->nx || j >= v->ny || k >= v->nz) continue; /* n == 1 axes */
                    size_t e = (size_t)comp * n + vox(v, i, j, k);
                    double xv = mean[e];
                    for (int m = 0; m < K; ++m) xv += U[(size_t)m * 3 * n + e] * w[m];
                    double wgt = (c0 ? t[0] : 1.0 - t[0]) * (c1 ? t[1] : 1.0 - t[1]) *
                                 (c2 ? t[2] : 1.0 - t[2]);
                    acc += wgt * xv;
                }
        out[comp] = acc;
    }
}

/*
 * Section 2.3: tumor position p in the current image, whose pull-back DVF maps
 * it to the reference-image tumor c0: p + x(p) = c0. Fixed-point iteration of
 * ref. 13 evaluated at one point: p <- c0 - x(p), starting from p = c0, until
 * the Euclidean step is below tol (mm) or max_iter steps. Returns the number of
 * steps taken.
 */
int or_tumor(const or_vol* v, const double* mean, const double* U, int K, const double* w,
             const double c0[3], double tol, int max_iter, double p[3]) {
    double cur[3] = {c0[0], c0[1], c0[2]};
    int it = 0;
    while (it < max_iter) {
        double x[3], nxt[3], d2 = 0.0;
        dvf_at(v, mean, U, K, w, cur, x);
        for (int c = 0; c < 3; ++c) {
            nxt[c] = c0[c] - x[c];
            d2 += (nxt[c] - cur[c]) * (nxt[c] - cur[c]);
            cur[c] = nxt[c];
        }
        ++it;
        if (sqrt(d2) < tol) break;
    }
    for (int c = 0; c < 3; ++c) p[c] = cur[c];
    return it;
}

/* DVF value at a world point (exported for the tumor round-trip check). */
void or_dvf_at(const or_vol* v, const double* mean, const double* U, int K, const double* w,
               const double p[3], double out[3]) {
    dvf_at(v, mean, U, K, w, p, out);
}

/*
 * Section 2.3 with ref. 13 over the whole grid: the push-forward DVF y that
 * inverts the pull-back field x = mean + sum_k u_k w_k, i.e. the displacement
 * with  u + y(u) + x(u + y(u)) = u  at every voxel centre u. Chen et al.'s
 * fixed-point iteration updates the whole field in each sweep,
 *     y_{m+1}(u) = -x(u + y_m(u)),   y_0 = 0,
 * with x trilinear and clamped to the grid edge (dvf_at), and stops when the
 * largest update of a sweep (Euclidean, mm) is below tol or after max_iter
 * sweeps. A voxel's update reads only its own previous value, so the sweep
 * runs in place. y: [3][nz][ny][nx] doubles (mm). Returns the sweep count.
 */
int or_invert(const or_vol* v, const double* mean, const double* U, int K, const double* w,
              double tol, int max_iter, double* y) {
    size_t n = (size_t)v->nx * v->ny * v->nz;
    double o[3];
    origin(v, o);
    memset(y, 0, 3 * n * sizeof(double));
    int sweeps = 0;
    while (sweeps < max_iter) {
        double largest = 0.0;
        for (int k = 0; k < v->nz; ++k)
            for (int j = 0; j < v->ny; ++j)
                for (int i = 0; i < v->nx; ++i) {
                    size_t e = vox(v, i, j, k);
                    double u[3] = {o[0] + i * v->dx, o[1] + j * v->dy, o[2] + k * v->dz};
                    double pt[3], x[3], d2 = 0.0;
                    for (int c = 0; c < 3; ++c) pt[c] = u[c] + y[(size_t)c * n + e];
                    dvf_at(v, mean, U, K, w, pt, x);
                    for (int c = 0; c < 3; ++c) {
                        double next = -x[c];
                        double step = next - y[(size_t)c * n + e];
                        d2 += step * step;
                        y[(size_t)c * n + e] = next;
                    }
                    if (d2 > largest) largest = d2;
                }
        ++sweeps;
        if (sqrt(largest) < tol) break;
    }
    return sweeps;
}
