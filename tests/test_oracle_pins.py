"""Pins of the FP64 oracle against facts it does not compute itself.

Each test ties one oracle routine to a closed form, an exact special case, a
library routine, a brute-force construction or a finite difference, so that a
dropped term, a wrong sign, a swapped axis or a transposed operand fails at
least one of them.
"""

import math

import numpy as np
import pytest

from oracle import oracle as O
from phantom import Geometry, Volume, build_pca, phantom_volume, training_dvfs, tumor_centre

RNG = np.random.default_rng(12345)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _grid_points(vol):
    ax, ay, az = vol.axes()
    return np.meshgrid(az, ay, ax, indexing="ij")  # z, y, x


# ----------------------------------------------------------------------------
# Eq. 1: DVF synthesis
# ----------------------------------------------------------------------------


def test_dvf_zero_w_is_mean_exactly():
    vol = Volume(7, 5, 4, 1.0, 2.0, 3.0)
    mean = RNG.standard_normal((3,) + vol.shape)
    U = RNG.standard_normal((3, 3) + vol.shape)
    assert np.array_equal(O.dvf(vol, mean, U, np.zeros(3)), mean)


def test_dvf_matches_tensor_contraction_and_is_affine_in_w():
    vol = Volume(6, 5, 4, 1.0, 2.0, 3.0)
    mean = RNG.standard_normal((3,) + vol.shape)
    U = RNG.standard_normal((4, 3) + vol.shape)
    w1, w2 = RNG.standard_normal(4), RNG.standard_normal(4)
    expect = mean + np.tensordot(w1, U, axes=(0, 0))
    assert _rel(O.dvf(vol, mean, U, w1), expect) < 1e-14
    lhs = O.dvf(vol, mean, U, w1 + w2) - mean
    rhs = (O.dvf(vol, mean, U, w1) - mean) + (O.dvf(vol, mean, U, w2) - mean)
    assert _rel(lhs, rhs) < 1e-13


# ----------------------------------------------------------------------------
# Section 2.2: trilinear warp and its exact derivative
# ----------------------------------------------------------------------------


def test_warp_zero_dvf_is_identity_bitwise():
    vol = Volume(9, 7, 5, 2.0, 2.0, 2.5)
    f0 = RNG.random(vol.shape)
    assert np.array_equal(O.warp(vol, f0, np.zeros((3,) + vol.shape)), f0)


def test_warp_integer_shift_is_exact_shift_with_zero_fill():
    vol = Volume(9, 8, 7, 2.0, 3.0, 2.5)
    f0 = RNG.random(vol.shape)
    sx, sy, sz = 2, -1, 3  # voxels; pull-back: f(v) = f0(v + s)
    x = np.zeros((3,) + vol.shape)
    x[0], x[1], x[2] = sx * vol.dx, sy * vol.dy, sz * vol.dz
    f = O.warp(vol, f0, x)
    expect = np.zeros(vol.shape)
    for k in range(vol.nz):
        for j in range(vol.ny):
            for i in range(vol.nx):
                ii, jj, kk = i + sx, j + sy, k + sz
                if 0 <= ii < vol.nx and 0 <= jj < vol.ny and 0 <= kk < vol.nz:
                    expect[k, j, i] = f0[kk, jj, ii]
    assert np.array_equal(f, expect)


def test_warp_reproduces_affine_image_under_subvoxel_shift():
    vol = Volume(10, 9, 8, 2.0, 3.0, 2.5)
    zi, yi, xi = np.meshgrid(np.arange(vol.nz), np.arange(vol.ny), np.arange(vol.nx), indexing="ij")
    beta = np.array([0.3, -0.7, 1.1])
    f0 = 2.0 + beta[0] * xi + beta[1] * yi + beta[2] * zi
    shift = np.array([0.37, -0.81, 0.55])  # mm
    x = np.zeros((3,) + vol.shape)
    for c in range(3):
        x[c] = shift[c]
    f = O.warp(vol, f0, x)
    q = shift / vol.spacing
    expect = 2.0 + beta[0] * (xi + q[0]) + beta[1] * (yi + q[1]) + beta[2] * (zi + q[2])
    inside = ((xi + q[0] >= 0) & (xi + q[0] <= vol.nx - 1) & (yi + q[1] >= 0) &
              (yi + q[1] <= vol.ny - 1) & (zi + q[2] >= 0) & (zi + q[2] <= vol.nz - 1))
    assert inside.sum() > 100
    assert np.max(np.abs(f[inside] - expect[inside])) < 1e-12
    # Beyond the support (-1, n) the interpolant is exactly zero.
    x[0] = -5.0 * vol.nx * vol.dx
    assert np.all(O.warp(vol, f0, x) == 0.0)


def test_warp_jacobian_of_affine_image_is_its_slope():
    vol = Volume(10, 9, 8, 2.0, 3.0, 2.5)
    zi, yi, xi = np.meshgrid(np.arange(vol.nz), np.arange(vol.ny), np.arange(vol.nx), indexing="ij")
    beta = np.array([0.3, -0.7, 1.1])  # per index step
    f0 = 2.0 + beta[0] * xi + beta[1] * yi + beta[2] * zi
    x = np.zeros((3,) + vol.shape)
    x[0], x[1], x[2] = 0.41, -0.93, 0.77
    U = RNG.standard_normal((2, 3) + vol.shape)
    h = O.warp_jac(vol, f0, x, U)
    q = np.array([0.41, -0.93, 0.77]) / vol.spacing
    inside = ((xi + q[0] > 0) & (xi + q[0] < vol.nx - 1) & (yi + q[1] > 0) &
              (yi + q[1] < vol.ny - 1) & (zi + q[2] > 0) & (zi + q[2] < vol.nz - 1))
    for k in range(2):
        expect = sum(beta[c] / vol.spacing[c] * U[k, c] for c in range(3))
        assert np.max(np.abs(h[k][inside] - expect[inside])) < 1e-12


def test_warp_jacobian_matches_central_differences():
    vol = Volume(12, 11, 10, 2.0, 3.0, 2.5)
    f0 = RNG.random(vol.shape)
    mean = 1.5 * RNG.standard_normal((3,) + vol.shape)
    U = RNG.standard_normal((3, 3) + vol.shape)
    w = np.array([0.3, -0.2, 0.4])
    x = O.dvf(vol, mean, U, w)
    h = O.warp_jac(vol, f0, x, U)
    eps = 1e-6
    q = np.stack([x[c] / vol.spacing[c] for c in range(3)])
    frac = q - np.floor(q)
    zi, yi, xi = np.meshgrid(np.arange(vol.nz), np.arange(vol.ny), np.arange(vol.nx), indexing="ij")
    idx = np.stack([xi, yi, zi]) + q
    dims = np.array([vol.nx, vol.ny, vol.nz]).reshape(3, 1, 1, 1)
    ok = np.all((frac > 1e-3) & (frac < 1 - 1e-3), axis=0) & np.all((idx > -1) & (idx < dims), axis=0)
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        fp = O.warp(vol, f0, O.dvf(vol, mean, U, w + e))
        fm = O.warp(vol, f0, O.dvf(vol, mean, U, w - e))
        fd = (fp - fm) / (2 * eps)
        assert ok.sum() > 200
        assert _rel(h[k][ok], fd[ok]) < 1e-7


# ----------------------------------------------------------------------------
# Eq. 2: cone-beam projection P
# ----------------------------------------------------------------------------


def test_central_ray_through_uniform_block_matches_closed_form():
    # nx, nz odd put the isocentre on a voxel centre, so the central ray (odd
    # detector) runs along +y through voxel centres. The interpolant of a
    # uniform block of n voxels integrates to mu * n * dy along y; the
    # source-anchored midpoint sum errs by at most |slope jump| ds^2 / 8 at each
    # of the four kinks: mu ds^2 / (2 dy) in total.
    vol = Volume(9, 11, 9, 2.0, 3.0, 2.5)
    mu = 0.02
    f = np.full(vol.shape, mu)
    for ds in (0.7, 0.35, 1.3):
        g = Geometry(1000.0, 1500.0, 3, 3, 1.0, 1.0, ds)
        p = O.project(vol, g, 0.0, f)
        exact = mu * vol.ny * vol.dy
        assert abs(p[1, 1] - exact) <= mu * ds * ds / (2 * vol.dy) + 1e-12


def test_projection_rotates_with_the_gantry():
    # Projecting f at angle th + 90 deg equals projecting f rotated by -90 deg
    # about z at angle th (square in-plane grid, so the rotation maps the grid
    # onto itself): g[k, j, i] = f[k, i, n - 1 - j].
    vol = Volume(10, 10, 6, 2.0, 2.0, 2.5)
    f = RNG.random(vol.shape)
    g = np.empty_like(f)
    n = vol.nx
    for j in range(n):
        for i in range(n):
            g[:, j, i] = f[:, i, n - 1 - j]
    geom = Geometry(1000.0, 1500.0, 12, 8, 2.0, 2.5, 0.6)
    th = 0.37
    assert _rel(O.project(vol, geom, th + math.pi / 2, f), O.project(vol, geom, th, g)) < 1e-12


def test_point_object_lands_at_pinhole_position():
    vol = Volume(21, 19, 17, 2.0, 2.0, 2.5)
    geom = Geometry(1000.0, 1500.0, 150, 130, 0.5, 0.5, 0.25)
    i0, j0, k0 = 14, 5, 12
    f = np.zeros(vol.shape)
    f[k0, j0, i0] = 1.0
    P = vol.origin + np.array([i0, j0, k0]) * vol.spacing
    for th in (0.0, 0.6, 2.3):
        S = np.array([geom.sad * math.sin(th), -geom.sad * math.cos(th), 0.0])
        e = np.array([-math.sin(th), math.cos(th), 0.0])
        u = np.array([math.cos(th), math.sin(th), 0.0])
        lam = (P - S) @ e
        iu = geom.sdd * ((P - S) @ u) / lam / geom.du + 0.5 * (geom.nu - 1)
        iv = geom.sdd * (P[2] - S[2]) / lam / geom.dv + 0.5 * (geom.nv - 1)
        p = O.project(vol, geom, th, f)
        assert p.sum() > 0
        vv, uu = np.meshgrid(np.arange(geom.nv), np.arange(geom.nu), indexing="ij")
        cu, cv = (p * uu).sum() / p.sum(), (p * vv).sum() / p.sum()
        assert abs(cu - iu) < 0.35 and abs(cv - iv) < 0.35


def _voxelised_sphere(vol, radius, sub=4):
    ax, ay, az = vol.axes()
    offs = (np.arange(sub) + 0.5) / sub - 0.5
    z, y, x = np.meshgrid(az, ay, ax, indexing="ij")
    acc = np.zeros(vol.shape)
    for ox in offs:
        for oy in offs:
            for oz in offs:
                px, py, pz = x + ox * vol.dx, y + oy * vol.dy, z + oz * vol.dz
                acc += (px * px + py * py + pz * pz < radius * radius)
    return acc / sub ** 3


def test_sphere_chords_converge_to_closed_form():
    radius = 14.0
    errs = []
    for d in (2.0, 1.0):
        n = int(round(40.0 / d))
        vol = Volume(n, n, n, d, d, d)
        f = _voxelised_sphere(vol, radius)
        geom = Geometry(1000.0, 1500.0, 15, 13, 2.4, 2.4, d / 2)
        th = 0.45
        p = O.project(vol, geom, th, f)
        chord = np.zeros_like(p)
        for iv in range(geom.nv):
            for iu in range(geom.nu):
                src, dr = O.ray(geom, th, iu, iv)
                tc = -src @ dr
                dist2 = src @ src - tc * tc
                chord[iv, iu] = 2 * math.sqrt(max(radius ** 2 - dist2, 0.0))
        core = chord > 2 * math.sqrt(radius ** 2 - (radius - 3.0) ** 2)
        errs.append(_rel(p[core], chord[core]))
    assert errs[0] < 0.02
    assert errs[1] < 0.6 * errs[0]


# ----------------------------------------------------------------------------
# P^T: exact transpose
# ----------------------------------------------------------------------------


def test_adjoint_identity():
    vol = Volume(12, 10, 8, 2.0, 3.0, 2.5)
    geom = Geometry(1000.0, 1500.0, 9, 7, 3.0, 3.5, 1.1)
    for th in (0.3, 1.9):
        x = RNG.standard_normal(vol.shape)
        y = RNG.standard_normal((geom.nv, geom.nu))
        lhs = float(np.sum(O.project(vol, geom, th, x) * y))
        rhs = float(np.sum(x * O.backproject(vol, geom, th, y)))
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_dense_transpose_on_8_cube():
    vol = Volume(8, 8, 8, 3.0, 3.0, 3.0)
    geom = Geometry(1000.0, 1500.0, 6, 6, 6.0, 6.0, 1.5)
    th = 0.8
    n, R = vol.n, geom.n_rays
    P = np.empty((R, n))
    for e in range(n):
        unit = np.zeros(n)
        unit[e] = 1.0
        P[:, e] = O.project(vol, geom, th, unit.reshape(vol.shape)).ravel()
    PT = np.empty((n, R))
    for r in range(R):
        unit = np.zeros(R)
        unit[r] = 1.0
        PT[:, r] = O.backproject(vol, geom, th, unit.reshape(geom.nv, geom.nu)).ravel()
    assert np.count_nonzero(P) > 1000
    assert np.max(np.abs(P - PT.T)) < 1e-13


# ----------------------------------------------------------------------------
# Eqs. 2-4: cost, intensity fit, gradient
# ----------------------------------------------------------------------------


def _tiny_model(K=3, n=16, d=4.0):
    vol = Volume(n, n, n, d, d, d)
    f0 = phantom_volume(vol)
    pca = build_pca(training_dvfs(vol), K)
    return O.Model(vol, f0, pca.mean, pca.U, tumor_centre(vol)), pca


def test_fit_ab_is_least_squares_minimiser():
    p = RNG.random((7, 9)) * 3
    y = 0.8 * p + 0.1 + 0.05 * RNG.standard_normal(p.shape)
    a, b = O.fit_ab(p, y)
    A = np.stack([y.ravel(), np.ones(y.size)], axis=1)
    ref = np.linalg.lstsq(A, p.ravel(), rcond=None)[0]
    assert abs(a - ref[0]) < 1e-12 and abs(b - ref[1]) < 1e-12
    J = O.cost(p, y, a, b)
    for da, db in ((1e-3, 0), (-1e-3, 0), (0, 1e-3), (0, -1e-3), (1e-3, -1e-3)):
        assert O.cost(p, y, a + da, b + db) > J
    assert abs(O.cost(p, y, a, b) - np.sum((p - a * y - b) ** 2)) < 1e-12


def test_gradient_matches_central_differences_of_J():
    m, pca = _tiny_model()
    geom = Geometry(1000.0, 1500.0, 24, 24, 3.2, 3.2, 2.0)
    th = 0.5
    y = O.evaluate(m, geom, th, np.array([0.6, -0.4, 0.2])).p
    y = y + 0.02 * RNG.standard_normal(y.shape)
    w = np.array([0.13, 0.21, -0.17])
    a, b = 1.07, 0.013
    g, J, _ = O.gradient(m, geom, th, w, a, b, y)
    eps = 1e-5
    fd = np.empty(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        Jp = O.cost(O.evaluate(m, geom, th, w + e).p, y, a, b)
        Jm = O.cost(O.evaluate(m, geom, th, w - e).p, y, a, b)
        fd[k] = (Jp - Jm) / (2 * eps)
    assert _rel(g, fd) < 1e-6
    assert abs(J - O.cost(O.evaluate(m, geom, th, w).p, y, a, b)) < 1e-12 * J


def test_gradient_equals_forward_mode_contraction():
    # sum_v (P^T r)(v) h_k(v) = sum_rays r (P h_k): the adjoint and the
    # forward-mode form of the same derivative.
    m, pca = _tiny_model(n=20, d=3.2)
    geom = Geometry(1000.0, 1500.0, 20, 18, 3.0, 3.0, 1.6)
    th = 1.1
    w = np.array([0.3, -0.1, 0.05])
    y = O.evaluate(m, geom, th, w * 1.3).p
    a, b = 0.97, -0.01
    g, J, p = O.gradient(m, geom, th, w, a, b, y)
    x = O.dvf(m.vol, m.mean, m.U, w)
    h = O.warp_jac(m.vol, m.f0, x, m.U)
    r = p - a * y - b
    fwd = np.array([2 * np.sum(r * O.project(m.vol, geom, th, h[k])) for k in range(3)])
    assert _rel(g, fwd) < 1e-10


# ----------------------------------------------------------------------------
# Section 2.2: alternation with Armijo's rule
# ----------------------------------------------------------------------------


# The two rules the solver offers: the paper's plain Armijo backtracking (the
# oracle's default) and the quadratic step model with power-of-two steps and the
# resolvability guard that the CUDA library runs by default.
RULES = {"plain": dict(), "model": dict(step_model=1, min_decrease=1e-6)}


@pytest.mark.parametrize("rule", sorted(RULES))
def test_cost_never_increases_across_steps(small_case, rule):
    c = small_case
    m = O.Model(c["vol"], c["f0"], c["pca"].mean, c["pca"].U, c["c0"])
    f_t = O.warp(c["vol"], c["f0"], c["x_test"])
    p_t = O.project(c["vol"], c["geom"], c["angle"], f_t)
    y = p_t + 0.01 * p_t * np.random.default_rng(0).standard_normal(p_t.shape)
    res = O.reconstruct(m, c["geom"], c["angle"], y, np.zeros(3), O.SolveOptions(max_iters=6, **RULES[rule]))
    a0, b0 = O.fit_ab(O.evaluate(m, c["geom"], c["angle"], np.zeros(3)).p, y)
    J_prev = O.cost(O.evaluate(m, c["geom"], c["angle"], np.zeros(3)).p, y, a0, b0)
    assert res.iters == 6
    for h in res.history:
        assert h["J_step1"] <= J_prev  # step 1 (Armijo, fixed a, b)
        assert h["J_step2"] <= h["J_step1"] + 1e-12 * J_prev  # step 2 (exact minimiser)
        J_prev = h["J_step2"]


def test_single_mode_recovers_true_coefficient():
    # One PCA mode, noise-free target inside the model: the alternation reaches
    # w_true, a = 1, b = 0 (the unique zero-cost point).
    m, pca = _tiny_model(K=1, n=24, d=3.0)
    geom = Geometry(1000.0, 1500.0, 32, 32, 2.4, 2.4, 1.5)
    th = 0.2
    w_true = np.array([0.9])
    y = O.evaluate(m, geom, th, w_true).p
    for rule in RULES.values():
        res = O.reconstruct(m, geom, th, y, np.zeros(1), O.SolveOptions(max_iters=40, grad_tol=1e-9, **rule))
        assert abs(res.w[0] - w_true[0]) < 1e-4
        assert abs(res.a - 1.0) < 1e-5 and abs(res.b) < 1e-5


# ---- one trial's decisions (step_choice), on hand-derived cases ----
#
# Along -g the cost of an exact quadratic is J(mu) = J0 - mu G + kappa mu^2 / 2
# (G = |g|^2), whose minimiser is mu* = G / kappa. The numbers below are chosen
# so that every quantity is exact in binary floating point and the expected
# factor is read off by hand.

PLAIN = O.SolveOptions()
MODEL = O.SolveOptions(step_model=1)  # quadratic model, guard off


def _quad(J0, G, kappa, mu):
    return J0 - mu * G + 0.5 * kappa * mu * mu


@pytest.mark.parametrize("kappa, expected", [
    (32.0, 0.125),   # mu* = 1/8 of mu: backtrack exactly to the minimiser
    (20.0, 0.125),   # mu* = 0.2 mu: rounded DOWN to a power of two (nearest would be 1/4)
    (64.0, 0.0625),  # mu* = 1/16 of mu: the lower clamp's edge
    (400.0, 0.0625),  # mu* = 0.01 mu: clamped up to 1/16
])
def test_step_choice_backtracks_to_the_quadratic_minimiser(kappa, expected):
    J0, G, mu = 10.0, 4.0, 1.0
    ok, stop, f = O.step_choice(J0, _quad(J0, G, kappa, mu), mu, G, 0, MODEL)
    assert (ok, stop) == (False, False)
    assert f == expected


def test_step_choice_backtrack_is_capped_by_beta():
    # mu* = 0.3 mu on a rejected trial; with beta = 1/8 the cap binds (1/8,
    # where the uncapped power-of-two floor of 0.3 would be 1/4)
    J0, G, mu = 10.0, 4.0, 1.0
    kappa = G / 0.3
    o = O.SolveOptions(step_model=1, beta=0.125)
    ok, stop, f = O.step_choice(J0, _quad(J0, G, kappa, mu), mu, G, 0, o)
    assert (ok, stop, f) == (False, False, 0.125)


@pytest.mark.parametrize("mu, kappa, expected", [
    (1.0, 4.0 / 1.5, 1.0),  # mu* = 1.5 mu: next first trial = mu (power-of-two floor)
    (1.0, 0.8, 2.0),        # mu* = 5 mu: capped at step_growth = 2 (uncapped floor would be 4)
    (2.0, 1.0, 2.0),        # mu* = 4 = exactly 2 mu: the cap's edge
])
def test_step_choice_next_step_after_acceptance(mu, kappa, expected):
    J0, G = 10.0, 4.0
    ok, stop, f = O.step_choice(J0, _quad(J0, G, kappa, mu), mu, G, 0, MODEL)
    assert (ok, stop) == (True, False)
    assert f == expected


def test_step_choice_without_positive_curvature_grows_by_the_plain_factor():
    # J(mu) at or below the tangent line: no quadratic minimiser, growth factor 2
    ok, stop, f = O.step_choice(10.0, 5.0, 1.0, 4.0, 0, MODEL)
    assert (ok, stop, f) == (True, False, 2.0)


def test_step_choice_armijo_test_flips_exactly_at_the_sufficient_decrease_line():
    # J = 10, mu = 1/2, |g|^2 = 8, c1 = 1/4: the line J - c1 mu |g|^2 is 9
    o = O.SolveOptions(c1=0.25)
    assert O.step_choice(10.0, 9.0, 0.5, 8.0, 0, o)[0] is True
    assert O.step_choice(10.0, float(np.nextafter(9.0, 10.0)), 0.5, 8.0, 0, o)[0] is False
    assert O.step_choice(10.0, float(np.nextafter(9.0, 0.0)), 0.5, 8.0, 0, o)[0] is True


def test_step_choice_plain_rule_uses_fixed_factors():
    o = O.SolveOptions(beta=0.3, step_growth=2.0, step_growth_bt=1.0)
    J0, G, mu = 10.0, 4.0, 1.0
    rej = _quad(J0, G, 32.0, mu)   # rejected (J rises)
    acc = _quad(J0, G, 0.8, mu)    # accepted
    assert O.step_choice(J0, rej, mu, G, 0, o) == (False, False, 0.3)   # beta, not a power of two
    assert O.step_choice(J0, acc, mu, G, 0, o) == (True, False, 2.0)    # first-try acceptance
    assert O.step_choice(J0, acc, mu, G, 3, o) == (True, False, 1.0)    # after backtracking
    assert O.step_choice(J0, rej, mu, G, 0, PLAIN)[:2] == (False, False)  # no guard: never a stop


def test_step_choice_resolvability_guard():
    # guard at 2^-20 of J = 2^20: a trial resolves a decrease above exactly 1
    o = O.SolveOptions(step_model=1, min_decrease=2.0 ** -20)
    J = 2.0 ** 20
    # predicted decrease mu G = 1, not above the threshold: a rejected trial stops
    assert O.step_choice(J, J, 1.0, 1.0, 0, o) == (False, True, 1.0)
    # the same trial with the guard off backtracks (to the model's minimiser,
    # mu* = mu / 2 here: kappa = 2 G / mu)
    assert O.step_choice(J, J, 1.0, 1.0, 0, MODEL) == (False, False, 0.5)
    # just above the threshold the guard lets the trial backtrack
    G = float(np.nextafter(1.0, 2.0))
    assert O.step_choice(J, J, 1.0, G, 0, o)[:2] == (False, False)
    # an accepted trial below the threshold ignores the model (mu* = 0.75 mu
    # would give 1/2) and grows by the plain factor 2
    G = 0.5
    Jt = _quad(J, G, G / 0.75, 1.0)
    assert O.step_choice(J, Jt, 1.0, G, 0, MODEL) == (True, False, 0.5)
    assert O.step_choice(J, Jt, 1.0, G, 0, o) == (True, False, 2.0)


def _quadratic_problem(K=2):
    """A model whose projections are exactly affine in w: f0 is an affine
    image and the modes vanish near the grid faces, so every pull-back point
    stays inside the grid, where trilinear interpolation reproduces the affine
    f0 exactly: f = f0 + s . x (s = f0's slope), p(w) = p(0) + A w, and J is an
    exact quadratic in (w, a, b)."""
    vol = Volume(16, 16, 16, 4.0, 4.0, 4.0)
    Z, Y, X = _grid_points(vol)
    f0 = 0.02 + 1e-4 * X + 2e-4 * Y - 1.5e-4 * Z
    bump = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 12.0 ** 2))
    bump *= (np.abs(X) < 20) & (np.abs(Y) < 20) & (np.abs(Z) < 20)  # 2 voxels of zero margin
    U = np.zeros((K, 3) + vol.shape)
    U[0, 2] = 3.0 * bump                 # SI
    U[1, 1] = 2.0 * bump * (X / 20.0)    # AP, sheared laterally
    m = O.Model(vol, f0, np.zeros((3,) + vol.shape), U, np.zeros(3))
    return m, vol


def test_solve_reaches_the_closed_form_minimiser_of_an_exact_quadratic():
    m, vol = _quadratic_problem()
    geom = Geometry(1000.0, 1500.0, 24, 24, 4.0, 4.0, 2.0)
    th = 0.7
    p0 = O.evaluate(m, geom, th, np.zeros(2)).p.ravel()
    A = np.stack([O.evaluate(m, geom, th, e).p.ravel() - p0 for e in np.eye(2)], axis=1)
    w_true = np.array([0.8, -0.6])
    # the model really is affine in w (brute force at another point)
    assert _rel(O.evaluate(m, geom, th, w_true).p.ravel(), p0 + A @ w_true) < 1e-12
    y = (p0 + A @ w_true) * (1.0 + 0.01 * RNG.standard_normal(p0.size))
    # closed form: min over (w, a, b) of |p0 + A w - a y - b|^2, by least squares
    M = np.concatenate([A, -y[:, None], -np.ones((p0.size, 1))], axis=1)
    sol = np.linalg.lstsq(M, -p0, rcond=None)[0]
    w_star, a_star, b_star = sol[:2], sol[2], sol[3]
    J_star = float(np.sum((p0 + A @ w_star - a_star * y - b_star) ** 2))
    yy = y.reshape(geom.nv, geom.nu)
    # the paper's plain backtracking and the quadratic step model (guard off)
    # both reach the minimiser
    for rule in (dict(), dict(step_model=1)):
        res = O.reconstruct(m, geom, th, yy, np.zeros(2), O.SolveOptions(max_iters=200, grad_tol=1e-10, **rule))
        assert _rel(res.w, w_star) < 1e-6, (rule, res.w, w_star, res.iters, res.stop_reason)
        assert abs(res.a - a_star) < 1e-6 * abs(a_star)
        assert (res.J - J_star) <= 1e-9 * J_star
    # with the resolvability guard at 1e-6 the solve stops once no step can
    # lower J by more than that fraction: J is then within 1e-6 of the minimum,
    # while w may still lie anywhere along the valley's flat direction
    res = O.reconstruct(m, geom, th, yy, np.zeros(2), O.SolveOptions(max_iters=200, grad_tol=1e-10, **RULES["model"]))
    assert res.stop_reason == O.STOP_RESOLVED
    assert 0.0 <= res.J - J_star <= 1e-6 * J_star


# ----------------------------------------------------------------------------
# Section 2.3: tumor by fixed-point inversion
# ----------------------------------------------------------------------------


def test_tumor_under_translation_is_c0_minus_shift():
    vol = Volume(16, 14, 12, 2.0, 2.0, 2.5)
    t = np.array([1.3, -2.1, 4.4])
    mean = np.zeros((3,) + vol.shape)
    for c in range(3):
        mean[c] = t[c]
    U = RNG.standard_normal((2, 3) + vol.shape)
    c0 = np.array([-3.0, 2.0, 1.5])
    p, steps = O.tumor(vol, mean, U, np.zeros(2), c0, tol=1e-12)
    assert np.max(np.abs(p - (c0 - t))) < 1e-12
    assert steps <= 3


def test_tumor_under_affine_dvf_solves_linear_system():
    # Trilinear interpolation reproduces an affine field exactly, so the fixed
    # point of p = c0 - (A p + t) is (I + A)^-1 (c0 - t).
    vol = Volume(20, 18, 16, 2.0, 2.5, 3.0)
    A = np.array([[0.05, -0.02, 0.01], [0.03, 0.04, -0.02], [-0.01, 0.02, 0.06]])
    t = np.array([0.7, -1.2, 2.0])
    z, y, x = _grid_points(vol)
    pts = np.stack([x, y, z])
    mean = np.einsum("ab,b...->a...", A, pts) + t.reshape(3, 1, 1, 1)
    U = np.zeros((1, 3) + vol.shape)
    c0 = np.array([4.0, -3.0, 2.5])
    p, _ = O.tumor(vol, mean, U, np.zeros(1), c0, tol=1e-13, max_iter=200)
    expect = np.linalg.solve(np.eye(3) + A, c0 - t)
    assert np.max(np.abs(p - expect)) < 1e-10


def test_tumor_round_trip_on_pca_dvf(small_case):
    c = small_case
    w = np.array([1.2, -0.3, 0.1])
    p, steps = O.tumor(c["vol"], c["pca"].mean, c["pca"].U, w, c["c0"], tol=1e-13, max_iter=200)
    x = O.dvf_at(c["vol"], c["pca"].mean, c["pca"].U, w, p)
    assert np.max(np.abs(p + x - c["c0"])) < 1e-9
    assert steps < 200


# ----------------------------------------------------------------------------
# Section 2.3 with ref. 13: the push-forward (inverse) DVF on the whole grid
# ----------------------------------------------------------------------------


def test_inverse_field_of_translation_is_minus_the_shift():
    vol = Volume(16, 14, 12, 2.0, 2.0, 2.5)
    t = np.array([1.3, -2.1, 4.4])
    mean = np.zeros((3,) + vol.shape)
    for c in range(3):
        mean[c] = t[c]
    U = RNG.standard_normal((2, 3) + vol.shape)
    y, sweeps = O.invert(vol, mean, U, np.zeros(2), tol=1e-12)
    for c in range(3):
        assert np.max(np.abs(y[c] + t[c])) < 1e-12
    assert sweeps <= 3


def test_inverse_field_of_affine_dvf_is_the_closed_form():
    # x(p) = A p + t (trilinear reproduces it inside the grid), so u + y + A(u + y) + t = u
    # gives y(u) = (I + A)^-1 (u - t) - u. Checked where every iterate stays inside the grid.
    vol = Volume(20, 18, 16, 2.0, 2.5, 3.0)
    A0 = np.array([[0.05, -0.02, 0.01], [0.03, 0.04, -0.02], [-0.01, 0.02, 0.06]])
    A1 = np.array([[0.02, 0.01, 0.0], [-0.01, 0.03, 0.01], [0.0, -0.02, 0.01]])
    t0, t1 = np.array([0.7, -1.2, 2.0]), np.array([0.3, 0.5, -0.4])
    z, yy, x = _grid_points(vol)
    pts = np.stack([x, yy, z])
    mean = np.einsum("ab,b...->a...", A0, pts) + t0.reshape(3, 1, 1, 1)
    U = (np.einsum("ab,b...->a...", A1, pts) + t1.reshape(3, 1, 1, 1))[None]
    w = np.array([0.7])
    y, _ = O.invert(vol, mean, U, w, tol=1e-13, max_iter=300)
    A, t = A0 + w[0] * A1, t0 + w[0] * t1
    expect = np.einsum("ab,b...->a...", np.linalg.inv(np.eye(3) + A), pts - t.reshape(3, 1, 1, 1)) - pts
    inner = (slice(None), slice(3, vol.nz - 3), slice(3, vol.ny - 3), slice(3, vol.nx - 3))
    assert np.max(np.abs(y - expect)[inner]) < 1e-10
    assert np.max(np.abs(expect[inner])) > 1.0  # displacements of a few mm, not a trivial field


def test_inverse_field_along_one_axis_matches_bisection():
    # x = (0, 0, a sin(2 pi z / L)) sampled on the nodes: along z the interpolant is
    # numpy's piecewise-linear interp (which also clamps to the end values), and each
    # voxel's inverse solves the scalar equation d + X(z_u + d) = 0 with X increasing
    # slower than d, found here by bisection.
    vol = Volume(6, 5, 40, 2.0, 2.0, 2.5)
    ax, ay, az = vol.axes()
    a, L = 3.0, 40.0
    xz = a * np.sin(2 * math.pi * az / L)
    mean = np.zeros((3,) + vol.shape)
    mean[2] = xz[:, None, None]
    U = np.zeros((1, 3) + vol.shape)
    y, _ = O.invert(vol, mean, U, np.zeros(1), tol=1e-13, max_iter=300)
    for k, zu in enumerate(az):
        lo, hi = -4 * a, 4 * a
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid + np.interp(zu + mid, az, xz) > 0:
                hi = mid
            else:
                lo = mid
        d = 0.5 * (lo + hi)
        assert np.max(np.abs(y[2, k] - d)) < 1e-10, k
    assert np.max(np.abs(y[0])) < 1e-13 and np.max(np.abs(y[1])) < 1e-13


def test_inverse_field_at_nodes_equals_pointwise_tumor_and_round_trips(small_case):
    c = small_case
    vol, mean, U = c["vol"], c["pca"].mean, c["pca"].U
    w = np.array([1.2, -0.3, 0.1])
    y, sweeps = O.invert(vol, mean, U, w, tol=1e-12, max_iter=200)
    assert sweeps < 200
    ax, ay, az = vol.axes()
    rng = np.random.default_rng(7)
    for _ in range(40):
        i, j, k = int(rng.integers(vol.nx)), int(rng.integers(vol.ny)), int(rng.integers(vol.nz))
        u = np.array([ax[i], ay[j], az[k]])
        p, _ = O.tumor(vol, mean, U, w, u, tol=1e-13, max_iter=200)
        assert np.max(np.abs(y[:, k, j, i] - (p - u))) < 1e-9
        x = O.dvf_at(vol, mean, U, w, u + y[:, k, j, i])
        assert np.max(np.abs(y[:, k, j, i] + x)) < 1e-9
