"""FP64 CPU oracle: the plain reference for the CUDA reconstruction path.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the library. It shares no code with the
CUDA path. The heavy loops (warp, projection, transpose, tumor fixed point)
are plain C in oracle.c, compiled by build_oracle(); the optimiser of
Section 2.2 is written here step by step in the paper's order.

Functions and the passages they follow:
  dvf          Eq. 1 (x = mean + U w)
  warp         Section 2.2, trilinear interpolation of f0 at v + x(v)
  warp_jac     Section 2.2, h_k = (df/dx) . u_k consistent with the interpolation
  project      Eq. 2, the projection matrix P
  backproject  gradient formula after Eq. 4, P^T
  cost         Eq. 2, J = ||P f - a y - b 1||^2
  fit_ab       Eq. 4, (a, b) = (Y^T Y)^-1 Y^T P f, Y = [y, 1]
  gradient     gradient formula after Eq. 4: 2 U^T (df/dx) P^T (P f - a y - b 1)
  reconstruct  Section 2.2: alternate Eq. 3 (Armijo step on w) and Eq. 4
  tumor        Section 2.3 with the fixed-point inversion of ref. 13
  invert       Section 2.3 with ref. 13: the push-forward field on the whole grid

Readings of the paper where it is silent (the CUDA path uses the same):
  * Armijo rule (Section 2.2 names it, gives no constants): sufficient
    decrease J(w - mu g; a, b) <= J(w; a, b) - c1 mu |g|^2 with c1 = 1e-4, at
    most 8 backtracks. The first trial step is mu = step0_mm / |g| (moves w by
    step0_mm). A solve warm-started from the previous frame starts with that
    frame's next trial step, as its w starts from that frame's w (Section 4
    initialises each frame from the previous one). No accepted step: w is
    kept, the solve stops with stop reason "line search failed" and the next
    trial step is forgotten.
  * Trial steps, SolveOptions.step_model (one trial's decision is the pure
    function step_choice):
      0 (the default: plain backtracking, the textbook form of Armijo's rule)
        a rejected trial backtracks mu <- beta mu (beta = 0.5); after an
        accepted step the next first trial is step_growth x mu (2) if mu was
        accepted at its first trial, else step_growth_bt x mu (1).
      1 (the CUDA library's default rule) each trial at mu also measures the
        curvature of J along -g, curv = 2 (J(mu) - J + mu |g|^2) / mu^2, whose
        quadratic model J - mu |g|^2 + curv mu^2 / 2 has its minimum at
        |g|^2 / curv; steps are that minimiser rounded down to a power of two
        times mu: a rejected trial backtracks to mu x pow2_floor(clamp(
        minimiser / mu, 1/16, beta)), and after an accepted step the next first
        trial is mu x pow2_floor(clamp(minimiser / mu, 1/2, step_growth)).
        Without a positive curvature the plain factors beta and step_growth
        apply.
  * Resolvability guard, SolveOptions.min_decrease (0 = off, the default;
    the CUDA library runs step_model 1 with 1e-6, the relative resolution of
    its FP32 cost at paper scale): the quadratic model is trusted only where
    the trial's predicted decrease mu |g|^2 exceeds min_decrease |J|, and a
    rejected trial below that threshold stops the solve ("resolved": no step
    along -g can then lower J by an amount the cost resolves).
  * (a, b) before the first step 1: Eq. 4 at the starting w.
  * Stop (Section 2.2: gradient "sufficiently small" or the iteration cap):
    |g| <= grad_tol * |g_0|, or max_iters accepted steps, or (with the guard
    on) the resolved stop above.
"""

from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

STOP_GRAD_TOL = 1
STOP_MAX_ITERS = 2
STOP_LINESEARCH_FAILED = 3
STOP_RESOLVED = 7


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build_oracle(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain -O2, single thread), or with
    openmp into liboracle_omp.so (the same source on all host cores; used only
    to time the method, see oracle.c)."""
    lib = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + ".tmp.%d" % os.getpid()
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared"] + flags + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


class _Vol(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class _Geom(ctypes.Structure):
    _fields_ = [("sad", ctypes.c_double), ("sdd", ctypes.c_double), ("nu", ctypes.c_int),
                ("nv", ctypes.c_int), ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("ds", ctypes.c_double)]


_lib = None
_openmp = False


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle(openmp=_openmp))
    return _lib


def use_openmp(flag: bool) -> int:
    """Route the oracle's loops through the OpenMP build (all host cores) or
    the plain one; returns the threads the loops will use."""
    global _lib, _openmp
    if flag != _openmp or _lib is None:
        _openmp = flag
        _lib = ctypes.CDLL(build_oracle(openmp=flag))
    return int(_lib.or_threads())


def _vol(v) -> _Vol:
    return _Vol(v.nx, v.ny, v.nz, v.dx, v.dy, v.dz)


def _geom(g) -> _Geom:
    return _Geom(g.sad, g.sdd, g.nu, g.nv, g.du, g.dv, g.ds)


def _d(a):
    """C-contiguous float64 copy/view and its pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------
# Operators
# ----------------------------------------------------------------------------


def dvf(vol, mean, U, w):
    """Eq. 1: x = mean + sum_k u_k w_k, [3][nz][ny][nx]."""
    mean, pm = _d(mean)
    U, pu = _d(U)
    w, pw = _d(np.atleast_1d(w))
    out = np.empty(mean.shape, dtype=np.float64)
    _L().or_dvf(ctypes.byref(_vol(vol)), pm, pu, ctypes.c_int(U.shape[0]), pw,
                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def warp(vol, f0, x):
    """Section 2.2: f(v) = F0(v + x(v)) (trilinear, zero outside the grid)."""
    f0, pf = _d(f0)
    x, px = _d(x)
    out = np.empty(f0.shape, dtype=np.float64)
    _L().or_warp(ctypes.byref(_vol(vol)), pf, px, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def warp_jac(vol, f0, x, U):
    """h_k(v) = (df/dx)(v) . u_k(v), [K][nz][ny][nx]."""
    f0, pf = _d(f0)
    x, px = _d(x)
    U, pu = _d(U)
    K = U.shape[0]
    out = np.empty((K,) + f0.shape, dtype=np.float64)
    _L().or_warp_jac(ctypes.byref(_vol(vol)), pf, px, pu, ctypes.c_int(K),
                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def project(vol, geom, angle, f):
    """Eq. 2: P f at gantry angle `angle` (rad), [nv][nu]."""
    f, pf = _d(f)
    out = np.empty((geom.nv, geom.nu), dtype=np.float64)
    _L().or_project(ctypes.byref(_vol(vol)), ctypes.byref(_geom(geom)), ctypes.c_double(angle), pf,
                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def backproject(vol, geom, angle, r):
    """P^T r, [nz][ny][nx]."""
    r, pr = _d(r)
    out = np.empty(vol.shape, dtype=np.float64)
    _L().or_backproject(ctypes.byref(_vol(vol)), ctypes.byref(_geom(geom)), ctypes.c_double(angle),
                        pr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def ray(geom, angle, iu, iv):
    """Source and unit direction of the ray to pixel (iu, iv)."""
    src = np.empty(3)
    d = np.empty(3)
    _L().or_ray(ctypes.byref(_geom(geom)), ctypes.c_double(angle), ctypes.c_int(iu), ctypes.c_int(iv),
                src.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return src, d


def tumor(vol, mean, U, w, c0, tol=1e-6, max_iter=100):
    """Section 2.3 / ref. 13: p with p + x(p) = c0 by p <- c0 - x(p). Returns (p, steps)."""
    mean, pm = _d(mean)
    U, pu = _d(U)
    w, pw = _d(np.atleast_1d(w))
    c0, pc = _d(c0)
    p = np.empty(3)
    it = _L().or_tumor(ctypes.byref(_vol(vol)), pm, pu, ctypes.c_int(U.shape[0]), pw, pc,
                       ctypes.c_double(tol), ctypes.c_int(max_iter),
                       p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return p, int(it)


def invert(vol, mean, U, w, tol=1e-9, max_iter=200):
    """Section 2.3 with ref. 13 over the whole grid: the push-forward DVF y
    [3][nz][ny][nx] (mm) with u + y(u) + x(u + y(u)) = u at every voxel centre,
    by Chen et al.'s whole-field fixed-point sweeps y <- -x(u + y) from y = 0
    (x trilinear, clamped to the grid edge). Returns (y, sweeps)."""
    mean, pm = _d(mean)
    U, pU = _d(U)
    w = np.ascontiguousarray(w, dtype=np.float64)
    y = np.empty((3,) + tuple(vol.shape), dtype=np.float64)
    sweeps = _L().or_invert(ctypes.byref(_vol(vol)), pm, pU, ctypes.c_int(len(w)),
                            w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_double(tol),
                            ctypes.c_int(max_iter), y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return y, int(sweeps)


def dvf_at(vol, mean, U, w, point):
    """x = mean + U w interpolated (clamp-to-edge) at a world point (mm)."""
    mean, pm = _d(mean)
    U, pu = _d(U)
    w, pw = _d(np.atleast_1d(w))
    point, pp = _d(point)
    out = np.empty(3)
    _L().or_dvf_at(ctypes.byref(_vol(vol)), pm, pu, ctypes.c_int(U.shape[0]), pw, pp,
                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


# ----------------------------------------------------------------------------
# Cost, intensity fit, gradient (Eqs. 2-4)
# ----------------------------------------------------------------------------


def cost(p, y, a, b):
    """Eq. 2: J = || p - a y - b 1 ||_2^2."""
    r = np.asarray(p, dtype=np.float64) - a * np.asarray(y, dtype=np.float64) - b
    return float(np.sum(r * r))


def fit_ab(p, y):
    """Eq. 4: (a, b)^T = (Y^T Y)^-1 Y^T p with Y = [y, 1]."""
    yv = np.asarray(y, dtype=np.float64).ravel()
    Y = np.stack([yv, np.ones_like(yv)], axis=1)
    a, b = np.linalg.solve(Y.T @ Y, Y.T @ np.asarray(p, dtype=np.float64).ravel())
    return float(a), float(b)


@dataclasses.dataclass
class Model:
    """A patient's PCA motion model as the solver sees it (all float64)."""

    vol: object
    f0: np.ndarray
    mean: np.ndarray
    U: np.ndarray
    c0: np.ndarray

    @property
    def K(self):
        return self.U.shape[0]


@dataclasses.dataclass
class Evaluation:
    w: np.ndarray
    f: np.ndarray
    p: np.ndarray


def evaluate(model, geom, angle, w):
    """x = mean + U w, f = warped f0, p = P f."""
    x = dvf(model.vol, model.mean, model.U, w)
    f = warp(model.vol, model.f0, x)
    p = project(model.vol, geom, angle, f)
    return Evaluation(np.array(w, dtype=np.float64), f, p)


def gradient(model, geom, angle, w, a, b, y):
    """dJ/dw = 2 U^T (df/dx) P^T (P f - a y - b 1), as the sum over voxels of
    2 (P^T r)(v) h_k(v). Returns (g, J, p)."""
    x = dvf(model.vol, model.mean, model.U, w)
    f = warp(model.vol, model.f0, x)
    h = warp_jac(model.vol, model.f0, x, model.U)
    p = project(model.vol, geom, angle, f)
    r = p - a * np.asarray(y, dtype=np.float64) - b
    bp = backproject(model.vol, geom, angle, r)
    g = np.array([2.0 * np.sum(bp * h[k]) for k in range(model.K)])
    return g, float(np.sum(r * r)), p


def pow2_floor(x: float) -> float:
    """The largest power of two not above x (x > 0)."""
    m, e = math.frexp(x)  # x = m 2^e, 0.5 <= m < 1
    return math.ldexp(1.0, e - 1)


@dataclasses.dataclass
class SolveOptions:
    """Section 2.2's solver constants. The defaults are the paper's rule:
    Armijo backtracking by beta, stop on a small gradient or the cap."""

    max_iters: int = 10
    grad_tol: float = 1e-6
    c1: float = 1e-4
    beta: float = 0.5
    max_backtracks: int = 8
    step0_mm: float = 1.0
    step_growth: float = 2.0
    step_growth_bt: float = 1.0
    step_model: int = 0        # 0: plain factors; 1: quadratic model, power-of-two steps
    min_decrease: float = 0.0  # resolvability guard (0 = off), see the module docstring
    tumor_tol: float = 1e-6
    tumor_max_iter: int = 100


def step_choice(J: float, J_t: float, mu: float, gn2: float, bt: int, o: SolveOptions):
    """One line-search trial's decisions (Section 2.2, Armijo's rule) from the
    cost J at w, the cost J_t at the trial w - mu g (same a, b), the step mu,
    |g|^2 and the backtracks bt already taken in this step.

    Returns (accepted, stop, factor): accepted is Armijo's sufficient-decrease
    test; stop is the guard's resolved stop (rejected trials only); factor
    scales mu for the next trial (the backtrack after a rejection, the next
    step's first trial after an acceptance)."""
    ok = J_t <= J - o.c1 * mu * gn2
    resolvable = o.min_decrease <= 0.0 or mu * gn2 > o.min_decrease * abs(J)
    # curvature of J along -g from this trial: J(mu) = J - mu |g|^2 + (curv/2) mu^2
    curv = 2.0 * (J_t - J + mu * gn2) / (mu * mu)
    use_model = o.step_model == 1 and resolvable and curv > 0.0 and math.isfinite(curv)
    if ok:
        if o.step_model == 1:
            ratio = min(o.step_growth, gn2 / curv / mu) if use_model else o.step_growth
            return True, False, pow2_floor(max(ratio, 0.5))
        return True, False, (o.step_growth if bt == 0 else o.step_growth_bt)
    if not resolvable:
        return False, True, 1.0
    if o.step_model == 1:
        ratio = min(o.beta, max(1.0 / 16.0, gn2 / curv / mu)) if use_model else o.beta
        return False, False, pow2_floor(ratio)
    return False, False, o.beta


@dataclasses.dataclass
class SolveResult:
    w: np.ndarray
    a: float
    b: float
    J: float
    grad: np.ndarray
    iters: int
    backtracks: int
    stop_reason: int
    tumor: np.ndarray
    tumor_steps: int
    mu: float  # first trial step of the next warm-started frame (0 = none)
    history: list  # per accepted step: dict(J_after_step1, J_after_step2, mu, w)
    log: list = dataclasses.field(default_factory=list)    # per trial: (accepted, stop, e), see reconstruct
    trace: list = dataclasses.field(default_factory=list)  # per trial: the FP64 quantities behind each choice


def reconstruct(model, geom, angle, y, w0, opts: SolveOptions | None = None,
                mu_next: float | None = None, replay: list | None = None) -> SolveResult:
    """Section 2.2: alternate step 1 (Eq. 3, gradient step with Armijo's rule at
    fixed a, b) and step 2 (Eq. 4, exact a, b at fixed w), then Section 2.3.
    mu_next: the previous frame's next trial step (None or 0 = cold).

    Every line-search trial makes three floating-point choices, logged as
    (accepted, stop, e): the Armijo test; a stop (a rejected trial whose
    predicted decrease is unresolvable, or an accepted step after which the
    gradient test is met); and e, the power-of-two exponent of the factor that
    scales mu next (the backtrack after a rejection, the next first trial after
    an acceptance; 0 with step_model 0, whose factors are fixed). With
    `replay` (such a log, e.g. the CUDA path's), trial i takes the logged
    choices instead of its own; `trace` keeps, per trial, the FP64 quantities
    from which its own choices follow, so a test can tell a tie from an error."""
    o = opts or SolveOptions()
    y = np.asarray(y, dtype=np.float64)
    w = np.array(w0, dtype=np.float64)
    # (a, b) at the starting w by Eq. 4.
    a, b = fit_ab(evaluate(model, geom, angle, w).p, y)
    g, J, _ = gradient(model, geom, angle, w, a, b, y)
    g0 = float(np.linalg.norm(g))
    n = 0
    backtracks = 0
    stop = STOP_MAX_ITERS
    history = []
    log, trace = [], []
    grad_stop = False
    while True:
        gn = float(np.linalg.norm(g))
        if grad_stop or (not log and (gn <= o.grad_tol * g0 or gn == 0.0)):
            stop = STOP_GRAD_TOL
            break
        if n >= o.max_iters:
            stop = STOP_MAX_ITERS
            break
        # Step 1: w <- w - mu g, mu by backtracking from the initial trial.
        mu = mu_next if mu_next else o.step0_mm / gn
        accepted = None
        resolved = False
        for bt in range(o.max_backtracks + 1):
            trial = evaluate(model, geom, angle, w - mu * g)
            J_t = cost(trial.p, y, a, b)
            # this trial's own choices (see the docstring)
            ok, stop_t, factor = step_choice(J, J_t, mu, gn * gn, bt, o)
            own = (ok, stop_t, _exp2(factor) if (o.step_model == 1 and not stop_t) else 0)
            trace.append(dict(J=J, J_t=J_t, mu=mu, gn2=gn * gn, curv=2.0 * (J_t - J + mu * gn * gn) / (mu * mu),
                              bt=bt, own=own, margin=J_t - (J - o.c1 * mu * gn * gn)))
            choice = own
            if replay is not None and len(log) < len(replay):
                choice = tuple(replay[len(log)])
                if choice[0] != own[0] or choice[2] != own[2]:
                    if o.step_model == 1:
                        factor = 2.0 ** choice[2]
                    elif choice[0]:
                        factor = o.step_growth if bt == 0 else o.step_growth_bt
                    else:
                        factor = o.beta
            log.append(choice)
            if choice[0]:
                accepted = trial
                break
            backtracks += 1
            if choice[1]:
                resolved = True  # no step along -g changes J by a resolvable amount
                break
            mu *= factor
        if resolved:
            stop = STOP_RESOLVED
            mu_next = mu
            break
        if accepted is None:
            stop = STOP_LINESEARCH_FAILED
            mu_next = 0.0
            break
        mu_next = mu * factor
        w = accepted.w
        # Step 2: (a, b) by Eq. 4 at the new w.
        a, b = fit_ab(accepted.p, y)
        g, J, _ = gradient(model, geom, angle, w, a, b, y)
        history.append(dict(J_step1=J_t, J_step2=J, mu=mu, w=w.copy()))
        n += 1
        # the gradient test after this step is the accepted trial's stop choice
        gn_new = float(np.linalg.norm(g))
        own_stop = gn_new <= o.grad_tol * g0 or gn_new == 0.0
        trace[-1]["gn_after"] = gn_new
        trace[-1]["g0"] = g0
        trace[-1]["own_grad_stop"] = own_stop
        if replay is not None and len(log) <= len(replay):
            grad_stop = bool(log[-1][1])
        else:
            grad_stop = own_stop
            log[-1] = (True, own_stop, log[-1][2])
    p_t, steps = tumor(model.vol, model.mean, model.U, w, model.c0, o.tumor_tol, o.tumor_max_iter)
    return SolveResult(w=w, a=a, b=b, J=J, grad=g, iters=n, backtracks=backtracks, stop_reason=stop,
                       tumor=p_t, tumor_steps=steps, mu=mu_next or 0.0, history=history, log=log, trace=trace)


def _exp2(factor: float) -> int:
    """Exponent e of a power of two factor = 2^e."""
    m, e = math.frexp(factor)
    return e - 1
