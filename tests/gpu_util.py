"""Shared helpers of the GPU tests: seeded inputs, oracle targets, error report."""

from __future__ import annotations

import json
import os

import numpy as np

from phantom import Geometry, Volume

# Tolerances (relative L2 unless stated), as stated for the method's results:
# projections and gradients 1e-4, recovered w 1e-3, tumor position 0.1 mm.
TOL_PROJ = 1e-4
TOL_GRAD = 1e-4
TOL_W = 1e-3
TOL_TUMOR_MM = 0.1


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def report(name: str, **values):
    """Print the FP64-reference error of a result and append it to the JSON
    report named by PR_PARITY_REPORT (if set)."""
    line = {"case": name}
    for k, v in values.items():
        line[k] = float(v) if np.ndim(v) == 0 else [float(x) for x in np.ravel(v)]
    print("PARITY", json.dumps(line))
    path = os.environ.get("PR_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(line) + "\n")


def noisy(p: np.ndarray, seed: int, level: float = 0.01) -> np.ndarray:
    """Measured projection: p + level * p * N(0, 1) draws of the given seed."""
    from phantom import standard_normal

    return p + level * p * standard_normal(seed, p.shape)


def random_volume(vol: Volume, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).random(vol.shape)


RAGGED_VOL = Volume(13, 11, 9, 3.0, 3.5, 4.0)
RAGGED_GEOM = Geometry(1000.0, 1500.0, 37, 21, 2.1, 2.7, 1.3)


# ----------------------------------------------------------------------------
# Line-search paths: the CUDA path decides Armijo's test, the step model and the
# stops in FP64 on FP32-computed costs, the oracle on FP64 costs. Where a choice
# is a rounding tie the two may take different branches, and both are correct.
# A GPU choice that differs from the oracle's own is accepted only as a tie:
#   - Armijo: |J_t - (J - c1 mu |g|^2)| <= TIE_J |J| in FP64, TIE_J ten times the
#     largest cost error measured against the oracle at equal w (about 1e-6);
#   - comparisons on |g| (the guard's resolvability test mu |g|^2 > min_decrease J
#     and the gradient stop): within TIE_G relative, the gradient tolerance;
#   - the step exponent: one that the FP64 trial allows once J and J_t carry
#     TIE_J each.
# The oracle then replays the GPU's choices in FP64, and the GPU's result is
# compared with that solve at the usual tolerances.
# ----------------------------------------------------------------------------
TIE_J = 1e-5
TIE_G = 1e-4


def library_opts(**kw):
    """Oracle options with the CUDA library's default line-search rule: the
    quadratic step model with power-of-two steps (step_model 1) and the
    resolvability guard at 1e-6 of J. The oracle's own default is the paper's
    plain Armijo backtracking."""
    from oracle import oracle as O

    kw.setdefault("step_model", 1)
    kw.setdefault("min_decrease", 1e-6)
    return O.SolveOptions(**kw)


def _exp2(f: float) -> int:
    import math

    return math.frexp(f)[1] - 1


def _pow2_floor(x: float) -> float:
    import math

    return math.ldexp(1.0, math.frexp(x)[1] - 1)


def _model_choices(t, opts) -> set:
    if opts.min_decrease <= 0.0:
        return {True}
    pred, thr = t["mu"] * t["gn2"], opts.min_decrease * abs(t["J"])
    if abs(pred - thr) <= TIE_G * max(pred, thr):
        return {True, False}
    return {pred > thr}


def allowed_exponents(t, accepted: bool, opts) -> set:
    """Step exponents consistent with trace entry t within the tie tolerances."""
    mu, gn2, J, Jt = t["mu"], t["gn2"], t["J"], t["J_t"]
    dJ = TIE_J * abs(J)
    out = set()
    for model in _model_choices(t, opts):
        for s in (-2.0 * dJ, 0.0, 2.0 * dJ):
            c = 2.0 * (Jt - J + mu * gn2 + s) / (mu * mu)
            use = model and c > 0
            if accepted:
                f = _pow2_floor(max(min(opts.step_growth, gn2 / c / mu), 0.5)) if use else \
                    _pow2_floor(max(opts.step_growth, 0.5))
            else:
                f = _pow2_floor(min(opts.beta, max(1.0 / 16.0, gn2 / c / mu))) if use else _pow2_floor(opts.beta)
            out.add(_exp2(f))
    return set(range(min(out), max(out) + 1))


def checked_oracle_solve(gpu_log, run_oracle, opts):
    """The oracle solve to compare a GPU solve with, the number of ties the
    GPU broke the other way, and the oracle's own (un-replayed) solve.
    run_oracle(replay) runs the oracle's reconstruct with replay=None (its own
    choices) or the GPU's trial log."""
    ores = run_oracle(None)
    if [tuple(x) for x in ores.log] == list(gpu_log):
        return ores, 0, ores
    rep = run_oracle(list(gpu_log))
    assert [tuple(x) for x in rep.log] == list(gpu_log), "the oracle could not follow the GPU's path"
    ties = 0
    for i, (t, g) in enumerate(zip(rep.trace, gpu_log)):
        own = t["own"]
        if g[0] != own[0]:
            assert abs(t["margin"]) <= TIE_J * abs(t["J"]), ("Armijo choice %d is not a tie" % i, t)
            ties += 1
        if not g[0]:
            # a rejected trial stops exactly when the guard finds its predicted
            # decrease unresolvable (whatever the oracle's own Armijo choice)
            stops = {not m for m in _model_choices(t, opts)}
            assert g[1] in stops, ("resolvability stop %d is not a tie" % i, t)
            if len(stops) == 2 and not own[0] and g[1] != own[1]:
                ties += 1
        if g[0] and g[1] != t.get("own_grad_stop", False):
            gn, thr = t["gn_after"], opts.grad_tol * t["g0"]
            assert abs(gn - thr) <= TIE_G * max(gn, thr), ("gradient stop %d is not a tie" % i, t)
            ties += 1
        if opts.step_model == 1 and not g[1] and (g[0] != own[0] or g[2] != own[2]):
            assert g[2] in allowed_exponents(t, g[0], opts), ("step exponent %d is not a tie" % i, t)
            ties += int(g[0] == own[0])
    return rep, ties, ores


def own_path_errors(res, own) -> dict:
    """Distance of a GPU solve from the oracle's own solve (its own line-search
    choices, not the GPU's): relative J, relative w and tumor distance (mm).
    After a tie broken the other way the two paths part; J, the quantity the
    method minimises, stays within the projection tolerance, while w may move
    along a flat valley of J."""
    return dict(own_J_rel=abs(res["J"] - own.J) / abs(own.J), own_w_rel=rel(res["w"], own.w),
                own_tumor_mm=float(np.max(np.abs(np.asarray(res["tumor"]) - own.tumor))),
                own_iters=own.iters, own_stop=own.stop_reason)
