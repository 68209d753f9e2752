"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle
on identical seeded inputs (float32 inputs, upcast exactly for the oracle)."""

import math

import numpy as np
import pytest

from gpu_util import (RAGGED_GEOM, RAGGED_VOL, TOL_GRAD, TOL_PROJ, TOL_TUMOR_MM, TOL_W, checked_oracle_solve, library_opts,
                      own_path_errors,
                      noisy, random_volume, rel, report)
from oracle import oracle as O
from phantom import Geometry, Volume

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_1004_0014_b300 import Context

    assert torch.cuda.is_available()
    c = Context(0)
    yield c
    c.close()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _up(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def small(ctx, small_case):
    c = small_case
    f0, mean, U = _f32(c["f0"]), _f32(c["pca"].mean), _f32(c["pca"].U)
    mid = ctx.load_model(c["vol"], c["geom"], f0, mean, U, c["c0"])
    om = O.Model(c["vol"], _up(f0), _up(mean), _up(U), c["c0"])
    # Measured projection: oracle warp by the 1.5x analytic field, oracle
    # projection, 1% noise (seed 0); float32 as the GPU receives it.
    ft = O.warp(c["vol"], om.f0, c["x_test"])
    y = _f32(noisy(O.project(c["vol"], c["geom"], c["angle"], ft), c["seed"]))
    return dict(c, mid=mid, om=om, y=y)


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


# ----------------------------------------------------------------------------
# a1: DVF synthesis + warp (+ h_k)
# ----------------------------------------------------------------------------


def _warp_check(ctx, mid, om, vol, w, name):
    f, h = ctx.warp(mid, w)
    f, h = f.cpu().numpy(), h.cpu().numpy()
    x = O.dvf(vol, om.mean, om.U, w)
    fo = O.warp(vol, om.f0, x)
    ho = O.warp_jac(vol, om.f0, x, om.U)
    # h_k jumps across trilinear cell faces (the derivative is one-sided
    # there), so a point within rounding of a face may take either cell in
    # float32. Compare where the cell is unambiguous: clear of every face, or
    # exactly on one with a zero displacement component (both paths then
    # compute the same integer).
    q = np.stack([x[c] / vol.spacing[c] for c in range(3)])
    frac = q - np.floor(q)
    ambiguous = (frac > 0) & ((frac < 1e-4) | (frac > 1 - 1e-4))
    clear = ~np.any(ambiguous, axis=0)
    assert clear.mean() > 0.99
    ef = rel(f, fo)
    eh = max(rel(h[k][clear], ho[k][clear]) for k in range(om.K))
    report(name, f_rel=ef, h_rel=eh, clear_frac=clear.mean())
    assert ef < 1e-5
    assert eh < 1e-5


def test_warp_matches_oracle(ctx, small):
    for w in (np.zeros(3), np.array([0.7, -0.4, 0.2]), np.array([-1.3, 0.5, 0.9])):
        _warp_check(ctx, small["mid"], small["om"], small["vol"], w, "warp64")


def test_warp_ragged_grid_matches_oracle(ctx):
    vol = RAGGED_VOL  # N = 1287: odd (the two-voxel vector loads fall back), rows not aligned
    rng = np.random.default_rng(7)
    f0 = _f32(rng.random(vol.shape))
    mean = _f32(2.0 * rng.standard_normal((3,) + vol.shape))
    U = _f32(rng.standard_normal((2, 3) + vol.shape))
    mid = ctx.load_model(vol, RAGGED_GEOM, f0, mean, U, np.zeros(3))
    om = O.Model(vol, _up(f0), _up(mean), _up(U), np.zeros(3))
    _warp_check(ctx, mid, om, vol, np.array([0.3, -0.8]), "warp_ragged")
    ctx.release_model(mid)


# ----------------------------------------------------------------------------
# a2: projector
# ----------------------------------------------------------------------------


def test_project_matches_oracle(ctx, small):
    vol, geom = small["vol"], small["geom"]
    f = _f32(O.warp(vol, small["om"].f0, O.dvf(vol, small["om"].mean, small["om"].U, [0.5, 0.2, -0.1])))
    fd = _cuda(f)
    for th in (0.0, 0.7, 2.5, 4.0, math.pi / 2):
        p = ctx.project(vol, geom, th, fd).cpu().numpy()
        po = O.project(vol, geom, th, _up(f))
        e = rel(p, po)
        report("project64", angle=th, rel=e)
        assert e < TOL_PROJ


def test_project_ragged_matches_oracle(ctx):
    vol, geom = RAGGED_VOL, RAGGED_GEOM
    f = _f32(random_volume(vol, 3))
    for th in (0.3, 1.9, 3.3):
        p = ctx.project(vol, geom, th, _cuda(f)).cpu().numpy()
        e = rel(p, O.project(vol, geom, th, _up(f)))
        report("project_ragged", angle=th, rel=e)
        assert e < TOL_PROJ


# ----------------------------------------------------------------------------
# a4: gather transpose
# ----------------------------------------------------------------------------


def test_backproject_is_transpose_and_matches_oracle(ctx, small):
    for vol, geom, th in ((RAGGED_VOL, RAGGED_GEOM, 0.4), (small["vol"], small["geom"], 2.2)):
        rng = np.random.default_rng(11)
        x = _f32(rng.standard_normal(vol.shape))
        r = _f32(rng.standard_normal((geom.nv, geom.nu)))
        px = ctx.project(vol, geom, th, _cuda(x)).cpu().numpy().astype(np.float64)
        g = ctx.backproject(vol, geom, th, _cuda(r)).cpu().numpy().astype(np.float64)
        lhs, rhs = float(np.sum(px * r)), float(np.sum(_up(x) * g))
        e_adj = abs(lhs - rhs) / abs(lhs)
        e = rel(g, O.backproject(vol, geom, th, _up(r)))
        report("backproject", n=vol.n, adjoint_rel=e_adj, rel=e)
        assert e_adj < 1e-5
        assert e < TOL_GRAD


# ----------------------------------------------------------------------------
# a2-a4: cost and gradient at the same (w, a, b)
# ----------------------------------------------------------------------------


def test_cost_and_gradient_match_oracle(ctx, small):
    yd = _cuda(small["y"])
    y = _up(small["y"])
    for w, a, b in ((np.zeros(3), 1.0, 0.0), (np.array([0.4, -0.3, 0.2]), 1.02, -0.01),
                    (np.array([-1.1, 0.6, 0.3]), 0.97, 0.02)):
        go, Jo, _ = O.gradient(small["om"], small["geom"], small["angle"], w, a, b, y)
        for mode in (0, 1):
            J, g = ctx.cost_grad(small["mid"], yd, small["angle"], w, a, b, mode)
            eJ, eg = abs(J - Jo) / Jo, rel(g, go)
            report("cost_grad64", mode=mode, J_rel=eJ, g_rel=eg)
            assert eJ < TOL_PROJ
            assert eg < TOL_GRAD


@pytest.mark.parametrize("deg", [0.0, 10.0, 14.0, 16.0, 45.0, 80.0, 100.0, 200.0])
def test_solver_projector_matches_oracle_for_both_warp_tiles(ctx, small, deg):
    """The solver-pass projector (P f, P h_k and the fused moments) takes 4 x 8
    detector pixels per warp within 15 degrees of a volume axis and 2 x 16
    elsewhere: P f, J and the forward-mode gradient against the oracle on both
    sides of the switch and around the rotation."""
    vol, geom, om = small["vol"], small["geom"], small["om"]
    th = math.radians(deg)
    ft = O.warp(vol, om.f0, small["x_test"])
    y = _f32(noisy(O.project(vol, geom, th, ft), small["seed"]))
    w, a, b = np.array([0.4, -0.3, 0.2]), 1.02, -0.01
    J, g, p = ctx.cost_grad(small["mid"], _cuda(y), th, w, a, b, 0, return_p=True)
    po = O.project(vol, geom, th, O.warp(vol, om.f0, O.dvf(vol, om.mean, om.U, w)))
    go, Jo, _ = O.gradient(om, geom, th, w, a, b, _up(y))
    ep, eJ, eg = rel(p.cpu().numpy(), po), abs(J - Jo) / Jo, rel(g, go)
    report("solver_projector_tiles", deg=deg, p_rel=ep, J_rel=eJ, g_rel=eg)
    assert ep < TOL_PROJ
    assert eJ < TOL_PROJ
    assert eg < TOL_GRAD


@pytest.mark.parametrize("th", [0.1, 0.8])
def test_solver_projector_ragged_matches_oracle(ctx, th):
    """The solver projector on a ragged grid and a 37 x 21 detector (partial
    warp tiles along both detector axes), with 4 x 8 (0.1 rad) and 2 x 16
    (0.8 rad) warp tiles: P f, J and the forward-mode gradient against the
    oracle."""
    vol, geom = RAGGED_VOL, RAGGED_GEOM
    rng = np.random.default_rng(11)
    f0 = _f32(rng.random(vol.shape))
    mean = _f32(2.0 * rng.standard_normal((3,) + vol.shape))
    U = _f32(rng.standard_normal((2, 3) + vol.shape))
    mid = ctx.load_model(vol, geom, f0, mean, U, np.zeros(3))
    om = O.Model(vol, _up(f0), _up(mean), _up(U), np.zeros(3))
    try:
        w, a, b = np.array([0.3, -0.8]), 0.9, 0.05
        f = O.warp(vol, om.f0, O.dvf(vol, om.mean, om.U, w))
        po = O.project(vol, geom, th, f)
        y = _f32(noisy(po, 5))
        J, g, p = ctx.cost_grad(mid, _cuda(y), th, w, a, b, 0, return_p=True)
        go, Jo, _ = O.gradient(om, geom, th, w, a, b, _up(y))
        ep, eJ, eg = rel(p.cpu().numpy(), po), abs(J - Jo) / Jo, rel(g, go)
        report("solver_projector_ragged", angle=th, p_rel=ep, J_rel=eJ, g_rel=eg)
        assert ep < TOL_PROJ
        assert eJ < TOL_PROJ
        assert eg < TOL_GRAD
    finally:
        ctx.release_model(mid)


def test_forward_and_vjp_match_oracle(ctx, small):
    import torch

    vol, geom, th = small["vol"], small["geom"], 0.9
    w = np.array([0.6, 0.1, -0.2])
    p = ctx.forward(small["mid"], w, th).cpu().numpy()
    po = O.evaluate(small["om"], geom, th, w).p
    ep = rel(p, po)
    gp = np.random.default_rng(5).standard_normal((geom.nv, geom.nu))
    v = ctx.vjp(small["mid"], w, th, torch.from_numpy(_f32(gp)).cuda())
    x = O.dvf(vol, small["om"].mean, small["om"].U, w)
    h = O.warp_jac(vol, small["om"].f0, x, small["om"].U)
    bp = O.backproject(vol, geom, th, _up(_f32(gp)))
    vo = np.array([np.sum(bp * h[k]) for k in range(3)])
    ev = rel(v, vo)
    report("forward_vjp64", p_rel=ep, vjp_rel=ev)
    assert ep < TOL_PROJ
    assert ev < TOL_GRAD


# ----------------------------------------------------------------------------
# a7: tumor
# ----------------------------------------------------------------------------


def test_tumor_matches_oracle(ctx, small):
    om = small["om"]
    for w in (np.zeros(3), np.array([1.5, -0.5, 0.3]), np.array([-2.0, 0.8, -0.4])):
        xyz, steps = ctx.tumor(small["mid"], w)
        xo, so = O.tumor(small["vol"], om.mean, om.U, w, om.c0)
        d = float(np.max(np.abs(xyz - xo)))
        report("tumor64", max_abs_mm=d, steps=steps)
        assert d < 1e-6
        assert steps == so


# ----------------------------------------------------------------------------
# a1-a8: the whole alternation
# ----------------------------------------------------------------------------


def _opts(**kw):
    from paper_1004_0014_b300 import default_opts

    return default_opts(**kw)


def test_reconstruct_matches_oracle(ctx, small):
    om, geom, th = small["om"], small["geom"], small["angle"]
    it = small["max_iters"]
    res = ctx.reconstruct(small["mid"], small["y"], th, _opts(max_iters=it, cold_start=1, w0=[0, 0, 0]))
    so = library_opts(max_iters=it)
    ores, ties, own = checked_oracle_solve(
        ctx.trial_log(small["mid"]),
        lambda rp: O.reconstruct(om, geom, th, _up(small["y"]), np.zeros(3), so, replay=rp), so)
    eJ = abs(res["J"] - ores.J) / ores.J
    ew = rel(res["w"], ores.w)
    et = float(np.max(np.abs(res["tumor"] - ores.tumor)))
    eo = own_path_errors(res, own)
    report("reconstruct64", iters=res["iters"], J_rel=eJ, w_rel=ew, tumor_mm=et,
           a_rel=abs(res["a"] - ores.a) / abs(ores.a), trials=res["trials"], backtracks=res["backtracks"],
           oracle_backtracks=ores.backtracks, ties=ties, **eo)
    assert res["iters"] == ores.iters == it
    assert res["stop_reason"] == ores.stop_reason
    assert eJ < TOL_PROJ
    assert ew < TOL_W
    assert et < TOL_TUMOR_MM
    assert eo["own_J_rel"] < TOL_PROJ
    # The FP32 solve at its own final w agrees with the oracle's cost and
    # gradient there. The final gradient is a small difference of large sums,
    # so its error is measured against the scale the per-step gradient
    # tolerance is stated on: the gradient at the start of the solve.
    go, Jo, _ = O.gradient(om, geom, th, res["w"], res["a"], res["b"], _up(small["y"]))
    assert abs(res["J"] - Jo) / Jo < TOL_PROJ
    g_start = np.sqrt(ores.trace[0]["gn2"])
    assert np.linalg.norm(res["grad"] - go) / g_start < TOL_GRAD


def test_reconstruct_plain_armijo_matches_oracle_default(ctx, small):
    """The paper's rule as the oracle runs it by default (backtracking by beta,
    no step model, no resolvability guard): the CUDA path's step_model 0 over
    a solve that is still far from the FP32 resolution of J."""
    om, geom, th = small["om"], small["geom"], small["angle"]
    it = 6
    res = ctx.reconstruct(small["mid"], small["y"], th, _opts(max_iters=it, cold_start=1, w0=[0, 0, 0],
                                                              step_model=0))
    so = O.SolveOptions(max_iters=it)
    ores, ties, own = checked_oracle_solve(
        ctx.trial_log(small["mid"]),
        lambda rp: O.reconstruct(om, geom, th, _up(small["y"]), np.zeros(3), so, replay=rp), so)
    eo = own_path_errors(res, own)
    report("reconstruct64_plain_armijo", iters=res["iters"], J_rel=abs(res["J"] - ores.J) / ores.J,
           w_rel=rel(res["w"], ores.w), backtracks=res["backtracks"], oracle_backtracks=ores.backtracks, ties=ties,
           **eo)
    assert res["iters"] == ores.iters
    assert res["backtracks"] == ores.backtracks
    assert abs(res["J"] - ores.J) / ores.J < TOL_PROJ
    assert rel(res["w"], ores.w) < TOL_W
    assert eo["own_J_rel"] < TOL_PROJ


def test_host_loop_equals_device_loop_bitwise(ctx, small):
    from paper_1004_0014_b300 import PR_LOOP_HOST

    kw = dict(max_iters=8, cold_start=1, w0=[0.2, 0.0, 0.0])
    a = ctx.reconstruct(small["mid"], small["y"], small["angle"], _opts(**kw))
    b = ctx.reconstruct(small["mid"], small["y"], small["angle"], _opts(loop_mode=PR_LOOP_HOST, **kw))
    c = ctx.reconstruct(small["mid"], small["y"], small["angle"], _opts(**kw))
    for k in ("w", "a", "b", "J", "tumor"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k
    assert a["iters"] == b["iters"] and a["trials"] == b["trials"]


def test_warm_start_carries_w(ctx, small):
    w_set = np.array([0.3, -0.2, 0.05])
    ctx.set_state(small["mid"], w_set)
    assert np.array_equal(ctx.get_state(small["mid"]), w_set)
    res = ctx.reconstruct(small["mid"], small["y"], small["angle"], _opts(max_iters=0))
    assert np.array_equal(res["w"], w_set)
    assert res["iters"] == 0
    res2 = ctx.reconstruct(small["mid"], small["y"], small["angle"], _opts(max_iters=3))
    # a warm-started solve starts from the state and leaves its answer there
    assert np.array_equal(ctx.get_state(small["mid"]), res2["w"])
    so = library_opts(max_iters=3)
    ores, _, _ = checked_oracle_solve(
        ctx.trial_log(small["mid"]),
        lambda rp: O.reconstruct(small["om"], small["geom"], small["angle"], _up(small["y"]), w_set, so,
                                 replay=rp), so)
    assert rel(res2["w"], ores.w) < TOL_W


def test_volume_output_matches_warp(ctx, small):
    res = ctx.reconstruct(small["mid"], small["y"], small["angle"],
                          _opts(max_iters=2, cold_start=1, w0=[0.1, 0, 0]), volume=True)
    f, _ = ctx.warp(small["mid"], res["w"], with_h=False)
    assert np.array_equal(res["volume"], f.cpu().numpy())


def test_nonfinite_and_singular_inputs_stop_cleanly(ctx, small):
    from paper_1004_0014_b300 import PR_STOP_NONFINITE, PR_STOP_SINGULAR_FIT

    y = small["y"].copy()
    y[3, 4] = np.nan
    w0 = [0.25, 0.0, 0.0]
    res = ctx.reconstruct(small["mid"], y, 0.0, _opts(cold_start=1, w0=w0))
    assert res["stop_reason"] == PR_STOP_NONFINITE
    assert np.array_equal(res["w"], np.array(w0))
    res = ctx.reconstruct(small["mid"], np.full_like(small["y"], 2.0), 0.0, _opts(cold_start=1, w0=w0))
    assert res["stop_reason"] == PR_STOP_SINGULAR_FIT
    assert np.array_equal(res["w"], np.array(w0))
    # the context stays usable
    res = ctx.reconstruct(small["mid"], small["y"], small["angle"], _opts(max_iters=1, cold_start=1, w0=w0))
    assert res["iters"] == 1


def test_invalid_arguments_are_rejected(ctx, small):
    from paper_1004_0014_b300 import Context, PcaReconError

    with pytest.raises(PcaReconError) as e:
        ctx.reconstruct(12345, small["y"], 0.0)
    assert e.value.code == -6
    with pytest.raises(PcaReconError) as e:
        ctx.reconstruct(small["mid"], small["y"], float("nan"))
    assert e.value.code == -1
    with pytest.raises(PcaReconError) as e:
        ctx.reconstruct(small["mid"], small["y"], 0.0, _opts(beta=1.5))
    assert e.value.code == -1
    vol = Volume(8, 8, 8, 1.0, 1.0, 1.0)
    z = np.zeros((1, 3) + vol.shape, np.float32)
    with pytest.raises(PcaReconError) as e:
        ctx.load_model(vol, Geometry(1000, 1500, 8, 8, 1, 1, 0), np.zeros(vol.shape, np.float32),
                       np.zeros((3,) + vol.shape, np.float32), np.zeros((9, 3) + vol.shape, np.float32),
                       np.zeros(3))
    assert e.value.code == -1  # K > 7
    small_ctx = Context(0, hbm_budget_bytes=1 << 16)
    with pytest.raises(PcaReconError) as e:
        small_ctx.load_model(vol, Geometry(1000, 1500, 8, 8, 1, 1, 0), np.zeros(vol.shape, np.float32),
                             np.zeros((3,) + vol.shape, np.float32), z, np.zeros(3))
    assert e.value.code == -3
    small_ctx.close()


def test_warm_started_frames_match_oracle(ctx, small):
    # Two frames at different angles: the second starts from the first's w and
    # last accepted step, on the GPU (model state) and in the oracle (arguments).
    om, geom, vol = small["om"], small["geom"], small["vol"]
    from phantom import dvf_analytic

    angles = (0.3, 0.32)
    ys = []
    for i, th in enumerate(angles):
        ft = O.warp(vol, om.f0, dvf_analytic(vol, 1.0 + i / 6.0, 1.5))
        ys.append(_f32(noisy(O.project(vol, geom, th, ft), 10 + i)))
    so = library_opts(max_iters=6)
    a = ctx.reconstruct(small["mid"], ys[0], angles[0], _opts(max_iters=6, cold_start=1, w0=[0, 0, 0]))
    log_a = ctx.trial_log(small["mid"])
    b = ctx.reconstruct(small["mid"], ys[1], angles[1], _opts(max_iters=6))
    log_b = ctx.trial_log(small["mid"])
    oa, ties_a, own_a = checked_oracle_solve(
        log_a, lambda rp: O.reconstruct(om, geom, angles[0], _up(ys[0]), np.zeros(3), so, replay=rp), so)
    ob, ties_b, _ = checked_oracle_solve(
        log_b, lambda rp: O.reconstruct(om, geom, angles[1], _up(ys[1]), oa.w, so, mu_next=oa.mu, replay=rp), so)
    # the oracle's own two-frame chain (its own first frame's w and step)
    own_b = O.reconstruct(om, geom, angles[1], _up(ys[1]), own_a.w, so, mu_next=own_a.mu)
    eo = own_path_errors(b, own_b)
    report("warm_frames64", w_rel=rel(b["w"], ob.w), mu_rel=abs(b["mu"] - ob.mu) / ob.mu,
           backtracks=b["backtracks"], oracle_backtracks=ob.backtracks, ties=ties_a + ties_b, **eo)
    assert eo["own_J_rel"] < TOL_PROJ
    # the step is step0 / |grad J| times powers of beta and step_growth, so it
    # carries the gradient's tolerance
    assert abs(a["mu"] - oa.mu) / oa.mu < TOL_GRAD
    assert b["backtracks"] == ob.backtracks
    assert rel(b["w"], ob.w) < TOL_W
    assert abs(b["J"] - ob.J) / ob.J < TOL_PROJ


def test_predicted_start_matches_oracle_chain(ctx, small):
    # Four frames with the linear predictor: the oracle chain starts frame j
    # from 2 w(j-1) - w(j-2) of its own earlier solves (and the warm step).
    from phantom import dvf_analytic

    om, geom, vol = small["om"], small["geom"], small["vol"]
    frames = []
    for j in range(4):
        th = 0.2 + 0.02 * j
        ft = O.warp(vol, om.f0, dvf_analytic(vol, 0.6 + j / 6.0, 1.5))
        frames.append((th, _f32(noisy(O.project(vol, geom, th, ft), 40 + j))))
    gpu, logs = [], []
    for j, (th, y) in enumerate(frames):
        kw = dict(max_iters=5, predict=1)
        if j == 0:
            kw.update(cold_start=1, w0=[0, 0, 0])
        gpu.append(ctx.reconstruct(small["mid"], y, th, _opts(**kw)))
        logs.append(ctx.trial_log(small["mid"]))
    ws, mu = [], None
    ws_own, mu_own = [], None
    so = library_opts(max_iters=5)
    for j, (th, y) in enumerate(frames):
        w0 = np.zeros(3) if j == 0 else (ws[-1] if j == 1 else 2 * ws[-1] - ws[-2])
        r, ties, _ = checked_oracle_solve(
            logs[j], lambda rp: O.reconstruct(om, geom, th, _up(y), w0, so, mu_next=mu, replay=rp), so)
        ws.append(r.w)
        mu = r.mu
        # the oracle's own chain, every frame on its own choices
        w0_own = np.zeros(3) if j == 0 else (ws_own[-1] if j == 1 else 2 * ws_own[-1] - ws_own[-2])
        own = O.reconstruct(om, geom, th, _up(y), w0_own, so, mu_next=mu_own)
        ws_own.append(own.w)
        mu_own = own.mu
        eo = own_path_errors(gpu[j], own)
        report("predict_chain64", frame=j, w_rel=rel(gpu[j]["w"], r.w), backtracks=gpu[j]["backtracks"],
               oracle_backtracks=r.backtracks, ties=ties, **eo)
        assert eo["own_J_rel"] < TOL_PROJ
        assert gpu[j]["backtracks"] == r.backtracks
        assert rel(gpu[j]["w"], r.w) < TOL_W
