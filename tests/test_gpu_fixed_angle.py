"""Fixed-angle geometry (Section 5): the transpose's per-voxel footprint weights
stored once for an angle give the same adjoint results, bit for bit, as the
weights computed on the fly; other angles are untouched; the table is counted
against the HBM budget and can be dropped."""

import math

import numpy as np
import pytest

from gpu_util import noisy, rel, report
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(small_case):
    import torch

    from paper_1004_0014_b300 import Context

    c = small_case
    f0, mean, U = (np.ascontiguousarray(a, dtype=np.float32) for a in (c["f0"], c["pca"].mean, c["pca"].U))
    ctx = Context(0)
    mid = ctx.load_model(c["vol"], c["geom"], f0, mean, U, c["c0"])
    om = O.Model(c["vol"], f0.astype(np.float64), mean.astype(np.float64), U.astype(np.float64), c["c0"])
    th = 0.35
    y = noisy(O.project(c["vol"], c["geom"], th, O.warp(c["vol"], om.f0, c["x_test"])), 3).astype(np.float32)
    rng = np.random.default_rng(5)
    gp = torch.from_numpy(rng.standard_normal((c["geom"].nv, c["geom"].nu)).astype(np.float32)).cuda()
    yield dict(c, ctx=ctx, mid=mid, om=om, th=th, y=y, yd=torch.from_numpy(y).cuda(), gp=gp)
    ctx.close()


def test_fixed_angle_adjoint_is_bitwise_the_same(setup):
    s = setup
    ctx, mid, th = s["ctx"], s["mid"], s["th"]
    w = np.array([0.7, -0.2, 0.1])
    v_free = ctx.vjp(mid, w, th, s["gp"])
    before = ctx.footprint(mid)  # after the adjoint's h scratch was allocated
    v_other = ctx.vjp(mid, w, th + 0.5, s["gp"])
    J_free, g_free = ctx.cost_grad(mid, s["yd"], th, w, 1.0, 0.0, 1)
    nbytes = ctx.fix_angle(mid, th)
    assert nbytes > 0 and ctx.footprint(mid) == before + nbytes
    v_fix = ctx.vjp(mid, w, th, s["gp"])
    J_fix, g_fix = ctx.cost_grad(mid, s["yd"], th, w, 1.0, 0.0, 1)
    assert np.array_equal(v_fix, v_free)
    assert J_fix == J_free and np.array_equal(g_fix, g_free)
    assert np.array_equal(ctx.vjp(mid, w, th + 0.5, s["gp"]), v_other)  # not the cached angle
    # and against the oracle: the adjoint form of the gradient
    go, Jo, _ = O.gradient(s["om"], s["geom"], th, w, 1.0, 0.0, s["y"].astype(np.float64))
    report("fixed_angle_adjoint64", table_mb=nbytes / 2**20, g_rel=rel(g_fix, go), J_rel=abs(J_fix - Jo) / Jo)
    assert rel(g_fix, go) < 1e-4
    ctx.fix_angle(mid, math.nan)
    assert ctx.footprint(mid) == before
    assert np.array_equal(ctx.vjp(mid, w, th, s["gp"]), v_free)


def test_fixed_angle_table_is_admitted_by_budget(setup):
    from paper_1004_0014_b300 import Context, PcaReconError

    s = setup
    need = s["ctx"].footprint(s["mid"])
    f0, mean, U = (np.ascontiguousarray(a, dtype=np.float32) for a in (s["f0"], s["pca"].mean, s["pca"].U))
    small = Context(0, hbm_budget_bytes=need + 1024)  # the model fits, its table does not
    try:
        mid = small.load_model(s["vol"], s["geom"], f0, mean, U, s["c0"])
        fp0 = small.footprint(mid)
        with pytest.raises(PcaReconError) as e:
            small.fix_angle(mid, s["th"])
        assert e.value.code == -3
        assert small.footprint(mid) == fp0
        with pytest.raises(PcaReconError) as e:
            small.fix_angle(mid, math.inf)
        assert e.value.code == -1
    finally:
        small.close()


def test_adjoint_scratch_is_charged_to_the_budget(setup):
    """The adjoint's h scratch is allocated on first use: it must fit the
    context's HBM budget, and releasing the model returns exactly what was
    charged (a later model of the same size is admitted again)."""
    from paper_1004_0014_b300 import Context, PcaReconError

    s = setup
    f0, mean, U = (np.ascontiguousarray(a, dtype=np.float32) for a in (s["f0"], s["pca"].mean, s["pca"].U))
    probe = Context(0)
    need = probe.footprint(probe.load_model(s["vol"], s["geom"], f0, mean, U, s["c0"]))
    probe.close()
    c = Context(0, hbm_budget_bytes=need + 1024)  # the model fits, its adjoint scratch does not
    try:
        mid = c.load_model(s["vol"], s["geom"], f0, mean, U, s["c0"])
        with pytest.raises(PcaReconError) as e:
            c.vjp(mid, np.zeros(3), s["th"], s["gp"])
        assert e.value.code == -3
        assert c.footprint(mid) == need
        c.release_model(mid)
        mid = c.load_model(s["vol"], s["geom"], f0, mean, U, s["c0"])
        assert c.footprint(mid) == need
    finally:
        c.close()
    roomy = Context(0, hbm_budget_bytes=2 * need + 8 * s["vol"].nx * s["vol"].ny * s["vol"].nz * 4)
    try:
        for _ in range(3):  # load, use the adjoint, release: the budget must not drift
            mid = roomy.load_model(s["vol"], s["geom"], f0, mean, U, s["c0"])
            roomy.vjp(mid, np.zeros(3), s["th"], s["gp"])
            roomy.release_model(mid)
    finally:
        roomy.close()
