"""Degenerate and edge cases of the method on the GPU: a single PCA mode, an
all-zero reference volume, a one-pixel detector (Eq. 4 singular) and a
one-slice volume, each against the oracle or the method's defined stop."""

import numpy as np
import pytest

from gpu_util import (TOL_GRAD, TOL_PROJ, TOL_W, checked_oracle_solve, library_opts, noisy, own_path_errors, rel,
                      report)
from oracle import oracle as O
from phantom import Geometry, Volume

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1004_0014_b300 import Context

    c = Context(0)
    yield c
    c.close()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def test_single_mode_model(ctx, small_case):
    from paper_1004_0014_b300 import default_opts

    c = small_case
    f0, mean, U = _f32(c["f0"]), _f32(c["pca"].mean), _f32(c["pca"].U[:1])
    mid = ctx.load_model(c["vol"], c["geom"], f0, mean, U, c["c0"])
    om = O.Model(c["vol"], f0.astype(np.float64), mean.astype(np.float64), U.astype(np.float64), c["c0"])
    y = _f32(noisy(O.project(c["vol"], c["geom"], c["angle"], O.warp(c["vol"], om.f0, c["x_test"])), 1))
    try:
        import torch

        yd = torch.from_numpy(y).cuda()
        go, Jo, _ = O.gradient(om, c["geom"], c["angle"], np.array([0.8]), 1.0, 0.0, y.astype(np.float64))
        for mode in (0, 1):
            J, g = ctx.cost_grad(mid, yd, c["angle"], np.array([0.8]), 1.0, 0.0, mode)
            assert abs(J - Jo) / Jo < TOL_PROJ and rel(g, go) < TOL_GRAD
        res = ctx.reconstruct(mid, y, c["angle"], default_opts(max_iters=10, cold_start=1))
        so = library_opts(max_iters=10)
        ores, ties, own = checked_oracle_solve(
            ctx.trial_log(mid),
            lambda rp: O.reconstruct(om, c["geom"], c["angle"], y.astype(np.float64), np.zeros(1), so, replay=rp),
            so)
        eo = own_path_errors(res, own)
        report("k1_solve", w_rel=rel(res["w"], ores.w), J_rel=abs(res["J"] - ores.J) / ores.J, ties=ties, **eo)
        assert eo["own_J_rel"] < TOL_PROJ
        assert res["iters"] == ores.iters and rel(res["w"], ores.w) < TOL_W
    finally:
        ctx.release_model(mid)


def test_all_zero_reference_volume(ctx, small_case):
    # p = 0 for every w: Eq. 4 gives a = b = 0, the gradient is 0, and the
    # solve stops on the gradient test at its start, as the oracle does
    from paper_1004_0014_b300 import PR_STOP_GRAD_TOL, default_opts

    c = small_case
    f0 = np.zeros(c["vol"].shape, np.float32)
    mean, U = _f32(c["pca"].mean), _f32(c["pca"].U)
    mid = ctx.load_model(c["vol"], c["geom"], f0, mean, U, c["c0"])
    om = O.Model(c["vol"], f0.astype(np.float64), mean.astype(np.float64), U.astype(np.float64), c["c0"])
    y = _f32(1.0 + np.random.default_rng(3).random((c["geom"].nv, c["geom"].nu)))
    try:
        w0 = [0.3, -0.1, 0.05]
        res = ctx.reconstruct(mid, y, 0.4, default_opts(max_iters=5, cold_start=1, w0=w0))
        ores = O.reconstruct(om, c["geom"], 0.4, y.astype(np.float64), np.array(w0), library_opts(max_iters=5))
        assert res["stop_reason"] == ores.stop_reason == PR_STOP_GRAD_TOL
        assert res["iters"] == ores.iters == 0
        assert np.array_equal(res["w"], np.array(w0))
        assert res["a"] == 0.0 and res["b"] == 0.0 and res["J"] == 0.0
        assert ctx.count_samples(mid, 0.4, np.array(w0)) == 0
    finally:
        ctx.release_model(mid)


def test_one_pixel_detector_stops_on_singular_fit(ctx, small_case):
    from paper_1004_0014_b300 import PR_STOP_SINGULAR_FIT, default_opts

    c = small_case
    geom = Geometry(1000.0, 1500.0, 1, 1, 1.6, 1.6, 0.0)
    f0, mean, U = _f32(c["f0"]), _f32(c["pca"].mean), _f32(c["pca"].U)
    mid = ctx.load_model(c["vol"], geom, f0, mean, U, c["c0"])
    try:
        w0 = [0.2, 0.0, 0.0]
        res = ctx.reconstruct(mid, np.array([[3.0]], np.float32), 0.0, default_opts(cold_start=1, w0=w0))
        assert res["stop_reason"] == PR_STOP_SINGULAR_FIT
        assert np.array_equal(res["w"], np.array(w0)) and np.all(np.isfinite(res["tumor"]))
    finally:
        ctx.release_model(mid)


def test_one_slice_volume(ctx):
    # a 1-voxel-thick volume: the interpolant runs from the slice to the zero
    # padding along z; warp and projection (forward model) against the oracle
    vol = Volume(32, 28, 1, 4.0, 4.0, 4.0)
    geom = Geometry(1000.0, 1500.0, 40, 8, 4.0, 4.0, 0.0)
    rng = np.random.default_rng(9)
    f0 = _f32(rng.random(vol.shape))
    mean = _f32(0.5 * rng.standard_normal((3,) + vol.shape))
    U = _f32(0.5 * rng.standard_normal((2, 3) + vol.shape))
    mid = ctx.load_model(vol, geom, f0, mean, U, np.zeros(3))
    om = O.Model(vol, f0.astype(np.float64), mean.astype(np.float64), U.astype(np.float64), np.zeros(3))
    try:
        w = np.array([0.7, -0.4])
        f, _ = ctx.warp(mid, w, with_h=False)
        fo = O.warp(vol, om.f0, O.dvf(vol, om.mean, om.U, w))
        gg = Geometry(geom.sad, geom.sdd, geom.nu, geom.nv, geom.du, geom.dv, 2.0)
        for th in (0.0, 0.9):
            p = ctx.forward(mid, w, th).cpu().numpy()
            po = O.project(vol, gg, th, fo)
            report("one_slice", angle=th, f_rel=rel(f.cpu().numpy(), fo), p_rel=rel(p, po))
            assert rel(p, po) < TOL_PROJ
        assert rel(f.cpu().numpy(), fo) < 1e-5
    finally:
        ctx.release_model(mid)
