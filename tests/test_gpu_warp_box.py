"""The solver's warp pass (Eq. 1 and the pull-back of Section 2.2) evaluates
only the 512-voxel chunks of the grid that meet the support box of the warped
volume: the displacement bound around the nonzero voxels of f0. Every other chunk is
written as zeros without reading a field, or left alone where no earlier pass
can have left a nonzero in it. These tests check the bound itself
(every nonzero f or h_k of the unrestricted warp lies in the reported box),
that the box really restricts the work on the phantoms, projections and
gradients at displacements of several voxels against the oracle, and that the
solver volume survives the whole-grid inversion that borrows it as scratch."""

import numpy as np
import pytest

from gpu_util import TOL_GRAD, TOL_PROJ, noisy, rel, report
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


def _compact_model():
    """A 40x36x28 grid whose reference volume is nonzero only in a sub-block
    (random values there), with smooth fields of up to about 3 voxels."""
    vol = Volume(40, 36, 28, 2.0, 2.0, 2.5)
    geom = Geometry(1000.0, 1500.0, 96, 80, 1.6, 1.6, 1.0)
    rng = np.random.default_rng(21)
    f0 = np.zeros(vol.shape)
    f0[8:20, 10:26, 12:30] = rng.random((12, 16, 18)) + 0.1
    z, y, x = np.meshgrid(*(np.linspace(0.0, 1.0, n) for n in vol.shape), indexing="ij")
    mean = np.stack([1.5 * np.sin(2.0 * y), 1.0 * np.cos(3.0 * x), 2.0 * z])
    U = np.stack([np.stack([np.sin(3.0 * x + k), np.cos(2.0 * z - k), 1.5 * np.sin(y + z + k)]) for k in range(2)])
    return vol, geom, _f32(f0), _f32(mean), _f32(U)


def _nonzero_inside(f, h, box):
    (x0, y0, z0), (x1, y1, z1) = box
    nz = (f != 0) | np.any(h != 0, axis=0)
    kk, jj, ii = np.nonzero(nz)
    inside = (ii >= x0) & (ii <= x1) & (jj >= y0) & (jj <= y1) & (kk >= z0) & (kk <= z1)
    return int(nz.sum()), bool(np.all(inside))


def test_box_holds_every_nonzero_voxel_compact(ctx):
    vol, geom, f0, mean, U = _compact_model()
    mid = ctx.load_model(vol, geom, f0, mean, U, np.zeros(3))
    try:
        for w in ([0.0, 0.0], [1.5, -0.7], [-3.0, 2.5], [4.0, 4.0]):
            box = ctx.warp_box(mid, np.array(w))
            f, h = ctx.warp(mid, np.array(w))
            count, ok = _nonzero_inside(f.cpu().numpy(), h.cpu().numpy(), box)
            frac = np.prod([box[1][c] - box[0][c] + 1 for c in range(3)]) / (vol.nx * vol.ny * vol.nz)
            report("warp_box_compact", w=w, box=box, nonzero=count, box_frac=frac)
            assert count > 0 and ok
            assert frac < 1.0  # the compact volume's box leaves part of the grid out
    finally:
        ctx.release_model(mid)


def test_box_holds_every_nonzero_voxel_phantom(ctx, small_case):
    c = small_case
    mid = ctx.load_model(c["vol"], c["geom"], _f32(c["f0"]), _f32(c["pca"].mean), _f32(c["pca"].U), c["c0"])
    try:
        for w in ([0.0, 0.0, 0.0], [1.2, -0.4, 0.2], [-3.0, 1.0, -0.5]):
            box = ctx.warp_box(mid, np.array(w))
            f, h = ctx.warp(mid, np.array(w))
            count, ok = _nonzero_inside(f.cpu().numpy(), h.cpu().numpy(), box)
            report("warp_box_phantom", w=w, box=box, nonzero=count)
            assert count > 0 and ok
    finally:
        ctx.release_model(mid)


def test_restricted_projection_and_gradient_match_oracle(ctx):
    """cost_grad mode 0 (restricted (f, h) volume, forward-mode gradient) and
    mode 1 (restricted f, gather adjoint) at displacements of several voxels,
    in an order that grows and shrinks the box: blocks that held nonzeros at
    the larger box must read as zeros at the smaller one."""
    import torch

    vol, geom, f0, mean, U = _compact_model()
    om = O.Model(vol, f0.astype(np.float64), mean.astype(np.float64), U.astype(np.float64), np.zeros(3))
    mid = ctx.load_model(vol, geom, f0, mean, U, np.zeros(3))
    try:
        big, small = ctx.warp_box(mid, np.array([4.0, 4.0])), ctx.warp_box(mid, np.array([0.2, -0.1]))
        assert any(small[0][c] > big[0][c] or small[1][c] < big[1][c] for c in range(3))
        th = 0.6
        y = _f32(noisy(O.evaluate(om, geom, th, np.array([2.0, -1.0])).p, 3))
        yd = torch.from_numpy(y).cuda()
        for w in ([-3.0, 2.5], [4.0, 4.0], [0.2, -0.1], [4.0, 4.0], [0.2, -0.1]):
            w = np.array(w)
            go, Jo, po = O.gradient(om, geom, th, w, 1.02, 0.01, y.astype(np.float64))
            for mode in (0, 1):
                J, g, pd = ctx.cost_grad(mid, yd, th, w, 1.02, 0.01, mode, return_p=True)
                ep, eJ, eg = rel(pd.cpu().numpy(), po), abs(J - Jo) / Jo, rel(g, go)
                report("warp_box_cost_grad", w=list(w), mode=mode, p_rel=ep, J_rel=eJ, g_rel=eg)
                assert ep < TOL_PROJ and eJ < TOL_PROJ and eg < TOL_GRAD
    finally:
        ctx.release_model(mid)


def test_inversion_scratch_leaves_solves_unchanged(ctx):
    """pr_invert_dvf borrows the solver volume as scratch; a solve after it
    must be bitwise the solve before it (the zero border is restored). The
    reference volume is nonzero up to the grid's faces, so rays sample the
    border."""
    from paper_1004_0014_b300 import default_opts

    vol = Volume(24, 20, 16, 2.0, 2.0, 2.5)
    geom = Geometry(1000.0, 1500.0, 64, 48, 1.6, 1.6, 1.0)
    rng = np.random.default_rng(4)
    f0 = _f32(rng.random(vol.shape) + 0.2)
    mean = _f32(0.5 * rng.standard_normal((3,) + vol.shape))
    U = _f32(rng.standard_normal((2, 3) + vol.shape))
    om = O.Model(vol, f0.astype(np.float64), mean.astype(np.float64), U.astype(np.float64), np.zeros(3))
    mid = ctx.load_model(vol, geom, f0, mean, U, np.zeros(3))
    try:
        th = 0.3
        y = _f32(noisy(O.evaluate(om, geom, th, np.array([0.4, -0.2])).p, 8))
        opts = default_opts(max_iters=6, cold_start=1)
        r0 = ctx.reconstruct(mid, y, th, opts)
        ctx.invert_dvf(mid, np.array([1.0, 0.5]), tol=1e-5, max_iter=64)
        r1 = ctx.reconstruct(mid, y, th, opts)
        report("invert_then_solve", w0=list(r0["w"]), w1=list(r1["w"]), J0=r0["J"], J1=r1["J"])
        assert np.array_equal(r0["w"], r1["w"]) and r0["J"] == r1["J"]
    finally:
        ctx.release_model(mid)
