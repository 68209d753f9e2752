"""Whole-grid inversion of the pull-back DVF (Section 2.3 with ref. 13): the
CUDA path through the C ABI against the oracle's whole-field fixed-point
sweeps on the same float32 fields (upcast exactly). The field is compared
voxel by voxel; its values are displacements in mm, so the bar is absolute:
1e-3 mm, a hundredth of the tumor-position tolerance (FP32 keeps the iterates
to about 1e-5 mm)."""

import numpy as np
import pytest

from gpu_util import report
from oracle import oracle as O
from phantom import Geometry, Volume

pytestmark = pytest.mark.gpu

TOL_FIELD_MM = 1e-3
GPU_TOL_MM = 1e-5


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _up(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def ctx():
    from paper_1004_0014_b300 import Context

    c = Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small(ctx, small_case):
    c = small_case
    f0, mean, U = _f32(c["f0"]), _f32(c["pca"].mean), _f32(c["pca"].U)
    mid = ctx.load_model(c["vol"], c["geom"], f0, mean, U, c["c0"])
    return dict(c, mid=mid, mean=_up(mean), U=_up(U))


@pytest.mark.parametrize("w", [[0.0, 0.0, 0.0], [1.2, -0.3, 0.1], [-2.5, 0.8, -0.4]])
def test_inverse_field_matches_oracle(ctx, small, w):
    w = np.array(w)
    y, steps, open_ = ctx.invert_dvf(small["mid"], w, tol=GPU_TOL_MM, max_iter=64)
    yo, sweeps = O.invert(small["vol"], small["mean"], small["U"], w, tol=1e-10, max_iter=200)
    err = float(np.max(np.abs(y.cpu().numpy().astype(np.float64) - yo)))
    report("invert64", w=w, max_abs_mm=err, max_steps=steps, oracle_sweeps=sweeps, unconverged=open_,
           field_max_mm=float(np.max(np.abs(yo))))
    assert open_ == 0
    assert err < TOL_FIELD_MM
    assert np.max(np.abs(yo)) > 1.0  # the mean field alone moves voxels by millimetres


def test_inverse_field_of_translation_and_ragged_grid(ctx):
    # a constant field on a grid whose size is not a multiple of 4 and with one
    # axis of length 1: y = -t everywhere, reached in two updates
    vol = Volume(7, 5, 1, 2.0, 2.5, 3.0)
    geom = Geometry(1000.0, 1500.0, 16, 8, 2.0, 2.0, 0.0)
    t = np.array([1.3, -2.1, 4.4])
    mean = np.zeros((3,) + vol.shape, np.float32)
    for c in range(3):
        mean[c] = t[c]
    U = np.zeros((1, 3) + vol.shape, np.float32)
    f0 = np.ones(vol.shape, np.float32)
    mid = ctx.load_model(vol, geom, f0, mean, U, np.zeros(3))
    try:
        y, steps, open_ = ctx.invert_dvf(mid, np.zeros(1), tol=GPU_TOL_MM, max_iter=64)
        yo, _ = O.invert(vol, mean.astype(np.float64), U.astype(np.float64), np.zeros(1), tol=1e-12)
        err = float(np.max(np.abs(y.cpu().numpy() - yo)))
        report("invert_translation_ragged", max_abs_mm=err, max_steps=steps)
        assert err < 1e-5
        assert steps <= 2 and open_ == 0
    finally:
        ctx.release_model(mid)


def test_inverse_field_arguments_are_checked(ctx, small):
    import torch

    from paper_1004_0014_b300 import PcaReconError, capi

    vol = small["vol"]
    y = torch.empty((3, vol.nz, vol.ny, vol.nx), dtype=torch.float32, device="cuda")
    for tol, it in ((-1.0, 10), (1e-5, 0), (1e-5, 100001), (float("nan"), 10)):
        with pytest.raises(PcaReconError) as e:
            capi.pr_invert_dvf(ctx._ctx, small["mid"], np.zeros(3), y, tol, it)
        assert e.value.code == -1
    with pytest.raises(PcaReconError) as e:
        capi.pr_invert_dvf(ctx._ctx, 9999, np.zeros(3), y, 1e-5, 10)
    assert e.value.code == -6
    # an iteration cap that stops short is reported, not hidden
    _, steps, open_ = ctx.invert_dvf(small["mid"], np.array([1.2, -0.3, 0.1]), tol=0.0, max_iter=3)
    assert steps == 3 and open_ == vol.nx * vol.ny * vol.nz
