"""Batched solves in one CUDA graph: frames of several patients (different
volume sizes and K) solved by one pr_reconstruct_batch launch give, frame by
frame, exactly the results of solving them one at a time in the same order
(the kernels' reductions are deterministic)."""

import numpy as np
import pytest

from gpu_util import noisy
from oracle import oracle as O
from phantom import Geometry, Volume, build_pca, dvf_analytic, phantom_volume, training_dvfs, tumor_centre

pytestmark = pytest.mark.gpu

SHAPES = [((48, 48, 40), 3), ((64, 56, 48), 5), ((40, 36, 30), 4)]
GEOM = Geometry(1000.0, 1500.0, 96, 80, 2.0, 2.0, 0.0)
FRAMES = 4
KEYS = ("w", "a", "b", "J", "tumor", "iters", "trials", "backtracks", "stop_reason")


def _patient(i):
    (nx, ny, nz), K = SHAPES[i]
    vol = Volume(nx, ny, nz, 4.0, 4.0, 5.0)
    f0 = phantom_volume(vol).astype(np.float32)
    pca = build_pca(training_dvfs(vol), K)
    g = Geometry(GEOM.sad, GEOM.sdd, GEOM.nu, GEOM.nv, GEOM.du, GEOM.dv, 0.5 * min(vol.dx, vol.dy, vol.dz))
    frames = []
    for j in range(FRAMES):
        th, t = np.deg2rad(11.0 * j + 40 * i), 0.3 + j / 6.0
        ft = O.warp(vol, f0.astype(np.float64), dvf_analytic(vol, t, 1.5))
        frames.append((th, noisy(O.project(vol, g, th, ft), 500 + 10 * i + j).astype(np.float32)))
    return dict(vol=vol, f0=f0, mean=pca.mean.astype(np.float32), U=pca.U.astype(np.float32), K=K,
                c0=tumor_centre(vol), frames=frames)


@pytest.fixture(scope="module")
def setup():
    from paper_1004_0014_b300 import Context

    pats = [_patient(i) for i in range(len(SHAPES))]
    ctx = Context(0)
    mids = [ctx.load_model(p["vol"], GEOM, p["f0"], p["mean"], p["U"], p["c0"]) for p in pats]
    order = [(i, j) for j in range(FRAMES) for i in range(len(pats))]  # interleaved arrivals
    yield dict(ctx=ctx, pats=pats, mids=mids, order=order)
    ctx.close()


def _reset(s):
    for p, mid in zip(s["pats"], s["mids"]):
        s["ctx"].set_state(mid, np.zeros(p["K"]))


def _opts():
    from paper_1004_0014_b300 import default_opts

    return default_opts(max_iters=6)


def test_batch_equals_one_at_a_time(setup):
    s = setup
    ctx, pats, mids, order = s["ctx"], s["pats"], s["mids"], s["order"]
    _reset(s)
    solo = [ctx.reconstruct(mids[i], pats[i]["frames"][j][1], pats[i]["frames"][j][0], _opts()) for i, j in order]
    for rnd in range(2):  # the second call reuses the instantiated graph
        _reset(s)
        got = ctx.reconstruct_batch([mids[i] for i, _ in order], [pats[i]["frames"][j][1] for i, j in order],
                                    [pats[i]["frames"][j][0] for i, j in order], _opts())
        for n, (a, b) in enumerate(zip(solo, got)):
            for k in KEYS:
                assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), (rnd, n, k)
    # the models keep the batch's last states as warm starts
    for i, mid in enumerate(mids):
        last = max(n for n, (pi, _) in enumerate(order) if pi == i)
        assert np.array_equal(ctx.get_state(mid), np.asarray(got[last]["w"]))


def test_batch_arguments_and_release(setup):
    from paper_1004_0014_b300 import PcaReconError, capi

    s = setup
    ctx, pats, mids = s["ctx"], s["pats"], s["mids"]
    y0, th0 = pats[0]["frames"][0][1], pats[0]["frames"][0][0]
    with pytest.raises(PcaReconError) as e:
        ctx.reconstruct_batch([9999], [y0], [th0])
    assert e.value.code == -6
    with pytest.raises(PcaReconError) as e:
        ctx.reconstruct_batch([mids[0]], [y0], [float("nan")])
    assert e.value.code == -1
    with pytest.raises(PcaReconError) as e:
        capi.pr_reconstruct_batch(ctx._ctx, [], [], [])
    assert e.value.code == -1
    ctx.serve_start(slots=2)
    with pytest.raises(PcaReconError) as e:
        ctx.reconstruct_batch([mids[0]], [y0], [th0])
    assert e.value.code == -1
    ctx.serve_stop()
    # a batch over a model that is then released: the next batch rebuilds its graph
    p = pats[2]
    extra = ctx.load_model(p["vol"], GEOM, p["f0"], p["mean"], p["U"], p["c0"])
    ctx.reconstruct_batch([mids[0], extra], [y0, p["frames"][0][1]], [th0, p["frames"][0][0]], _opts())
    ctx.release_model(extra)
    r = ctx.reconstruct_batch([mids[0], mids[1]], [y0, pats[1]["frames"][0][1]], [th0, pats[1]["frames"][0][0]],
                              _opts())
    assert len(r) == 2 and all(x["iters"] >= 1 for x in r)
