"""Serving: frames of several patients (different volume sizes) submitted
together run concurrently, in stream slots or in tick-batched launches (one
graph launch per tick over the pending frames of every patient); every
frame's result must be the same as when that patient's frames are solved
alone, one after the other (the kernels' reductions are deterministic, so
the same means bitwise). Over-budget patients wait in the admission queue
until a release frees memory."""

import numpy as np
import pytest

from gpu_util import noisy
from oracle import oracle as O
from phantom import Geometry, Volume, build_pca, dvf_analytic, phantom_volume, training_dvfs, tumor_centre

pytestmark = pytest.mark.gpu

SHAPES = [(48, 48, 40), (64, 64, 64), (40, 36, 30)]
GEOM = Geometry(1000.0, 1500.0, 96, 80, 2.0, 2.0, 0.0)
FRAMES = 6


def _patient(i):
    nx, ny, nz = SHAPES[i]
    vol = Volume(nx, ny, nz, 4.0, 4.0, 5.0)
    f0 = phantom_volume(vol).astype(np.float32)
    pca = build_pca(training_dvfs(vol), 3)
    frames = []
    for j in range(FRAMES):
        th, t = np.deg2rad(7.0 * j + 30 * i), 0.5 + j / 6.0
        ft = O.warp(vol, f0.astype(np.float64), dvf_analytic(vol, t, 1.5))
        g = Geometry(GEOM.sad, GEOM.sdd, GEOM.nu, GEOM.nv, GEOM.du, GEOM.dv, 0.5 * min(vol.dx, vol.dy, vol.dz))
        frames.append((th, noisy(O.project(vol, g, th, ft), 100 * i + j).astype(np.float32)))
    return dict(vol=vol, f0=f0, mean=pca.mean.astype(np.float32), U=pca.U.astype(np.float32),
                c0=tumor_centre(vol), frames=frames)


@pytest.fixture(scope="module")
def patients():
    return [_patient(i) for i in range(len(SHAPES))]


def _opts():
    from paper_1004_0014_b300 import default_opts

    return default_opts(max_iters=6)


def _solo(ctx, mids, patients):
    solo = {}
    for i, (mid, p) in enumerate(zip(mids, patients)):
        ctx.set_state(mid, np.zeros(3))
        for j, (th, y) in enumerate(p["frames"]):
            solo[(i, j)] = ctx.reconstruct(mid, y, th, _opts())
    return solo


def _same(a, b, key):
    for k in ("w", "a", "b", "J", "tumor", "iters", "trials"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), (key, k)


@pytest.mark.parametrize("storage", ["f32", "bf16", "mixed"])
@pytest.mark.parametrize("mode", ["slots", "batched"])
def test_served_results_equal_solo_results(patients, mode, storage):
    """storage: every model in float32 or bfloat16, or "mixed" (the middle
    patient in float32, the others in bfloat16)."""
    from paper_1004_0014_b300 import PR_BF16, PR_F32, Context

    def st(i):
        if storage == "mixed":
            return PR_F32 if i == 1 else PR_BF16
        return PR_BF16 if storage == "bf16" else PR_F32

    ctx = Context(0)
    try:
        mids = [ctx.load_model(p["vol"], GEOM, p["f0"], p["mean"], p["U"], p["c0"], storage=st(i))
                for i, p in enumerate(patients)]
        solo = _solo(ctx, mids, patients)
        for mid in mids:
            ctx.set_state(mid, np.zeros(3))
        if mode == "slots":
            ctx.serve_start(slots=3)
        else:
            ctx.serve_start(batched_lanes=2)
        # interleave the patients' frames as they would arrive
        for j in range(FRAMES):
            for i, (mid, p) in enumerate(zip(mids, patients)):
                th, y = p["frames"][j]
                ctx.submit(mid, y, th, _opts(), tag=1000 * i + j)
        served = {}
        while len(served) < len(solo):
            r = ctx.poll(timeout_ms=60000)
            assert r is not None and r["status"] == 0
            served[(r["tag"] // 1000, r["tag"] % 1000)] = r
            assert r["latency_ms"] >= r["gpu_ms"] * 0.999 >= 0.0
        ctx.serve_stop()
        for key, a in solo.items():
            _same(a, served[key], key)
    finally:
        ctx.close()


def test_admission_and_release_rules(patients):
    from paper_1004_0014_b300 import Context, PcaReconError

    p0, p1 = patients[0], patients[1]
    probe = Context(0)
    need0 = probe.footprint(probe.load_model(p0["vol"], GEOM, p0["f0"], p0["mean"], p0["U"], p0["c0"]))
    need1 = probe.footprint(probe.load_model(p1["vol"], GEOM, p1["f0"], p1["mean"], p1["U"], p1["c0"]))
    probe.close()
    # a budget that holds either patient alone but not both together
    budget = max(need0, need1) + min(need0, need1) // 2
    ctx = Context(0, hbm_budget_bytes=budget)
    try:
        a = ctx.load_model(p0["vol"], GEOM, p0["f0"], p0["mean"], p0["U"], p0["c0"])
        with pytest.raises(PcaReconError) as e:
            ctx.load_model(p1["vol"], GEOM, p1["f0"], p1["mean"], p1["U"], p1["c0"])
        assert e.value.code == -3
        ctx.serve_start(slots=2)
        with pytest.raises(PcaReconError):
            ctx.poll(timeout_ms=0)  # nothing outstanding
        for j, (th, y) in enumerate(p0["frames"]):  # one patient's frames run in order
            ctx.submit(a, y, th, _opts(), tag=j)
        with pytest.raises(PcaReconError) as e:
            ctx.release_model(a)  # frames outstanding
        assert e.value.code == -1
        tags = sorted(ctx.poll(timeout_ms=60000)["tag"] for _ in p0["frames"])
        assert tags == list(range(len(p0["frames"])))
        ctx.serve_stop()
        ctx.release_model(a)
        # the freed budget admits the other patient
        b = ctx.load_model(p1["vol"], GEOM, p1["f0"], p1["mean"], p1["U"], p1["c0"])
        ctx.serve_start(slots=2)
        th, y = p1["frames"][0]
        ctx.submit(b, y, th, _opts(), tag=8)
        assert ctx.poll(timeout_ms=60000)["tag"] == 8
        ctx.serve_stop()
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", ["batched", "slots"])
def test_admission_queue_admits_a_waiting_patient_after_a_release(patients, mode):
    """A budget that holds one of two patients: the second is queued
    (PR_QUEUED, status waiting), its submitted frames wait, and releasing
    the first admits it; its served frames then equal its solo results."""
    from paper_1004_0014_b300 import Context, PcaReconError, capi

    p0, p1 = patients[0], patients[1]
    ref = Context(0)
    try:
        r0 = ref.load_model(p0["vol"], GEOM, p0["f0"], p0["mean"], p0["U"], p0["c0"])
        r1 = ref.load_model(p1["vol"], GEOM, p1["f0"], p1["mean"], p1["U"], p1["c0"])
        need0, need1 = ref.footprint(r0), ref.footprint(r1)
        solo1 = _solo(ref, [r1], [p1])
    finally:
        ref.close()
    budget = max(need0, need1) + min(need0, need1) // 2
    ctx = Context(0, hbm_budget_bytes=budget)
    try:
        ctx.set_admission_queue(True)
        a = ctx.load_model(p0["vol"], GEOM, p0["f0"], p0["mean"], p0["U"], p0["c0"])
        b = ctx.load_model(p1["vol"], GEOM, p1["f0"], p1["mean"], p1["U"], p1["c0"])
        assert ctx.model_status(a) == capi.PR_MODEL_RESIDENT
        assert ctx.model_status(b) == capi.PR_MODEL_WAITING
        with pytest.raises(PcaReconError) as e:
            ctx.reconstruct(b, p1["frames"][0][1], 0.0)  # not resident yet
        assert e.value.code == -6
        ctx.set_state(a, np.zeros(3))
        if mode == "batched":
            ctx.serve_start(batched_lanes=2)
        else:
            ctx.serve_start(slots=2)
        for j, (th, y) in enumerate(p1["frames"]):
            ctx.submit(b, y, th, _opts(), tag=100 + j)
        for j, (th, y) in enumerate(p0["frames"][:2]):
            ctx.submit(a, y, th, _opts(), tag=j)
        got = sorted(ctx.poll(timeout_ms=60000)["tag"] for _ in range(2))
        assert got == [0, 1]  # the resident patient's frames are served
        assert ctx.poll(timeout_ms=300) is None  # the waiting patient's frames stay queued
        ctx.release_model(a)  # frees the budget: b is admitted and its frames run
        assert ctx.model_status(b) == capi.PR_MODEL_RESIDENT
        served = {}
        for _ in p1["frames"]:
            r = ctx.poll(timeout_ms=60000)
            assert r["status"] == 0
            served[(0, r["tag"] - 100)] = r
        ctx.serve_stop()
        for key, s1 in solo1.items():
            _same(s1, served[key], key)
    finally:
        ctx.close()
