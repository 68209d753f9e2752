"""Host-side arithmetic of the benchmark (no GPU): the count of voxels the
support-restricted warp pass evaluates (chunks of 512 consecutive voxels of
the flat grid that meet the warp box) against a brute-force count, the
algorithmic flops per projector sample, the reading of the clock samples taken
during the timed region (a run that saw a slowdown reason must say so), and
the oracle's time per reconstruction."""

import numpy as np
import pytest

from phantom import Volume


def _brute(vol, box, block=512):
    (x0, y0, z0), (x1, y1, z1) = box
    n = vol.nx * vol.ny * vol.nz
    total = 0
    for b0 in range(0, n, block):
        vs = np.arange(b0, min(b0 + block, n))
        i, jk = vs % vol.nx, vs // vol.nx
        j, k = jk % vol.ny, jk // vol.ny
        hit = (i >= x0) & (i <= x1) & (j >= y0) & (j <= y1) & (k >= z0) & (k <= z1)
        if hit.any():
            total += len(vs)
    return total


@pytest.mark.parametrize("shape", [(13, 11, 9), (40, 36, 28), (256, 7, 5), (1, 1, 3000), (37, 1, 1)])
def test_warp_voxels_evaluated_matches_brute_force(shape):
    import bench

    vol = Volume(*shape, 2.0, 2.0, 2.5)
    rng = np.random.default_rng(sum(shape))
    boxes = [((0, 0, 0), (vol.nx - 1, vol.ny - 1, vol.nz - 1)),  # whole grid
             ((1, 1, 1), (0, 0, 0))]                              # empty box (all-zero volume)
    for _ in range(12):
        lo = [int(rng.integers(0, n)) for n in (vol.nx, vol.ny, vol.nz)]
        hi = [int(rng.integers(l, n)) for l, n in zip(lo, (vol.nx, vol.ny, vol.nz))]
        boxes.append((tuple(lo), tuple(hi)))
    for box in boxes:
        assert bench.warp_voxels_evaluated(vol, box) == _brute(vol, box), box


def test_flops_per_sample():
    import bench

    # 8 trilinear taps x nch channels x one multiply-add (2 flop)
    assert [bench.flops_per_sample(c) for c in (4, 6, 8)] == [64, 96, 128]


def test_timed_frames_spread_over_the_rotation():
    import bench

    fr = bench.timed_frames(20, 5)
    assert fr[:5] == [-5, -4, -3, -2, -1]
    assert fr[5:] == [18 * i for i in range(20)]
    assert bench.timed_frames(360, 3)[3:] == list(range(360))
    assert bench.timed_frames(400, 3)[3:] == list(range(400))
    assert bench.frame_list_text(fr[5:]) == "0, 18, ..., 342"


def test_openmp_oracle_matches_the_plain_build():
    """The all-cores build times the same method: the projection and warp
    bitwise, the scatter-form transpose to rounding (another summation order)."""
    from oracle import oracle as O
    from phantom import Geometry, Volume, phantom_volume

    vol = Volume(20, 18, 16, 4.0, 4.0, 5.0)
    geom = Geometry(1000.0, 1500.0, 24, 20, 3.6, 3.6, 2.0)
    f = phantom_volume(vol)
    r = np.random.default_rng(4).random((geom.nv, geom.nu))
    out = {}
    try:
        for omp in (False, True):
            O.use_openmp(omp)
            out[omp] = (O.project(vol, geom, 0.7, f), O.backproject(vol, geom, 0.7, r))
    finally:
        O.use_openmp(False)
    assert np.array_equal(out[False][0], out[True][0])
    bp0, bp1 = out[False][1], out[True][1]
    assert np.max(np.abs(bp0 - bp1)) <= 1e-12 * np.max(np.abs(bp0))


def _sampler(lines):
    import bench

    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_reports_slowdowns_and_busy_median():
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2032, 2032, 700.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2032, 2032, 910.4, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 1980, 2032, 1050.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 345, 2032, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # idle sample
             "garbage line",
             "0, 2010, 2032, 990.0, 0x20, Not Active, Active, Not Active, Not Active"]
    s = _sampler(lines)
    assert s["samples"] == 5
    assert s["sm_max_mhz"] == 2032.0
    assert s["sm_mhz"] == 2021.0  # median of the busy samples (the 345 MHz one is idle)
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    s = _sampler([])
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == ["no samples"]


def test_oracle_reconstruction_time():
    import bench

    # Eq. 4 at the start costs one evaluation and one gradient; each trial one
    # evaluation; each accepted step one gradient
    assert bench.oracle_recon_seconds(2.0, 5.0, iters=10, trials=11) == 12 * 2.0 + 11 * 5.0
