"""The line-search path checker used by the GPU solve tests (CPU only): the
oracle replays its own choices bitwise, and a choice flipped where it is not a
rounding tie is rejected."""

import numpy as np
import pytest

from gpu_util import TIE_J, checked_oracle_solve, library_opts
from oracle import oracle as O


@pytest.fixture(scope="module")
def solve(small_case):
    c = small_case
    from gpu_util import noisy

    m = O.Model(c["vol"], c["f0"], c["pca"].mean, c["pca"].U, c["c0"])
    y = noisy(O.project(c["vol"], c["geom"], c["angle"], O.warp(c["vol"], m.f0, c["x_test"])), c["seed"])
    so = library_opts(max_iters=8)

    def run(replay):
        return O.reconstruct(m, c["geom"], c["angle"], y, np.zeros(3), so, replay=replay)

    return run, so


def test_replaying_own_choices_is_bitwise(solve):
    run, so = solve
    r = run(None)
    rr = run(r.log)
    assert rr.log == r.log and np.array_equal(rr.w, r.w) and rr.J == r.J
    res, ties, own = checked_oracle_solve(r.log, run, so)
    assert ties == 0 and np.array_equal(res.w, r.w) and own is res


def test_flipping_a_clear_choice_is_rejected(solve):
    run, so = solve
    r = run(None)
    i = max(range(len(r.trace)), key=lambda k: abs(r.trace[k]["margin"]) / abs(r.trace[k]["J"]))
    assert abs(r.trace[i]["margin"]) > 100 * TIE_J * abs(r.trace[i]["J"])
    bad = list(r.log)
    ok, stop, e = bad[i]
    bad[i] = (not ok, False, -1 if ok else 1)
    full = run(bad[:i + 1]).log  # the path that follows the flipped choice
    assert full[:i + 1] == bad[:i + 1]
    with pytest.raises(AssertionError, match="is not a tie"):
        checked_oracle_solve(full, run, so)
