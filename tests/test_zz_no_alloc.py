"""The allocation-free cost/gradient entry point, pr_cost_grad_static.

It serves callers that cannot allocate device memory while they run (a
real-time loop with all memory reserved at start-up, or device memory owned by
another allocator): its scratch is a fixed array inside the library. Here it is
called through the C ABI twice in a row (the second call reuses the array that
the first left behind) and must agree with pr_cost_grad, the allocating entry
point that computes the same cost and gradient, within the gradient tolerance.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""

import numpy as np
import pytest

from gpu_util import TOL_GRAD, TOL_PROJ, rel

pytestmark = pytest.mark.gpu


def test_static_cost_grad_matches_allocating_entry_point(small_case):
    import torch

    from paper_1004_0014_b300 import Context, PcaReconError, capi

    c = small_case
    vol, geom, th = c["vol"], c["geom"], 0.8
    ctx = Context(0)
    try:
        f0 = np.ascontiguousarray(c["f0"], dtype=np.float32)
        mean = np.ascontiguousarray(c["pca"].mean, dtype=np.float32)
        U = np.ascontiguousarray(c["pca"].U, dtype=np.float32)
        mid = ctx.load_model(vol, geom, f0, mean, U, c["c0"])
        K, R = U.shape[0], geom.nu * geom.nv
        # a measured projection: the forward model at other coefficients + 1% noise
        p_true = ctx.forward(mid, np.array([0.9, -0.2, 0.1]), th)
        gen = torch.Generator(device="cpu").manual_seed(3)
        noise = torch.randn(p_true.shape, generator=gen).cuda()
        y = (p_true * (1.0 + 0.01 * noise)).contiguous()
        # projections of f and h_k at the evaluation point
        w = np.array([0.4, -0.3, 0.2])
        f, h = ctx.warp(mid, w)
        p = ctx.project(vol, geom, th, f).contiguous()
        q = torch.stack([ctx.project(vol, geom, th, h[k].contiguous()) for k in range(K)]).contiguous()
        torch.cuda.synchronize()
        for a, b in ((1.02, -0.01), (0.97, 0.03)):
            out = torch.full((1 + K,), float("nan"), dtype=torch.float64, device="cuda")
            capi.pr_cost_grad_static(0, ctx.stream.cuda_stream, p, q, y, R, K, a, b, out)
            ctx.stream.synchronize()
            J, g = out[0].item(), out[1:].cpu().numpy()
            J_ref, g_ref = ctx.cost_grad(mid, y, th, w, a, b, mode=0)
            assert abs(J - J_ref) / J_ref < TOL_PROJ
            assert rel(g, g_ref) < TOL_GRAD
        # sizes beyond the scratch are rejected with a clear error
        with pytest.raises(PcaReconError) as e:
            capi.pr_cost_grad_static(0, ctx.stream.cuda_stream, p, q, y, R, 8, 1.0, 0.0, out)
        assert e.value.code == -1 and "K must be 1..7" in str(e.value)
    finally:
        ctx.close()


@pytest.mark.parametrize("R, K", [(20011, 7), (1, 7), (1, 1), (37, 3)])
def test_static_cost_grad_limits_against_float64_sums(R, K):
    """At the header's limits: K = 7 fills every per-block sum slot, and with
    R = 1 nearly all of the reduction's blocks publish empty rows. Seeded
    synthetic p, q, y (no model needed), two calls in a row, each against
    float64 sums, and the out_dev entries past 1 + K keep a sentinel."""
    import torch

    from paper_1004_0014_b300 import capi

    gen = torch.Generator(device="cpu").manual_seed(1000 * K + R)
    p = (1.0 + torch.rand(R, generator=gen, dtype=torch.float32)).cuda()
    q = torch.randn((K, R), generator=gen, dtype=torch.float32).cuda()
    y = (1.0 + torch.rand(R, generator=gen, dtype=torch.float32)).cuda()
    stream = torch.cuda.Stream()
    for a, b in ((0.9, 0.05), (1.1, -0.02)):
        out = torch.full((1 + K + 3,), -7.25, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        capi.pr_cost_grad_static(0, stream.cuda_stream, p, q, y, R, K, a, b, out)
        stream.synchronize()
        r = p.double() - a * y.double() - b
        J_ref = float(torch.sum(r * r))
        g_ref = (2.0 * (q.double() * r[None, :]).sum(dim=1)).cpu().numpy()
        o = out.cpu().numpy()
        assert abs(o[0] - J_ref) / J_ref < TOL_PROJ
        assert rel(o[1:1 + K], g_ref) < TOL_GRAD
        assert np.all(o[1 + K:] == -7.25)
