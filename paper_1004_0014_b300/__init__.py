"""pcarecon: single-projection volumetric reconstruction and tumor localisation
with a PCA lung-motion model (Li et al.), as a C-ABI CUDA library for B300
(sm_103a) with a thin Python binding.

    from paper_1004_0014_b300 import Context
    ctx = Context(device=0)
    mid = ctx.load_model(vol, geom, f0, mean_dvf, U, tumor_ref_xyz)
    res = ctx.reconstruct(mid, y, angle_rad)

Device memory and streams come from PyTorch; every step of the method runs in
the library's CUDA kernels. There is no CPU fallback.
"""

from __future__ import annotations

import numpy as np

from . import capi
from .capi import (  # noqa: F401
    PR_BF16, PR_DEVICE, PR_F32, PR_HOST, PR_LOOP_GRAPH, PR_LOOP_HOST, PR_MAX_K,
    PR_STOP_GRAD_TOL, PR_STOP_LINESEARCH_FAILED, PR_STOP_MAX_ITERS, PR_STOP_NONFINITE,
    PR_STOP_RESOLVED, PR_STOP_SINGULAR_FIT, Geometry, PcaReconError, Result, SolveOpts, VolumeDesc,
)


def volume_desc(vol) -> VolumeDesc:
    """VolumeDesc from any object with nx, ny, nz, dx, dy, dz."""
    return VolumeDesc(int(vol.nx), int(vol.ny), int(vol.nz), float(vol.dx), float(vol.dy), float(vol.dz))


def geometry(geom) -> Geometry:
    """Geometry from any object with sad, sdd, nu, nv, du, dv, ds."""
    return Geometry(float(geom.sad), float(geom.sdd), int(geom.nu), int(geom.nv), float(geom.du),
                    float(geom.dv), float(geom.ds))


class Context:
    """One pcarecon context on one CUDA device (wraps pr_create / pr_destroy)."""

    def __init__(self, device: int = 0, stream=None, hbm_budget_bytes: int = 0):
        """stream: a torch.cuda.Stream to run on (default: a new one). All of
        the context's device work is ordered on it; time it with events
        recorded on `self.stream`."""
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("pcarecon needs a CUDA device")
        self.device = device
        if stream is None:
            stream = torch.cuda.Stream(device=device)
        self.stream = stream
        self._ctx = capi.pr_create(device, stream.cuda_stream, hbm_budget_bytes)
        self._models = {}

    def close(self):
        if getattr(self, "_ctx", None):
            capi.pr_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- models -----------------------------------------------------------
    def load_model(self, vol, geom, f0, mean_dvf, U, tumor_ref_xyz, storage: int = PR_F32) -> int:
        U = np.asarray(U, dtype=np.float32) if not hasattr(U, "data_ptr") else U
        K = int(U.shape[0])
        vd, gd = volume_desc(vol), geometry(geom)
        mid = capi.pr_load_model(self._ctx, vd, gd, f0, mean_dvf, U, K, storage, tumor_ref_xyz)
        self._models[mid] = dict(K=K, vol=vd, geom=gd)
        return mid

    def release_model(self, mid: int):
        capi.pr_release_model(self._ctx, mid)
        self._models.pop(mid, None)

    def footprint(self, mid: int) -> int:
        return capi.pr_model_footprint(self._ctx, mid)

    def K(self, mid: int) -> int:
        return self._models[mid]["K"]

    # --- solves -----------------------------------------------------------
    def reconstruct(self, mid: int, y, angle_rad: float, opts: SolveOpts | None = None,
                    volume: bool = False):
        vo = None
        if volume:
            v = self._models[mid]["vol"]
            vo = np.empty((v.nz, v.ny, v.nx), dtype=np.float32)
        res = capi.pr_reconstruct(self._ctx, mid, y, angle_rad, opts, vo).as_dict()
        if volume:
            res["volume"] = vo
        return res

    def reconstruct_batch(self, mids, ys, angles, opts: SolveOpts | None = None):
        """Solves frame i of model mids[i] for every i in one graph launch
        (host ys); results as dicts, in order."""
        return [r.as_dict() for r in capi.pr_reconstruct_batch(self._ctx, mids, ys, angles, opts)]

    def reconstruct_async(self, mid: int, y_dev, angle_rad: float, opts: SolveOpts | None = None):
        capi.pr_reconstruct_async(self._ctx, mid, y_dev, angle_rad, opts)

    def fetch_result(self, mid: int):
        return capi.pr_fetch_result(self._ctx, mid).as_dict()

    def get_state(self, mid: int) -> np.ndarray:
        return capi.pr_get_state(self._ctx, mid, self.K(mid))

    def set_state(self, mid: int, w):
        capi.pr_set_state(self._ctx, mid, w)

    # --- step-level operators ----------------------------------------------
    def warp(self, mid: int, w, with_h: bool = True):
        import torch

        v = self._models[mid]["vol"]
        f = torch.empty((v.nz, v.ny, v.nx), dtype=torch.float32, device="cuda:%d" % self.device)
        h = None
        if with_h:
            h = torch.empty((self.K(mid), v.nz, v.ny, v.nx), dtype=torch.float32, device=f.device)
        capi.pr_warp(self._ctx, mid, w, f, h)
        return f, h

    def project(self, vol, geom, angle_rad: float, f_dev):
        import torch

        gd = geometry(geom)
        p = torch.empty((gd.nv, gd.nu), dtype=torch.float32, device=f_dev.device)
        capi.pr_project(self._ctx, volume_desc(vol), gd, angle_rad, f_dev.contiguous(), p)
        return p

    def backproject(self, vol, geom, angle_rad: float, r_dev):
        import torch

        vd = volume_desc(vol)
        g = torch.empty((vd.nz, vd.ny, vd.nx), dtype=torch.float32, device=r_dev.device)
        capi.pr_backproject(self._ctx, vd, geometry(geom), angle_rad, r_dev.contiguous(), g)
        return g

    def forward(self, mid: int, w, angle_rad: float):
        import torch

        gd = self._models[mid]["geom"]
        p = torch.empty((gd.nv, gd.nu), dtype=torch.float32, device="cuda:%d" % self.device)
        capi.pr_forward(self._ctx, mid, w, angle_rad, p)
        return p

    def vjp(self, mid: int, w, angle_rad: float, grad_p):
        return capi.pr_vjp(self._ctx, mid, w, angle_rad, grad_p.contiguous(), self.K(mid))

    def cost_grad(self, mid: int, y_dev, angle_rad: float, w, a: float, b: float, mode: int = 0,
                  return_p: bool = False):
        import torch

        p = None
        if return_p:
            gd = self._models[mid]["geom"]
            p = torch.empty((gd.nv, gd.nu), dtype=torch.float32, device=y_dev.device)
        J, g = capi.pr_cost_grad(self._ctx, mid, y_dev.contiguous(), angle_rad, w, a, b, mode,
                                 self.K(mid), p)
        return (J, g, p) if return_p else (J, g)

    def tumor(self, mid: int, w, tol: float = 1e-6, max_iter: int = 100):
        return capi.pr_tumor(self._ctx, mid, w, tol, max_iter)

    def count_samples(self, mid: int, angle_rad: float, w) -> int:
        """Ray samples the solver-pass projector evaluates at this angle and w."""
        return capi.pr_count_samples(self._ctx, mid, angle_rad, w)

    def warp_box(self, mid: int, w):
        """Inclusive voxel box ((x0, y0, z0), (x1, y1, z1)) the solver's warp evaluates at w."""
        return capi.pr_warp_box(self._ctx, mid, w)

    def fix_angle(self, mid: int, angle_rad: float) -> int:
        """Fixed-angle transpose table for the model at this angle (NaN drops it)."""
        return capi.pr_fix_angle(self._ctx, mid, angle_rad)

    def trial_log(self, mid: int):
        """The last solve's line-search choices: (accepted, stop, e) per trial."""
        return capi.pr_trial_log(self._ctx, mid)

    def invert_dvf(self, mid: int, w, tol: float = 1e-5, max_iter: int = 64):
        """Push-forward DVF (3, nz, ny, nx) float32 mm on the device, the largest
        per-voxel step count and the number of voxels not converged to tol."""
        import torch

        vol = self._models[mid]["vol"]
        y = torch.empty((3, vol.nz, vol.ny, vol.nx), dtype=torch.float32, device="cuda:%d" % self.device)
        steps, open_ = capi.pr_invert_dvf(self._ctx, mid, w, y, tol, max_iter)
        return y, steps, open_

    # --- serving -------------------------------------------------------------
    def serve_start(self, slots: int = 4, batched_lanes: int = 0, tick_frames: int = 0):
        """Slot mode (`slots` concurrent solve streams) or, with batched_lanes
        > 0, tick-batched mode (one graph launch per tick over the models'
        pending frames, at most tick_frames of them (0 = all), that many ticks
        in flight)."""
        if batched_lanes:
            capi.pr_serve_start_batched(self._ctx, batched_lanes, tick_frames)
        else:
            capi.pr_serve_start(self._ctx, slots)

    def set_admission_queue(self, enable: bool = True):
        capi.pr_set_admission_queue(self._ctx, enable)

    def model_status(self, mid: int) -> int:
        return capi.pr_model_status(self._ctx, mid)

    def submit(self, mid: int, y, angle_rad: float, opts: SolveOpts | None = None, tag: int = 0):
        capi.pr_submit(self._ctx, mid, y, angle_rad, opts, tag)

    def poll(self, timeout_ms: int = -1):
        return capi.pr_poll(self._ctx, timeout_ms)

    def serve_stop(self):
        capi.pr_serve_stop(self._ctx)

    # --- measurement -------------------------------------------------------
    def time_kernel(self, mid: int, which: int, angle_rad: float = 0.0, iters: int = 20) -> float:
        return capi.pr_time_kernel(self._ctx, mid, which, angle_rad, iters)

    def stats(self, mid: int) -> dict:
        return capi.pr_model_stats(self._ctx, mid)

    def io_bytes(self, mid: int):
        return capi.pr_io_bytes(self._ctx, mid)


def default_opts(**overrides) -> SolveOpts:
    return capi.pr_default_opts(**overrides)
