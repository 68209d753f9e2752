"""ctypes binding of the pcarecon C ABI (include/pcarecon.h).

Argument marshalling only: every function here forwards to the function of
the same name in libpcarecon.so, which does all the work in CUDA kernels.
Device buffers are torch CUDA tensors (passed by data_ptr()); host buffers are
numpy arrays or CPU tensors. There is no fallback: if the library is missing
or a call fails, an exception is raised.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PR_OK = 0
PR_EINVAL = -1
PR_ENOMEM = -2
PR_EADMIT = -3
PR_ECUDA = -4
PR_ETIMEOUT = -5
PR_ENOMODEL = -6
PR_EUNSUPPORTED = -7

PR_STOP_GRAD_TOL = 1
PR_STOP_MAX_ITERS = 2
PR_STOP_LINESEARCH_FAILED = 3
PR_STOP_NONFINITE = 4
PR_STOP_SINGULAR_FIT = 5
PR_STOP_RESOLVED = 7

PR_MAX_K = 7
PR_HOST, PR_DEVICE = 0, 1
PR_F32, PR_BF16 = 0, 1
PR_LOOP_GRAPH, PR_LOOP_HOST = 0, 1

EXPORTED = [
    "pr_version", "pr_last_error", "pr_default_opts", "pr_create", "pr_destroy", "pr_load_model",
    "pr_release_model", "pr_model_footprint", "pr_reconstruct", "pr_reconstruct_batch", "pr_reconstruct_async",
    "pr_fetch_result", "pr_get_state", "pr_set_state", "pr_warp", "pr_project", "pr_backproject",
    "pr_forward", "pr_vjp", "pr_cost_grad", "pr_tumor", "pr_invert_dvf", "pr_trial_log", "pr_fix_angle",
    "pr_count_samples", "pr_warp_box", "pr_time_kernel", "pr_model_stats",
    "pr_io_bytes", "pr_cost_grad_static", "pr_serve_start", "pr_submit", "pr_poll", "pr_serve_stop",
    "pr_serve_start_batched", "pr_set_admission_queue", "pr_model_status",
]

PR_QUEUED = 1
PR_MODEL_RESIDENT, PR_MODEL_WAITING = 0, 1

PR_KERNEL_WARP_FH, PR_KERNEL_PROJECT_FH, PR_KERNEL_REGRAD = 0, 1, 2
PR_KERNEL_BACKPROJECT, PR_KERNEL_WARP_F, PR_KERNEL_PROJECT_F, PR_KERNEL_INVERT = 3, 4, 5, 6
PR_KERNEL_PROJECT_FH_TRIAL = 7


class Stats(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_longlong), ("trials", ctypes.c_longlong), ("kernels", ctypes.c_longlong),
                ("iters", ctypes.c_longlong), ("line_search_failures", ctypes.c_longlong)]


class PcaReconError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pcarecon error %d: %s" % (code, msg))
        self.code = code


class VolumeDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class Geometry(ctypes.Structure):
    _fields_ = [("sad", ctypes.c_double), ("sdd", ctypes.c_double), ("nu", ctypes.c_int),
                ("nv", ctypes.c_int), ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("ds", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("grad_tol", ctypes.c_double), ("c1", ctypes.c_double),
                ("beta", ctypes.c_double), ("max_backtracks", ctypes.c_int),
                ("step0_mm", ctypes.c_double), ("cold_start", ctypes.c_int),
                ("w0", ctypes.c_double * PR_MAX_K), ("loop_mode", ctypes.c_int),
                ("tumor_tol", ctypes.c_double), ("tumor_max_iter", ctypes.c_int),
                ("step_growth", ctypes.c_double), ("step_growth_bt", ctypes.c_double),
                ("warm_step", ctypes.c_int), ("predict", ctypes.c_int), ("step_model", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("w", ctypes.c_double * PR_MAX_K), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("J", ctypes.c_double), ("grad", ctypes.c_double * PR_MAX_K),
                ("grad_norm", ctypes.c_double), ("grad_norm0", ctypes.c_double),
                ("iters", ctypes.c_int), ("trials", ctypes.c_int), ("backtracks", ctypes.c_int),
                ("stop_reason", ctypes.c_int), ("tumor_xyz", ctypes.c_double * 3),
                ("tumor_steps", ctypes.c_int), ("mu", ctypes.c_double)]

    def as_dict(self):
        K = self.K
        return dict(w=np.array(self.w[:K]), a=self.a, b=self.b, J=self.J,
                    grad=np.array(self.grad[:K]), grad_norm=self.grad_norm,
                    grad_norm0=self.grad_norm0, iters=self.iters, trials=self.trials,
                    backtracks=self.backtracks, stop_reason=self.stop_reason,
                    tumor=np.array(self.tumor_xyz[:]), tumor_steps=self.tumor_steps, mu=self.mu)


class Served(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("model_id", ctypes.c_int), ("status", ctypes.c_int),
                ("result", Result), ("queue_ms", ctypes.c_double), ("gpu_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        d = self.result.as_dict()
        d.update(tag=self.tag, model_id=self.model_id, status=self.status, queue_ms=self.queue_ms,
                 gpu_ms=self.gpu_ms, latency_ms=self.latency_ms)
        return d


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)


def load_library(path: str | None = None):
    """Load libpcarecon.so (built in-tree by paper_1004_0014_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libpcarecon.so not found at %s: run `python -m paper_1004_0014_b300.build`"
                           % path)
    lib = ctypes.CDLL(path)
    sig = {
        "pr_version": (ctypes.c_char_p, []),
        "pr_last_error": (ctypes.c_char_p, []),
        "pr_default_opts": (None, [ctypes.POINTER(SolveOpts)]),
        "pr_create": (_I, [ctypes.POINTER(_P), _I, _P, ctypes.c_size_t]),
        "pr_destroy": (None, [_P]),
        "pr_load_model": (_I, [_P, ctypes.POINTER(VolumeDesc), ctypes.POINTER(Geometry), _I, _P, _P, _P,
                               _I, _I, _DP, ctypes.POINTER(_I)]),
        "pr_release_model": (_I, [_P, _I]),
        "pr_model_footprint": (_I, [_P, _I, ctypes.POINTER(ctypes.c_size_t)]),
        "pr_reconstruct": (_I, [_P, _I, _P, _I, _D, ctypes.POINTER(SolveOpts), ctypes.POINTER(Result), _P]),
        "pr_reconstruct_async": (_I, [_P, _I, _P, _D, ctypes.POINTER(SolveOpts)]),
        "pr_reconstruct_batch": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_P), _DP, ctypes.POINTER(SolveOpts),
                                      ctypes.POINTER(Result)]),
        "pr_fetch_result": (_I, [_P, _I, ctypes.POINTER(Result)]),
        "pr_get_state": (_I, [_P, _I, _DP]),
        "pr_set_state": (_I, [_P, _I, _DP]),
        "pr_warp": (_I, [_P, _I, _DP, _P, _P]),
        "pr_project": (_I, [_P, ctypes.POINTER(VolumeDesc), ctypes.POINTER(Geometry), _D, _P, _P]),
        "pr_backproject": (_I, [_P, ctypes.POINTER(VolumeDesc), ctypes.POINTER(Geometry), _D, _P, _P]),
        "pr_forward": (_I, [_P, _I, _DP, _D, _P]),
        "pr_vjp": (_I, [_P, _I, _DP, _D, _P, _DP]),
        "pr_cost_grad": (_I, [_P, _I, _P, _D, _DP, _D, _D, _I, _DP, _DP, _P]),
        "pr_tumor": (_I, [_P, _I, _DP, _D, _I, _DP, ctypes.POINTER(_I)]),
        "pr_invert_dvf": (_I, [_P, _I, _DP, _D, _I, _P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong)]),
        "pr_trial_log": (_I, [_P, _I, _P, _I, ctypes.POINTER(_I)]),
        "pr_fix_angle": (_I, [_P, _I, _D, ctypes.POINTER(ctypes.c_size_t)]),
        "pr_count_samples": (_I, [_P, _I, _D, _DP, ctypes.POINTER(ctypes.c_longlong)]),
        "pr_warp_box": (_I, [_P, _I, _DP, ctypes.POINTER(ctypes.c_int)]),
        "pr_time_kernel": (_I, [_P, _I, _I, _D, _I, _DP]),
        "pr_model_stats": (_I, [_P, _I, ctypes.POINTER(Stats)]),
        "pr_io_bytes": (_I, [_P, _I, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
        "pr_cost_grad_static": (_I, [_I, _P, _P, _P, _P, _I, _I, _D, _D, _P]),
        "pr_serve_start": (_I, [_P, _I]),
        "pr_serve_start_batched": (_I, [_P, _I, _I]),
        "pr_set_admission_queue": (_I, [_P, _I]),
        "pr_model_status": (_I, [_P, _I, ctypes.POINTER(_I)]),
        "pr_submit": (_I, [_P, _I, _P, _D, ctypes.POINTER(SolveOpts), ctypes.c_uint64]),
        "pr_poll": (_I, [_P, _I, ctypes.POINTER(Served)]),
        "pr_serve_stop": (_I, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != PR_OK:
        raise PcaReconError(rc, _lib.pr_last_error().decode())
    return rc


def _dvec(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(_DP)


def _ptr(x):
    """(pointer, location) of a torch tensor or numpy array."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), (PR_DEVICE if x.is_cuda else PR_HOST)
    if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data), PR_HOST


def _f32(x):
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float32:
            raise TypeError("expected float32")
        return x.contiguous()
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def _dev(x, what):
    if not (hasattr(x, "data_ptr") and x.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % what)
    return ctypes.c_void_p(x.data_ptr())


# ---------------------------------------------------------------------------
# Functions with the C names
# ---------------------------------------------------------------------------


def pr_version() -> str:
    return load_library().pr_version().decode()


def pr_last_error() -> str:
    return load_library().pr_last_error().decode()


def pr_default_opts(**overrides) -> SolveOpts:
    o = SolveOpts()
    load_library().pr_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "w0":
            for i, x in enumerate(v):
                o.w0[i] = float(x)
        else:
            setattr(o, k, v)
    return o


def pr_create(device: int = 0, stream=None, hbm_budget_bytes: int = 0):
    lib = load_library()
    ctx = ctypes.c_void_p()
    # A zero handle is the legacy default stream; pass it through as such.
    s = ctypes.c_void_p(stream) if stream else None
    _check(lib.pr_create(ctypes.byref(ctx), int(device), s, int(hbm_budget_bytes)))
    return ctx


def pr_destroy(ctx):
    load_library().pr_destroy(ctx)


def pr_load_model(ctx, vol: VolumeDesc, geom: Geometry, f0, mean_dvf, U, K: int, storage: int,
                  tumor_ref_xyz) -> int:
    f0, mean_dvf, U = _f32(f0), _f32(mean_dvf), _f32(U)
    pf, lf = _ptr(f0)
    pm, lm = _ptr(mean_dvf)
    pu, lu = _ptr(U)
    if not (lf == lm == lu):
        raise ValueError("f0, mean_dvf and U must all be on the host or all on the device")
    c0, pc = _dvec(tumor_ref_xyz)
    mid = ctypes.c_int()
    rc = _lib.pr_load_model(ctx, ctypes.byref(vol), ctypes.byref(geom), lf, pf, pm, pu, int(K), int(storage), pc,
                            ctypes.byref(mid))
    if rc != PR_QUEUED:  # queued for admission: a handle, not an error
        _check(rc)
    return mid.value


def pr_set_admission_queue(ctx, enable: bool):
    _check(_lib.pr_set_admission_queue(ctx, 1 if enable else 0))


def pr_model_status(ctx, model_id: int) -> int:
    st = _I()
    _check(_lib.pr_model_status(ctx, int(model_id), ctypes.byref(st)))
    return st.value


def pr_release_model(ctx, model_id: int):
    _check(_lib.pr_release_model(ctx, int(model_id)))


def pr_model_footprint(ctx, model_id: int) -> int:
    b = ctypes.c_size_t()
    _check(_lib.pr_model_footprint(ctx, int(model_id), ctypes.byref(b)))
    return b.value


def pr_reconstruct(ctx, model_id: int, y, angle_rad: float, opts: SolveOpts | None = None,
                   volume_out=None) -> Result:
    y = _f32(y)
    py, ly = _ptr(y)
    res = Result()
    vo = None
    if volume_out is not None:
        vo, lv = _ptr(volume_out)
        if lv != PR_HOST:
            raise ValueError("volume_out must be host memory")
    _check(_lib.pr_reconstruct(ctx, int(model_id), py, ly, float(angle_rad),
                               ctypes.byref(opts) if opts is not None else None, ctypes.byref(res), vo))
    return res


def pr_reconstruct_batch(ctx, model_ids, ys, angles, opts: SolveOpts | None = None):
    """Solves n frames (host arrays) in one graph launch; returns n Results."""
    n = len(model_ids)
    if not (len(ys) == len(angles) == n):
        raise ValueError("model_ids, ys and angles must have the same length")
    arrs = [_f32(y) for y in ys]
    ids = (_I * n)(*[int(i) for i in model_ids])
    ptrs = (_P * n)(*[a.ctypes.data for a in arrs])
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    out = (Result * n)()
    _check(_lib.pr_reconstruct_batch(ctx, n, ids, ptrs, ang.ctypes.data_as(_DP),
                                     ctypes.byref(opts) if opts is not None else None, out))
    return list(out)


def pr_reconstruct_async(ctx, model_id: int, y_dev, angle_rad: float, opts: SolveOpts | None = None):
    _check(_lib.pr_reconstruct_async(ctx, int(model_id), _dev(y_dev, "y_dev"), float(angle_rad),
                                     ctypes.byref(opts) if opts is not None else None))


def pr_fetch_result(ctx, model_id: int) -> Result:
    res = Result()
    _check(_lib.pr_fetch_result(ctx, int(model_id), ctypes.byref(res)))
    return res


def pr_get_state(ctx, model_id: int, K: int) -> np.ndarray:
    w = np.zeros(K)
    _check(_lib.pr_get_state(ctx, int(model_id), w.ctypes.data_as(_DP)))
    return w


def pr_set_state(ctx, model_id: int, w):
    w, pw = _dvec(w)
    _check(_lib.pr_set_state(ctx, int(model_id), pw))


def pr_warp(ctx, model_id: int, w, f_dev=None, h_dev=None):
    w, pw = _dvec(w)
    _check(_lib.pr_warp(ctx, int(model_id), pw, _dev(f_dev, "f_dev") if f_dev is not None else None,
                        _dev(h_dev, "h_dev") if h_dev is not None else None))


def pr_project(ctx, vol: VolumeDesc, geom: Geometry, angle_rad: float, f_dev, p_dev):
    _check(_lib.pr_project(ctx, ctypes.byref(vol), ctypes.byref(geom), float(angle_rad),
                           _dev(f_dev, "f_dev"), _dev(p_dev, "p_dev")))


def pr_backproject(ctx, vol: VolumeDesc, geom: Geometry, angle_rad: float, r_dev, g_dev):
    _check(_lib.pr_backproject(ctx, ctypes.byref(vol), ctypes.byref(geom), float(angle_rad),
                               _dev(r_dev, "r_dev"), _dev(g_dev, "g_dev")))


def pr_forward(ctx, model_id: int, w, angle_rad: float, p_dev):
    w, pw = _dvec(w)
    _check(_lib.pr_forward(ctx, int(model_id), pw, float(angle_rad), _dev(p_dev, "p_dev")))


def pr_vjp(ctx, model_id: int, w, angle_rad: float, grad_p_dev, K: int) -> np.ndarray:
    w, pw = _dvec(w)
    out = np.zeros(K)
    _check(_lib.pr_vjp(ctx, int(model_id), pw, float(angle_rad), _dev(grad_p_dev, "grad_p_dev"),
                       out.ctypes.data_as(_DP)))
    return out


def pr_cost_grad(ctx, model_id: int, y_dev, angle_rad: float, w, a: float, b: float, mode: int,
                 K: int, p_dev=None):
    w, pw = _dvec(w)
    J = ctypes.c_double()
    g = np.zeros(K)
    _check(_lib.pr_cost_grad(ctx, int(model_id), _dev(y_dev, "y_dev"), float(angle_rad), pw, float(a),
                             float(b), int(mode), ctypes.byref(J), g.ctypes.data_as(_DP),
                             _dev(p_dev, "p_dev") if p_dev is not None else None))
    return J.value, g


def pr_tumor(ctx, model_id: int, w, tol: float = 1e-6, max_iter: int = 100):
    w, pw = _dvec(w)
    xyz = np.zeros(3)
    steps = ctypes.c_int()
    _check(_lib.pr_tumor(ctx, int(model_id), pw, float(tol), int(max_iter), xyz.ctypes.data_as(_DP),
                         ctypes.byref(steps)))
    return xyz, steps.value


def pr_invert_dvf(ctx, model_id: int, w, y_dev, tol: float = 1e-5, max_iter: int = 64):
    """Fills y_dev [3][nz][ny][nx] (device float32, mm); returns (max steps, unconverged voxels)."""
    w, pw = _dvec(w)
    steps = ctypes.c_int()
    open_ = ctypes.c_longlong()
    _check(_lib.pr_invert_dvf(ctx, int(model_id), pw, float(tol), int(max_iter), _dev(y_dev, "y_dev"),
                              ctypes.byref(steps), ctypes.byref(open_)))
    return steps.value, open_.value


def pr_count_samples(ctx, model_id: int, angle_rad: float, w) -> int:
    w, pw = _dvec(w)
    n = ctypes.c_longlong()
    _check(_lib.pr_count_samples(ctx, int(model_id), float(angle_rad), pw, ctypes.byref(n)))
    return n.value


def pr_warp_box(ctx, model_id: int, w):
    """((x0, y0, z0), (x1, y1, z1)): inclusive voxel box the solver's warp evaluates at w."""
    w, pw = _dvec(w)
    box = (ctypes.c_int * 6)()
    _check(_lib.pr_warp_box(ctx, int(model_id), pw, box))
    return tuple(box[0:3]), tuple(box[3:6])


def pr_fix_angle(ctx, model_id: int, angle_rad: float) -> int:
    """Builds the fixed-angle transpose table (NaN drops it); returns its bytes."""
    nb = ctypes.c_size_t()
    _check(_lib.pr_fix_angle(ctx, int(model_id), float(angle_rad), ctypes.byref(nb)))
    return nb.value


def pr_trial_log(ctx, model_id: int):
    """The last solve's trial choices as a list of (accepted, stop, e)."""
    buf = (ctypes.c_ubyte * 1024)()
    n = ctypes.c_int()
    _check(_lib.pr_trial_log(ctx, int(model_id), ctypes.cast(buf, _P), 1024, ctypes.byref(n)))
    return [(bool(b & 0x80), bool(b & 0x40), (b & 0x3F) - 32) for b in buf[:min(n.value, 1024)]]


def pr_time_kernel(ctx, model_id: int, which: int, angle_rad: float, iters: int) -> float:
    ms = ctypes.c_double()
    _check(_lib.pr_time_kernel(ctx, int(model_id), int(which), float(angle_rad), int(iters), ctypes.byref(ms)))
    return ms.value


def pr_model_stats(ctx, model_id: int) -> dict:
    st = Stats()
    _check(_lib.pr_model_stats(ctx, int(model_id), ctypes.byref(st)))
    return dict(solves=st.solves, trials=st.trials, kernels=st.kernels, iters=st.iters,
                line_search_failures=st.line_search_failures)


def pr_io_bytes(ctx, model_id: int):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.pr_io_bytes(ctx, int(model_id), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def pr_cost_grad_static(device: int, stream, p_dev, q_dev, y_dev, R: int, K: int, a: float, b: float, out_dev):
    """Allocation-free cost and gradient from projections (see include/pcarecon.h).
    stream: a cudaStream_t handle (int) or None; all buffers are CUDA tensors."""
    load_library()
    s = ctypes.c_void_p(stream) if stream else None
    _check(_lib.pr_cost_grad_static(int(device), s, _dev(p_dev, "p_dev"), _dev(q_dev, "q_dev"),
                                    _dev(y_dev, "y_dev"), int(R), int(K), float(a), float(b),
                                    _dev(out_dev, "out_dev")))


def pr_serve_start(ctx, slots: int = 4):
    _check(_lib.pr_serve_start(ctx, int(slots)))


def pr_serve_start_batched(ctx, lanes: int = 2, tick_frames: int = 0):
    _check(_lib.pr_serve_start_batched(ctx, int(lanes), int(tick_frames)))


def pr_submit(ctx, model_id: int, y, angle_rad: float, opts: SolveOpts | None = None, tag: int = 0):
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float32))
    _check(_lib.pr_submit(ctx, int(model_id), ctypes.c_void_p(y.ctypes.data), float(angle_rad),
                          ctypes.byref(opts) if opts is not None else None, ctypes.c_uint64(tag)))


def pr_poll(ctx, timeout_ms: int = -1):
    """Next finished frame as a dict, or None on timeout."""
    out = Served()
    rc = _lib.pr_poll(ctx, int(timeout_ms), ctypes.byref(out))
    if rc == PR_ETIMEOUT:
        return None
    _check(rc)
    return out.as_dict()


def pr_serve_stop(ctx):
    _check(_lib.pr_serve_stop(ctx))
