"""GB300-native TNLM 4DCT reconstruction (arXiv:1009.1351).

Thin Python binding of the C ABI declared in include/tnlm.h.  Every function
here only marshals arguments (torch CUDA tensors or raw device pointers,
the CUDA stream) and calls the library of the same name; all computation
runs in the library's CUDA kernels.  There is no CPU fallback: if the
library has not been built (``python -c "import __graft_entry__ as g;
g.build()"``) or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Any, Dict, List, Optional, Tuple

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libtnlm.so")

TNLM_OK = 0
TNLM_ERR_INVALID_ARG = 1
TNLM_ERR_OOM = 2
TNLM_ERR_CUDA = 3
TNLM_ERR_NUMERIC = 4
TNLM_ERR_TIMEOUT = 5
TNLM_DETECTOR_ARC = 0
TNLM_DATA_CGLS = 0
TNLM_DATA_GRAD = 1

EXPORTED = ("tnlm_create_geometry", "tnlm_destroy_geometry", "tnlm_project", "tnlm_backproject",
            "tnlm_weights_size", "tnlm_weights", "tnlm_workspace_bytes", "tnlm_reconstruct",
            "tnlm_last_error", "tnlm_debug_fail_alloc_after", "tnlm_debug_wait_limit", "tnlm_profile_enable",
            "tnlm_profile_read", "tnlm_project_static", "tnlm_fbp", "tnlm_autotune",
            "tnlm_reconstruct_batch", "tnlm_batch_last_was_loop", "tnlm_fbp_phases", "tnlm_unet_create", "tnlm_unet_destroy", "tnlm_unet_param_count",
            "tnlm_unet_set_params", "tnlm_unet_get_params", "tnlm_unet_forward", "tnlm_unet_grads",
            "tnlm_unet_adam_step", "tnlm_unet_last_error", "tnlm_measure_peaks")
KCLASSES = ("prep", "project", "backproject", "cgls", "weights", "gj")
PREC_FP32, PREC_MIXED = 0, 1


class GeometryDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pixel_mm", ctypes.c_double),
                ("n_phases", ctypes.c_int), ("n_views", ctypes.c_int), ("n_bins", ctypes.c_int),
                ("bin_mm", ctypes.c_double), ("sid_mm", ctypes.c_double),
                ("sdd_mm", ctypes.c_double), ("detector", ctypes.c_int),
                ("view_angles_rad", ctypes.POINTER(ctypes.c_double)), ("device", ctypes.c_int)]


class ParamsC(ctypes.Structure):
    _fields_ = [("mu_hat", ctypes.c_double), ("h", ctypes.c_double), ("beta", ctypes.c_double),
                ("patch", ctypes.c_int), ("window", ctypes.c_int), ("m1", ctypes.c_int),
                ("m2", ctypes.c_int), ("k_outer", ctypes.c_int), ("data_step", ctypes.c_int),
                ("clamp", ctypes.c_int), ("tol", ctypes.c_double),
                ("tol_check_every", ctypes.c_int), ("precision", ctypes.c_int),
                ("monitor", ctypes.c_int), ("recompute", ctypes.c_int)]


class ReportC(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_change", ctypes.c_double),
                ("data_residual", ctypes.c_double),
                ("rel_change_hist", ctypes.POINTER(ctypes.c_double)),
                ("residual_hist", ctypes.POINTER(ctypes.c_double)),
                ("clamped", ctypes.c_longlong),
                ("clamped_hist", ctypes.POINTER(ctypes.c_longlong)),
                ("tnlm_term", ctypes.c_double), ("objective", ctypes.c_double),
                ("tnlm_hist", ctypes.POINTER(ctypes.c_double)),
                ("data_hist", ctypes.POINTER(ctypes.c_double)),
                ("objective_hist", ctypes.POINTER(ctypes.c_double))]


def _new_report(k_outer: int):
    """A ReportC with history arrays for k_outer iterations (kept alive by the tuple)."""
    k = max(int(k_outer), 1)
    arrs = [(ctypes.c_double * k)() for _ in range(5)] + [(ctypes.c_longlong * k)()]
    rep = ReportC(0, 0.0, 0.0, arrs[0], arrs[1], 0, arrs[5], 0.0, 0.0, arrs[2], arrs[3], arrs[4])
    return rep, arrs


def _report_dict(rep, arrs, monitor: bool):
    n = rep.iterations
    out = {"iterations": n, "rel_change": rep.rel_change, "data_residual": rep.data_residual,
           "rel_change_hist": list(arrs[0][:n]), "residual_hist": list(arrs[1][:n]),
           "clamped": int(rep.clamped), "clamped_hist": [int(v) for v in arrs[5][:n]]}
    if monitor:
        out.update({"tnlm_term": rep.tnlm_term, "objective": rep.objective,
                    "tnlm_hist": list(arrs[2][:n]), "data_hist": list(arrs[3][:n]),
                    "objective_hist": list(arrs[4][:n])})
    return out


class TnlmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tnlm status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtnlm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.tnlm_create_geometry.argtypes = [ctypes.POINTER(GeometryDesc), ctypes.POINTER(vp)]
    lib.tnlm_destroy_geometry.argtypes = [vp]
    lib.tnlm_destroy_geometry.restype = None
    lib.tnlm_project.argtypes = [vp, vp, vp, vp]
    lib.tnlm_backproject.argtypes = [vp, vp, vp, vp]
    lib.tnlm_project_static.argtypes = [vp, vp, vp, vp]
    lib.tnlm_fbp.argtypes = [vp, vp, vp, vp]
    lib.tnlm_fbp_phases.argtypes = [vp, vp, vp, vp]
    lib.tnlm_weights_size.argtypes = [vp, ctypes.POINTER(ParamsC), ctypes.POINTER(ctypes.c_size_t),
                                      ctypes.POINTER(ctypes.c_size_t)]
    lib.tnlm_weights.argtypes = [vp, ctypes.POINTER(ParamsC), vp, vp, vp, vp]
    lib.tnlm_workspace_bytes.argtypes = [vp, ctypes.POINTER(ParamsC), ctypes.POINTER(ctypes.c_size_t)]
    lib.tnlm_reconstruct.argtypes = [vp, ctypes.POINTER(ParamsC), vp, vp, vp,
                                     ctypes.POINTER(ReportC), vp]
    lib.tnlm_autotune.argtypes = [vp, ctypes.POINTER(ParamsC), vp, vp, vp, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), vp]
    lib.tnlm_reconstruct_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ParamsC), ctypes.c_int,
                                           ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(ReportC), ctypes.c_int, vp]
    lib.tnlm_unet_create.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(vp)]
    lib.tnlm_unet_destroy.argtypes = [vp]
    lib.tnlm_unet_destroy.restype = None
    lib.tnlm_unet_param_count.argtypes = [vp]
    lib.tnlm_unet_param_count.restype = ctypes.c_longlong
    lib.tnlm_unet_set_params.argtypes = [vp, vp]
    lib.tnlm_unet_get_params.argtypes = [vp, vp, vp]
    lib.tnlm_unet_forward.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.tnlm_unet_grads.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), vp]
    lib.tnlm_unet_adam_step.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, vp]
    lib.tnlm_unet_last_error.restype = ctypes.c_char_p
    lib.tnlm_measure_peaks.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.tnlm_measure_peaks.restype = ctypes.c_int
    lib.tnlm_batch_last_was_loop.restype = ctypes.c_int
    lib.tnlm_last_error.restype = ctypes.c_char_p
    lib.tnlm_debug_fail_alloc_after.argtypes = [ctypes.c_int]
    lib.tnlm_debug_fail_alloc_after.restype = None
    lib.tnlm_debug_wait_limit.argtypes = [ctypes.c_long]
    lib.tnlm_debug_wait_limit.restype = None
    lib.tnlm_profile_enable.argtypes = [vp, ctypes.c_uint]
    lib.tnlm_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    for name in ("tnlm_create_geometry", "tnlm_project", "tnlm_project_static", "tnlm_fbp",
                 "tnlm_backproject",
                 "tnlm_weights_size",
                 "tnlm_weights", "tnlm_workspace_bytes", "tnlm_reconstruct", "tnlm_profile_enable",
                 "tnlm_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != TNLM_OK:
        msg = load_library().tnlm_last_error().decode(errors="replace")
        raise TnlmError(status, msg)


def _ptr(t: Any) -> Optional[int]:
    """Device pointer of a torch CUDA tensor (float32, contiguous) or a raw int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    import torch
    if t.dtype != torch.float32:
        raise ValueError("expected float32")
    return t.data_ptr()


def _stream(stream: Any) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def params_c(p: Any) -> ParamsC:
    """Marshal an object with the tnlm_params fields (e.g. synth.Params)."""
    return ParamsC(float(p.mu_hat), float(p.h), float(getattr(p, "beta", 0.0)), int(p.patch),
                   int(p.window), int(p.m1), int(p.m2), int(p.k_outer),
                   int(getattr(p, "data_step", 0)), int(getattr(p, "clamp", 1)),
                   float(getattr(p, "tol", 0.0)), int(getattr(p, "tol_check_every", 1)),
                   int(getattr(p, "precision", PREC_FP32)), int(getattr(p, "monitor", 0)),
                   int(getattr(p, "recompute", 0)))


class Geometry:
    """Owns a tnlm_geometry handle (created by tnlm_create_geometry)."""

    def __init__(self, handle: int, desc: GeometryDesc):
        self.handle = handle
        self.nx, self.ny = desc.nx, desc.ny
        self.n_phases, self.n_views, self.n_bins = desc.n_phases, desc.n_views, desc.n_bins

    @property
    def img_shape(self) -> Tuple[int, int, int]:
        return (self.n_phases, self.ny, self.nx)

    @property
    def sino_shape(self) -> Tuple[int, int, int]:
        return (self.n_phases, self.n_views, self.n_bins)

    def close(self) -> None:
        if self.handle:
            load_library().tnlm_destroy_geometry(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tnlm_create_geometry(g: Any, angles=None, device: int = 0) -> Geometry:
    """g: an object with nx, ny, pixel_mm, n_phases, n_views, n_bins, bin_mm,
    sid_mm, sdd_mm (e.g. synth.Geometry); angles: [N*V] source angles."""
    import numpy as np
    ang = np.ascontiguousarray(g.view_angles() if angles is None else angles, dtype=np.float64)
    desc = GeometryDesc(int(g.nx), int(g.ny), float(g.pixel_mm), int(g.n_phases), int(g.n_views),
                        int(g.n_bins), float(g.bin_mm), float(g.sid_mm), float(g.sdd_mm),
                        TNLM_DETECTOR_ARC, ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        int(device))
    h = ctypes.c_void_p()
    _check(load_library().tnlm_create_geometry(ctypes.byref(desc), ctypes.byref(h)))
    return Geometry(h.value, desc)


def tnlm_project(geom: Geometry, img, sino, stream=None) -> None:
    _check(load_library().tnlm_project(geom.handle, _ptr(img), _ptr(sino), _stream(stream)))


def tnlm_project_static(geom: Geometry, img, sino, stream=None) -> None:
    """tnlm_project without any device allocation (fixed-size static scratch)."""
    _check(load_library().tnlm_project_static(geom.handle, _ptr(img), _ptr(sino), _stream(stream)))


def tnlm_fbp(geom: Geometry, y, img, stream=None) -> None:
    """Initial image: fan-beam FBP of all phases' projections (every phase the same)."""
    _check(load_library().tnlm_fbp(geom.handle, _ptr(y), _ptr(img), _stream(stream)))


def tnlm_fbp_phases(geom: Geometry, y, img, stream=None) -> None:
    """Per-phase fan-beam FBP: phase i from its own views only."""
    _check(load_library().tnlm_fbp_phases(geom.handle, _ptr(y), _ptr(img), _stream(stream)))


def tnlm_backproject(geom: Geometry, sino, img, stream=None) -> None:
    _check(load_library().tnlm_backproject(geom.handle, _ptr(sino), _ptr(img), _stream(stream)))


def tnlm_weights_size(geom: Geometry, params) -> Tuple[int, int]:
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    pc = params_c(params)
    _check(load_library().tnlm_weights_size(geom.handle, ctypes.byref(pc), ctypes.byref(a),
                                            ctypes.byref(b)))
    return a.value, b.value


def tnlm_workspace_bytes(geom: Geometry, params) -> int:
    a = ctypes.c_size_t()
    pc = params_c(params)
    _check(load_library().tnlm_workspace_bytes(geom.handle, ctypes.byref(pc), ctypes.byref(a)))
    return a.value


def tnlm_weights(geom: Geometry, params, g, dist, norm, stream=None) -> None:
    pc = params_c(params)
    _check(load_library().tnlm_weights(geom.handle, ctypes.byref(pc), _ptr(g), _ptr(dist),
                                       _ptr(norm), _stream(stream)))


def tnlm_reconstruct(geom: Geometry, params, y, winv, f, report: bool = True,
                     stream=None) -> Optional[Dict[str, Any]]:
    """Run the TNLM iteration in place on f.  With report=True the call
    synchronises and returns the report (iterations, final relative change,
    data residual, clamped pixels and their per-iteration histories; with
    params.monitor = 1 also the TNLM term, data term and Eq. 1 objective)."""
    pc = params_c(params)
    lib = load_library()
    if not report:
        _check(lib.tnlm_reconstruct(geom.handle, ctypes.byref(pc), _ptr(y), _ptr(winv), _ptr(f),
                                    None, _stream(stream)))
        return None
    rep, arrs = _new_report(pc.k_outer)
    _check(lib.tnlm_reconstruct(geom.handle, ctypes.byref(pc), _ptr(y), _ptr(winv), _ptr(f),
                                ctypes.byref(rep), _stream(stream)))
    return _report_dict(rep, arrs, bool(pc.monitor))


def tnlm_autotune(geom: Geometry, params, y, winv, f0, stream=None) -> Dict[str, int]:
    """Measure and keep the fastest launch shapes for this handle (f0 is not
    modified).  Returns {"bp_groups": G, "gj_tiles": T, "gj_split": S}."""
    pc = params_c(params)
    bg, gt, gs = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load_library().tnlm_autotune(geom.handle, ctypes.byref(pc), _ptr(y), _ptr(winv), _ptr(f0),
                                        ctypes.byref(bg), ctypes.byref(gt), ctypes.byref(gs),
                                        _stream(stream)))
    return {"bp_groups": bg.value, "gj_tiles": gt.value, "gj_split": gs.value}


def tnlm_reconstruct_batch(geoms, params, ys, winvs, fs, autotune: bool = True,
                           stream=None) -> List[Dict[str, Any]]:
    """Run the TNLM iteration in place on every f of the batch as one graph
    launch (each slice stops at its own k_outer or tolerance, decided on the
    device).  params: one parameter set or one per slice (objects with the
    tnlm_params fields; tol and tol_check_every optional).  Returns one
    report per slice."""
    n = len(geoms)
    if not (len(ys) == len(winvs) == len(fs) == n):
        raise ValueError("geoms, ys, winvs and fs must have the same length")
    plist = list(params) if isinstance(params, (list, tuple)) else [params] * n
    if len(plist) != n:
        raise ValueError("one parameter set per slice expected")
    pcs = (ParamsC * n)(*[params_c(p) for p in plist])
    vp = ctypes.c_void_p
    hs = (vp * n)(*[g.handle for g in geoms])
    yp = (vp * n)(*[_ptr(t) for t in ys])
    wp = (vp * n)(*[_ptr(t) for t in winvs])
    fp = (vp * n)(*[_ptr(t) for t in fs])
    hist = []
    reps = (ReportC * n)()
    for k in range(n):
        rep, arrs = _new_report(pcs[k].k_outer)
        hist.append(arrs)
        reps[k] = rep
    _check(load_library().tnlm_reconstruct_batch(hs, pcs, n, yp, wp, fp, reps, 1 if autotune else 0,
                                                 _stream(stream)))
    return [_report_dict(reps[k], hist[k], bool(pcs[k].monitor)) for k in range(n)]


def tnlm_batch_last_was_loop() -> bool:
    """Whether the last batched call on this thread ran as one loop-graph launch."""
    return bool(load_library().tnlm_batch_last_was_loop())


def tnlm_measure_peaks(device: int = 0) -> Dict[str, float]:
    """Measured FP32 FMA and ex2.approx rates (lane operations per second)."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load_library().tnlm_measure_peaks(int(device), ctypes.byref(a), ctypes.byref(b)))
    return {"fp32_ops": a.value, "ex2_ops": b.value}


def tnlm_debug_fail_alloc_after(n: int) -> None:
    load_library().tnlm_debug_fail_alloc_after(int(n))


def tnlm_debug_wait_limit(polls: int) -> None:
    """Poll limit of the TMA sweep's pipeline waits (< 0: built-in); a test
    hook for the timeout path."""
    load_library().tnlm_debug_wait_limit(int(polls))


def tnlm_profile_enable(geom: Geometry, classes=()) -> None:
    """Time the launches of these kernel classes (names from KCLASSES) with
    CUDA events on their stream; () turns timing off (counting stays on)."""
    mask = 0
    for c in classes:
        mask |= 1 << KCLASSES.index(c)
    _check(load_library().tnlm_profile_enable(geom.handle, mask))


def tnlm_profile_read(geom: Geometry, reset: bool = True) -> Dict[str, Dict[str, float]]:
    """{class: {"ms": device time of timed launches, "launches": count}}."""
    ms = (ctypes.c_double * len(KCLASSES))()
    n = (ctypes.c_longlong * len(KCLASSES))()
    _check(load_library().tnlm_profile_read(geom.handle, ms, n, 1 if reset else 0))
    return {c: {"ms": ms[k], "launches": int(n[k])} for k, c in enumerate(KCLASSES)}


# ---------------------------------------------------------------------------
# learned warm start (include/tnlm_unet.h)
# ---------------------------------------------------------------------------
def _ucheck(status: int) -> None:
    if status != TNLM_OK:
        msg = load_library().tnlm_unet_last_error().decode(errors="replace")
        raise TnlmError(status, msg)


class UNet:
    """Owns a tnlm_unet (2D U-Net over phases as channels, BF16 storage)."""

    def __init__(self, in_ch: int = 10, out_ch: int = 10, base: int = 32, levels: int = 4,
                 device: int = 0):
        self.in_ch, self.out_ch, self.base, self.levels = in_ch, out_ch, base, levels
        h = ctypes.c_void_p()
        _ucheck(load_library().tnlm_unet_create(in_ch, out_ch, base, levels, device, ctypes.byref(h)))
        self.handle = h.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tnlm_unet_destroy(self.handle)
            self.handle = None

    @property
    def param_count(self) -> int:
        return int(load_library().tnlm_unet_param_count(self.handle))

    def set_params(self, flat) -> None:
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.param_count:
            raise ValueError(f"expected {self.param_count} parameters, got {a.size}")
        _ucheck(load_library().tnlm_unet_set_params(self.handle, a.ctypes.data))

    def get_params(self, grads: bool = False):
        import numpy as np
        n = self.param_count
        p = np.zeros(n, dtype=np.float32)
        g = np.zeros(n, dtype=np.float32) if grads else None
        _ucheck(load_library().tnlm_unet_get_params(self.handle, p.ctypes.data,
                                                    g.ctypes.data if grads else None))
        return (p, g) if grads else p

    def forward(self, x, out, stream=None) -> None:
        b, c, h, w = x.shape
        _ucheck(load_library().tnlm_unet_forward(self.handle, _ptr(x), _ptr(out), b, h, w,
                                                 _stream(stream)))

    def grads(self, x, target, stream=None) -> float:
        b, c, h, w = x.shape
        loss = ctypes.c_double(0.0)
        _ucheck(load_library().tnlm_unet_grads(self.handle, _ptr(x), _ptr(target), b, h, w,
                                               ctypes.byref(loss), _stream(stream)))
        return loss.value

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                  stream=None) -> None:
        _ucheck(load_library().tnlm_unet_adam_step(self.handle, lr, beta1, beta2, eps, _stream(stream)))
