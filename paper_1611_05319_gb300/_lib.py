"""ctypes binding of libguidefill.so (include/guidefill.h): argument marshalling only.

The shared library is built in-tree by ``paper_1611_05319_gb300.build.build()``.
If it is missing, loading fails with an error: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libguidefill.so")

GF_FLAG_GHOST = 1
GF_FLAG_SMART = 2
GF_FLAG_RESCAN = 4
GF_FLAG_DATA = 8

STATUS = {0: "ok", 1: "incomplete", -1: "invalid argument", -2: "CUDA error", -3: "timeout",
          -4: "no progress", -5: "out of memory", -6: "unsupported device", -7: "internal error",
          -8: "frame too large for gf_fill_noalloc"}

# every function declared in include/guidefill.h
EXPORTS = ["gf_create", "gf_destroy", "gf_status_string", "gf_last_cuda_error", "gf_fill",
           "gf_fill_batched", "gf_fill_batched_ex", "gf_fill_batched_host", "gf_guidance_from_splines", "gf_guidance_batched",
           "gf_set_launch_config", "gf_get_last_launch", "gf_max_active_clusters", "gf_fill_backward",
           "gf_guide_from_angle", "gf_autotune", "gf_fill_noalloc", "gf_set_split", "gf_get_last_split",
           "gf_detect_splines", "gf_detect_splines_batched", "gf_fill_batched_splines"]


class Frame(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("rgba", C.c_void_p), ("labels", C.c_void_p),
                ("guide", C.c_void_p), ("out_rgba", C.c_void_p), ("out_shell", C.c_void_p),
                ("out_enter", C.c_void_p), ("out_stall", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("eps", C.c_float), ("mu", C.c_float), ("c", C.c_float), ("flags", C.c_uint32),
                ("snap_tau", C.c_float), ("max_shells", C.c_int32)]


class SplineFrame(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("labels", C.c_void_p), ("n_splines", C.c_int32),
                ("n_points", C.c_int32), ("offsets", C.c_void_p), ("pts", C.c_void_p), ("guide", C.c_void_p),
                ("weight", C.c_void_p)]


class DetectParams(C.Structure):
    _fields_ = [("sigma", C.c_float), ("rho", C.c_float), ("ring_dist", C.c_int32), ("annulus", C.c_int32),
                ("t_high", C.c_float), ("t_low", C.c_float), ("length", C.c_float), ("Lambda", C.c_float)]


class DetectFrame(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("rgba", C.c_void_p), ("labels", C.c_void_p),
                ("max_splines", C.c_int32), ("pts", C.c_void_p), ("weight", C.c_void_p), ("offsets", C.c_void_p),
                ("base", C.c_void_p), ("edges", C.c_void_p), ("result", C.c_void_p)]


class AdjointFrame(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("out_rgba", C.c_void_p), ("guide", C.c_void_p),
                ("shell", C.c_void_p), ("stall", C.c_void_p), ("grad_out", C.c_void_p), ("grad_in", C.c_void_p),
                ("grad_phi", C.c_void_p), ("grad_mu", C.c_void_p)]


STATS_DTYPE = np.dtype([("shells", np.int32), ("stalls", np.int32), ("status", np.int32), ("rechecks", np.int32),
                        ("filled", np.int64), ("evaluations", np.int64), ("max_front", np.int64),
                        ("holes", np.int64), ("data_switch", np.int32), ("reserved", np.int32)])
STATS_BYTES = STATS_DTYPE.itemsize  # 56


class GuidefillError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1611_05319_gb300.build.build() "
                               "(requires nvcc); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.gf_create.argtypes = [C.POINTER(P), C.c_int]
        L.gf_create.restype = C.c_int
        L.gf_destroy.argtypes = [P]
        L.gf_destroy.restype = None
        L.gf_status_string.argtypes = [C.c_int]
        L.gf_status_string.restype = C.c_char_p
        L.gf_last_cuda_error.argtypes = [P]
        L.gf_last_cuda_error.restype = C.c_int
        L.gf_fill.argtypes = [P, C.POINTER(Frame), C.POINTER(Params), P, P]
        L.gf_fill.restype = C.c_int
        L.gf_fill_batched.argtypes = [P, C.c_int, C.POINTER(Frame), C.POINTER(Params), P, P]
        L.gf_fill_batched.restype = C.c_int
        L.gf_fill_batched_ex.argtypes = [P, C.c_int, C.POINTER(Frame), C.POINTER(Params), P, P, P, P]
        L.gf_fill_batched_ex.restype = C.c_int
        L.gf_fill_batched_host.argtypes = [P, C.c_int, P, P, P, P, P, P, P, P, P, C.c_float, P, P,
                                           C.POINTER(Params), P, P]
        L.gf_fill_batched_host.restype = C.c_int
        L.gf_guidance_from_splines.argtypes = [P, C.c_int, C.c_int, P, C.c_int, P, C.c_int, P, C.c_float, P, P]
        L.gf_guidance_from_splines.restype = C.c_int
        L.gf_guidance_batched.argtypes = [P, C.c_int, C.POINTER(SplineFrame), C.c_float, P]
        L.gf_guidance_batched.restype = C.c_int
        L.gf_set_launch_config.argtypes = [P, C.c_int, C.c_int, C.c_int]
        L.gf_set_launch_config.restype = C.c_int
        L.gf_get_last_launch.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.gf_get_last_launch.restype = C.c_int
        L.gf_max_active_clusters.argtypes = [P, C.c_float, C.c_int]
        L.gf_max_active_clusters.restype = C.c_int
        L.gf_fill_backward.argtypes = [P, C.c_int, C.POINTER(AdjointFrame), C.POINTER(Params), P]
        L.gf_fill_backward.restype = C.c_int
        L.gf_guide_from_angle.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P]
        L.gf_guide_from_angle.restype = C.c_int
        L.gf_autotune.argtypes = [P, C.c_int, C.POINTER(Frame), C.POINTER(Params), P, P, C.c_int,
                                  C.POINTER(C.c_int), C.POINTER(C.c_float)]
        L.gf_autotune.restype = C.c_int
        L.gf_fill_noalloc.argtypes = [C.POINTER(Frame), C.POINTER(Params), P, P]
        L.gf_fill_noalloc.restype = C.c_int
        L.gf_set_split.argtypes = [P, C.c_int, C.c_int, C.c_int]
        L.gf_set_split.restype = C.c_int
        L.gf_get_last_split.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.gf_get_last_split.restype = C.c_int
        L.gf_fill_batched_splines.argtypes = [P, C.c_int, C.POINTER(Frame), C.POINTER(SplineFrame), C.c_float,
                                              C.POINTER(Params), P, P, P, P]
        L.gf_fill_batched_splines.restype = C.c_int
        L.gf_detect_splines.argtypes = [P, C.POINTER(DetectFrame), C.POINTER(DetectParams), P]
        L.gf_detect_splines.restype = C.c_int
        L.gf_detect_splines_batched.argtypes = [P, C.c_int, C.POINTER(DetectFrame), C.POINTER(DetectParams), P]
        L.gf_detect_splines_batched.restype = C.c_int
        _lib = L
    return _lib


def check(code: int, what: str, ctx=None):
    if code < 0:
        extra = ""
        if ctx is not None and code == -2:
            extra = f" (cudaError {lib().gf_last_cuda_error(ctx)})"
        raise GuidefillError(code, what + extra)
    return code


def make_params(eps=3.0, mu=50.0, c=0.05, ghost=True, smart=True, rescan=False, snap_tau=1e-5, max_shells=0,
                data_term=False):
    flags = (GF_FLAG_GHOST if ghost else 0) | (GF_FLAG_SMART if smart else 0) | (GF_FLAG_RESCAN if rescan else 0) | \
        (GF_FLAG_DATA if data_term else 0)
    return Params(float(eps), float(mu), float(c), flags, float(snap_tau), int(max_shells))


# Section 3.3's example values sigma = 2, rho = 4 and Lambda = 1e-5; thresholds on
# |grad u_sigma| for colours in [0, 1]
DETECT_DEFAULTS = dict(sigma=2.0, rho=4.0, ring_dist=0, annulus=2, t_high=0.04, t_low=0.015, length=48.0,
                       Lambda=1e-5)


def make_detect_params(**kw):
    d = dict(DETECT_DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise TypeError(f"unknown detection parameters: {sorted(unknown)}")
    d.update(kw)
    return DetectParams(float(d["sigma"]), float(d["rho"]), int(d["ring_dist"]), int(d["annulus"]),
                        float(d["t_high"]), float(d["t_low"]), float(d["length"]), float(d["Lambda"]))
