"""CPU oracle for the Guidefill shell fill — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product library never calls it.  The C source
``guidefill_oracle.c`` is compiled with gcc (no fast-math, no FP contraction)
into ``liboracle.so`` beside it on first use, or by ``build()``.

Functions follow the paper (arxiv 1611.05319):
  fill       Algorithm 1 with the rotated ghost-pixel ball, eq. weight,
             eq. bilinearDef, eqs. confidence / ready (smart order)
  guidance   guide field from splines, Section 3.3 (optionally weighted by
             each spline's coherence factor |g_Gamma|)
  detect_splines   automatic spline detection, Section 3.3 (ring R, Canny on
             an annulus, structure tensor eq. structureTensor, g_Gamma)
  alg_bytes  algorithmic bytes of a fill under Algorithm 1's per-step semantics
  frozen_fill / fill_backward   (see the adjoint section below)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "guidefill_oracle.c")
_SRC_ADJ = os.path.join(_HERE, "guidefill_oracle_adjoint.c")
_SRC_SPL = os.path.join(_HERE, "guidefill_oracle_splines.c")
_LIB = os.path.join(_HERE, "liboracle.so")

GHOST = 1
SMART = 2
DATA = 8  # data term of eq. ready2

KNOWN, UNFILLED, BYSTANDER = -1, -2, -3


class Stats(C.Structure):
    _fields_ = [("shells", C.c_int32), ("stalls", C.c_int32), ("evaluations", C.c_int64),
                ("filled", C.c_int64), ("unreachable", C.c_int64), ("max_front", C.c_int64),
                ("min_margin", C.c_double), ("data_switch", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DetParams(C.Structure):
    _fields_ = [("sigma", C.c_float), ("rho", C.c_float), ("ring_dist", C.c_int32), ("annulus", C.c_int32),
                ("t_high", C.c_float), ("t_low", C.c_float), ("length", C.c_float), ("Lambda", C.c_float)]


class DetDebug(C.Structure):
    _fields_ = [("d_hole", C.c_void_p), ("d_all", C.c_void_p), ("edge_nms", C.c_void_p), ("edge", C.c_void_p),
                ("us", C.c_void_p), ("T", C.c_void_p), ("J", C.c_void_p)]


# defaults of the detection (sigma = 2, rho = 4 as in the example of Section 3.3.1;
# Lambda = 1e-5 as in Section 3.3)
DETECT_DEFAULTS = dict(sigma=2.0, rho=4.0, ring_dist=0, annulus=2, t_high=0.04, t_low=0.015, length=48.0,
                       Lambda=1e-5)


def build(force: bool = False) -> str:
    srcs = [s for s in (_SRC, _SRC_ADJ, _SRC_SPL) if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp] + srcs + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.oracle_fill.restype = C.c_int
        _lib.oracle_fill.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, C.c_double, C.c_double,
                                     C.c_double, C.c_uint, C.c_float, C.c_int, P, P, P, P]
        _lib.oracle_guidance.restype = C.c_int
        _lib.oracle_guidance.argtypes = [C.c_int, C.c_int, P, C.c_int, P, P, C.c_float, P, P, P, P,
                                         C.POINTER(C.c_double)]
        _lib.oracle_detect_splines.restype = C.c_int
        _lib.oracle_detect_splines.argtypes = [C.c_int, C.c_int, P, P, C.POINTER(DetParams), C.c_int, P, P, P,
                                               C.POINTER(DetDebug)]
        _lib.oracle_gauss_taps.restype = C.c_int
        _lib.oracle_gauss_taps.argtypes = [C.c_float, P]
        _lib.oracle_alg_bytes.restype = C.c_int64
        _lib.oracle_alg_bytes.argtypes = [C.c_int, C.c_int, P, P, C.c_double, C.c_uint, C.c_float,
                                          P, P]
        if hasattr(_lib, "oracle_frozen_fill"):
            _lib.oracle_frozen_fill.restype = C.c_int
            _lib.oracle_frozen_fill.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, C.c_double,
                                                C.c_double, C.c_float, P, P, C.c_int, P]
            _lib.oracle_fill_backward.restype = C.c_int
            _lib.oracle_fill_backward.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, C.c_double, C.c_double,
                                                  C.c_float, P, P, C.c_int, P, P, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f32(x):
    return float(np.float32(x))


def fill(rgb, labels, guide, eps=3.0, mu=50.0, c=0.05, ghost=True, smart=True, tau=1e-5,
         max_shells=0, data_term=False):
    """Runs Algorithm 1 on a copy of ``rgb`` (float32/64 [H, W, C]) in FP64.
    Parameters are rounded to FP32 first (the library takes FP32 parameters).
    Returns dict(u=float64 [H, W, C], shell, enter, stall_steps, stats, status)."""
    lab = np.ascontiguousarray(labels, np.uint8)
    H, W = lab.shape
    u = np.ascontiguousarray(rgb, np.float64).copy()
    Cn = u.shape[2]
    g = np.ascontiguousarray(guide, np.float32)
    assert g.shape == (H, W, 2)
    shell = np.empty((H, W), np.int32)
    enter = np.empty((H, W), np.int32)
    n_hole = int((lab == 1).sum())
    cap = max_shells if max_shells > 0 else n_hole + 1
    stall = np.zeros(cap + 1, np.uint8)
    st = Stats()
    flags = (GHOST if ghost else 0) | (SMART if smart else 0) | (DATA if data_term else 0)
    rc = lib().oracle_fill(H, W, Cn, _p(u), _p(lab), _p(g), _f32(eps), _f32(mu), _f32(c), flags,
                           _f32(tau), int(max_shells), _p(shell), _p(enter), _p(stall),
                           C.byref(st))
    if rc < 0:
        raise ValueError("oracle_fill: bad arguments")
    s = st.as_dict()
    return dict(u=u, shell=shell, enter=enter, stall_steps=stall[:s["shells"]].copy(), stats=s,
                status=rc)


def guidance(labels, offsets, pts, eta=3.0, H=None, W=None, weight=None):
    """Guide field from polylines (Section 3.3), float32 [H, W, 2]; zero outside
    the hole.  weight: optional float32 [n_splines], the magnitude |g_Gamma| of
    each spline's direction (1 when omitted)."""
    return guidance_ties(labels, offsets, pts, eta, weight=weight)["guide"]


SEG_TIE_PX = 1e-3  # width of the tie band of the nearest-segment and 3-eta decisions (px)


def guidance_ties(labels, offsets, pts, eta=3.0, weight=None):
    """Guide field (as ``guidance``) with its near-ties: dict(guide, alt, tie,
    n_ties, min_gap).  Where ``tie`` is set the nearest-segment choice or the
    3 eta cut is within SEG_TIE_PX px of a tie and ``alt`` holds the value of the
    other choice (both are valid); ``min_gap`` is the smallest decision gap (px)
    over the other hole pixels."""
    lab = np.ascontiguousarray(labels, np.uint8)
    H, W = lab.shape
    off = np.ascontiguousarray(offsets, np.int32)
    P = np.ascontiguousarray(pts, np.float32)
    g = np.zeros((H, W, 2), np.float32)
    alt = np.zeros((H, W, 2), np.float32)
    tie = np.zeros((H, W), np.uint8)
    mg = C.c_double(0.0)
    w = None if weight is None else np.ascontiguousarray(weight, np.float32)
    assert w is None or w.shape == (len(off) - 1,)
    rc = lib().oracle_guidance(H, W, _p(lab), len(off) - 1, _p(off), _p(P), _f32(eta), _p(w), _p(g), _p(alt),
                               _p(tie), C.byref(mg))
    if rc < 0:
        raise ValueError("oracle_guidance: bad arguments")
    return dict(guide=g, alt=alt, tie=tie.astype(bool), n_ties=int(rc), min_gap=mg.value)


def alg_bytes(labels, guide, eps, shell, enter, ghost=True, tau=1e-5):
    lab = np.ascontiguousarray(labels, np.uint8)
    H, W = lab.shape
    g = np.ascontiguousarray(guide, np.float32)
    return int(lib().oracle_alg_bytes(H, W, _p(lab), _p(g), _f32(eps), GHOST if ghost else 0,
                                      _f32(tau), _p(np.ascontiguousarray(shell, np.int32)),
                                      _p(np.ascontiguousarray(enter, np.int32))))


# ---------------------------------------------------------------------------
# adjoint (frozen schedule): see guidefill_oracle_adjoint.c
# ---------------------------------------------------------------------------
def _stall_u8(stall_steps, K):
    s = np.zeros(max(K, 1), np.uint8)
    if stall_steps is not None and len(stall_steps):
        s[:len(stall_steps)] = np.asarray(stall_steps, np.uint8)[:K]
    return s


def frozen_fill(u_in, labels, guide, shell, stall_steps, eps=3.0, mu=50.0, phi=None, tau=1e-5):
    """FP64 fill with the schedule (shell map, stall steps) and the ghost-sample
    taps of a forward run held fixed, at angle field ``phi`` (FP64 [H, W]; None =
    angle of ``guide``) and ``mu``.  Returns u_out FP64 [H, W, C]."""
    lab = np.ascontiguousarray(labels, np.uint8)
    H, W = lab.shape
    u = np.ascontiguousarray(u_in, np.float64)
    Cn = u.shape[2]
    out = np.empty_like(u)
    g = np.ascontiguousarray(guide, np.float32)
    sh = np.ascontiguousarray(shell, np.int32)
    K = int(sh.max()) + 1 if sh.size else 0
    ph = None if phi is None else np.ascontiguousarray(phi, np.float64)
    lib().oracle_frozen_fill(H, W, Cn, _p(u), _p(lab), _p(g), _p(ph), _f32(eps), float(mu), _f32(tau), _p(sh),
                             _p(_stall_u8(stall_steps, K)), K, _p(out))
    return out


def fill_backward(u_out, labels, guide, shell, stall_steps, grad_out, eps=3.0, mu=50.0, tau=1e-5):
    """FP64 reverse sweep of the frozen fill.  Returns (grad_in [H,W,C],
    grad_phi [H,W], grad_mu)."""
    lab = np.ascontiguousarray(labels, np.uint8)
    H, W = lab.shape
    u = np.ascontiguousarray(u_out, np.float64)
    Cn = u.shape[2]
    go = np.ascontiguousarray(grad_out, np.float64)
    gi = np.empty_like(go)
    gphi = np.empty((H, W), np.float64)
    gmu = C.c_double(0.0)
    sh = np.ascontiguousarray(shell, np.int32)
    K = int(sh.max()) + 1 if sh.size else 0
    g = np.ascontiguousarray(guide, np.float32)
    lib().oracle_fill_backward(H, W, Cn, _p(u), _p(lab), _p(g), _f32(eps), float(mu), _f32(tau), _p(sh),
                               _p(_stall_u8(stall_steps, K)), K, _p(go), _p(gi), _p(gphi), C.byref(gmu))
    return gi, gphi, gmu.value


def gauss_taps(s):
    """The normalised FP32 taps of g_s the detection uses (radius ceil(2 s))."""
    w = np.zeros(129, np.float32)
    r = lib().oracle_gauss_taps(_f32(s), _p(w))
    return w[:2 * r + 1].copy()


def detect_splines(rgb, labels, max_splines=4096, debug=False, **kw):
    """Automatic spline detection of Section 3.3 on an RGB(A) image (float32
    [H, W, >=3]; the first three channels are used) with labels (0 known, 1
    hole, 2 bystander).  Returns dict(count, pts [n, 2, 2] (base, end), weight
    [n], base [n] (pixel index y W + x)) for the first n = min(count,
    max_splines) splines in raster order of their base; with debug=True also
    the per-pixel maps d_hole, d_all, edge_nms, edge, us, T, J."""
    prm = dict(DETECT_DEFAULTS)
    prm.update(kw)
    lab = np.ascontiguousarray(labels, np.uint8)
    H, W = lab.shape
    rgb3 = np.ascontiguousarray(np.asarray(rgb)[..., :3], np.float32)
    assert rgb3.shape == (H, W, 3)
    P = DetParams(_f32(prm["sigma"]), _f32(prm["rho"]), int(prm["ring_dist"]), int(prm["annulus"]),
                  _f32(prm["t_high"]), _f32(prm["t_low"]), _f32(prm["length"]), _f32(prm["Lambda"]))
    pts = np.zeros((max(max_splines, 1), 2, 2), np.float32)
    wt = np.zeros(max(max_splines, 1), np.float32)
    base = np.zeros(max(max_splines, 1), np.int32)
    maps = {}
    dbg = None
    if debug:
        maps = dict(d_hole=np.zeros((H, W), np.int32), d_all=np.zeros((H, W), np.int32),
                    edge_nms=np.zeros((H, W), np.uint8), edge=np.zeros((H, W), np.uint8),
                    us=np.zeros((H, W, 3), np.float32), T=np.zeros((H, W, 3), np.float32),
                    J=np.zeros((H, W, 3), np.float32))
        dbg = DetDebug(*[_p(maps[k]) for k, _ in DetDebug._fields_])
    rc = lib().oracle_detect_splines(H, W, _p(rgb3), _p(lab), C.byref(P), int(max_splines), _p(pts), _p(wt),
                                     _p(base), C.byref(dbg) if dbg is not None else None)
    if rc < 0:
        raise ValueError("oracle_detect_splines: bad arguments")
    n = min(rc, max_splines)
    out = dict(count=rc, pts=pts[:n].copy(), weight=wt[:n].copy(), base=base[:n].copy())
    out.update(maps)
    return out
