"""GB300-native Guidefill shell fill (arxiv 1611.05319): PyTorch-facing binding.

PyTorch provides device memory and streams only; every step of the fill runs in
the CUDA kernels of ``libguidefill.so`` behind the C ABI in
``include/guidefill.h``.  This module marshals tensors into that ABI.

    ctx = Context(0)
    out = ctx.fill(rgba, labels, guide, eps=3.0, mu=50.0, c=0.05)
    out.rgba, out.shell, out.stats()
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import STATS_BYTES, STATS_DTYPE, GuidefillError, check, lib, make_params

__all__ = ["Context", "HostBatch", "context", "fill", "fill_batched", "guidance", "detect_splines", "guidance_auto",
           "FillResult", "DetectResult", "GuidefillError", "to_rgba", "STATS_DTYPE"]


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def to_rgba(img: torch.Tensor) -> torch.Tensor:
    """[H, W, 3|4] float32 -> contiguous [H, W, 4] float32 (alpha = 1 when padded)."""
    if img.dim() != 3 or img.shape[2] not in (3, 4):
        raise ValueError("image must be [H, W, 3] or [H, W, 4]")
    img = img.to(torch.float32)
    if img.shape[2] == 3:
        img = torch.cat([img, torch.ones_like(img[..., :1])], dim=2)
    return img.contiguous()


@dataclass
class FillResult:
    rgba: torch.Tensor
    shell: torch.Tensor
    enter: Optional[torch.Tensor]
    stall: Optional[torch.Tensor]
    _stats_dev: torch.Tensor = field(repr=False)

    def stats(self) -> dict:
        """Synchronises with the device and returns the frame's gf_stats."""
        rec = np.frombuffer(self._stats_dev.cpu().numpy().tobytes(), dtype=STATS_DTYPE)[0]
        d = {k: int(rec[k]) for k in STATS_DTYPE.names}
        return d

    def stall_steps(self) -> np.ndarray:
        """Boolean array over steps 0..K-1: step filled by the stall rule."""
        K = self.stats()["shells"]
        bits = self.stall.cpu().numpy().view(np.uint32)
        idx = np.arange(K)
        return ((bits[idx >> 5] >> (idx & 31)) & 1).astype(bool)


@dataclass
class DetectResult:
    """Splines of one frame from gf_detect_splines (device tensors): pts
    [max_splines, 2, 2] (base, end), weight [max_splines] (|g_Gamma|), offsets
    [max_splines + 1] (polyline offsets 2 min(s, n)), base [max_splines] (pixel
    index of each base), result [2] (n found, status), edges [H, W] or None."""
    pts: torch.Tensor
    weight: torch.Tensor
    offsets: torch.Tensor
    base: torch.Tensor
    result: torch.Tensor
    edges: Optional[torch.Tensor]
    max_splines: int

    def count(self) -> int:
        """Synchronises; the number of splines found (may exceed max_splines)."""
        r = self.result.cpu().tolist()
        if r[1] != 0:
            raise GuidefillError(r[1], "gf_detect_splines (device)")
        return int(r[0])

    def splines(self):
        """Synchronises; (pts [n, 2, 2], weight [n], base [n]) as numpy for the n written."""
        n = min(self.count(), self.max_splines)
        return (self.pts[:n].cpu().numpy(), self.weight[:n].cpu().numpy(), self.base[:n].cpu().numpy())


class Context:
    """Owns a gf_ctx (scratch memory, cached graphs) on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().gf_create(C.byref(h), self.device), "gf_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().gf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- config
    def set_launch_config(self, cluster_size: int = 0, n_clusters: int = 0, use_graph: bool = True):
        check(lib().gf_set_launch_config(self._h, cluster_size, n_clusters, int(use_graph)), "gf_set_launch_config")

    def last_launch(self):
        a, b = C.c_int(), C.c_int()
        check(lib().gf_get_last_launch(self._h, C.byref(a), C.byref(b)), "gf_get_last_launch")
        return a.value, b.value

    def set_split(self, split_m: int = 0, cluster_size: int = 0, n_clusters: int = 0):
        """Split schedule: the split_m largest holes on n_clusters clusters of
        cluster_size CTAs beside the main launch (split_m = 0: one launch)."""
        check(lib().gf_set_split(self._h, split_m, cluster_size, n_clusters), "gf_set_split")

    def last_split(self):
        m, a, b = C.c_int(), C.c_int(), C.c_int()
        check(lib().gf_get_last_split(self._h, C.byref(m), C.byref(a), C.byref(b)), "gf_get_last_split")
        return m.value, a.value, b.value

    def autotune(self, frames, stats: torch.Tensor, params, trials: int = 3, stream=None):
        """Runs gf_autotune on prepared ctypes frames; returns (cluster_size, ms)."""
        cs, ms = C.c_int(), C.c_float()
        check(lib().gf_autotune(self._h, len(frames), frames, C.byref(params), _ptr(stats), _stream(stream),
                                int(trials), C.byref(cs), C.byref(ms)), "gf_autotune", self._h)
        return cs.value, ms.value

    def max_active_clusters(self, eps: float, cluster_size: int) -> int:
        return lib().gf_max_active_clusters(self._h, float(eps), int(cluster_size))

    # ------------------------------------------------------------------ fill
    def _frame(self, rgba, labels, guide, out, want_enter, want_stall):
        dev = torch.device("cuda", self.device)
        rgba = to_rgba(rgba.to(dev))
        H, W = rgba.shape[:2]
        labels = labels.to(dev, torch.uint8).contiguous()
        guide = guide.to(dev, torch.float32).contiguous()
        if labels.shape != (H, W) or guide.shape != (H, W, 2):
            raise ValueError("labels must be [H, W] and guide [H, W, 2]")
        out_rgba = rgba if out == "inplace" else (out if out is not None else torch.empty_like(rgba))
        shell = torch.empty((H, W), dtype=torch.int32, device=dev)
        enter = torch.empty((H, W), dtype=torch.int32, device=dev) if want_enter else None
        stall = torch.empty(((H * W + 1 + 31) // 32,), dtype=torch.int32, device=dev) if want_stall else None
        fr = _lib.Frame(H, W, rgba.data_ptr(), labels.data_ptr(), guide.data_ptr(), out_rgba.data_ptr(),
                        shell.data_ptr(), enter.data_ptr() if enter is not None else None,
                        stall.data_ptr() if stall is not None else None)
        keep = (rgba, labels, guide)
        return fr, out_rgba, shell, enter, stall, keep

    def fill(self, rgba, labels, guide, eps=3.0, mu=50.0, c=0.05, ghost=True, smart=True, rescan=False,
             snap_tau=1e-5, max_shells=0, out=None, enter=False, stall=False, stream=None,
             data_term=False) -> FillResult:
        """Fills one frame.  rgba [H,W,3|4] float32, labels [H,W] uint8 (0 known, 1 hole, 2 bystander),
        guide [H,W,2] float32.  out=None allocates the output, out="inplace" fills rgba in place
        (rgba must then already be a contiguous [H,W,4] float32 CUDA tensor)."""
        return self.fill_batched([rgba], [labels], [guide], eps, mu, c, ghost, smart, rescan, snap_tau, max_shells,
                                 out=None if out is None else [out], enter=enter, stall=stall, stream=stream,
                                 data_term=data_term)[0]

    def fill_batched(self, rgba: Sequence[torch.Tensor], labels: Sequence[torch.Tensor],
                     guide: Sequence[torch.Tensor], eps=3.0, mu=50.0, c=0.05, ghost=True, smart=True,
                     rescan=False, snap_tau=1e-5, max_shells=0, out=None, enter=False, stall=False,
                     stream=None, data_term=False) -> List[FillResult]:
        n = len(rgba)
        if not (len(labels) == len(guide) == n) or n == 0:
            raise ValueError("rgba, labels and guide must have the same non-zero length")
        outs = out if isinstance(out, (list, tuple)) else [out] * n
        frames = (_lib.Frame * n)()
        res, keep = [], []
        for i in range(n):
            fr, o, sh, en, st, kp = self._frame(rgba[i], labels[i], guide[i], outs[i], enter, stall)
            frames[i] = fr
            keep.append(kp)
            res.append((o, sh, en, st))
        stats = torch.empty((n * STATS_BYTES,), dtype=torch.uint8, device=torch.device("cuda", self.device))
        prm = make_params(eps, mu, c, ghost, smart, rescan, snap_tau, max_shells, data_term)
        with torch.cuda.device(self.device):
            check(lib().gf_fill_batched(self._h, n, frames, C.byref(prm), _ptr(stats), _stream(stream)),
                  "gf_fill_batched", self._h)
        self._keep = keep  # inputs stay alive until the next call on this context
        return [FillResult(o, sh, en, st, stats[i * STATS_BYTES:(i + 1) * STATS_BYTES])
                for i, (o, sh, en, st) in enumerate(res)]

    def fill_frames(self, frames, stats: torch.Tensor, params, stream=None, events=None):
        """Lowest-overhead batched call: ``frames`` is a prepared ctypes array of
        _lib.Frame, ``stats`` a device buffer of n*56 bytes (_lib.STATS_BYTES each), ``params`` a _lib.Params;
        ``events`` an optional pair of recorded torch.cuda.Event placed around the
        persistent fill kernel."""
        e0 = C.c_void_p(events[0].cuda_event) if events else None
        e1 = C.c_void_p(events[1].cuda_event) if events else None
        check(lib().gf_fill_batched_ex(self._h, len(frames), frames, C.byref(params), _ptr(stats), _stream(stream),
                                       e0, e1), "gf_fill_batched_ex", self._h)

    # --------------------------------------------------------------- adjoint
    def fill_backward(self, results: Sequence[FillResult], guides: Sequence[torch.Tensor],
                      grad_out: Sequence[torch.Tensor], eps=3.0, mu=50.0, c=0.05, smart=True, snap_tau=1e-5,
                      max_shells=0, stream=None):
        """Adjoint of ``fill_batched`` (ghost ball): returns lists (grad_in [H,W,4],
        grad_phi [H,W]) and a device tensor grad_mu [n] (one value per frame).
        ``results`` must come from a fill with ``stall=True`` when it had stall steps."""
        n = len(results)
        dev = torch.device("cuda", self.device)
        frames = (_lib.AdjointFrame * n)()
        gi, gp, keep = [], [], []
        gmu = torch.zeros((n,), dtype=torch.float32, device=dev)
        for i, r in enumerate(results):
            H, W = r.shell.shape
            go = grad_out[i].to(dev, torch.float32).contiguous()
            if go.shape[-1] == 3:
                go = torch.cat([go, torch.zeros_like(go[..., :1])], dim=2).contiguous()
            g = guides[i].to(dev, torch.float32).contiguous()
            a = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
            b = torch.empty((H, W), dtype=torch.float32, device=dev)
            frames[i] = _lib.AdjointFrame(H, W, r.rgba.data_ptr(), g.data_ptr(), r.shell.data_ptr(),
                                          r.stall.data_ptr() if r.stall is not None else None, go.data_ptr(),
                                          a.data_ptr(), b.data_ptr(), gmu.data_ptr() + 4 * i)
            gi.append(a)
            gp.append(b)
            keep.append((go, g))
        prm = make_params(eps, mu, c, True, smart, False, snap_tau, max_shells)
        with torch.cuda.device(self.device):
            check(lib().gf_fill_backward(self._h, n, frames, C.byref(prm), _stream(stream)), "gf_fill_backward",
                  self._h)
        self._akeep = keep
        return gi, gp, gmu

    def guide_from_angle(self, labels, mag, phi, out=None, stream=None) -> torch.Tensor:
        """g = mag (cos phi, sin phi) at hole pixels (FP64, rounded once)."""
        dev = torch.device("cuda", self.device)
        lab = labels.to(dev, torch.uint8).contiguous()
        m = mag.to(dev, torch.float32).contiguous()
        p = phi.to(dev, torch.float32).contiguous()
        H, W = lab.shape
        g = out if out is not None else torch.zeros((H, W, 2), dtype=torch.float32, device=dev)
        with torch.cuda.device(self.device):
            check(lib().gf_guide_from_angle(self._h, H, W, _ptr(lab), _ptr(m), _ptr(p), _ptr(g), _stream(stream)),
                  "gf_guide_from_angle", self._h)
        self._gakeep = (lab, m, p)
        return g

    # -------------------------------------------------------------- guidance
    def guidance(self, labels, offsets, pts, eta=3.0, out=None, stream=None, weight=None) -> torch.Tensor:
        """Guide field from polylines (Section 3.3), written at hole pixels of ``out``
        (zero-initialised [H,W,2] float32 when not given); ``weight`` [n_splines]
        scales each spline's field (|g_Gamma|, 1 when omitted)."""
        return self.guidance_batched([labels], [offsets], [pts], eta, None if out is None else [out], stream,
                                     None if weight is None else [weight])[0]

    def guidance_batched(self, labels, offsets, pts, eta=3.0, out=None, stream=None, weight=None):
        dev = torch.device("cuda", self.device)
        n = len(labels)
        frames = (_lib.SplineFrame * n)()
        outs, keep = [], []
        for i in range(n):
            lab = labels[i].to(dev, torch.uint8).contiguous()
            off = torch.as_tensor(offsets[i], dtype=torch.int32).to(dev).contiguous()
            P = torch.as_tensor(pts[i], dtype=torch.float32).to(dev).contiguous()
            H, W = lab.shape
            g = out[i] if out is not None else torch.zeros((H, W, 2), dtype=torch.float32, device=dev)
            w = None
            if weight is not None and weight[i] is not None:
                w = torch.as_tensor(weight[i], dtype=torch.float32).to(dev).contiguous()
                if w.numel() != off.numel() - 1:
                    raise ValueError("weight needs one value per spline")
            frames[i] = _lib.SplineFrame(H, W, lab.data_ptr(), off.numel() - 1, P.reshape(-1, 2).shape[0],
                                         off.data_ptr(), P.data_ptr(), g.data_ptr(), _ptr(w))
            outs.append(g)
            keep.append((lab, off, P, w))
        with torch.cuda.device(self.device):
            check(lib().gf_guidance_batched(self._h, n, frames, C.c_float(eta), _stream(stream)),
                  "gf_guidance_batched", self._h)
        self._gkeep = keep
        return outs

    # ----------------------------------------------------- spline detection
    def detect_splines_batched(self, rgba: Sequence[torch.Tensor], labels: Sequence[torch.Tensor], max_splines=4096,
                               edges=False, stream=None, **params) -> List[DetectResult]:
        """Automatic spline detection (Section 3.3) on device frames: rgba [H,W,4]
        (or [H,W,3]) float32, labels [H,W] uint8.  ``params``: sigma, rho,
        ring_dist, annulus, t_high, t_low, length, Lambda (see ``_lib.DETECT_DEFAULTS``).
        Results stay on the device; ``count`` is a device int32 tensor [2]
        (number found, status)."""
        dev = torch.device("cuda", self.device)
        n = len(rgba)
        frames = (_lib.DetectFrame * n)()
        outs, keep = [], []
        for i in range(n):
            img = to_rgba(rgba[i].to(dev, torch.float32))
            lab = labels[i].to(dev, torch.uint8).contiguous()
            H, W = lab.shape
            m = int(max_splines)
            pts = torch.zeros((max(m, 1), 2, 2), dtype=torch.float32, device=dev)
            wt = torch.zeros((max(m, 1),), dtype=torch.float32, device=dev)
            off = torch.zeros((m + 1,), dtype=torch.int32, device=dev)
            base = torch.zeros((max(m, 1),), dtype=torch.int32, device=dev)
            res = torch.zeros((2,), dtype=torch.int32, device=dev)
            ed = torch.zeros((H, W), dtype=torch.uint8, device=dev) if edges else None
            frames[i] = _lib.DetectFrame(H, W, img.data_ptr(), lab.data_ptr(), m, pts.data_ptr(), wt.data_ptr(),
                                         off.data_ptr(), base.data_ptr(), _ptr(ed), res.data_ptr())
            outs.append(DetectResult(pts, wt, off, base, res, ed, m))
            keep.append((img, lab))
        prm = _lib.make_detect_params(**params)
        with torch.cuda.device(self.device):
            check(lib().gf_detect_splines_batched(self._h, n, frames, C.byref(prm), _stream(stream)),
                  "gf_detect_splines_batched", self._h)
        self._dkeep = keep
        return outs

    def detect_splines(self, rgba, labels, **kw) -> "DetectResult":
        return self.detect_splines_batched([rgba], [labels], **kw)[0]

    def guidance_auto_batched(self, rgba, labels, eta=3.0, max_splines=4096, out=None, stream=None, **params):
        """Detected splines (Section 3.3) straight into the guide field, with no
        host synchronisation: each frame's guide field comes from its detected
        splines weighted by their coherence factor.  Returns (guides, detections)."""
        det = self.detect_splines_batched(rgba, labels, max_splines=max_splines, stream=stream, **params)
        dev = torch.device("cuda", self.device)
        n = len(rgba)
        frames = (_lib.SplineFrame * n)()
        outs, keep = [], []
        for i in range(n):
            lab = labels[i].to(dev, torch.uint8).contiguous()
            H, W = lab.shape
            g = out[i] if out is not None else torch.zeros((H, W, 2), dtype=torch.float32, device=dev)
            d = det[i]
            frames[i] = _lib.SplineFrame(H, W, lab.data_ptr(), d.max_splines, 2 * d.max_splines, d.offsets.data_ptr(),
                                         d.pts.data_ptr(), g.data_ptr(), d.weight.data_ptr())
            outs.append(g)
            keep.append(lab)
        with torch.cuda.device(self.device):
            check(lib().gf_guidance_batched(self._h, n, frames, C.c_float(eta), _stream(stream)),
                  "gf_guidance_batched", self._h)
        self._gkeep = keep
        return outs, det

    # ---------------------------------------------------- host-buffer path
    def fill_batched_host(self, rgba, labels=None, guide=None, out_rgba=None, out_shell=None, splines=None,
                          eta=3.0, eps=3.0, mu=50.0, c=0.05, ghost=True, smart=True, rescan=False, snap_tau=1e-5,
                          max_shells=0, stream=None, data_term=False) -> np.ndarray:
        """Fills frames held in HOST memory (numpy; rgba [H,W,4] float32, labels [H,W] uint8,
        guide [H,W,2] float32 or None with ``splines[i] = (offsets, pts)``); the library
        copies them to the device, fills, and copies out_rgba / out_shell back.  ``rgba``
        may instead be a ``HostBatch`` (the frames' pointer tables built once).
        Returns the stats records."""
        b = rgba if isinstance(rgba, HostBatch) else HostBatch(rgba, labels, guide, out_rgba, out_shell, splines)
        st = np.zeros(b.n, dtype=STATS_DTYPE)
        prm = make_params(eps, mu, c, ghost, smart, rescan, snap_tau, max_shells, data_term)
        with torch.cuda.device(self.device):
            check(lib().gf_fill_batched_host(self._h, b.n, b.Hs, b.Ws, b.p_rgba, b.p_labels, b.p_guide, b.ns,
                                             b.p_offs, b.npts, b.p_pts, C.c_float(eta), b.p_out_rgba,
                                             b.p_out_shell, C.byref(prm), st.ctypes.data, _stream(stream)),
                  "gf_fill_batched_host", self._h)
        return st


class HostBatch:
    """The pointer tables of a batch of host frames for ``Context.fill_batched_host``,
    built once for frames that are filled repeatedly (a serving loop): the arrays
    (same arguments as ``fill_batched_host``) are referenced, must stay alive, and
    must not be resized while the batch is in use.  Every call still reads the
    inputs from and writes the outputs to these host buffers."""

    def __init__(self, rgba: Sequence[np.ndarray], labels: Sequence[np.ndarray],
                 guide: Optional[Sequence[Optional[np.ndarray]]], out_rgba: Sequence[np.ndarray],
                 out_shell: Sequence[np.ndarray], splines=None):
        n = len(rgba)
        self.n = n
        self.Hs = (C.c_int32 * n)(*[a.shape[0] for a in rgba])
        self.Ws = (C.c_int32 * n)(*[a.shape[1] for a in rgba])

        def arr(xs):
            return (C.c_void_p * n)(*[(x.ctypes.data if x is not None else None) for x in xs])

        if guide is None:
            guide = [None] * n
        self.ns = (C.c_int32 * n)()
        self.npts = (C.c_int32 * n)()
        offs = [None] * n
        pts = [None] * n
        if splines is not None:
            for i, sp in enumerate(splines):
                if sp is None:
                    continue
                o = np.ascontiguousarray(sp[0], np.int32)
                p = np.ascontiguousarray(sp[1], np.float32)
                offs[i], pts[i] = o, p
                self.ns[i] = len(o) - 1
                self.npts[i] = p.shape[0]
        self.p_rgba, self.p_labels, self.p_guide = arr(rgba), arr(labels), arr(guide)
        self.p_offs, self.p_pts = arr(offs), arr(pts)
        self.p_out_rgba, self.p_out_shell = arr(out_rgba), arr(out_shell)
        self._keep = (list(rgba), list(labels), list(guide), offs, pts, list(out_rgba), list(out_shell))


_contexts = {}


def context(device: Optional[int] = None) -> Context:
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _contexts:
        _contexts[d] = Context(d)
    return _contexts[d]


def fill(rgba, labels, guide, **kw) -> FillResult:
    return context(rgba.device.index if rgba.is_cuda else None).fill(rgba, labels, guide, **kw)


def fill_batched(rgba, labels, guide, **kw) -> List[FillResult]:
    return context().fill_batched(rgba, labels, guide, **kw)


def guidance(labels, offsets, pts, eta=3.0, **kw) -> torch.Tensor:
    return context().guidance(labels, offsets, pts, eta, **kw)


def detect_splines(rgba, labels, **kw) -> DetectResult:
    return context(rgba.device.index if rgba.is_cuda else None).detect_splines(rgba, labels, **kw)


def guidance_auto(rgba, labels, eta=3.0, **kw):
    """Guide field from automatically detected splines; returns (guide, detection)."""
    ctx = context(rgba.device.index if rgba.is_cuda else None)
    g, d = ctx.guidance_auto_batched([rgba], [labels], eta, **kw)
    return g[0], d[0]
