"""The five synthetic workloads (seeded), built only from ``synth`` primitives.

Each builder returns a dict with
  rgb     float32 [H, W, 3]  input image; hole and bystander pixels are set to
                             NaN when ``poison`` is true (they must never be read)
  gt      float32 [H, W, 3]  the image before the hole was cut (ground truth)
  labels  uint8   [H, W]     0 known, 1 hole, 2 bystander
  guide   float32 [H, W, 2]  only for constant-guidance workloads, else None
  splines (offsets, pts)     polylines for the guidance-field sampler, else None
  eps, mu, c, eta            parameters
Guidance fields from splines are *not* built here: they are the sampler's job.
"""
from __future__ import annotations

import numpy as np

from . import (annulus_mask, bands_with_fraction, const_guide, flatten_beziers, labels_from,
               polygon_image, rect_mask, _rng)


def _finish(img, hole, bystander=None, poison=False, **kw):
    labels = labels_from(hole, bystander)
    rgb = img.copy()
    if poison:
        rgb[labels != 0] = np.nan
    d = dict(rgb=rgb, gt=img, labels=labels, guide=None, splines=None,
             eps=3.0, mu=50.0, c=0.05, eta=3.0)
    d.update(kw)
    return d


def plain_128(seed: int = 1, poison: bool = False):
    """128x128 polygons + N(0, 0.01) noise; annulus hole of width 8 px centred
    (radii 24..32); constant guidance at 30 degrees; eps=3, mu=50."""
    H = W = 128
    img = polygon_image(H, W, 8, seed)
    hole = annulus_mask(H, W, 24.0, 32.0)
    return _finish(img, hole, poison=poison, guide=const_guide(H, W, 30.0))


def frame_1080(seed: int = 2, poison: bool = False, H: int = 1080, W: int = 1920,
               fraction: float = 0.03):
    """1920x1080 piecewise-smooth frame; hole = union of bands of width U[3, 15] px
    along 20 cubic Beziers, about 3% of the pixels; eps=3, mu=50."""
    img = polygon_image(H, W, 40, seed)
    ctrl, hws, hole = bands_with_fraction(H, W, 20, seed, (1.5, 7.5), fraction)
    return _finish(img, hole, poison=poison, splines=flatten_beziers(ctrl), half_widths=hws)


def frame_4k_blob(seed: int = 3, poison: bool = False, H: int = 2160, W: int = 3840,
                  blob: int = 400, fraction: float = 0.02):
    """3840x2160 frame with one blob x blob square hole at a random position
    plus thin bands along 20 Beziers; eps=4, mu=50."""
    img = polygon_image(H, W, 40, seed)
    ctrl, hws, hole = bands_with_fraction(H, W, 20, seed, (1.5, 7.5), fraction)
    rng = _rng(seed + 31337)
    bx = int(rng.integers(64, W - blob - 64))
    by = int(rng.integers(64, H - blob - 64))
    hole = hole | rect_mask(H, W, bx, by, blob, blob)
    return _finish(img, hole, poison=poison, splines=flatten_beziers(ctrl), half_widths=hws,
                   eps=4.0, blob_xy=(bx, by))


def batch_hole_fraction(seed: int) -> float:
    """The target hole fraction of batch frame ``seed`` (U[0.5%, 8%]), without
    building the frame."""
    return float(_rng(seed + 4242).uniform(0.005, 0.08))


def batch_frame(seed: int, poison: bool = False, H: int = 1080, W: int = 1920):
    """One frame of the uneven batch: hole fraction U[0.5%, 8%], band widths
    U[2, 40] px (half-widths U[1, 20])."""
    frac = batch_hole_fraction(seed)
    img = polygon_image(H, W, 40, seed)
    ctrl, hws, hole = bands_with_fraction(H, W, 20, seed, (1.0, 20.0), frac)
    return _finish(img, hole, poison=poison, splines=flatten_beziers(ctrl), half_widths=hws,
                   target_fraction=frac)


def batch_1080(n: int = 64, seed0: int = 100, poison: bool = False, H: int = 1080, W: int = 1920):
    """The batched workload: n frames, seeds seed0 .. seed0+n-1."""
    return [batch_frame(seed0 + i, poison=poison, H=H, W=W) for i in range(n)]


def diff_frame(seed: int, poison: bool = False, H: int = 512, W: int = 512):
    """One 512x512 frame of the differentiable workload: thin bands, ~5% of pixels."""
    img = polygon_image(H, W, 12, seed)
    ctrl, hws, hole = bands_with_fraction(H, W, 12, seed, (1.5, 4.5), 0.05, margin=24.0)
    return _finish(img, hole, poison=poison, splines=flatten_beziers(ctrl), half_widths=hws)


def diff_batch(n: int = 16, seed0: int = 200, poison: bool = False):
    return [diff_frame(seed0 + i, poison=poison) for i in range(n)]


def line_problem(H: int, poison: bool = False):
    """The line problem of the complexity validation (Section 7): image domain
    [0, 4] x [0, 1] rendered at (4H) x H px (pixel centres), a horizontal line
    0.45 <= y <= 0.55 of one colour on a background of another, hole
    D = [0.4, 3.96] x [0.2, 0.8]; no splines (guide field 0), smart order off."""
    W = 4 * H
    xc = (np.arange(W, dtype=np.float64) + 0.5) * (4.0 / W)
    yc = (np.arange(H, dtype=np.float64) + 0.5) * (1.0 / H)
    line = (yc >= 0.45) & (yc <= 0.55)
    img = np.empty((H, W, 3), np.float32)
    img[:] = np.array([0.1, 0.3, 0.8], np.float32)
    img[line] = np.array([0.9, 0.2, 0.1], np.float32)
    hole = ((yc >= 0.2) & (yc <= 0.8))[:, None] & ((xc >= 0.4) & (xc <= 3.96))[None, :]
    return _finish(img, hole, poison=poison, guide=np.zeros((H, W, 2), np.float32), smart=False)


def corridor(L: int = 2048, poison: bool = False):
    """A one-pixel-wide corridor of L hole pixels (row 1, x = 1..L) between two
    rows of bystanders, open to one known pixel at its left end (0, 1) and closed
    by a bystander at its right end: under onion order each step can fill only
    the next pixel of the corridor, so the fill takes exactly L steps of one
    pixel each (the per-step cost of the shell loop with no work in it).
    Guide field 0, smart order off."""
    H, W = 3, L + 2
    img = np.full((H, W, 3), 0.5, np.float32)
    img[1, 0] = (0.9, 0.2, 0.1)
    hole = np.zeros((H, W), bool)
    hole[1, 1:L + 1] = True
    byst = np.ones((H, W), bool)
    byst[1, 0:L + 1] = False
    return _finish(img, hole, byst, poison=poison, guide=np.zeros((H, W, 2), np.float32), smart=False)
