"""Seeded synthetic inputs for the Guidefill shell fill.

This module is the only code shared by the CPU oracle side and the CUDA side.
It draws images, hole / bystander labels and spline polylines; it contains none
of the method's arithmetic (no weights, no ghost-pixel geometry, no guidance
field, no distance-to-polyline computation).  Every function is deterministic
for a given seed (numpy PCG64 via ``default_rng``).

Conventions shared by every caller:
  * images are float32 ``[H, W, C]`` (C = 3 RGB or 4 RGBA), values in [0, 1];
  * labels are uint8 ``[H, W]``: 0 known, 1 hole (inpainting domain D_h),
    2 bystander (B_h, Section 2.1 of the paper);
  * pixel (x, y) has centre at integer coordinates, x = column, y = row;
  * a polyline set is ``(offsets int32[n+1], pts float32[P, 2])``: polyline i
    uses points ``pts[offsets[i]:offsets[i+1]]`` as (x, y).
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

KNOWN, HOLE, BYSTANDER = 0, 1, 2


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------
def polygon_image(H: int, W: int, n_polys: int, seed: int, noise_sigma: float = 0.01,
                  channels: int = 3) -> np.ndarray:
    """Piecewise-smooth image: random convex polygons, each with its own linear
    colour gradient, painted in order over a linear-gradient background, plus
    N(0, noise_sigma) noise, clamped to [0, 1]."""
    rng = _rng(seed)
    ys = np.arange(H, dtype=np.float32)[:, None]
    xs = np.arange(W, dtype=np.float32)[None, :]
    img = np.empty((H, W, channels), np.float32)
    base = rng.uniform(0.2, 0.8, channels)
    gx = rng.uniform(-0.2, 0.2, channels)
    gy = rng.uniform(-0.2, 0.2, channels)
    for ch in range(channels):
        img[:, :, ch] = base[ch] + gx[ch] * (xs / W) + gy[ch] * (ys / H)
    s = float(min(H, W))
    for _ in range(n_polys):
        nv = int(rng.integers(3, 8))
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        r = rng.uniform(0.05, 0.3) * s
        ang = np.sort(rng.uniform(0, 2 * np.pi, nv))
        sx, sy = rng.uniform(0.5, 1.5), rng.uniform(0.5, 1.5)
        rot = rng.uniform(0, 2 * np.pi)
        px = r * sx * np.cos(ang)
        py = r * sy * np.sin(ang)
        vx = cx + px * np.cos(rot) - py * np.sin(rot)
        vy = cy + px * np.sin(rot) + py * np.cos(rot)
        c0 = rng.uniform(0.0, 1.0, channels)
        cgx = rng.uniform(-0.5, 0.5, channels)
        cgy = rng.uniform(-0.5, 0.5, channels)
        x0, x1 = int(max(0, np.floor(vx.min()))), int(min(W, np.ceil(vx.max()) + 1))
        y0, y1 = int(max(0, np.floor(vy.min()))), int(min(H, np.ceil(vy.max()) + 1))
        if x0 >= x1 or y0 >= y1:
            continue
        X = xs[:, x0:x1]
        Y = ys[y0:y1, :]
        inside = np.ones((y1 - y0, x1 - x0), bool)
        # vertices are in angular order of an affine image of a circle: convex;
        # orientation sign is taken from the polygon's signed area
        area = 0.5 * np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy)
        sgn = 1.0 if area >= 0 else -1.0
        for i in range(nv):
            ax, ay = vx[i], vy[i]
            bx, by = vx[(i + 1) % nv], vy[(i + 1) % nv]
            cross = (bx - ax) * (Y - ay) - (by - ay) * (X - ax)
            inside &= (sgn * cross) >= 0
        for ch in range(channels):
            val = c0[ch] + cgx[ch] * (X - cx) / r + cgy[ch] * (Y - cy) / r
            sub = img[y0:y1, x0:x1, ch]
            sub[inside] = np.broadcast_to(val, inside.shape)[inside]
    if noise_sigma > 0:
        img += rng.normal(0.0, noise_sigma, img.shape).astype(np.float32)
    np.clip(img, 0.0, 1.0, out=img)
    return img


def to_rgba(img: np.ndarray) -> np.ndarray:
    """Pads an RGB float32 image with an alpha channel equal to 1."""
    if img.shape[2] == 4:
        return np.ascontiguousarray(img, dtype=np.float32)
    out = np.ones(img.shape[:2] + (4,), np.float32)
    out[:, :, :3] = img
    return out


# --------------------------------------------------------------------------
# splines
# --------------------------------------------------------------------------
def _bezier(ctrl: np.ndarray, t: np.ndarray) -> np.ndarray:
    p0, p1, p2, p3 = ctrl
    u = 1.0 - t
    return ((u ** 3)[:, None] * p0 + (3 * u * u * t)[:, None] * p1
            + (3 * u * t * t)[:, None] * p2 + (t ** 3)[:, None] * p3)


def random_beziers(n: int, H: int, W: int, seed: int, scale: float, margin: float = 40.0):
    """n cubic Bezier control polygons ([n, 4, 2] float64).  Each curve starts at
    a uniform point inside the frame minus ``margin``; the three further control
    points follow a random walk of step ``scale`` (with jitter), clipped to the
    same box, so every curve lies inside the frame."""
    rng = _rng(seed)
    lo = np.array([margin, margin])
    hi = np.array([W - 1 - margin, H - 1 - margin])
    out = np.empty((n, 4, 2))
    for i in range(n):
        p = rng.uniform(lo, hi)
        heading = rng.uniform(0, 2 * np.pi)
        pts = [p]
        for _ in range(3):
            heading += rng.normal(0.0, 0.6)
            step = scale * rng.uniform(0.6, 1.4) / 3.0
            p = np.clip(p + step * np.array([np.cos(heading), np.sin(heading)]), lo, hi)
            pts.append(p)
        out[i] = np.array(pts)
    return out


def flatten_beziers(ctrl: np.ndarray, n_seg: int = 64):
    """Flattens Beziers into polylines of n_seg segments each (uniform in t)."""
    t = np.linspace(0.0, 1.0, n_seg + 1)
    pts = np.concatenate([_bezier(c, t) for c in ctrl]).astype(np.float32)
    offsets = np.arange(0, (n_seg + 1) * (len(ctrl) + 1), n_seg + 1, dtype=np.int32)
    return offsets, pts


def band_mask(H: int, W: int, ctrl: np.ndarray, half_widths) -> np.ndarray:
    """Union of bands: pixels within half_widths[i] of Bezier i.  The curve is
    sampled densely, its samples are rounded to pixels and a Euclidean distance
    transform of that raster gives the band (a pixel-quantised centreline)."""
    mask = np.zeros((H, W), bool)
    for c, hw in zip(ctrl, half_widths):
        length = np.sum(np.linalg.norm(np.diff(c, axis=0), axis=1)) + 1.0
        t = np.linspace(0.0, 1.0, int(length * 4) + 2)
        p = _bezier(c, t)
        pad = int(np.ceil(hw)) + 2
        x0 = max(0, int(np.floor(p[:, 0].min())) - pad)
        x1 = min(W, int(np.ceil(p[:, 0].max())) + pad + 1)
        y0 = max(0, int(np.floor(p[:, 1].min())) - pad)
        y1 = min(H, int(np.ceil(p[:, 1].max())) + pad + 1)
        grid = np.ones((y1 - y0, x1 - x0), bool)
        ix = np.clip(np.rint(p[:, 0]).astype(int) - x0, 0, x1 - x0 - 1)
        iy = np.clip(np.rint(p[:, 1]).astype(int) - y0, 0, y1 - y0 - 1)
        grid[iy, ix] = False
        dist = ndimage.distance_transform_edt(grid)
        mask[y0:y1, x0:x1] |= dist <= hw
    return mask


def bands_with_fraction(H: int, W: int, n: int, seed: int, half_width_range, target_fraction: float,
                        margin: float = 40.0, iters: int = 3):
    """Bezier bands whose union covers about ``target_fraction`` of the frame.
    The walk step is rescaled a few times (deterministically) to approach the
    target.  Returns (ctrl, half_widths, mask)."""
    rng = _rng(seed + 7919)
    hws = rng.uniform(half_width_range[0], half_width_range[1], n)
    scale = 0.25 * min(H, W)
    for _ in range(iters):
        ctrl = random_beziers(n, H, W, seed, scale, margin)
        mask = band_mask(H, W, ctrl, hws)
        frac = mask.mean()
        if frac <= 0:
            scale *= 2.0
            continue
        scale = float(np.clip(scale * target_fraction / frac, 8.0, 4.0 * max(H, W)))
    ctrl = random_beziers(n, H, W, seed, scale, margin)
    mask = band_mask(H, W, ctrl, hws)
    return ctrl, hws, mask


# --------------------------------------------------------------------------
# masks / labels / simple guidance fields
# --------------------------------------------------------------------------
def annulus_mask(H: int, W: int, r_in: float, r_out: float, cx: float | None = None,
                 cy: float | None = None) -> np.ndarray:
    cx = (W - 1) / 2.0 if cx is None else cx
    cy = (H - 1) / 2.0 if cy is None else cy
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = (xx - cx) ** 2 + (yy - cy) ** 2
    return (d2 >= r_in * r_in) & (d2 <= r_out * r_out)


def rect_mask(H: int, W: int, x0: int, y0: int, w: int, h: int) -> np.ndarray:
    m = np.zeros((H, W), bool)
    m[max(0, y0):min(H, y0 + h), max(0, x0):min(W, x0 + w)] = True
    return m


def labels_from(hole: np.ndarray, bystander: np.ndarray | None = None) -> np.ndarray:
    lab = np.zeros(hole.shape, np.uint8)
    if bystander is not None:
        lab[bystander] = BYSTANDER
    lab[hole] = HOLE
    return lab


def const_guide(H: int, W: int, theta_deg: float, magnitude: float = 1.0) -> np.ndarray:
    """Constant guidance vector magnitude*(cos theta, sin theta), float32 [H, W, 2],
    computed in float64 and rounded once."""
    th = np.deg2rad(np.float64(theta_deg))
    g = np.empty((H, W, 2), np.float32)
    g[:, :, 0] = np.float32(magnitude * np.cos(th))
    g[:, :, 1] = np.float32(magnitude * np.sin(th))
    return g


def random_guide(H: int, W: int, seed: int, zero_fraction: float = 0.2) -> np.ndarray:
    """Random guidance vectors (uniform angle, magnitude U[0, 1]) with a random
    subset set exactly to zero; used by edge-case tests."""
    rng = _rng(seed)
    ang = rng.uniform(0, 2 * np.pi, (H, W))
    mag = rng.uniform(0, 1, (H, W))
    mag[rng.uniform(0, 1, (H, W)) < zero_fraction] = 0.0
    g = np.stack([mag * np.cos(ang), mag * np.sin(ang)], -1).astype(np.float32)
    return g
