"""Theorem 1 (eqs. limitDirection, ctgf_limits) reproduced from the CUDA fill:
the transport direction of a straight edge continued into a half-plane hole
(Section 4 setting: data below, hole above, constant guidance, onion order) is
the centre of mass of the readable half ball under the weights -- for the
rotated ball of ghost pixels (Guidefill) and for the lattice ball (coherence
transport), at r = eps/h = 3 and 5."""
import math

import numpy as np
import pytest

import synth
from _gpu import gpu_fill

pytestmark = pytest.mark.gpu


def _g_star(theta_deg, mu, r, ghost):
    """Weighted centre of mass of the samples of the ball of radius r that lie in
    rows already filled (y >= 1, array coordinates, data below)."""
    th = math.radians(theta_deg)
    gh = (math.cos(th), math.sin(th))
    gp = (-gh[1], gh[0])
    sx = sy = sw = 0.0
    coef = mu * mu / (2.0 * r * r)
    for m in range(-r, r + 1):
        for n in range(-r, r + 1):
            if (n, m) == (0, 0) or n * n + m * m > r * r:
                continue
            if ghost:
                px, py, proj = n * gh[0] + m * gp[0], n * gh[1] + m * gp[1], m
            else:
                px, py, proj = n, m, -gh[1] * n + gh[0] * m
            if py < 1.0:
                continue
            w = math.exp(-coef * proj * proj) / math.hypot(n, m)
            sx, sy, sw = sx + w * px, sy + w * py, sw + w
    return sx / sw, sy / sw


def _gpu_edge_slope(theta_deg, mu, ghost, r, H=64, W=480, data_rows=8):
    th = math.radians(theta_deg)
    s_data = math.cos(th) / math.sin(th)
    hole = np.zeros((H, W), bool)
    hole[: H - data_rows] = True
    lab = synth.labels_from(hole)
    xs = np.arange(W)[None, :]
    ys = np.arange(H)[:, None]
    u = (xs < W / 2.0 + s_data * (ys - (H - 1))).astype(np.float32)
    img = np.repeat(u[..., None], 3, axis=2)
    g = synth.const_guide(H, W, theta_deg)
    f = gpu_fill(img, lab, g, eps=float(r), mu=mu, smart=False, ghost=ghost)["u"][..., 0].astype(np.float64)
    rows = list(range(6, H - data_rows - 12))
    cents = []
    for y in rows:
        p = f[y, :-1] - f[y, 1:]
        lo, hi = int(W * 0.3), int(W * 0.7)
        pw = p[lo:hi]
        cents.append(np.sum(pw * (np.arange(lo, hi) + 0.5)) / np.sum(pw))
    return np.polyfit(np.array(rows, float), np.array(cents), 1)[0]


@pytest.mark.parametrize("r", [3, 5])
@pytest.mark.parametrize("ghost", [True, False])
@pytest.mark.parametrize("theta", [45.0, 60.0, 73.0, 90.0, 110.0, 135.0])
def test_transport_direction_matches_theorem1(theta, ghost, r):
    gx, gy = _g_star(theta, 50.0, r, ghost)
    assert abs(_gpu_edge_slope(theta, 50.0, ghost, r) - gx / gy) < 2e-3


def test_guidefill_does_not_kink_where_coherence_transport_does():
    """Figure connectLine at r = 3 and 5: theta* = theta for the ghost ball,
    theta* pulled to a lattice direction for the lattice ball (73 degrees, mu = 50)."""
    target = math.cos(math.radians(73.0)) / math.sin(math.radians(73.0))
    assert abs(_gpu_edge_slope(73.0, 50.0, True, 3) - target) < 2e-3
    assert abs(_gpu_edge_slope(73.0, 50.0, False, 3) - target) > 0.1
    assert abs(_gpu_edge_slope(73.0, 50.0, True, 5) - target) < 2e-3
