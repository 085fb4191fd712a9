"""Pins of the oracle's adjoint (frozen-schedule reverse sweep) -- no GPU.

The reverse sweep is checked against quantities computed without it: the
frozen forward (which must reproduce Algorithm 1's fill), the transpose
identity <w, J v> = <J^T w, v> for the colour Jacobian (the fill is linear in
the known colours with the schedule fixed), and central finite differences of
the FP64 frozen forward for the guidance angle and mu.
"""
import numpy as np
import pytest

import oracle
import synth


def _problem(seed, H=40, W=44, mu=10.0, band=False):
    rng = np.random.default_rng(seed)
    if band:
        hole = np.zeros((H, W), bool)
        hole[14:22, :] = True
        g = synth.const_guide(H, W, 0.0)
    else:
        yy, xx = np.mgrid[0:H, 0:W]
        hole = np.zeros((H, W), bool)
        for _ in range(5):
            cx, cy, r = rng.uniform(6, W - 6), rng.uniform(6, H - 6), rng.uniform(2, 6)
            hole |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
        g = synth.random_guide(H, W, seed + 1, zero_fraction=0.1)
    lab = synth.labels_from(hole)
    u = rng.uniform(0, 1, (H, W, 3))
    gt = rng.uniform(0, 1, (H, W, 3))
    f = oracle.fill(u, lab, g, eps=3.0, mu=mu, c=0.05)
    return lab, g, u, gt, f


def _loss(out, gt):
    return 0.5 * float(np.sum((out - gt) ** 2))


@pytest.mark.parametrize("seed", [1, 2])
def test_frozen_forward_reproduces_the_fill(seed):
    lab, g, u, gt, f = _problem(seed)
    out = oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], eps=3.0, mu=10.0)
    assert np.abs(out - f["u"]).max() < 1e-5  # FP64 vs FP32-rounded ghost positions


@pytest.mark.parametrize("seed,band", [(3, False), (4, False), (5, True)])
def test_colour_adjoint_is_the_transpose(seed, band):
    lab, g, u, gt, f = _problem(seed, band=band)
    if band:
        assert f["stats"]["stalls"] > 0
    rng = np.random.default_rng(seed + 100)
    v = rng.normal(size=u.shape) * (lab == 0)[..., None]
    w = rng.normal(size=u.shape)
    Jv = oracle.frozen_fill(u + v, lab, g, f["shell"], f["stall_steps"], mu=10.0) - \
        oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], mu=10.0)
    gi, _, _ = oracle.fill_backward(f["u"], lab, g, f["shell"], f["stall_steps"], w, mu=10.0)
    lhs, rhs = float(np.sum(w * Jv)), float(np.sum(gi * v))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    # filled hole pixels: their input colour is never used
    assert np.all(gi[f["shell"] >= 0] == 0.0)


@pytest.mark.parametrize("seed", [6, 7])
def test_angle_gradient_matches_central_differences(seed):
    lab, g, u, gt, f = _problem(seed)
    phi0 = np.arctan2(g[..., 1].astype(np.float64), g[..., 0].astype(np.float64))
    out0 = oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], mu=10.0, phi=phi0)
    _, gphi, _ = oracle.fill_backward(out0, lab, g, f["shell"], f["stall_steps"], out0 - gt, mu=10.0)
    rng = np.random.default_rng(seed)
    filled = np.argwhere((f["shell"] >= 0) & (np.hypot(g[..., 0], g[..., 1]) > 0))
    pick = filled[rng.choice(len(filled), 20, replace=False)]
    h = 1e-6
    for y, x in pick:
        ph = phi0.copy()
        ph[y, x] += h
        lp = _loss(oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], mu=10.0, phi=ph), gt)
        ph[y, x] -= 2 * h
        lm = _loss(oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], mu=10.0, phi=ph), gt)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gphi[y, x]) <= 1e-6 + 1e-5 * abs(fd), (y, x, fd, gphi[y, x])


@pytest.mark.parametrize("mu", [3.0, 10.0])
def test_mu_gradient_matches_central_differences(mu):
    lab, g, u, gt, f = _problem(8, mu=mu)
    out0 = oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], mu=mu)
    _, _, gmu = oracle.fill_backward(out0, lab, g, f["shell"], f["stall_steps"], out0 - gt, mu=mu)
    h = 1e-6
    lp = _loss(oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], mu=mu + h), gt)
    lm = _loss(oracle.frozen_fill(u, lab, g, f["shell"], f["stall_steps"], mu=mu - h), gt)
    fd = (lp - lm) / (2 * h)
    assert abs(gmu) > 1e-6
    assert abs(fd - gmu) <= 1e-6 * max(1.0, abs(fd)), (fd, gmu)


def test_stall_pixels_carry_no_angle_or_mu_gradient():
    lab, g, u, gt, f = _problem(9, band=True)
    stall = np.zeros(f["stats"]["shells"], bool)
    stall[:len(f["stall_steps"])] = f["stall_steps"].astype(bool)
    _, gphi, _ = oracle.fill_backward(f["u"], lab, g, f["shell"], f["stall_steps"], f["u"] - gt, mu=10.0)
    sh = f["shell"]
    at_stall = (sh >= 0) & stall[np.clip(sh, 0, None)]
    assert at_stall.any()
    assert np.all(gphi[at_stall] == 0.0)
