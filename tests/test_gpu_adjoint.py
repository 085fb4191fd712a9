"""Adjoint kernel vs the oracle's FP64 reverse sweep and FP64 finite
differences of the oracle's frozen forward (needs a GB300)."""
import numpy as np
import pytest

import oracle
import synth
from synth import configs

from _gpu import rgba

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ctx(cuda_device):
    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import build
    build.build()
    return gf.context(0)


def _angle_problem(seed, H=128, W=128, mu=10.0, band=False):
    """Differentiable workload at a given size: thin bands, guide from the band
    splines re-expressed as magnitude and angle."""
    f = configs.diff_frame(seed, H=H, W=W)
    lab = f["labels"]
    if band:
        lab = np.zeros((H, W), np.uint8)
        lab[H // 2 - 4:H // 2 + 4, :] = 1
        g0 = synth.const_guide(H, W, 0.0) * (lab == 1)[..., None]
    else:
        g0 = oracle.guidance(lab, *f["splines"], eta=3.0)
    mag = np.hypot(g0[..., 0].astype(np.float64), g0[..., 1].astype(np.float64)).astype(np.float32)
    phi = np.arctan2(g0[..., 1].astype(np.float64), g0[..., 0].astype(np.float64)).astype(np.float32)
    guide = np.zeros((H, W, 2), np.float32)
    hole = lab == 1
    guide[..., 0][hole] = (mag.astype(np.float64) * np.cos(phi.astype(np.float64))).astype(np.float32)[hole]
    guide[..., 1][hole] = (mag.astype(np.float64) * np.sin(phi.astype(np.float64))).astype(np.float32)[hole]
    img = rgba(f["gt"])
    gt = rgba(f["gt"])
    return img, lab, mag, phi, guide, gt


def _gpu_fwd_bwd(img, lab, mag, phi, grad_out, mu, eps=3.0):
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    lab_t = torch.from_numpy(lab).cuda()
    g = ctx.guide_from_angle(lab_t, torch.from_numpy(mag).cuda(), torch.from_numpy(phi).cuda())
    r = ctx.fill_batched([torch.from_numpy(img).cuda()], [lab_t], [g], eps=eps, mu=mu, stall=True, enter=True)
    gi, gp, gmu = ctx.fill_backward(r, [g], [torch.from_numpy(grad_out.astype(np.float32)).cuda()], eps=eps, mu=mu)
    torch.cuda.synchronize()
    return dict(guide=g.cpu().numpy(), u=r[0].rgba.cpu().numpy(), shell=r[0].shell.cpu().numpy(),
                stats=r[0].stats(), gi=gi[0].cpu().numpy(), gphi=gp[0].cpu().numpy(), gmu=float(gmu[0]))


# Per-pixel bound on the angle gradient: |g_gpu - g_oracle| <= ANG_RTOL * max(|g_oracle|, floor)
# with floor = ANG_FLOOR * max |g_oracle| over the frame (below the floor the FP32
# sums' absolute error, a few ulp of the largest terms times the number of steps,
# dominates any relative bound).
ANG_RTOL, ANG_FLOOR = 1e-3, 1e-2


def assert_angle_grad(got, want):
    """Element by element; reports the worst pixel."""
    top = float(np.abs(want).max())
    if top == 0.0:
        assert np.abs(got).max() == 0.0
        return 0.0
    den = np.maximum(np.abs(want), ANG_FLOOR * top)
    rel = np.abs(got - want) / den
    i = np.unravel_index(int(np.argmax(rel)), rel.shape)
    assert rel[i] <= ANG_RTOL, f"worst pixel {i}: gpu {got[i]} oracle {want[i]} (rel {rel[i]:.2e}, max {top:.3e})"
    return float(rel[i])


def test_guide_from_angle_bitexact():
    img, lab, mag, phi, guide, gt = _angle_problem(201)
    r = _gpu_fwd_bwd(img, lab, mag, phi, np.zeros_like(img), 10.0)
    hole = lab == 1
    assert np.array_equal(r["guide"][hole], guide[hole])


@pytest.mark.parametrize("seed,mu,band", [(202, 10.0, False), (203, 50.0, False), (204, 3.0, False),
                                          (205, 10.0, True)])
def test_adjoint_matches_oracle_reverse_sweep(seed, mu, band):
    img, lab, mag, phi, guide, gt = _angle_problem(seed, mu=mu, band=band)
    o = oracle.fill(img, lab, guide, eps=3.0, mu=mu)
    grad_out = np.random.default_rng(seed).normal(size=img.shape)
    r = _gpu_fwd_bwd(img, lab, mag, phi, grad_out, mu)
    assert np.array_equal(r["shell"], o["shell"])
    if band:
        assert o["stats"]["stalls"] > 0
    gi, gphi, gmu = oracle.fill_backward(o["u"], lab, guide, o["shell"], o["stall_steps"], grad_out, eps=3.0, mu=mu)
    scale = np.abs(gi).max()
    assert np.abs(r["gi"] - gi).max() <= 1e-4 * max(1.0, scale)
    assert_angle_grad(r["gphi"], gphi)
    assert abs(r["gmu"] - gmu) <= 1e-3 * max(abs(gmu), 1e-6) + 1e-6


def test_fd_on_64x64_crop():
    """FP64 central differences of the oracle's frozen forward (loss 1/2 |u - gt|^2)
    against the GPU gradients for the angle at 24 pixels and for mu."""
    mu = 10.0
    img, lab, mag, phi, guide, gt = _angle_problem(206, H=64, W=64, mu=mu)
    o = oracle.fill(img, lab, guide, eps=3.0, mu=mu)
    r = _gpu_fwd_bwd(img, lab, mag, phi, (o["u"] - gt), mu)
    assert np.array_equal(r["shell"], o["shell"])

    def loss(**kw):
        u = oracle.frozen_fill(img, lab, guide, o["shell"], o["stall_steps"], eps=3.0, **kw)
        return 0.5 * float(np.sum((u - gt) ** 2))

    phi0 = np.arctan2(guide[..., 1].astype(np.float64), guide[..., 0].astype(np.float64))
    rng = np.random.default_rng(7)
    cand = np.argwhere((o["shell"] >= 0) & (mag > 0.05))
    pick = cand[rng.choice(len(cand), min(24, len(cand)), replace=False)]
    h = 1e-6
    fd, got = [], []
    for y, x in pick:
        ph = phi0.copy()
        ph[y, x] += h
        lp = loss(mu=mu, phi=ph)
        ph[y, x] -= 2 * h
        lm = loss(mu=mu, phi=ph)
        fd.append((lp - lm) / (2 * h))
        got.append(r["gphi"][y, x])
    fd, got = np.array(fd), np.array(got)
    # each sampled pixel on its own: relative 1e-3 above a floor of 1e-2 of the largest
    assert_angle_grad(got, fd)
    fdm = (loss(mu=mu + 1e-5, phi=phi0) - loss(mu=mu - 1e-5, phi=phi0)) / 2e-5
    assert abs(fdm - r["gmu"]) <= 1e-3 * abs(fdm) + 1e-7, (fdm, r["gmu"])


def test_autograd_function_batch():
    import torch

    from paper_1611_05319_gb300.autograd import guidefill_fill
    probs = [_angle_problem(210 + i, H=96, W=112) for i in range(3)]
    img = torch.from_numpy(np.stack([p[0] for p in probs])).cuda().requires_grad_(True)
    lab = torch.from_numpy(np.stack([p[1] for p in probs])).cuda()
    mag = torch.from_numpy(np.stack([p[2] for p in probs])).cuda()
    phi = torch.from_numpy(np.stack([p[3] for p in probs])).cuda().requires_grad_(True)
    gt = torch.from_numpy(np.stack([p[5] for p in probs])).cuda()
    mu = torch.tensor(10.0, requires_grad=True)
    out = guidefill_fill(img, lab, mag, phi, mu)
    loss = 0.5 * ((out - gt) ** 2).sum()
    loss.backward()
    for i, p in enumerate(probs):
        o = oracle.fill(p[0], p[1], p[4], eps=3.0, mu=10.0)
        gi, gphi, gmu = oracle.fill_backward(o["u"], p[1], p[4], o["shell"], o["stall_steps"], o["u"] - p[5],
                                             eps=3.0, mu=10.0)
        assert np.abs(img.grad[i].cpu().numpy() - gi).max() <= 1e-4 * max(1.0, np.abs(gi).max())
        assert_angle_grad(phi.grad[i].cpu().numpy(), gphi)
    assert mu.grad is not None and np.isfinite(float(mu.grad))


def test_differentiable_config_two_frames_of_sixteen():
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    frames = configs.diff_batch(16)
    probs = []
    for f in frames:
        lab = f["labels"]
        g0 = oracle.guidance(lab, *f["splines"], eta=3.0)
        mag = np.hypot(g0[..., 0].astype(np.float64), g0[..., 1].astype(np.float64)).astype(np.float32)
        phi = np.arctan2(g0[..., 1].astype(np.float64), g0[..., 0].astype(np.float64)).astype(np.float32)
        probs.append((rgba(f["gt"]), lab, mag, phi))
    lab_t = [torch.from_numpy(p[1]).cuda() for p in probs]
    guides = [ctx.guide_from_angle(lab_t[i], torch.from_numpy(p[2]).cuda(), torch.from_numpy(p[3]).cuda())
              for i, p in enumerate(probs)]
    res = ctx.fill_batched([torch.from_numpy(p[0]).cuda() for p in probs], lab_t, guides, mu=50.0, stall=True)
    grads = [(r.rgba - torch.from_numpy(p[0]).cuda()) for r, p in zip(res, probs)]
    gi, gp, gmu = ctx.fill_backward(res, guides, grads, mu=50.0)
    torch.cuda.synchronize()
    for i in (0, 15):
        p = probs[i]
        hole = p[1] == 1
        guide = np.zeros(p[1].shape + (2,), np.float32)  # the CPU's own FP64 evaluation, rounded once
        guide[..., 0][hole] = (p[2].astype(np.float64) * np.cos(p[3].astype(np.float64))).astype(np.float32)[hole]
        guide[..., 1][hole] = (p[2].astype(np.float64) * np.sin(p[3].astype(np.float64))).astype(np.float32)[hole]
        assert np.array_equal(guides[i].cpu().numpy()[hole], guide[hole])
        o = oracle.fill(p[0], p[1], guide, eps=3.0, mu=50.0)
        assert np.array_equal(o["shell"], res[i].shell.cpu().numpy())
        go = o["u"] - p[0]
        ogi, ogp, ogm = oracle.fill_backward(o["u"], p[1], guide, o["shell"], o["stall_steps"], go, eps=3.0,
                                             mu=50.0)
        assert np.abs(gi[i].cpu().numpy() - ogi).max() <= 1e-4 * max(1.0, np.abs(ogi).max())
        assert_angle_grad(gp[i].cpu().numpy(), ogp)
        assert abs(float(gmu[i]) - ogm) <= 1e-3 * abs(ogm) + 1e-6
        if i == 0:
            # FP64 central difference of the loss in mu on the whole 512 x 512 frame
            # (frozen schedule, the adjoint's semantics), against the GPU's d/dmu
            def loss(m):
                u = oracle.frozen_fill(p[0], p[1], guide, o["shell"], o["stall_steps"], eps=3.0, mu=m)
                return 0.5 * float(np.sum((u - p[0]) ** 2))
            h = 1e-4
            fdm = (loss(50.0 + h) - loss(50.0 - h)) / (2 * h)
            assert fdm != 0.0
            assert abs(float(gmu[i]) - fdm) <= 1e-3 * abs(fdm), (float(gmu[i]), fdm)
