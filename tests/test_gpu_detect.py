"""Automatic spline detection (Section 3.3) on the CUDA path against the oracle:
ring, Canny edges on the annulus, hysteresis, and the splines (base pixels and
end points bit-exact, coherence weights to 1e-6), at small ragged sizes, with
every parameter at its limits, batched, at the full 1920x1080 size of the
batched workload, and through to the guide field."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import hole_blobs
from synth import configs

pytestmark = pytest.mark.gpu

WEIGHT_RTOL = 1e-6  # tanh in FP64 on both sides, rounded once to FP32


def _gpu_detect_batched(imgs, labs, max_splines=4096, **kw):
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    dets = ctx.detect_splines_batched([torch.from_numpy(np.ascontiguousarray(i, np.float32)).cuda() for i in imgs],
                                      [torch.from_numpy(np.ascontiguousarray(l)).cuda() for l in labs],
                                      max_splines=max_splines, edges=True, **kw)
    torch.cuda.synchronize()
    out = []
    for d in dets:
        res = d.result.cpu().numpy()
        n = min(int(res[0]), max_splines)
        out.append(dict(count=int(res[0]), status=int(res[1]), pts=d.pts[:n].cpu().numpy(),
                        weight=d.weight[:n].cpu().numpy(), base=d.base[:n].cpu().numpy(),
                        offsets=d.offsets.cpu().numpy(), edges=d.edges.cpu().numpy()))
    return out


def _gpu_detect(img, lab, **kw):
    return _gpu_detect_batched([img], [lab], **kw)[0]


def _assert_detect_parity(o, g, max_splines=4096):
    assert g["status"] == 0
    assert g["count"] == o["count"], (g["count"], o["count"])
    np.testing.assert_array_equal(g["edges"], (o["edge"] == 2).astype(np.uint8))
    np.testing.assert_array_equal(g["base"], o["base"])
    np.testing.assert_array_equal(g["pts"], o["pts"])
    np.testing.assert_allclose(g["weight"], o["weight"], rtol=WEIGHT_RTOL, atol=0)
    n = o["count"]
    s = np.arange(max_splines + 1)
    np.testing.assert_array_equal(g["offsets"], 2 * np.minimum(s, n))


def _scene(H, W, seed, bystanders=True, poison=True):
    rng = np.random.default_rng(seed)
    img = synth.polygon_image(H, W, max(4, H * W // 6000), seed)
    hole = hole_blobs(H, W, seed, n=max(1, H * W // 4000), rmin=3, rmax=14)
    b = None
    if bystanders:
        b = np.zeros((H, W), bool)
        for _ in range(2):
            y0, x0 = rng.integers(0, H), rng.integers(0, W)
            b[y0:y0 + rng.integers(3, 12), x0:x0 + rng.integers(3, 12)] = True
        b &= ~hole
    lab = synth.labels_from(hole, b)
    if poison:
        img = img.copy()
        img[lab != 0] = np.nan  # never read by a ring pixel's tensor or an annulus pixel's gradient
    return img, lab


def _check(img, lab, max_splines=4096, **kw):
    o = oracle.detect_splines(img, lab, max_splines=max_splines, debug=True, **kw)
    g = _gpu_detect(img, lab, max_splines=max_splines, **kw)
    _assert_detect_parity(o, g, max_splines)
    return o, g


def test_paper_example_45_degrees():
    H = W = 96
    y, x = np.mgrid[0:H, 0:W]
    img = np.where((x - 48) > (y - 60), 1.0, 0.5).astype(np.float32)[..., None].repeat(3, 2)
    lab = np.zeros((H, W), np.uint8)
    lab[60:] = 1
    o, g = _check(img, lab, sigma=2.0, rho=4.0)
    assert g["count"] >= 1


@pytest.mark.parametrize("H,W,seed", [(64, 64, 1), (97, 129, 2), (200, 333, 3), (130, 70, 4)])
def test_random_scenes_ragged_sizes(H, W, seed):
    o, g = _check(*_scene(H, W, seed))
    assert g["count"] > 0


@pytest.mark.parametrize("kw", [
    dict(sigma=1.0, rho=2.0, annulus=0),
    dict(sigma=4.0, rho=8.0, annulus=4),  # largest windows
    dict(sigma=1.5, rho=3.0, ring_dist=20, annulus=6, length=10.0),
    dict(t_high=0.0, t_low=0.0),          # every suppression survivor is strong
    dict(t_high=0.2, t_low=0.01, Lambda=0.5),  # long hysteresis chains, unsaturated weights
])
def test_parameters_at_their_limits(kw):
    _check(*_scene(180, 210, 11), **kw)


def test_largest_distance_cap():
    # ring_dist + annulus = 96: a small hole at the centre, the ring 90 px out
    img = synth.polygon_image(200, 200, 12, 12)
    lab = np.zeros((200, 200), np.uint8)
    lab[96:104, 95:106] = 1
    _, g = _check(img, lab, sigma=0.5, rho=0.5, ring_dist=90, annulus=6)
    assert g["count"] > 0


def test_degenerate_frames():
    rng = np.random.default_rng(7)
    # no hole: no ring, no edges, no splines
    img = rng.random((50, 60, 3), dtype=np.float32)
    _, g = _check(img, np.zeros((50, 60), np.uint8))
    assert g["count"] == 0 and not g["edges"].any()
    # hole everywhere
    _, g = _check(img, np.ones((50, 60), np.uint8))
    assert g["count"] == 0
    # constant image
    lab = np.zeros((50, 60), np.uint8)
    lab[20:30, 20:40] = 1
    _, g = _check(np.full((50, 60, 3), 0.25, np.float32), lab)
    assert g["count"] == 0
    # frames smaller than a tile, single rows and columns, a hole at the border
    for H, W in ((20, 17), (1, 90), (90, 1), (33, 33)):
        img = synth.polygon_image(H, W, 3, H * 100 + W) if H > 1 and W > 1 else rng.random((H, W, 3), dtype=np.float32)
        lab = np.zeros((H, W), np.uint8)
        lab[: max(1, H // 4), : max(1, W // 3)] = 1
        _check(img, lab, t_high=0.0, t_low=0.0, sigma=1.0, rho=1.0)


def test_truncation_keeps_the_first_splines_in_raster_order():
    img, lab = _scene(200, 240, 21)
    full = oracle.detect_splines(img, lab, t_high=0.0, t_low=0.0)
    assert full["count"] > 10
    for m in (0, 1, 7):
        o = oracle.detect_splines(img, lab, max_splines=m, debug=True, t_high=0.0, t_low=0.0)
        g = _gpu_detect(img, lab, max_splines=m, t_high=0.0, t_low=0.0)
        _assert_detect_parity(o, g, m)
        assert g["count"] == full["count"]


def test_batched_frames_of_different_sizes():
    scenes = [_scene(H, W, s) for H, W, s in ((64, 96, 31), (150, 40, 32), (120, 200, 33), (33, 65, 34))]
    gs = _gpu_detect_batched([s[0] for s in scenes], [s[1] for s in scenes])
    for (img, lab), g in zip(scenes, gs):
        _assert_detect_parity(oracle.detect_splines(img, lab, debug=True), g)


def test_full_size_frame_of_the_batched_workload():
    d = configs.batch_frame(100, poison=True)
    o = oracle.detect_splines(d["rgb"], d["labels"], debug=True)
    g = _gpu_detect(d["rgb"], d["labels"])
    _assert_detect_parity(o, g)
    assert g["count"] > 50


def test_batched_launch_equals_single_launches_on_the_workload():
    # a property that holds at any size: the 16-frame launch gives every frame
    # what a launch of that frame alone gives
    fr = [configs.batch_frame(100 + i, poison=True, H=540, W=960) for i in range(16)]
    gb = _gpu_detect_batched([f["rgb"] for f in fr], [f["labels"] for f in fr])
    for f, g in zip(fr[:4], gb[:4]):
        gs = _gpu_detect(f["rgb"], f["labels"])
        for k in ("count", "status"):
            assert g[k] == gs[k]
        for k in ("pts", "weight", "base", "edges", "offsets"):
            np.testing.assert_array_equal(g[k], gs[k])
    o = oracle.detect_splines(fr[9]["rgb"], fr[9]["labels"], debug=True)
    _assert_detect_parity(o, gb[9])


def test_guide_field_from_detected_splines():
    import torch

    import paper_1611_05319_gb300 as gf
    img, lab = _scene(160, 200, 41)
    kw = dict(t_high=0.02, t_low=0.01, Lambda=0.05)  # weights below 1 at weak edges
    o = oracle.detect_splines(img, lab, **kw)
    assert (o["weight"] < 1.0).any()
    n = o["count"]
    go = oracle.guidance(lab, 2 * np.arange(n + 1, dtype=np.int32), o["pts"].reshape(-1, 2), eta=3.0,
                         weight=o["weight"])
    gg, det = gf.context(0).guidance_auto_batched([torch.from_numpy(img).cuda()], [torch.from_numpy(lab).cuda()],
                                                  eta=3.0, max_splines=512, **kw)
    gg = gg[0].cpu().numpy()
    assert det[0].count() == n
    np.testing.assert_array_equal(gg != 0, go != 0)
    np.testing.assert_allclose(gg, go, rtol=2e-6, atol=1e-30)
    # unweighted splines through the same entry point give the unit-weight field
    g1 = gf.context(0).guidance(torch.from_numpy(lab).cuda(), 2 * np.arange(n + 1, dtype=np.int32),
                                o["pts"].reshape(-1, 2))
    np.testing.assert_array_equal(g1.cpu().numpy(), oracle.guidance(lab, 2 * np.arange(n + 1, dtype=np.int32),
                                                                     o["pts"].reshape(-1, 2), eta=3.0))


def test_argument_errors_launch_nothing():
    import torch

    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import GuidefillError
    img = torch.zeros((40, 40, 4), device="cuda")
    lab = torch.zeros((40, 40), dtype=torch.uint8, device="cuda")
    ctx = gf.context(0)
    for bad in (dict(sigma=0.0), dict(sigma=4.5), dict(rho=9.0), dict(annulus=17), dict(annulus=14),
                dict(ring_dist=95, annulus=2), dict(length=0.0), dict(Lambda=0.0), dict(t_high=float("nan"))):
        with pytest.raises(GuidefillError):
            ctx.detect_splines(img, lab, **bad)


@pytest.mark.parametrize("seed", [100, 102])
def test_detected_guidance_through_the_fill(seed):
    # the paper's automatic pipeline end to end: splines detected on the frame,
    # their guide field, the fill; each side from its own detection (Lambda = 1e-5
    # saturates every weight to 1, so the two guide fields agree exactly)
    import torch

    import paper_1611_05319_gb300 as gf
    from _gpu import assert_parity, oracle_fill
    f = configs.batch_frame(seed, poison=True, H=270, W=480)
    img, lab = f["rgb"], f["labels"]
    o = oracle.detect_splines(img, lab)
    n = o["count"]
    go = oracle.guidance(lab, 2 * np.arange(n + 1, dtype=np.int32), o["pts"].reshape(-1, 2), eta=3.0,
                         weight=o["weight"])
    assert ((np.abs(go).sum(-1) > 0) & (lab == 1)).sum() > 1000
    ctx = gf.context(0)
    gg, det = ctx.guidance_auto_batched([torch.from_numpy(img).cuda()], [torch.from_numpy(lab).cuda()], eta=3.0)
    assert det[0].count() == n
    gg = gg[0]
    np.testing.assert_array_equal(gg.cpu().numpy(), go)
    r = ctx.fill(torch.from_numpy(synth.to_rgba(img)).cuda(), torch.from_numpy(lab).cuda(), gg, enter=True, stall=True)
    torch.cuda.synchronize()
    g = dict(u=r.rgba.cpu().numpy(), shell=r.shell.cpu().numpy(), enter=r.enter.cpu().numpy(), stats=r.stats(),
             stall_steps=r.stall_steps())
    ref = oracle_fill(img, lab, go, eps=3.0, mu=50.0, c=0.05)
    assert_parity(ref, g, lab)


def test_bench_launch_64_frames_sampled():
    # the launch the benchmark times: all 64 frames of the 1920x1080 batch in one
    # call; two frames checked in full against the oracle, every frame's count,
    # offsets and base order checked for validity
    fr = [configs.batch_frame(100 + i, poison=False) for i in range(64)]
    gb = _gpu_detect_batched([f["rgb"] for f in fr], [f["labels"] for f in fr])
    for i in (7, 41):
        _assert_detect_parity(oracle.detect_splines(fr[i]["rgb"], fr[i]["labels"], debug=True), gb[i])
    for f, g in zip(fr, gb):
        assert g["status"] == 0 and g["count"] > 0
        assert (np.diff(g["base"]) > 0).all()  # raster order, no duplicates
        lab = f["labels"].reshape(-1)
        assert (lab[g["base"]] == 0).all()  # bases are known pixels
        v = g["pts"][:, 1] - g["pts"][:, 0]
        np.testing.assert_allclose(np.hypot(v[:, 0], v[:, 1]), 48.0, rtol=1e-5)
