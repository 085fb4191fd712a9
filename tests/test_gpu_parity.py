"""CUDA path vs the CPU oracle on the same seeded inputs (needs a GB300).

Bar: shell indices and front-entry steps bit-exact, per-frame counts equal,
colours within 1e-4 max-abs of the FP64 oracle.  Inputs at hole and bystander
pixels are NaN: the fill must never read them.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import configs

from _gpu import assert_guide_parity, assert_parity, gpu_fill, hole_blobs, oracle_fill, rgba

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ctx(cuda_device):
    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import build
    build.build()
    return gf.context(0)


def _case(H, W, seed, byst=0.03, zero_g=0.2, n=None, rmax=7):
    rng = np.random.default_rng(seed)
    n = n if n is not None else max(1, H * W // 300)
    hole = hole_blobs(H, W, seed, n=n, rmax=rmax, margin=3)
    b = (rng.uniform(0, 1, (H, W)) < byst) & ~hole
    lab = synth.labels_from(hole, b)
    img = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    img[lab != 0] = np.nan
    g = synth.random_guide(H, W, seed + 1, zero_fraction=zero_g)
    return img, lab, g


def test_plain_128_annulus():
    d = configs.plain_128(poison=True)
    o = oracle_fill(d["rgb"], d["labels"], d["guide"], eps=3.0, mu=50.0, c=0.05)
    g = gpu_fill(d["rgb"], d["labels"], d["guide"], eps=3.0, mu=50.0, c=0.05)
    assert_parity(o, g, d["labels"])
    assert g["stats"]["status"] == 0


@pytest.mark.parametrize("H,W", [(37, 53), (64, 64), (8, 8), (5, 200), (200, 5), (129, 131), (1, 1), (2, 9)])
@pytest.mark.parametrize("eps", [3.0, 4.0])
def test_random_frames_ragged(H, W, eps):
    img, lab, g = _case(H, W, 1000 + H * 7 + W)
    o = oracle_fill(img, lab, g, eps=eps, mu=50.0)
    r = gpu_fill(img, lab, g, eps=eps, mu=50.0)
    assert_parity(o, r, lab)


@pytest.mark.parametrize("eps", [1.0, 1.5, 2.5, 3.3, 5.0, 6.5, 7.0])
@pytest.mark.parametrize("mu", [0.0, 10.0, 50.0])
def test_eps_mu_grid(eps, mu):
    img, lab, g = _case(48, 56, int(eps * 100 + mu))
    o = oracle_fill(img, lab, g, eps=eps, mu=mu)
    r = gpu_fill(img, lab, g, eps=eps, mu=mu)
    assert_parity(o, r, lab)


@pytest.mark.parametrize("ghost", [True, False])
@pytest.mark.parametrize("smart", [True, False])
@pytest.mark.parametrize("rescan", [False, True])
def test_flags(ghost, smart, rescan):
    img, lab, g = _case(60, 72, 77 + ghost + 2 * smart)
    o = oracle_fill(img, lab, g, eps=3.0, mu=10.0, ghost=ghost, smart=smart)
    r = gpu_fill(img, lab, g, eps=3.0, mu=10.0, ghost=ghost, smart=smart, rescan=rescan)
    assert_parity(o, r, lab)


def test_rescan_equals_tracking_and_counts_every_front_pixel():
    d = configs.plain_128(poison=True)
    a = gpu_fill(d["rgb"], d["labels"], d["guide"], rescan=False)
    b = gpu_fill(d["rgb"], d["labels"], d["guide"], rescan=True)
    o = oracle_fill(d["rgb"], d["labels"], d["guide"])
    assert np.array_equal(a["shell"], b["shell"]) and np.array_equal(a["enter"], b["enter"])
    # Same fills; the colours agree to FP32 rounding (the lanes that share a pixel's
    # samples follow the tile's front-pixel count, which a rescan sees larger).
    assert np.nanmax(np.abs(a["u"] - b["u"])) <= 2e-6
    assert b["stats"]["evaluations"] == o["stats"]["evaluations"]  # rescan evaluates the whole front every step
    assert a["stats"]["evaluations"] < b["stats"]["evaluations"]


@pytest.mark.parametrize("c", [1e-6, 0.05, 0.3, 0.9])
def test_confidence_thresholds(c):
    img, lab, g = _case(50, 50, 5)
    o = oracle_fill(img, lab, g, eps=3.0, mu=5.0, c=c)
    r = gpu_fill(img, lab, g, eps=3.0, mu=5.0, c=c)
    assert_parity(o, r, lab)


def test_stall_rule_band_across_image():
    H, W = 24, 40
    hole = np.zeros((H, W), bool)
    hole[8:16, :] = True
    lab = synth.labels_from(hole)
    g = synth.const_guide(H, W, 0.0)
    img = np.random.default_rng(9).uniform(0, 1, (H, W, 3)).astype(np.float32)
    img[hole] = np.nan
    o = oracle_fill(img, lab, g, mu=50.0)
    r = gpu_fill(img, lab, g, mu=50.0)
    assert o["stats"]["stalls"] > 0
    assert_parity(o, r, lab)


@pytest.mark.parametrize("cs", [4, 16])
def test_corridor_one_pixel_per_step(cs):
    """The benchmark's per-step floor workload: a one-pixel corridor walled by
    bystanders fills one pixel per step under onion order."""
    import torch

    import paper_1611_05319_gb300 as gf
    d = configs.corridor(300, poison=True)
    ctx = gf.Context(0)
    ctx.set_launch_config(cs, 1)
    lab = d["labels"]
    r = ctx.fill(torch.from_numpy(rgba(d["rgb"])).cuda(), torch.from_numpy(lab).cuda(),
                 torch.from_numpy(d["guide"]).cuda(), smart=False, enter=True, stall=True)
    torch.cuda.synchronize()
    g = dict(u=r.rgba.cpu().numpy(), shell=r.shell.cpu().numpy(), enter=r.enter.cpu().numpy(), stats=r.stats(),
             stall_steps=r.stall_steps())
    o = oracle_fill(d["rgb"], lab, d["guide"], smart=False)
    assert o["stats"]["shells"] == 300 and o["stats"]["max_front"] == 1
    assert_parity(o, g, lab)
    ctx.close()


def test_walled_region_incomplete():
    H, W = 30, 30
    hole = synth.rect_mask(H, W, 5, 5, 8, 8) | synth.rect_mask(H, W, 20, 20, 3, 3)
    byst = synth.rect_mask(H, W, 19, 19, 5, 5) & ~synth.rect_mask(H, W, 20, 20, 3, 3)
    lab = synth.labels_from(hole, byst)
    img = np.random.default_rng(3).uniform(0, 1, (H, W, 3)).astype(np.float32)
    img[lab == 2] = np.nan
    g = synth.random_guide(H, W, 4)
    o = oracle_fill(img, lab, g)
    r = gpu_fill(img, lab, g)
    assert_parity(o, r, lab)
    assert r["stats"]["status"] == 1 and (r["shell"][20:23, 20:23] == -2).all()


def test_all_hole_and_no_hole():
    H, W = 20, 28
    g = synth.random_guide(H, W, 1)
    img = np.random.default_rng(2).uniform(0, 1, (H, W, 3)).astype(np.float32)
    lab = np.ones((H, W), np.uint8)
    r = gpu_fill(img, lab, g)
    assert r["stats"]["filled"] == 0 and r["stats"]["status"] == 1 and (r["shell"] == -2).all()
    lab0 = np.zeros((H, W), np.uint8)
    r0 = gpu_fill(img, lab0, g)
    assert r0["stats"]["filled"] == 0 and r0["stats"]["status"] == 0 and (r0["shell"] == -1).all()
    assert np.array_equal(r0["u"][..., :3], img)


def test_hole_touching_every_border():
    H, W = 33, 47
    hole = np.zeros((H, W), bool)
    hole[:4, :] = True
    hole[-3:, :] = True
    hole[:, :2] = True
    hole[:, -5:] = True
    lab = synth.labels_from(hole)
    img = np.random.default_rng(4).uniform(0, 1, (H, W, 3)).astype(np.float32)
    img[hole] = np.nan
    g = synth.random_guide(H, W, 5)
    o = oracle_fill(img, lab, g)
    r = gpu_fill(img, lab, g)
    assert_parity(o, r, lab)


@pytest.mark.parametrize("cs", [1, 2, 4, 8, 16])
def test_launch_shape_does_not_change_results(cs):
    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    d = configs.plain_128(poison=True)
    o = oracle_fill(d["rgb"], d["labels"], d["guide"])
    if ctx.max_active_clusters(3.0, cs) <= 0:
        pytest.skip(f"cluster size {cs} not schedulable")
    ctx.set_launch_config(cluster_size=cs)
    try:
        r = gpu_fill(d["rgb"], d["labels"], d["guide"])
        assert ctx.last_launch()[0] == cs
    finally:
        ctx.set_launch_config(0)
    assert_parity(o, r, d["labels"])


def test_batched_mixed_sizes_and_params():
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    cases = [_case(H, W, 300 + i) for i, (H, W) in enumerate([(40, 40), (17, 93), (128, 64), (9, 9), (70, 71)])]
    res = ctx.fill_batched([torch.from_numpy(rgba(c[0])).cuda() for c in cases],
                           [torch.from_numpy(c[1]).cuda() for c in cases],
                           [torch.from_numpy(c[2]).cuda() for c in cases], eps=3.0, mu=20.0, enter=True, stall=True)
    torch.cuda.synchronize()
    for (img, lab, g), r in zip(cases, res):
        gg = dict(u=r.rgba.cpu().numpy(), shell=r.shell.cpu().numpy(), enter=r.enter.cpu().numpy(),
                  stats=r.stats(), stall_steps=r.stall_steps())
        o = oracle_fill(img, lab, g, eps=3.0, mu=20.0)
        assert_parity(o, gg, lab)


def test_in_place_and_host_buffers_match():
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    img, lab, g = _case(64, 80, 11)
    a = gpu_fill(img, lab, g)
    x = torch.from_numpy(rgba(img)).cuda()
    r = ctx.fill(x, torch.from_numpy(lab).cuda(), torch.from_numpy(g).cuda(), out="inplace")
    torch.cuda.synchronize()
    assert r.rgba.data_ptr() == x.data_ptr()
    assert np.array_equal(x.cpu().numpy()[a["shell"] >= 0], a["u"][a["shell"] >= 0])
    out_rgba = np.zeros((64, 80, 4), np.float32)
    out_shell = np.zeros((64, 80), np.int32)
    st = ctx.fill_batched_host([rgba(img)], [lab], [g], [out_rgba], [out_shell])
    assert np.array_equal(out_shell, a["shell"])
    assert np.array_equal(out_rgba[a["shell"] >= 0], a["u"][a["shell"] >= 0])
    assert st[0]["filled"] == a["stats"]["filled"]


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_in_place_moves_only_what_the_fill_touches(pinned):
    """In place on host buffers: pinned buffers take the sparse path (colours near
    the holes in, hole colours out, written by the device), pageable ones full
    copies; both leave the buffers exactly as the device-buffer fill leaves its
    output: hole pixels filled, every other pixel untouched (NaN bystanders,
    unreachable pixels included)."""
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    cases = [_case(96 + 8 * i, 136 - 5 * i, 700 + i) for i in range(5)]
    # frame 1: a walled region (unreachable pixels keep their colour); frame 3 takes
    # its guide field from splines
    im, lb, g = cases[1]
    lb = lb.copy()
    lb[10:19, 10:19] = 2
    lb[12:17, 12:17] = 1
    cases[1] = (im, lb, g)
    H3, W3 = cases[3][1].shape
    spl = {3: (np.array([0, 3], np.int32), np.array([[2.0, 2.0], [W3 / 2.0, H3 / 2.0], [W3 - 3.0, H3 - 3.0]],
                                                     np.float32))}
    dev = torch.device("cuda", 0)
    guides = [ctx.guidance(torch.from_numpy(lb).to(dev), *spl[i], 3.0).cpu().numpy() if i in spl else g
              for i, (_, lb, g) in enumerate(cases)]
    ref = ctx.fill_batched([torch.from_numpy(rgba(im)).to(dev) for im, _, _ in cases],
                           [torch.from_numpy(lb).to(dev) for _, lb, _ in cases],
                           [torch.from_numpy(np.ascontiguousarray(g, np.float32)).to(dev) for g in guides], mu=10.0)
    torch.cuda.synchronize()

    def host(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return (t.pin_memory() if pinned else t.clone()).numpy()
    bufs = [host(rgba(im)) for im, _, _ in cases]
    before = [b.copy() for b in bufs]
    labs = [host(lb) for _, lb, _ in cases]
    gds = [None if i in spl else host(np.ascontiguousarray(g, np.float32)) for i, (_, _, g) in enumerate(cases)]
    shells = [np.full(lb.shape, 9, np.int32) for _, lb, _ in cases]
    # later calls on the filled buffers give the same result, also through a HostBatch
    batch = gf.HostBatch(bufs, labs, gds, bufs, shells, splines=[spl.get(i) for i in range(5)])
    for rep in range(3):
        if rep == 0:
            st = ctx.fill_batched_host(bufs, labs, gds, bufs, shells, splines=[spl.get(i) for i in range(5)], eta=3.0,
                                       mu=10.0)
        else:
            st = ctx.fill_batched_host(batch, eta=3.0, mu=10.0)
        for i, r in enumerate(ref):
            sh = r.shell.cpu().numpy()
            assert np.array_equal(shells[i], sh), i
            filled = sh >= 0
            assert np.array_equal(bufs[i][filled], r.rgba.cpu().numpy()[filled]), i
            assert np.array_equal(np.nan_to_num(bufs[i][~filled], nan=-7.0),
                                  np.nan_to_num(before[i][~filled], nan=-7.0)), i
            assert st[i]["filled"] == r.stats()["filled"], i
    assert (shells[1][12:17, 12:17] == -2).all()


def test_repeated_calls_are_deterministic():
    d = configs.plain_128(poison=True)
    a = gpu_fill(d["rgb"], d["labels"], d["guide"])
    b = gpu_fill(d["rgb"], d["labels"], d["guide"])
    assert np.array_equal(a["shell"], b["shell"]) and np.array_equal(a["u"], b["u"])


# ---------------------------------------------------------------------------
# guide field from splines
# ---------------------------------------------------------------------------
def _gpu_guidance(lab, off, pts, eta):
    import torch

    import paper_1611_05319_gb300 as gf
    g = gf.context(0).guidance(torch.from_numpy(lab).cuda(), off, pts, eta)
    torch.cuda.synchronize()
    return g.cpu().numpy()


def test_guidance_small_bitexact():
    H, W = 90, 130
    ctrl = synth.random_beziers(5, H, W, 3, 40.0, margin=5)
    off, pts = synth.flatten_beziers(ctrl, 16)
    lab = synth.labels_from(synth.band_mask(H, W, ctrl, [6.0] * 5))
    ties = oracle.guidance_ties(lab, off, pts, 3.0)
    gg = _gpu_guidance(lab, off, pts, 3.0)
    assert_guide_parity(ties, gg, lab)


def test_guidance_overflowing_bins_bitexact():
    """Many short segments through one bin: the bin list overflows and the
    kernel scans every segment of the frame."""
    H, W = 64, 64
    t = np.linspace(0, 2 * np.pi, 200)
    pts = np.stack([32 + 10 * np.cos(t), 32 + 10 * np.sin(t)], 1).astype(np.float32)
    off = np.array([0, 200], np.int32)
    lab = np.ones((H, W), np.uint8)
    ties = oracle.guidance_ties(lab, off, pts, 2.0)
    gg = _gpu_guidance(lab, off, pts, 2.0)
    assert_guide_parity(ties, gg, lab)


# ---------------------------------------------------------------------------
# full-size workloads (launch configuration of the benchmark)
# ---------------------------------------------------------------------------
def test_frame_1080_full_size_sampler_and_fill():
    d = configs.frame_1080(poison=True)
    lab = d["labels"]
    ties = oracle.guidance_ties(lab, *d["splines"], eta=3.0)
    go = ties["guide"]
    gg = _gpu_guidance(lab, *d["splines"], eta=3.0)
    assert_guide_parity(ties, gg, lab)
    assert ties["min_gap"] > oracle.SEG_TIE_PX
    o = oracle_fill(d["rgb"], lab, go)
    assert o["stats"]["min_margin"] > 1e-10
    r = gpu_fill(d["rgb"], lab, go)
    assert_parity(o, r, lab)


@pytest.mark.slow
def test_frame_4k_blob_full_size():
    d = configs.frame_4k_blob(poison=True)
    lab = d["labels"]
    go = oracle.guidance(lab, *d["splines"], eta=3.0)
    o = oracle_fill(d["rgb"], lab, go, eps=4.0)
    for rescan in (False, True):
        r = gpu_fill(d["rgb"], lab, go, eps=4.0, rescan=rescan)
        assert_parity(o, r, lab)


def test_autotuned_launch_gives_identical_results():
    import ctypes as C

    import torch

    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import _lib
    ctx = gf.Context(0)
    cases = [_case(72, 96, 500 + i) for i in range(6)]
    imgs = [torch.from_numpy(rgba(c[0])).cuda() for c in cases]
    labs = [torch.from_numpy(c[1]).cuda() for c in cases]
    gds = [torch.from_numpy(c[2]).cuda() for c in cases]
    outs = [torch.empty_like(i) for i in imgs]
    shells = [torch.empty(c[1].shape, dtype=torch.int32, device="cuda") for c in cases]
    fr = (_lib.Frame * 6)()
    for i in range(6):
        fr[i] = _lib.Frame(72, 96, imgs[i].data_ptr(), labs[i].data_ptr(), gds[i].data_ptr(), outs[i].data_ptr(),
                           shells[i].data_ptr(), None, None)
    stats = torch.zeros((6 * _lib.STATS_BYTES,), dtype=torch.uint8, device="cuda")
    prm = _lib.make_params()
    cs, ms = ctx.autotune(fr, stats, prm, trials=1)
    assert cs in (1, 2, 4, 8, 16) and ms > 0
    ctx.fill_frames(fr, stats, prm)
    torch.cuda.synchronize()
    assert ctx.last_launch()[0] == cs
    for i, (img, lab, g) in enumerate(cases):
        o = oracle_fill(img, lab, g)
        assert np.array_equal(o["shell"], shells[i].cpu().numpy())
        filled = o["shell"] >= 0
        assert np.abs(o["u"][filled] - outs[i].cpu().numpy()[filled]).max() <= 1e-4
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("H", [70, 140])
def test_line_problem_of_the_complexity_validation(H):
    """Section 7's line problem (onion order, no splines) at the two smallest
    sizes of the complexity sweep: tracked and rescanned fills against the oracle."""
    d = configs.line_problem(H, poison=True)
    o = oracle_fill(d["rgb"], d["labels"], d["guide"], smart=False)
    for rescan in (False, True):
        r = gpu_fill(d["rgb"], d["labels"], d["guide"], smart=False, rescan=rescan)
        assert_parity(o, r, d["labels"])
    # onion order on a rectangle: one Chebyshev ring per step from both long sides
    rows = int(d["labels"].any(axis=1).sum())
    assert o["stats"]["shells"] == (rows + 1) // 2


def test_split_schedule_gives_identical_results():
    """The split schedule (largest holes on a second launch of larger clusters,
    beside the main launch) fills every frame exactly as one launch does."""
    import torch

    import paper_1611_05319_gb300 as gf
    frames = [_case(40 + 8 * i, 48 + 4 * i, 900 + i) for i in range(9)]
    dev = torch.device("cuda", 0)
    outs = []
    for split in ((0, 0, 0), (3, 8, 2), (1, 16, 1)):
        ctx = gf.Context(0)
        ctx.set_launch_config(2, 0)
        ctx.set_split(*split)
        rs = ctx.fill_batched([torch.from_numpy(rgba(im)).to(dev) for im, _, _ in frames],
                              [torch.from_numpy(lb).to(dev) for _, lb, _ in frames],
                              [torch.from_numpy(g).to(dev) for _, _, g in frames], eps=3.0, mu=10.0, enter=True)
        torch.cuda.synchronize()
        outs.append(([r.shell.cpu().numpy() for r in rs], [r.rgba.cpu().numpy() for r in rs],
                     [r.enter.cpu().numpy() for r in rs], [r.stats() for r in rs]))
        m, cs, nc = ctx.last_split()
        assert (m, cs) == (split[0], split[1]) and (nc > 0) == (split[0] > 0)
        ctx.close()
    for o in outs[1:]:
        for a, b in zip(outs[0][0], o[0]):
            assert np.array_equal(a, b)
        for a, b in zip(outs[0][1], o[1]):
            assert np.array_equal(a, b, equal_nan=True)
        for a, b in zip(outs[0][2], o[2]):
            assert np.array_equal(a, b)
        for a, b in zip(outs[0][3], o[3]):
            assert (a["shells"], a["filled"], a["status"]) == (b["shells"], b["filled"], b["status"])
    o = oracle_fill(*frames[8], eps=3.0, mu=10.0)
    assert np.array_equal(o["shell"], outs[1][0][8])


def test_host_buffer_pipeline_many_frames_matches_device_path():
    """The host-buffer call pipelines its frames over four chunks (frames dealt
    round-robin); seven frames of different sizes, some with guide fields and some
    with splines, must come back in order and equal the device-buffer fills."""
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    cases = [_case(40 + 6 * i, 56 + 2 * i, 400 + i) for i in range(7)]
    dev = torch.device("cuda", 0)
    # frames 1, 4 take their guide field from splines (a short diagonal polyline each)
    spl = {}
    for i in (1, 4):
        H, W = cases[i][1].shape
        pts = np.array([[2.0, 2.0], [W / 2.0, H / 2.0], [W - 3.0, H - 3.0]], np.float32)
        spl[i] = (np.array([0, 3], np.int32), pts)
    guides = []
    for i, (im, lb, g) in enumerate(cases):
        if i in spl:
            guides.append(ctx.guidance(torch.from_numpy(lb).to(dev), spl[i][0], spl[i][1], 3.0).cpu().numpy())
        else:
            guides.append(g)
    ref = ctx.fill_batched([torch.from_numpy(rgba(im)).to(dev) for im, _, _ in cases],
                           [torch.from_numpy(lb).to(dev) for _, lb, _ in cases],
                           [torch.from_numpy(np.ascontiguousarray(g, np.float32)).to(dev) for g in guides], mu=10.0)
    torch.cuda.synchronize()
    outs = [np.zeros(lb.shape + (4,), np.float32) for _, lb, _ in cases]
    shells = [np.zeros(lb.shape, np.int32) for _, lb, _ in cases]
    st = ctx.fill_batched_host([rgba(im) for im, _, _ in cases], [lb for _, lb, _ in cases],
                               [None if i in spl else g for i, (_, _, g) in enumerate(cases)], outs, shells,
                               splines=[spl.get(i) for i in range(7)], eta=3.0, mu=10.0)
    for i, r in enumerate(ref):
        sh = r.shell.cpu().numpy()
        assert np.array_equal(shells[i], sh), i
        assert np.array_equal(outs[i][sh >= 0], r.rgba.cpu().numpy()[sh >= 0]), i
        rs = r.stats()
        assert (st[i]["filled"], st[i]["shells"], st[i]["holes"]) == (rs["filled"], rs["shells"], rs["holes"]), i


@pytest.mark.parametrize("data_term", [False, True])
def test_fill_batched_splines_equals_guidance_then_fill(data_term):
    """gf_fill_batched_splines builds the guide fields beside the fill's preparation;
    the results equal the guide fields followed by the batched fill, bit for bit,
    and the guide fields themselves equal gf_guidance_batched's."""
    import ctypes as C

    import torch

    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import _lib
    from synth import configs, to_rgba
    ctx = gf.context(0)
    dev = torch.device("cuda", 0)
    fr_ = [configs.batch_frame(300 + i, poison=True, H=270, W=480) for i in range(6)]
    n = len(fr_)
    labs = [torch.from_numpy(f["labels"]).to(dev) for f in fr_]
    offs = [torch.from_numpy(f["splines"][0]).to(dev) for f in fr_]
    pts = [torch.from_numpy(f["splines"][1]).to(dev) for f in fr_]
    ref_g = ctx.guidance_batched(labs, [f["splines"][0] for f in fr_], [f["splines"][1] for f in fr_], 3.0)
    ref = ctx.fill_batched([torch.from_numpy(to_rgba(f["rgb"])).to(dev) for f in fr_], labs, ref_g, eps=3.0, mu=50.0,
                           c=0.05, data_term=data_term)
    torch.cuda.synchronize()
    imgs = [torch.from_numpy(to_rgba(f["rgb"])).to(dev) for f in fr_]
    guides = [torch.full((f["labels"].shape[0], f["labels"].shape[1], 2), 7.0, dtype=torch.float32, device=dev)
              for f in fr_]
    shells = [torch.empty(f["labels"].shape, dtype=torch.int32, device=dev) for f in fr_]
    stats = torch.zeros((n * _lib.STATS_BYTES,), dtype=torch.uint8, device=dev)
    frames = (_lib.Frame * n)()
    sfr = (_lib.SplineFrame * n)()
    for i, f in enumerate(fr_):
        H, W = f["labels"].shape
        frames[i] = _lib.Frame(H, W, imgs[i].data_ptr(), labs[i].data_ptr(), guides[i].data_ptr(), imgs[i].data_ptr(),
                               shells[i].data_ptr(), None, None)
        sfr[i] = _lib.SplineFrame(H, W, labs[i].data_ptr(), offs[i].numel() - 1, pts[i].shape[0], offs[i].data_ptr(),
                                  pts[i].data_ptr(), guides[i].data_ptr(), None)
    prm = _lib.make_params(eps=3.0, mu=50.0, c=0.05, data_term=data_term)
    L = _lib.lib()
    sp = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # the second call replays the cached graphs
        for im, f in zip(imgs, fr_):
            im.copy_(torch.from_numpy(to_rgba(f["rgb"])).to(dev))
        _lib.check(L.gf_fill_batched_splines(ctx._h, n, frames, sfr, C.c_float(3.0), C.byref(prm),
                                             C.c_void_p(stats.data_ptr()), sp, None, None), "fill_batched_splines",
                   ctx._h)
        torch.cuda.synchronize()
        st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=_lib.STATS_DTYPE)
        for i, r in enumerate(ref):
            lab = fr_[i]["labels"]
            hole = lab == 1
            assert np.array_equal(guides[i].cpu().numpy()[hole], ref_g[i].cpu().numpy()[hole]), i
            sh = r.shell.cpu().numpy()
            assert np.array_equal(shells[i].cpu().numpy(), sh), i
            assert np.array_equal(imgs[i].cpu().numpy()[sh >= 0], r.rgba.cpu().numpy()[sh >= 0]), i
            rs = r.stats()
            assert (st[i]["filled"], st[i]["shells"], st[i]["data_switch"]) == \
                (rs["filled"], rs["shells"], rs["data_switch"]), i
