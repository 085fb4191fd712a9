"""Pins of the spline-detection oracle (Section 3.3) against facts that do not
come from the oracle: the worked example of Section 3.3.1, closed forms,
library routines for the special cases they cover (chessboard distance
transform, separable correlation, connected components, symmetric eigensolver)
and geometric invariants."""
import math

import numpy as np
import pytest

import oracle

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def _half_plane_45(H=96, W=96, hole_row=60):
    """Section 3.3.1: inpaint the lower half plane; above it white below a 45
    degree line and grey above it (here in image coordinates, rows down)."""
    y, x = np.mgrid[0:H, 0:W]
    img = np.where((x - 48) > (y - hole_row), 1.0, 0.5).astype(np.float32)[..., None].repeat(3, 2)
    lab = np.zeros((H, W), np.uint8)
    lab[hole_row:] = 1
    return img, lab


def test_paper_example_structure_tensor_gives_45_degrees():
    # sigma = 2, rho = 4 as in the example; the ordinary structure tensor at a
    # point far enough from the hole gives the correct 45 degrees
    img, lab = _half_plane_45()
    r = oracle.detect_splines(img, lab, sigma=2.0, rho=4.0)
    assert r["count"] >= 1
    for p, w in zip(r["pts"], r["weight"]):
        v = p[1] - p[0]
        assert abs(math.degrees(math.atan2(v[1], v[0])) - 45.0) < 0.5
        assert p[1][1] > p[0][1]  # points into the hole (down)
        assert abs(float(np.hypot(*v)) - 48.0) < 1e-3
        assert w == 1.0  # tanh saturates: lambda+ - lambda- >> 1e-5 at a real edge
    # the base lies on the ring dR = ceil(2 sigma) + ceil(2 rho) + 2 = 14 rows above the hole
    assert set(int(b) // 96 for b in r["base"]) == {60 - 14}


def test_gaussian_taps_and_window():
    for s in (0.7, 1.0, 2.0, 2.5, 4.0):
        w = oracle.gauss_taps(s)
        r = math.ceil(2 * s)
        assert len(w) == 2 * r + 1  # window 4 s + 1 for integer s
        i = np.arange(-r, r + 1)
        ref = np.exp(-i * i / (2.0 * s * s))
        np.testing.assert_allclose(w, ref / ref.sum(), rtol=3e-7, atol=0)


def test_distance_maps_are_chessboard_distances():
    rng = np.random.default_rng(5)
    H, W = 70, 90
    lab = np.zeros((H, W), np.uint8)
    for _ in range(4):
        y0, x0 = rng.integers(0, H - 10), rng.integers(0, W - 10)
        lab[y0:y0 + rng.integers(2, 12), x0:x0 + rng.integers(2, 12)] = rng.integers(1, 3)
    lab[5, 5] = 1
    lab[60, 80] = 2
    img = rng.random((H, W, 3), dtype=np.float32)
    r = oracle.detect_splines(img, lab, debug=True, annulus=2)
    cap = 14 + 2 + 1
    ref_h = scipy_ndimage.distance_transform_cdt((lab != 1).astype(np.int32), metric="chessboard")
    ref_a = scipy_ndimage.distance_transform_cdt((lab == 0).astype(np.int32), metric="chessboard")
    np.testing.assert_array_equal(r["d_hole"], np.minimum(ref_h, cap + 1))
    np.testing.assert_array_equal(r["d_all"], np.minimum(ref_a, cap + 1))


def test_smoothing_is_separable_clamped_correlation():
    rng = np.random.default_rng(6)
    H, W = 40, 53
    img = rng.random((H, W, 3), dtype=np.float32)
    lab = np.zeros((H, W), np.uint8)
    lab[18:22, 20:30] = 1
    for s in (1.0, 2.0, 3.0):
        r = oracle.detect_splines(img, lab, sigma=s, debug=True)
        w = oracle.gauss_taps(s).astype(np.float64)
        ref = scipy_ndimage.correlate1d(img.astype(np.float64), w, axis=1, mode="nearest")
        ref = scipy_ndimage.correlate1d(ref, w, axis=0, mode="nearest")
        np.testing.assert_allclose(r["us"], ref, rtol=0, atol=2e-6)


def test_tensor_of_a_linear_ramp_is_the_gradient_outer_product():
    # u_c = a_c x + b_c y + o_c: away from the border grad u_sigma = (a_c, b_c),
    # T = J = sum_c (a_c, b_c) (x) (a_c, b_c); v- is perpendicular to the
    # dominant gradient; lambda+ - lambda- from the closed form
    H, W = 64, 64
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    a = np.array([0.010, -0.004, 0.006])
    b = np.array([0.003, 0.002, 0.009])
    o = np.array([0.2, 0.5, 0.1])
    img = (a[None, None] * x[..., None] + b[None, None] * y[..., None] + o).astype(np.float32)
    lab = np.zeros((H, W), np.uint8)
    lab[28:36, 28:36] = 1
    r = oracle.detect_splines(img, lab, debug=True, sigma=1.0, rho=2.0)
    Txx, Txy, Tyy = (a * a).sum(), (a * b).sum(), (b * b).sum()
    inner = (slice(12, 52), slice(12, 52))
    for k, ref in enumerate((Txx, Txy, Tyy)):
        np.testing.assert_allclose(r["T"][inner][..., k], ref, rtol=2e-4, atol=1e-9)
        np.testing.assert_allclose(r["J"][inner][..., k], ref, rtol=2e-4, atol=1e-9)
    # ring of a square hole: 4 (s + 2 dR) - 4 pixels at chessboard distance dR = 1 .. 2 + 4 + 2
    dR = 2 + 4 + 2
    ring = (lab == 0) & (r["d_hole"] == dR) & (r["d_all"] == dR)
    assert ring.sum() == 4 * (8 + 2 * dR) - 4
    lam = np.linalg.eigh(np.array([[Txx, Txy], [Txy, Tyy]]))
    vmin = lam[1][:, 0]
    for p, w in zip(r["pts"], r["weight"]):
        v = (p[1] - p[0]) / np.linalg.norm(p[1] - p[0])
        assert abs(abs(float(v @ vmin)) - 1.0) < 1e-4
        assert w == np.float32(math.tanh((lam[0][1] - lam[0][0]) / 1e-5))


def test_coherence_weight_and_minor_eigenvector_match_eigh():
    # a weak edge and a large Lambda so that tanh does not saturate
    rng = np.random.default_rng(8)
    H, W = 80, 80
    y, x = np.mgrid[0:H, 0:W]
    img = (0.5 + 0.02 * np.tanh((x - 0.6 * y - 20) / 3.0))[..., None].repeat(3, 2).astype(np.float32)
    img += rng.normal(0, 0.001, img.shape).astype(np.float32)
    lab = np.zeros((H, W), np.uint8)
    lab[50:, :] = 1
    r = oracle.detect_splines(img, lab, debug=True, t_high=0.004, t_low=0.002, Lambda=2e-4)
    assert r["count"] >= 1
    for p, w, bse in zip(r["pts"], r["weight"], r["base"]):
        J = r["J"].reshape(-1, 3)[bse].astype(np.float64)
        lam, vec = np.linalg.eigh(np.array([[J[0], J[1]], [J[1], J[2]]]))
        assert 0.0 < w < 1.0
        assert abs(w - math.tanh((lam[1] - lam[0]) / 2e-4)) < 2e-6
        v = (p[1] - p[0]) / np.linalg.norm(p[1] - p[0])
        assert abs(abs(float(v @ vec[:, 0])) - 1.0) < 1e-5
        assert p[1][1] > p[0][1]


def test_non_maximum_suppression_keeps_the_ridge_column():
    # a vertical ramp edge symmetric about column 40: the gradient magnitude has
    # a unique maximum per row there, so only column 40 survives suppression
    H, W = 64, 80
    x = np.arange(W)
    prof = np.clip((x - 40) / 4.0 + 0.5, 0.0, 1.0)
    img = np.broadcast_to(prof[None, :, None], (H, W, 3)).astype(np.float32).copy()
    lab = np.zeros((H, W), np.uint8)
    lab[40:, :] = 1
    r = oracle.detect_splines(img, lab, debug=True)
    cols = np.unique(np.nonzero(r["edge_nms"])[1])
    assert cols.tolist() == [40]
    assert r["count"] == 1 and int(r["base"][0]) % W == 40
    p = r["pts"][0]
    assert p[1][0] == p[0][0] and p[1][1] > p[0][1]  # straight down into the hole


def test_hysteresis_is_the_union_of_components_with_a_strong_pixel():
    rng = np.random.default_rng(22)
    H, W = 120, 120
    y, x = np.mgrid[0:H, 0:W]
    img = np.zeros((H, W, 3), np.float32)
    for k in range(12):
        ang = rng.uniform(0, np.pi)
        c = rng.uniform(0.02, 0.3)
        off = rng.uniform(-60, 60)
        img += (c * ((np.cos(ang) * (x - 60) + np.sin(ang) * (y - 60) - off) > 0))[..., None]
    img += rng.normal(0, 0.01, img.shape).astype(np.float32)
    lab = np.zeros((H, W), np.uint8)
    lab[40:80, 35:85] = 1
    r = oracle.detect_splines(img, lab, debug=True, annulus=3, t_high=0.05, t_low=0.01)
    pre = r["edge_nms"]
    assert (pre == 1).any() and (pre == 2).any()
    comp, n = scipy_ndimage.label(pre > 0, structure=np.ones((3, 3), int))
    strong = np.unique(comp[pre == 2])
    ref = np.isin(comp, strong[strong > 0])
    np.testing.assert_array_equal(r["edge"] > 0, ref)
    # the case needs the diagonal links: with 4-connectivity fewer pixels are kept
    comp4, _ = scipy_ndimage.label(pre > 0)
    assert (np.isin(comp4, np.unique(comp4[pre == 2])) != ref).sum() > 10
    # the splines are the ring pixels among the kept edge pixels, in raster order
    dR = 14
    ring = (lab == 0) & (r["d_hole"] == dR) & (r["d_all"] == dR)
    np.testing.assert_array_equal(r["base"], np.flatnonzero(ring & ref))


def test_radial_edges_give_radial_splines_into_the_hole():
    # 12 angular sectors of different colours around the centre of a square
    # hole: the edges are radial, so every spline points at the centre
    H, W = 160, 160
    y, x = np.mgrid[0:H, 0:W]
    cx = cy = 79.5
    ang = np.arctan2(y - cy, x - cx)
    sector = np.floor((ang + np.pi) / (2 * np.pi / 12)).astype(int) % 12
    pal = np.random.default_rng(10).random((12, 3)).astype(np.float32)
    img = pal[sector]
    lab = np.zeros((H, W), np.uint8)
    lab[60:100, 60:100] = 1
    r = oracle.detect_splines(img, lab, length=30.0)
    assert r["count"] >= 12
    for p in r["pts"]:
        v = (p[1] - p[0]) / np.linalg.norm(p[1] - p[0])
        rad = np.array([cx, cy]) - p[0]
        rad /= np.linalg.norm(rad)
        assert float(v @ rad) > math.cos(math.radians(6.0))


def test_bystanders_keep_the_ring_away():
    rng = np.random.default_rng(11)
    H, W = 100, 100
    img = rng.random((H, W, 3), dtype=np.float32)
    lab = np.zeros((H, W), np.uint8)
    lab[40:60, 40:60] = 1
    lab[40:60, 62:70] = 2  # a bystander object beside the hole
    r = oracle.detect_splines(img, lab, debug=True, t_high=0.0, t_low=0.0)
    ring = (lab == 0) & (r["d_hole"] == 14) & (r["d_all"] == 14)
    near_b = scipy_ndimage.distance_transform_cdt((lab != 2).astype(np.int32), metric="chessboard") < 14
    assert not (ring & near_b).any()
    for b in r["base"]:
        assert ring.reshape(-1)[b]
    assert not (r["edge_nms"][lab != 0]).any()


def test_degenerate_inputs():
    H, W = 50, 60
    img = np.full((H, W, 3), 0.3, np.float32)
    lab = np.zeros((H, W), np.uint8)
    lab[20:30, 20:30] = 1
    assert oracle.detect_splines(img, lab)["count"] == 0  # no edges
    img2 = np.random.default_rng(12).random((H, W, 3), dtype=np.float32)
    assert oracle.detect_splines(img2, np.zeros((H, W), np.uint8))["count"] == 0  # no hole
    full = oracle.detect_splines(img2, lab, t_high=0.0, t_low=0.0)
    part = oracle.detect_splines(img2, lab, t_high=0.0, t_low=0.0, max_splines=3)
    assert part["count"] == full["count"] > 3
    np.testing.assert_array_equal(part["base"], full["base"][:3])
    with pytest.raises(ValueError):
        oracle.detect_splines(img2, lab, sigma=0.0)


def test_weighted_guidance_scales_each_splines_field():
    H, W = 64, 64
    lab = np.zeros((H, W), np.uint8)
    lab[16:48, 8:56] = 1
    pts = np.array([[10, 20], [54, 22], [10, 44], [54, 40]], np.float32)
    off = np.array([0, 2, 4], np.int32)
    wt = np.array([0.25, 0.8], np.float32)
    g1 = oracle.guidance(lab, off, pts, eta=3.0)
    gw = oracle.guidance(lab, off, pts, eta=3.0, weight=wt)
    top = np.zeros((H, W), bool)
    top[16:32] = True
    np.testing.assert_allclose(gw[top], g1[top] * 0.25, rtol=2e-7, atol=1e-30)
    np.testing.assert_allclose(gw[~top], g1[~top] * np.float32(0.8), rtol=2e-7, atol=1e-30)
    assert np.abs(g1).max() > 0.9
