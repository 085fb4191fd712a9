"""Pins of the CPU oracle to facts the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than its own code: hand
worked values, closed forms from Theorem 1, invariants of Algorithm 1, the
iteration bound of Theorem complexity2, brute-force restatements of set
definitions.  A plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed offset) breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
S2 = math.sqrt(2.0)


def _hole_blobs(H, W, seed, n=6, rmax=7, margin=4):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    hole = np.zeros((H, W), bool)
    for _ in range(n):
        cx, cy = rng.uniform(margin + rmax, W - margin - rmax), rng.uniform(margin + rmax, H - margin - rmax)
        r = rng.uniform(2, rmax)
        hole |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    return hole


# ----------------------------------------------------------------------------
# Hand-worked 3x3 hole (Algorithm 1, eq. weight, eqs. confidence / ready)
# ----------------------------------------------------------------------------
def _hand_case(seed=0):
    H = W = 7
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 1, (H, W, 3))
    hole = synth.rect_mask(H, W, 2, 2, 3, 3)
    lab = synth.labels_from(hole)
    g = np.zeros((H, W, 2), np.float32)
    return u, lab, g


def test_hand_3x3_shells_and_colours_c005():
    gold = json.load(open(os.path.join(HERE, "golden", "hand_3x3.json")))
    u, lab, g = _hand_case()
    r = oracle.fill(u, lab, g, eps=1.5, mu=50.0, c=0.05)
    assert np.array_equal(r["shell"][2:5, 2:5], np.array(gold["shell_c005"]))
    assert r["stats"]["shells"] == 2 and r["stats"]["stalls"] == 0
    # corner (2,2): readable = axial (2,1),(1,2); diagonal (1,1),(3,1),(1,3)
    w_ax, w_dg = 1.0, 1.0 / S2
    exp_corner = (w_ax * (u[1, 2] + u[2, 1]) + w_dg * (u[1, 1] + u[1, 3] + u[3, 1])) / (2 * w_ax + 3 * w_dg)
    assert np.allclose(r["u"][2, 2], exp_corner, atol=1e-14)
    # edge-middle (x=3, y=2): axial (3,1); diagonal (2,1),(4,1)
    exp_edge = (w_ax * u[1, 3] + w_dg * (u[1, 2] + u[1, 4])) / (w_ax + 2 * w_dg)
    assert np.allclose(r["u"][2, 3], exp_edge, atol=1e-14)
    # centre at step 1 from the eight step-0 values
    f = r["u"]
    exp_c = (w_ax * (f[2, 3] + f[4, 3] + f[3, 2] + f[3, 4]) + w_dg * (f[2, 2] + f[2, 4] + f[4, 2] + f[4, 4])) \
        / (4 * w_ax + 4 * w_dg)
    assert np.allclose(f[3, 3], exp_c, atol=1e-14)
    # confidence values of the hand derivation lie on the expected side of c
    assert abs((2 + 3 / S2) / (4 + 2 * S2) - 0.60355339) < 1e-8
    assert abs((1 + 2 / S2) / (4 + 2 * S2) - 0.35355339) < 1e-8


def test_hand_3x3_smart_order_threshold_c05():
    """c = 0.5 lies between the edge (0.354) and corner (0.604) confidences: the
    corners fill first, the edge-middles next (0.646), the centre last (its
    step-1 confidence is 0.414 < 0.5)."""
    gold = json.load(open(os.path.join(HERE, "golden", "hand_3x3.json")))
    u, lab, g = _hand_case(1)
    r = oracle.fill(u, lab, g, eps=1.5, mu=50.0, c=0.5)
    assert np.array_equal(r["shell"][2:5, 2:5], np.array(gold["shell_c05"]))
    f = r["u"]
    # edge-middle (x=3,y=2) at step 1: known (3,1) axial, (2,1),(4,1) diagonal; corners (2,2),(4,2) axial
    exp_edge = (u[1, 3] + f[2, 2] + f[2, 4] + (u[1, 2] + u[1, 4]) / S2) / (3 + 2 / S2)
    assert np.allclose(f[2, 3], exp_edge, atol=1e-14)
    # front entry: ring pixels at 0, centre at 1
    assert r["enter"][3, 3] == 1 and (r["enter"][2:5, 2:5] == np.array([[0, 0, 0], [0, 1, 0], [0, 0, 0]])).all()


def test_alg_bytes_hand_3x3():
    gold = json.load(open(os.path.join(HERE, "golden", "hand_3x3.json")))
    u, lab, g = _hand_case()
    r = oracle.fill(u, lab, g, eps=1.5, mu=50.0, c=0.05)
    assert oracle.alg_bytes(lab, g, 1.5, r["shell"], r["enter"]) == gold["alg_bytes_c005"]


# ----------------------------------------------------------------------------
# Invariants of Algorithm 1
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("ghost", [True, False])
@pytest.mark.parametrize("smart", [True, False])
def test_constant_image_stays_constant(ghost, smart):
    """Every fill is a normalised weighted average of bilinear values (a partition
    of unity), so a constant image stays constant (Algorithm 1, eq. bilinearDef)."""
    H, W = 40, 48
    hole = _hole_blobs(H, W, 3)
    rng = np.random.default_rng(5)
    byst = (rng.uniform(0, 1, (H, W)) < 0.05) & ~hole
    lab = synth.labels_from(hole, byst)
    g = synth.random_guide(H, W, 7)
    u = np.empty((H, W, 3))
    u[:] = [0.25, 0.5, 0.875]
    u[lab != 0] = np.nan  # never read
    r = oracle.fill(u, lab, g, eps=3.0, mu=10.0, c=0.05, ghost=ghost, smart=smart)
    filled = r["shell"] >= 0
    assert filled.sum() > 0
    assert np.allclose(r["u"][filled], [0.25, 0.5, 0.875], atol=1e-13)


def test_linear_in_known_colours():
    """The schedule depends only on g, eps, mu, c and the sets D^(k), B (eqs.
    confidence/ready), never on colours, so the output is linear in the known
    colours."""
    H, W = 36, 40
    hole = _hole_blobs(H, W, 11)
    lab = synth.labels_from(hole)
    g = synth.random_guide(H, W, 12)
    rng = np.random.default_rng(13)
    u1 = rng.uniform(0, 1, (H, W, 3))
    u2 = rng.uniform(0, 1, (H, W, 3))
    a, b = 0.3, -1.7
    r1 = oracle.fill(u1, lab, g, mu=10.0)
    r2 = oracle.fill(u2, lab, g, mu=10.0)
    r3 = oracle.fill(a * u1 + b * u2, lab, g, mu=10.0)
    assert np.array_equal(r1["shell"], r2["shell"]) and np.array_equal(r1["shell"], r3["shell"])
    assert np.allclose(r3["u"], a * r1["u"] + b * r2["u"], atol=1e-12)


def test_guide_sign_invariance():
    """g and -g give the same ball (symmetric under (n,m) -> (-n,-m)) and the same
    weights (even in g_perp.(y-x)), hence the same fill (eq. weight)."""
    H, W = 36, 44
    hole = _hole_blobs(H, W, 21)
    lab = synth.labels_from(hole)
    g = synth.random_guide(H, W, 22)
    rng = np.random.default_rng(23)
    u = rng.uniform(0, 1, (H, W, 3))
    r1 = oracle.fill(u, lab, g, mu=10.0)
    r2 = oracle.fill(u, lab, -g, mu=10.0)
    assert r1["stats"]["min_margin"] > 1e-9
    assert np.array_equal(r1["shell"], r2["shell"])
    assert np.allclose(r1["u"], r2["u"], atol=1e-12)


@pytest.mark.parametrize("vec", [(1.0, 0.0), (0.0, 1.0), (0.0, -0.6), (0.0, 0.0)])
def test_axis_aligned_guidance_ghost_equals_lattice(vec):
    """For g parallel to e1 or e2 (or g = 0), the rotated ball is the lattice ball
    and g_perp.(y - x) agrees, so Guidefill and coherence transport coincide
    (Notation: B~ = R(B); Section 4, g = 0 case)."""
    H, W = 30, 34
    hole = _hole_blobs(H, W, 31)
    lab = synth.labels_from(hole)
    g = np.zeros((H, W, 2), np.float32)
    g[..., 0], g[..., 1] = vec
    rng = np.random.default_rng(32)
    u = rng.uniform(0, 1, (H, W, 3))
    r1 = oracle.fill(u, lab, g, mu=10.0, ghost=True)
    r2 = oracle.fill(u, lab, g, mu=10.0, ghost=False)
    assert np.array_equal(r1["shell"], r2["shell"])
    assert np.allclose(r1["u"], r2["u"], atol=1e-12)


def test_transpose_symmetry():
    """Transposing the image and swapping the guide components transposes the
    result (the method has no preferred axis)."""
    H, W = 32, 38
    hole = _hole_blobs(H, W, 41)
    lab = synth.labels_from(hole)
    g = synth.random_guide(H, W, 42)
    rng = np.random.default_rng(43)
    u = rng.uniform(0, 1, (H, W, 3))
    r1 = oracle.fill(u, lab, g, mu=10.0)
    gt = np.ascontiguousarray(g.transpose(1, 0, 2)[..., ::-1])
    r2 = oracle.fill(u.transpose(1, 0, 2), lab.T, gt, mu=10.0)
    assert r1["stats"]["min_margin"] > 1e-9
    assert np.array_equal(r1["shell"], r2["shell"].T)
    assert np.allclose(r1["u"], r2["u"].transpose(1, 0, 2), atol=1e-12)


def test_front_entry_equals_bruteforce_definition():
    """The step at which each pixel joins the active boundary (Notation,
    d_active D^(k)_h) recomputed by brute force from the shell map: the first k
    at which some 8-neighbour is known or filled before k."""
    H, W = 40, 40
    hole = _hole_blobs(H, W, 51)
    rng = np.random.default_rng(52)
    byst = (rng.uniform(0, 1, (H, W)) < 0.08) & ~hole
    lab = synth.labels_from(hole, byst)
    g = synth.random_guide(H, W, 53)
    u = rng.uniform(0, 1, (H, W, 3))
    r = oracle.fill(u, lab, g, mu=50.0)
    sh, en = r["shell"], r["enter"]
    INF = 10 ** 9
    for y in range(H):
        for x in range(W):
            if lab[y, x] != 1:
                assert en[y, x] == -1
                continue
            best = INF
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == 0 and dy == 0:
                        continue
                    xx, yy = x + dx, y + dy
                    if 0 <= xx < W and 0 <= yy < H:
                        if lab[yy, xx] == 0:
                            best = min(best, 0)
                        elif lab[yy, xx] == 1 and sh[yy, xx] >= 0:
                            best = min(best, sh[yy, xx] + 1)
            if sh[y, x] >= 0:
                assert best <= sh[y, x]
                assert en[y, x] == best
            else:
                # never filled: it either never joined the front, or joined and the run ended
                assert en[y, x] == (-1 if best == INF else best)


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_onion_iteration_bound(seed):
    """Theorem complexity2: with smart order off and no bystanders on the outer
    boundary, Algorithm 1 ends within ceil(sqrt(N)/2) steps, N = |D_h|."""
    H, W = 48, 48
    hole = _hole_blobs(H, W, seed, n=5, rmax=9)
    lab = synth.labels_from(hole)
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 1, (H, W, 3))
    g = np.zeros((H, W, 2), np.float32)
    r = oracle.fill(u, lab, g, smart=False)
    N = int(hole.sum())
    assert r["stats"]["unreachable"] == 0
    assert r["stats"]["shells"] <= math.ceil(math.sqrt(N) / 2)


def test_onion_square_hole_shells():
    """Onion order on an s x s square hole with the 8-neighbour ball fills one
    ring per step: K = ceil(s/2), ring i (Chebyshev distance to the rim) at step i."""
    s = 9
    H = W = s + 8
    hole = synth.rect_mask(H, W, 4, 4, s, s)
    lab = synth.labels_from(hole)
    u = np.random.default_rng(1).uniform(0, 1, (H, W, 3))
    r = oracle.fill(u, lab, np.zeros((H, W, 2), np.float32), eps=1.5, smart=False)
    assert r["stats"]["shells"] == math.ceil(s / 2)
    yy, xx = np.mgrid[0:s, 0:s]
    ring = np.minimum(np.minimum(xx, yy), np.minimum(s - 1 - xx, s - 1 - yy))
    assert np.array_equal(r["shell"][4:4 + s, 4:4 + s], ring)


# ----------------------------------------------------------------------------
# Weights: response to a single bright pixel (eq. weight)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("mu", [0.0, 2.0, 10.0])
@pytest.mark.parametrize("vec", [(1.0, 0.0), (0.0, 0.5)])
def test_single_pixel_hole_delta_response(mu, vec):
    """One hole pixel surrounded by known pixels, axis-aligned g: every sample is
    a lattice pixel, so the filled value is the normalised weight of the bright
    pixel, w(x, y) = exp(-mu^2/(2 eps^2) (g_perp.(y-x))^2)/|y-x| (eq. weight)."""
    eps = 3.0
    H = W = 11
    hole = np.zeros((H, W), bool)
    hole[5, 5] = True
    lab = synth.labels_from(hole)
    g = np.zeros((H, W, 2), np.float32)
    g[..., 0], g[..., 1] = vec
    gx, gy = vec
    pts = [(dx, dy) for dy in range(-3, 4) for dx in range(-3, 4) if (dx, dy) != (0, 0) and dx * dx + dy * dy <= 9]

    def w(dx, dy):
        proj = -gy * dx + gx * dy
        return math.exp(-mu * mu / (2 * eps * eps) * proj * proj) / math.hypot(dx, dy)

    tot = sum(w(dx, dy) for dx, dy in pts)
    for (bx, by) in [(1, 0), (0, 2), (2, -2), (-1, 2), (-1, 3)]:
        u = np.zeros((H, W, 1))
        u[5 + by, 5 + bx] = 1.0
        r = oracle.fill(u, lab, g, eps=eps, mu=mu, c=1e-6)
        assert r["shell"][5, 5] == 0
        expect = w(bx, by) / tot if bx * bx + by * by <= 9 else 0.0   # (-1, 3) is outside the ball
        assert abs(r["u"][5, 5, 0] - expect) < 1e-14


# ----------------------------------------------------------------------------
# Theorem 1: transport direction g* (eqs. limitDirection, ctgf_limits)
# ----------------------------------------------------------------------------
def _g_star(theta_deg, mu, r, ghost):
    """Centre of mass of the half ball A^-_r under the weights (eq.
    limitDirection), in array coordinates (y down, data below the hole)."""
    th = math.radians(theta_deg)
    gh = (math.cos(th), math.sin(th))
    gp = (-gh[1], gh[0])
    num_x = num_y = den = 0.0
    coef = mu * mu / (2.0 * r * r)
    for m in range(-r, r + 1):
        for n in range(-r, r + 1):
            if (n, m) == (0, 0) or n * n + m * m > r * r:
                continue
            if ghost:
                yx = n * gh[0] + m * gp[0]
                yy = n * gh[1] + m * gp[1]
                proj = m
            else:
                yx, yy = n, m
                proj = -gh[1] * n + gh[0] * m
            if yy < 1.0:  # only rows already filled (onion order, rows below)
                continue
            w = math.exp(-coef * proj * proj) / math.hypot(n, m)
            num_x += w * yx
            num_y += w * yy
            den += w
    return num_x / den, num_y / den


def _edge_slope(theta_deg, mu, ghost, r=3, H=64, W=360, data_rows=8):
    """Onion-order fill of the half-plane problem (Section 4 assumptions, data
    below, hole above) with a straight step edge in the data; returns the
    per-row displacement of the edge centroid deep inside the hole."""
    th = math.radians(theta_deg)
    s_data = math.cos(th) / math.sin(th)
    hole = np.zeros((H, W), bool)
    hole[: H - data_rows] = True
    lab = synth.labels_from(hole)
    xs = np.arange(W)[None, :]
    ys = np.arange(H)[:, None]
    x0 = W / 2.0
    u = (xs < x0 + s_data * (ys - (H - 1))).astype(np.float64)[..., None]
    g = synth.const_guide(H, W, theta_deg)
    rr = oracle.fill(u, lab, g, eps=float(r), mu=mu, smart=False, ghost=ghost)
    f = rr["u"][..., 0]
    cents = []
    rows = list(range(6, H - data_rows - 12))
    for y in rows:
        p = f[y, :-1] - f[y, 1:]
        lo, hi = int(W * 0.3), int(W * 0.7)
        pw = p[lo:hi]
        cents.append(np.sum(pw * (np.arange(lo, hi) + 0.5)) / np.sum(pw))
    slope = np.polyfit(np.array(rows, float), np.array(cents), 1)[0]
    return slope


@pytest.mark.parametrize("theta,mu,ghost", [(73.0, 50.0, True), (73.0, 50.0, False), (60.0, 10.0, True),
                                            (60.0, 10.0, False), (110.0, 3.0, True), (48.0, 50.0, True)])
def test_theorem1_transport_direction(theta, mu, ghost):
    gx, gy = _g_star(theta, mu, 3, ghost)
    pred = gx / gy
    got = _edge_slope(theta, mu, ghost)
    assert abs(got - pred) < 2e-3, (got, pred)


def test_theorem1_no_kink_guidefill_kink_coherence_transport():
    """Section 3.4 / Figure connectLine: at 73 degrees with mu = 50, Guidefill
    continues the edge along g (theta* = theta) while coherence transport bends
    it toward the nearest lattice direction."""
    target = math.cos(math.radians(73)) / math.sin(math.radians(73))
    assert abs(_edge_slope(73.0, 50.0, True) - target) < 2e-3
    assert abs(_edge_slope(73.0, 50.0, False) - target) > 0.1


# ----------------------------------------------------------------------------
# Bystanders, unreachable pixels, stalls
# ----------------------------------------------------------------------------
def test_bystanders_never_read_and_walled_hole_unfilled():
    H, W = 30, 30
    hole = synth.rect_mask(H, W, 5, 5, 8, 8) | synth.rect_mask(H, W, 20, 20, 3, 3)
    byst = synth.rect_mask(H, W, 19, 19, 5, 5) & ~synth.rect_mask(H, W, 20, 20, 3, 3)
    lab = synth.labels_from(hole, byst)
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, (H, W, 3))
    u[lab == 2] = np.nan
    before = u.copy()
    g = synth.random_guide(H, W, 4)
    r = oracle.fill(u, lab, g)
    assert r["status"] == 1 and r["stats"]["unreachable"] == 9
    assert (r["shell"][20:23, 20:23] == -2).all()
    assert (r["enter"][20:23, 20:23] == -1).all()
    assert np.allclose(r["u"][20:23, 20:23], before[20:23, 20:23])
    assert (r["shell"][lab == 2] == -3).all() and (r["shell"][lab == 0] == -1).all()
    assert np.isfinite(r["u"][r["shell"] >= 0]).all()


def test_stall_rule_band_across_image():
    """A band crossing the whole image with guidance along it: interior pixels
    have no readable sample on their guidance line, so every front pixel waits
    (Remark smartOrder); the stall rule fills the front isotropically."""
    H, W = 24, 40
    hole = np.zeros((H, W), bool)
    hole[8:16, :] = True
    lab = synth.labels_from(hole)
    g = synth.const_guide(H, W, 0.0)
    rng = np.random.default_rng(9)
    u = rng.uniform(0, 1, (H, W, 3))
    r = oracle.fill(u, lab, g, mu=50.0)
    assert r["stats"]["stalls"] > 0
    assert r["stats"]["unreachable"] == 0
    assert r["stall_steps"].sum() == r["stats"]["stalls"]
    assert np.isfinite(r["u"]).all()


def _stall_band_failures():
    """Runs the oracle on the hand-worked stall band (tests/golden/stall_band.json)
    and returns the list of disagreements with the hand-worked values."""
    gold = json.load(open(os.path.join(HERE, "golden", "stall_band.json")))
    H, W = 24, 40
    hole = np.zeros((H, W), bool)
    hole[8:16, :] = True
    lab = synth.labels_from(hole)
    g = synth.const_guide(H, W, 0.0)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = np.stack([0.1 + xx / 50, 0.2 + yy / 30, 0.3 + (xx + 2 * yy) / 100], axis=2)
    r = oracle.fill(u, lab, g, eps=3.0, mu=50.0, c=0.05)
    bad = []
    want = np.full((H, W), gold["shell_outside_hole"], np.int32)
    for row, k in gold["shell_of_row"].items():
        want[int(row), :] = k
    if not np.array_equal(r["shell"], want):
        bad.append(f"shell map differs at {(r['shell'] != want).sum()} pixels")
    if r["stats"]["stalls"] != gold["stalls"] or r["stats"]["shells"] != gold["shells"]:
        bad.append(f"stalls/shells {r['stats']['stalls']}/{r['stats']['shells']}")
    if list(r["stall_steps"]) != [1] * gold["shells"]:
        bad.append(f"stall steps {list(r['stall_steps'])}")

    def from_offsets(x, y, offs, img):
        # the weighted average written out from the hand-listed readable offsets
        ws = [eval(e, {"sqrt": math.sqrt}) for _, _, e in offs]
        return sum(w * img[y + m, x + n] for (n, m, _), w in zip(offs, ws)) / sum(ws)

    for key, (x, y) in (("pixel_20_8_step0", (20, 8)), ("pixel_0_8_step0", (0, 8))):
        exp = np.array(gold[key]["colour"])
        if np.abs(from_offsets(x, y, gold[key]["readable_offsets"], u) - exp).max() > 1e-12:
            bad.append(f"{key}: the listed offsets do not give the listed colour")
        if np.abs(r["u"][y, x] - exp).max() > 1e-12:
            bad.append(f"{key}: oracle {r['u'][y, x]} vs {exp}")
    exp = np.array(gold["pixel_20_9_step1"]["colour"])
    if np.abs(r["u"][9, 20] - exp).max() > 1e-12:
        bad.append(f"pixel_20_9_step1: oracle {r['u'][9, 20]} vs {exp}")
    return bad


def test_stall_band_hand_worked():
    """Reading 8 (stall rule) pinned by hand: the 24 x 40 band with g parallel to
    it stalls at every step, fills one row from each edge per step, and fills
    with the 1/|(n, m)|-weighted average of the readable lattice points."""
    assert _stall_band_failures() == []


def _mutant_oracle(tmp_path, edits):
    """The oracle compiled from a copy of its source with `edits` applied
    (each old text must occur in the source)."""
    import ctypes as C
    import subprocess
    src = open(os.path.join(os.path.dirname(oracle.__file__), "guidefill_oracle.c")).read()
    for old, new in edits:
        assert old in src, old
        src = src.replace(old, new)
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o",
                    str(so), str(c), "-lm"], check=True)
    lib = C.CDLL(str(so))
    lib.oracle_fill.restype = C.c_int
    lib.oracle_fill.argtypes = oracle.lib().oracle_fill.argtypes
    return lib


@pytest.mark.parametrize("name,edits", [
    ("weights 1/|d|^2", [("/ sqrt((double)(n * n + m * m));", "/ (double)(n * n + m * m);")]),
    ("rotated weights in the stall pass", [("    if (isotropic) return 0.0;\n", "")]),
])
def test_stall_band_catches_planted_mistakes(tmp_path, monkeypatch, name, edits):
    """A slip in the stall rule's weights, planted in a copy of the oracle, fails the hand-worked band."""
    monkeypatch.setattr(oracle, "_lib", _mutant_oracle(tmp_path, edits))
    assert _stall_band_failures() != [], name


# ----------------------------------------------------------------------------
# Guide field from splines (Section 3.3)
# ----------------------------------------------------------------------------
def test_guidance_single_segment_closed_form():
    H, W = 40, 64
    lab = np.ones((H, W), np.uint8)
    off = np.array([0, 2], np.int32)
    pts = np.array([[10, 20], [50, 20]], np.float32)
    g = oracle.guidance(lab, off, pts, eta=3.0)
    assert np.allclose(g[23, 30], [math.exp(-9 / 18), 0.0], atol=1e-7)
    assert np.allclose(g[20, 30], [1.0, 0.0], atol=1e-7)
    assert np.allclose(g[29, 30], [math.exp(-81 / 18), 0.0], atol=1e-7)   # d = 9 = 3 eta: kept
    assert np.allclose(g[30, 30], [0.0, 0.0])                            # d = 10 > 3 eta
    assert np.allclose(g[20, 5], [math.exp(-25 / 18), 0.0], atol=1e-7)   # nearest point: endpoint
    lab2 = lab.copy()
    lab2[23, 30] = 0
    g2 = oracle.guidance(lab2, off, pts, eta=3.0)
    assert (g2[23, 30] == 0).all()                                       # non-hole pixels untouched


def test_guidance_nearest_of_two_splines_and_tangent():
    H, W = 48, 48
    lab = np.ones((H, W), np.uint8)
    off = np.array([0, 3, 5], np.int32)
    pts = np.array([[5, 10], [20, 10], [20, 30], [30, 40], [40, 30]], np.float32)
    g = oracle.guidance(lab, off, pts, eta=2.0)
    # (12, 12): nearest is segment (5,10)-(20,10), d = 2
    assert np.allclose(g[12, 12], [math.exp(-4 / 8), 0.0], atol=1e-7)
    # (22, 20): nearest is segment (20,10)-(20,30) (tangent +y), d = 2
    assert np.allclose(g[20, 22], [0.0, math.exp(-4 / 8)], atol=1e-7)
    # (35, 35) lies on the second spline's segment (30,40)-(40,30): d = 0, tangent (1,-1)/sqrt2
    assert np.allclose(g[35, 35], [1 / S2, -1 / S2], atol=1e-7)
    # (36, 36) is sqrt(2) away from it
    assert np.allclose(g[36, 36], [math.exp(-2 / 8) / S2, -math.exp(-2 / 8) / S2], atol=1e-7)


def test_guidance_tie_lowest_index():
    """Equidistant from two parallel segments: the lowest segment index wins."""
    H, W = 30, 30
    lab = np.ones((H, W), np.uint8)
    off = np.array([0, 2, 4], np.int32)
    pts = np.array([[5, 10], [25, 10], [25, 14], [5, 14]], np.float32)
    g = oracle.guidance(lab, off, pts, eta=3.0)
    assert np.allclose(g[12, 15], [math.exp(-4 / 18), 0.0], atol=1e-7)


def test_guidance_ties_report_the_other_choice():
    """Near-ties of the nearest-segment choice and of the 3 eta cut are flagged
    with the other choice's value (closed forms); decisions clear of a tie are
    not, and their smallest gap is reported."""
    H, W = 40, 40
    lab = np.ones((H, W), np.uint8)
    # two parallel segments 4 px apart (index 0 at y = 10 pointing +x, index 1 at
    # y = 14 pointing -x): row 12 is equidistant; a corner polyline (5,30)-(20,30)-(20,35)
    off = np.array([0, 2, 4, 7], np.int32)
    pts = np.array([[5, 10], [25, 10], [25, 14], [5, 14], [5, 30], [20, 30], [20, 35]], np.float32)
    r = oracle.guidance_ties(lab, off, pts, eta=3.0)
    g, alt, tie = r["guide"], r["alt"], r["tie"]
    e2 = math.exp(-4 / 18)
    assert tie[12, 15] and np.allclose(g[12, 15], [e2, 0.0], atol=1e-7) and np.allclose(alt[12, 15], [-e2, 0.0],
                                                                                         atol=1e-7)
    assert not tie[11, 15] and np.array_equal(alt[11, 15], g[11, 15])
    # outside the corner at (20, 30), on the bisector: both segments' nearest point is the vertex
    d = math.hypot(2, 2)
    e = math.exp(-d * d / 18)
    assert tie[28, 22] and np.allclose(g[28, 22], [e, 0.0], atol=1e-7) and np.allclose(alt[28, 22], [0.0, e],
                                                                                        atol=1e-7)
    # d = 9 = 3 eta above the upper parallel segment (nothing else within 9 px): the cut is a tie
    assert tie[1, 15] and np.allclose(g[1, 15], [math.exp(-81 / 18), 0.0], atol=1e-7)
    assert np.array_equal(alt[1, 15], [0.0, 0.0])
    assert not tie[2, 15] and not tie[0, 15] and np.array_equal(g[0, 15], [0.0, 0.0])
    assert r["n_ties"] == int(tie.sum()) > 0
    assert oracle.SEG_TIE_PX < r["min_gap"] < 0.5


# ----------------------------------------------------------------------------
# Data term (eq. ready2, Section 3.5 possible extensions)
# ----------------------------------------------------------------------------
def _mixed_hole(H=48, W=64, seed=5):
    """A horizontal band with guidance along it (g != 0) joined to a square blob
    with g = 0."""
    rng = np.random.default_rng(seed)
    hole = np.zeros((H, W), bool)
    hole[20:27, 6:40] = True          # band
    hole[12:36, 40:58] = True         # blob
    g = np.zeros((H, W, 2), np.float32)
    g[20:27, 6:40] = (1.0, 0.0)
    lab = synth.labels_from(hole)
    u = rng.uniform(0, 1, (H, W, 3))
    return u, lab, g, hole


def test_data_term_without_guidance_is_the_plain_fill():
    u, lab, _, _ = _mixed_hole()
    g0 = np.zeros(lab.shape + (2,), np.float32)
    a = oracle.fill(u, lab, g0)
    b = oracle.fill(u, lab, g0, data_term=True)
    assert np.array_equal(a["shell"], b["shell"]) and np.array_equal(a["u"], b["u"])
    assert b["stats"]["data_switch"] == 0 and a["stats"]["data_switch"] == -1


def test_data_term_fills_guided_pixels_first():
    u, lab, g, hole = _mixed_hole()
    r = oracle.fill(u, lab, g, data_term=True)
    ks = r["stats"]["data_switch"]
    sh = r["shell"]
    gnz = (g[..., 0] != 0) | (g[..., 1] != 0)
    assert ks > 0
    # phase 1: every pixel filled before the switch has g != 0
    assert np.all(gnz[(sh >= 0) & (sh < ks)])
    # the switch: either every guided pixel is filled, or phase 1 had nothing ready
    guided_left = np.any(gnz & hole & ((sh < 0) | (sh >= ks)))
    if guided_left:
        plain = oracle.fill(u, lab, g)
        assert not np.array_equal(plain["shell"], sh)
    # a constant image stays constant under the data term as well
    c = oracle.fill(np.full_like(u, 0.375), lab, g, data_term=True)
    assert np.allclose(c["u"][hole], 0.375, atol=1e-12)
    # eq. ready2 changes the order: the plain fill reaches blob pixels earlier
    plain = oracle.fill(u, lab, g)
    blob = hole & ~gnz
    assert sh[blob].min() >= ks and plain["shell"][blob].min() < ks
