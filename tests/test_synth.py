"""The seeded synthetic workloads follow their stated recipe: same seed, same
arrays; sizes, hole fractions, band half-widths, spline counts and guidance as
the workload table gives them; hole pixels poisoned with NaN on request.  CPU
only (each frame takes well under two seconds to build)."""
import math

import numpy as np
import pytest

from synth import configs


def _same(a, b):
    assert np.array_equal(a["labels"], b["labels"])
    assert np.array_equal(a["rgb"], b["rgb"], equal_nan=True)
    assert np.array_equal(a["splines"][0], b["splines"][0]) and np.array_equal(a["splines"][1], b["splines"][1])
    assert np.array_equal(a["half_widths"], b["half_widths"])


def test_same_seed_same_arrays_other_seed_other_arrays():
    a, b = configs.batch_frame(123), configs.batch_frame(123)
    _same(a, b)
    c = configs.batch_frame(124)
    assert not np.array_equal(a["labels"], c["labels"])


def test_plain_128_recipe():
    d = configs.plain_128(poison=True)
    lab = d["labels"]
    assert lab.shape == (128, 128) and not (lab == 2).any()
    area = math.pi * (32.0 ** 2 - 24.0 ** 2)  # annulus of radii 24 and 32
    assert abs((lab == 1).sum() - area) < 0.03 * area
    g = d["guide"].reshape(-1, 2)
    assert np.allclose(g, [math.cos(math.radians(30.0)), math.sin(math.radians(30.0))], atol=1e-7)
    assert np.isnan(d["rgb"][lab == 1]).all() and np.isfinite(d["rgb"][lab == 0]).all()
    assert d["gt"].min() >= 0.0 and d["gt"].max() <= 1.0
    assert (d["eps"], d["mu"], d["c"]) == (3.0, 50.0, 0.05)


def test_frame_1080_recipe():
    d = configs.frame_1080(poison=True)
    lab = d["labels"]
    assert lab.shape == (1080, 1920) and d["rgb"].shape == (1080, 1920, 3)
    assert abs((lab == 1).mean() - 0.03) < 0.001
    assert len(d["splines"][0]) - 1 == 20
    assert d["half_widths"].min() >= 1.5 and d["half_widths"].max() <= 7.5
    assert np.isnan(d["rgb"][lab == 1]).all() and np.isfinite(d["gt"]).all()
    assert d["gt"].min() >= 0.0 and d["gt"].max() <= 1.0


@pytest.mark.parametrize("seed", [100, 119, 137, 163])
def test_batch_frame_recipe(seed):
    d = configs.batch_frame(seed)
    lab = d["labels"]
    f = d["target_fraction"]
    assert lab.shape == (1080, 1920) and not (lab == 2).any()
    assert 0.005 <= f <= 0.08
    assert abs((lab == 1).mean() - f) < 0.1 * f
    assert len(d["splines"][0]) - 1 == 20
    assert d["half_widths"].min() >= 1.0 and d["half_widths"].max() <= 20.0


def test_frame_4k_blob_recipe():
    d = configs.frame_4k_blob()
    lab = d["labels"]
    bx, by = d["blob_xy"]
    assert lab.shape == (2160, 3840) and d["eps"] == 4.0
    assert (lab[by:by + 400, bx:bx + 400] == 1).all()
    blob = 400 * 400 / lab.size
    assert 0.02 + blob - 0.004 < (lab == 1).mean() < 0.02 + blob + 0.001  # bands may overlap the blob


@pytest.mark.parametrize("H", [70, 140])
def test_line_problem_geometry(H):
    d = configs.line_problem(H)
    lab = d["labels"]
    W = 4 * H
    yc = (np.arange(H) + 0.5) / H
    xc = (np.arange(W) + 0.5) * 4.0 / W
    rows = ((yc >= 0.2) & (yc <= 0.8)).sum()
    cols = ((xc >= 0.4) & (xc <= 3.96)).sum()
    assert lab.shape == (H, W) and (lab == 1).sum() == rows * cols
    line = (yc >= 0.45) & (yc <= 0.55)
    assert np.allclose(d["gt"][line], [0.9, 0.2, 0.1]) and np.allclose(d["gt"][~line], [0.1, 0.3, 0.8])
    assert not d["guide"].any() and d["smart"] is False


def test_corridor_recipe():
    """One-pixel corridor: L hole pixels in row 1, bystander walls, one known pixel at the open end."""
    d = configs.corridor(50)
    lab = d["labels"]
    assert lab.shape == (3, 52)
    assert (lab[1, 1:51] == 1).all() and lab[1, 0] == 0 and lab[1, 51] == 2
    assert (lab[0] == 2).all() and (lab[2] == 2).all()
    assert (d["guide"] == 0).all() and d["smart"] is False


def test_batch_hole_fraction_is_the_frame_target():
    for s in (100, 119, 163):
        assert configs.batch_hole_fraction(s) == configs.batch_frame(s, H=108, W=192)["target_fraction"]
