"""The data term of eq. ready2 (Section 3.5, possible extensions) on the CUDA
path against the oracle: while hole pixels with g != 0 remain, only they are
ready; eq. ready from the first step at which none is left or none would fill."""
import numpy as np
import pytest

import synth
from _gpu import assert_parity, gpu_fill, hole_blobs, oracle_fill

pytestmark = pytest.mark.gpu


def _mixed(H=48, W=64, seed=5):
    rng = np.random.default_rng(seed)
    hole = np.zeros((H, W), bool)
    hole[20:27, 6:40] = True
    hole[12:36, 40:58] = True
    g = np.zeros((H, W, 2), np.float32)
    g[20:27, 6:40] = (1.0, 0.0)
    lab = synth.labels_from(hole)
    img = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    img[lab != 0] = np.nan
    return img, lab, g


def _random(H, W, seed):
    rng = np.random.default_rng(seed)
    hole = hole_blobs(H, W, seed, n=max(1, H * W // 300), rmax=7, margin=3)
    b = (rng.uniform(0, 1, (H, W)) < 0.03) & ~hole
    lab = synth.labels_from(hole, b)
    img = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    img[lab != 0] = np.nan
    g = synth.random_guide(H, W, seed + 1, zero_fraction=0.2)
    return img, lab, g


def test_mixed_hole_guided_band_first():
    img, lab, g = _mixed()
    o = oracle_fill(img, lab, g, data_term=True)
    r = gpu_fill(img, lab, g, data_term=True)
    assert_parity(o, r, lab)
    assert r["stats"]["data_switch"] == o["stats"]["data_switch"] > 0


@pytest.mark.parametrize("ghost,smart,rescan", [(True, True, False), (True, False, False), (False, True, False),
                                                (True, True, True)])
@pytest.mark.parametrize("seed", [31, 32])
def test_random_frames(ghost, smart, rescan, seed):
    img, lab, g = _random(60, 76, seed)
    o = oracle_fill(img, lab, g, eps=3.0, mu=10.0, ghost=ghost, smart=smart, data_term=True)
    r = gpu_fill(img, lab, g, eps=3.0, mu=10.0, ghost=ghost, smart=smart, rescan=rescan, data_term=True)
    assert_parity(o, r, lab)


def test_no_guidance_switches_at_step_zero():
    img, lab, _ = _random(40, 48, 33)
    g0 = np.zeros(lab.shape + (2,), np.float32)
    o = oracle_fill(img, lab, g0, data_term=True)
    r = gpu_fill(img, lab, g0, data_term=True)
    assert_parity(o, r, lab)
    assert r["stats"]["data_switch"] == 0
    p = gpu_fill(img, lab, g0)
    assert np.array_equal(p["shell"], r["shell"]) and p["stats"]["data_switch"] == -1
