"""CUDA path vs the oracle with the caller's buffers at the smallest offsets the
C ABI allows: labels at any byte, guide vectors and spline points at 8 bytes,
state words, entry steps and stall bits at 4 bytes, colours at 16 bytes.  Such
offsets take the kernels' scalar load and store paths (their 16-byte row loads
and stores need 16-byte aligned rows), so the results must not change.

Bar as in the parity tests: shell indices and entry steps bit-exact, counts
equal, colours within 1e-4 of the FP64 oracle; guide fields and detected
spline end points bit-exact, their weights within 1e-6 relative."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from synth import configs

from _gpu import COLOUR_ATOL, hole_blobs, rgba

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ctx(cuda_device):
    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import build
    build.build()
    return gf.context(0)


def _at(a, off, dev):
    """A contiguous device copy of `a` that starts `off` elements into a larger buffer."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a).reshape(-1))
    big = torch.zeros(t.numel() + off, dtype=t.dtype, device=dev)
    big[off:].copy_(t)
    return big, big[off:].view(a.shape)


def _empty_at(n, dtype, off, dev):
    import torch
    big = torch.zeros(n + off, dtype=dtype, device=dev)
    return big, big[off:]


def _case(H, W, seed):
    rng = np.random.default_rng(seed)
    hole = hole_blobs(H, W, seed, n=max(1, H * W // 300), rmax=7, margin=3)
    b = (rng.uniform(0, 1, (H, W)) < 0.03) & ~hole
    lab = synth.labels_from(hole, b)
    img = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    img[lab != 0] = np.nan
    g = synth.random_guide(H, W, seed + 1, zero_fraction=0.2)
    return img, lab, g


@pytest.mark.parametrize("H,W", [(48, 64), (37, 61), (64, 256)])
@pytest.mark.parametrize("lab_off", [1, 3])
def test_fill_with_offset_buffers(H, W, lab_off, cuda_device):
    import torch

    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import _lib
    img, lab, g = _case(H, W, 4000 + H + W + lab_off)
    o = oracle.fill(rgba(img), lab, g, eps=3.0, mu=50.0)
    dev = cuda_device
    keep = []
    for x in (_at(rgba(img), 4, dev), _at(lab, lab_off, dev), _at(g.astype(np.float32), 2, dev)):
        keep.append(x)
    (_, x_rgba), (_, x_lab), (_, x_g) = keep
    _, o_rgba = _empty_at(H * W * 4, torch.float32, 4, dev)
    _, o_shell = _empty_at(H * W, torch.int32, 1, dev)
    _, o_enter = _empty_at(H * W, torch.int32, 3, dev)
    _, o_stall = _empty_at((H * W + 1 + 31) // 32, torch.int32, 1, dev)
    assert x_lab.data_ptr() % 16 == lab_off and x_g.data_ptr() % 16 == 8 and o_shell.data_ptr() % 16 == 4
    stats = torch.zeros((_lib.STATS_BYTES,), dtype=torch.uint8, device=dev)
    fr = (_lib.Frame * 1)(_lib.Frame(H, W, x_rgba.data_ptr(), x_lab.data_ptr(), x_g.data_ptr(), o_rgba.data_ptr(),
                                     o_shell.data_ptr(), o_enter.data_ptr(), o_stall.data_ptr()))
    prm = _lib.make_params(eps=3.0, mu=50.0)
    ctx = gf.context(0)
    _lib.check(_lib.lib().gf_fill_batched(ctx._h, 1, fr, C.byref(prm), C.c_void_p(stats.data_ptr()),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream)), "fill", ctx._h)
    torch.cuda.synchronize()
    st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=_lib.STATS_DTYPE)[0]
    shell = o_shell.cpu().numpy().reshape(H, W)
    enter = o_enter.cpu().numpy().reshape(H, W)
    u = o_rgba.cpu().numpy().reshape(H, W, 4)
    assert np.array_equal(shell, o["shell"])
    assert np.array_equal(enter, o["enter"])
    for k in ("shells", "stalls", "filled", "max_front"):
        assert int(st[k]) == int(o["stats"][k]), k
    assert int(st["status"]) == 0 and int(st["holes"]) == int((lab == 1).sum())
    bits = o_stall.cpu().numpy().view(np.uint32)
    steps = np.array([(bits[k >> 5] >> (k & 31)) & 1 for k in range(int(st["shells"]))], bool)
    assert np.array_equal(steps, o["stall_steps"][:int(st["shells"])].astype(bool))
    filled = o["shell"] >= 0
    if filled.any():
        assert np.abs(u[filled] - o["u"][filled]).max() <= COLOUR_ATOL
    known = lab == 0
    assert np.array_equal(u[known], rgba(img)[known])


@pytest.mark.parametrize("lab_off", [1, 2, 5])
def test_guidance_with_offset_labels(lab_off, cuda_device):
    import torch

    import paper_1611_05319_gb300 as gf
    H, W = 96, 160
    ctrl = synth.random_beziers(6, H, W, 3, 40.0, margin=5)
    off, pts = synth.flatten_beziers(ctrl, 16)
    lab = synth.labels_from(synth.band_mask(H, W, ctrl, [5.0] * 6))
    go = oracle.guidance(lab, off, pts, 3.0)
    _, x_lab = _at(lab, lab_off, cuda_device)
    _, x_pts = _at(pts.astype(np.float32), 2, cuda_device)
    _, x_off = _at(off.astype(np.int32), 1, cuda_device)
    assert x_lab.data_ptr() % 16 == lab_off and x_pts.data_ptr() % 16 == 8
    gg = gf.context(0).guidance(x_lab, x_off, x_pts, 3.0)
    torch.cuda.synchronize()
    gg = gg.cpu().numpy()
    hole = lab == 1
    assert hole.any()
    assert np.array_equal(go[hole], gg[hole])


@pytest.mark.parametrize("lab_off", [1, 7])
def test_detection_with_offset_labels(lab_off, cuda_device):
    import torch

    import paper_1611_05319_gb300 as gf
    d = configs.plain_128(poison=True)
    img = rgba(d["rgb"])
    kw = dict(sigma=1.0, rho=2.0, t_high=0.02, t_low=0.01)
    od = oracle.detect_splines(img, d["labels"], **kw)
    _, x_img = _at(img, 4, cuda_device)
    _, x_lab = _at(d["labels"], lab_off, cuda_device)
    det = gf.context(0).detect_splines(x_img, x_lab, **kw)
    torch.cuda.synchronize()
    pts, wt, base = det.splines()
    assert od["count"] > 0
    assert det.count() == od["count"]
    assert np.array_equal(base, od["base"]) and np.array_equal(pts, od["pts"])
    np.testing.assert_allclose(wt, od["weight"], rtol=1e-6, atol=0)  # as in the detection parity tests
