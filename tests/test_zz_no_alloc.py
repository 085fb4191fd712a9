"""gf_fill_noalloc: the fill entry point that allocates no device memory.

It is for callers that cannot call cudaMalloc: hosts that own all device memory
and hand libraries none, and loops that must not allocate once they run.  Its
scratch is a fixed __device__ array in the library.  Its output must equal
gf_fill's, and the oracle's, on the same frame, on two calls in a row (the
array keeps the previous call's contents, so the second call checks that
everything that must start at zero is cleared).  This file is collected last so
that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth

from _gpu import assert_parity, oracle_fill

pytestmark = pytest.mark.gpu


def _frame(H, W, seed, n=None):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    hole = np.zeros((H, W), bool)
    for _ in range(n if n is not None else max(1, H * W // 400)):
        cx, cy, r = rng.uniform(0, W), rng.uniform(0, H), rng.uniform(2, 8)
        hole |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    byst = (rng.uniform(0, 1, (H, W)) < 0.02) & ~hole
    lab = synth.labels_from(hole, byst)
    img = synth.to_rgba(rng.uniform(0, 1, (H, W, 3)).astype(np.float32))
    img[lab != 0] = np.nan
    return img, lab, synth.random_guide(H, W, seed + 1, zero_fraction=0.3)


def _run(fn_name, img, lab, g, ctx=None, data_term=False):
    import torch

    from paper_1611_05319_gb300 import _lib
    H, W = lab.shape
    x = torch.from_numpy(img).cuda()
    lt = torch.from_numpy(lab).cuda()
    gt = torch.from_numpy(g).cuda()
    out = torch.full((H, W, 4), -5.0, dtype=torch.float32, device="cuda")
    shell = torch.full((H, W), 7, dtype=torch.int32, device="cuda")
    enter = torch.full((H, W), 7, dtype=torch.int32, device="cuda")
    stall = torch.full(((H * W + 1 + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    stats = torch.zeros((_lib.STATS_BYTES,), dtype=torch.uint8, device="cuda")
    fr = _lib.Frame(H, W, x.data_ptr(), lt.data_ptr(), gt.data_ptr(), out.data_ptr(), shell.data_ptr(),
                    enter.data_ptr(), stall.data_ptr())
    prm = _lib.make_params(eps=3.0, mu=50.0, c=0.05, data_term=data_term)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = _lib.lib()
    if fn_name == "gf_fill":
        rc = L.gf_fill(ctx._h, C.byref(fr), C.byref(prm), C.c_void_p(stats.data_ptr()), stream)
    else:
        rc = L.gf_fill_noalloc(C.byref(fr), C.byref(prm), C.c_void_p(stats.data_ptr()), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=_lib.STATS_DTYPE)[0]
    K = int(st["shells"])
    sb = stall.cpu().numpy().view(np.uint32)
    steps = np.array([(sb[k >> 5] >> (k & 31)) & 1 for k in range(K)], bool)
    return dict(u=out.cpu().numpy(), shell=shell.cpu().numpy(), enter=enter.cpu().numpy(), stall_steps=steps,
                stats={k: int(st[k]) for k in st.dtype.names})


@pytest.mark.parametrize("data_term", [False, True])
def test_noalloc_matches_oracle_and_gf_fill_on_two_calls_in_a_row(cuda_device, data_term):
    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import build
    build.build()
    ctx = gf.Context(0)
    # two different frames, the second smaller than the first, so stale
    # contents of the shared scratch would show
    for (H, W, seed) in [(300, 420, 11), (97, 131, 12)]:
        img, lab, g = _frame(H, W, seed)
        got = _run("gf_fill_noalloc", img, lab, g, data_term=data_term)
        o = oracle_fill(img, lab, g, eps=3.0, mu=50.0, c=0.05, data_term=data_term)
        assert got["stats"]["shells"] > 0 and (got["shell"] >= 0).sum() > 0
        assert_parity(o, got, lab)
        ref = _run("gf_fill", img, lab, g, ctx, data_term=data_term)
        assert np.array_equal(ref["shell"], got["shell"]) and np.array_equal(ref["enter"], got["enter"])
        filled = ref["shell"] >= 0
        assert np.abs(ref["u"][filled] - got["u"][filled]).max() <= 1e-4
        for k in ("shells", "stalls", "filled", "max_front", "holes", "status", "data_switch"):
            assert ref["stats"][k] == got["stats"][k], k
    ctx.close()


def test_noalloc_largest_allowed_frame(cuda_device):
    """4096 x 1024 = 4,194,304 px, the largest frame the fixed scratch holds."""
    import paper_1611_05319_gb300 as gf
    ctx = gf.Context(0)
    img, lab, g = _frame(1024, 4096, 21, n=40)
    got = _run("gf_fill_noalloc", img, lab, g)
    ref = _run("gf_fill", img, lab, g, ctx)
    assert got["stats"]["status"] == 0 and got["stats"]["filled"] == int((lab == 1).sum())
    assert np.array_equal(ref["shell"], got["shell"]) and np.array_equal(ref["enter"], got["enter"])
    filled = ref["shell"] >= 0
    assert np.array_equal(ref["u"][filled], got["u"][filled])
    ctx.close()


@pytest.mark.parametrize("H,W", [(16, 4097), (4097, 16), (1025, 4096), (4096, 1025)])
def test_noalloc_rejects_frames_beyond_its_scratch(cuda_device, H, W):
    """One side over 4096 px, or both within 4096 but over 4,194,304 px in total."""
    import torch

    from paper_1611_05319_gb300 import _lib
    L = _lib.lib()
    buf = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    lab = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    g = torch.zeros((H, W, 2), dtype=torch.float32, device="cuda")
    sh = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    stats = torch.zeros((_lib.STATS_BYTES,), dtype=torch.uint8, device="cuda")
    fr = _lib.Frame(H, W, buf.data_ptr(), lab.data_ptr(), g.data_ptr(), buf.data_ptr(), sh.data_ptr(), None, None)
    prm = _lib.make_params()
    rc = L.gf_fill_noalloc(C.byref(fr), C.byref(prm), C.c_void_p(stats.data_ptr()), None)
    assert rc == -8
    assert b"4096" in L.gf_status_string(rc)
