"""gf_fill_noalloc: the fill entry point that allocates no device memory.

It is for callers that cannot call cudaMalloc (work enqueued while a stream is
being captured into a CUDA graph, hosts that own all device memory, loops that
must not allocate after start-up); its scratch is a fixed __device__ array in
the library.  Its output must equal gf_fill's on the same frame, on two calls in
a row (the array keeps the previous call's contents, so the second call checks
that everything that must start at zero is cleared).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _frame(H, W, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    hole = np.zeros((H, W), bool)
    for _ in range(max(1, H * W // 400)):
        cx, cy, r = rng.uniform(0, W), rng.uniform(0, H), rng.uniform(2, 8)
        hole |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    byst = (rng.uniform(0, 1, (H, W)) < 0.02) & ~hole
    lab = synth.labels_from(hole, byst)
    img = synth.to_rgba(rng.uniform(0, 1, (H, W, 3)).astype(np.float32))
    img[lab != 0] = np.nan
    return img, lab, synth.random_guide(H, W, seed + 1)


def _run(fn_name, img, lab, g, ctx=None):
    import torch

    from paper_1611_05319_gb300 import _lib
    H, W = lab.shape
    x = torch.from_numpy(img).cuda()
    lt = torch.from_numpy(lab).cuda()
    gt = torch.from_numpy(g).cuda()
    out = torch.full((H, W, 4), -5.0, dtype=torch.float32, device="cuda")
    shell = torch.full((H, W), 7, dtype=torch.int32, device="cuda")
    enter = torch.full((H, W), 7, dtype=torch.int32, device="cuda")
    stats = torch.zeros((_lib.STATS_BYTES,), dtype=torch.uint8, device="cuda")
    fr = _lib.Frame(H, W, x.data_ptr(), lt.data_ptr(), gt.data_ptr(), out.data_ptr(), shell.data_ptr(),
                    enter.data_ptr(), None)
    prm = _lib.make_params(eps=3.0, mu=50.0, c=0.05)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = _lib.lib()
    if fn_name == "gf_fill":
        rc = L.gf_fill(ctx._h, C.byref(fr), C.byref(prm), C.c_void_p(stats.data_ptr()), stream)
    else:
        rc = L.gf_fill_noalloc(C.byref(fr), C.byref(prm), C.c_void_p(stats.data_ptr()), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=_lib.STATS_DTYPE)[0]
    return out.cpu().numpy(), shell.cpu().numpy(), enter.cpu().numpy(), st


def test_noalloc_matches_gf_fill_on_two_calls_in_a_row(cuda_device):
    import paper_1611_05319_gb300 as gf
    from paper_1611_05319_gb300 import build
    build.build()
    ctx = gf.Context(0)
    # two different frames, the second smaller than the first, so stale
    # contents of the shared scratch would show
    for (H, W, seed) in [(300, 420, 11), (97, 131, 12)]:
        img, lab, g = _frame(H, W, seed)
        ref = _run("gf_fill", img, lab, g, ctx)
        got = _run("gf_fill_noalloc", img, lab, g)
        assert np.array_equal(ref[1], got[1])  # shell indices bit-exact
        assert np.array_equal(ref[2], got[2])  # front-entry steps bit-exact
        filled = ref[1] >= 0
        assert filled.sum() > 0
        assert np.abs(ref[0][filled] - got[0][filled]).max() <= 1e-4
        for k in ("shells", "stalls", "filled", "max_front", "holes", "status"):
            assert ref[3][k] == got[3][k], k
    ctx.close()


def test_noalloc_rejects_frames_beyond_its_scratch(cuda_device):
    import torch

    from paper_1611_05319_gb300 import _lib
    L = _lib.lib()
    H, W = 16, 4097  # one side over 4096
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
