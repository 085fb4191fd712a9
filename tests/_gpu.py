"""Helpers for the GPU parity tests: run the CUDA path and the oracle on the same
seeded inputs and compare element by element."""
import numpy as np

import oracle
import synth

COLOUR_ATOL = 1e-4  # max-abs on colours in [0, 1] against the FP64 oracle


def rgba(img):
    return synth.to_rgba(np.asarray(img, np.float32))


def gpu_fill(img, labels, guide, **kw):
    import torch

    import paper_1611_05319_gb300 as gf
    ctx = gf.context(0)
    r = ctx.fill(torch.from_numpy(rgba(img)).cuda(), torch.from_numpy(np.ascontiguousarray(labels)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(guide, np.float32)).cuda(), enter=True, stall=True, **kw)
    torch.cuda.synchronize()
    st = r.stats()
    return dict(u=r.rgba.cpu().numpy(), shell=r.shell.cpu().numpy(), enter=r.enter.cpu().numpy(), stats=st,
                stall_steps=r.stall_steps())


def oracle_fill(img, labels, guide, **kw):
    kw = dict(kw)
    kw.pop("rescan", None)
    return oracle.fill(rgba(img), labels, guide, **kw)


def assert_parity(o, g, labels, atol=COLOUR_ATOL, check_enter=True):
    assert np.array_equal(o["shell"], g["shell"]), _diff(o["shell"], g["shell"])
    if check_enter:
        assert np.array_equal(o["enter"], g["enter"]), _diff(o["enter"], g["enter"])
    so, sg = o["stats"], g["stats"]
    for k in ("shells", "stalls", "filled", "max_front", "data_switch"):
        assert so[k] == sg[k], (k, so[k], sg[k])
    assert sg["holes"] == int((labels == 1).sum())
    assert np.array_equal(o["stall_steps"].astype(bool), g["stall_steps"])
    filled = o["shell"] >= 0
    if filled.any():
        err = np.abs(o["u"][filled] - g["u"][filled]).max()
        assert err <= atol, err
    # pixels that were not filled keep their input value exactly
    known = labels == 0
    assert np.array_equal(np.nan_to_num(o["u"][known].astype(np.float32), nan=-7.0),
                          np.nan_to_num(g["u"][known], nan=-7.0))
    return True


def assert_guide_parity(ties, gg, labels):
    """GPU guide field against oracle.guidance_ties: bit-exact wherever the
    nearest-segment choice and the 3 eta cut are clear of a tie (the value is
    unique there), and one of the two valid values at the near-ties.  Returns
    the number of near-tie pixels."""
    hole = labels == 1
    g, alt, tie = ties["guide"], ties["alt"], ties["tie"]
    clear = hole & ~tie
    assert np.array_equal(g[clear], gg[clear]), _diff(g[clear], gg[clear])
    t = hole & tie
    ok = np.all(gg[t] == g[t], axis=-1) | np.all(gg[t] == alt[t], axis=-1)
    assert ok.all(), f"{(~ok).sum()} near-tie pixels hold neither valid value"
    return int(t.sum())


def _diff(a, b):
    idx = np.argwhere(a != b)
    return f"{len(idx)} mismatches, first {idx[:5].tolist()}: {a[tuple(idx[0])] if len(idx) else ''} vs " \
           f"{b[tuple(idx[0])] if len(idx) else ''}"


def hole_blobs(H, W, seed, n=6, rmin=2, rmax=7, margin=0):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    hole = np.zeros((H, W), bool)
    for _ in range(n):
        cx, cy = rng.uniform(-margin, W + margin), rng.uniform(-margin, H + margin)
        r = rng.uniform(rmin, rmax)
        hole |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    return hole


def oracle_batch_job(args):
    """Oracle side of one frame of the 64-frame batch, for a spawned worker:
    the guide field with its near-ties from the frame's splines, and the fill of
    the frame with the guide field the GPU built (its input; the guide fields
    are compared separately).  Returns compact arrays."""
    seed, gpu_guide = args
    from synth import configs
    f = configs.batch_frame(seed, poison=True)
    ties = oracle.guidance_ties(f["labels"], *f["splines"], eta=3.0)
    o = oracle.fill(rgba(f["rgb"]), f["labels"], gpu_guide, eps=3.0, mu=50.0, c=0.05)
    filled = o["shell"] >= 0
    return dict(seed=seed, shell=o["shell"], enter=o["enter"], u_filled=o["u"][filled], stats=o["stats"],
                stall_steps=o["stall_steps"], ties={k: ties[k] for k in ("guide", "alt", "tie", "min_gap", "n_ties")})
