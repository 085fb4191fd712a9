"""Writes tests/golden/alg_bytes.json: the algorithmic bytes of each benchmark
frame under Algorithm 1's per-step semantics, counted by the oracle
(oracle.alg_bytes over the oracle's own shell / front-entry maps).

Calls only ``oracle`` and ``synth``.  Usage: python tests/golden/make_alg_bytes.py
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def _one(item):
    name, seed = item
    import oracle
    from synth import configs
    if name == "batch_1080":
        f = configs.batch_frame(seed)
    elif name == "frame_1080":
        f = configs.frame_1080(seed)
    elif name == "frame_4k_blob":
        f = configs.frame_4k_blob(seed)
    elif name == "plain_128":
        f = configs.plain_128(seed)
    else:
        raise ValueError(name)
    g = f["guide"] if f["guide"] is not None else oracle.guidance(f["labels"], *f["splines"], eta=f["eta"])
    r = oracle.fill(f["rgb"], f["labels"], g, eps=f["eps"], mu=f["mu"], c=f["c"])
    b = oracle.alg_bytes(f["labels"], g, f["eps"], r["shell"], r["enter"])
    H, W = f["labels"].shape
    return name, seed, dict(alg_bytes=b, filled=r["stats"]["filled"], shells=r["stats"]["shells"],
                            stalls=r["stats"]["stalls"], evaluations=r["stats"]["evaluations"],
                            holes=int((f["labels"] == 1).sum()), H=H, W=W)


def main():
    items = [("batch_1080", s) for s in range(100, 164)] + [("frame_1080", 2), ("plain_128", 1),
                                                           ("frame_4k_blob", 3)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(items), os.cpu_count() or 1)) as pool:
        res = pool.map(_one, items)
    out = {"cite": "Algorithm 1 per-step byte model: sum_k |E_k|*12 + |T_k|*4 + |U_k|*12 + |F_k|*16 "
                   "+ |front_{k+1}|*4 bytes (oracle.alg_bytes)",
           "frames": {}}
    for name, seed, d in res:
        out["frames"].setdefault(name, {})[str(seed)] = d
    with open(os.path.join(HERE, "alg_bytes.json"), "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    tot = sum(d["alg_bytes"] for d in out["frames"]["batch_1080"].values())
    px = sum(d["filled"] for d in out["frames"]["batch_1080"].values())
    print(f"batch_1080: {tot} bytes for {px} filled px ({tot / px:.1f} B/px)")


if __name__ == "__main__":
    main()
