"""Accuracy versus speed: the contact network against UCF-GJK (Sec. IV-B,
Claim 1: the paper plots collision-check speed against accuracy for its
network and for a uniform-flow GJK over convex decompositions, sweeping the
GJK hyper-parameters).

Accuracy: collision decisions on a labelled test set written by the test
infrastructure (labels from the geometric contact detector).  Speed: pairs/s
of one call on the test set's pairs replicated to a batch of about 200 k
pairs, device-resident inputs, CUDA-event timing, median of repeats with L2
flushed between them.  GJK sweeps the hull vertices kept per convex element
(farthest-point sampling of each component's vertices) and the fixed
iteration count.

    python -m paper_2304_09439_b300.gjk_sweep --data data/test_known.npz --out report.md
"""

from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _time(fn, stream, flush, reps=7):
    import torch
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts[2:]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", default=os.path.join(ROOT, "data", "test_known.npz"))
    ap.add_argument("--weights", default=os.path.join(HERE, "weights", "locc_trained.bin"))
    ap.add_argument("--replicate", type=int, default=32)
    ap.add_argument("--vertices", default="8,16,32,64", help="0 = all vertices")
    ap.add_argument("--iterations", default="4,6,9,16")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()

    import torch
    import synth
    from paper_2304_09439_b300 import GJK, Detector
    from paper_2304_09439_b300.train import LIBRARIES

    dev = torch.device("cuda:0")
    d = np.load(args.data)
    n_lib, seed = LIBRARIES[str(d["library"])]
    lib = synth.make_library(n_lib, seed)
    truth = d["targets"][:, 0] > 0.5
    P = len(d["pairs"])
    # replicated batch for timing: copies share the poses, pairs point into them
    reps = args.replicate
    poses = torch.from_numpy(d["poses"]).to(dev)
    osh = torch.from_numpy(d["obj_shape"]).to(dev)
    pairs = torch.from_numpy(d["pairs"]).to(dev)
    big = pairs.repeat(reps, 1).contiguous()
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)

    rows = []
    with open(args.weights, "rb") as f:
        blob = f.read()
    for prec in ("bf16", "fp8", "fp32"):
        with Detector(lib.points, lib.aabb, blob, 0.25, prec) as det:
            det.reserve(len(big))
            out = det.detect(poses, osh, pairs, stream=stream).cpu().numpy()
            det.status(stream)
            acc = float(np.mean((out[:, 0] > 0) == truth))
            ms = _time(lambda: det.detect(poses, osh, big, stream=stream), stream, flush)
            rows.append({"method": f"network ({prec})", "setting": "trained, local crops",
                         "accuracy": acc, "pairs_per_s": len(big) / (ms * 1e-3)})
    for nv in (int(x) for x in args.vertices.split(",")):
        eo, vo, vv = synth.convex_elements(lib, nv)
        with GJK(eo, vo, vv) as g:
            for it in (int(x) for x in args.iterations.split(",")):
                col = g.detect(poses, osh, pairs, it, stream=stream).cpu().numpy()
                g.status(stream)
                acc = float(np.mean((col == 1) == truth))
                ms = _time(lambda: g.detect(poses, osh, big, it, stream=stream), stream, flush)
                rows.append({"method": "UCF-GJK", "setting": f"{nv or 'all'} vertices / element, "
                                                           f"{it} iterations",
                             "accuracy": acc, "pairs_per_s": len(big) / (ms * 1e-3),
                             "elements": int(eo[-1]), "vertices": int(vo[-1])})
    for r in rows:
        print(json.dumps(r), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(f"# Accuracy vs speed on {os.path.basename(args.data)} ({P} labelled pairs; "
                    f"timing on {len(big)} pairs)\n\n")
            f.write("| method | setting | accuracy | pairs/s |\n|---|---|---:|---:|\n")
            for r in rows:
                f.write(f"| {r['method']} | {r['setting']} | {r['accuracy']:.4f} | "
                        f"{r['pairs_per_s']:.3e} |\n")


if __name__ == "__main__":
    main()
