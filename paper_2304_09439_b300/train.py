"""Train the crop network on the GPU and evaluate it against geometric labels.

    python -m paper_2304_09439_b300.train --data data/train64.npz \
        --test data/test_known.npz data/test_unknown.npz \
        --steps 20000 --batch 256 --out paper_2304_09439_b300/weights/locc_trained.bin

Datasets are .npz files with poses [2n,7], obj_shape [2n], pairs [n,2] and
world-frame targets [n,8] = {collide, contact point, normal, depth} (written by
the dataset script of the test infrastructure from the geometric contact
detector) and the name of the procedural shape library they were drawn from.
Every step runs in liblocc: crop gather, float32 forward, loss, backward and
Adam (``locc_train_step``); this script only samples batches and rotations.
Rotation augmentation (Sec. III-A): each pair's canonical crop frame gets a
uniformly random rotation.  The paper trains with batch 32; a larger batch
keeps the GPU busy and is stated in the output.
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# procedural shape libraries by name: (number of shapes, seed)
LIBRARIES = {"train64": (64, 4), "unknown32": (32, 7)}
RADIUS = 0.25


def load_dataset(path):
    d = np.load(path)
    return {k: d[k] for k in ("poses", "obj_shape", "pairs", "targets")}, str(d["library"])


def make_library(name):
    import synth
    n, seed = LIBRARIES[name]
    return synth.make_library(n, seed)


def random_rotations(n, rng):
    """Uniform rotations (Shoemake quaternions) as row-major 3x3, float32 [n, 9]."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    x, y = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    z, w = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=1)
    return R.astype(np.float32)


def metrics(pred, tgt, near=0.05):
    """Collision accuracy / precision / recall / F1 (logit > 0 vs label), normal
    angle error in degrees on true collisions, depth MAE on pairs whose true
    depth is within `near` of contact (depth > -near)."""
    yp = pred[:, 0] > 0
    yt = tgt[:, 0] > 0.5
    tp = np.sum(yp & yt)
    fp = np.sum(yp & ~yt)
    fn = np.sum(~yp & yt)
    acc = float(np.mean(yp == yt))
    prec = float(tp / max(tp + fp, 1))
    rec = float(tp / max(tp + fn, 1))
    f1 = float(2 * prec * rec / max(prec + rec, 1e-12))
    m = yt & yp
    cosv = np.sum(pred[m, 4:7] * tgt[m, 4:7], axis=1)
    ang = float(np.degrees(np.arccos(np.clip(cosv, -1, 1))).mean()) if m.any() else float("nan")
    nm = tgt[:, 7] > -near
    mae = float(np.abs(pred[nm, 7] - tgt[nm, 7]).mean()) if nm.any() else float("nan")
    return {"accuracy": acc, "precision": prec, "recall": rec, "f1": f1,
            "normal_angle_deg": ang, "depth_mae": mae, "n": int(len(tgt))}


def evaluate(det, lib_name, data, dev, cache):
    """Run the detector on a dataset (its own shape library)."""
    import torch
    from paper_2304_09439_b300 import Detector
    if lib_name != cache["train_lib"]:
        if lib_name not in cache:
            cache[lib_name] = make_library(lib_name)
        lib = cache[lib_name]
        blob = cache["blob"]()
        with Detector(lib.points, lib.aabb, blob, RADIUS, det.precision) as d2:
            return _run(d2, data, dev)
    return _run(det, data, dev)


def _run(det, data, dev):
    import torch
    out = det.detect(torch.from_numpy(data["poses"]).to(dev),
                     torch.from_numpy(data["obj_shape"]).to(dev),
                     torch.from_numpy(data["pairs"]).to(dev)).cpu().numpy()
    det.status()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--test", nargs="*", default=[])
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-every", type=int, default=5000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    args = ap.parse_args()

    import torch
    import synth
    from paper_2304_09439_b300 import Detector, Trainer, weights

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    train, lib_name = load_dataset(args.data)
    lib = make_library(lib_name)
    tests = [(p,) + load_dataset(p) for p in args.test]
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(args.seed), RADIUS, "fp32")
    tr = Trainer(det, args.batch, lr=args.lr)
    cache = {"train_lib": lib_name, "blob": lambda: weights.pack(
        weights.from_flat(tr.params().cpu().numpy()))}

    report = {"train": args.data, "n_train": int(len(train["pairs"])), "batch": args.batch,
              "steps": args.steps, "lr": args.lr, "evals": []}

    def run_eval(step):
        row = {"step": step}
        for path, data, name in tests:
            tr.commit()
            for prec in ("fp32", "bf16"):
                det.set_precision(prec)
                row[f"{os.path.basename(path)}:{prec}"] = metrics(
                    evaluate(det, name, data, dev, cache), data["targets"])
            det.set_precision("fp32")
        report["evals"].append(row)
        print(json.dumps(row), flush=True)

    run_eval(0)
    P = len(train["pairs"])
    d_poses = torch.from_numpy(train["poses"]).to(dev)
    d_shape = torch.from_numpy(train["obj_shape"]).to(dev)
    d_tgt = torch.from_numpy(train["targets"]).to(dev)
    rng = np.random.default_rng(args.seed)
    B = args.batch
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hist = []
    t0 = time.time()
    for step in range(1, args.steps + 1):
        idx = rng.integers(0, P, B)
        objs = np.stack([2 * idx, 2 * idx + 1], 1).ravel()
        bp = d_poses[torch.from_numpy(objs).to(dev)]
        bs = d_shape[torch.from_numpy(objs).to(dev)]
        pairs = torch.arange(2 * B, dtype=torch.int32, device=dev).view(B, 2)
        bt = d_tgt[torch.from_numpy(idx).to(dev)]
        rot = torch.from_numpy(random_rotations(B, rng)).to(dev)
        tr.step(bp.contiguous(), bs.contiguous(), pairs, bt.contiguous(), rot, True, loss)
        if step % 200 == 0:
            hist.append((step, float(loss.item())))
        if step % args.eval_every == 0 or step == args.steps:
            print(f"step {step} loss {hist[-1][1]:.4f} {time.time() - t0:.0f} s", flush=True)
            run_eval(step)
    report["loss_history"] = hist
    report["train_seconds"] = time.time() - t0
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        with open(args.out, "wb") as f:
            f.write(weights.pack(weights.from_flat(tr.params().cpu().numpy())))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)
    tr.close()
    det.close()


if __name__ == "__main__":
    main()
