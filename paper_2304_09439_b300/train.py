"""Train the crop network on the GPU and evaluate it against geometric labels.

    python -m paper_2304_09439_b300.train --data data/train64.npz data/train64b.npz \
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
LIBRARIES = {"train64": (64, 4), "unknown32": (32, 7),
             # the data-efficiency comparison (Sec. IV-B): 5 / 20 / 50 / 100 shapes
             "few5": (5, 31), "few20": (20, 32), "few50": (50, 33), "few100": (100, 34)}
RADIUS = 0.25


def load_dataset(path):
    d = np.load(path)
    return {k: d[k] for k in ("poses", "obj_shape", "pairs", "targets")}, str(d["library"])


def concat(parts):
    """Concatenate datasets whose objects are numbered per file."""
    out = {"poses": [], "obj_shape": [], "pairs": [], "targets": []}
    base = 0
    for d in parts:
        out["poses"].append(d["poses"])
        out["obj_shape"].append(d["obj_shape"])
        out["pairs"].append(d["pairs"] + base)
        out["targets"].append(d["targets"])
        base += len(d["poses"])
    return {k: np.concatenate(v) for k, v in out.items()}


def split(data, n_val, rng):
    """Hold out n_val pairs (with their two objects) for checkpoint selection.
    Training files store pair i as objects (2i, 2i+1)."""
    n = len(data["pairs"])
    perm = rng.permutation(n)
    parts = []
    for idx in (perm[n_val:], perm[:n_val]):
        objs = data["pairs"][idx].ravel()
        parts.append({"poses": data["poses"][objs], "obj_shape": data["obj_shape"][objs],
                      "pairs": np.arange(2 * len(idx), dtype=np.int32).reshape(-1, 2),
                      "targets": data["targets"][idx]})
    return parts


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
    mn = m & (np.abs(tgt[:, 7]) < near)
    cosn = np.sum(pred[mn, 4:7] * tgt[mn, 4:7], axis=1)
    ang_near = (float(np.degrees(np.arccos(np.clip(cosn, -1, 1))).mean())
                if mn.any() else float("nan"))
    return {"accuracy": acc, "precision": prec, "recall": rec, "f1": f1,
            "normal_angle_deg": ang, "normal_angle_deg_near": ang_near,
            "depth_mae": mae, "n": int(len(tgt))}


def aabb_overlap(lib, data):
    """The method without the network: a pair collides when the world AABBs
    of the two posed OBBs overlap (the broadphase test).  Returns [n, 8] with
    +1/-1 logits and zero regression outputs, so ``metrics`` applies."""
    q = data["poses"][:, :4].astype(np.float64)
    w, x, y, z = q.T
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
                 axis=1).reshape(-1, 3, 3)
    box = np.asarray(lib.aabb, np.float64)[data["obj_shape"]]
    c = 0.5 * (box[:, :3] + box[:, 3:])
    h = 0.5 * (box[:, 3:] - box[:, :3])
    wc = np.einsum("nij,nj->ni", R, c) + data["poses"][:, 4:]
    wh = np.einsum("nij,nj->ni", np.abs(R), h)
    a, b = data["pairs"][:, 0], data["pairs"][:, 1]
    hit = np.all(np.abs(wc[a] - wc[b]) <= wh[a] + wh[b], axis=1)
    out = np.zeros((len(a), 8), np.float32)
    out[:, 0] = np.where(hit, 1.0, -1.0)
    return out


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
            d2.set_crop_mode(cache.get("crop_mode", "local"))
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
    ap.add_argument("--data", nargs="+", required=True)
    ap.add_argument("--test", nargs="*", default=[])
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=0.02,
                    help="cosine decay to lr * lr_final at the last step (1 = constant)")
    ap.add_argument("--val", type=int, default=4096, help="held-out pairs for checkpoint selection")
    ap.add_argument("--eval-every", type=int, default=5000)
    ap.add_argument("--val-every", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--w-len", type=float, default=0.0,
                    help="weight of the raw-normal length term (|n| - 1)^2 on every pair")
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    ap.add_argument("--checkpoint", default=None,
                    help="write a training checkpoint (parameters, Adam state, step, sampler "
                         "state, best-so-far) here at every validation and at the end")
    ap.add_argument("--resume", default=None, help="continue from a checkpoint of this run")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="trainer arithmetic: float32 CUDA cores, or the dense products on "
                         "the tensor cores with bf16 operands (float32 accumulation and state)")
    ap.add_argument("--crop-mode", default="local", choices=["local", "global"],
                    help="local crops (the method) or global crops (the ablation without "
                         "locality)")
    args = ap.parse_args()

    import torch
    import synth
    from paper_2304_09439_b300 import Detector, Trainer, weights

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    loaded = [load_dataset(p) for p in args.data]
    lib_name = loaded[0][1]
    if any(n != lib_name for _, n in loaded):
        raise SystemExit("all --data files must use one shape library")
    rng = np.random.default_rng(args.seed)
    train, val = split(concat([d for d, _ in loaded]), args.val, rng)
    lib = make_library(lib_name)
    tests = [(p,) + load_dataset(p) for p in args.test]
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(args.seed), RADIUS, "fp32")
    det.set_crop_mode(args.crop_mode)
    tr = Trainer(det, args.batch, lr=args.lr, w_len=args.w_len, precision=args.precision)
    cache = {"train_lib": lib_name, "crop_mode": args.crop_mode, "blob": lambda: weights.pack(
        weights.from_flat(tr.params().cpu().numpy()))}

    report = {"train": args.data, "n_train": int(len(train["pairs"])),
              "n_val": int(len(val["pairs"])), "batch": args.batch, "steps": args.steps,
              "lr": args.lr, "lr_final": args.lr_final, "schedule": "cosine",
              "crop_mode": args.crop_mode, "precision": args.precision, "evals": [],
              "val": []}

    def run_eval(step):
        row = {"step": step}
        for path, data, name in tests:
            tr.commit()
            for prec in ("fp32", "bf16", "fp8"):
                det.set_precision(prec)
                pred = evaluate(det, name, data, dev, cache)
                row[f"{os.path.basename(path)}:{prec}"] = metrics(pred, data["targets"])
                if prec == "fp32":
                    # pairs within 5 cm of contact (true depth > -0.05) and the rest
                    near = data["targets"][:, 7] > -0.05
                    for tag, m in (("near", near), ("far", ~near)):
                        if m.any():
                            row[f"{os.path.basename(path)}:fp32:{tag}"] = metrics(
                                pred[m], data["targets"][m])
            det.set_precision("fp32")
            tl = lib if name == lib_name else cache.setdefault(name, make_library(name))
            row[f"{os.path.basename(path)}:aabb"] = metrics(aabb_overlap(tl, data),
                                                            data["targets"])
        report["evals"].append(row)
        print(json.dumps(row), flush=True)

    def run_val():
        tr.commit()
        return metrics(_run(det, val, dev), val["targets"])

    P = len(train["pairs"])
    d_poses = torch.from_numpy(train["poses"]).to(dev)
    d_shape = torch.from_numpy(train["obj_shape"]).to(dev)
    d_tgt = torch.from_numpy(train["targets"]).to(dev)
    B = args.batch
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hist = []
    best = (-1.0, 0, None)
    first = 1
    if args.resume:
        first, best, hist = load_checkpoint(args.resume, tr, rng, report, dev)
    else:
        run_eval(0)
    # batches go to the device from page-locked buffers without blocking, so
    # the host draws batch k + 1 while the GPU runs step k; each of the
    # NBUF buffers is reused only once its copy has run (same draws, in the
    # same order, as a blocking copy)
    NBUF = 3
    h_objs = [torch.empty(2 * B, dtype=torch.int64).pin_memory() for _ in range(NBUF)]
    h_idx = [torch.empty(B, dtype=torch.int64).pin_memory() for _ in range(NBUF)]
    h_rot = [torch.empty((B, 9), dtype=torch.float32).pin_memory() for _ in range(NBUF)]
    copied = [None] * NBUF
    pairs = torch.arange(2 * B, dtype=torch.int32, device=dev).view(B, 2)
    t0 = time.time()
    for step in range(first, args.steps + 1):
        tr.set_lr(tr_lr(args, step))
        k = step % NBUF
        if copied[k] is not None:
            copied[k].synchronize()
        idx = rng.integers(0, P, B)
        h_idx[k].numpy()[:] = idx
        h_objs[k].numpy()[:] = np.stack([2 * idx, 2 * idx + 1], 1).ravel()
        h_rot[k].numpy()[:] = random_rotations(B, rng)
        d_objs = h_objs[k].to(dev, non_blocking=True)
        d_idx = h_idx[k].to(dev, non_blocking=True)
        rot = h_rot[k].to(dev, non_blocking=True)
        copied[k] = torch.cuda.Event()
        copied[k].record()
        bp = d_poses[d_objs]
        bs = d_shape[d_objs]
        bt = d_tgt[d_idx]
        tr.step(bp.contiguous(), bs.contiguous(), pairs, bt.contiguous(), rot, True, loss)
        if step % 200 == 0:
            hist.append((step, float(loss.item())))
        if step % args.val_every == 0 or step == args.steps:
            v = run_val()
            report["val"].append({"step": step, **v})
            # checkpoint selection: collision accuracy first, regression error second
            score = v["f1"] - 1e-3 * v["depth_mae"]
            if score > best[0]:
                best = (score, step, tr.params().clone())
            if args.checkpoint:
                save_checkpoint(args.checkpoint, tr, step, rng, best, hist, report)
        if step % args.eval_every == 0 or step == args.steps:
            print(f"step {step} loss {hist[-1][1]:.4f} lr {tr_lr(args, step):.2e} "
                  f"{time.time() - t0:.0f} s", flush=True)
            run_eval(step)
    report["loss_history"] = hist
    report["train_seconds"] = time.time() - t0
    report["best_step"] = best[1]
    tr.set_params(best[2])
    run_eval(-best[1])
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        with open(args.out, "wb") as f:
            f.write(weights.pack(weights.from_flat(best[2].cpu().numpy())))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)
    tr.close()
    det.close()


def save_checkpoint(path, tr, step, rng, best, hist, report):
    """Everything a resumed run needs, written atomically: parameters, Adam
    moments and step count, the last finished step, the batch sampler's state,
    the best-so-far parameters and the history kept for the report."""
    m, v, adam_step = tr.state()
    js = lambda o: np.frombuffer(json.dumps(o).encode(), np.uint8)
    state = dict(params=tr.params().cpu().numpy(), m=m.cpu().numpy(), v=v.cpu().numpy(),
                 adam_step=np.int64(adam_step), step=np.int64(step),
                 rng=js(rng.bit_generator.state), best_score=np.float64(best[0]),
                 best_step=np.int64(best[1]),
                 best_params=(best[2].cpu().numpy() if best[2] is not None
                              else np.zeros(0, np.float32)),
                 hist=np.array(hist, np.float64).reshape(-1, 2),
                 report=js({"val": report["val"], "evals": report["evals"]}))
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, **state)
    os.replace(tmp, path)


def load_checkpoint(path, tr, rng, report, dev):
    """Restore a checkpoint written by save_checkpoint into the trainer, the
    sampler and the report; returns (first step to run, best, history)."""
    import torch
    ck = np.load(path)
    tr.set_params(torch.from_numpy(ck["params"]).to(dev))
    tr.set_state(torch.from_numpy(ck["m"]).to(dev), torch.from_numpy(ck["v"]).to(dev),
                 int(ck["adam_step"]))
    rng.bit_generator.state = json.loads(bytes(ck["rng"]).decode())
    saved = json.loads(bytes(ck["report"]).decode())
    report["val"], report["evals"] = saved["val"], saved["evals"]
    bp = ck["best_params"]
    best = (float(ck["best_score"]), int(ck["best_step"]),
            torch.from_numpy(bp).to(dev) if bp.size else None)
    hist = [(int(a), float(b)) for a, b in ck["hist"]]
    return int(ck["step"]) + 1, best, hist


def tr_lr(args, step):
    """Cosine decay from lr to lr * lr_final over the run."""
    frac = (step - 1) / max(args.steps - 1, 1)
    return args.lr * (args.lr_final + (1 - args.lr_final) * 0.5 * (1 + np.cos(np.pi * frac)))


if __name__ == "__main__":
    main()
