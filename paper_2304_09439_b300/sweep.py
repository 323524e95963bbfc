"""Precision sweep: the contact path in FP32, BF16 and FP8 on 1,048,576 pairs.

    python -m paper_2304_09439_b300.sweep --data data/sweep_1m.npz \
        --weights paper_2304_09439_b300/weights/locc_trained.bin --md report.md

The input file (written by the oracle's sweep script) holds the pairs over the
64-shape library (half uniform relative poses, half near contact), a
stratified subset of 16,384 of them labelled by the geometric oracle (a), and
the float64 network outputs of oracle (b) on that subset.  For every
precision this runs ``locc_detect`` on all pairs and reports
* agreement with the FP32 path on all pairs: collision decisions, normal
  components and depth within 1e-2;
* error against oracle (b) (same network, float64) on the subset;
* accuracy against oracle (a) (geometry) on the subset: collision accuracy /
  F1, normal angle, contact-point distance, depth MAE;
* throughput of one ``locc_detect`` call on all pairs (CUDA events, median of
  three after a warm-up).
"""

from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PRECISIONS = ("fp32", "bf16", "fp8")


def _agree(a, b, tol=1e-2):
    """FP32 rows a vs another precision's rows b (all pairs)."""
    dn = np.abs(a[:, 4:7] - b[:, 4:7]).max(axis=1)
    dd = np.abs(a[:, 7] - b[:, 7])
    same = (a[:, 0] > 0) == (b[:, 0] > 0)
    return {"collide_agree": float(same.mean()),
            "normal_within_1e-2": float((dn <= tol).mean()),
            "depth_within_1e-2": float((dd <= tol).mean()),
            "all_within": float((same & (dn <= tol) & (dd <= tol)).mean()),
            "normal_absdiff_p50": float(np.percentile(dn, 50)),
            "normal_absdiff_p99": float(np.percentile(dn, 99)),
            "depth_absdiff_p50": float(np.percentile(dd, 50)),
            "depth_absdiff_p99": float(np.percentile(dd, 99)),
            "logit_absdiff_p99": float(np.percentile(np.abs(a[:, 0] - b[:, 0]), 99))}


def _vs_oracle_b(y, ref):
    """Against the float64 network: max and rms of the difference per output
    group, relative to the rms of the reference."""
    groups = {"logit": [0], "point": [1, 2, 3], "normal": [4, 5, 6], "depth": [7]}
    out = {}
    for name, cols in groups.items():
        d = np.abs(y[:, cols] - ref[:, cols])
        scale = float(np.sqrt(np.mean(ref[:, cols] ** 2))) or 1.0
        out[name] = {"max_abs": float(d.max()), "rms_abs": float(np.sqrt(np.mean(d ** 2))),
                     "rms_rel": float(np.sqrt(np.mean(d ** 2)) / scale)}
    out["collide_agree"] = float(np.mean((y[:, 0] > 0) == (ref[:, 0] > 0)))
    return out


def _vs_geometry(y, tgt):
    from .train import metrics
    m = metrics(y.astype(np.float32), tgt.astype(np.float32))
    hit = (y[:, 0] > 0) & (tgt[:, 0] > 0.5)
    m["point_err_mean"] = (float(np.linalg.norm(y[hit, 1:4] - tgt[hit, 1:4], axis=1).mean())
                           if hit.any() else float("nan"))
    return m


def run(data_path: str, weights_path: str, reps: int = 3) -> dict:
    import torch
    import synth
    from . import Detector
    d = np.load(data_path)
    lib = synth.make_library(64, 4)
    with open(weights_path, "rb") as f:
        blob = f.read()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    poses = torch.from_numpy(d["poses"]).to(dev)
    osh = torch.from_numpy(d["obj_shape"]).to(dev)
    pairs = torch.from_numpy(d["pairs"]).to(dev)
    P = pairs.shape[0]
    sub = d["subset"]
    report = {"pairs": int(P), "subset": int(len(sub)), "weights": os.path.basename(weights_path),
              "precisions": {}}
    outs = {}
    with Detector(lib.points, lib.aabb, blob, 0.25, "fp32") as det:
        det.reserve(P, 0)
        out = torch.empty((P, 8), dtype=torch.float32, device=dev)
        stream = torch.cuda.current_stream()
        for prec in PRECISIONS:
            det.set_precision(prec)
            det.detect(poses, osh, pairs, out=out)
            det.status()
            ms = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                det.detect(poses, osh, pairs, out=out)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            det.status()
            outs[prec] = out.cpu().numpy().copy()
            report["precisions"][prec] = {"pairs_per_s": P / (float(np.median(ms)) * 1e-3),
                                          "ms_per_call": float(np.median(ms))}
    for prec in PRECISIONS:
        r = report["precisions"][prec]
        if prec != "fp32":
            r["vs_fp32_all_pairs"] = _agree(outs["fp32"], outs[prec])
        r["vs_oracle_b_subset"] = _vs_oracle_b(outs[prec][sub].astype(np.float64), d["oracle_b"])
        r["vs_oracle_a_subset"] = _vs_geometry(outs[prec][sub], d["targets"])
    return report


def markdown(rep: dict, cmd: str) -> str:
    P = rep["precisions"]
    lines = [f"# Precision sweep: {rep['pairs']:,} pairs, FP32 vs BF16 vs FP8",
             "", f"Command: `{cmd}`", "",
             f"Weights: `{rep['weights']}`; oracle subset: {rep['subset']:,} pairs "
             "(half near contact, half uniform).", "",
             "| precision | pairs/s (one call) | collide agree vs FP32 | normal ≤1e-2 | "
             "depth ≤1e-2 | all three | F1 vs oracle (a) | accuracy | normal angle (deg, near) "
             "| depth MAE | max |Δ| depth vs oracle (b) |",
             "|---|---|---|---|---|---|---|---|---|---|---|"]
    for prec in PRECISIONS:
        r = P[prec]
        a = r.get("vs_fp32_all_pairs")
        g = r["vs_oracle_a_subset"]
        b = r["vs_oracle_b_subset"]
        ag = (f"{a['collide_agree']:.5f} | {a['normal_within_1e-2']:.5f} | "
              f"{a['depth_within_1e-2']:.5f} | {a['all_within']:.5f}") if a else "— | — | — | —"
        lines.append(f"| {prec} | {r['pairs_per_s']:.4g} | {ag} | {g['f1']:.4f} | "
                     f"{g['accuracy']:.4f} | {g['normal_angle_deg_near']:.1f} | "
                     f"{g['depth_mae']:.4f} | {b['depth']['max_abs']:.3g} |")
    lines += ["", "```json", json.dumps(rep, indent=1), "```", ""]
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--weights", required=True)
    ap.add_argument("--md", default=None)
    args = ap.parse_args()
    rep = run(args.data, args.weights)
    print(json.dumps(rep), flush=True)
    if args.md:
        cmd = " ".join(["python -m paper_2304_09439_b300.sweep"] + sys.argv[1:])
        with open(args.md, "w") as f:
            f.write(markdown(rep, cmd))


if __name__ == "__main__":
    main()
