"""Write the precision-sweep workload and its oracle values (test infrastructure).

1,048,576 pairs over the 64-shape library (seed 5): half at uniform relative
poses, half placed near contact (approximate surface gap uniform in
[-0.05, 0.05]).  Oracle (a) is too slow for a million pairs, so it labels a
seeded stratified subset (half near-contact, half uniform; 16,384 pairs by
default) with {collide, contact point, normal, depth} in the world frame;
oracle (b) computes the float64 network outputs of the same subset for the
given weights.  This script calls only ``oracle`` and ``synth``; the product's
sweep runner reads the file it writes.

    python -m oracle.make_sweep --weights paper_2304_09439_b300/weights/locc_trained.bin \
        --out data/sweep_1m.npz
"""

from __future__ import annotations

import argparse
import os
import struct
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def read_blob(path: str) -> np.ndarray:
    """Flat float64 parameters of a LOCCW001 blob (W[out][in] then b[out] per
    layer, in the layer order of the network)."""
    with open(path, "rb") as f:
        raw = f.read()
    if raw[:8] != b"LOCCW001":
        raise ValueError("not a LOCCW001 blob")
    ver, n_layers = struct.unpack_from("<II", raw, 8)
    dims = [struct.unpack_from("<II", raw, 16 + 8 * i) for i in range(n_layers)]
    if ver != 1 or [tuple(d) for d in dims] != oracle.LAYER_DIMS:
        raise ValueError("unexpected blob header")
    o = 16 + 8 * n_layers
    flat = np.frombuffer(raw, "<f4", count=oracle.N_PARAMS, offset=o)
    return flat.astype(np.float64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--subset", type=int, default=16384)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--weights", required=True)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    t0 = time.time()
    lib = synth.make_library(64, 4)
    poses, osh, pairs, near = synth.sweep_pairs(lib, args.n, args.seed)
    rng = np.random.default_rng(args.seed + 1)
    half = args.subset // 2
    sub = np.sort(np.concatenate([rng.choice(np.nonzero(near)[0], half, replace=False),
                                  rng.choice(np.nonzero(~near)[0], args.subset - half,
                                             replace=False)]))
    t1 = time.time()
    objs = pairs[sub].ravel()
    sp = {"poses": poses[objs], "obj_shape": osh[objs],
          "pairs": np.arange(2 * len(sub), dtype=np.int32).reshape(-1, 2)}
    tgt = np.concatenate([oracle.contact(lib.meshes, lib.points, sp["poses"], sp["obj_shape"],
                                         sp["pairs"][i:i + 2048], n_threads=args.threads)
                          for i in range(0, len(sub), 2048)])
    t2 = time.time()
    params = read_blob(args.weights)
    res = oracle.crop_forward(lib.points, lib.aabb, sp["poses"], sp["obj_shape"], sp["pairs"],
                              0.25, params, n_threads=args.threads)
    t3 = time.time()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez_compressed(args.out, poses=poses, obj_shape=osh, pairs=pairs, near=near,
                        subset=sub.astype(np.int64), targets=tgt, oracle_b=res["out"],
                        weights=os.path.basename(args.weights), seed=args.seed)
    print(f"{args.out}: {args.n} pairs, subset {len(sub)}: generate {t1 - t0:.0f} s, "
          f"oracle (a) {t2 - t1:.0f} s, oracle (b) {t3 - t2:.0f} s, "
          f"{tgt[:, 0].mean():.3f} colliding in the subset", flush=True)


if __name__ == "__main__":
    main()
