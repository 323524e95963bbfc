"""Write a labelled contact dataset with the oracle (test infrastructure).

Training pairs follow the paper's data generation (Sec. III-A, Fig. 4): two
objects are placed far apart at random orientations, the shortest-distance
vector delta between them is computed, and one object is moved along delta so
that the remaining signed gap is a target s ~ N(0, 0.02 m) (negative = overlap;
the paper's |delta'| taken signed, see the readings of the paper in the design
notes).  Test pairs use uniform relative poses (the paper's test-set recipe,
Sec. IV-A) mixed half and half with near-contact placements.  Every label and
regression target -- {collide, contact point, normal, depth} in the world frame
-- comes from oracle (a); this script calls only ``oracle`` and ``synth``.

    python -m oracle.make_dataset --library train64 --mode train --n 60000 --out data/train.npz
"""

from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

LIBRARIES = {
    "train64": (64, 4),    # the benchmark library: "known objects"
    "unknown32": (32, 7),  # shapes never seen in training: "unknown objects"
    # training libraries of the data-efficiency comparison (Sec. IV-B,
    # Table I: 5 / 20 / 50 / 100 training objects)
    "few5": (5, 31),
    "few20": (20, 32),
    "few50": (50, 33),
    "few100": (100, 34),
}


def library(name: str):
    n, seed = LIBRARIES[name]
    return synth.make_library(n, seed)


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def distance_manipulated(lib, n, rng, sigma=0.02, far=3.0, threads=8, chunk=2048):
    """Pairs moved along their shortest-distance vector to a signed gap."""
    poses = np.zeros((2 * n, 7), np.float32)
    poses[0::2, :4] = synth.random_quaternions(n, rng)
    poses[1::2, :4] = synth.random_quaternions(n, rng)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    poses[0::2, 4:] = rng.uniform(-2, 2, size=(n, 3))
    poses[1::2, 4:] = poses[0::2, 4:] + far * u
    osh = rng.integers(0, lib.n_shapes, size=2 * n).astype(np.int32)
    pairs = np.stack([np.arange(0, 2 * n, 2), np.arange(1, 2 * n, 2)], 1).astype(np.int32)
    first = np.concatenate([oracle.contact(lib.meshes, lib.points, poses, osh,
                                           pairs[i:i + chunk], n_threads=threads)
                            for i in range(0, n, chunk)])
    s = rng.normal(0.0, sigma, size=n)
    for i in range(n):
        if first[i, 0] > 0:  # already touching at the far placement: keep as is
            continue
        gap = -first[i, 7]
        normal = first[i, 4:7]
        poses[2 * i + 1, 4:] -= ((gap - s[i]) * normal).astype(np.float32)
    return poses, osh, pairs


def uniform_and_near(lib, n, rng):
    poses, osh, pairs, near = synth.sweep_pairs(lib, n, int(rng.integers(1 << 30)),
                                                n_unique_near=max(64, n // 4))
    return poses, osh, pairs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--library", default="train64", choices=sorted(LIBRARIES))
    ap.add_argument("--mode", default="train", choices=["train", "test"])
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    rng = np.random.default_rng(args.seed)
    lib = library(args.library)
    t0 = time.time()
    if args.mode == "train":
        poses, osh, pairs = distance_manipulated(lib, args.n, rng, threads=args.threads)
    else:
        poses, osh, pairs = uniform_and_near(lib, args.n, rng)
    chunk = 2048
    tgt = np.concatenate([oracle.contact(lib.meshes, lib.points, poses, osh, pairs[i:i + chunk],
                                         n_threads=args.threads)
                          for i in range(0, len(pairs), chunk)])
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez_compressed(args.out, poses=poses, obj_shape=osh, pairs=pairs,
                        targets=tgt.astype(np.float32), library=args.library,
                        mode=args.mode, seed=args.seed)
    print(f"{args.out}: {len(pairs)} pairs, {tgt[:, 0].mean():.3f} colliding, "
          f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
