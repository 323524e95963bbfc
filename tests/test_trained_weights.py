"""CPU: the committed trained weights, checked without the GPU.

The weights blob parses and is finite, and run through oracle (b) (float64
crop network on the CPU) it beats the AABB broadphase alone on geometric
labels from oracle (a), on 512 pairs over shapes never seen in training
(the GPU test does the same on 2048 pairs through the CUDA path).
"""

import os

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2304_09439_b300", "weights", "locc_trained.bin")


def test_blob_parses():
    from paper_2304_09439_b300 import weights
    with open(WEIGHTS, "rb") as f:
        layers = weights.unpack(f.read())
    flat = weights.flat(layers)
    assert flat.shape == (oracle.N_PARAMS,) and np.all(np.isfinite(flat))
    assert [w.shape for w, _ in layers] == [(o, i) for i, o in oracle.LAYER_DIMS]


def test_trained_beats_broadphase_on_oracle():
    from paper_2304_09439_b300 import weights
    from paper_2304_09439_b300.train import aabb_overlap, metrics
    with open(WEIGHTS, "rb") as f:
        params = weights.flat(weights.unpack(f.read())).astype(np.float64)
    lib = synth.make_library(32, 7)
    poses, osh, pairs, _ = synth.sweep_pairs(lib, 512, 9002, n_unique_near=128)
    cores = os.cpu_count() or 1
    tgt = oracle.contact(lib.meshes, lib.points, poses, osh, pairs, n_threads=cores)
    res = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, 0.25, params,
                              n_threads=cores)
    data = {"poses": poses, "obj_shape": osh, "pairs": pairs}
    m = metrics(res["out"].astype(np.float32), tgt)
    base = metrics(aabb_overlap(lib, data), tgt)
    assert m["accuracy"] >= base["accuracy"] + 0.03, (m, base)
    assert m["f1"] >= base["f1"], (m, base)
