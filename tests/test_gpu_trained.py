"""GPU: what the trained crop network gains over the method without it.

Test set: 2048 pairs over a 32-shape library never used in training
(procedural, seed 7), half at uniform relative poses and half placed near
contact (gap in [-0.05, 0.05]), labelled by the geometric oracle (a).

Compared on the same pairs:
* the method without a learned detector: the AABB broadphase alone (a pair
  collides when the world boxes of its two objects overlap; no contact point,
  normal or depth);
* the same network untrained (Xavier initialisation);
* the committed trained weights (trained on the GPU by this library's own
  forward / backward kernels), in FP32, BF16 and FP8.

Bars: the trained network beats the broadphase on collision accuracy and F1
and beats the untrained network on F1; its normals near contact are far
better than chance (mean angle 90 degrees) and its depth error is below that
of predicting zero depth.
"""

import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2304_09439_b300", "weights", "locc_trained.bin")
R = 0.25


@pytest.fixture(scope="module")
def testset():
    lib = synth.make_library(32, 7)
    poses, osh, pairs, near = synth.sweep_pairs(lib, 2048, 9001, n_unique_near=512)
    tgt = oracle.contact(lib.meshes, lib.points, poses, osh, pairs,
                         n_threads=os.cpu_count() or 1)
    return lib, {"poses": poses, "obj_shape": osh, "pairs": pairs, "targets": tgt}


def _run(lib, layers, prec, data):
    from paper_2304_09439_b300 import Detector
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    with Detector(lib.points, lib.aabb, layers, R, prec) as det:
        out = det.detect(*(torch.from_numpy(data[k]).to(dev)
                           for k in ("poses", "obj_shape", "pairs")))
        det.status()
        return out.cpu().numpy()


def test_trained_network_gain(testset):
    from paper_2304_09439_b300.train import aabb_overlap, metrics
    lib, data = testset
    tgt = data["targets"]
    with open(WEIGHTS, "rb") as f:
        blob = f.read()
    base = metrics(aabb_overlap(lib, data), tgt)
    untrained = metrics(_run(lib, synth.xavier_weights(1), "fp32", data), tgt)
    zero_depth = float(np.abs(tgt[tgt[:, 7] > -0.05, 7]).mean())
    for prec in ("fp32", "bf16", "fp8"):
        m = metrics(_run(lib, blob, prec, data), tgt)
        print(prec, m, "aabb", base, "untrained", untrained)
        assert m["accuracy"] >= base["accuracy"] + 0.04, (prec, m, base)
        assert m["f1"] >= base["f1"] + 0.01, (prec, m, base)
        assert m["f1"] >= untrained["f1"] + 0.02, (prec, m, untrained)
        assert m["normal_angle_deg_near"] <= 55.0, (prec, m)
        assert m["depth_mae"] <= 0.9 * zero_depth, (prec, m, zero_depth)
