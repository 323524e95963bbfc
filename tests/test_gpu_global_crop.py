"""GPU: global crops (the ablation without locality) against oracle (b).

With the crop mode set to global, every object keeps its first 64 surface
samples in the canonical crop frame: indices, counts and coordinates must
equal oracle (b)'s global mode bit for bit, and the FP32 network outputs must
match within 1e-4 (relative to max(|y|, rms of the column)).  The mode is a
property of the handle: switching back gives the local crops again.
"""

import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_global_crops_match_oracle_and_switch_back():
    from paper_2304_09439_b300 import Detector
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = synth.make_library(8, 3)
    layers = synth.xavier_weights(1, bias_scale=0.05)
    params = oracle.flatten_params(layers)
    poses, osh, env = synth.uneven_scene(64, 8, seed=9)
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)[:300]
    tp, ts, tq = (torch.from_numpy(a).to(dev) for a in (poses, osh, pairs))
    with Detector(lib.points, lib.aabb, layers, 0.25, "fp32") as det:
        det.set_crop_mode("global")
        crop = det.crop(tp, ts, tq)
        out = det.detect(tp, ts, tq).cpu().numpy()
        det.status()
        ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, 0.25, params,
                                  n_threads=os.cpu_count() or 1, mode="global")
        np.testing.assert_array_equal(crop["cnt"].cpu().numpy(), ref["cnt"])
        np.testing.assert_array_equal(crop["idx"].cpu().numpy(), ref["idx"])
        np.testing.assert_array_equal(crop["xyz"].cpu().numpy()[..., :3], ref["xyz"])
        y = ref["out"]
        scale = np.maximum(np.abs(y), np.sqrt((y ** 2).mean(axis=0)) + 1e-30)
        assert (np.abs(out - y) <= 1e-4 * scale).all()
        # back to the method's local crops
        det.set_crop_mode("local")
        loc = det.crop(tp, ts, tq)
        det.status()
        ref_l = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, 0.25,
                                    n_threads=os.cpu_count() or 1)
        np.testing.assert_array_equal(loc["cnt"].cpu().numpy(), ref_l["cnt"])
        # the two modes select different points
        assert not np.array_equal(loc["idx"].cpu().numpy(), crop["idx"].cpu().numpy())
