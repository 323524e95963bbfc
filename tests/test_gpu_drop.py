"""GPU: the FP32 plain path on drop scenes against the oracle.

4096 environments, each dropping two objects of the 16-shape procedural
library (seed 3) onto a plane, 240 steps at dt = 1/240 s.  The poses come
from an integrator with analytic contacts (no input ever comes from the path
under test).  Every step runs ``locc_step`` (broadphase + detection) on the
device; at four steps the broadphase pairs must equal the oracle's bit for
bit, and a sample of the pairs must match oracle (b): crop index sets and
canonical coordinates bit-exact, float32 outputs within 1e-4 relative.
"""

import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R = 0.25
N_ENV = 4096
CHECK = (0, 80, 160, 239)


def test_drop_scene_fp32_matches_oracle():
    from paper_2304_09439_b300 import Detector, weights
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = synth.make_library(16, 3)
    with open(os.path.join(ROOT, "paper_2304_09439_b300", "weights", "locc_trained.bin"),
              "rb") as f:
        blob = f.read()
    params = oracle.flatten_params(weights.unpack(blob))
    max_pairs = N_ENV  # two objects per environment: at most one pair each
    checked = 0
    with Detector(lib.points, lib.aabb, blob, R, "fp32") as det:
        det.reserve(max_pairs, N_ENV)
        for step, poses, osh, env in synth.drop_scene(lib, N_ENV, 240, 8):
            tp, ts, te = (torch.from_numpy(a).to(dev) for a in (poses, osh, env))
            pairs, n_dev, out = det.step(tp, ts, te, max_pairs)
            if step not in CHECK:
                continue
            det.status()
            n = int(n_dev.item())
            ref_pairs = oracle.broadphase(lib.aabb, poses, osh, env)
            got = pairs[:n].cpu().numpy()
            np.testing.assert_array_equal(got, ref_pairs)
            if n == 0:
                continue
            rng = np.random.default_rng(step)
            sel = np.sort(rng.choice(n, min(n, 256), replace=False))
            ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, got[sel], R, params,
                                      n_threads=os.cpu_count() or 1)
            crop = det.crop(tp, ts, pairs[:n][torch.from_numpy(sel).to(dev)].contiguous())
            det.status()
            cnt = crop["cnt"].cpu().numpy()
            np.testing.assert_array_equal(cnt, ref["cnt"])
            gi = np.sort(np.where(np.arange(64) < cnt[..., None], crop["idx"].cpu().numpy(),
                                  1 << 30), axis=-1)
            ri = np.sort(np.where(np.arange(64) < ref["cnt"][..., None], ref["idx"], 1 << 30),
                         axis=-1)
            np.testing.assert_array_equal(gi, ri)
            o = out[:n].cpu().numpy()[sel].astype(np.float64)
            y = ref["out"]
            scale = np.maximum(np.abs(y), np.sqrt((y ** 2).mean(axis=0)) + 1e-30)
            bad = np.abs(o - y) > 1e-4 * scale
            assert not bad.any(), f"step {step}: {bad.sum()} outputs off, worst " \
                f"{np.max(np.abs(o - y) / scale):.3g}"
            checked += len(sel)
    assert checked >= 512
