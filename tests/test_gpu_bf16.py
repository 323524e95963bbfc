"""GPU: the tcgen05 BF16 path against the oracle and against the FP32 path.

Bars:
* pooled features (bf16 operands, fp32 accumulation) against the float64
  oracle: |f - f*| <= 2e-2 * rms(f*) element-wise.  Each of the encoder's two
  bf16 matrix products rounds both operands (relative 2^-9 each); over the two
  layers and K <= 128 terms with mixed signs this stays below ~1 % of the
  feature scale, so 2 % leaves a margin of two;
* outputs against the FP32 GPU path on the full uneven scene: normals and
  depth within 1e-2, identical collision decisions (logit > 0) on >= 99.9 % of
  pairs;
* structure: empty crops pool to exact zeros, results are deterministic and do
  not depend on the batch they are in.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 0.25


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _det(lib, layers, prec):
    from paper_2304_09439_b300 import Detector
    _dev()
    return Detector(lib.points, lib.aabb, layers, R, prec)


@pytest.fixture(scope="module")
def tiny():
    lib = synth.tiny_library()
    poses, osh, pairs = synth.compose_relative_tiny(256, 0)
    layers = synth.xavier_weights(1, bias_scale=0.05)
    return lib, poses, osh, pairs, layers


@pytest.fixture(scope="module")
def scene64():
    lib = synth.make_library(64, 4)
    poses, osh, env = synth.uneven_scene(8192, 64, 4)
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    layers = synth.xavier_weights(1, bias_scale=0.05)
    return lib, poses, osh, env, pairs, layers


def test_bf16_features_match_oracle(tiny):
    lib, poses, osh, pairs, layers = tiny
    dev = _dev()
    params = oracle.flatten_params(layers)
    ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, R, params)
    xyz = np.zeros((len(pairs), 2, 64, 4), np.float32)
    xyz[..., :3] = ref["xyz"]
    xyz[..., 3] = np.arange(64)[None, None] < ref["cnt"][:, :, None]
    with _det(lib, layers, "bf16") as det:
        y, f = det.network(_t(xyz, dev), with_feat=True)
        det.status()
    f = f.cpu().numpy().astype(np.float64)
    fr = ref["feat"]
    rms = np.sqrt((fr ** 2).mean())
    err = np.abs(f - fr)
    print(f"bf16 features: max err / rms = {err.max() / rms:.3e}, mean {err.mean() / rms:.3e}")
    assert err.max() <= 2e-2 * rms
    empty = ref["cnt"] == 0
    fe = f.reshape(-1, 2, 256)
    assert np.all(fe[empty] == 0.0)
    yr, _ = oracle.network(params, ref["xyz"], ref["cnt"])
    yrms = np.sqrt((yr ** 2).mean(axis=0))
    yerr = np.abs(y.cpu().numpy() - yr) / yrms
    print("bf16 raw outputs: max err / column rms =", np.array2string(yerr.max(axis=0), precision=3))
    assert yerr.max() <= 5e-2


def test_bf16_vs_fp32_full_scene(scene64):
    lib, poses, osh, env, pairs, layers = scene64
    dev = _dev()
    tp, ts, tq = _t(poses, dev), _t(osh, dev), _t(pairs, dev)
    with _det(lib, layers, "fp32") as det:
        o32 = det.detect(tp, ts, tq).cpu().numpy()
        det.set_precision("bf16")
        o16 = det.detect(tp, ts, tq).cpu().numpy()
        o16b = det.detect(tp, ts, tq).cpu().numpy()
        det.status()
    assert np.array_equal(o16, o16b)
    dn = np.abs(o16[:, 4:7] - o32[:, 4:7]).max(axis=1)
    dd = np.abs(o16[:, 7] - o32[:, 7])
    agree = np.mean((o16[:, 0] > 0) == (o32[:, 0] > 0))
    print(f"bf16 vs fp32 on {len(pairs)} pairs: decisions agree {agree:.5f}, "
          f"normal err max {dn.max():.3e} p99.9 {np.quantile(dn, 0.999):.3e}, "
          f"depth err max {dd.max():.3e}")
    assert agree >= 0.999
    assert dd.max() <= 1e-2
    assert np.quantile(dn, 0.999) <= 1e-2


def test_bf16_batch_invariance_and_ragged_tiles(tiny):
    lib, poses, osh, pairs, layers = tiny
    dev = _dev()
    with _det(lib, layers, "bf16") as det:
        full = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs, dev)).cpu().numpy()
        for lo, hi in ((0, 1), (5, 132), (100, 229), (200, 256)):
            part = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs[lo:hi], dev)).cpu().numpy()
            np.testing.assert_array_equal(part, full[lo:hi])
        det.status()
