"""GPU: the tcgen05 FP8 (e4m3) path against the oracle and the FP32 path.

e4m3 keeps 3 mantissa bits: one rounding has relative error u <= 2^-4.  Each
product in encoder layers 2-3 and the head rounds both operands once (scaled
per row / per output channel, so no value saturates); to first order a dot
product is off by at most 2u sum|a_k w_k|, which exceeds |sum a_k w_k| where
terms cancel, and the max-pool keeps the largest (upward) error of 64 points.
Bars, with the measured values printed (rms over all features, zeros of
empty crops included):
* pooled features vs the float64 oracle: mean |f - f*| <= 0.03 rms(f*),
  max <= 0.5 rms(f*);
* raw outputs vs the oracle: max error <= 0.5 of the column rms;
* decisions vs the FP32 path on the full uneven scene: >= 98 % identical.
Structure as for BF16: empty crops pool to exact zeros, batch invariance."""

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


def test_fp8_features_match_oracle():
    dev = _dev()
    lib = synth.tiny_library()
    poses, osh, pairs = synth.compose_relative_tiny(256, 0)
    layers = synth.xavier_weights(1, bias_scale=0.05)
    params = oracle.flatten_params(layers)
    ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, R, params)
    xyz = np.zeros((len(pairs), 2, 64, 4), np.float32)
    xyz[..., :3] = ref["xyz"]
    xyz[..., 3] = np.arange(64)[None, None] < ref["cnt"][:, :, None]
    with _det(lib, layers, "fp8") as det:
        y, f = det.network(_t(xyz, dev), with_feat=True)
        full = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs, dev)).cpu().numpy()
        part = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs[37:201], dev)).cpu().numpy()
        det.status()
    np.testing.assert_array_equal(part, full[37:201])
    f = f.cpu().numpy().astype(np.float64)
    fr = ref["feat"]
    rms = np.sqrt((fr ** 2).mean())
    err = np.abs(f - fr)
    print(f"fp8 features: max err / rms = {err.max() / rms:.3e}, mean {err.mean() / rms:.3e}")
    assert err.mean() <= 0.03 * rms and err.max() <= 0.5 * rms
    fe = f.reshape(-1, 2, 256)
    assert np.all(fe[ref["cnt"] == 0] == 0.0)
    yr, _ = oracle.network(params, ref["xyz"], ref["cnt"])
    yerr = np.abs(y.cpu().numpy() - yr) / np.sqrt((yr ** 2).mean(axis=0))
    print("fp8 raw outputs: max err / column rms =", np.array2string(yerr.max(axis=0), precision=3))
    assert yerr.max() <= 0.5


def test_fp8_vs_fp32_full_scene():
    dev = _dev()
    lib = synth.make_library(64, 4)
    poses, osh, env = synth.uneven_scene(8192, 64, 4)
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    layers = synth.xavier_weights(1, bias_scale=0.05)
    tp, ts, tq = _t(poses, dev), _t(osh, dev), _t(pairs, dev)
    with _det(lib, layers, "fp32") as det:
        o32 = det.detect(tp, ts, tq).cpu().numpy()
        det.set_precision("fp8")
        o8 = det.detect(tp, ts, tq).cpu().numpy()
        o8b = det.detect(tp, ts, tq).cpu().numpy()
        det.status()
    assert np.array_equal(o8, o8b)
    agree = np.mean((o8[:, 0] > 0) == (o32[:, 0] > 0))
    dn = np.abs(o8[:, 4:7] - o32[:, 4:7]).max(axis=1)
    dd = np.abs(o8[:, 7] - o32[:, 7])
    print(f"fp8 vs fp32 on {len(pairs)} pairs: decisions agree {agree:.5f}, normal err "
          f"p99 {np.quantile(dn, 0.99):.3e} max {dn.max():.3e}, depth err max {dd.max():.3e}")
    assert agree >= 0.98
