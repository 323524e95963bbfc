"""GPU: the voxel-latent variant against its oracle (``oracle/voxel.py``).

* latents of every library shape: float32 within 1e-4 of the float64 oracle
  (relative to max(|y|, rms of the latents));
* cell selection: the selected cell sets of both objects of every pair equal
  the oracle's bit for bit (float32 geometry in the same fixed order);
* pooled features and logits within 1e-4 (same guard);
* batch invariance at ragged sizes around the 32-pair tile, empty selections,
  out-of-range indices (NaN logit and BAD_INDEX), zero pairs.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import voxel as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _close(got, want, tol=1e-4):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.maximum(np.abs(want), np.sqrt(np.mean(want ** 2)) + 1e-30)
    err = np.abs(got - want) / scale
    assert err.max() <= tol, f"max scaled error {err.max():.3g} at {np.unravel_index(err.argmax(), err.shape)}"


def _masks_from_ranges(r):
    """[P, 2, 6] index ranges -> [P, 2, 6, 6, 6] masks."""
    P = r.shape[0]
    m = np.zeros((P, 2, 6, 6, 6), bool)
    i = np.arange(6)
    for p in range(P):
        for o in range(2):
            a = (i >= r[p, o, 0]) & (i <= r[p, o, 1])
            b = (i >= r[p, o, 2]) & (i <= r[p, o, 3])
            c = (i >= r[p, o, 4]) & (i <= r[p, o, 5])
            m[p, o] = a[:, None, None] & b[None, :, None] & c[None, None, :]
    return m


@pytest.fixture(scope="module")
def setup():
    from paper_2304_09439_b300 import VoxelDetector
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = synth.make_library(6, 3)
    flat = synth.voxel_weights(V.LAYERS, 7)
    prm = V.split_params(flat)
    lat_ref = V.encode_library(lib.points, lib.aabb, prm)
    det = VoxelDetector(lib.points, lib.aabb, flat)
    poses, osh, env = synth.uneven_scene(96, 6, seed=5)
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    yield dict(lib=lib, prm=prm, lat_ref=lat_ref, det=det, poses=poses, osh=osh, pairs=pairs)
    det.close()


def test_latents_match_oracle(setup):
    lat = setup["det"].latents().cpu().numpy()
    setup["det"].status()
    _close(lat, setup["lat_ref"].reshape(lat.shape))


def test_selection_pooling_and_logits_match_oracle(setup):
    dev = torch.device("cuda:0")
    det, pairs = setup["det"], setup["pairs"]
    assert len(pairs) > 200
    tp, ts, tq = (torch.from_numpy(a).to(dev) for a in (setup["poses"], setup["osh"], pairs))
    logit, ranges, pooled = det.detect(tp, ts, tq, details=True)
    det.status()
    ref = V.detect(setup["lat_ref"], setup["lib"].aabb, setup["poses"], setup["osh"], pairs,
                   setup["prm"])
    masks = _masks_from_ranges(ranges.cpu().numpy())
    np.testing.assert_array_equal(masks, ref["mask"])
    np.testing.assert_array_equal(masks.reshape(len(pairs), 2, -1).sum(-1), ref["cnt"])
    _close(pooled.cpu().numpy(), ref["feat"])
    _close(logit.cpu().numpy(), ref["logit"])
    # the scene has both decisions and both empty and full selections
    assert (ref["logit"] > 0).any() and (ref["logit"] <= 0).any()
    assert (ref["cnt"] == 0).any() and (ref["cnt"] > 8).any()


@pytest.mark.parametrize("n", [1, 31, 32, 33, 65, 200])
def test_batch_invariance_at_ragged_sizes(setup, n):
    dev = torch.device("cuda:0")
    det, pairs = setup["det"], setup["pairs"]
    tp, ts = (torch.from_numpy(a).to(dev) for a in (setup["poses"], setup["osh"]))
    full = det.detect(tp, ts, torch.from_numpy(pairs).to(dev)).cpu().numpy()
    part = det.detect(tp, ts, torch.from_numpy(np.ascontiguousarray(pairs[:n])).to(dev))
    det.status()
    np.testing.assert_array_equal(part.cpu().numpy(), full[:n])


def test_empty_selection_and_bad_indices(setup):
    from paper_2304_09439_b300 import LoccError
    dev = torch.device("cuda:0")
    det, lib = setup["det"], setup["lib"]
    poses = np.array([[1, 0, 0, 0, 0, 0, 0], [1, 0, 0, 0, 50.0, 0, 0],
                      [1, 0, 0, 0, 0.1, 0, 0]], np.float32)
    osh = np.array([0, 1, 2], np.int32)
    pairs = np.array([[0, 1], [0, 2], [0, 7], [2, 0]], np.int32)
    tp, ts, tq = (torch.from_numpy(a).to(dev) for a in (poses, osh, pairs))
    logit, ranges, pooled = det.detect(tp, ts, tq, details=True)
    with pytest.raises(LoccError):
        det.status()
    lg = logit.cpu().numpy()
    assert np.isnan(lg[2]) and np.isfinite(lg[[0, 1, 3]]).all()
    ok = np.array([0, 1, 3])
    ref = V.detect(setup["lat_ref"], lib.aabb, poses, osh, pairs[ok], setup["prm"])
    np.testing.assert_array_equal(_masks_from_ranges(ranges.cpu().numpy()[ok]), ref["mask"])
    assert ref["cnt"][0].tolist() == [0, 0]
    assert np.all(pooled.cpu().numpy()[0] == 0)
    _close(lg[ok], ref["logit"])
    # zero pairs: nothing to do, no error
    det.detect(tp, ts, torch.zeros((0, 2), dtype=torch.int32, device=dev))
    det.status()


def test_larger_library_sampled_against_oracle():
    # 16 shapes, 1024 environments: a sample of the pairs against the oracle
    from paper_2304_09439_b300 import VoxelDetector
    dev = torch.device("cuda:0")
    lib = synth.make_library(16, 4)
    flat = synth.voxel_weights(V.LAYERS, 11)
    prm = V.split_params(flat)
    poses, osh, env = synth.uneven_scene(1024, 16, seed=6)
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(len(pairs), 256, replace=False))
    with VoxelDetector(lib.points, lib.aabb, flat) as det:
        tp, ts, tq = (torch.from_numpy(a).to(dev) for a in (poses, osh, pairs))
        logit, ranges, pooled = det.detect(tp, ts, tq, details=True)
        lat = det.latents().cpu().numpy()
        det.status()
    used = np.unique(osh[pairs[sel]].ravel())
    lat_ref = np.zeros((16, 6, 6, 6, 16))
    for s in used:
        lat_ref[s] = V.encode_shape(lib.points[s], lib.aabb[s], prm)
    _close(lat[used], lat_ref[used].reshape(len(used), 216, 16))
    ref = V.detect(lat_ref, lib.aabb, poses, osh, pairs[sel], prm)
    np.testing.assert_array_equal(_masks_from_ranges(ranges.cpu().numpy()[sel]), ref["mask"])
    _close(pooled.cpu().numpy()[sel], ref["feat"])
    _close(logit.cpu().numpy()[sel], ref["logit"])


def test_bf16_tensor_core_predictor(setup):
    """tcgen05 predictor (bf16 operands, float32 accumulation): cell ranges
    and pooled features unchanged (they stay float32), logits within 5e-2 of
    max(|y|, rms) of the float64 oracle (seven layers of bf16 rounding,
    ~2^-9 per operand), the same decision on >= 97 % of pairs, batch-size
    invariant at tile edges; back to FP32 gives the FP32 results again."""
    dev = torch.device("cuda:0")
    det, pairs = setup["det"], setup["pairs"]
    tp, ts, tq = (torch.from_numpy(a).to(dev) for a in (setup["poses"], setup["osh"], pairs))
    l32, r32, f32 = det.detect(tp, ts, tq, details=True)
    det.set_precision("bf16")
    try:
        l16, r16, f16 = det.detect(tp, ts, tq, details=True)
        det.status()
        np.testing.assert_array_equal(r16.cpu().numpy(), r32.cpu().numpy())
        np.testing.assert_array_equal(f16.cpu().numpy(), f32.cpu().numpy())
        ref = V.detect(setup["lat_ref"], setup["lib"].aabb, setup["poses"], setup["osh"], pairs,
                       setup["prm"])["logit"]
        _close(l16.cpu().numpy(), ref, tol=5e-2)
        agree = np.mean((l16.cpu().numpy() > 0) == (ref > 0))
        assert agree >= 0.97, agree
        full = l16.cpu().numpy()
        for n in (1, 127, 128, 129, 255, 257):
            part = det.detect(tp, ts, torch.from_numpy(np.ascontiguousarray(pairs[:n])).to(dev))
            np.testing.assert_array_equal(part.cpu().numpy(), full[:n])
        det.status()
    finally:
        det.set_precision("fp32")
    again = det.detect(tp, ts, tq).cpu().numpy()
    det.status()
    np.testing.assert_array_equal(again, l32.cpu().numpy())
