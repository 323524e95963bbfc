"""GPU parity: the CUDA path through the C ABI against the oracle.

* crop index sets, counts, centres and canonical coordinates: bit-exact;
* float32 network outputs: |x - y| <= 1e-4 max(|y|, rms of the column);
* broadphase pair lists: bit-exact.
Sizes span several tiles with ragged tails; the full-size uneven scene is
checked on a sampled subset of its pairs."""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 0.25
TOL = 1e-4


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def assert_close_rel(got, ref, tol=TOL, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    rms = np.sqrt((ref ** 2).mean(axis=0, keepdims=True)) + 1e-30
    scale = np.maximum(np.abs(ref), rms)
    err = np.abs(got - ref) / scale
    bad = np.argwhere(err > tol)
    assert bad.size == 0, f"{what}: {len(bad)} elements off, worst {err.max():.3g} at {bad[:5]}"


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


def _detector(lib, layers, prec="fp32"):
    from paper_2304_09439_b300 import Detector
    _dev()
    return Detector(lib.points, lib.aabb, layers, R, prec)


def canonical_order(idx, xyz, cnt):
    """Selected points of every object crop in ascending library index (the
    crop's point order is a fixed storage order, not part of the result: the
    network max-pools over points, so only the selected set matters)."""
    idx = idx.copy()
    xyz = xyz.copy()
    for p in range(idx.shape[0]):
        for o in range(2):
            c = int(cnt[p, o])
            order = np.argsort(idx[p, o, :c], kind="stable")
            idx[p, o, :c] = idx[p, o, :c][order]
            xyz[p, o, :c] = xyz[p, o, :c][order]
    return idx, xyz


def _check_crop(det, lib, poses, osh, pairs, sample=None, points=None, radius=R):
    dev = _dev()
    c = det.crop(_t(poses, dev), _t(osh, dev), _t(pairs, dev))
    det.status()
    sel = np.arange(len(pairs)) if sample is None else sample
    pts = lib.points if points is None else points
    ref = oracle.crop_forward(pts, lib.aabb, poses, osh, pairs[sel], radius, n_threads=8)
    cnt = c["cnt"].cpu().numpy()[sel]
    idx = c["idx"].cpu().numpy()[sel]
    xyz = c["xyz"].cpu().numpy()[sel]
    cen = c["centre"].cpu().numpy()[sel]
    np.testing.assert_array_equal(cnt, ref["cnt"])
    idx, xyz = canonical_order(idx, xyz, cnt)
    ridx, rxyz = canonical_order(ref["idx"], ref["xyz"], ref["cnt"])
    np.testing.assert_array_equal(idx, ridx)
    np.testing.assert_array_equal(cen[:, :3], ref["centre"])
    np.testing.assert_array_equal(xyz[..., :3], rxyz)
    valid = np.arange(64)[None, None, :] < cnt[:, :, None]
    np.testing.assert_array_equal(xyz[..., 3], valid.astype(np.float32))
    return ref


def test_crop_bit_exact_tiny(tiny):
    lib, poses, osh, pairs, layers = tiny
    with _detector(lib, layers) as det:
        ref = _check_crop(det, lib, poses, osh, pairs)
    assert (ref["cnt"] == 64).sum() > 10 and (ref["cnt"] == 0).sum() > 10


@pytest.mark.parametrize("copies,radius", [(48, 0.35), (128, 0.4), (1, 0.6), (1, 1.5)])
def test_crop_selection_paths(tiny, copies, radius):
    # samples repeated `copies` times (many equal distances: ties go to the
    # lower index, and the histogram bin that holds the 64th key can hold more
    # keys than the rank buffer) and large balls (hundreds to thousands of
    # in-ball samples: the histogram re-scan and streaming top-64 path)
    from paper_2304_09439_b300 import Detector
    lib, poses, osh, pairs, layers = tiny
    pts = lib.points.copy()
    if copies > 1:
        for s_ in range(pts.shape[0]):
            pts[s_] = pts[s_][(np.arange(pts.shape[1]) // copies) * copies]
    _dev()
    with Detector(pts, lib.aabb, layers, radius, "fp32") as det:
        ref = _check_crop(det, lib, poses, osh, pairs, points=pts, radius=radius)
    assert (ref["cnt"] == 64).sum() > 10


def test_fp32_outputs_match_oracle_tiny(tiny):
    lib, poses, osh, pairs, layers = tiny
    dev = _dev()
    ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, R,
                              oracle.flatten_params(layers))
    with _detector(lib, layers) as det:
        out = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs, dev))
        det.status()
        assert_close_rel(out.cpu().numpy(), ref["out"], what="detect fp32")
        # network alone on the oracle's crops
        xyz = np.zeros((len(pairs), 2, 64, 4), np.float32)
        xyz[..., :3] = ref["xyz"]
        xyz[..., 3] = (np.arange(64)[None, None] < ref["cnt"][:, :, None])
        y, f = det.network(_t(xyz, dev), with_feat=True)
        yr, fr = oracle.network(oracle.flatten_params(layers), ref["xyz"], ref["cnt"])
        assert_close_rel(f.cpu().numpy(), fr, what="pooled features")
        assert_close_rel(y.cpu().numpy(), yr, what="raw head outputs")


def test_detect_ragged_sizes_and_determinism(tiny):
    lib, poses, osh, pairs, layers = tiny
    dev = _dev()
    params = oracle.flatten_params(layers)
    with _detector(lib, layers) as det:
        for n in (1, 31, 33, 200):
            sub = pairs[:n]
            ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, sub, R, params)
            a = det.detect(_t(poses, dev), _t(osh, dev), _t(sub, dev)).cpu().numpy()
            b = det.detect(_t(poses, dev), _t(osh, dev), _t(sub, dev)).cpu().numpy()
            assert np.array_equal(a, b)
            assert_close_rel(a, ref["out"], what=f"n={n}")
        # empty call is a no-op
        empty = torch.zeros((0, 2), dtype=torch.int32, device=dev)
        out = det.detect(_t(poses, dev), _t(osh, dev), empty)
        assert out.shape == (0, 8)
        det.status()


def test_detect_host_matches_device(tiny):
    lib, poses, osh, pairs, layers = tiny
    dev = _dev()
    with _detector(lib, layers) as det:
        a = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs, dev)).cpu().numpy()
        b = det.detect_host(poses, osh, pairs)
        assert np.array_equal(a, b)


def test_bad_index_flags_error_and_nan_row(tiny):
    from paper_2304_09439_b300 import LoccError
    lib, poses, osh, pairs, layers = tiny
    dev = _dev()
    bad = pairs[:4].copy()
    bad[2, 1] = 10_000
    with _detector(lib, layers) as det:
        out = det.detect(_t(poses, dev), _t(osh, dev), _t(bad, dev)).cpu().numpy()
        with pytest.raises(LoccError) as e:
            det.status()
        assert e.value.code == -6
        assert np.all(np.isnan(out[2])) and np.all(np.isfinite(out[[0, 1, 3]]))
        det.status()  # flag cleared


def test_identical_overlapping_objects_and_small_libraries():
    # same shape at the same pose (full overlap); libraries whose point count
    # is not a multiple of 32 and smaller than the crop size
    dev = _dev()
    layers = synth.xavier_weights(1, bias_scale=0.05)
    params = oracle.flatten_params(layers)
    for n_points in (1000, 40, 7):
        lib = synth.tiny_library(n_points=n_points, seed=3)
        rng = np.random.default_rng(n_points)
        poses = synth.random_poses(40, rng, -0.3, 0.3)
        poses[1] = poses[0]
        osh = rng.integers(0, 2, 40).astype(np.int32)
        osh[1] = osh[0]
        pairs = rng.integers(0, 40, (97, 2)).astype(np.int32)
        pairs[0] = (0, 1)
        pairs[1] = (5, 5)
        with _detector(lib, layers) as det:
            _check_crop(det, lib, poses, osh, pairs)
            ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, R, params)
            out = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs, dev)).cpu().numpy()
            assert_close_rel(out, ref["out"], what=f"n_points={n_points}")


def test_crop_full_size_uneven_scene_sampled(scene64):
    lib, poses, osh, env, pairs, layers = scene64
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(len(pairs), 3000, replace=False))
    with _detector(lib, layers) as det:
        ref = _check_crop(det, lib, poses, osh, pairs, sample)
    assert (ref["cnt"] == 64).mean() > 0.2


def test_fp32_full_size_uneven_scene_sampled(scene64):
    lib, poses, osh, env, pairs, layers = scene64
    dev = _dev()
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(len(pairs), 1500, replace=False))
    ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs[sample], R,
                              oracle.flatten_params(layers), n_threads=8)
    with _detector(lib, layers) as det:
        out = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs, dev))
        det.status()
        assert_close_rel(out.cpu().numpy()[sample], ref["out"], what="uneven fp32")


def test_broadphase_bit_exact(scene64):
    lib, poses, osh, env, pairs, layers = scene64
    dev = _dev()
    with _detector(lib, layers) as det:
        got, n = det.broadphase(_t(poses, dev), _t(osh, dev), _t(env, dev), 400_000)
        det.status()
        n = int(n.item())
        assert n == len(pairs)
        np.testing.assert_array_equal(got[:n].cpu().numpy(), pairs)
        # truncated output keeps the full count and the first max_pairs pairs
        got2, n2 = det.broadphase(_t(poses, dev), _t(osh, dev), _t(env, dev), 1000)
        assert int(n2.item()) == len(pairs)
        np.testing.assert_array_equal(got2[:1000].cpu().numpy(), pairs[:1000])
        # small ragged case: environments of 0, 1, 2, 25, 40 objects
        counts = np.array([0, 1, 2, 25, 40, 3], np.int64)
        off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        rng = np.random.default_rng(9)
        p2 = synth.random_poses(int(off[-1]), rng, -0.8, 0.8)
        s2 = rng.integers(0, 64, int(off[-1])).astype(np.int32)
        ref = oracle.broadphase(lib.aabb, p2, s2, off)
        got3, n3 = det.broadphase(_t(p2, dev), _t(s2, dev), _t(off, dev), 5000)
        assert int(n3.item()) == len(ref)
        np.testing.assert_array_equal(got3[:len(ref)].cpu().numpy(), ref)


def test_step_matches_broadphase_then_detect(scene64):
    lib, poses, osh, env, pairs, layers = scene64
    dev = _dev()
    params = oracle.flatten_params(layers)
    with _detector(lib, layers) as det:
        det.reserve(400_000, len(env) - 1)
        tp, ts, te = _t(poses, dev), _t(osh, dev), _t(env, dev)
        pr, n, out = det.step(tp, ts, te, 400_000)
        det.status()
        n = int(n.item())
        assert n == len(pairs)
        np.testing.assert_array_equal(pr[:n].cpu().numpy(), pairs)
        ref_dev = det.detect(tp, ts, _t(pairs, dev)).cpu().numpy()
        np.testing.assert_array_equal(out[:n].cpu().numpy(), ref_dev)
        # host-buffer step returns the same pairs and outputs
        hp, ho, hn = det.step_host(poses, osh, env, 400_000)
        assert hn == n
        np.testing.assert_array_equal(hp, pairs)
        np.testing.assert_array_equal(ho, ref_dev)
        # page-locked buffers (copied directly, no staging); rows beyond the
        # count untouched
        def pin(a):
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        h_out = torch.full((400_000, 8), -7.0, dtype=torch.float32).pin_memory().numpy()
        h_pairs = torch.zeros((400_000, 2), dtype=torch.int32).pin_memory().numpy()
        hp, ho, hn = det.step_host(pin(poses), pin(osh), pin(env), 400_000, pairs_out=h_pairs,
                                   out=h_out)
        assert hn == n
        np.testing.assert_array_equal(hp, pairs)
        np.testing.assert_array_equal(ho, ref_dev)
        assert np.all(h_out[n:] == -7.0)
        h_out[:] = 0.0
        hp, ho, hn = det.step_host(poses, osh, env, 400_000, out=h_out)  # mixed pageable / pinned
        np.testing.assert_array_equal(hp, pairs)
        np.testing.assert_array_equal(ho, ref_dev)
        # a step with fewer pair slots than candidates detects only the first ones
        pr2, n2, out2 = det.step(tp, ts, te, 777)
        assert int(n2.item()) == n
        np.testing.assert_array_equal(out2[:777].cpu().numpy(), ref_dev[:777])
        rng = np.random.default_rng(3)
        sample = rng.choice(n, 500, replace=False)
        ref = oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs[sample], R, params,
                                  n_threads=8)
        assert_close_rel(ref_dev[sample], ref["out"], what="step outputs")


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_pipelined_step_is_bit_identical(scene64, prec):
    lib, poses, osh, env, pairs, layers = scene64
    dev = _dev()
    with _detector(lib, layers, prec) as det:
        det.reserve(400_000, len(env) - 1)
        tp, ts, te = _t(poses, dev), _t(osh, dev), _t(env, dev)
        _, n, ref = det.step(tp, ts, te, 400_000)
        n = int(n.item())
        ref = ref[:n].cpu().numpy()
        for chunks, cap in ((2, 0), (4, 6), (8, 4), (3, 8)):
            det.set_pipeline(chunks, cap)
            _, n2, out = det.step(tp, ts, te, 400_000)
            assert int(n2.item()) == n
            np.testing.assert_array_equal(out[:n].cpu().numpy(), ref)
            d = det.detect(tp, ts, _t(pairs, dev)).cpu().numpy()
            np.testing.assert_array_equal(d, ref)
        best, ms = det.autotune(tp, ts, te, 400_000, reps=1)
        assert best[0] in (0, 1, 2, 4, 8) and ms > 0  # 0: the fused launch (BF16)
        _, _, out = det.step(tp, ts, te, 400_000)
        np.testing.assert_array_equal(out[:n].cpu().numpy(), ref)
        det.status()


def test_step_replays_as_cuda_graph(scene64):
    lib, poses, osh, env, pairs, layers = scene64
    dev = _dev()
    with _detector(lib, layers, "bf16") as det:
        det.reserve(400_000, len(env) - 1)
        det.set_pipeline(4, 6)
        tp, ts, te = _t(poses, dev), _t(osh, dev), _t(env, dev)
        pr = torch.empty((400_000, 2), dtype=torch.int32, device=dev)
        n = torch.zeros(1, dtype=torch.int32, device=dev)
        out = torch.empty((400_000, 8), dtype=torch.float32, device=dev)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            det.step(tp, ts, te, 400_000, pr, n, out)  # warm-up outside capture
            ref = out[:len(pairs)].clone()
            g = torch.cuda.CUDAGraph()
            out.zero_()
            with torch.cuda.graph(g, stream=s):
                det.step(tp, ts, te, 400_000, pr, n, out)
        torch.cuda.synchronize()
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(n.item()) == len(pairs)
        assert torch.equal(out[:len(pairs)], ref)
        # new poses in the same buffers: the replay follows them
        p2 = synth.random_poses(len(poses), np.random.default_rng(11), -1, 1)
        tp.copy_(_t(p2, dev))
        g.replay()
        torch.cuda.synchronize()
        ref2 = oracle.broadphase(lib.aabb, p2, osh, env)
        assert int(n.item()) == len(ref2)
        np.testing.assert_array_equal(pr[:len(ref2)].cpu().numpy(), ref2)
        det.status()
