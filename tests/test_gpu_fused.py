"""The fused crop + BF16 encoder launch (locc_set_pipeline(h, 0, crop_warps))
against the separate crop and encoder kernels: outputs bit-identical on the
bench scene (8192 environments, 64 shapes; also as a CUDA-graph replay), on
ragged pair counts with invalid object indices, and on libraries with
duplicated samples and large crop balls, where many objects are deferred to
the exact fallback crop and its list-driven encoder pass.  Each object's
arithmetic is the same in both paths (the same MMA shapes over its 64 rows,
the same pooling), so equality is exact."""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 0.25


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return dev


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _detect_all_modes(det, tp, ts, tq):
    outs = {}
    for mode in ((1, 0), (0, 8), (0, 6)):
        det.set_pipeline(*mode)
        outs[mode] = det.detect(tp, ts, tq).cpu().numpy()
        det.status()
    return outs


def test_fused_step_bit_identical_on_bench_scene():
    from paper_2304_09439_b300 import Detector
    dev = _dev()
    lib = synth.make_library(64, 4)
    poses, osh, env = synth.uneven_scene(8192, 64, 5)
    layers = synth.xavier_weights(1, bias_scale=0.05)
    with Detector(lib.points, lib.aabb, layers, R, "bf16") as det:
        det.reserve(400_000, len(env) - 1)
        tp, ts, te = _t(poses, dev), _t(osh, dev), _t(env, dev)
        det.set_pipeline(1, 0)
        pairs, n_dev, ref = det.step(tp, ts, te, 400_000)
        n = int(n_dev.item())
        assert n > 100_000
        ref = ref[:n].cpu().numpy()
        tq = pairs[:n].clone()
        for w in (8, 6):
            det.set_pipeline(0, w)
            _, n2, out = det.step(tp, ts, te, 400_000)
            assert int(n2.item()) == n
            np.testing.assert_array_equal(out[:n].cpu().numpy(), ref)
            np.testing.assert_array_equal(det.detect(tp, ts, tq).cpu().numpy(), ref)
            det.status()
        # the fused step replays as a CUDA graph
        det.set_pipeline(0, 8)
        out = torch.empty((400_000, 8), dtype=torch.float32, device=dev)
        pb = torch.empty((400_000, 2), dtype=torch.int32, device=dev)
        nb = torch.zeros(1, dtype=torch.int32, device=dev)
        stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(stream):
            det.step(tp, ts, te, 400_000, pairs_out=pb, n_pairs_out=nb, out=out)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                det.step(tp, ts, te, 400_000, pairs_out=pb, n_pairs_out=nb, out=out)
            out.fill_(0.0)
            g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out[:n].cpu().numpy(), ref)
        det.status()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 128, 129, 1000])
def test_fused_ragged_counts_and_invalid_indices(n):
    from paper_2304_09439_b300 import Detector, LoccError
    dev = _dev()
    lib = synth.tiny_library()
    poses, osh, pairs = synth.compose_relative_tiny(max(n, 4), 3)
    pairs = pairs[:n].copy()
    if n >= 3:
        pairs[1, 1] = poses.shape[0] + 3  # out of range: NaN row, BAD_INDEX
    layers = synth.xavier_weights(2, bias_scale=0.05)
    with Detector(lib.points, lib.aabb, layers, R, "bf16") as det:
        outs = {}
        for mode in ((1, 0), (0, 8), (0, 6)):
            det.set_pipeline(*mode)
            outs[mode] = det.detect(_t(poses, dev), _t(osh, dev), _t(pairs, dev)).cpu().numpy()
            if n >= 3:
                with pytest.raises(LoccError):
                    det.status()
            else:
                det.status()
        for mode in ((0, 8), (0, 6)):
            np.testing.assert_array_equal(outs[mode], outs[(1, 0)])
        if n >= 3:
            assert np.all(np.isnan(outs[(0, 8)][1]))
            assert np.all(np.isfinite(np.delete(outs[(0, 8)], 1, axis=0)))


@pytest.mark.parametrize("copies,radius", [(128, 0.6), (48, 1.0), (1, 1.5)])
def test_fused_with_deferred_objects(copies, radius):
    # many equal distances (duplicated samples) and large balls: the bin
    # holding the 64th key overflows the rank buffer, objects are deferred
    from paper_2304_09439_b300 import Detector
    dev = _dev()
    lib = synth.tiny_library()
    poses, osh, pairs = synth.compose_relative_tiny(512, 4)
    pts = lib.points.copy()
    if copies > 1:
        for s_ in range(pts.shape[0]):
            pts[s_] = pts[s_][(np.arange(pts.shape[1]) // copies) * copies]
    layers = synth.xavier_weights(3, bias_scale=0.05)
    with Detector(pts, lib.aabb, layers, radius, "bf16") as det:
        outs = _detect_all_modes(det, _t(poses, dev), _t(osh, dev), _t(pairs, dev))
        crop = det.crop(_t(poses, dev), _t(osh, dev), _t(pairs, dev), with_idx=False)
        assert int((crop["cnt"] == 64).sum().item()) > 100
    for mode in ((0, 8), (0, 6)):
        np.testing.assert_array_equal(outs[mode], outs[(1, 0)])
