"""The allocation-free entry point against the ordinary one.

locc_detect_noalloc serves callers that may not allocate device memory at call
time (a simulator whose pool allocator owns HBM, a latency-critical loop): its
scratch is a library-owned static device array.  This test calls it through the
C ABI twice in a row and checks both results against locc_detect on the same
inputs with the float32 parity tolerance, plus the size limit.  It sits in a
file of its own, named to run last, and needs nothing from other tests."""

import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


def _close(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), np.sqrt((ref ** 2).mean(axis=0, keepdims=True)) + 1e-30)
    assert np.all(np.abs(got - ref) <= TOL * scale)


def test_noalloc_matches_detect_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_09439_b300 import Detector, abi
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    lib = synth.tiny_library()
    layers = synth.xavier_weights(1, bias_scale=0.05)
    so = abi.load()
    with Detector(lib.points, lib.aabb, layers, 0.25, "fp32") as det:
        stream = torch.cuda.current_stream()
        for seed, n in ((0, 1000), (1, 1024)):
            poses, osh, pairs = synth.compose_relative_tiny(n, seed)
            tp = torch.from_numpy(poses).to(dev)
            ts = torch.from_numpy(osh).to(dev)
            tq = torch.from_numpy(pairs).to(dev)
            ref = det.detect(tp, ts, tq).cpu().numpy()
            outs = []
            for _ in range(2):
                out = torch.full((n, 8), float("nan"), dtype=torch.float32, device=dev)
                rc = so.locc_detect_noalloc(det._h, tp.data_ptr(), ts.data_ptr(), tp.shape[0],
                                            tq.data_ptr(), n, out.data_ptr(),
                                            ctypes.c_void_p(stream.cuda_stream))
                assert rc == 0, so.locc_last_error()
                det.status()
                outs.append(out.cpu().numpy())
            for o in outs:
                _close(o, ref)
            np.testing.assert_array_equal(outs[0], outs[1])
        # beyond the stated maximum: a clear error, nothing launched
        big = torch.zeros((abi.NOALLOC_MAX_PAIRS + 1, 2), dtype=torch.int32, device=dev)
        out = torch.zeros((big.shape[0], 8), dtype=torch.float32, device=dev)
        rc = so.locc_detect_noalloc(det._h, tp.data_ptr(), ts.data_ptr(), tp.shape[0],
                                    big.data_ptr(), big.shape[0], out.data_ptr(),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert rc == -1
        assert b"LOCC_NOALLOC_MAX_PAIRS" in so.locc_last_error()
