"""The allocation-free entry point against the ordinary one.

locc_detect_noalloc serves callers that may not allocate device memory at call
time (a simulator whose pool allocator owns HBM, a latency-critical loop): its
scratch is a library-owned static device array.  These tests call it through
the C ABI twice in a row and check both results against locc_detect on the
same inputs with the float32 parity tolerance, check the size limit, check
that its first call on a new handle changes the device's free memory by
nothing (locc_create already loaded the array and the kernels), and check
that a BF16 handle still gets the float32 network.  The file sits on its own,
named to run last, and needs nothing from other tests."""

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


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_09439_b300 import abi
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return dev, abi.load(), abi


def _inputs(dev, n, seed):
    poses, osh, pairs = synth.compose_relative_tiny(n, seed)
    return (torch.from_numpy(poses).to(dev), torch.from_numpy(osh).to(dev),
            torch.from_numpy(pairs).to(dev))


def _noalloc(so, det, tp, ts, tq, out, stream):
    return so.locc_detect_noalloc(det._h, tp.data_ptr(), ts.data_ptr(), tp.shape[0],
                                  tq.data_ptr(), tq.shape[0], out.data_ptr(),
                                  ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_first_call_allocates_nothing():
    dev, so, _ = _setup()
    from paper_2304_09439_b300 import Detector
    lib = synth.tiny_library()
    layers = synth.xavier_weights(1, bias_scale=0.05)
    tp, ts, tq = _inputs(dev, 1024, 3)
    out = torch.full((1024, 8), float("nan"), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    with Detector(lib.points, lib.aabb, layers, 0.25, "fp32") as det:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        rc = _noalloc(so, det, tp, ts, tq, out, stream)
        assert rc == 0, so.locc_last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"first call changed free device memory by {free0 - free1} bytes"
        det.status()
        ref = det.detect(tp, ts, tq).cpu().numpy()
        _close(out.cpu().numpy(), ref)


def test_noalloc_matches_detect_twice():
    dev, so, abi = _setup()
    from paper_2304_09439_b300 import Detector
    lib = synth.tiny_library()
    layers = synth.xavier_weights(1, bias_scale=0.05)
    with Detector(lib.points, lib.aabb, layers, 0.25, "fp32") as det:
        stream = torch.cuda.current_stream()
        for seed, n in ((0, 1000), (1, 1024)):
            tp, ts, tq = _inputs(dev, n, seed)
            ref = det.detect(tp, ts, tq).cpu().numpy()
            outs = []
            for _ in range(2):
                out = torch.full((n, 8), float("nan"), dtype=torch.float32, device=dev)
                rc = _noalloc(so, det, tp, ts, tq, out, stream)
                assert rc == 0, so.locc_last_error()
                det.status()
                outs.append(out.cpu().numpy())
            for o in outs:
                _close(o, ref)
            np.testing.assert_array_equal(outs[0], outs[1])
        # beyond the stated maximum: a clear error, nothing launched
        big = torch.zeros((abi.NOALLOC_MAX_PAIRS + 1, 2), dtype=torch.int32, device=dev)
        out = torch.zeros((big.shape[0], 8), dtype=torch.float32, device=dev)
        rc = _noalloc(so, det, tp, ts, big, out, stream)
        assert rc == -1
        msg = so.locc_last_error()
        assert b"LOCC_NOALLOC_MAX_PAIRS" in msg and str(abi.NOALLOC_MAX_PAIRS).encode() in msg


def test_noalloc_on_bf16_handle_runs_float32_network():
    dev, so, _ = _setup()
    from paper_2304_09439_b300 import Detector
    lib = synth.tiny_library()
    layers = synth.xavier_weights(1, bias_scale=0.05)
    tp, ts, tq = _inputs(dev, 777, 4)
    stream = torch.cuda.current_stream()
    with Detector(lib.points, lib.aabb, layers, 0.25, "fp32") as d32:
        ref = d32.detect(tp, ts, tq).cpu().numpy()
    with Detector(lib.points, lib.aabb, layers, 0.25, "bf16") as d16:
        for _ in range(2):
            out = torch.full((777, 8), float("nan"), dtype=torch.float32, device=dev)
            rc = _noalloc(so, d16, tp, ts, tq, out, stream)
            assert rc == 0, so.locc_last_error()
            d16.status()
            _close(out.cpu().numpy(), ref)
