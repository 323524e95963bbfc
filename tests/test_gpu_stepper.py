"""Pipelined host-buffer stepping (locc_stepper_*) against locc_step on the
device: for several scenes of different sizes submitted back to back with
up to three steps in flight, every step's pair list, count and outputs equal
the device step's bit for bit, whatever the order of the waits.  Also: more
steps than slots is refused with BUSY, pageable arrays and unknown or
already waited tickets with INVALID_ARG, and the handle keeps working."""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 0.25
MAX_PAIRS = 60_000


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return dev


def _pin(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.fixture(scope="module")
def scenes():
    lib = synth.make_library(16, 3)
    out = [synth.uneven_scene(n, 16, seed) for n, seed in ((2048, 1), (700, 2), (2500, 3), (1, 4))]
    return lib, out


def _check(got, want):
    pairs, out, n = got
    wp, wo, wn = want
    assert n == wn
    np.testing.assert_array_equal(pairs, wp)
    np.testing.assert_array_equal(out, wo)


def _reference(det, scs, dev):
    ref = []
    for p, s, e in scs:
        pr, n, o = det.step(torch.from_numpy(p).to(dev), torch.from_numpy(s).to(dev),
                            torch.from_numpy(e).to(dev), MAX_PAIRS)
        n = int(n.item())
        assert n <= MAX_PAIRS
        ref.append((pr[:n].cpu().numpy(), o[:n].cpu().numpy(), n))
    det.status()
    return ref


@pytest.mark.parametrize("depth,order", [(1, "fifo"), (2, "fifo"), (3, "fifo"), (3, "lifo")])
def test_stepper_matches_device_step(scenes, depth, order):
    from paper_2304_09439_b300 import Detector, Stepper
    dev = _dev()
    lib, scs = scenes
    layers = synth.xavier_weights(2, bias_scale=0.05)
    max_env = max(len(e) - 1 for _, _, e in scs)
    max_obj = max(len(p) for p, _, _ in scs)
    with Detector(lib.points, lib.aabb, layers, R, "bf16") as det:
        ref = _reference(det, scs, dev)
        inputs = [tuple(_pin(a) for a in sc) for sc in scs]
        free = [(_pin(np.zeros((MAX_PAIRS, 2), np.int32)), _pin(np.zeros((MAX_PAIRS, 8), np.float32)))
                for _ in range(depth)]
        with Stepper(det, MAX_PAIRS, max_env, max_obj, depth) as st:
            flight = []  # (ticket, scene, buffers)

            def finish():
                t, k, buf = flight.pop(0 if order == "fifo" else -1)
                _check(st.wait(t), ref[k])
                free.append(buf)

            for k in list(range(len(scs))) * 2:  # every slot used more than once
                if len(flight) == depth:
                    finish()
                buf = free.pop()
                flight.append((st.submit(*inputs[k], *buf), k, buf))
            while flight:
                finish()
        det.status()


def test_stepper_refusals(scenes):
    from paper_2304_09439_b300 import Detector, LoccError, Stepper, abi
    dev = _dev()
    lib, scs = scenes
    p, s, e = scs[0]
    layers = synth.xavier_weights(2, bias_scale=0.05)
    with Detector(lib.points, lib.aabb, layers, R, "fp32") as det:
        ref = _reference(det, [scs[0]], dev)[0]
        with Stepper(det, MAX_PAIRS, len(e) - 1, len(p), 2) as st:
            inp = tuple(_pin(a) for a in (p, s, e))
            bufs = [(_pin(np.zeros((MAX_PAIRS, 2), np.int32)),
                     _pin(np.zeros((MAX_PAIRS, 8), np.float32))) for _ in range(3)]
            with pytest.raises(LoccError):  # pageable inputs
                st.submit(np.ascontiguousarray(p), inp[1], inp[2], *bufs[0])
            t0 = st.submit(*inp, *bufs[0])
            t1 = st.submit(*inp, *bufs[1])
            with pytest.raises(LoccError) as busy:  # both slots in flight
                st.submit(*inp, *bufs[2])
            assert busy.value.code == -7
            _check(st.wait(t1), ref)
            _check(st.wait(t0), ref)
            with pytest.raises(LoccError):  # already waited for
                abi.check(st._lib.locc_stepper_wait(st._t, t0))
            _check(st.wait(st.submit(*inp, *bufs[2])), ref)
        det.status()
        # the handle still steps on its own afterwards
        assert _reference(det, [scs[0]], dev)[0][2] == ref[2]


def test_stepper_empty_scenes(scenes):
    # no environment at all, and environments of one object each (no pair):
    # count 0 and nothing else changes; a normal scene afterwards still matches
    from paper_2304_09439_b300 import Detector, Stepper
    dev = _dev()
    lib, scs = scenes
    layers = synth.xavier_weights(2, bias_scale=0.05)
    p, s, e = scs[1]
    single = (p[:5].copy(), s[:5].copy(), np.arange(6, dtype=np.int32))
    with Detector(lib.points, lib.aabb, layers, R, "bf16") as det:
        ref = _reference(det, [scs[1]], dev)[0]
        with Stepper(det, MAX_PAIRS, len(e) - 1, len(p), 2) as st:
            buf = (_pin(np.zeros((MAX_PAIRS, 2), np.int32)), _pin(np.zeros((MAX_PAIRS, 8), np.float32)))
            none = (_pin(np.zeros((0, 7), np.float32)), _pin(np.zeros(0, np.int32)),
                    _pin(np.zeros(1, np.int32)))
            for inp in (none, tuple(_pin(a) for a in single)):
                pairs, out, n = st.wait(st.submit(*inp, *buf))
                assert n == 0 and len(pairs) == 0 and len(out) == 0
            _check(st.wait(st.submit(*(_pin(a) for a in (p, s, e)), *buf)), ref)
        det.status()
