"""GPU: the failure path of the tensor-core kernels, without a fault.

Every mbarrier wait in the encoder and head kernels is bounded: when it runs
out, the CTA raises the timeout bit of the handle's error flag, drains its
own copies, releases its TMEM and returns.  ``locc_selftest_wait_timeout``
launches one CTA that takes exactly that path (a wait on an mbarrier that
nothing completes, bounded to a few hundred microseconds); ``status`` must
then report TIMEOUT once, and the same handle must go on producing the same
outputs as before.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_survives():
    from paper_2304_09439_b300 import Detector, LoccError
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = synth.make_library(8, 3)
    poses, osh, env = synth.uneven_scene(64, 8, seed=9)
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)[:500]
    tp, ts, tq = (torch.from_numpy(a).to(dev) for a in (poses, osh, pairs))
    with Detector(lib.points, lib.aabb, synth.xavier_weights(1), 0.25, "bf16") as det:
        before = det.detect(tp, ts, tq).cpu().numpy()
        det.status()
        det.selftest_wait_timeout(1_000_000)  # about 0.5 ms at 2 GHz
        with pytest.raises(LoccError) as e:
            det.status()
        assert e.value.code == -4
        det.status()  # reported once, then cleared
        after = det.detect(tp, ts, tq).cpu().numpy()
        det.status()
        np.testing.assert_array_equal(after, before)
        with pytest.raises(LoccError):
            det.selftest_wait_timeout(0)
