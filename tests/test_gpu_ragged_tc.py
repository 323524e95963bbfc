"""GPU: the tensor-core paths on ragged batch sizes.

The heads work on tiles of 128 pairs and the encoders on one pair per slot;
every row must not depend on which tile, slot or batch it falls in.  For
sizes around the tile edges (1, 127, 128, 129, 255, 257, 1000, 4097) the
output rows of a detect call on the first n pairs equal, bit for bit, the
same rows of one call on all pairs, in BF16 and FP8; the pooled features of
the network entry point do too.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 0.25
SIZES = (1, 127, 128, 129, 255, 257, 1000, 4097)


@pytest.fixture(scope="module")
def scene():
    lib = synth.make_library(16, 3)
    poses, osh, env = synth.uneven_scene(1024, 16, 21)
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    assert len(pairs) >= max(SIZES)
    return lib, poses, osh, pairs


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_rows_do_not_depend_on_batch(scene, prec):
    from paper_2304_09439_b300 import Detector
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib, poses, osh, pairs = scene
    tp, ts = torch.from_numpy(poses).to(dev), torch.from_numpy(osh).to(dev)
    N = max(SIZES)
    tq = torch.from_numpy(pairs[:N]).to(dev)
    with Detector(lib.points, lib.aabb, synth.xavier_weights(1, bias_scale=0.05), R, prec) as det:
        full = det.detect(tp, ts, tq).cpu().numpy()
        crops = det.crop(tp, ts, tq)
        y_full, f_full = det.network(crops["xyz"], with_feat=True)
        y_full, f_full = y_full.cpu().numpy(), f_full.cpu().numpy()
        for n in SIZES:
            part = det.detect(tp, ts, tq[:n].contiguous()).cpu().numpy()
            assert np.array_equal(part.view(np.uint32), full[:n].view(np.uint32)), f"{prec} n={n}"
            y, f = det.network(crops["xyz"][:n].contiguous(), with_feat=True)
            assert np.array_equal(y.cpu().numpy().view(np.uint32), y_full[:n].view(np.uint32))
            assert np.array_equal(f.cpu().numpy().view(np.uint32), f_full[:n].view(np.uint32))
        det.status()
    assert np.isfinite(full).all()
