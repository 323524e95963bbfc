"""GPU: UCF-GJK on convex decompositions against the exact hull test.

With enough iterations GJK decides whether two convex hulls intersect: on
random pairs of decomposed library shapes every pair whose answer is robust
(unchanged when the hulls shrink or grow by 0.2 %) must match the LP oracle
(``oracle/convex.py``).  Fewer iterations only add false positives (an
undecided element pair counts as colliding), never false negatives.  Bad
indices give 0xff and BAD_INDEX.
"""

import numpy as np
import pytest

import synth
from oracle import convex as CX

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_gjk_matches_exact_hull_test():
    from paper_2304_09439_b300 import GJK
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = synth.make_library(6, 3)
    eo, vo, vv = synth.convex_elements(lib, 16)
    rng = np.random.default_rng(3)
    P = 300
    poses = np.zeros((2 * P, 7), np.float32)
    poses[:, :4] = synth.random_quaternions(2 * P, rng)
    poses[1::2, 4:] = rng.uniform(-0.7, 0.7, (P, 3))
    osh = rng.integers(0, 6, 2 * P).astype(np.int32)
    pairs = np.stack([np.arange(0, 2 * P, 2), np.arange(1, 2 * P, 2)], 1).astype(np.int32)
    tp, ts, tq = (torch.from_numpy(a).to(dev) for a in (poses, osh, pairs))
    with GJK(eo, vo, vv) as g:
        full = g.detect(tp, ts, tq, 64).cpu().numpy()
        few = g.detect(tp, ts, tq, 3).cpu().numpy()
        g.status()
    n_rob = 0
    for p in range(P):
        want, robust = CX.decomposition_collide(eo, vo, vv, poses, osh, pairs[p])
        if not robust:
            continue
        n_rob += 1
        assert full[p] == int(want), (p, full[p], want)
        if want:
            assert few[p] == 1  # a capped run never misses a collision
    assert n_rob > 250
    assert 0.2 < full.mean() < 0.9


def test_gjk_bad_index():
    from paper_2304_09439_b300 import GJK, LoccError
    dev = torch.device("cuda:0")
    lib = synth.make_library(2, 3)
    eo, vo, vv = synth.convex_elements(lib, 8)
    poses = torch.tensor([[1, 0, 0, 0, 0, 0, 0]] * 2, dtype=torch.float32, device=dev)
    osh = torch.tensor([0, 5], dtype=torch.int32, device=dev)
    pairs = torch.tensor([[0, 1], [0, 0]], dtype=torch.int32, device=dev)
    with GJK(eo, vo, vv) as g:
        out = g.detect(poses, osh, pairs, 8).cpu().numpy()
        with pytest.raises(LoccError):
            g.status()
    assert out[0] == 0xff and out[1] == 1
