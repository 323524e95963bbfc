"""Training checkpoints round-trip on the host (no GPU): ``train.save_checkpoint``
followed by ``train.load_checkpoint`` restores the parameters, Adam's moments
and step count, the best-so-far parameters, the loss history and the report,
and the batch sampler continues with exactly the draws an uninterrupted run
would have made.  A stand-in trainer with the same four methods as the GPU
``Trainer`` (CPU tensors) takes the place of the real one."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_09439_b300 import train  # noqa: E402


class FakeTrainer:
    def __init__(self, n, seed):
        g = np.random.default_rng(seed)
        self.p = torch.from_numpy(g.normal(size=n).astype(np.float32))
        self.m = torch.from_numpy(g.normal(size=n).astype(np.float32))
        self.v = torch.from_numpy(g.random(n).astype(np.float32))
        self.step = int(g.integers(1, 10_000))

    def params(self):
        return self.p.clone()

    def state(self):
        return self.m.clone(), self.v.clone(), self.step

    def set_params(self, p):
        self.p = p.clone()

    def set_state(self, m, v, step):
        self.m, self.v, self.step = m.clone(), v.clone(), int(step)


def test_checkpoint_round_trip_and_sampler_continuation(tmp_path):
    n = 1000
    src = FakeTrainer(n, 1)
    rng = np.random.default_rng(7)
    rng.integers(0, 100, 37)  # some draws before the checkpoint
    best = (0.91, 400, torch.from_numpy(np.arange(n, dtype=np.float32)))
    hist = [(200, 0.5), (400, 0.25)]
    report = {"val": [{"step": 400, "f1": 0.9}], "evals": [{"step": 0}]}
    path = str(tmp_path / "ck.npz")
    train.save_checkpoint(path, src, 400, rng, best, hist, report)
    expect_next = rng.integers(0, 1 << 30, 16)  # what the run would draw next

    dst = FakeTrainer(n, 2)
    rng2 = np.random.default_rng(99)
    rep2 = {"val": [], "evals": []}
    first, best2, hist2 = train.load_checkpoint(path, dst, rng2, rep2, "cpu")
    assert first == 401
    assert torch.equal(dst.p, src.p) and torch.equal(dst.m, src.m) and torch.equal(dst.v, src.v)
    assert dst.step == src.step
    assert best2[0] == best[0] and best2[1] == best[1] and torch.equal(best2[2], best[2])
    assert hist2 == hist
    assert rep2 == report
    np.testing.assert_array_equal(rng2.integers(0, 1 << 30, 16), expect_next)


def test_checkpoint_without_best_parameters(tmp_path):
    src = FakeTrainer(10, 3)
    rng = np.random.default_rng(0)
    path = str(tmp_path / "ck.npz")
    train.save_checkpoint(path, src, 5, rng, (-1.0, 0, None), [], {"val": [], "evals": []})
    dst = FakeTrainer(10, 4)
    first, best, hist = train.load_checkpoint(path, dst, np.random.default_rng(1),
                                              {"val": [], "evals": []}, "cpu")
    assert first == 6 and best[2] is None and hist == []
