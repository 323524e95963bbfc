"""GPU: training checkpoints resume exactly (optimizer state included).

Adam's moments and step count are read out with ``Trainer.state`` and put
back with ``Trainer.set_state``.  Three runs from the same start on the same
batches: 8 + 8 steps straight; 8 steps, a checkpoint, then a new trainer that
restores parameters and Adam state and runs the last 8; and the same restart
with the parameters alone.  The restored run must reproduce the straight run
(up to the float32 reduction order of the weight gradients), while the
parameters-only restart must not -- so the test would notice a lost moment or
a wrong bias-correction exponent.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batches(lib, n_batches, B, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_batches):
        poses = synth.random_poses(2 * B, rng, -0.4, 0.4)
        osh = rng.integers(0, lib.n_shapes, 2 * B).astype(np.int32)
        pairs = np.stack([np.arange(0, 2 * B, 2), np.arange(1, 2 * B, 2)], 1).astype(np.int32)
        tgt = np.zeros((B, 8), np.float32)
        tgt[:, 0] = rng.integers(0, 2, B)
        tgt[:, 1:4] = poses[0::2, 4:] + rng.normal(0, 0.1, (B, 3))
        nv = rng.normal(size=(B, 3))
        tgt[:, 4:7] = nv / np.linalg.norm(nv, axis=1, keepdims=True)
        tgt[:, 7] = rng.normal(0, 0.02, B)
        out.append((poses, osh, pairs, tgt))
    return out


def test_resume_from_checkpoint_matches_uninterrupted_training():
    from paper_2304_09439_b300 import Detector, Trainer
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = synth.make_library(8, 3)
    B = 64
    batches = [tuple(torch.from_numpy(a).to(dev) for a in b) for b in _batches(lib, 16, B, 4)]

    def run(tr, bs):
        for poses, osh, pairs, tgt in bs:
            tr.step(poses, osh, pairs, tgt, None, True)
        torch.cuda.synchronize()

    with Detector(lib.points, lib.aabb, synth.xavier_weights(2), 0.25, "fp32") as det:
        tr = Trainer(det, B, lr=3e-3)
        p0 = tr.params().clone()
        run(tr, batches[:8])
        ck_p = tr.params().clone()
        ck_m, ck_v, ck_step = tr.state()
        ck_m, ck_v = ck_m.clone(), ck_v.clone()
        assert ck_step == 8
        run(tr, batches[8:])
        straight = tr.params().cpu().numpy()
        tr.close()

        tr = Trainer(det, B, lr=3e-3)
        tr.set_params(ck_p)
        tr.set_state(ck_m, ck_v, ck_step)
        m, v, step = tr.state()
        assert step == 8 and torch.equal(m, ck_m) and torch.equal(v, ck_v)
        run(tr, batches[8:])
        resumed = tr.params().cpu().numpy()
        tr.close()

        tr = Trainer(det, B, lr=3e-3)
        tr.set_params(ck_p)
        run(tr, batches[8:])
        params_only = tr.params().cpu().numpy()
        tr.close()

    moved = np.abs(straight - ck_p.cpu().numpy()).max()
    assert moved > 1e-4  # the last 8 steps changed the parameters
    assert np.abs(resumed - straight).max() <= 1e-3 * moved
    assert np.abs(params_only - straight).max() > 0.05 * moved
    assert not np.array_equal(p0.cpu().numpy(), straight)
