"""CPU: the seeded scene generators produce well-formed inputs."""

import numpy as np

import oracle
import synth


def test_drop_scene_well_formed():
    lib = synth.make_library(16, 3)
    seen = 0
    for step, poses, osh, env in synth.drop_scene(lib, 256, 200, 8):
        assert poses.dtype == np.float32 and poses.shape == (512, 7)
        assert np.all(np.isfinite(poses))
        np.testing.assert_allclose(np.linalg.norm(poses[:, :4], axis=1), 1.0, atol=1e-5)
        if step % 50 == 0:
            pairs = oracle.broadphase(lib.aabb, poses, osh, env)
            assert len(pairs) <= 256  # at most one pair per two-object environment
            assert np.all(pairs[:, 1] == pairs[:, 0] + 1) and np.all(pairs[:, 0] % 2 == 0)
            seen += len(pairs)
    assert poses[:, 6].min() > 0.0  # nothing fell through the plane
    assert seen > 0


def test_client_batch_pairs_stay_in_their_environment():
    p, s, q = synth.client_batch(64, 300, 5000, 11)
    assert p.shape[1] == 7 and len(s) == len(p) and q.shape == (5000, 2)
    assert np.all(q[:, 0] != q[:, 1]) and q.min() >= 0 and q.max() < len(p)
    # rebuild the environment of every object from the Poisson counts
    _, _, off = synth.uneven_scene(300, 64, int(np.random.default_rng(11).integers(1 << 30)),
                                   8.0, n_min=2, n_max=25, extent=1.0)
    env_of = np.repeat(np.arange(300), np.diff(off))
    assert np.all(env_of[q[:, 0]] == env_of[q[:, 1]])
