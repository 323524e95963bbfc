"""Pins of oracle (b): crop selection and the crop network forward / backward.

Expected values come from independent routes: scipy's rotation routines,
float64 geometry worked out by hand, invariants of the selection rule,
hand-built networks whose output has a closed form, and central finite
differences of the oracle's own loss for its backward pass."""

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import synth

KMAX = oracle.KMAX


def _one_pair_lib(ptsA, ptsB, aabbA, aabbB):
    n = max(len(ptsA), len(ptsB))
    P = np.zeros((2, n, 3), np.float32)
    P[0, :len(ptsA)] = ptsA
    P[1, :len(ptsB)] = ptsB
    if len(ptsA) < n:
        P[0, len(ptsA):] = 1e6  # far away, never selected
    if len(ptsB) < n:
        P[1, len(ptsB):] = 1e6
    return P, np.array([aabbA, aabbB], np.float32)


def _R64(pose):
    w, x, y, z = (float(v) for v in pose[:4])
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def test_rotation_matches_scipy():
    # the crop frame of A is R(q_A); with B at the identity and A's box
    # covering everything, B's canonical coords are R_A^T (p - t_A) - c
    rng = np.random.default_rng(0)
    q = synth.random_quaternions(50, rng)
    for i in range(50):
        poseA = np.array([*q[i], 0, 0, 0], np.float32)
        poseB = np.array([1, 0, 0, 0, 0, 0, 0], np.float32)
        ptsB = rng.uniform(-0.1, 0.1, size=(8, 3)).astype(np.float32)
        P, aabb = _one_pair_lib(np.zeros((1, 3)), ptsB, [-5, -5, -5, 5, 5, 5],
                                [-0.1, -0.1, -0.1, 0.1, 0.1, 0.1])
        r = oracle.crop_forward(P, aabb, np.stack([poseA, poseB]),
                                np.array([0, 1], np.int32),
                                np.array([[0, 1]], np.int32), 10.0)
        RA = _R64(poseA)
        c = r["centre"][0].astype(np.float64)
        # B's box in A's frame: centre R_A^T 0 = 0, half |R_A^T| 0.1
        half = np.abs(RA.T) @ np.full(3, 0.1)
        np.testing.assert_allclose(c, 0.0, atol=1e-6)
        assert np.all(half >= 0.1 - 1e-9)
        got = r["xyz"][0, 1, :8].astype(np.float64)
        idx = r["idx"][0, 1, :8]
        expect = (RA.T @ ptsB[idx].astype(np.float64).T).T - c
        np.testing.assert_allclose(got, expect, atol=2e-6)


@pytest.mark.parametrize("angle,expect_x", [(0.0, 0.85),
                                            (np.pi / 4, (1.2 - 0.5 * np.sqrt(2) + 1.0) / 2)])
def test_crop_centre_closed_form(angle, expect_x):
    # A: box [-1,1]^3 at the origin; B: box [-.5,.5]^3 at (1.2, 0, 0) turned by
    # `angle` about z.  B's A-frame box spans x in [1.2 - h, 1.2 + h] with
    # h = 0.5 (|cos| + |sin|); the intersection with [-1, 1] is [1.2 - h, 1].
    P, aabb = _one_pair_lib(np.zeros((1, 3)), np.zeros((1, 3)),
                            [-1, -1, -1, 1, 1, 1], [-.5, -.5, -.5, .5, .5, .5])
    q = Rotation.from_euler("z", angle).as_quat()
    poses = np.array([[1, 0, 0, 0, 0, 0, 0],
                      [q[3], q[0], q[1], q[2], 1.2, 0, 0]], np.float32)
    r = oracle.crop_forward(P, aabb, poses, np.array([0, 1], np.int32),
                            np.array([[0, 1]], np.int32), 0.25)
    np.testing.assert_allclose(r["centre"][0], [expect_x, 0, 0], atol=1e-6)


def test_crop_centre_of_separated_boxes_is_gap_midpoint():
    # no overlap on x: the centre sits half-way between the facing faces
    P, aabb = _one_pair_lib(np.zeros((1, 3)), np.zeros((1, 3)),
                            [-1, -1, -1, 1, 1, 1], [-.5, -.5, -.5, .5, .5, .5])
    poses = np.array([[1, 0, 0, 0, 0, 0, 0], [1, 0, 0, 0, 2.5, 0.25, 0]], np.float32)
    r = oracle.crop_forward(P, aabb, poses, np.array([0, 1], np.int32),
                            np.array([[0, 1]], np.int32), 0.25)
    # x: faces at 1.0 and 2.0 -> 1.5; y: [-1,1] and [-.25,.75] -> [-.25,.75] -> .25
    np.testing.assert_allclose(r["centre"][0], [1.5, 0.25, 0.0], atol=1e-6)


def test_crop_selection_invariants(tiny_lib, tiny_case):
    poses, osh, pairs = tiny_case
    r = oracle.crop_forward(tiny_lib.points, tiny_lib.aabb, poses, osh, pairs, 0.25)
    rr = 0.25
    n_full = 0
    for p in range(pairs.shape[0]):
        a, b = pairs[p]
        RA, RB = _R64(poses[a]), _R64(poses[b])
        tA, tB = poses[a, 4:].astype(np.float64), poses[b, 4:].astype(np.float64)
        c = r["centre"][p].astype(np.float64)
        for side, (o, R, t) in enumerate([(a, RA, tA), (b, RB, tB)]):
            pts = tiny_lib.points[osh[o]].astype(np.float64)
            # canonical: A's axes, origin at the crop centre
            can = (RA.T @ (R @ pts.T + t[:, None] - tA[:, None])).T - c
            d = np.linalg.norm(can, axis=1)
            cnt = r["cnt"][p, side]
            idx = r["idx"][p, side]
            assert np.all(idx[cnt:] == -1) and np.all(idx[:cnt] >= 0)
            assert np.all(r["xyz"][p, side, cnt:] == 0)
            sel = idx[:cnt]
            assert len(np.unique(sel)) == cnt
            np.testing.assert_allclose(r["xyz"][p, side, :cnt], can[sel], atol=3e-6)
            assert np.all(d[sel] <= rr + 1e-5)
            # nearest first
            assert np.all(np.diff(d[sel]) >= -1e-5)
            n_in = np.sum(d <= rr - 1e-5)
            n_in_loose = np.sum(d <= rr + 1e-5)
            assert min(KMAX, n_in) <= cnt <= min(KMAX, n_in_loose)
            if cnt == KMAX:
                n_full += 1
                rest = np.setdiff1d(np.nonzero(d <= rr + 1e-5)[0], sel)
                if len(rest):
                    assert d[rest].min() >= d[sel].max() - 1e-5
    assert n_full > 10


def _passthrough_params(bias3=0.0):
    """Encoder that copies relu(+-x, +-y, +-z) into channels 0..5; head whose
    logit is sum_k fA[k] - sum_k fB[k] and whose other outputs are fA[0..6]."""
    W = [np.zeros((o, i)) for i, o in oracle.LAYER_DIMS]
    b = [np.zeros(o) for _, o in oracle.LAYER_DIMS]
    for k in range(3):
        W[0][2 * k, k] = 1.0
        W[0][2 * k + 1, k] = -1.0
    for k in range(6):
        W[1][k, k] = 1.0
        W[2][k, k] = 1.0
    b[2][6] = bias3  # a channel that is relu(bias3) for every point
    for k in range(7):
        W[3][k, k] = 1.0          # g1[k] = fA[k]
        W[3][7 + k, 256 + k] = 1.0  # g1[7+k] = fB[k]
    for k in range(14):
        W[4][k, k] = 1.0
    W[5][0, :7] = 1.0
    W[5][0, 7:14] = -1.0
    for k in range(1, 8):
        W[5][k, k - 1] = 1.0
    return oracle.flatten_params(list(zip(W, b)))


def test_network_closed_form_passthrough():
    rng = np.random.default_rng(1)
    P = 5
    xyz = np.zeros((P, 2, KMAX, 3), np.float32)
    cnt = np.array([[3, 7], [0, 5], [64, 0], [1, 1], [10, 64]], np.int32)
    for p in range(P):
        for s in range(2):
            xyz[p, s, :cnt[p, s]] = rng.uniform(-0.25, 0.25, (cnt[p, s], 3))
            # garbage in padded slots must not matter
            xyz[p, s, cnt[p, s]:] = rng.uniform(-9, 9, (KMAX - cnt[p, s], 3))
    y, f = oracle.network(_passthrough_params(bias3=0.7), xyz, cnt)
    for p in range(P):
        feats = []
        for s in range(2):
            v = xyz[p, s, :cnt[p, s]].astype(np.float64)
            if len(v):
                e = [max(0, v[:, k].max()) if j == 0 else max(0, (-v[:, k]).max())
                     for k in range(3) for j in range(2)]
                e.append(0.7)
            else:
                e = [0.0] * 7
            feats.append(np.array(e))
        np.testing.assert_allclose(f[p, :7], feats[0], atol=1e-7)
        np.testing.assert_allclose(f[p, 256:263], feats[1], atol=1e-7)
        assert np.all(f[p, 7:256] == 0) and np.all(f[p, 263:] == 0)
        np.testing.assert_allclose(y[p, 0], feats[0].sum() - feats[1].sum(), atol=1e-7)
        np.testing.assert_allclose(y[p, 1:8], feats[0][:7], atol=1e-7)


def test_network_point_permutation_invariance():
    rng = np.random.default_rng(2)
    W = synth.xavier_weights(3, bias_scale=0.1)
    params = oracle.flatten_params(W)
    xyz = rng.uniform(-0.25, 0.25, (4, 2, KMAX, 3)).astype(np.float32)
    cnt = np.array([[64, 64], [13, 40], [0, 9], [64, 1]], np.int32)
    y0, f0 = oracle.network(params, xyz, cnt)
    xyz2 = xyz.copy()
    for p in range(4):
        for s in range(2):
            perm = rng.permutation(cnt[p, s])
            xyz2[p, s, :cnt[p, s]] = xyz[p, s, perm]
    y1, f1 = oracle.network(params, xyz2, cnt)
    np.testing.assert_allclose(y0, y1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(f0, f1, rtol=1e-12, atol=1e-12)


def test_epilogue_maps_canonical_outputs_to_world(tiny_lib):
    # a head whose raw outputs are its biases: point (0.1,-0.2,0.05) and
    # normal (3,4,0) in the crop frame
    W = [np.zeros((o, i)) for i, o in oracle.LAYER_DIMS]
    b = [np.zeros(o) for _, o in oracle.LAYER_DIMS]
    b[5][:] = [0.5, 0.1, -0.2, 0.05, 3.0, 4.0, 0.0, -0.02]
    params = oracle.flatten_params(list(zip(W, b)))
    rng = np.random.default_rng(4)
    poses = synth.random_poses(6, rng, -0.5, 0.5)
    osh = np.array([0, 1, 1, 0, 0, 0], np.int32)
    pairs = np.array([[0, 1], [2, 3], [4, 5]], np.int32)
    r = oracle.crop_forward(tiny_lib.points, tiny_lib.aabb, poses, osh, pairs,
                            0.25, params)
    for p, (a, _) in enumerate(pairs):
        RA = _R64(poses[a])
        c = r["centre"][p].astype(np.float64)
        pw = RA @ (np.array([0.1, -0.2, 0.05]) + c) + poses[a, 4:]
        nw = RA @ np.array([0.6, 0.8, 0.0])
        np.testing.assert_allclose(r["out"][p, 0], 0.5)
        np.testing.assert_allclose(r["out"][p, 1:4], pw, atol=2e-6)
        np.testing.assert_allclose(r["out"][p, 4:7], nw, atol=2e-6)
        np.testing.assert_allclose(r["out"][p, 7], -0.02)


@pytest.mark.parametrize("w_len", [0.0, 0.3])
def test_backward_matches_finite_differences(w_len):
    rng = np.random.default_rng(5)
    W = synth.xavier_weights(7, bias_scale=0.2)
    params = oracle.flatten_params(W)
    P = 3
    xyz = rng.uniform(-0.25, 0.25, (P, 2, KMAX, 3)).astype(np.float32)
    cnt = np.array([[20, 5], [64, 0], [3, 64]], np.int32)
    tgt = np.zeros((P, 8))
    tgt[:, 0] = [1, 0, 1]
    tgt[:, 1:4] = rng.normal(0, 0.1, (P, 3))
    n = rng.normal(size=(P, 3))
    tgt[:, 4:7] = n / np.linalg.norm(n, axis=1, keepdims=True)
    tgt[:, 7] = rng.normal(0, 0.05, P)
    hp = (1.0, 1.0, 1.0, 0.5, 0.5, w_len)  # wide huber so the depth term is smooth
    L, g = oracle.loss_grad(params, xyz, cnt, tgt, hp)
    # probe parameters with a large gradient in every layer
    offs = np.cumsum([0] + [i * o + o for i, o in oracle.LAYER_DIMS])
    h = 1e-6
    checked = 0
    for l in range(6):
        seg = np.arange(offs[l], offs[l + 1])
        pick = seg[np.argsort(-np.abs(g[seg]))[:6]]
        for k in pick:
            if g[k] == 0:
                continue
            pp = params.copy(); pp[k] += h
            pm = params.copy(); pm[k] -= h
            fd = (oracle.loss_grad(pp, xyz, cnt, tgt, hp)[0]
                  - oracle.loss_grad(pm, xyz, cnt, tgt, hp)[0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(g[k])) + 1e-7, (l, k, fd, g[k])
            checked += 1
    assert checked >= 30
