"""Pins of the oracle-(b) functions that the GPU path is compared against but
whose own correctness the other oracle tests do not fix:

* the broad phase (Sec. II, footnote 1: far-apart objects are ruled out
  before the narrow phase) against a float64 brute force over the posed boxes,
  built from scipy's rotations, with touching, rotated and elongated boxes and
  environments of 0, 1, 2 and 25 objects;
* the global crop of the ablation without locality (Sec. IV-B, GLOBAL-OCN):
  the first 64 samples of each object, zero padding below 64, and B's
  coordinates R_rel (p - c_B) recomputed in float64;
* the training loss value (Sec. III-A: binary cross-entropy on the collision
  logit plus alpha |f|^2 on the shape embedding, alpha = 0.5; this library's
  regression terms) against numbers worked out by hand on networks whose
  outputs are their biases;
* the selection's tie rule (equal squared distances go to the lower sample
  index) on samples placed at exactly equal float32 distances;
* the bf16 operand mode of the loss and gradient (the arithmetic of a bf16
  tensor-core trainer): its rounding against PyTorch's CPU bfloat16
  conversion, and the loss and gradient against PyTorch CPU autograd through
  the same network whose matrix products round their operands (forward and
  backward, straight through) at the places the oracle's header lists.

None of the expected values comes from the oracle itself or from the CUDA
path."""

import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle

KMAX = oracle.KMAX


# ------------------------------------------------------------------ broad phase

def _world_boxes64(aabb, poses, obj_shape):
    """float64 world axis-aligned box (centre, half extents) of each posed body
    box, with the rotation taken from scipy (not from the oracle)."""
    c = np.empty((len(obj_shape), 3))
    h = np.empty((len(obj_shape), 3))
    for i, s in enumerate(obj_shape):
        lo = aabb[s, :3].astype(np.float64)
        hi = aabb[s, 3:].astype(np.float64)
        w, x, y, z = (float(v) for v in poses[i, :4])
        R = Rotation.from_quat([x, y, z, w]).as_matrix()
        c[i] = R @ ((lo + hi) / 2) + poses[i, 4:].astype(np.float64)
        h[i] = np.abs(R) @ ((hi - lo) / 2)
    return c, h


def _brute_pairs64(aabb, poses, obj_shape, env_offsets):
    c, h = _world_boxes64(aabb, poses, obj_shape)
    out, margin = [], []
    for e in range(len(env_offsets) - 1):
        for i in range(env_offsets[e], env_offsets[e + 1]):
            for j in range(i + 1, env_offsets[e + 1]):
                m = np.min(h[i] + h[j] - np.abs(c[i] - c[j]))
                margin.append(((i, j), m))
                if m >= 0:
                    out.append((i, j))
    return np.array(out, np.int32).reshape(-1, 2), dict(margin)


def _ident(t):
    return [1, 0, 0, 0, *t]


def test_broadphase_touching_and_separated_axis_aligned():
    # unit cubes on the x axis: centres 1.0 apart touch (|dc| == h_i + h_j,
    # counts as overlap), 1.0 + 2^-20 apart do not; the y and z extents overlap
    aabb = np.array([[-0.5, -0.5, -0.5, 0.5, 0.5, 0.5]], np.float32)
    poses = np.array([_ident([0, 0, 0]), _ident([1.0, 0, 0]),
                      _ident([2.0 + 2.0 ** -20, 0.25, 0]),
                      _ident([-1.0, 0.999, -0.999])], np.float32)
    osh = np.zeros(4, np.int32)
    got = oracle.broadphase(aabb, poses, osh, np.array([0, 4], np.int32))
    # 0-1 touch on x; 1-2 separated by 2^-20 on x; 0-3 touch on x, overlap y, z;
    # 0-2, 1-3, 2-3 far apart
    np.testing.assert_array_equal(got, [[0, 1], [0, 3]])


def test_broadphase_touching_after_half_turn():
    # a half turn about z (q = (0, 0, 0, 1), exact in float32) mirrors the
    # off-centre box [0, 1] x [-0.5, 0.5] x [-0.5, 0.5] to [-1, 0] in x: a box
    # at x = -1.5 of half width 0.5 touches it, one at x = +0.75 does not
    aabb = np.array([[0.0, -0.5, -0.5, 1.0, 0.5, 0.5],
                     [-0.5, -0.5, -0.5, 0.5, 0.5, 0.5]], np.float32)
    poses = np.array([[0, 0, 0, 1, 0, 0, 0], _ident([-1.5, 0, 0]),
                      _ident([0.5 + 2.0 ** -20, 0, 0])], np.float32)
    osh = np.array([0, 1, 1], np.int32)
    got = oracle.broadphase(aabb, poses, osh, np.array([0, 2, 3], np.int32))
    np.testing.assert_array_equal(got, [[0, 1]])
    # without the half turn the body box spans [0, 1]: the box at -1.5 misses
    poses[0, :4] = [1, 0, 0, 0]
    got = oracle.broadphase(aabb, poses, osh, np.array([0, 2, 3], np.int32))
    assert got.shape == (0, 2)


def test_broadphase_rotated_elongated_boxes_hand_computed():
    # a rod of half extents (1, 0.1, 0.1) under q = (0.5, 0.5, -0.5, 0.5)
    # (90 deg about z, then 90 deg about x; exact in float32): R maps body x
    # to world z, so its world half extents are (0.1, 0.1, 1.0).  The
    # transposed |R^T| h would give (0.1, 1.0, 0.1) instead.
    q = np.array([0.5, 0.5, -0.5, 0.5])
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    np.testing.assert_allclose(np.abs(R) @ [1.0, 0.1, 0.1], [0.1, 0.1, 1.0], atol=1e-15)
    aabb = np.array([[-1, -0.1, -0.1, 1, 0.1, 0.1],
                     [-0.05, -0.05, -0.05, 0.05, 0.05, 0.05]], np.float32)
    # one environment (rod, probe) per probe: along z at 0.9 (within reach)
    # and 1.2 (beyond 1.0 + 0.05); along y at 0.12 (0.1 + 0.05 > 0.12) and 0.9
    probes = [[0, 0, 0.9], [0, 0, 1.2], [0, 0.12, 0], [0, 0.9, 0]]
    poses = np.concatenate([np.array([[*q, 0, 0, 0], _ident(t)], np.float32)
                            for t in probes])
    osh = np.array([0, 1] * 4, np.int32)
    env = np.arange(0, 9, 2, dtype=np.int32)
    got = oracle.broadphase(aabb, poses, osh, env)
    np.testing.assert_array_equal(got, [[0, 1], [4, 5]])


@pytest.mark.parametrize("sizes", [[0], [1], [2], [25], [0, 1, 25, 0, 2, 7, 25]])
def test_broadphase_matches_float64_brute_force(sizes):
    rng = np.random.default_rng(sum(sizes) + 11 * len(sizes))
    S = 6
    lo = rng.uniform(-0.6, -0.05, (S, 3))
    hi = rng.uniform(0.05, 0.9, (S, 3))  # off-centre boxes: R c matters
    hi[0] = [1.2, 0.08, 0.1]             # a rod: |R| h vs |R^T| h matters
    lo[0] = [-0.9, -0.06, -0.1]
    aabb = np.concatenate([lo, hi], 1).astype(np.float32)
    n = sum(sizes)
    q = Rotation.random(max(n, 1), random_state=int(rng.integers(1 << 30))).as_quat()
    poses = np.zeros((max(n, 1), 7), np.float32)
    poses[:, 0] = q[:, 3]
    poses[:, 1:4] = q[:, :3]
    poses[:, 4:] = rng.uniform(-1.2, 1.2, (max(n, 1), 3))
    osh = rng.integers(0, S, max(n, 1)).astype(np.int32)
    env = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    got = oracle.broadphase(aabb, poses, osh, env)
    want, margin = _brute_pairs64(aabb, poses, osh, env)
    # the oracle works in float32: only pairs whose float64 margin is within
    # 1e-5 of zero may be decided either way
    got_s = {tuple(p) for p in got}
    want_s = {tuple(p) for p in want}
    for p in got_s ^ want_s:
        assert abs(margin[p]) < 1e-5, (p, margin[p])
    # environment, then i, then j
    if len(got):
        key = got[:, 0].astype(np.int64) * 4096 + got[:, 1]
        assert np.all(np.diff(key) > 0)
        e_of = np.searchsorted(env, np.arange(len(osh)), side="right") - 1
        assert np.all(e_of[got[:, 0]] == e_of[got[:, 1]])
    if sizes == [25]:
        assert 10 < len(got) < 300  # a dense environment with many overlaps


# ------------------------------------------------------------------ global crops

def _R64(pose):
    w, x, y, z = (float(v) for v in pose[:4])
    return Rotation.from_quat([x, y, z, w]).as_matrix()


@pytest.mark.parametrize("n_points", [2048, 64, 40, 1])
def test_global_crop_first_samples_in_canonical_frame(n_points):
    rng = np.random.default_rng(n_points)
    pts = rng.uniform(-0.8, 0.8, (2, n_points, 3)).astype(np.float32)
    aabb = np.array([[-0.8, -0.8, -0.8, 0.8, 0.8, 0.8],
                     [-0.8, -0.6, -0.7, 0.8, 0.5, 0.8]], np.float32)
    q = Rotation.random(6, random_state=3).as_quat()
    poses = np.zeros((6, 7), np.float32)
    poses[:, 0] = q[:, 3]
    poses[:, 1:4] = q[:, :3]
    poses[:, 4:] = rng.uniform(-1, 1, (6, 3))
    osh = np.array([0, 1, 1, 0, 0, 1], np.int32)
    pairs = np.array([[0, 1], [2, 3], [4, 5]], np.int32)
    r = oracle.crop_forward(pts, aabb, poses, osh, pairs, 0.01, mode="global")
    cnt_want = min(KMAX, n_points)
    for p, (a, b) in enumerate(pairs):
        RA, RB = _R64(poses[a]), _R64(poses[b])
        tA, tB = poses[a, 4:].astype(np.float64), poses[b, 4:].astype(np.float64)
        Rrel = RA.T @ RB
        trel = RA.T @ (tB - tA)
        c = r["centre"][p].astype(np.float64)
        cB = Rrel.T @ (c - trel)
        for side, (o, cX, M) in enumerate([(a, c, np.eye(3)), (b, cB, Rrel)]):
            assert r["cnt"][p, side] == cnt_want
            np.testing.assert_array_equal(r["idx"][p, side, :cnt_want], np.arange(cnt_want))
            assert np.all(r["idx"][p, side, cnt_want:] == -1)
            assert np.all(r["xyz"][p, side, cnt_want:] == 0)
            # the radius plays no part: points far outside 0.01 are taken
            src = pts[osh[o], :cnt_want].astype(np.float64)
            want = (M @ (src - cX).T).T
            np.testing.assert_allclose(r["xyz"][p, side, :cnt_want], want, atol=4e-6)
            # and B's canonical coordinates are A's body frame about the centre
            if side == 1:
                world = (RB @ src.T).T + tB
                can = (RA.T @ (world - tA).T).T - c
                np.testing.assert_allclose(r["xyz"][p, 1, :cnt_want], can, atol=4e-6)


# ------------------------------------------------------------------ loss value

def _bias_net(y, f_chan=None):
    """All weights zero; the head's last bias is y (so the raw outputs are y),
    and the encoder's last bias puts f_chan[c] into pooled channel c of every
    object with a non-empty crop (ReLU of a constant)."""
    W = [np.zeros((o, i)) for i, o in oracle.LAYER_DIMS]
    b = [np.zeros(o) for _, o in oracle.LAYER_DIMS]
    b[5][:] = y
    if f_chan is not None:
        for c, v in f_chan.items():
            b[2][c] = v
    return oracle.flatten_params(list(zip(W, b)))


def _one_pair(cnt_a=3, cnt_b=5):
    xyz = np.zeros((1, 2, KMAX, 3), np.float32)
    xyz[0, :, :, :] = 0.01
    return xyz, np.array([[cnt_a, cnt_b]], np.int32)


HP = (1.0, 1.0, 1.0, 0.01, 0.5)  # w_pt, w_n, w_d, Huber beta, alpha


def _loss(y, tgt, f_chan=None, cnt=(3, 5), hp=HP):
    xyz, c = _one_pair(*cnt)
    L, _ = oracle.loss_grad(_bias_net(y, f_chan), xyz, c, np.array([tgt], np.float64), hp)
    return L


def test_loss_value_collision_terms():
    # logit ln 3, label 1: BCE = log(1 + e^{-ln 3}) = log(4/3)
    # point (0.1, -0.2, 0.3) vs (0.1, 0.1, -0.1): |d|^2 = 0.09 + 0.16 = 0.25
    # normal (3, 4, 0) vs (1, 0, 0): cos = 0.6 -> 1 - cos = 0.4
    # depth 0.012 vs 0.007: |e| = 0.005 < beta -> 0.5 e^2 / beta = 1.25e-3
    y = [math.log(3.0), 0.1, -0.2, 0.3, 3.0, 4.0, 0.0, 0.012]
    tgt = [1, 0.1, 0.1, -0.1, 1.0, 0.0, 0.0, 0.007]
    want = math.log(4 / 3) + 0.25 + 0.4 + 1.25e-3
    assert _loss(y, tgt) == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_loss_value_separated_pair_ignores_point_and_normal():
    # label 0, logit ln 3: BCE = ln 3 + log(4/3) = log 4; the point and normal
    # errors are large but do not count; depth error -0.03 (|e| >= beta):
    # |e| - beta / 2 = 0.025
    y = [math.log(3.0), 5.0, 5.0, 5.0, -1.0, 0.0, 0.0, -0.03]
    tgt = [0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    assert _loss(y, tgt) == pytest.approx(math.log(4.0) + 0.025, rel=1e-12)


def test_loss_value_opposite_normal_zero_logit_and_embedding():
    # logit 0, label 1: log 2; normal opposite the target: 1 - cos = 2;
    # point exact; depth exact.  Embedding: channel 0 = 0.5, channel 7 = 0.25
    # in both objects (non-empty crops), channel 9 = -1 (ReLU -> 0):
    # alpha * mean(f^2) = 0.5 * 2 (0.25 + 0.0625) / 512
    y = [0.0, 0.3, 0.0, 0.0, 0.0, -2.0, 0.0, 0.1]
    tgt = [1, 0.3, 0.0, 0.0, 0.0, 0.5, 0.0, 0.1]
    f = {0: 0.5, 7: 0.25, 9: -1.0}
    want = math.log(2.0) + 2.0 + 0.5 * 2 * (0.25 + 0.0625) / 512
    assert _loss(y, tgt, f) == pytest.approx(want, rel=1e-12)
    # an empty crop pools to zero: only object A's embedding counts
    want_a = math.log(2.0) + 2.0 + 0.5 * (0.25 + 0.0625) / 512
    assert _loss(y, tgt, f, cnt=(4, 0)) == pytest.approx(want_a, rel=1e-12)


def test_loss_value_weights_and_huber_branch_edge():
    # weights w_pt = 2, w_n = 3, w_d = 5, beta = 0.1; large negative logit with
    # label 1: BCE = log(1 + e^{20}) = 20 + log(1 + e^{-20})
    # point error (0, 0, 0.5): 2 * 0.25; normal orthogonal: 3 * 1;
    # depth error exactly -beta (the linear branch): 5 (0.1 - 0.05) = 0.25
    y = [-20.0, 0.0, 0.0, 0.5, 0.0, 0.0, 1.0, 0.1]
    tgt = [1, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.2]
    hp = (2.0, 3.0, 5.0, 0.1, 0.0)
    want = 20 + math.log1p(math.exp(-20)) + 0.5 + 3.0 + 0.25
    assert _loss(y, tgt, hp=hp) == pytest.approx(want, rel=1e-10)


def test_loss_value_raw_normal_length_term():
    # w_len (|n| - 1)^2 on every pair: raw normal (3, 4, 0) has length 5 ->
    # 0.25 * 16 = 4; label 0 (the term does not depend on the label), logit
    # 0: log 2; depth exact; the normal's direction plays no part (cos term
    # off for label 0)
    y = [0.0, 0.0, 0.0, 0.0, 3.0, 4.0, 0.0, 0.0]
    tgt = [0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    hp = (1.0, 1.0, 1.0, 0.01, 0.0, 0.25)
    assert _loss(y, tgt, hp=hp) == pytest.approx(math.log(2.0) + 4.0, rel=1e-12)
    # unit length: no contribution; length 0.5 with label 1 and the target
    # along n: log(1 + e^{-2}) + 0.25 * 0.25
    y = [2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.5, 0.0]
    tgt = [1, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0]
    assert _loss(y, tgt, hp=hp) == pytest.approx(math.log1p(math.exp(-2.0)) + 0.0625, rel=1e-12)
    y[6] = 1.0
    assert _loss(y, tgt, hp=hp) == pytest.approx(math.log1p(math.exp(-2.0)), rel=1e-12)


def test_loss_is_mean_over_pairs():
    y = [0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    xyz = np.zeros((2, 2, KMAX, 3), np.float32)
    cnt = np.array([[0, 0], [0, 0]], np.int32)
    tgt = np.array([[0, 0, 0, 0, 1, 0, 0, 0.0],      # log 2
                    [1, 0, 0, 0, -1, 0, 0, 0.0]])    # log 2 + 2
    L, _ = oracle.loss_grad(_bias_net(y), xyz, cnt, tgt, HP)
    assert L == pytest.approx(math.log(2.0) + 1.0, rel=1e-12)


# ------------------------------------------------------------------ tie rule

def _tie_lib(pts_a, pts_b):
    n = 2048
    P = np.full((2, n, 3), 5.0, np.float32)  # far outside the ball
    P[0, :len(pts_a)] = pts_a
    P[1, :len(pts_b)] = pts_b
    aabb = np.array([[-1, -1, -1, 1, 1, 1]] * 2, np.float32)
    return P, aabb


def _perm_slots(rng, n, k):
    return np.sort(rng.choice(n, k, replace=False))


def test_selection_ties_go_to_lower_index():
    # both objects at the identity with the same box: the crop centre is 0 in
    # both frames.  Object A: 100 samples at float32-equal squared distance
    # 0.1^2 (the six axis points (+-0.1, 0, 0), ... each have the key
    # fl(0.1 * 0.1) exactly), scattered over the index range, plus 30 samples
    # nearer (0.05 along axes) that always win.  Only the 34 lowest-index
    # distance-0.1 samples may fill the crop.
    rng = np.random.default_rng(9)
    axis_pts = np.array([[0.1, 0, 0], [-0.1, 0, 0], [0, 0.1, 0], [0, -0.1, 0],
                         [0, 0, 0.1], [0, 0, -0.1]], np.float32)
    slots_far = _perm_slots(rng, 2048, 100)
    rest = np.setdiff1d(np.arange(2048), slots_far)
    slots_near = np.sort(rng.choice(rest, 30, replace=False))
    pa = np.full((2048, 3), 5.0, np.float32)
    pa[slots_far] = axis_pts[rng.integers(0, 6, 100)]
    near = np.array([[0.05, 0, 0], [0, -0.05, 0], [0, 0, 0.05]], np.float32)
    pa[slots_near] = near[rng.integers(0, 3, 30)]
    # object B: 64 + 1 exact duplicates of one point; the highest index is out
    pb = np.full((2048, 3), 5.0, np.float32)
    slots_b = _perm_slots(rng, 2048, 65)
    pb[slots_b] = [0.0, 0.2, 0.0]
    P = np.stack([pa, pb])
    aabb = np.array([[-1, -1, -1, 1, 1, 1]] * 2, np.float32)
    poses = np.array([_ident([0, 0, 0]), _ident([0, 0, 0])], np.float32)
    r = oracle.crop_forward(P, aabb, poses, np.array([0, 1], np.int32),
                            np.array([[0, 1]], np.int32), 0.25)
    np.testing.assert_array_equal(r["centre"][0], [0, 0, 0])
    assert r["cnt"][0, 0] == KMAX and r["cnt"][0, 1] == KMAX
    # nearest first, ties by index: the 30 near samples in index order... the
    # near samples all have d^2 = fl(0.05^2), one key: index order
    np.testing.assert_array_equal(r["idx"][0, 0, :30], slots_near)
    np.testing.assert_array_equal(r["idx"][0, 0, 30:], slots_far[:34])
    np.testing.assert_array_equal(r["idx"][0, 1], slots_b[:64])
    assert slots_b[64] not in r["idx"][0, 1]


def test_selection_tie_at_the_boundary_of_the_ball():
    # r = 0.25: samples at squared distance exactly fl(0.25 * 0.25) = r2 are
    # inside (d^2 <= r2); 70 of them, only the 64 lowest indices are kept;
    # samples just beyond (0.25 + 2^-24 * 4) are outside
    rng = np.random.default_rng(10)
    slots = _perm_slots(rng, 2048, 70)
    pa = np.full((2048, 3), 5.0, np.float32)
    pa[slots] = [0.25, 0, 0]
    out_slots = np.setdiff1d(np.arange(2048), slots)[:5]
    pa[out_slots] = [np.nextafter(np.float32(0.25), np.float32(1)), 0, 0]
    pb = np.full((2048, 3), 5.0, np.float32)
    P = np.stack([pa, pb])
    aabb = np.array([[-1, -1, -1, 1, 1, 1]] * 2, np.float32)
    poses = np.array([_ident([0, 0, 0]), _ident([0, 0, 0])], np.float32)
    r = oracle.crop_forward(P, aabb, poses, np.array([0, 1], np.int32),
                            np.array([[0, 1]], np.int32), 0.25)
    assert r["cnt"][0, 0] == KMAX and r["cnt"][0, 1] == 0
    np.testing.assert_array_equal(r["idx"][0, 0], slots[:64])
    assert np.all(r["idx"][0, 1] == -1)


# ------------------------------------------------------------- bf16 operands

def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    # exact ties and neighbours of ties: 1 + (2j + 1) 2^-8 at binade scales
    j = np.arange(0, 128)
    ties = np.concatenate([(1 + (2 * j + 1) * 2.0 ** -8) * s_ for s_ in (1.0, -2.0 ** 5, 2.0 ** -9)])
    ties = ties.astype(np.float32)
    nxt = np.nextafter(ties, np.float32(np.inf))
    prv = np.nextafter(ties, np.float32(-np.inf))
    v = np.concatenate([v, ties, nxt, prv, np.float32([0.0, -0.0, 1.0, -1.0, 3.0e38])])
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(v), want)
    # float64 inputs are rounded to float32 first, as a float32 producer holds them
    w = rng.standard_normal(1000)
    want = torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(w), want)


def _st_net_loss(torch, flat, xyz, cnt, lab, alpha):
    """Mean of BCE(y0, lab) + alpha mean(f^2) through the crop network in
    float64 autograd, with straight-through bf16 operands (torch's rounding)
    in encoder layers 2 and 3 and head layers 1 and 2; layer 3's backward
    unrounded."""
    def r(x):
        return x.float().to(torch.bfloat16).double()

    class RoundedLinear(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, W, b, round_back):
            ctx.save_for_backward(x, W)
            ctx.round_back = round_back
            return r(x) @ r(W).T + b

        @staticmethod
        def backward(ctx, gy):
            x, W = ctx.saved_tensors
            if ctx.round_back:
                return r(gy) @ r(W), r(gy).T @ r(x), gy.sum(0), None
            return gy @ W, gy.T @ x, gy.sum(0), None

    offs = np.cumsum([0] + [i * o + o for i, o in oracle.LAYER_DIMS])
    prm = torch.tensor(flat, dtype=torch.float64, requires_grad=True)
    Ws, bs = [], []
    for l, (fi, fo) in enumerate(oracle.LAYER_DIMS):
        Ws.append(prm[offs[l]:offs[l] + fi * fo].view(fo, fi))
        bs.append(prm[offs[l] + fi * fo:offs[l + 1]])
    P = cnt.shape[0]
    feats = []
    for p in range(P):
        f = []
        for o in range(2):
            n = int(cnt[p, o])
            if n == 0:
                f.append(torch.zeros(256, dtype=torch.float64))
                continue
            x = torch.tensor(xyz[p, o, :n].astype(np.float64))
            h1 = torch.relu(x @ Ws[0].T + bs[0])
            h2 = torch.relu(RoundedLinear.apply(h1, Ws[1], bs[1], True))
            h3 = torch.relu(RoundedLinear.apply(h2, Ws[2], bs[2], False))
            f.append(h3.max(dim=0).values)
        feats.append(torch.cat(f))
    F = torch.stack(feats)
    g1 = torch.relu(RoundedLinear.apply(F, Ws[3], bs[3], True))
    g2 = torch.relu(RoundedLinear.apply(g1, Ws[4], bs[4], True))
    y = g2 @ Ws[5].T + bs[5]
    bce = torch.nn.functional.binary_cross_entropy_with_logits(
        y[:, 0], torch.tensor(lab, dtype=torch.float64), reduction="none")
    L = (bce + alpha * (F * F).mean(dim=1)).mean()
    L.backward()
    return float(L.detach()), prm.grad.numpy()


def test_bf16_operand_mode_matches_straight_through_autograd():
    torch = pytest.importorskip("torch")
    import synth
    rng = np.random.default_rng(8)
    P = 4
    cnt = np.array([[64, 17], [5, 0], [33, 64], [1, 40]], np.int32)
    xyz = np.zeros((P, 2, KMAX, 3), np.float32)
    for p in range(P):
        for o in range(2):
            xyz[p, o, :cnt[p, o]] = rng.uniform(-0.25, 0.25, (cnt[p, o], 3))
    flat = oracle.flatten_params(synth.xavier_weights(9, bias_scale=0.1)).astype(np.float64)
    lab = np.array([1.0, 0.0, 1.0, 0.0])
    tgt = np.zeros((P, 8))
    tgt[:, 0] = lab
    hp = (0.0, 0.0, 0.0, 0.01, 0.5, 0.0)  # BCE and the embedding term only
    L_b, g_b = oracle.loss_grad(flat, xyz, cnt, tgt, hp, operands="bf16")
    L_e, g_e = oracle.loss_grad(flat, xyz, cnt, tgt, hp, operands="exact")
    L_t, g_t = _st_net_loss(torch, flat, xyz, cnt, lab, hp[4])
    assert abs(L_b - L_t) <= 1e-12 * abs(L_t)
    assert np.linalg.norm(g_b - g_t) <= 1e-10 * np.linalg.norm(g_t)
    # the rounding is really applied (the two modes differ at bf16 scale)
    d = np.linalg.norm(g_b - g_e) / np.linalg.norm(g_e)
    assert 1e-5 < d < 5e-2, d
