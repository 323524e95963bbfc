"""Pins of the voxel-latent oracle (``oracle/voxel.py``) against things the
oracle does not compute itself: library routines for the convolutions, the
adjoint identity of convolution and transposed convolution, closed forms of
the U-Net wiring, exact box-box geometry for the cell selection, invariances.
"""

import numpy as np
import pytest
from scipy import signal

from oracle import voxel as V

RNG = np.random.default_rng(1234)


def test_conv3d_matches_scipy_correlate():
    # out[o] = b[o] + sum_i correlate(pad(x[i]), w[o, i], 'valid')
    for pad in (0, 1):
        x = RNG.standard_normal((2, 5, 5, 5))
        w = RNG.standard_normal((3, 2, 3, 3, 3))
        b = RNG.standard_normal(3)
        got = V.conv3d(x, w, b, pad)
        xp = np.pad(x, ((0, 0), (pad, pad), (pad, pad), (pad, pad)))
        ref = np.stack([b[o] + sum(signal.correlate(xp[i], w[o, i], mode="valid")
                                   for i in range(2)) for o in range(3)])
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_conv_transpose3d_matches_scipy_convolve():
    # transposed convolution = full convolution with the kernel, cropped by pad
    for pad in (0, 1):
        x = RNG.standard_normal((2, 4, 4, 4))
        w = RNG.standard_normal((2, 3, 3, 3, 3))          # [in, out, k, k, k]
        b = RNG.standard_normal(3)
        got = V.conv_transpose3d(x, w, b, pad)
        full = np.stack([sum(signal.convolve(x[i], w[i, o], mode="full") for i in range(2))
                         for o in range(3)])
        n = full.shape[1] - 2 * pad
        ref = full[:, pad:pad + n, pad:pad + n, pad:pad + n] + b[:, None, None, None]
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("pad,d", [(0, 6), (1, 4)])
def test_transposed_convolution_is_the_adjoint(pad, d):
    # <conv(x; W), y> = <x, convT(y; W)> with the same W read as [out][in]
    # by the convolution and [in][out] by the transposed one
    x = RNG.standard_normal((4, d, d, d))
    w = RNG.standard_normal((5, 4, 3, 3, 3))
    y = RNG.standard_normal((5,) + (d + 2 * pad - 2,) * 3)
    lhs = np.sum(V.conv3d(x, w, np.zeros(5), pad) * y)
    rhs = np.sum(x * V.conv_transpose3d(y, w, np.zeros(4), pad))
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))


def _params(seed=3):
    import synth
    return V.split_params(synth.voxel_weights(V.LAYERS, seed))


def _shape(seed=0, n=512):
    rng = np.random.default_rng(seed)
    pts = (rng.uniform(-1, 1, (n, 3)) * np.array([0.8, 0.5, 0.3])).astype(np.float32)
    aabb = np.concatenate([pts.min(0), pts.max(0)]).astype(np.float32)
    return pts, aabb


def test_point_cells_contain_their_points():
    pts, aabb = _shape(1, 4096)
    cell = V.point_cells(pts, aabb)
    assert cell.min() >= 0 and cell.max() <= V.M - 1
    lo, hi = aabb[:3].astype(np.float64), aabb[3:].astype(np.float64)
    a = (hi - lo) / V.M
    tol = 1e-5 * (hi - lo)
    assert np.all(pts >= lo + cell * a - tol) and np.all(pts <= lo + (cell + 1) * a + tol)
    # points on the upper face land in the last cell
    top = pts.copy()
    top[:, 0] = aabb[3]
    assert np.all(V.point_cells(top, aabb)[:, 0] == V.M - 1)


def test_encoder_closed_form_with_zero_weights():
    # all weights zero: every U-Net layer outputs relu(bias); the global feature
    # is [max || mean] of relu(c4.b) = [relu(c4.b) || relu(c4.b)]; the latent of
    # every cell is f.w [relu(d4.b) || g] + f.b
    prm = _params()
    for k in prm:
        if k.endswith(".w") and k[0] in "ecd":
            prm[k] = np.zeros_like(prm[k])
    pts, aabb = _shape(2)
    lat = V.encode_shape(pts, aabb, prm)
    g = np.concatenate([np.maximum(prm["c4.b"], 0), np.maximum(prm["c4.b"], 0)])
    want = prm["f.w"] @ np.concatenate([np.maximum(prm["d4.b"], 0), g]) + prm["f.b"]
    np.testing.assert_allclose(lat, np.broadcast_to(want, lat.shape), rtol=1e-12, atol=1e-12)


def test_encoder_global_feature_is_max_then_mean():
    # only the global half of the final layer reads its input: f.w columns
    # 128..255 pick max-pooled channels, 256..383 mean-pooled ones
    prm = _params(5)
    pts, aabb = _shape(3)
    prm_max = {k: v.copy() for k, v in prm.items()}
    prm_max["f.w"][:, :128] = 0
    prm_max["f.w"][:, 256:] = 0
    prm_mean = {k: v.copy() for k, v in prm.items()}
    prm_mean["f.w"][:, :256] = 0
    # recompute the last convolution's output independently
    h = np.maximum(pts.astype(np.float64) @ prm["e1.w"].T + prm["e1.b"], 0)
    h = np.maximum(h @ prm["e2.w"].T + prm["e2.b"], 0)
    h = np.maximum(h @ prm["e3.w"].T + prm["e3.b"], 0)
    cell = V.point_cells(pts, aabb)
    grid = np.zeros((V.H, 6, 6, 6))
    for n in range(len(pts)):
        grid[:, cell[n, 0], cell[n, 1], cell[n, 2]] = np.maximum(
            grid[:, cell[n, 0], cell[n, 1], cell[n, 2]], h[n])
    s = grid
    for name, pad in (("c1", 0), ("c2", 1), ("c3", 1), ("c4", 1)):
        xp = np.pad(s, ((0, 0), (pad, pad), (pad, pad), (pad, pad)))
        w = prm[name + ".w"]
        s = np.maximum(np.stack([prm[name + ".b"][o] + sum(
            signal.correlate(xp[i], w[o, i], mode="valid") for i in range(w.shape[1]))
            for o in range(w.shape[0])]), 0)
    mx, mean = s.reshape(128, -1).max(1), s.reshape(128, -1).mean(1)
    want_max = prm["f.w"][:, 128:256] @ mx + prm["f.b"]
    want_mean = prm["f.w"][:, 256:] @ mean + prm["f.b"]
    np.testing.assert_allclose(V.encode_shape(pts, aabb, prm_max)[2, 3, 1], want_max, rtol=1e-9)
    np.testing.assert_allclose(V.encode_shape(pts, aabb, prm_mean)[0, 5, 4], want_mean, rtol=1e-9)


def test_encoder_is_invariant_to_point_order():
    prm = _params(6)
    pts, aabb = _shape(4)
    perm = np.random.default_rng(0).permutation(len(pts))
    np.testing.assert_allclose(V.encode_shape(pts, aabb, prm),
                               V.encode_shape(pts[perm], aabb, prm), rtol=1e-12, atol=1e-12)


def _quat_rot64(q):
    w, x, y, z = np.asarray(q, np.float64)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _obb_overlap(c1, R1, h1, c2, R2, h2, slack=0.0):
    """Separating-axis test of two oriented boxes (float64): centres c, axes
    the columns of R, half extents h.  True if no axis separates them by more
    than ``slack``."""
    axes = [R1[:, i] for i in range(3)] + [R2[:, i] for i in range(3)]
    axes += [np.cross(R1[:, i], R2[:, j]) for i in range(3) for j in range(3)]
    d = c2 - c1
    for ax in axes:
        n = np.linalg.norm(ax)
        if n < 1e-12:
            continue
        ax = ax / n
        r1 = np.sum(h1 * np.abs(R1.T @ ax))
        r2 = np.sum(h2 * np.abs(R2.T @ ax))
        if abs(d @ ax) > r1 + r2 + slack:
            return False
    return True


def test_selection_has_no_false_negatives():
    # every cell of A whose box meets B's oriented box (exact SAT in float64)
    # is selected, and likewise for B; the margin (cell half-diagonal) makes
    # this hold for cells that only graze the region
    import synth
    lib = synth.make_library(3, 9)
    rng = np.random.default_rng(7)
    checked = 0
    for trial in range(60):
        sa, sb = rng.integers(0, 3, 2)
        q = synth.random_quaternions(2, rng)
        poses = np.zeros((2, 7), np.float32)
        poses[:, :4] = q
        poses[1, 4:] = rng.uniform(-1.2, 1.2, 3)
        osh = np.array([sa, sb], np.int32)
        mA, mB = V.pair_selection(lib.aabb, poses, osh, np.array([0, 1]))
        for obj, other, mask in ((0, 1, mA), (1, 0, mB)):
            box = lib.aabb[osh[obj]].astype(np.float64)
            obox = lib.aabb[osh[other]].astype(np.float64)
            Ro, Rt = _quat_rot64(poses[obj, :4]), _quat_rot64(poses[other, :4])
            a = (box[3:] - box[:3]) / 6
            cO = (obox[:3] + obox[3:]) / 2
            hO = (obox[3:] - obox[:3]) / 2
            for i in range(6):
                for j in range(6):
                    for k in range(6):
                        cen = box[:3] + (np.array([i, j, k]) + 0.5) * a
                        hit = _obb_overlap(Ro @ cen + poses[obj, 4:], Ro, a / 2,
                                           Rt @ cO + poses[other, 4:], Rt, hO, slack=-1e-6)
                        if hit:
                            assert mask[i, j, k], (trial, obj, i, j, k)
                            checked += 1
    assert checked > 500


def test_selection_is_the_widened_intersection_box():
    # recompute the region in float64 and compare the masks away from ties
    import synth
    lib = synth.make_library(3, 9)
    rng = np.random.default_rng(8)
    for trial in range(40):
        q = synth.random_quaternions(2, rng)
        poses = np.zeros((2, 7), np.float32)
        poses[:, :4] = q
        poses[1, 4:] = rng.uniform(-1.0, 1.0, 3)
        osh = np.array(rng.integers(0, 3, 2), np.int32)
        masks = V.pair_selection(lib.aabb, poses, osh, np.array([0, 1]))
        R = [_quat_rot64(poses[i, :4]) for i in range(2)]
        for obj, other in ((0, 1), (1, 0)):
            box = lib.aabb[osh[obj]].astype(np.float64)
            obox = lib.aabb[osh[other]].astype(np.float64)
            Rr = R[obj].T @ R[other]                     # other -> obj frame
            tr = R[obj].T @ (poses[other, 4:].astype(np.float64) - poses[obj, 4:])
            c = Rr @ ((obox[:3] + obox[3:]) / 2) + tr
            h = np.abs(Rr) @ ((obox[3:] - obox[:3]) / 2)
            a = (box[3:] - box[:3]) / 6
            eps = np.linalg.norm(a) / 2
            lo = np.maximum(box[:3], c - h) - eps
            hi = np.minimum(box[3:], c + h) + eps
            cen = box[:3, None] + (np.arange(6) + 0.5) * a[:, None]
            ins = (cen >= lo[:, None]) & (cen <= hi[:, None])
            near = (np.abs(cen - lo[:, None]) < 1e-5) | (np.abs(cen - hi[:, None]) < 1e-5)
            want = ins[0][:, None, None] & ins[1][None, :, None] & ins[2][None, None, :]
            ok = ~(near[0][:, None, None] | near[1][None, :, None] | near[2][None, None, :])
            np.testing.assert_array_equal(masks[obj][ok], want[ok])


def test_predictor_is_symmetric_in_the_objects():
    prm = _params(9)
    fA, fB = RNG.standard_normal(16), RNG.standard_normal(16)
    pA, pB = RNG.standard_normal(7), RNG.standard_normal(7)
    assert V.predictor(fA, pA, fB, pB, prm) == V.predictor(fB, pB, fA, pA, prm)
    # and it pools by a maximum (not a sum or mean): two identical objects give
    # the second MLP applied to one object's branch
    x = np.concatenate([fA, pA])
    z = np.maximum(prm["p1.w"] @ x + prm["p1.b"], 0)
    z = np.maximum(prm["p2.w"] @ z + prm["p2.b"], 0)
    z = np.maximum(prm["p3.w"] @ z + prm["p3.b"], 0)
    for k in ("q1", "q2", "q3"):
        z = np.maximum(prm[k + ".w"] @ z + prm[k + ".b"], 0)
    want = float(prm["q4.w"][0] @ z + prm["q4.b"][0])
    assert abs(V.predictor(fA, pA, fA, pA, prm) - want) <= 1e-12 * max(1.0, abs(want))


def test_relative_pose_of_a_pair():
    # A at the identity: B's relative pose is B's pose; a common rigid motion
    # leaves it unchanged up to the sign of the quaternion
    import synth
    rng = np.random.default_rng(11)
    q = synth.random_quaternions(3, rng).astype(np.float64)
    poseB = np.concatenate([q[0], rng.uniform(-1, 1, 3)])
    ident = np.array([1.0, 0, 0, 0, 0, 0, 0])
    np.testing.assert_allclose(V.relative_pose(ident, poseB), poseB, atol=1e-7)
    poseA = np.concatenate([q[1], rng.uniform(-1, 1, 3)])
    g_q, g_t = q[2], rng.uniform(-1, 1, 3)
    Rg = _quat_rot64(g_q)
    moved = [np.concatenate([V.quat_mul(g_q, p[:4]), Rg @ p[4:] + g_t]) for p in (poseA, poseB)]
    r0 = V.relative_pose(poseA, poseB)
    r1 = V.relative_pose(*moved)
    s = np.sign(r0[0] * r1[0]) or 1.0
    np.testing.assert_allclose(r1[:4] * s, r0[:4], atol=2e-6)
    np.testing.assert_allclose(r1[4:], r0[4:], atol=2e-6)


def test_empty_selection_pools_to_zero():
    # two boxes far apart: no cell is selected and the pooled features are 0
    import synth
    lib = synth.make_library(2, 9)
    prm = _params(10)
    lat = np.ones((2, 6, 6, 6, 16))
    poses = np.array([[1, 0, 0, 0, 0, 0, 0], [1, 0, 0, 0, 9.0, 0, 0]], np.float32)
    r = V.detect(lat, lib.aabb, poses, np.array([0, 1], np.int32), np.array([[0, 1]]), prm)
    assert r["cnt"].tolist() == [[0, 0]]
    assert np.all(r["feat"] == 0)
    # the same boxes at the same place: every cell is selected, the pool is the mean
    poses[1, 4] = 0.0
    r = V.detect(lat * np.arange(1, 17), lib.aabb, poses, np.array([0, 0], np.int32),
                 np.array([[0, 1]]), prm)
    assert r["cnt"].tolist() == [[216, 216]]
    np.testing.assert_allclose(r["feat"][0, 0], np.arange(1, 17))


def test_voxel_blob_round_trip_and_layout():
    # the product's blob layout lists the same tensors in the same order as
    # the oracle, and packing / unpacking is lossless
    from paper_2304_09439_b300 import weights as W
    import synth
    assert [(n, tuple(s)) for n, s in W.VOXEL_LAYERS] == [(n, tuple(s)) for n, s in V.LAYERS]
    assert W.N_VOXEL_PARAMS == V.N_PARAMS
    flat = synth.voxel_weights(V.LAYERS, 2)
    blob = W.pack_voxel(flat)
    assert blob[:8] == b"LOCCV001" and len(blob) == 16 + 4 * V.N_PARAMS
    np.testing.assert_array_equal(W.unpack_voxel(blob), flat)
