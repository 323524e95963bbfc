"""Pins of oracle (a), the float64 geometric contact detector, against closed
forms, a textbook separating-axis test, symmetries and its own brute force.

Each expected value below comes from geometry worked out by hand (or from the
separating-axis theorem, the textbook convex test the paper contrasts with in
Sec. II), never from the oracle itself."""

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import synth
from synth.shapes import box_mesh, ellipsoid_mesh, torus_mesh


def _pose(q_wxyz=(1, 0, 0, 0), t=(0, 0, 0)):
    return np.array(list(q_wxyz) + list(t), np.float32)


def _contact_two(mA, mB, pA, pB, samples=None, culled=True):
    rng = np.random.default_rng(0)
    if samples is None:
        samples = [synth.sample_surface(m, 512, rng) for m in (mA, mB)]
    S = np.stack(samples).astype(np.float32)
    poses = np.stack([pA, pB])
    return oracle.contact([mA, mB], S, poses, np.array([0, 1], np.int32),
                          np.array([[0, 1]], np.int32), culled=culled)[0]


def _rigid(R, t, pose):
    """Apply world motion (R, t) to a (w,x,y,z,t) pose."""
    r0 = Rotation.from_quat([pose[1], pose[2], pose[3], pose[0]])
    r1 = Rotation.from_matrix(R) * r0
    q = r1.as_quat()  # x y z w
    tt = R @ pose[4:].astype(np.float64) + t
    return np.array([q[3], q[0], q[1], q[2], *tt], np.float32)


def test_sphere_sphere_overlap_depth():
    # two UV spheres; the equator rings hold vertices exactly at +-r on x, so
    # the deepest candidate is A's vertex (rA,0,0): depth = rA + rB - d
    rA, rB, d = 0.5, 0.4, 0.8
    A = ellipsoid_mesh((rA, rA, rA), 24, 48)
    B = ellipsoid_mesh((rB, rB, rB), 24, 48)
    out = _contact_two(A, B, _pose(), _pose(t=(d, 0, 0)))
    assert out[0] == 1.0
    # inscribed tessellation: surface within r (1 - cos(pi/48)) ~ 1e-3 of the sphere
    assert abs(out[7] - (rA + rB - d)) < 5e-3
    assert out[4] > 0.99  # normal from A towards B is +x
    assert np.linalg.norm(out[1:4] - [(rA + d - rB) / 2, 0, 0]) < 2e-2


def test_sphere_sphere_gap_exact():
    # separated: both meshes have a vertex on the x axis facing each other,
    # and the polytopes lie inside their spheres, so the gap is d - rA - rB
    rA, rB, d = 0.5, 0.4, float(np.float32(1.2))  # poses are float32
    A = ellipsoid_mesh((rA, rA, rA), 24, 48)
    B = ellipsoid_mesh((rB, rB, rB), 24, 48)
    out = _contact_two(A, B, _pose(), _pose(t=(d, 0, 0)))
    assert out[0] == 0.0
    assert abs(out[7] - (-(d - rA - rB))) < 1e-9
    np.testing.assert_allclose(out[4:7], [1, 0, 0], atol=1e-9)
    np.testing.assert_allclose(out[1:4], [(rA + d - rB) / 2, 0, 0], atol=1e-9)


@pytest.mark.parametrize("seed", [0, 1])
def test_box_on_plane(seed):
    # small box sinking delta into a large slab whose top face is z = 0
    delta = 0.03
    box = box_mesh((0.2, 0.15, 0.1), (4, 3, 2))
    plane = box_mesh((3.0, 3.0, 0.25), (6, 6, 1))
    pA = _pose(t=(0.1, -0.2, 0.1 - delta))
    pB = _pose(t=(0, 0, -0.25))
    rng = np.random.default_rng(seed)
    R = Rotation.random(random_state=seed).as_matrix()
    t = rng.uniform(-1, 1, 3)
    out = _contact_two(box, plane, _rigid(R, t, pA), _rigid(R, t, pB))
    assert out[0] == 1.0
    assert abs(out[7] - delta) < 1e-6
    np.testing.assert_allclose(out[4:7], R @ [0, 0, -1], atol=1e-6)
    # point lies half-way between the sunk face and the slab top
    local = R.T @ (out[1:4] - t)
    assert abs(local[2] - (-delta / 2)) < 1e-6
    assert abs(local[0] - 0.1) <= 0.2 + 1e-9 and abs(local[1] + 0.2) <= 0.15 + 1e-9


@pytest.mark.parametrize("off", [(0.9, 0.0, 0.0), (0.8, 0.45, 0.0),
                                 (0.75, 0.5, 0.42)])
def test_separated_boxes_distance(off):
    hA, hB = np.array([0.3, 0.2, 0.1]), np.array([0.25, 0.15, 0.2])
    A = box_mesh(hA, (3, 2, 2))
    B = box_mesh(hB, (2, 2, 2))
    out = _contact_two(A, B, _pose(), _pose(t=off))
    gaps = np.maximum(0.0, np.abs(off) - hA - hB)
    expect = np.sqrt((gaps ** 2).sum())
    assert expect > 0
    assert out[0] == 0.0
    assert abs(-out[7] - expect) < 1e-7


def _sat_overlap(cA, RA, hA, cB, RB, hB):
    """Separating-axis test for two oriented boxes (15 axes)."""
    axes = [RA[:, i] for i in range(3)] + [RB[:, i] for i in range(3)]
    for i in range(3):
        for j in range(3):
            c = np.cross(RA[:, i], RB[:, j])
            if np.linalg.norm(c) > 1e-9:
                axes.append(c / np.linalg.norm(c))
    d = cB - cA
    margin = np.inf
    for a in axes:
        ra = np.sum(hA * np.abs(RA.T @ a))
        rb = np.sum(hB * np.abs(RB.T @ a))
        margin = min(margin, ra + rb - abs(d @ a))
    return margin


def test_box_box_label_matches_sat():
    rng = np.random.default_rng(7)
    hits = 0
    n = 0
    while n < 40:
        hA = rng.uniform(0.1, 0.4, 3)
        hB = rng.uniform(0.1, 0.4, 3)
        RA = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        RB = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        cB = rng.uniform(-0.7, 0.7, 3)
        m = _sat_overlap(np.zeros(3), RA, hA, cB, RB, hB)
        if abs(m) < 1e-3:
            continue  # too close to touching to call either way
        A = box_mesh(hA, (2, 2, 2))
        B = box_mesh(hB, (2, 2, 2))
        qa = Rotation.from_matrix(RA).as_quat()
        qb = Rotation.from_matrix(RB).as_quat()
        pA = _pose((qa[3], qa[0], qa[1], qa[2]))
        pB = _pose((qb[3], qb[0], qb[1], qb[2]), cB)
        out = _contact_two(A, B, pA, pB)
        assert out[0] == float(m > 0), (m, out)
        hits += m > 0
        n += 1
    assert 5 < hits < 35


def test_winding_inside_matches_analytic():
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1.5, 1.5, size=(400, 3))
    tor = torus_mesh()
    got = oracle.inside(tor, _pose(), pts)
    rho = np.hypot(pts[:, 0], pts[:, 1])
    analytic = (rho - 1.0) ** 2 + pts[:, 2] ** 2 < 0.3 ** 2
    # the 32 x 8 polytope is inscribed in the torus: disagreements only near it
    tube = np.sqrt((rho - 1.0) ** 2 + pts[:, 2] ** 2)
    far = np.abs(tube - 0.3) > 0.3 * (1 - np.cos(np.pi / 8)) + 0.05
    assert np.array_equal(got[far], analytic[far])
    box = box_mesh((0.3, 0.2, 0.1), (2, 2, 2))
    got = oracle.inside(box, _pose(), pts)
    assert np.array_equal(got, np.all(np.abs(pts) < [0.3, 0.2, 0.1], axis=1))


def _lib_pairs(n, seed):
    lib = synth.tiny_library(n_points=512)
    rng = np.random.default_rng(seed)
    poses = synth.random_poses(2 * n, rng, -0.6, 0.6)
    obj_shape = np.tile(np.array([0, 1], np.int32), n)
    pairs = np.stack([np.arange(0, 2 * n, 2), np.arange(1, 2 * n, 2)], 1).astype(np.int32)
    return lib, poses, obj_shape, pairs


def test_swap_symmetry():
    lib, poses, osh, pairs = _lib_pairs(24, 11)
    a = oracle.contact(lib.meshes, lib.points, poses, osh, pairs)
    b = oracle.contact(lib.meshes, lib.points, poses, osh, pairs[:, ::-1].copy())
    assert 3 < a[:, 0].sum() < 21
    np.testing.assert_array_equal(a[:, 0], b[:, 0])
    np.testing.assert_allclose(a[:, 7], b[:, 7], atol=1e-12)
    np.testing.assert_allclose(a[:, 1:4], b[:, 1:4], atol=1e-9)
    np.testing.assert_allclose(a[:, 4:7], -b[:, 4:7], atol=1e-9)


def test_rigid_motion_invariance():
    lib, poses, osh, pairs = _lib_pairs(16, 12)
    R = Rotation.random(random_state=5).as_matrix()
    t = np.array([0.3, -2.0, 1.1])
    moved = np.stack([_rigid(R, t, p) for p in poses])
    a = oracle.contact(lib.meshes, lib.points, poses, osh, pairs)
    b = oracle.contact(lib.meshes, lib.points, moved, osh, pairs)
    np.testing.assert_array_equal(a[:, 0], b[:, 0])
    # poses are stored in float32, so the motion is exact only to ~1e-6
    np.testing.assert_allclose(a[:, 7], b[:, 7], atol=2e-5)
    np.testing.assert_allclose(a[:, 1:4] @ R.T + t, b[:, 1:4], atol=5e-5)
    ok = np.abs(a[:, 7]) > 1e-3
    np.testing.assert_allclose((a[:, 4:7] @ R.T)[ok], b[ok, 4:7], atol=1e-3)


def test_brute_equals_culled():
    lib, poses, osh, pairs = _lib_pairs(12, 13)
    a = oracle.contact(lib.meshes, lib.points, poses, osh, pairs, culled=True)
    b = oracle.contact(lib.meshes, lib.points, poses, osh, pairs, culled=False)
    np.testing.assert_array_equal(a, b)
