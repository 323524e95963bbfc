"""Pins of the convex-hull intersection oracle (``oracle/convex.py``) against
closed forms: axis-aligned boxes (interval overlap per axis), rotated boxes
(the separating-axis theorem), a point inside / outside a tetrahedron, and
symmetry / rigid-motion invariance."""

import numpy as np

from oracle import convex as CX

RNG = np.random.default_rng(5)


def _box(c, h, R=np.eye(3)):
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    return (corners * h) @ R.T + c


def _rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    return CX.posed(np.eye(3), np.concatenate([q, [0, 0, 0]])).T


def test_axis_aligned_boxes_match_interval_overlap():
    for _ in range(200):
        c1, c2 = RNG.uniform(-1, 1, 3), RNG.uniform(-1, 1, 3)
        h1, h2 = RNG.uniform(0.1, 0.6, 3), RNG.uniform(0.1, 0.6, 3)
        gap = np.abs(c1 - c2) - (h1 + h2)
        if np.abs(gap).min() < 1e-6:
            continue
        want = bool(np.all(gap < 0))
        assert CX.hulls_intersect(_box(c1, h1), _box(c2, h2)) == want


def test_rotated_boxes_match_separating_axis_theorem():
    def sat(c1, R1, h1, c2, R2, h2):
        axes = [R1[:, i] for i in range(3)] + [R2[:, i] for i in range(3)]
        axes += [np.cross(R1[:, i], R2[:, j]) for i in range(3) for j in range(3)]
        margin = np.inf
        for ax in axes:
            n = np.linalg.norm(ax)
            if n < 1e-9:
                continue
            ax = ax / n
            r = np.sum(h1 * np.abs(R1.T @ ax)) + np.sum(h2 * np.abs(R2.T @ ax))
            margin = min(margin, r - abs((c2 - c1) @ ax))
        return margin
    n = 0
    for _ in range(300):
        R1, R2 = _rot(RNG), _rot(RNG)
        c1, c2 = RNG.uniform(-0.8, 0.8, 3), RNG.uniform(-0.8, 0.8, 3)
        h1, h2 = RNG.uniform(0.1, 0.5, 3), RNG.uniform(0.1, 0.5, 3)
        m = sat(c1, R1, h1, c2, R2, h2)
        if abs(m) < 1e-6:
            continue
        assert CX.hulls_intersect(_box(c1, h1, R1), _box(c2, h2, R2)) == (m > 0)
        n += 1
    assert n > 250


def test_point_in_tetrahedron():
    T = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    assert CX.hulls_intersect(T, [[0.2, 0.2, 0.2]])
    assert not CX.hulls_intersect(T, [[0.5, 0.5, 0.5]])      # beyond the face x+y+z=1
    assert CX.hulls_intersect(T, [[1 / 3, 1 / 3, 1 / 3]])    # on the face
    assert not CX.hulls_intersect(T, [[-0.01, 0.2, 0.2]])


def test_symmetry_and_rigid_motion():
    for _ in range(50):
        A = RNG.normal(size=(12, 3)) * 0.4
        B = RNG.normal(size=(10, 3)) * 0.4 + RNG.uniform(-1, 1, 3)
        ans, robust = CX.robust_intersect(A, B)
        if not robust:
            continue
        assert CX.hulls_intersect(B, A) == ans
        q = RNG.normal(size=4)
        q /= np.linalg.norm(q)
        pose = np.concatenate([q, RNG.uniform(-2, 2, 3)])
        assert CX.hulls_intersect(CX.posed(A, pose), CX.posed(B, pose)) == ans
