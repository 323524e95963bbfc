"""Oracle of the UCF-GJK comparator: exact intersection of convex hulls.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` alone; the product library
never imports it and shares no code with it).

Two convex hulls conv(A) and conv(B) intersect exactly when some convex
combination of A's vertices equals some convex combination of B's:
    lambda >= 0, mu >= 0, sum lambda = 1, sum mu = 1, A^T lambda = B^T mu,
a linear feasibility problem (solved with scipy's HiGHS, float64).  A union of
convex elements collides with another when any pair of elements intersects --
what GJK on a convex decomposition decides, given enough iterations.
"""

from __future__ import annotations

import numpy as np
from scipy.optimize import linprog


def hulls_intersect(A, B) -> bool:
    """Do conv(A) and conv(B) intersect?  A [n, 3], B [m, 3] float64 points."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    n, m = len(A), len(B)
    A_eq = np.zeros((5, n + m))
    A_eq[:3, :n] = A.T
    A_eq[:3, n:] = -B.T
    A_eq[3, :n] = 1.0
    A_eq[4, n:] = 1.0
    b_eq = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    # HiGHS' default can end undecided on degenerate instances; the dual
    # simplex and the interior-point solver are tried next
    for method in ("highs", "highs-ds", "highs-ipm"):
        res = linprog(np.zeros(n + m), A_eq=A_eq, b_eq=b_eq, bounds=(0, None), method=method)
        if res.status in (0, 2):
            return res.status == 0
    raise RuntimeError(f"linprog undecided: {res.message}")


def scaled(V, s):
    """Points scaled by s about their centroid."""
    V = np.asarray(V, np.float64)
    c = V.mean(axis=0)
    return c + s * (V - c)


def robust_intersect(A, B, delta: float = 2e-3):
    """(answer, robust): robust when shrinking and growing both hulls by
    delta about their centroids does not change the answer."""
    try:
        lo = hulls_intersect(scaled(A, 1 - delta), scaled(B, 1 - delta))
        hi = hulls_intersect(scaled(A, 1 + delta), scaled(B, 1 + delta))
        mid = hulls_intersect(A, B)
    except RuntimeError:  # solver undecided: not a case to compare on
        return False, False
    return mid, lo == hi


def posed(V, pose):
    """Body-frame points -> world with pose (w, x, y, z, tx, ty, tz)."""
    w, x, y, z = np.asarray(pose[:4], np.float64)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    return np.asarray(V, np.float64) @ R.T + np.asarray(pose[4:7], np.float64)


def decomposition_collide(elem_off, vert_off, verts, poses, obj_shape, pair):
    """(collide, robust) of one pair of decomposed shapes: any intersecting
    element pair; robust when every element pair's answer is robust."""
    a, b = int(pair[0]), int(pair[1])
    sa, sb = int(obj_shape[a]), int(obj_shape[b])
    hit, robust = False, True
    for i in range(elem_off[sa], elem_off[sa + 1]):
        Va = posed(verts[vert_off[i]:vert_off[i + 1]], poses[a])
        for j in range(elem_off[sb], elem_off[sb + 1]):
            Vb = posed(verts[vert_off[j]:vert_off[j + 1]], poses[b])
            ans, rob = robust_intersect(Va, Vb)
            hit |= ans
            robust &= rob
    return hit, robust
