"""Scenes: many environments of objects, and random pair sweeps.

``uneven_scene``: n_env environments, each with Poisson(lam) objects (clipped
to [1, 25]) drawn from a shape library, uniform rotations, positions uniform in
[-1, 1]^3.  Objects of environment e are obj[env_offsets[e]:env_offsets[e+1]].

``sweep_pairs``: independent object pairs; half with B at a uniform pose
relative to A, half placed near contact (approximate surface gap uniform in
[-gap, gap]) along a random direction.  The near-contact placement bisects the
centre distance until the two surface-sample clouds come within a touching
threshold (a k-d tree query, scipy), then shifts by the drawn gap; the realised
gap is approximate, exact labels come from the geometric contact detector.
"""

from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .poses import random_poses, random_quaternions, quat_multiply
from .shapes import ShapeLibrary


def _quat_to_matrix64(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def uneven_scene(n_env: int, n_shapes: int, seed: int, lam: float = 8.0,
                 n_min: int = 1, n_max: int = 25, extent: float = 1.0):
    """Returns (poses f32 [n_obj,7], obj_shape i32 [n_obj], env_offsets i32
    [n_env+1])."""
    rng = np.random.default_rng(seed)
    counts = np.clip(rng.poisson(lam, size=n_env), n_min, n_max)
    offsets = np.zeros(n_env + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    n_obj = int(offsets[-1])
    poses = random_poses(n_obj, rng, -extent, extent)
    obj_shape = rng.integers(0, n_shapes, size=n_obj).astype(np.int32)
    return poses, obj_shape, offsets.astype(np.int32)


def _touching_distance(pa: np.ndarray, tree_a: cKDTree, pb: np.ndarray,
                       u: np.ndarray, thresh: float, iters: int = 18) -> float:
    """Smallest s (bisection) at which cloud B shifted by s*u is within
    ``thresh`` of cloud A."""
    ra = np.linalg.norm(pa, axis=1).max()
    rb = np.linalg.norm(pb, axis=1).max()
    lo, hi = 0.0, ra + rb + 2 * thresh
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        d, _ = tree_a.query(pb + mid * u, k=1)
        if d.min() <= thresh:
            lo = mid
        else:
            hi = mid
    return hi


def sweep_pairs(lib: ShapeLibrary, n_pairs: int, seed: int,
                near_frac: float = 0.5, gap: float = 0.05,
                n_unique_near: int = 2048, world_extent: float = 4.0,
                sub: int = 512, touch: float = 0.01):
    """Returns (poses f32 [2n,7], obj_shape i32 [2n], pairs i32 [n,2],
    near mask bool [n])."""
    rng = np.random.default_rng(seed)
    n = int(n_pairs)
    n_near = int(round(n * near_frac))
    sa = rng.integers(0, lib.n_shapes, size=n).astype(np.int32)
    sb = rng.integers(0, lib.n_shapes, size=n).astype(np.int32)
    # world pose of A
    qa = random_quaternions(n, rng)
    ta = rng.uniform(-world_extent, world_extent, size=(n, 3))
    # relative pose of B in A's frame: uniform for the far half
    rel = random_poses(n, rng).astype(np.float64)
    near = np.zeros(n, bool)
    near[:n_near] = True
    rng.shuffle(near)
    idx_near = np.nonzero(near)[0]
    if len(idx_near):
        k = min(n_unique_near, len(idx_near))
        base = []  # (shapeA, shapeB, q_rel, u, s_touch)
        for j in range(k):
            a_s, b_s = int(sa[idx_near[j]]), int(sb[idx_near[j]])
            q = random_quaternions(1, rng)[0]
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            pa = lib.points[a_s].astype(np.float64)
            pb = lib.points[b_s].astype(np.float64) @ _quat_to_matrix64(q).T
            sel_a = rng.choice(len(pa), size=min(sub, len(pa)), replace=False)
            sel_b = rng.choice(len(pb), size=min(sub, len(pb)), replace=False)
            s0 = _touching_distance(pa[sel_a], cKDTree(pa[sel_a]), pb[sel_b], u,
                                    touch)
            base.append((a_s, b_s, q, u, s0))
        for j, i in enumerate(idx_near):
            a_s, b_s, q, u, s0 = base[j % k]
            sa[i], sb[i] = a_s, b_s
            g = rng.uniform(-gap, gap)
            rel[i, :4] = q
            rel[i, 4:] = (s0 + g) * u
    # compose world pose of B = A o rel
    qb = quat_multiply(qa, rel[:, :4])
    qb /= np.linalg.norm(qb, axis=1, keepdims=True)
    tb = np.empty((n, 3))
    for i in range(n):
        tb[i] = _quat_to_matrix64(qa[i]) @ rel[i, 4:] + ta[i]
    poses = np.empty((2 * n, 7), np.float32)
    poses[0::2, :4] = qa
    poses[0::2, 4:] = ta
    poses[1::2, :4] = qb
    poses[1::2, 4:] = tb
    obj_shape = np.empty(2 * n, np.int32)
    obj_shape[0::2] = sa
    obj_shape[1::2] = sb
    pairs = np.stack([np.arange(0, 2 * n, 2), np.arange(1, 2 * n, 2)],
                     axis=1).astype(np.int32)
    return poses, obj_shape, pairs, near


def client_batch(n_shapes: int, n_env: int, n_pairs: int, seed: int,
                 lam: float = 8.0, extent: float = 1.0):
    """A simulator client's contact-query batch: ``n_env`` environments of
    Poisson(lam) objects (clipped to [2, 25]) at uniform poses in
    [-extent, extent]^3, and ``n_pairs`` candidate pairs, each two distinct
    objects of one uniformly drawn environment.  Returns (poses f32 [n_obj,7],
    obj_shape i32 [n_obj], pairs i32 [n_pairs,2])."""
    rng = np.random.default_rng(seed)
    poses, obj_shape, off = uneven_scene(n_env, n_shapes, int(rng.integers(1 << 30)), lam,
                                         n_min=2, n_max=25, extent=extent)
    e = rng.integers(0, n_env, size=n_pairs)
    k = (off[e + 1] - off[e]).astype(np.int64)
    a = rng.integers(0, k)
    b = (a + 1 + rng.integers(0, k - 1)) % k
    pairs = np.stack([off[e] + a, off[e] + b], axis=1).astype(np.int32)
    return poses, obj_shape, pairs
