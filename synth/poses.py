"""Uniformly random rigid poses.

A pose is 7 float32 numbers (w, x, y, z, tx, ty, tz): a unit quaternion in
(w, x, y, z) order followed by a translation; the body-to-world map is
p_world = R(q) p_body + t.  Rotations are drawn uniformly on SO(3) with
Shoemake's method (Graphics Gems III, "Uniform random rotations").
"""

from __future__ import annotations

import numpy as np


def random_quaternions(n: int, rng: np.random.Generator) -> np.ndarray:
    """n uniform unit quaternions, float64 [n, 4] in (w, x, y, z) order."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    return np.stack([w, x, y, z], axis=1)


def random_poses(n: int, rng: np.random.Generator, lo: float = -1.5,
                 hi: float = 1.5) -> np.ndarray:
    """n poses: uniform SO(3) rotation, translation uniform in [lo, hi]^3."""
    q = random_quaternions(n, rng)
    t = rng.uniform(lo, hi, size=(n, 3))
    return np.concatenate([q, t], axis=1).astype(np.float32)


def quat_multiply(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product a * b for (w, x, y, z) quaternions (float64)."""
    aw, ax, ay, az = np.moveaxis(np.asarray(a, np.float64), -1, 0)
    bw, bx, by, bz = np.moveaxis(np.asarray(b, np.float64), -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def compose_relative_tiny(n: int = 256, seed: int = 0):
    """The tiny case: object A (shape 0) at the identity, object B (shape 1)
    at n uniform relative poses; returns (poses [2n,7], obj_shape [2n],
    pairs [n,2])."""
    rng = np.random.default_rng(seed)
    rel = random_poses(n, rng)
    ident = np.zeros((n, 7), np.float32)
    ident[:, 0] = 1.0
    poses = np.empty((2 * n, 7), np.float32)
    poses[0::2] = ident
    poses[1::2] = rel
    obj_shape = np.tile(np.array([0, 1], np.int32), n)
    pairs = np.stack([np.arange(0, 2 * n, 2), np.arange(1, 2 * n, 2)],
                     axis=1).astype(np.int32)
    return poses, obj_shape, pairs
