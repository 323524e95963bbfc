"""Drop scenes: environments of two objects falling onto a plane.

Every environment holds two objects of a shape library that start above the
plane z = 0 at random orientations, spins and small horizontal offsets and
fall under gravity.  Poses advance with a minimal float32 penalty integrator
whose contacts are analytic -- the corners of each object's posed body box
against the plane, bounding spheres between the two objects -- so the poses
never depend on the contact detector under test.  The generator yields the
poses of every step; the detector sees about one candidate pair per
environment once the objects have landed.
"""

from __future__ import annotations

import numpy as np

from .poses import random_quaternions


def _rotate(q, v):
    """Rotate vectors v [n, k, 3] by unit quaternions q [n, 4] (w, x, y, z)."""
    w = q[:, None, 0:1]
    u = q[:, None, 1:4]
    t = 2.0 * np.cross(u, v)
    return v + w * t + np.cross(u, t)


def drop_scene(lib, n_env: int, n_steps: int, seed: int, dt: float = 1.0 / 240.0,
               g: float = 9.81, k_plane: float = 4000.0, k_obj: float = 2000.0,
               damping: float = 4.0):
    """Yields (step, poses f32 [2 n_env, 7], obj_shape i32 [2 n_env],
    env_offsets i32 [n_env + 1]) for steps 0 .. n_steps - 1."""
    rng = np.random.default_rng(seed)
    n = 2 * n_env
    shape = rng.integers(0, lib.n_shapes, size=n).astype(np.int32)
    lo, hi = lib.aabb[shape, :3].astype(np.float64), lib.aabb[shape, 3:].astype(np.float64)
    corners = np.stack([np.stack([np.where(b & 1, hi[:, 0], lo[:, 0]),
                                  np.where(b & 2, hi[:, 1], lo[:, 1]),
                                  np.where(b & 4, hi[:, 2], lo[:, 2])], 1)
                        for b in range(8)], 1)               # [n, 8, 3] body frame
    radius = np.linalg.norm(lib.points[shape], axis=2).max(axis=1).astype(np.float64)
    q = random_quaternions(n, rng).astype(np.float64)
    x = np.zeros((n, 3))
    x[:, 2] = 1.0 + rng.uniform(0.0, 0.5, n) + np.tile([0.0, 1.2], n_env)  # second one above
    x[:, :2] = rng.uniform(-0.3, 0.3, (n, 2))
    x[1::2, :2] = x[0::2, :2] + rng.uniform(-0.2, 0.2, (n_env, 2))
    v = np.zeros((n, 3))
    w = rng.normal(0.0, 2.0, (n, 3))
    env = np.arange(0, n + 1, 2, dtype=np.int32)
    for step in range(n_steps):
        poses = np.concatenate([q, x], 1).astype(np.float32)
        yield step, poses, shape, env
        f = np.zeros((n, 3))
        f[:, 2] -= g
        # plane: penalty on box corners below z = 0
        wc = _rotate(q, corners) + x[:, None, :]
        pen = np.maximum(-wc[:, :, 2], 0.0)
        f[:, 2] += k_plane * pen.sum(1) - damping * v[:, 2] * (pen.sum(1) > 0)
        # objects: bounding-sphere penalty within each environment
        d = x[1::2] - x[0::2]
        dist = np.linalg.norm(d, axis=1) + 1e-9
        over = np.maximum(radius[0::2] + radius[1::2] - dist, 0.0)
        push = (k_obj * over / dist)[:, None] * d
        f[0::2] -= push
        f[1::2] += push
        v = (v + dt * f) * (1.0 - 0.5 * dt)
        x = x + dt * v
        # spin: integrate the angular velocity into the quaternion
        w *= 1.0 - 0.5 * dt
        dq = np.concatenate([np.zeros((n, 1)), w], 1)
        qd = 0.5 * np.stack([
            dq[:, 0] * q[:, 0] - np.sum(dq[:, 1:] * q[:, 1:], 1),
            *(dq[:, 0:1] * q[:, 1:] + q[:, 0:1] * dq[:, 1:] + np.cross(dq[:, 1:], q[:, 1:])).T], 1)
        q = q + dt * qd
        q /= np.linalg.norm(q, axis=1, keepdims=True)


def drop_initial_state(lib, n_env: int, seed: int):
    """Initial state of drop scenes for a simulator driven by the detector:
    two objects per environment drawn from the library, the second 1.2 m above
    the first, random orientations and spins, small horizontal offsets (the
    same recipe as ``drop_scene``).  Returns poses float32 [2 n_env, 7],
    velocities float32 [2 n_env, 6] (linear, angular), obj_shape int32
    [2 n_env] and env_offsets int32 [n_env + 1]."""
    rng = np.random.default_rng(seed)
    n = 2 * n_env
    shape = rng.integers(0, lib.n_shapes, size=n).astype(np.int32)
    q = random_quaternions(n, rng).astype(np.float32)
    x = np.zeros((n, 3), np.float32)
    x[:, 2] = 1.0 + rng.uniform(0.0, 0.5, n) + np.tile([0.0, 1.2], n_env)
    x[:, :2] = rng.uniform(-0.3, 0.3, (n, 2))
    x[1::2, :2] = x[0::2, :2] + rng.uniform(-0.2, 0.2, (n_env, 2))
    vel = np.zeros((n, 6), np.float32)
    vel[:, 3:] = rng.normal(0.0, 2.0, (n, 3))
    poses = np.concatenate([q, x], 1).astype(np.float32)
    env = np.arange(0, n + 1, 2, dtype=np.int32)
    return poses, vel, shape, env
