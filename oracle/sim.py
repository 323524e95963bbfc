"""Oracle of the contact-resolution step (test infrastructure only).

Plain float64 restatement of one rigid-body step driven by contact rows in
the detector's output format, for the drop-scene fidelity measurement
(Sec. IV-C: the contact network inside a GPU simulator; Table 2 measures
interpenetration whenever a contact arises).  The paper names its contact
solver only by reference, so the step is this library's reading, a penalty
method:

1. every pair contact {logit, point p, normal n (A towards B), depth d} with
   logit > 0 pushes B by F = max(0, k_c max(d, 0) - c_c v_n) n and A by -F,
   both applied at p, where v_n = (v_B(p) - v_A(p)) . n and
   v_X(p) = v_X + w_X x (p - x_X);
2. each corner of an object's body box below the plane z = 0 (depth
   pen = -z) adds the force (-mu v_x, -mu v_y, max(0, k_p pen - c_p v_z)) at
   the corner, v the corner's velocity;
3. gravity -g e_z on a unit mass;
4. torques about the object's centre, inertia of a solid unit-mass box
   filling the body AABB (principal moments (e_j^2 + e_k^2) / 12 in the body
   frame), world angular acceleration R I^-1 R^T T;
5. semi-implicit Euler: v += dt F, w += dt alpha, each damped by
   max(0, 1 - damping dt); x += dt v (new v); q += dt/2 (0, w) q, then q is
   normalised.

Only tests import this module; it shares no code with the CUDA path.
"""

from __future__ import annotations

import numpy as np


def rotation(q) -> np.ndarray:
    """Rotation matrix of the unit quaternion (w, x, y, z), body -> world."""
    w, x, y, z = (float(v) for v in q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def step(params: dict, poses, vel, obj_shape, aabb, pairs, contacts):
    """One step.  params: dict with dt, gravity, k_contact, c_contact, k_plane,
    c_plane, mu_plane, lin_damp, ang_damp.  poses [n][7] (w, x, y, z, t),
    vel [n][6] (linear, angular, world), obj_shape [n], aabb [S][6] (lo, hi),
    pairs [m][2], contacts [m][8].  Returns new (poses, vel) as float64."""
    P = np.asarray(poses, np.float64).copy()
    V = np.asarray(vel, np.float64).copy()
    n = len(P)
    force = np.zeros((n, 3))
    torque = np.zeros((n, 3))
    # 1. pair contacts
    for (a, b), row in zip(np.asarray(pairs), np.asarray(contacts, np.float64)):
        if not row[0] > 0 or not (0 <= a < n and 0 <= b < n):
            continue
        d = max(row[7], 0.0)
        p, nrm = row[1:4], row[4:7]
        rA, rB = p - P[a, 4:], p - P[b, 4:]
        vA = V[a, :3] + np.cross(V[a, 3:], rA)
        vB = V[b, :3] + np.cross(V[b, 3:], rB)
        vn = float(np.dot(vB - vA, nrm))
        f = max(params["k_contact"] * d - params["c_contact"] * vn, 0.0)
        if f == 0.0:
            continue
        F = f * nrm
        force[b] += F
        torque[b] += np.cross(rB, F)
        force[a] -= F
        torque[a] -= np.cross(rA, F)
    dt = params["dt"]
    for i in range(n):
        s = int(obj_shape[i])
        if not 0 <= s < len(aabb):
            continue
        lo, hi = np.asarray(aabb[s][:3], np.float64), np.asarray(aabb[s][3:], np.float64)
        R = rotation(P[i, :4])
        F, T = force[i].copy(), torque[i].copy()
        # 2. ground plane at the body-box corners
        for c in range(8):
            corner = np.array([hi[0] if c & 1 else lo[0], hi[1] if c & 2 else lo[1],
                               hi[2] if c & 4 else lo[2]])
            r = R @ corner
            z = r[2] + P[i, 6]
            if z >= 0.0:
                continue
            vc = V[i, :3] + np.cross(V[i, 3:], r)
            fz = max(params["k_plane"] * (-z) - params["c_plane"] * vc[2], 0.0)
            fc = np.array([-params["mu_plane"] * vc[0], -params["mu_plane"] * vc[1], fz])
            F += fc
            T += np.cross(r, fc)
        # 3. gravity on a unit mass
        F[2] -= params["gravity"]
        # 4. inertia of a solid unit-mass box
        e = hi - lo
        inv_I = np.array([12.0 / max(e[1] ** 2 + e[2] ** 2, 1e-12),
                          12.0 / max(e[0] ** 2 + e[2] ** 2, 1e-12),
                          12.0 / max(e[0] ** 2 + e[1] ** 2, 1e-12)])
        alpha = R @ (inv_I * (R.T @ T))
        # 5. semi-implicit Euler with damping
        ld = max(1.0 - params["lin_damp"] * dt, 0.0)
        ad = max(1.0 - params["ang_damp"] * dt, 0.0)
        V[i, :3] = (V[i, :3] + dt * F) * ld
        V[i, 3:] = (V[i, 3:] + dt * alpha) * ad
        P[i, 4:] = P[i, 4:] + dt * V[i, :3]
        w, x, y, z = P[i, :4]
        ox, oy, oz = V[i, 3:]
        # (0, w) q, quaternion product
        dq = np.array([-ox * x - oy * y - oz * z,
                       ox * w + oy * z - oz * y,
                       oy * w + oz * x - ox * z,
                       oz * w + ox * y - oy * x])
        q = P[i, :4] + 0.5 * dt * dq
        P[i, :4] = q / np.linalg.norm(q)
    return P, V
