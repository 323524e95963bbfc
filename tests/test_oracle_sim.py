"""Pins of the contact-resolution oracle (oracle/sim.py) from closed forms of
rigid-body mechanics: free fall, a box resting on the plane, equal and
opposite pair forces, the world inertia tensor of a turned box, the rotation
angle of the quaternion update, and the symmetry of swapping A and B."""

import math

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import sim

PRM = dict(dt=1 / 240, gravity=9.81, k_contact=2e4, c_contact=100.0, k_plane=2e4,
           c_plane=100.0, mu_plane=2.0, lin_damp=0.5, ang_damp=1.0)
CUBE = np.array([[-0.5, -0.5, -0.5, 0.5, 0.5, 0.5]])
NO_PAIRS = (np.zeros((0, 2), int), np.zeros((0, 8)))


def _ld(p):
    return 1 - p["lin_damp"] * p["dt"]


def _ad(p):
    return 1 - p["ang_damp"] * p["dt"]


def test_free_fall():
    poses = np.array([[1, 0, 0, 0, 0.3, -0.2, 5.0]])
    vel = np.zeros((1, 6))
    P, V = sim.step(PRM, poses, vel, [0], CUBE, *NO_PAIRS)
    vz = -PRM["gravity"] * PRM["dt"] * _ld(PRM)
    np.testing.assert_allclose(V[0], [0, 0, vz, 0, 0, 0], atol=1e-15)
    np.testing.assert_allclose(P[0], [1, 0, 0, 0, 0.3, -0.2, 5.0 + PRM["dt"] * vz], atol=1e-15)


def test_box_resting_in_the_plane():
    # a unit cube whose bottom face sits 1 mm below z = 0: four corners push
    # up with k pen each, their torques cancel; the friction term is zero at
    # rest
    pen = 1e-3
    poses = np.array([[1, 0, 0, 0, 0, 0, 0.5 - pen]])
    P, V = sim.step(PRM, poses, np.zeros((1, 6)), [0], CUBE, *NO_PAIRS)
    vz = PRM["dt"] * (4 * PRM["k_plane"] * pen - PRM["gravity"]) * _ld(PRM)
    np.testing.assert_allclose(V[0], [0, 0, vz, 0, 0, 0], atol=1e-12)
    np.testing.assert_allclose(P[0, :4], [1, 0, 0, 0], atol=1e-15)


def test_pair_forces_equal_and_opposite_with_torque():
    # two cubes far above the plane; a contact along +x at a point off the
    # centre line: B gets +F, A gets -F; torques r x F about each centre;
    # identity poses, unit cube inertia 1/6 -> angular acceleration 6 tau
    d, f_expect = 0.01, 2e4 * 0.01
    poses = np.array([[1, 0, 0, 0, 0, 0, 10.0], [1, 0, 0, 0, 0.99, 0, 10.0]])
    pt = np.array([0.495, 0.2, 10.1])
    row = np.array([[3.0, *pt, 1.0, 0.0, 0.0, d]])
    P, V = sim.step(PRM, poses, np.zeros((2, 6)), [0, 0], np.repeat(CUBE, 1, 0),
                    np.array([[0, 1]]), row)
    g = PRM["gravity"]
    F = np.array([f_expect, 0, 0])
    for i, sign in ((0, -1.0), (1, 1.0)):
        lin = (sign * F + np.array([0, 0, -g])) * PRM["dt"] * _ld(PRM)
        np.testing.assert_allclose(V[i, :3], lin, rtol=1e-12, atol=1e-14)
        tau = np.cross(pt - poses[i, 4:], sign * F)
        np.testing.assert_allclose(V[i, 3:], 6.0 * tau * PRM["dt"] * _ad(PRM), rtol=1e-12,
                                   atol=1e-14)
    # momentum: the pair forces cancel
    np.testing.assert_allclose(V[0, :3] + V[1, :3],
                               2 * np.array([0, 0, -g]) * PRM["dt"] * _ld(PRM), atol=1e-13)


def test_no_force_without_contact_and_damping_only_force():
    poses = np.array([[1, 0, 0, 0, 0, 0, 10.0], [1, 0, 0, 0, 1.2, 0, 10.0]])
    vel = np.zeros((2, 6))
    vel[1, 0] = -0.5  # B approaches A along -x
    base = sim.step(PRM, poses, vel, [0, 0], CUBE, *NO_PAIRS)
    # logit <= 0: ignored
    row = np.array([[-1.0, 0.6, 0, 10.0, 1, 0, 0, 0.2]])
    P, V = sim.step(PRM, poses, vel, [0, 0], CUBE, np.array([[0, 1]]), row)
    np.testing.assert_array_equal(V, base[1])
    # a contact with a gap (depth < 0 counts as 0) still damps the approach:
    # f = -c v_n = 100 * 0.5, at a point on the centre line (no torque)
    row[0, 0], row[0, 7] = 1.0, -0.05
    P, V = sim.step(PRM, poses, vel, [0, 0], CUBE, np.array([[0, 1]]), row)
    dv = (V - base[1])[:, :3] / (PRM["dt"] * _ld(PRM))
    np.testing.assert_allclose(dv[1], [50.0, 0, 0], rtol=1e-12)
    np.testing.assert_allclose(dv[0], [-50.0, 0, 0], rtol=1e-12)
    np.testing.assert_allclose(V[:, 3:], 0.0, atol=1e-15)


def test_world_inertia_of_a_turned_box():
    # a 1 x 2 x 3 box turned by a random rotation: the angular acceleration
    # from a contact torque solves I_world alpha = tau with
    # I_world = R diag((e_y^2 + e_z^2) / 12, ...) R^T
    aabb = np.array([[-0.5, -1.0, -1.5, 0.5, 1.0, 1.5], [-0.5, -0.5, -0.5, 0.5, 0.5, 0.5]])
    rot = Rotation.from_euler("xyz", [0.3, -1.1, 2.0])
    q = rot.as_quat()
    poses = np.array([[q[3], q[0], q[1], q[2], 0, 0, 20.0], [1, 0, 0, 0, 3.0, 0, 20.0]])
    pt = np.array([0.8, 0.4, 19.7])
    nrm = np.array([0.6, 0.0, 0.8])
    row = np.array([[1.0, *pt, *nrm, 0.02]])
    P, V = sim.step(PRM, poses, np.zeros((2, 6)), [0, 1], aabb, np.array([[0, 1]]), row)
    F = 2e4 * 0.02 * nrm
    tau = np.cross(pt - poses[0, 4:], -F)
    e = np.array([1.0, 2.0, 3.0])
    I_body = np.diag([(e[1] ** 2 + e[2] ** 2) / 12, (e[0] ** 2 + e[2] ** 2) / 12,
                      (e[0] ** 2 + e[1] ** 2) / 12])
    R = rot.as_matrix()
    alpha = np.linalg.solve(R @ I_body @ R.T, tau)
    np.testing.assert_allclose(V[0, 3:], alpha * PRM["dt"] * _ad(PRM), rtol=1e-10)


def test_quaternion_update_angle():
    # spin about z from the identity: q' = normalise(1, 0, 0, dt w / 2), a
    # rotation by 2 atan(dt w / 2) with w the damped rate
    w0 = 7.0
    poses = np.array([[1, 0, 0, 0, 0, 0, 10.0]])
    vel = np.array([[0, 0, 0, 0, 0, w0]])
    P, V = sim.step(PRM, poses, vel, [0], CUBE, *NO_PAIRS)
    w = w0 * _ad(PRM)
    ang = 2 * math.atan(PRM["dt"] * w / 2)
    np.testing.assert_allclose(P[0, :4], [math.cos(ang / 2), 0, 0, math.sin(ang / 2)], atol=1e-14)
    # the same update from a turned orientation composes on the left:
    # q' = normalise(q + dt/2 (0, w) q) = r q with r the rotation above
    q0 = Rotation.from_euler("xyz", [0.4, 0.1, -0.7]).as_quat()
    poses[0, :4] = [q0[3], q0[0], q0[1], q0[2]]
    P2, _ = sim.step(PRM, poses, vel, [0], CUBE, *NO_PAIRS)
    want = (Rotation.from_rotvec([0, 0, ang]) * Rotation.from_quat(q0)).as_quat()
    got = P2[0, [1, 2, 3, 0]]
    assert min(np.abs(got - want).max(), np.abs(got + want).max()) < 1e-13


def test_swapping_a_and_b_with_the_normal_flipped():
    rng = np.random.default_rng(3)
    q = Rotation.random(2, random_state=4).as_quat()
    poses = np.zeros((2, 7))
    poses[:, :4] = q[:, [3, 0, 1, 2]]
    poses[:, 4:] = [[0, 0, 0.4], [0.7, 0.1, 0.5]]
    vel = rng.normal(0, 0.5, (2, 6))
    aabb = np.array([[-0.4, -0.3, -0.2, 0.4, 0.3, 0.2], [-0.3, -0.3, -0.3, 0.3, 0.3, 0.3]])
    nrm = np.array([0.8, 0.0, 0.6])
    row = np.array([[2.0, 0.35, 0.05, 0.45, *nrm, 0.03]])
    P1, V1 = sim.step(PRM, poses, vel, [0, 1], aabb, np.array([[0, 1]]), row)
    row2 = row.copy()
    row2[0, 4:7] = -nrm
    P2, V2 = sim.step(PRM, poses, vel, [0, 1], aabb, np.array([[1, 0]]), row2)
    np.testing.assert_allclose(P1, P2, atol=1e-14)
    np.testing.assert_allclose(V1, V2, atol=1e-12)


def test_quaternion_update_about_a_general_axis():
    # q' = normalise((1, dt w / 2) q): a rotation by 2 atan(dt |w| / 2) about
    # w, composed on the left of the current orientation
    w0 = np.array([3.0, -2.0, 5.0])
    q0 = Rotation.from_euler("zyx", [1.0, -0.4, 0.3]).as_quat()
    poses = np.array([[q0[3], q0[0], q0[1], q0[2], 0, 0, 10.0]])
    vel = np.concatenate([[0.0, 0.0, 0.0], w0])[None]
    P, V = sim.step(PRM, poses, vel, [0], CUBE, *NO_PAIRS)
    w = w0 * _ad(PRM)
    ang = 2 * math.atan(PRM["dt"] * np.linalg.norm(w) / 2)
    want = (Rotation.from_rotvec(ang * w / np.linalg.norm(w)) * Rotation.from_quat(q0)).as_quat()
    got = P[0, [1, 2, 3, 0]]
    assert min(np.abs(got - want).max(), np.abs(got + want).max()) < 1e-13


def test_tilted_box_on_one_edge_turns_level():
    # a unit cube turned by +0.1 rad about x rests on its lower edge (two
    # corners, at y < 0, 1 mm into the plane): the upward corner forces give
    # a torque about -x (the box levels out); magnitude from the corner
    # positions computed with scipy's rotation
    th, pen = 0.1, 1e-3
    rot = Rotation.from_rotvec([th, 0, 0])
    corners = np.array([[x, y, z] for z in (-0.5, 0.5) for y in (-0.5, 0.5) for x in (-0.5, 0.5)])
    r = rot.apply(corners)
    zc = -r[:, 2].min() - pen  # centre height: the lowest corners at -pen
    q = rot.as_quat()
    poses = np.array([[q[3], q[0], q[1], q[2], 0, 0, zc]])
    P, V = sim.step(PRM, poses, np.zeros((1, 6)), [0], CUBE, *NO_PAIRS)
    low = r[:, 2] + zc < 0
    assert low.sum() == 2 and np.all(r[low, 1] < 0)
    f = PRM["k_plane"] * -(r[low, 2] + zc)
    tau_x = float(np.sum(r[low, 1] * f))
    assert tau_x < 0
    np.testing.assert_allclose(V[0, 3:], [6.0 * tau_x * PRM["dt"] * _ad(PRM), 0, 0], rtol=1e-10,
                               atol=1e-14)
