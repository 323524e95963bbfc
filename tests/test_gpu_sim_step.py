"""The device contact-resolution step (locc_sim_step) against its float64
oracle (oracle/sim.py): poses and velocities element by element after each of
several steps, every step started from the same state on both sides.  The
scene mixes objects resting in or above the plane, turned boxes, contacts with
and without penetration, separated rows (logit <= 0), repeated objects (forces
summed by atomics on the device) and invalid object indices."""

import numpy as np
import pytest

import synth
from oracle import sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRM = dict(dt=1 / 240, gravity=9.81, k_contact=2e4, c_contact=100.0, k_plane=2e4,
           c_plane=100.0, mu_plane=2.0, lin_damp=0.5, ang_damp=1.0)


def _scene(lib, n_obj, n_pairs, rng):
    q = synth.random_quaternions(n_obj, rng)
    poses = np.zeros((n_obj, 7), np.float32)
    poses[:, :4] = q
    poses[:, 4:6] = rng.uniform(-2, 2, (n_obj, 2))
    poses[:, 6] = rng.uniform(0.3, 1.5, n_obj)  # some body boxes dip into the plane
    vel = rng.normal(0, 0.8, (n_obj, 6)).astype(np.float32)
    osh = rng.integers(0, lib.n_shapes, n_obj).astype(np.int32)
    pairs = rng.integers(0, n_obj, (n_pairs, 2)).astype(np.int32)
    pairs[:3, 1] = n_obj + 5  # invalid index: ignored
    rows = np.zeros((n_pairs, 8), np.float32)
    rows[:, 0] = rng.normal(0.5, 1.0, n_pairs)  # about a third separated
    mid = 0.5 * (poses[pairs[:, 0] % n_obj, 4:] + poses[pairs[:, 1] % n_obj, 4:])
    rows[:, 1:4] = mid + rng.normal(0, 0.05, (n_pairs, 3))
    nrm = rng.normal(size=(n_pairs, 3))
    rows[:, 4:7] = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    rows[:, 7] = rng.uniform(-0.05, 0.03, n_pairs)
    return poses, vel, osh, pairs, rows


def test_sim_step_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_09439_b300 import Detector, simulate
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    lib = synth.make_library(16, 3)
    rng = np.random.default_rng(21)
    n_obj, n_pairs = 300, 400
    poses, vel, osh, pairs, rows = _scene(lib, n_obj, n_pairs, rng)
    prm = simulate.default_params()
    for k, v in PRM.items():
        assert abs(getattr(prm, k) - v) <= 1e-6 * abs(v), k
    layers = synth.xavier_weights(1)
    with Detector(lib.points, lib.aabb, layers, 0.25, "fp32") as det:
        tq = torch.from_numpy(pairs).to(dev)
        tr = torch.from_numpy(rows).to(dev)
        ts = torch.from_numpy(osh).to(dev)
        acc = torch.zeros((n_obj, 6), dtype=torch.float32, device=dev)
        for step in range(6):
            tp = torch.from_numpy(poses).to(dev)
            tv = torch.from_numpy(vel).to(dev)
            det.sim_step(prm, tp, tv, ts, tq, None, tr, acc)
            det.status()
            gp, gv = tp.cpu().numpy(), tv.cpu().numpy()
            op, ov = sim.step(PRM, poses, vel, osh, lib.aabb, pairs, rows)
            # float32 on the device (contraction, summation order of the
            # per-object force atomics) against float64, relative to the
            # largest velocity component of the object (terms of that size
            # cancel in its update); a velocity error moves the pose by dt
            # times itself.  A corner within rounding of the plane is decided
            # differently in float32 and float64, and the plane's damping force
            # jumps there: such objects are left out (a handful)
            edge = np.any(np.abs(_corner_z(lib, poses, osh)) < 1e-4, axis=1)
            assert edge.sum() <= 3
            keep = ~edge
            tol_v = 5e-5 + 1e-4 * np.abs(ov).max(axis=1, keepdims=True)
            tol_p = 2e-6 + 2e-6 * np.abs(op)
            tol_p[:, 4:] += PRM["dt"] * tol_v
            tol_p[:, :4] += PRM["dt"] * tol_v
            np.testing.assert_array_less(np.abs(gv - ov)[keep], tol_v.repeat(6, 1)[keep])
            np.testing.assert_array_less(np.abs(gp - op)[keep], tol_p[keep])
            assert np.all(acc.cpu().numpy() == 0)  # scratch left zero
            # next step from the device's state (both sides start equal)
            poses, vel = gp, gv
            rows[:, 0] = rng.normal(0.5, 1.0, n_pairs).astype(np.float32)
            tr = torch.from_numpy(rows).to(dev)
        assert np.sum(_lowest_corner(lib, poses, osh) < 0) > 10  # the plane was in play


def _corner_z(lib, poses, osh):
    """World z of the eight body-box corners of each object [n][8]."""
    out = np.empty((len(poses), 8))
    for i in range(len(poses)):
        lo, hi = lib.aabb[osh[i], :3], lib.aabb[osh[i], 3:]
        corners = np.array([[(hi if c & 1 else lo)[0], (hi if c & 2 else lo)[1],
                             (hi if c & 4 else lo)[2]] for c in range(8)], np.float64)
        out[i] = (corners @ sim.rotation(poses[i, :4]).T)[:, 2] + poses[i, 6]
    return out


def _lowest_corner(lib, poses, osh):
    return _corner_z(lib, poses, osh).min(axis=1)
