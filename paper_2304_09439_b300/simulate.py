"""Drop simulations whose object-object contacts come from the detector.

Every step runs on the device: the AABB broadphase and the contact network
(``locc_step``), optionally a proxy contact source in its place
(``locc_sphere_contacts``), then the contact-resolution step
(``locc_sim_step``).  The harness keeps the poses, pairs and contact rows of
every step on the device and returns them at the end, so that the contacts a
run produced can be examined afterwards (e.g. their true signed distances).
"""

from __future__ import annotations

from . import abi


def default_params(dt: float = 1.0 / 240.0) -> "abi.SimParams":
    """Penalty parameters for objects of about 1 m at 240 Hz (unit masses):
    contact stiffness 2e4 N/m (a body landing at 5 m/s sinks about 3.5 cm
    before the spring stops it; sqrt(k/m) dt = 0.59 keeps the explicit step
    stable), damping 100 N s/m."""
    return abi.SimParams(dt=dt, gravity=9.81, k_contact=20000.0, c_contact=100.0,
                         k_plane=20000.0, c_plane=100.0, mu_plane=2.0, lin_damp=0.5,
                         ang_damp=1.0)


def run_drop(det, poses, vel, obj_shape, env_offsets, n_steps: int, params=None,
             source: str = "locc", radius=None, max_pairs=None, stream=None):
    """Simulate ``n_steps`` steps in place on the device.

    poses float32 [n, 7], vel float32 [n, 6], obj_shape int32 [n],
    env_offsets int32 [n_env + 1] (device tensors); ``source`` is "locc"
    (the detector's contacts) or "sphere" (bounding spheres of ``radius``
    [n_shapes] device float32).  Returns host arrays: poses [T, n, 7] (the
    poses each step's contacts were computed from), pairs [T, M, 2],
    contacts [T, M, 8], n_pairs [T]."""
    import torch
    if source not in ("locc", "sphere"):
        raise ValueError("source must be 'locc' or 'sphere'")
    if source == "sphere" and radius is None:
        raise ValueError("the sphere source needs radii")
    dev = poses.device
    n_obj = poses.shape[0]
    n_env = env_offsets.shape[0] - 1
    M = int(max_pairs if max_pairs is not None else max(n_env, 1))
    params = params or default_params()
    pairs = torch.zeros((M, 2), dtype=torch.int32, device=dev)
    n_dev = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.zeros((M, 8), dtype=torch.float32, device=dev)
    acc = torch.zeros((n_obj, 6), dtype=torch.float32, device=dev)
    h_poses = torch.empty((n_steps, n_obj, 7), dtype=torch.float32, device=dev)
    h_pairs = torch.empty((n_steps, M, 2), dtype=torch.int32, device=dev)
    h_out = torch.empty((n_steps, M, 8), dtype=torch.float32, device=dev)
    h_n = torch.empty(n_steps, dtype=torch.int32, device=dev)
    for t in range(n_steps):
        h_poses[t].copy_(poses)
        det.step(poses, obj_shape, env_offsets, M, pairs_out=pairs, n_pairs_out=n_dev, out=out,
                 stream=stream)
        if source == "sphere":
            det.sphere_contacts(poses, obj_shape, pairs, n_dev, radius, out, stream=stream)
        h_pairs[t].copy_(pairs)
        h_out[t].copy_(out)
        h_n[t] = n_dev[0]
        det.sim_step(params, poses, vel, obj_shape, pairs, n_dev, out, acc, stream=stream)
    det.status(stream)
    return {"poses": h_poses.cpu().numpy(), "pairs": h_pairs.cpu().numpy(),
            "contacts": h_out.cpu().numpy(), "n_pairs": h_n.cpu().numpy()}
