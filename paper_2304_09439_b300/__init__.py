"""B300-native local-crop contact detection (LOCC, Son & Kim, RSS 2023).

The compute path lives in the sm_103a library ``liblocc.so`` behind the C ABI
of ``include/locc.h``; this package is its thin Python binding.  PyTorch is
used only for device memory and streams.

    det = Detector(points, aabb, weights, radius=0.25, precision="bf16")
    out = det.detect(poses, obj_shape, pairs)   # [P, 8] on the device
"""

from __future__ import annotations

import ctypes
from typing import Optional

from . import abi, weights
from .abi import LoccError, LOCC_FP32, LOCC_BF16, LOCC_FP8, PRECISIONS

KMAX = 64
OUT_DIM = 8

__all__ = ["Detector", "VoxelDetector", "GJK", "Trainer", "Server", "Stepper", "LoccError", "LOCC_FP32", "LOCC_BF16", "LOCC_FP8", "weights",
           "abi", "KMAX", "OUT_DIM"]


def _prec(p) -> int:
    if isinstance(p, str):
        return PRECISIONS[p.lower()]
    return int(p)


def _need(t, dtype, name, device=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, detector on cuda:{device}")


class Detector:
    """Owns one ``locc_handle`` on the current CUDA device."""

    def __init__(self, points, aabb, layers, radius: float = 0.25, precision="fp32"):
        import torch
        self._lib = abi.load()
        self.device = torch.cuda.current_device()
        blob = layers if isinstance(layers, (bytes, bytearray)) else weights.pack(layers)
        self._h = abi.create(points, aabb, bytes(blob), radius, _prec(precision))
        self.radius = float(radius)
        self.precision = _prec(precision)

    # -- lifetime ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.locc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration ----------------------------------------------------
    def set_precision(self, precision) -> None:
        abi.check(self._lib.locc_set_precision(self._h, _prec(precision)))
        self.precision = _prec(precision)

    def set_crop_mode(self, mode: str) -> None:
        """"local" (the method) or "global" (each object's first 64 samples)."""
        abi.check(self._lib.locc_set_crop_mode(self._h, abi.CROP_MODES[mode]))

    def reserve(self, max_pairs: int, max_envs: int = 0) -> None:
        abi.check(self._lib.locc_reserve(self._h, int(max_pairs), int(max_envs)))

    def profile(self, enable: bool = True) -> None:
        abi.check(self._lib.locc_profile(self._h, int(bool(enable))))

    def set_pipeline(self, n_chunks: int, crop_ctas_per_sm: int = 0) -> None:
        abi.check(self._lib.locc_set_pipeline(self._h, int(n_chunks), int(crop_ctas_per_sm)))

    def autotune(self, poses, obj_shape, env_offsets, max_pairs: int, reps: int = 3,
                 pairs_out=None, n_pairs_out=None, out=None, stream=None):
        """Pick the fastest pipelining setting for these step inputs; returns
        ((n_chunks, crop_ctas_per_sm), ms per step).  n_chunks 0 is the fused
        crop + encoder launch (BF16), crop_ctas_per_sm then its crop warps per
        CTA."""
        import numpy as np
        import torch
        dev = poses.device
        M = int(max_pairs)
        if pairs_out is None:
            pairs_out = torch.empty((max(M, 1), 2), dtype=torch.int32, device=dev)
        if n_pairs_out is None:
            n_pairs_out = torch.zeros(1, dtype=torch.int32, device=dev)
        if out is None:
            out = torch.empty((max(M, 1), OUT_DIM), dtype=torch.float32, device=dev)
        best = np.zeros(2, np.int32)
        ms = np.zeros(1, np.float32)
        abi.check(self._lib.locc_autotune(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                          poses.shape[0], abi.ptr(env_offsets),
                                          env_offsets.shape[0] - 1, abi.ptr(pairs_out),
                                          abi.ptr(n_pairs_out), M, abi.ptr(out), int(reps),
                                          abi.ptr(best), abi.ptr(ms), abi.stream_ptr(stream)))
        return (int(best[0]), int(best[1])), float(ms[0])

    def stage_times(self):
        """Durations (ms) of the last call's stages: broadphase, crop, encoder,
        head (each summed over pipeline chunks), whole call."""
        import numpy as np
        ms = np.zeros(5, np.float32)
        n = self._lib.locc_stage_times(self._h, abi.ptr(ms), 5)
        if n < 0:
            abi.check(n)
        return ms[:n]

    def status(self, stream=None) -> None:
        """Wait for the stream; raise if a kernel flagged a bad index or a
        bounded device wait ran out."""
        abi.check(self._lib.locc_status(self._h, abi.stream_ptr(stream)))

    def selftest_wait_timeout(self, max_cycles: int = 1_000_000, stream=None) -> None:
        """Test hook: one CTA waits (bounded) on an mbarrier nothing completes
        and takes the kernels' timeout path; the next ``status`` raises
        ``LoccError`` with code -4 (TIMEOUT)."""
        abi.check(self._lib.locc_selftest_wait_timeout(self._h, int(max_cycles),
                                                       abi.stream_ptr(stream)))

    # -- the path -----------------------------------------------------------
    def detect(self, poses, obj_shape, pairs, out=None, stream=None):
        import torch
        _need(poses, torch.float32, "poses", self.device)
        _need(obj_shape, torch.int32, "obj_shape", self.device)
        _need(pairs, torch.int32, "pairs", self.device)
        P = pairs.shape[0]
        if out is None:
            out = torch.empty((P, OUT_DIM), dtype=torch.float32, device=pairs.device)
        _need(out, torch.float32, "out", self.device)
        abi.check(self._lib.locc_detect(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                        poses.shape[0], abi.ptr(pairs), P, abi.ptr(out),
                                        abi.stream_ptr(stream)))
        return out

    def detect_host(self, poses, obj_shape, pairs, out=None, stream=None):
        """Host (numpy) arrays in and out; copies and waits inside the call."""
        import numpy as np
        poses = np.ascontiguousarray(poses, np.float32)
        obj_shape = np.ascontiguousarray(obj_shape, np.int32)
        pairs = np.ascontiguousarray(pairs, np.int32)
        P = pairs.shape[0]
        if out is None:
            out = np.empty((P, OUT_DIM), np.float32)
        abi.check(self._lib.locc_detect_host(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                             poses.shape[0], abi.ptr(pairs), P, abi.ptr(out),
                                             abi.stream_ptr(stream)))
        return out

    def crop(self, poses, obj_shape, pairs, with_idx=True, stream=None):
        import torch
        _need(poses, torch.float32, "poses", self.device)
        _need(obj_shape, torch.int32, "obj_shape", self.device)
        _need(pairs, torch.int32, "pairs", self.device)
        P = pairs.shape[0]
        dev = pairs.device
        xyz = torch.empty((P, 2, KMAX, 4), dtype=torch.float32, device=dev)
        idx = torch.empty((P, 2, KMAX), dtype=torch.int32, device=dev) if with_idx else None
        cnt = torch.empty((P, 2), dtype=torch.int32, device=dev)
        centre = torch.empty((P, 4), dtype=torch.float32, device=dev)
        abi.check(self._lib.locc_crop(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                      poses.shape[0], abi.ptr(pairs), P, abi.ptr(xyz),
                                      abi.ptr(idx), abi.ptr(cnt), abi.ptr(centre),
                                      abi.stream_ptr(stream)))
        return dict(xyz=xyz, idx=idx, cnt=cnt, centre=centre)

    def network(self, xyz, with_feat=False, stream=None):
        import torch
        _need(xyz, torch.float32, "xyz", self.device)
        P = xyz.shape[0]
        y = torch.empty((P, OUT_DIM), dtype=torch.float32, device=xyz.device)
        f = torch.empty((P, 512), dtype=torch.float32, device=xyz.device) if with_feat else None
        abi.check(self._lib.locc_network(self._h, abi.ptr(xyz), P, abi.ptr(y), abi.ptr(f),
                                         abi.stream_ptr(stream)))
        return (y, f) if with_feat else y

    def broadphase(self, poses, obj_shape, env_offsets, max_pairs: int, pairs_out=None,
                   n_pairs_out=None, stream=None):
        import torch
        _need(poses, torch.float32, "poses", self.device)
        _need(obj_shape, torch.int32, "obj_shape", self.device)
        _need(env_offsets, torch.int32, "env_offsets", self.device)
        dev = poses.device
        if pairs_out is None:
            pairs_out = torch.empty((max(int(max_pairs), 1), 2), dtype=torch.int32, device=dev)
        if n_pairs_out is None:
            n_pairs_out = torch.zeros(1, dtype=torch.int32, device=dev)
        abi.check(self._lib.locc_broadphase(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                            abi.ptr(env_offsets), env_offsets.shape[0] - 1,
                                            abi.ptr(pairs_out), abi.ptr(n_pairs_out),
                                            int(max_pairs), abi.stream_ptr(stream)))
        return pairs_out, n_pairs_out

    def step(self, poses, obj_shape, env_offsets, max_pairs: int, pairs_out=None,
             n_pairs_out=None, out=None, stream=None):
        """Broadphase + detection on the device; returns (pairs, n_pairs, out)
        with the count left on the device."""
        import torch
        _need(poses, torch.float32, "poses", self.device)
        _need(obj_shape, torch.int32, "obj_shape", self.device)
        _need(env_offsets, torch.int32, "env_offsets", self.device)
        dev = poses.device
        M = int(max_pairs)
        if pairs_out is None:
            pairs_out = torch.empty((max(M, 1), 2), dtype=torch.int32, device=dev)
        if n_pairs_out is None:
            n_pairs_out = torch.zeros(1, dtype=torch.int32, device=dev)
        if out is None:
            out = torch.empty((max(M, 1), OUT_DIM), dtype=torch.float32, device=dev)
        abi.check(self._lib.locc_step(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                      poses.shape[0], abi.ptr(env_offsets),
                                      env_offsets.shape[0] - 1, abi.ptr(pairs_out),
                                      abi.ptr(n_pairs_out), M, abi.ptr(out),
                                      abi.stream_ptr(stream)))
        return pairs_out, n_pairs_out, out

    def sim_step(self, params, poses, vel, obj_shape, pairs, n_pairs_dev, contacts, acc,
                 stream=None):
        """One contact-resolution step of every object in place (poses, vel)
        from contact rows in the detector's output format."""
        import torch
        _need(poses, torch.float32, "poses", self.device)
        _need(vel, torch.float32, "vel", self.device)
        _need(obj_shape, torch.int32, "obj_shape", self.device)
        _need(acc, torch.float32, "acc", self.device)
        abi.check(self._lib.locc_sim_step(self._h, ctypes.byref(params), abi.ptr(poses),
                                          abi.ptr(vel), abi.ptr(obj_shape), poses.shape[0],
                                          abi.ptr(pairs), abi.ptr(n_pairs_dev), pairs.shape[0],
                                          abi.ptr(contacts), abi.ptr(acc),
                                          abi.stream_ptr(stream)))

    def sphere_contacts(self, poses, obj_shape, pairs, n_pairs_dev, radius, out, stream=None):
        """Bounding-sphere contact rows (a proxy-geometry contact source)."""
        abi.check(self._lib.locc_sphere_contacts(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                                 poses.shape[0], abi.ptr(pairs),
                                                 abi.ptr(n_pairs_dev), pairs.shape[0],
                                                 abi.ptr(radius), abi.ptr(out),
                                                 abi.stream_ptr(stream)))

    def step_host(self, poses, obj_shape, env_offsets, max_pairs: int, pairs_out=None,
                  out=None, stream=None):
        """Host arrays in and out; returns (pairs [n,2], out [n,8]) as numpy."""
        import numpy as np
        poses = np.ascontiguousarray(poses, np.float32)
        obj_shape = np.ascontiguousarray(obj_shape, np.int32)
        env_offsets = np.ascontiguousarray(env_offsets, np.int32)
        M = int(max_pairs)
        if pairs_out is None:
            pairs_out = np.empty((max(M, 1), 2), np.int32)
        if out is None:
            out = np.empty((max(M, 1), OUT_DIM), np.float32)
        n = np.zeros(1, np.int32)
        abi.check(self._lib.locc_step_host(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                           poses.shape[0], abi.ptr(env_offsets),
                                           env_offsets.shape[0] - 1, abi.ptr(pairs_out),
                                           abi.ptr(n), M, abi.ptr(out), abi.stream_ptr(stream)))
        m = min(int(n[0]), M)
        return pairs_out[:m], out[:m], int(n[0])


class Stepper:
    """Owns one ``locc_stepper`` on a Detector: host-buffer steps with up to
    ``depth`` in flight, their copies overlapping the neighbouring steps.

    ``submit`` takes page-locked numpy arrays (e.g. from
    ``torch.empty(..., pin_memory=True).numpy()``) and returns a ticket; the
    arrays must stay alive and the inputs unchanged until ``wait`` returns
    for it.  ``wait`` returns (pairs [n, 2], out [n, 8], n) as views of the
    caller's output arrays."""

    def __init__(self, det: "Detector", max_pairs: int, max_env: int, max_obj: int,
                 depth: int = 2):
        self._lib = abi.load()
        self.det = det
        self.max_pairs = int(max_pairs)
        self._t = ctypes.c_void_p()
        abi.check(self._lib.locc_stepper_create(det._h, self.max_pairs, int(max_env),
                                                int(max_obj), int(depth), ctypes.byref(self._t)))
        self._pending = {}

    def close(self) -> None:
        if getattr(self, "_t", None) is not None and self._t.value:
            self._lib.locc_stepper_destroy(self._t)
            self._t = None
            self._pending = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, poses, obj_shape, env_offsets, pairs_out, out) -> int:
        import numpy as np
        for name, a, dt in (("poses", poses, np.float32), ("obj_shape", obj_shape, np.int32),
                            ("env_offsets", env_offsets, np.int32),
                            ("pairs_out", pairs_out, np.int32), ("out", out, np.float32)):
            if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"{name} must be a C-contiguous {np.dtype(dt).name} array")
        if pairs_out.size < 2 * self.max_pairs or out.size < OUT_DIM * self.max_pairs:
            raise ValueError("pairs_out / out must hold max_pairs rows")
        n = np.zeros(1, np.int32)
        t = ctypes.c_int64(-1)
        abi.check(self._lib.locc_stepper_submit(self._t, abi.ptr(poses), abi.ptr(obj_shape),
                                                poses.shape[0], abi.ptr(env_offsets),
                                                env_offsets.shape[0] - 1, abi.ptr(pairs_out),
                                                abi.ptr(n), abi.ptr(out), ctypes.byref(t)))
        # keep the arrays alive until the wait
        self._pending[int(t.value)] = (poses, obj_shape, env_offsets, pairs_out, out, n)
        return int(t.value)

    def wait(self, ticket: int):
        abi.check(self._lib.locc_stepper_wait(self._t, int(ticket)))
        _, _, _, pairs_out, out, n = self._pending.pop(int(ticket))
        m = min(int(n[0]), self.max_pairs)
        return pairs_out.reshape(-1, 2)[:m], out.reshape(-1, OUT_DIM)[:m], int(n[0])


class VoxelDetector:
    """Owns one ``locc_voxel`` handle (the voxel-latent variant) on the current
    CUDA device: the library's latents are computed at construction."""

    def __init__(self, points, aabb, params):
        import torch
        self._lib = abi.load()
        self.device = torch.cuda.current_device()
        blob = params if isinstance(params, (bytes, bytearray)) else weights.pack_voxel(params)
        self._h = abi.voxel_create(points, aabb, bytes(blob))
        self.n_shapes = int(len(aabb))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.locc_voxel_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_precision(self, precision) -> None:
        """"fp32" (CUDA cores) or "bf16" (tcgen05) for the predictor."""
        abi.check(self._lib.locc_voxel_set_precision(self._h, _prec(precision)))

    def encode(self, stream=None) -> None:
        """Recompute the latents (asynchronous on ``stream``)."""
        abi.check(self._lib.locc_voxel_encode(self._h, abi.stream_ptr(stream)))

    def latents(self, stream=None):
        import torch
        out = torch.empty((self.n_shapes, 216, 16), dtype=torch.float32, device=self.device)
        abi.check(self._lib.locc_voxel_latents(self._h, abi.ptr(out), abi.stream_ptr(stream)))
        return out

    def detect(self, poses, obj_shape, pairs, logit=None, details=False, stream=None):
        """Logits [P] (and, with ``details``, cell ranges [P, 2, 6] and pooled
        features [P, 2, 16])."""
        import torch
        _need(poses, torch.float32, "poses", self.device)
        _need(obj_shape, torch.int32, "obj_shape", self.device)
        _need(pairs, torch.int32, "pairs", self.device)
        P = pairs.shape[0]
        if logit is None:
            logit = torch.empty(P, dtype=torch.float32, device=pairs.device)
        _need(logit, torch.float32, "logit", self.device)
        if not details:
            abi.check(self._lib.locc_voxel_detect(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                                  poses.shape[0], abi.ptr(pairs), P,
                                                  abi.ptr(logit), abi.stream_ptr(stream)))
            return logit
        ranges = torch.empty((P, 2, 6), dtype=torch.int32, device=pairs.device)
        pooled = torch.empty((P, 2, 16), dtype=torch.float32, device=pairs.device)
        abi.check(self._lib.locc_voxel_detect_ex(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                                 poses.shape[0], abi.ptr(pairs), P,
                                                 abi.ptr(logit), abi.ptr(ranges), abi.ptr(pooled),
                                                 abi.stream_ptr(stream)))
        return logit, ranges, pooled

    def status(self, stream=None) -> None:
        abi.check(self._lib.locc_voxel_status(self._h, abi.stream_ptr(stream)))


class GJK:
    """UCF-GJK comparator (``locc_gjk``): a convex decomposition on the current
    CUDA device; ``detect`` tests every pair with a fixed GJK iteration count."""

    def __init__(self, elem_off, vert_off, verts):
        import numpy as np
        import torch
        self._lib = abi.load()
        self.device = torch.cuda.current_device()
        eo = np.ascontiguousarray(elem_off, np.int32)
        vo = np.ascontiguousarray(vert_off, np.int32)
        vv = np.ascontiguousarray(verts, np.float32)
        self._h = ctypes.c_void_p()
        abi.check(self._lib.locc_gjk_create(len(eo) - 1, eo.ctypes.data, vo.ctypes.data,
                                            vv.ctypes.data, ctypes.byref(self._h)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.locc_gjk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def detect(self, poses, obj_shape, pairs, iterations: int, collide=None, stream=None):
        """uint8 [P] on the device: 1 collision, 0 none, 255 bad pair."""
        import torch
        _need(poses, torch.float32, "poses", self.device)
        _need(obj_shape, torch.int32, "obj_shape", self.device)
        _need(pairs, torch.int32, "pairs", self.device)
        P = pairs.shape[0]
        if collide is None:
            collide = torch.empty(P, dtype=torch.uint8, device=pairs.device)
        abi.check(self._lib.locc_gjk_detect(self._h, abi.ptr(poses), abi.ptr(obj_shape),
                                            poses.shape[0], abi.ptr(pairs), P, int(iterations),
                                            abi.ptr(collide), abi.stream_ptr(stream)))
        return collide

    def status(self, stream=None) -> None:
        abi.check(self._lib.locc_gjk_status(self._h, abi.stream_ptr(stream)))


class Trainer:
    """Owns one ``locc_trainer`` (GPU training of a Detector's network)."""

    def __init__(self, det: "Detector", max_batch: int, lr=1e-3, beta1=0.9, beta2=0.999,
                 eps=1e-8, w_pt=1.0, w_n=1.0, w_d=1.0, huber_beta=0.01, alpha=0.5, w_len=0.0,
                 precision: str = "fp32"):
        self._lib = abi.load()
        self.det = det
        self.max_batch = int(max_batch)
        cfg = abi.TrainConfig(lr, beta1, beta2, eps, w_pt, w_n, w_d, huber_beta, alpha, w_len)
        self._t = ctypes.c_void_p()
        abi.check(self._lib.locc_trainer_create(det._h, self.max_batch, ctypes.byref(cfg),
                                                ctypes.byref(self._t)))
        self.set_precision(precision)

    def set_precision(self, precision: str) -> None:
        """"fp32" (CUDA-core products) or "bf16" (tensor cores, bf16 operands,
        float32 accumulation and state) for the following steps."""
        if precision not in ("fp32", "bf16"):
            raise ValueError(f"training precision must be 'fp32' or 'bf16', not {precision!r}")
        abi.check(self._lib.locc_trainer_set_precision(self._t, abi.PRECISIONS[precision]))
        self.precision = precision

    def close(self) -> None:
        if getattr(self, "_t", None) is not None and self._t.value:
            self._lib.locc_trainer_destroy(self._t)
            self._t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, poses, obj_shape, pairs, targets, rot=None, update=True, loss_out=None,
             stream=None):
        """One step; returns the device scalar holding the batch's mean loss."""
        import torch
        dev = self.det.device
        _need(poses, torch.float32, "poses", dev)
        _need(obj_shape, torch.int32, "obj_shape", dev)
        _need(pairs, torch.int32, "pairs", dev)
        _need(targets, torch.float32, "targets", dev)
        if rot is not None:
            _need(rot, torch.float32, "rot", dev)
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float32, device=pairs.device)
        abi.check(self._lib.locc_train_step(self._t, abi.ptr(poses), abi.ptr(obj_shape),
                                            poses.shape[0], abi.ptr(pairs), pairs.shape[0],
                                            abi.ptr(targets), abi.ptr(rot), abi.ptr(loss_out),
                                            int(bool(update)), abi.stream_ptr(stream)))
        return loss_out

    def grad(self, stream=None):
        import torch
        g = torch.empty(weights.N_PARAMS, dtype=torch.float32, device=f"cuda:{self.det.device}")
        abi.check(self._lib.locc_trainer_grad(self._t, abi.ptr(g), abi.stream_ptr(stream)))
        return g

    def params(self, stream=None):
        import torch
        p = torch.empty(weights.N_PARAMS, dtype=torch.float32, device=f"cuda:{self.det.device}")
        abi.check(self._lib.locc_trainer_params(self._t, abi.ptr(p), abi.stream_ptr(stream)))
        return p

    def set_params(self, p, stream=None) -> None:
        import torch
        _need(p, torch.float32, "params", self.det.device)
        abi.check(self._lib.locc_trainer_set_params(self._t, abi.ptr(p), abi.stream_ptr(stream)))

    def state(self, stream=None):
        """Adam state for a checkpoint: (m, v) device tensors and the step count."""
        import torch
        m = torch.empty(weights.N_PARAMS, dtype=torch.float32, device=f"cuda:{self.det.device}")
        v = torch.empty_like(m)
        step = ctypes.c_int64(0)
        abi.check(self._lib.locc_trainer_get_state(self._t, abi.ptr(m), abi.ptr(v),
                                                   ctypes.byref(step), abi.stream_ptr(stream)))
        return m, v, int(step.value)

    def set_state(self, m, v, step: int, stream=None) -> None:
        """Restore Adam's moments and step count (from ``state``)."""
        import torch
        _need(m, torch.float32, "m", self.det.device)
        _need(v, torch.float32, "v", self.det.device)
        if m.numel() != weights.N_PARAMS or v.numel() != weights.N_PARAMS:
            raise ValueError(f"m and v need {weights.N_PARAMS} values")
        abi.check(self._lib.locc_trainer_set_state(self._t, abi.ptr(m), abi.ptr(v), int(step),
                                                   abi.stream_ptr(stream)))

    def set_lr(self, lr: float) -> None:
        """Learning rate of the following steps."""
        abi.check(self._lib.locc_trainer_set_lr(self._t, float(lr)))

    def commit(self) -> None:
        """Install the trained parameters as the detector's inference weights."""
        abi.check(self._lib.locc_trainer_commit(self._t))


class Server:
    """Owns one ``locc_server`` on a Detector (continuous batching of
    contact-query batches from many clients; see ``locc_server_*``).

    ``submit`` takes HOST numpy arrays (page-locked ones, e.g. from
    ``torch.empty(..., pin_memory=True).numpy()``, let the copies overlap) and
    keeps them alive until ``wait`` returns.  While the server exists it owns
    the detector's handle."""

    def __init__(self, det: Detector, arena_bytes: int = 0, max_batch_pairs: int = 131072,
                 max_active: int = 256, max_queued_pairs: int = 0, max_active_pairs: int = 0):
        self._lib = abi.load()
        self.det = det
        cfg = abi.ServerConfig(int(arena_bytes), int(max_batch_pairs), int(max_active),
                               int(max_queued_pairs), int(max_active_pairs))
        self._s = ctypes.c_void_p()
        abi.check(self._lib.locc_server_create(det._h, ctypes.byref(cfg), ctypes.byref(self._s)))
        self._keep = {}

    def close(self) -> None:
        if getattr(self, "_s", None) is not None and self._s.value:
            self._lib.locc_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, poses, obj_shape, pairs, out=None) -> int:
        """Queue a request; returns its id.  ``out`` (float32 [n_pairs, 8],
        host) receives the results; allocated when None (read it back with
        ``result``)."""
        import numpy as np
        poses = np.ascontiguousarray(poses, np.float32)
        obj_shape = np.ascontiguousarray(obj_shape, np.int32)
        pairs = np.ascontiguousarray(pairs, np.int32)
        if out is None:
            out = np.empty((pairs.shape[0], OUT_DIM), np.float32)
        if out.dtype != np.float32 or not out.flags.c_contiguous or \
                out.shape != (pairs.shape[0], OUT_DIM):
            raise ValueError("out must be a C-contiguous float32 [n_pairs, 8] array")
        rq = abi.Request(poses.ctypes.data, obj_shape.ctypes.data, poses.shape[0],
                         pairs.ctypes.data, pairs.shape[0], out.ctypes.data)
        rid = ctypes.c_int64()
        abi.check(self._lib.locc_server_submit(self._s, ctypes.byref(rq), ctypes.byref(rid)))
        self._keep[rid.value] = (poses, obj_shape, pairs, out)
        return rid.value

    def wait(self, rid: int, timeout_ms: int = -1) -> dict:
        """Block until request ``rid`` completes; returns its timeline
        (admit_us, done_us, launches) and output array."""
        info = abi.RequestInfo()
        code = self._lib.locc_server_wait(self._s, int(rid), int(timeout_ms), ctypes.byref(info))
        if code == -4:
            raise TimeoutError(f"request {rid} still running")
        keep = self._keep.pop(int(rid), None)
        abi.check(code)
        return {"admit_us": info.admit_us, "done_us": info.done_us, "launches": info.launches,
                "out": keep[3] if keep else None}

    def stats(self, reset: bool = False) -> dict:
        c = abi.ServerCounters()
        abi.check(self._lib.locc_server_stats(self._s, ctypes.byref(c), int(bool(reset))))
        return {name: getattr(c, name) for name, _ in abi.ServerCounters._fields_}
