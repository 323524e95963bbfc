"""ctypes binding of the C ABI in ``include/locc.h`` (argument marshalling only).

Every step of the contact path runs in ``liblocc.so``; this module converts
PyTorch tensors to device pointers and return codes to exceptions.  There is no
other implementation behind it: if the library cannot be loaded, importing the
package still works but every call raises ``LoccError``.
"""

from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

from . import build as _build

LOCC_FP32, LOCC_BF16, LOCC_FP8 = 0, 1, 2
CROP_MODES = {"local": 0, "global": 1}
PRECISIONS = {"fp32": LOCC_FP32, "bf16": LOCC_BF16, "fp8": LOCC_FP8}
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT",
          -5: "BAD_WEIGHTS", -6: "BAD_INDEX", -7: "BUSY"}

# every symbol include/locc.h declares
EXPORTS = ["locc_create", "locc_set_precision", "locc_detect", "locc_detect_host",
           "locc_crop", "locc_network", "locc_broadphase", "locc_step", "locc_step_host",
           "locc_reserve", "locc_profile", "locc_stage_times", "locc_status", "locc_destroy",
           "locc_last_error", "locc_detect_noalloc", "locc_trainer_create", "locc_train_step",
           "locc_trainer_grad", "locc_trainer_params", "locc_trainer_set_params",
           "locc_trainer_commit", "locc_trainer_set_lr", "locc_trainer_destroy", "locc_set_pipeline",
           "locc_autotune", "locc_server_create", "locc_server_submit", "locc_server_wait",
           "locc_server_stats", "locc_server_destroy", "locc_voxel_create", "locc_voxel_encode",
           "locc_voxel_latents", "locc_voxel_detect", "locc_voxel_detect_ex", "locc_voxel_status",
           "locc_voxel_set_precision",
           "locc_voxel_destroy", "locc_sim_step", "locc_sphere_contacts", "locc_set_crop_mode",
           "locc_gjk_create", "locc_gjk_detect", "locc_gjk_status", "locc_gjk_destroy",
           "locc_selftest_wait_timeout", "locc_trainer_get_state", "locc_trainer_set_state",
           "locc_trainer_set_precision", "locc_stepper_create", "locc_stepper_submit",
           "locc_stepper_wait", "locc_stepper_destroy"]
VOID_EXPORTS = ("locc_destroy", "locc_last_error", "locc_trainer_destroy", "locc_server_destroy",
                "locc_voxel_destroy", "locc_gjk_destroy", "locc_stepper_destroy")


def _header_define(name: str) -> int:
    """Integer value of a #define in include/locc.h (the header is the one
    place such a limit is written down)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "include", "locc.h")
    with open(hdr) as f:
        m = re.search(rf"^#define\s+{name}\s+(\d+)\s*$", f.read(), re.M)
    if not m:
        raise RuntimeError(f"{name} not found in {hdr}")
    return int(m.group(1))


NOALLOC_MAX_PAIRS = _header_define("LOCC_NOALLOC_MAX_PAIRS")


class LoccError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"locc error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class TrainConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("lr", "beta1", "beta2", "eps", "w_pt", "w_n", "w_d", "huber_beta", "alpha",
                 "w_len")]


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_int64), ("max_batch_pairs", ctypes.c_int32),
                ("max_active", ctypes.c_int32), ("max_queued_pairs", ctypes.c_int64),
                ("max_active_pairs", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("poses", ctypes.c_void_p), ("obj_shape", ctypes.c_void_p),
                ("n_obj", ctypes.c_int32), ("pairs", ctypes.c_void_p),
                ("n_pairs", ctypes.c_int32), ("out", ctypes.c_void_p)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("admit_us", ctypes.c_double), ("done_us", ctypes.c_double),
                ("launches", ctypes.c_int32), ("status", ctypes.c_int32)]


class ServerCounters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("submitted", "rejected", "completed", "failed", "queued", "active",
                 "pairs_completed", "launches", "arena_bytes", "arena_used", "arena_peak")] + \
               [(n, ctypes.c_double) for n in
                ("latency_p50_us", "latency_p99_us", "latency_max_us", "mean_pairs_per_launch")] + \
               [("max_active_seen", ctypes.c_int32)]


class SimParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("dt", "gravity", "k_contact", "c_contact", "k_plane", "c_plane", "mu_plane",
                 "lin_damp", "ang_damp")]


class _ShapeLibrary(ctypes.Structure):
    _fields_ = [("n_shapes", ctypes.c_int32), ("n_points", ctypes.c_int32),
                ("points", ctypes.c_void_p), ("aabb", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load liblocc.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.SO_PATH
        if build_if_needed and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise LoccError(-3, f"{path} is missing; build it with "
                                "`python -m paper_2304_09439_b300.build`")
        lib = ctypes.CDLL(path)
        P, I, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_float
        lib.locc_create.argtypes = [ctypes.POINTER(_ShapeLibrary), P, ctypes.c_size_t, F,
                                    ctypes.c_int, ctypes.POINTER(P)]
        lib.locc_set_precision.argtypes = [P, ctypes.c_int]
        lib.locc_detect.argtypes = [P, P, P, I, P, I, P, P]
        lib.locc_detect_host.argtypes = [P, P, P, I, P, I, P, P]
        lib.locc_detect_noalloc.argtypes = [P, P, P, I, P, I, P, P]
        lib.locc_crop.argtypes = [P, P, P, I, P, I, P, P, P, P, P]
        lib.locc_network.argtypes = [P, P, I, P, P, P]
        lib.locc_broadphase.argtypes = [P, P, P, P, I, P, P, I, P]
        lib.locc_step.argtypes = [P, P, P, I, P, I, P, P, I, P, P]
        lib.locc_step_host.argtypes = [P, P, P, I, P, I, P, P, I, P, P]
        lib.locc_reserve.argtypes = [P, I, I]
        lib.locc_set_pipeline.argtypes = [P, I, I]
        lib.locc_autotune.argtypes = [P, P, P, I, P, I, P, P, I, P, I, P, P, P]
        lib.locc_profile.argtypes = [P, ctypes.c_int]
        lib.locc_stage_times.argtypes = [P, P, ctypes.c_int]
        lib.locc_status.argtypes = [P, P]
        lib.locc_selftest_wait_timeout.argtypes = [P, ctypes.c_int64, P]
        lib.locc_trainer_get_state.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_int64), P]
        lib.locc_trainer_set_state.argtypes = [P, P, P, ctypes.c_int64, P]
        lib.locc_trainer_create.argtypes = [P, I, ctypes.POINTER(TrainConfig), ctypes.POINTER(P)]
        lib.locc_train_step.argtypes = [P, P, P, I, P, I, P, P, P, I, P]
        lib.locc_trainer_grad.argtypes = [P, P, P]
        lib.locc_trainer_params.argtypes = [P, P, P]
        lib.locc_trainer_set_params.argtypes = [P, P, P]
        lib.locc_trainer_commit.argtypes = [P]
        lib.locc_trainer_set_lr.argtypes = [P, ctypes.c_float]
        lib.locc_trainer_set_precision.argtypes = [P, I]
        lib.locc_stepper_create.argtypes = [P, I, I, I, I, ctypes.POINTER(P)]
        lib.locc_stepper_submit.argtypes = [P, P, P, I, P, I, P, P, P,
                                            ctypes.POINTER(ctypes.c_int64)]
        lib.locc_stepper_wait.argtypes = [P, ctypes.c_int64]
        lib.locc_stepper_destroy.argtypes = [P]
        lib.locc_stepper_destroy.restype = None
        lib.locc_trainer_destroy.argtypes = [P]
        lib.locc_trainer_destroy.restype = None
        lib.locc_server_create.argtypes = [P, ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
        lib.locc_server_submit.argtypes = [P, ctypes.POINTER(Request),
                                           ctypes.POINTER(ctypes.c_int64)]
        lib.locc_server_wait.argtypes = [P, ctypes.c_int64, I, ctypes.POINTER(RequestInfo)]
        lib.locc_server_stats.argtypes = [P, ctypes.POINTER(ServerCounters), I]
        lib.locc_server_destroy.argtypes = [P]
        lib.locc_server_destroy.restype = None
        lib.locc_set_crop_mode.argtypes = [P, I]
        lib.locc_gjk_create.argtypes = [I, P, P, P, ctypes.POINTER(P)]
        lib.locc_gjk_detect.argtypes = [P, P, P, I, P, I, I, P, P]
        lib.locc_gjk_status.argtypes = [P, P]
        lib.locc_gjk_destroy.argtypes = [P]
        lib.locc_gjk_destroy.restype = None
        lib.locc_sim_step.argtypes = [P, ctypes.POINTER(SimParams), P, P, P, I, P, P, I, P, P, P]
        lib.locc_sphere_contacts.argtypes = [P, P, P, I, P, P, I, P, P, P]
        lib.locc_voxel_create.argtypes = [ctypes.POINTER(_ShapeLibrary), P, ctypes.c_size_t,
                                          ctypes.POINTER(P)]
        lib.locc_voxel_encode.argtypes = [P, P]
        lib.locc_voxel_latents.argtypes = [P, P, P]
        lib.locc_voxel_detect.argtypes = [P, P, P, I, P, I, P, P]
        lib.locc_voxel_detect_ex.argtypes = [P, P, P, I, P, I, P, P, P, P]
        lib.locc_voxel_status.argtypes = [P, P]
        lib.locc_voxel_set_precision.argtypes = [P, I]
        lib.locc_voxel_destroy.argtypes = [P]
        lib.locc_voxel_destroy.restype = None
        lib.locc_destroy.argtypes = [P]
        lib.locc_destroy.restype = None
        lib.locc_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in VOID_EXPORTS:
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def check(code: int) -> None:
    if code != 0:
        msg = load().locc_last_error().decode(errors="replace")
        raise LoccError(code, msg)


def ptr(t) -> Optional[int]:
    """Device (or host) address of a tensor / numpy array, None for None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr() or None
    return t.ctypes.data or None


def stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return getattr(stream, "cuda_stream", stream) or None


def create(points, aabb, blob: bytes, radius: float, precision: int):
    import numpy as np
    lib = load()
    points = np.ascontiguousarray(points, np.float32)
    aabb = np.ascontiguousarray(aabb, np.float32)
    if points.ndim != 3 or points.shape[2] != 3 or aabb.shape != (points.shape[0], 6):
        raise ValueError("points must be [S, n_points, 3] and aabb [S, 6]")
    sl = _ShapeLibrary(points.shape[0], points.shape[1], points.ctypes.data, aabb.ctypes.data)
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    check(lib.locc_create(ctypes.byref(sl), ctypes.cast(buf, ctypes.c_void_p), len(blob),
                          float(radius), int(precision), ctypes.byref(h)))
    return h


def voxel_create(points, aabb, blob: bytes):
    import numpy as np
    lib = load()
    points = np.ascontiguousarray(points, np.float32)
    aabb = np.ascontiguousarray(aabb, np.float32)
    if points.ndim != 3 or points.shape[2] != 3 or aabb.shape != (points.shape[0], 6):
        raise ValueError("points must be [S, n_points, 3] and aabb [S, 6]")
    sl = _ShapeLibrary(points.shape[0], points.shape[1], points.ctypes.data, aabb.ctypes.data)
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    check(lib.locc_voxel_create(ctypes.byref(sl), ctypes.cast(buf, ctypes.c_void_p), len(blob),
                                ctypes.byref(h)))
    return h
