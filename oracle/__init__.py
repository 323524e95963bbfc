"""The oracle: plain, slow CPU implementations of what the contact path computes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()``, the
CPU-baseline / reference legs of ``bench.py`` and the scripts under
``oracle/`` and ``tests/golden/`` that write stored expected values may import
this package.  The product library never imports, links or runs it, and it
shares no code with the CUDA path.

Two parts, both plain C compiled with ``-ffp-contract=off`` (no fused
multiply-add, no fast-math):

* oracle (a), ``oracle_a.c``: float64 geometric contact detector on the
  triangle meshes (label, contact point, normal, penetration depth);
* oracle (b), ``oracle_b.c``: the crop selection in float32 (fixed operation
  order, reproducible bit for bit) and the crop network forward / backward in
  float64.

Each C function's header comment cites the passage of the paper it follows.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liblocc_oracle.so")
_SRCS = [os.path.join(_HERE, "oracle_a.c"), os.path.join(_HERE, "oracle_b.c")]
_lock = threading.Lock()
_lib = None

KMAX = 64
N_PARAMS = 240776
LAYER_DIMS = [(3, 64), (64, 128), (128, 256), (512, 256), (256, 256), (256, 8)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liblocc_oracle.so`` (gcc, -O2,
    -ffp-contract=off)."""
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", "-pthread", "-o", tmp] + _SRCS + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.orb_run.argtypes = [P, P, I, I, P, P, I, P, I, ctypes.c_float, I,
                                P, P, P, P, P, P, P, I]
        lib.orb_run.restype = I
        lib.orb_run_global.argtypes = [P, P, I, I, P, P, I, P, I, ctypes.c_float, I,
                                P, P, P, P, P, P, P, I]
        lib.orb_run_global.restype = I
        lib.orb_network.argtypes = [P, P, P, I, I, P, P]
        lib.orb_network.restype = I
        lib.orb_loss_grad.argtypes = [P, P, P, P, I, I, P, I, P]
        lib.orb_loss_grad.restype = ctypes.c_double
        lib.orb_bf16.argtypes = [ctypes.c_double]
        lib.orb_bf16.restype = ctypes.c_double
        lib.orb_n_params.restype = I
        lib.ora_contact_batch.argtypes = [P, P, P, P, P, P, I, P, P, P, I, I,
                                          P, I]
        lib.ora_contact_batch.restype = I
        lib.ora_inside.argtypes = [P, I, P, P, I, P, P, I, P]
        lib.ora_inside.restype = I
        lib.orb_broadphase.argtypes = [P, I, P, P, P, I, P, ctypes.c_longlong]
        lib.orb_broadphase.restype = ctypes.c_longlong
        assert lib.orb_n_params() == N_PARAMS
        _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def flatten_params(weights: Sequence[Tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    """[(W [out,in], b [out]) x 6] float32 -> flat float64 (W1 b1 W2 b2 ...)."""
    parts = []
    for (w, b), (fi, fo) in zip(weights, LAYER_DIMS):
        assert w.shape == (fo, fi) and b.shape == (fo,)
        parts += [np.asarray(w, np.float64).ravel(), np.asarray(b, np.float64)]
    flat = np.concatenate(parts)
    assert flat.size == N_PARAMS
    return flat


def unflatten_params(flat: np.ndarray):
    out, o = [], 0
    for fi, fo in LAYER_DIMS:
        w = flat[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        b = flat[o:o + fo]
        o += fo
        out.append((w, b))
    return out


def crop_forward(points, aabb, poses, obj_shape, pairs, r: float,
                 params: Optional[np.ndarray] = None, kmax: int = KMAX,
                 n_threads: int = 1, mode: str = "local"):
    """Oracle (b): crop selection (+ network forward when ``params`` given).
    ``mode`` "global": each object's first kmax samples instead of the local
    crop (the ablation without locality).

    Returns a dict with idx [P,2,kmax] int32 (-1 padded), cnt [P,2] int32,
    xyz [P,2,kmax,3] float32 canonical coordinates, centre [P,3] float32 and,
    with params, out [P,8] float64 world-frame outputs and feat [P,512] float64.
    """
    lib = _load()
    points = _c(points, np.float32)
    aabb = _c(aabb, np.float32)
    poses = _c(poses, np.float32)
    obj_shape = _c(obj_shape, np.int32)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    S, NP = points.shape[0], points.shape[1]
    P = pairs.shape[0]
    idx = np.empty((P, 2, kmax), np.int32)
    cnt = np.empty((P, 2), np.int32)
    xyz = np.empty((P, 2, kmax, 3), np.float32)
    centre = np.empty((P, 3), np.float32)
    out = feat = None
    if params is not None:
        params = _c(params, np.float64)
        assert params.size == N_PARAMS
        out = np.empty((P, 8), np.float64)
        feat = np.empty((P, 512), np.float64)
    run = {"local": lib.orb_run, "global": lib.orb_run_global}[mode]
    st = run(_ptr(points), _ptr(aabb), S, NP, _ptr(poses), _ptr(obj_shape),
                     poses.shape[0], _ptr(pairs), P, float(r), kmax, _ptr(params),
                     _ptr(idx), _ptr(cnt), _ptr(xyz), _ptr(centre), _ptr(out),
                     _ptr(feat), int(n_threads))
    if st != 0:
        raise ValueError(f"oracle crop_forward failed with status {st}")
    res = dict(idx=idx, cnt=cnt, xyz=xyz, centre=centre)
    if params is not None:
        res.update(out=out, feat=feat)
    return res


def network(params: np.ndarray, xyz: np.ndarray, cnt: np.ndarray,
            kmax: int = KMAX):
    """Oracle (b) network on given crops -> (raw canonical y [P,8], feat [P,512])."""
    lib = _load()
    params = _c(params, np.float64)
    xyz = _c(xyz, np.float32)
    cnt = _c(cnt, np.int32)
    P = cnt.shape[0]
    y = np.empty((P, 8), np.float64)
    f = np.empty((P, 512), np.float64)
    if lib.orb_network(_ptr(params), _ptr(xyz), _ptr(cnt), P, kmax, _ptr(y), _ptr(f)):
        raise ValueError("bad crop counts")
    return y, f


DEFAULT_LOSS_HP = (1.0, 1.0, 1.0, 0.01, 0.5, 0.0)  # w_pt, w_n, w_d, huber beta, alpha, w_len


def loss_grad(params: np.ndarray, xyz: np.ndarray, cnt: np.ndarray,
              tgt: np.ndarray, hp=DEFAULT_LOSS_HP, kmax: int = KMAX, operands: str = "exact"):
    """Mean training loss over the pairs and its gradient (flat float64).

    operands="bf16" rounds both operands of the matrix-product layers to
    bfloat16 before their float64 products (the arithmetic of a bf16
    tensor-core trainer; which products, in oracle_b.c's header)."""
    if operands not in ("exact", "bf16"):
        raise ValueError(f"operands must be 'exact' or 'bf16', not {operands!r}")
    lib = _load()
    params = _c(params, np.float64)
    xyz = _c(xyz, np.float32)
    cnt = _c(cnt, np.int32)
    tgt = _c(tgt, np.float64)
    hp = _c(tuple(hp) + (0.0,) * (6 - len(hp)), np.float64)  # w_len defaults to 0
    assert hp.size == 6
    g = np.empty(N_PARAMS, np.float64)
    L = lib.orb_loss_grad(_ptr(params), _ptr(xyz), _ptr(cnt), _ptr(tgt),
                          cnt.shape[0], kmax, _ptr(hp), int(operands == "bf16"), _ptr(g))
    return float(L), g


def round_bf16(x) -> np.ndarray:
    """The oracle's bfloat16 rounding (orb_bf16) of each value, as float64."""
    lib = _load()
    a = np.asarray(x, np.float64)
    return np.array([lib.orb_bf16(float(v)) for v in a.ravel()], np.float64).reshape(a.shape)


def broadphase(aabb, poses, obj_shape, env_offsets) -> np.ndarray:
    """Oracle broad phase: int32 [n_pairs, 2] overlapping pairs per environment,
    ordered by environment, then i, then j."""
    lib = _load()
    aabb = _c(aabb, np.float32)
    poses = _c(poses, np.float32)
    obj_shape = _c(obj_shape, np.int32)
    env_offsets = _c(env_offsets, np.int32)
    n_env = env_offsets.shape[0] - 1
    n = lib.orb_broadphase(_ptr(aabb), aabb.shape[0], _ptr(poses), _ptr(obj_shape),
                           _ptr(env_offsets), n_env, None, 0)
    if n < 0:
        raise ValueError("bad shape id")
    out = np.empty((max(n, 1), 2), np.int32)
    lib.orb_broadphase(_ptr(aabb), aabb.shape[0], _ptr(poses), _ptr(obj_shape),
                       _ptr(env_offsets), n_env, _ptr(out), n)
    return out[:n]


def _pack_meshes(meshes):
    V = np.concatenate([m.vertices for m in meshes]).astype(np.float64)
    F = np.concatenate([m.faces for m in meshes]).astype(np.int32)
    comp = np.concatenate([m.comp for m in meshes]).astype(np.int32)
    voff = np.zeros(len(meshes) + 1, np.int64)
    foff = np.zeros(len(meshes) + 1, np.int64)
    voff[1:] = np.cumsum([m.vertices.shape[0] for m in meshes])
    foff[1:] = np.cumsum([m.faces.shape[0] for m in meshes])
    return V, voff, F, comp, foff


def contact(meshes, samples, poses, obj_shape, pairs, culled: bool = True,
            n_threads: int = 1) -> np.ndarray:
    """Oracle (a): {label, point xyz, normal xyz, depth} [P,8] float64, world
    frame, normal from A towards B, depth > 0 penetration / < 0 gap."""
    lib = _load()
    V, voff, F, comp, foff = _pack_meshes(meshes)
    samples = _c(samples, np.float32)
    poses = _c(poses, np.float32)
    obj_shape = _c(obj_shape, np.int32)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    out = np.empty((pairs.shape[0], 8), np.float64)
    st = lib.ora_contact_batch(_ptr(V), _ptr(voff), _ptr(F), _ptr(comp), _ptr(foff),
                               _ptr(samples), samples.shape[1], _ptr(poses),
                               _ptr(obj_shape), _ptr(pairs), pairs.shape[0],
                               int(bool(culled)), _ptr(out), int(n_threads))
    if st:
        raise MemoryError("oracle contact failed")
    return out


def inside(mesh, pose, pts) -> np.ndarray:
    """Winding-number inside test of world points against one posed mesh."""
    lib = _load()
    V = _c(mesh.vertices, np.float64)
    F = _c(mesh.faces, np.int32)
    comp = _c(mesh.comp, np.int32)
    pose = _c(pose, np.float32)
    pts = _c(pts, np.float64).reshape(-1, 3)
    res = np.empty(pts.shape[0], np.int32)
    lib.ora_inside(_ptr(V), V.shape[0], _ptr(F), _ptr(comp), F.shape[0], _ptr(pose),
                   _ptr(pts), pts.shape[0], _ptr(res))
    return res.astype(bool)
