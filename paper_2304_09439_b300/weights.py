"""The "LOCCW001" parameter blob read by ``locc_create``.

Layout (little endian): 8-byte magic ``LOCCW001``, uint32 version (1), uint32
number of layers (6), six (uint32 in, uint32 out) pairs, then for every layer
float32 W[out][in] followed by float32 b[out].
"""

from __future__ import annotations

import struct
from typing import List, Sequence, Tuple

import numpy as np

MAGIC = b"LOCCW001"
LAYER_DIMS: List[Tuple[int, int]] = [(3, 64), (64, 128), (128, 256),
                                     (512, 256), (256, 256), (256, 8)]
N_PARAMS = sum(i * o + o for i, o in LAYER_DIMS)


def pack(layers: Sequence[Tuple[np.ndarray, np.ndarray]]) -> bytes:
    """[(W [out,in], b [out]) x 6] -> blob bytes."""
    if len(layers) != len(LAYER_DIMS):
        raise ValueError("expected 6 layers")
    head = MAGIC + struct.pack("<II", 1, len(LAYER_DIMS))
    body = []
    for (w, b), (fi, fo) in zip(layers, LAYER_DIMS):
        w = np.asarray(w, np.float32)
        b = np.asarray(b, np.float32)
        if w.shape != (fo, fi) or b.shape != (fo,):
            raise ValueError(f"layer {fi}->{fo}: got W{w.shape} b{b.shape}")
        head += struct.pack("<II", fi, fo)
        body += [w.astype("<f4").tobytes(), b.astype("<f4").tobytes()]
    return head + b"".join(body)


def unpack(blob: bytes):
    """Blob bytes -> [(W [out,in], b [out]) x 6] float32."""
    if blob[:8] != MAGIC:
        raise ValueError("bad magic")
    version, n = struct.unpack_from("<II", blob, 8)
    if version != 1 or n != 6:
        raise ValueError("unsupported blob")
    off = 16 + 8 * n
    out = []
    for fi, fo in LAYER_DIMS:
        w = np.frombuffer(blob, "<f4", fi * fo, off).reshape(fo, fi).copy()
        off += 4 * fi * fo
        b = np.frombuffer(blob, "<f4", fo, off).copy()
        off += 4 * fo
        out.append((w, b))
    return out


def flat(layers) -> np.ndarray:
    """Concatenate W1 b1 ... W6 b6 as float32."""
    return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(),
                                           np.asarray(b, np.float32)])
                           for w, b in layers])


def from_flat(flat) -> list:
    """Flat W1 b1 ... W6 b6 -> [(W [out,in], b [out]) x 6] float32."""
    flat = np.asarray(flat, np.float32).ravel()
    if flat.size != N_PARAMS:
        raise ValueError("wrong parameter count")
    out, o = [], 0
    for fi, fo in LAYER_DIMS:
        w = flat[o:o + fi * fo].reshape(fo, fi).copy()
        o += fi * fo
        b = flat[o:o + fo].copy()
        o += fo
        out.append((w, b))
    return out


# ------------------------------------------------------------------ voxel net
# The "LOCCV001" blob of the voxel-latent network read by locc_voxel_create:
# 8-byte magic, uint32 version (1), uint32 parameter count, then float32
# parameters in the order below.  Linear weights are [out][in], convolutions
# [out][in][3][3][3], transposed convolutions [in][out][3][3][3].
VOXEL_MAGIC = b"LOCCV001"
VOXEL_LAYERS = [
    ("e1.w", (256, 3)), ("e1.b", (256,)),
    ("e2.w", (256, 256)), ("e2.b", (256,)),
    ("e3.w", (256, 256)), ("e3.b", (256,)),
    ("c1.w", (128, 256, 3, 3, 3)), ("c1.b", (128,)),
    ("c2.w", (128, 128, 3, 3, 3)), ("c2.b", (128,)),
    ("c3.w", (128, 128, 3, 3, 3)), ("c3.b", (128,)),
    ("c4.w", (128, 128, 3, 3, 3)), ("c4.b", (128,)),
    ("d1.w", (128, 128, 3, 3, 3)), ("d1.b", (128,)),
    ("d2.w", (256, 128, 3, 3, 3)), ("d2.b", (128,)),
    ("d3.w", (256, 128, 3, 3, 3)), ("d3.b", (128,)),
    ("d4.w", (256, 128, 3, 3, 3)), ("d4.b", (128,)),
    ("f.w", (16, 384)), ("f.b", (16,)),
    ("p1.w", (128, 23)), ("p1.b", (128,)),
    ("p2.w", (128, 128)), ("p2.b", (128,)),
    ("p3.w", (128, 128)), ("p3.b", (128,)),
    ("q1.w", (128, 128)), ("q1.b", (128,)),
    ("q2.w", (128, 128)), ("q2.b", (128,)),
    ("q3.w", (128, 128)), ("q3.b", (128,)),
    ("q4.w", (1, 128)), ("q4.b", (1,)),
]
N_VOXEL_PARAMS = int(sum(int(np.prod(s)) for _, s in VOXEL_LAYERS))


def pack_voxel(flat_params) -> bytes:
    """Flat float32 parameters (VOXEL_LAYERS order) -> LOCCV001 blob."""
    v = np.asarray(flat_params, np.float32).ravel()
    if v.size != N_VOXEL_PARAMS:
        raise ValueError(f"expected {N_VOXEL_PARAMS} parameters, got {v.size}")
    return VOXEL_MAGIC + struct.pack("<II", 1, v.size) + v.astype("<f4").tobytes()


def unpack_voxel(blob: bytes) -> np.ndarray:
    """LOCCV001 blob -> flat float32 parameters."""
    if blob[:8] != VOXEL_MAGIC:
        raise ValueError("bad magic")
    version, n = struct.unpack_from("<II", blob, 8)
    if version != 1 or n != N_VOXEL_PARAMS:
        raise ValueError("unsupported voxel blob")
    return np.frombuffer(blob, "<f4", n, 16).copy()
