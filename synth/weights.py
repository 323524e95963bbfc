"""Xavier-initialised parameters of the crop network.

Layer list (in, out): per-point encoder 3 -> 64 -> 128 -> 256 (shared by both
objects of a pair), head 512 -> 256 -> 256 -> 8.  Weights are stored row-major
as [out, in] float32, biases as [out] float32.
"""

from __future__ import annotations

from typing import List, Tuple

import numpy as np

LAYER_DIMS: List[Tuple[int, int]] = [(3, 64), (64, 128), (128, 256),
                                     (512, 256), (256, 256), (256, 8)]


def xavier_weights(seed: int = 1, bias_scale: float = 0.0):
    """Glorot-uniform weights, U(-a, a) with a = sqrt(6 / (in + out)).

    Biases are zero unless ``bias_scale`` > 0, in which case they are drawn
    U(-bias_scale, bias_scale) (tests use this to exercise the bias paths).
    Returns a list of (W [out, in], b [out]) float32 pairs.
    """
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in LAYER_DIMS:
        a = np.sqrt(6.0 / (fi + fo))
        w = rng.uniform(-a, a, size=(fo, fi)).astype(np.float32)
        if bias_scale > 0:
            b = rng.uniform(-bias_scale, bias_scale, size=fo).astype(np.float32)
        else:
            b = np.zeros(fo, np.float32)
        out.append((w, b))
    return out


def voxel_weights(layers, seed: int = 7, bias_scale: float = 0.05) -> np.ndarray:
    """He-uniform parameters of the voxel-latent network (ReLU throughout) as
    one flat float32 vector in the order of ``layers`` ((name, shape) pairs;
    names ending in ".b" are biases): U(-a, a), a = sqrt(6 / fan_in), where
    fan_in = in * k for linear weights [out, in] and convolutions [out, in, 3,
    3, 3] (k = 27), and for transposed convolutions [in, out, 3, 3, 3] the
    number of inputs reaching one output, in * 27.  Biases are
    U(-bias_scale, bias_scale)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in layers:
        shape = tuple(shape)
        if name.endswith(".b"):
            parts.append(rng.uniform(-bias_scale, bias_scale, size=shape).astype(np.float32))
            continue
        k = int(np.prod(shape[2:])) if len(shape) > 2 else 1
        fan_in = (shape[0] if name.startswith("d") else shape[1]) * k
        a = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-a, a, size=shape).astype(np.float32).ravel())
    return np.concatenate([p.ravel() for p in parts])
