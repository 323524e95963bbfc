"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every symbol the header declares; the weights blob round-trips."""

import ctypes
import re
import os

import numpy as np
import pytest

import synth
from paper_2304_09439_b300 import abi, build, weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "locc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(locc_[a-z_]+)\s*\(", src)))


def test_library_exports_every_header_symbol():
    lib = abi.load()
    declared = _header_functions()
    assert set(declared) == set(abi.EXPORTS), declared
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.locc_last_error() is not None


def test_library_is_built_for_sm103a():
    so = build.build()
    assert os.path.exists(so)
    assert "compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_create_rejects_bad_arguments_without_gpu():
    # argument checks run before any CUDA call
    lib = abi.load()
    h = ctypes.c_void_p()
    assert lib.locc_create(None, None, 0, ctypes.c_float(0.25), 0, ctypes.byref(h)) == -1
    assert b"library" in lib.locc_last_error()
    assert lib.locc_detect(None, None, None, 0, None, 0, None, None) == -1
    assert lib.locc_status(None, None) == -1


def test_bad_weights_blob_is_rejected():
    lib = abi.load()
    pts = np.zeros((1, 32, 3), np.float32)
    aabb = np.array([[-1, -1, -1, 1, 1, 1]], np.float32)
    blob = bytearray(weights.pack(synth.xavier_weights(1)))
    blob[0:8] = b"XXXXXXXX"
    with pytest.raises(abi.LoccError) as e:
        abi.create(pts, aabb, bytes(blob), 0.25, 0)
    assert e.value.code == -5
    short = weights.pack(synth.xavier_weights(1))[:-4]
    with pytest.raises(abi.LoccError) as e:
        abi.create(pts, aabb, short, 0.25, 0)
    assert e.value.code == -5


def test_weights_blob_roundtrip():
    layers = synth.xavier_weights(2, bias_scale=0.1)
    blob = weights.pack(layers)
    assert len(blob) == 16 + 48 + 4 * weights.N_PARAMS
    back = weights.unpack(blob)
    for (w, b), (w2, b2) in zip(layers, back):
        assert np.array_equal(w, w2) and np.array_equal(b, b2)
