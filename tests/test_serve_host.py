"""Host bookkeeping of the request server, on the CPU: the device-arena
allocator (admission by free device memory) and the per-launch packing policy
of continuous batching (``csrc/arena.hpp``, plain C++ compiled here with g++),
plus the server's argument checks through the C ABI without a GPU."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_09439_b300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
def test_arena_and_packing(tmp_path):
    exe = str(tmp_path / "arena_check")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-I", CSRC, "-o", exe,
                           os.path.join(ROOT, "tests", "host", "arena_check.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_server_rejects_null_handle():
    import ctypes
    from paper_2304_09439_b300 import abi
    lib = abi.load()
    s = ctypes.c_void_p()
    assert lib.locc_server_create(None, None, ctypes.byref(s)) == -1
    assert not s.value
    rid = ctypes.c_int64()
    assert lib.locc_server_submit(None, None, ctypes.byref(rid)) == -1
    assert lib.locc_server_wait(None, 1, 0, None) == -1
    assert lib.locc_server_stats(None, None, 0) == -1
    lib.locc_server_destroy(None)
