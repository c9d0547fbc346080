"""The lattice storage's ghost-frame arithmetic (flb_layout.cuh, shared by all
step kernels), run on the host: every pull of every node reads the value its
periodic origin stored, every index stays inside the buffer, and interior rows
start 128-byte aligned (FP32) as the TMA tiles and coalesced stores assume."""
import ctypes
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    src = os.path.join(HERE, "helpers", "layout_check.cu")
    hdr = os.path.join(HERE, "..", "paper_1204_6734_gb300", "csrc", "flb_layout.cuh")
    out = os.path.join(HERE, "_build", "liblayout_check.so")
    if (not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(src),
                                                               os.path.getmtime(hdr))):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        if not os.path.exists(nvcc):
            pytest.skip("nvcc not available")
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-O1", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-Xcompiler", "-fPIC", "-shared", "-o", tmp, src], check=True)
        os.replace(tmp, out)
    L = ctypes.CDLL(out)
    L.layout_check.restype = ctypes.c_longlong
    L.layout_check.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_longlong)]
    return L


SHAPES = [(1, 1), (1, 2), (2, 1), (2, 2), (3, 3), (1, 7), (7, 1), (5, 7), (21, 21), (31, 33),
          (32, 32), (33, 1), (64, 5), (127, 3), (128, 4), (129, 2), (300, 17)]


@pytest.mark.parametrize("shape", SHAPES)
def test_ghost_frame_pulls_periodic_images(lib, shape):
    pitch, plane = ctypes.c_longlong(), ctypes.c_longlong()
    assert lib.layout_check(shape[0], shape[1], ctypes.byref(pitch), ctypes.byref(plane)) == 0
    assert pitch.value % 32 == 0 and pitch.value >= shape[0] + 33
    assert plane.value == pitch.value * (shape[1] + 2)
