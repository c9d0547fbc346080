import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def curand_ref():
    """The CUDA toolkit's Philox4x32-10 (curand_Philox4x32_10), compiled for the
    host from its header, as an implementation independent of ours."""
    import ctypes
    src = os.path.join(HERE, "helpers", "curand_philox_ref.cu")
    lib = os.path.join(BUILD, "libcurand_philox_ref.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        if not os.path.exists(nvcc):
            pytest.skip("nvcc not available to build the cuRAND reference")
        os.makedirs(BUILD, exist_ok=True)
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-Xcompiler", "-fPIC", "-shared", "-o", tmp, src], check=True)
        os.replace(tmp, lib)
    return ctypes.CDLL(lib)


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.lib()
    return O
