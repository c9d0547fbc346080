"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/flb.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1204_6734_gb300 import build, flb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "flb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("flb_create", "flb_step", "flb_correlations", "flb_destroy",
                 "flb_set_sampling", "flb_conservation", "flb_get_populations",
                 "flb_set_populations", "flb_run_host"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(flb.exported_symbols()) == declared_symbols()
    lib = flb.load()
    for n in declared_symbols():
        assert hasattr(flb, n), n


def test_pure_host_entry_points():
    """Calls that touch no device: version, error strings, argument checks."""
    lib = flb.load()
    assert flb.flb_version() >= 100
    for code in range(0, -8, -1):
        assert flb.flb_error_string(code)
    assert "unknown" in flb.flb_error_string(-99)
    # invalid parameters are rejected before any CUDA call
    from paper_1204_6734_gb300 import inputs
    bad = inputs.LatticeParams(0, 4)
    assert flb.flb_workspace_bytes(bad) == 0
    with pytest.raises(flb.FlbError) as e:
        flb.flb_create(bad)
    assert e.value.code == flb.ERR_ARG
    outside = inputs.LatticeParams(8, 8, ux0=0.6, uy0=0.6)        # some f_i^0(1,u0) < 0
    with pytest.raises(flb.FlbError):
        flb.flb_create(outside)
    bad_omega = inputs.LatticeParams(8, 8, omega=(0, 0, 0, 2.0, 1, 1, 1, 1, 1))
    with pytest.raises(flb.FlbError):
        flb.flb_create(bad_omega)
    assert lib.flb_destroy(None) == 0


def _compile_c_client(tmp_path):
    """Build tests/helpers/capi_example.c with gcc as C99, linked to the library."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    lib = build.build()
    exe = str(tmp_path / "capi_example")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "helpers", "capi_example.c"), "-o", exe,
           "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib), "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_is_c99_and_links_from_c(tmp_path):
    """The boundary is a C ABI: a C99 client compiles with warnings as errors
    and links against the library (it is not run without a GPU)."""
    assert os.path.exists(_compile_c_client(tmp_path))


@pytest.mark.gpu
def test_c_client_matches_the_binding(tmp_path):
    import subprocess

    import numpy as np
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _compile_c_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    t, n, m, jx, jy, c00, cmm33 = r.stdout.split()
    from paper_1204_6734_gb300 import inputs
    p = inputs.LatticeParams(96, 40, 1.0, 0.1, 0.0, 1e-4, inputs.omega_groups(1.1, 0.8, 1.3), "local", "fp32",
                             seed=2024)
    with flb.Lattice(p) as lat:
        lat.set_sampling(10, 1)
        lat.step(50)
        sums = lat.conservation()
        Cff, CMM, _, nn = lat.correlations("local")
    assert int(t) == 50 and int(n) == nn
    np.testing.assert_allclose([float(m), float(jx), float(jy)], sums, rtol=1e-12, atol=1e-12)
    assert float(c00) == pytest.approx(Cff[0, 0], rel=1e-9)
    assert float(cmm33) == pytest.approx(CMM[3, 3], rel=1e-9)
