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
