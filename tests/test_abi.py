"""The C-ABI library builds, loads and exports every entry point that
include/fsi.h declares; the ctypes binding covers the same set.  No compute
call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "fsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsi_\w+)\s*\(", src)))


def test_header_declares_the_step_entry_points():
    names = declared()
    for n in ("fsi_create_problem", "fsi_assemble_step", "fsi_solve_step", "fsi_advance", "fsi_destroy",
              "fsi_footprint_bytes", "fsi_get_state", "fsi_set_state"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2301_10041_gb300 import build, fsi
    try:
        path = build.build()
    except RuntimeError as e:  # no toolkit on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(fsi.EXPORTS) == declared()
    fsi.load_library(path)
    assert fsi.load_library().fsi_status_str(-4) == b"solid point outside the fluid domain"
