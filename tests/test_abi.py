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


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Offsets and sizes of the ctypes mirrors of fsi_params, fsi_solid_mesh
    and fsi_solve_info equal those a C compiler gives the header."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2301_10041_gb300 import fsi
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fsi.h"', "int main(void) {"]
    structs = {"fsi_params": fsi.fsi_params, "fsi_solid_mesh": fsi.fsi_solid_mesh,
               "fsi_solve_info": fsi.fsi_solve_info}
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_ctypes_structs_list_every_header_field_in_order():
    """A field missing from a ctypes mirror could hide in tail padding: the
    member names of each header struct equal the mirror's, in order."""
    from paper_2301_10041_gb300 import fsi
    src = open(os.path.join(ROOT, "include", "fsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for cname, cls in (("fsi_params", fsi.fsi_params), ("fsi_solid_mesh", fsi.fsi_solid_mesh),
                       ("fsi_solve_info", fsi.fsi_solve_info)):
        body = re.search(r"typedef struct " + cname + r"\s*\{(.*?)\}\s*" + cname + ";", src, flags=re.S).group(1)
        names = [re.findall(r"(\w+)\s*$", d.strip())[0] for d in body.split(";") if d.strip()]
        assert names == [f for f, _ in cls._fields_], cname


FOOTPRINT_SWEEP = r"""
import sys
sys.path.insert(0, sys.argv[1])
from paper_2301_10041_gb300 import fsi
fsi.load_library()
bad = []
for elem in (0, 1):
    for N in (8, 16):
        prm = fsi.make_params(N, 1.0, 0.1, 10.0, 0.01, solid_elem=elem)
        for nn in range(1, 14):
            for ne in (1, 2, 5, 17, 40):
                v = fsi.footprint_bytes(prm, nn, ne)
                valid = nn >= (4 if elem else 3)
                if (v > 0) != valid:
                    bad.append((elem, N, nn, ne, v))
print("bad", bad)
"""


def test_footprint_is_host_logic_and_never_crashes():
    """fsi_footprint_bytes counts bytes on the host (no device call): it is
    positive for every valid size, 0 for meshes too small for their element,
    never faults on tiny meshes (run in a child process), and grows with
    the grid and the solid."""
    import subprocess
    import sys
    from paper_2301_10041_gb300 import build, fsi
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    r = subprocess.run([sys.executable, "-c", FOOTPRINT_SWEEP, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().endswith("bad []"), r.stdout[-2000:]
    fsi.load_library()
    for elem in (0, 1):
        f = lambda N, nn, ne: fsi.footprint_bytes(fsi.make_params(N, 1.0, 0.1, 10.0, 0.01, solid_elem=elem), nn, ne)
        assert f(16, 60, 44) < f(32, 60, 44) < f(64, 60, 44)
        assert f(32, 60, 44) < f(32, 600, 440)
    assert fsi.footprint_bytes(fsi.make_params(15, 1.0, 0.1, 10.0, 0.01), 60, 44) == 0   # odd N
