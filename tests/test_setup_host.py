"""The library's host setup code (fsi_setup.cpp) without a GPU, through
`tests/setup_harness.cpp`:

* the fused pressure restriction: (R L) x equals R (L x) on every level;
* the matrix-free stencils of every level reproduce the assembled rows;
* the Q1 solid operators (Section 6's element): C_s and A_s equal the
  oracle's independent 3 x 3 Gauss assembly, and the Chebyshev interval for
  D^-1 C_s (Wathen's element bound) contains the whole spectrum; on a
  square mesh it is [1/4, 9/4].
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import fsi_inputs as fi
from oracle import fsi_oracle as fo

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2301_10041_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("setup") / "setup_harness")
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "setup_harness.cpp"),
                        os.path.join(CSRC, "fsi_setup.cpp"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


@pytest.mark.parametrize("N", [16, 24, 128])
def test_fused_pressure_restriction_product(harness, N):
    out = subprocess.run([harness, "products", str(N)], capture_output=True, text=True, check=True).stdout
    rows = [json.loads(l) for l in out.splitlines() if l.strip()]
    assert len(rows) >= 1
    for r in rows:
        assert r["rel_err"] < 1e-14, r


@pytest.mark.parametrize("N", [8, 24, 64, 128])
def test_matrix_free_stencils_are_the_assembled_rows(harness, N):
    """The constant-coefficient stencils used by the matrix-free multigrid
    kernels reproduce every row of the assembled velocity operator and
    pressure Laplacian of every level bit for bit (walls only remove
    neighbours of A; L has one stencil per wall variant), and the finest
    level's divergence table reproduces every entry of -B and -B^T."""
    out = subprocess.run([harness, "stencils", str(N)], capture_output=True, text=True, check=True).stdout
    rows = [json.loads(l) for l in out.splitlines() if l.strip()]
    assert len(rows) >= 1
    for r in rows:
        assert r["a_mismatch"] == 0 and r["l_mismatch"] == 0 and r["b_mismatch"] == 0, r


def _solid(harness, tmp_path, xy, quads, kappa):
    path = tmp_path / "mesh.txt"
    with open(path, "w") as f:
        f.write(f"{xy.shape[0]} {quads.shape[0]}\n")
        f.write("\n".join(f"{x:.17g} {y:.17g}" for x, y in xy) + "\n")
        f.write("\n".join(" ".join(str(int(v)) for v in q) for q in quads) + "\n")
    out = subprocess.run([harness, "solid", str(path), str(kappa)], capture_output=True, text=True, check=True).stdout
    d = json.loads(out)
    n = xy.shape[0]

    def mat(t):
        t = np.array(t)
        return sp.coo_matrix((t[:, 2], (t[:, 0].astype(int), t[:, 1].astype(int))), shape=(n, n)).toarray()

    return mat(d["Cs"]), mat(d["As"]), d["cs_lo"], d["cs_hi"]


def test_q1_solid_operators_match_the_oracle(harness, tmp_path):
    xy, quads = fi.annulus_mesh(3, 6, quads=True)
    kappa = 7.0
    C, A, lo, hi = _solid(harness, tmp_path, xy, quads, kappa)
    Co, Ao = fo.assemble_solid_q1(xy, quads.astype(np.int64), kappa)
    assert np.abs(C - Co.toarray()).max() <= 1e-14 * np.abs(Co).max()
    assert np.abs(A - Ao.toarray()).max() <= 1e-13 * np.abs(Ao).max()
    d = np.diag(C)
    ev = np.linalg.eigvalsh(C / np.sqrt(np.outer(d, d)))
    assert lo <= ev.min() * (1 + 1e-12) and ev.max() <= hi * (1 + 1e-12)


def test_q1_interval_on_squares_is_a_quarter_to_nine_quarters(harness, tmp_path):
    n = 4
    g = np.linspace(0.2, 0.6, n + 1)
    X, Y = np.meshgrid(g, g)
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    quads = np.array([(j * (n + 1) + i, j * (n + 1) + i + 1, (j + 1) * (n + 1) + i + 1, (j + 1) * (n + 1) + i)
                      for j in range(n) for i in range(n)])
    C, A, lo, hi = _solid(harness, tmp_path, xy, quads, 1.0)
    assert abs(lo - 0.25) < 1e-13 and abs(hi - 2.25) < 1e-13
    d = np.diag(C)
    ev = np.linalg.eigvalsh(C / np.sqrt(np.outer(d, d)))
    assert lo <= ev.min() + 1e-13 and ev.max() <= hi + 1e-13


@pytest.mark.parametrize("N,cu,cp,Ns,nu,np_", [
    (128, 16, 0, [128, 64, 32, 16], 4, 4),      # the default: both stop at 16 cells
    (128, 16, 32, [128, 64, 32, 16], 4, 3),     # a coarser pressure hierarchy
    (128, 8, 0, [128, 64, 32, 16, 8], 5, 5),
    (96, 16, 0, [96, 48, 24, 12], 4, 4),        # 3 * 2^5: the coarsest is 12 cells
    (24, 16, 32, [24, 12], 2, 1),               # the pressure takes the finest grid itself
    (16, 16, 0, [16], 1, 1),
    (12, 4, 0, [12, 6, 3], 3, 3),               # odd coarsest grid
])
def test_hierarchy_levels_and_dense_coarsest(harness, N, cu, cp, Ns, nu, np_):
    """Each hierarchy ends at its first grid of at most its limit of cells (or
    at an odd one); the dense coarsest matrices have the unknowns of that
    level: 2 (2 n - 1)^2 velocity, 3 n^2 pressure."""
    out = subprocess.run([harness, "levels", str(N), str(cu), str(cp)], capture_output=True, text=True,
                         check=True).stdout
    d = json.loads(out)
    assert d["Ns"] == Ns and d["nlev_u"] == nu and d["nlev_p"] == np_
    nc_u, nc_p = Ns[nu - 1], Ns[np_ - 1]
    assert d["coarse_nA"] == 2 * (2 * nc_u - 1) ** 2 and d["coarse_nL"] == 3 * nc_p ** 2
    assert d["dense_A"] == d["coarse_nA"] ** 2 and d["dense_L"] == d["coarse_nL"] ** 2
