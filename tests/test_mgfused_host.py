"""The fused matrix-free multigrid kernels (fsi_mgfused.cuh) without a GPU.

`tests/mgfused_emul.cu` runs the kernels' __host__ __device__ bodies on the
host, one thread per CTA, under AddressSanitizer (every shared-memory frame
is a separate heap block of exactly the launch's size), and compares each
launch with the same multigrid step written on the assembled level matrices
of the host setup: the down launch (Chebyshev pre-smoothing from
c0 D^-1 b, residual, Q2 / P1disc restriction, coarse smoother start) and the
up launch (prolongation, post-smoothing, Richardson and Cahouet-Chabard
epilogues), velocity and pressure, degrees 1-4, grids N = 16, 24, 48, 128 and the next coarser level, and N = 512 (the
larger tiles): FP64 to 1e-12, FP32 to 1e-5.  On the finest level the down
launch is also checked with the Stokes residual start of a Richardson step
(Section 5): its right-hand side b - A_f z_u - (-B^T) z_p (velocity; also
without z_u) and b - (-B) z_u (pressure) against the assembled A_f, -B^T and
-B, and the smoothing and restriction that follow.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2301_10041_gb300", "csrc")


def test_fused_multigrid_kernels_match_the_assembled_levels(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                    else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "mgfused_emul")
    base = [nvcc, "-std=c++17", "-O1", "-g", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
            os.path.join(HERE, "mgfused_emul.cu"), os.path.join(CSRC, "fsi_setup.cpp"), "-o", exe]
    r = subprocess.run(base[:1] + ["-Xcompiler", "-fsanitize=address,-fno-omit-frame-pointer"] + base[1:],
                       capture_output=True, text=True)
    if r.returncode != 0:   # no sanitizer runtime: plain build
        r = subprocess.run(base, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "failures=0" in r.stdout
    assert r.stdout.count("residual start: right-hand side") >= 20
