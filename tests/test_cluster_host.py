"""Host logic of the cluster-resident coarse multigrid levels, without a GPU.

`tests/cluster_emul.cu` builds the per-CTA shared-memory images with the
library's builder (`fsi_cluster_host.h`), replays the cluster kernel's phases
on the host with every shared-memory, remote and global access checked
against its buffer, and compares the result with a plain per-level V-cycle
(Section 5 smoother and transfers) on the host matrices: FP64 to 1e-12, FP32
images to 1e-5, for the velocity and pressure hierarchies, clusters of 16
and 8 CTAs, grids N = 16, 24, 96, 128.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2301_10041_gb300", "csrc")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_cluster_images_and_phases_match_per_level_vcycle(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "cluster_emul")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-I", CSRC,
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "cluster_emul.cu"),
           os.path.join(CSRC, "fsi_setup.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert "failures=0" in r.stdout
