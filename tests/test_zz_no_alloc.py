"""The allocation-free point location and binning entry point.

Callers that cannot allocate device memory (code running under stream
capture, hosts that forbid allocation after start-up) use
fsi_locate_bin_noalloc with buffers they own.  This file checks, through the
C ABI, that its cells and local coordinates equal the oracle's brute-force
location bit for bit (and the library's own assembly, fsi_get_points), that
points outside the domain get cell -1, are counted and left out of the lists,
and that the per-cell lists hold exactly the points of each cell in increasing
order.  Grids of N = 128 and N = 512 (the compiled-in maximum) take several
blocks of the scan; a call on the largest grid followed by one on a small grid
checks that each call clears what the previous one left in the shared
scratch.  It is collected last so that a run stopping at the first failure has
already run everything else.
"""
import numpy as np
import pytest

import fsi_inputs as fi
from oracle import fsi_oracle as fo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_10041_gb300 import build, fsi
    build.build()
    fsi.load_library()
    return torch, fsi


def _sheared24():
    xy, tris = fi.ring_disk_mesh(9, 0.23, (0.47, 0.52))
    d = xy - np.array([0.47, 0.52])
    X = np.stack([0.9 * d[:, 0] - 0.3 * d[:, 1], 0.3 * d[:, 0] + 0.9 * d[:, 1]], 1) + np.array([0.47, 0.52])
    return fi.FsiCase(N=24, rho_f=1.0, nu=0.1, kappa=10.0, dt=0.01, lid_u=0.0, ref_xy=xy, tris=tris,
                      u0=fi.wall_velocity(24, 0.0), X0=X)


def _partly_outside16():
    """The N = 16 disk moved so that it crosses x = 1 and y = 0."""
    c = fi.disk16_case()
    X = c.X0 + np.array([0.42, -0.38])
    return fi.FsiCase(N=16, rho_f=1.0, nu=1.0, kappa=10.0, dt=0.01, lid_u=0.0, ref_xy=c.ref_xy, tris=c.tris,
                      u0=c.u0, X0=X)


def _run_noalloc(torch, fsi, case):
    dev = torch.device("cuda")
    tris = torch.as_tensor(np.ascontiguousarray(case.tris, dtype=np.int32).ravel(), device=dev)
    X = torch.as_tensor(np.ascontiguousarray(case.X0, dtype=np.float64).ravel(), device=dev)
    npts = 6 * case.tris.shape[0]
    cell = torch.full((npts,), -7, dtype=torch.int32, device=dev)
    xi = torch.full((npts,), -7.0, dtype=torch.float64, device=dev)
    eta = torch.full((npts,), -7.0, dtype=torch.float64, device=dev)
    start = torch.full((case.N * case.N + 1,), -7, dtype=torch.int32, device=dev)
    pts = torch.full((npts,), -1, dtype=torch.int32, device=dev)
    nout = torch.full((1,), -1, dtype=torch.int32, device=dev)
    st = fsi.locate_bin_noalloc(case.N, case.tris.shape[0], tris.data_ptr(), X.data_ptr(), cell.data_ptr(),
                                xi.data_ptr(), eta.data_ptr(), start.data_ptr(), pts.data_ptr(), nout.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    return cell.cpu().numpy(), xi.cpu().numpy(), eta.cpu().numpy(), start.cpu().numpy(), pts.cpu().numpy(), \
        int(nout.item())


def _check(case, out, sample=None):
    """Compare one call's outputs with the oracle's brute-force location (all
    points, or the points of `sample` sampled triangles) and check the lists."""
    cell, xi, eta, start, pts, nout = out
    tris = case.tris.astype(np.int64)
    if sample is None:
        pid = np.arange(cell.size)
        x = fo.quadrature_points(case.X0, tris)
    else:
        rng = np.random.default_rng(case.N)
        t = np.sort(rng.choice(tris.shape[0], size=sample, replace=False))
        pid = (6 * t[:, None] + np.arange(6)[None, :]).ravel()
        x = fo.quadrature_points(case.X0, tris[t])
    ocell, oxi, oeta = fo.locate_brute_force(x, case.N)
    assert np.array_equal(cell[pid], ocell)
    assert np.array_equal(xi[pid], oxi) and np.array_equal(eta[pid], oeta)
    inside = cell >= 0
    assert nout == int((~inside).sum())
    nc = case.N * case.N
    assert start[0] == 0 and start[nc] == int(inside.sum())
    assert np.array_equal(np.diff(start), np.bincount(cell[inside], minlength=nc))
    ids = np.nonzero(inside)[0]
    order = ids[np.argsort(cell[ids], kind="stable")]    # by cell, then by point id
    assert np.array_equal(pts[:ids.size], order)


def test_noalloc_matches_oracle_and_library_assembly_twice(env):
    torch, fsi = env
    for case in (fi.disk16_case(), _sheared24(), fi.ellipse_case(128)):
        prob = fsi.problem_from_case(case)
        prob.assemble_step()
        rcell, rxi, reta = prob.get_points()
        prob.close()
        for _ in range(2):  # the second call sees the scratch the first one left
            out = _run_noalloc(torch, fsi, case)
            _check(case, out)
            assert out[5] == 0
            assert np.array_equal(out[0], rcell)
            assert np.array_equal(out[1], rxi) and np.array_equal(out[2], reta)


def test_noalloc_points_outside_the_domain(env):
    torch, fsi = env
    case = _partly_outside16()
    for _ in range(2):
        out = _run_noalloc(torch, fsi, case)
        _check(case, out)
        assert 0 < out[5] < out[0].size


def test_noalloc_largest_grid_then_a_small_one(env):
    """N = 512 fills the whole compiled-in scratch (256 scan blocks); the N =
    24 call after it must not see its counts."""
    torch, fsi = env
    big = fi.ellipse_case(512)
    out = _run_noalloc(torch, fsi, big)
    _check(big, out, sample=40000)
    assert out[5] == 0
    small = _sheared24()
    _check(small, _run_noalloc(torch, fsi, small))


def test_noalloc_rejects_grids_above_the_scratch(env):
    torch, fsi = env
    st = fsi.locate_bin_noalloc(513, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0)   # N*N > FSI_NOALLOC_MAX_CELLS
    assert st == fsi.FSI_ERR_INVALID
