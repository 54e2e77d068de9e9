"""The allocation-free point location and binning entry point.

Callers that cannot allocate device memory (code running under stream
capture, hosts that forbid allocation after start-up) use
fsi_locate_bin_noalloc with buffers they own.  This file checks, through the
C ABI, that two calls in a row give the same cells and local coordinates as
the library's normal assembly (fsi_get_points), bit for bit, and cell lists
that hold exactly those points in increasing order.  It is collected last so
that a run stopping at the first failure has already run everything else.
"""
import numpy as np
import pytest

import fsi_inputs as fi

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


def _cases():
    c0 = fi.disk16_case()
    xy, tris = fi.ring_disk_mesh(9, 0.23, (0.47, 0.52))
    d = xy - np.array([0.47, 0.52])
    X = np.stack([0.9 * d[:, 0] - 0.3 * d[:, 1], 0.3 * d[:, 0] + 0.9 * d[:, 1]], 1) + np.array([0.47, 0.52])
    c1 = fi.FsiCase(N=24, rho_f=1.0, nu=0.1, kappa=10.0, dt=0.01, lid_u=0.0, ref_xy=xy, tris=tris,
                    u0=fi.wall_velocity(24, 0.0), X0=X)
    return [c0, c1]


def _run_noalloc(torch, fsi, case):
    dev = torch.device("cuda")
    tris = torch.as_tensor(np.ascontiguousarray(case.tris, dtype=np.int32).ravel(), device=dev)
    X = torch.as_tensor(np.ascontiguousarray(case.X0, dtype=np.float64).ravel(), device=dev)
    npts = 6 * case.tris.shape[0]
    cell = torch.full((npts,), -7, dtype=torch.int32, device=dev)
    xi = torch.zeros(npts, dtype=torch.float64, device=dev)
    eta = torch.zeros(npts, dtype=torch.float64, device=dev)
    start = torch.zeros(case.N * case.N + 1, dtype=torch.int32, device=dev)
    pts = torch.full((npts,), -1, dtype=torch.int32, device=dev)
    nout = torch.full((1,), -1, dtype=torch.int32, device=dev)
    st = fsi.locate_bin_noalloc(case.N, case.tris.shape[0], tris.data_ptr(), X.data_ptr(), cell.data_ptr(),
                                xi.data_ptr(), eta.data_ptr(), start.data_ptr(), pts.data_ptr(), nout.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    return cell.cpu().numpy(), xi.cpu().numpy(), eta.cpu().numpy(), start.cpu().numpy(), pts.cpu().numpy(), \
        int(nout.item())


def test_noalloc_matches_library_assembly_twice(env):
    torch, fsi = env
    for case in _cases():
        prob = fsi.problem_from_case(case)
        prob.assemble_step()
        rcell, rxi, reta = prob.get_points()
        prob.close()
        for _ in range(2):  # the second call sees the scratch the first one left
            cell, xi, eta, start, pts, nout = _run_noalloc(torch, fsi, case)
            assert nout == 0
            assert np.array_equal(cell, rcell)
            assert np.array_equal(xi, rxi) and np.array_equal(eta, reta)
            assert start[0] == 0 and start[-1] == cell.size
            assert np.array_equal(np.diff(start), np.bincount(rcell, minlength=case.N * case.N))
            for c in np.nonzero(np.diff(start))[0]:
                assert np.array_equal(pts[start[c]:start[c + 1]], np.nonzero(rcell == c)[0])


def test_noalloc_rejects_grids_above_the_scratch(env):
    torch, fsi = env
    st = fsi.locate_bin_noalloc(1024, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0)   # N*N > FSI_NOALLOC_MAX_CELLS
    assert st == fsi.FSI_ERR_INVALID
