"""The exact coupling rule (Section 4: each mapped solid triangle intersected
with the fluid cells by Sutherland-Hodgman, the pieces integrated exactly)
on the GPU against the oracle's restatement of the same rule.

C_f entries to 1e-13 relative (same FP64 arithmetic, different summation
order), including solid triangles that span many fluid cells; one time step
with this coupling to 1e-7 relative at a 1e-12 solve; the bench workload at
full size through the oracle's operator and residual.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import bench
import fsi_inputs as fi
from oracle import fsi_oracle as fo
from tests.gpu_helpers import oracle_to_gpu_perm, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_10041_gb300 import build, fsi as f
    build.build()
    f.load_library()
    return f


def _ragged():
    xy, tris = fi.ring_disk_mesh(9, 0.23, (0.47, 0.52))
    c, s = np.cos(0.3), np.sin(0.3)
    d = xy - np.array([0.47, 0.52])
    X0 = np.stack([c * d[:, 0] - s * d[:, 1] + 0.2 * d[:, 1], s * d[:, 0] + c * d[:, 1]], 1) + np.array([0.47, 0.52])
    return fi.FsiCase(N=24, rho_f=1.3, nu=0.05, kappa=30.0, dt=0.005, lid_u=1.0, ref_xy=xy, tris=tris,
                      u0=fi.initial_velocity(24, 7, lid_u=1.0), X0=X0, precond=1, rtol=1e-12)


def _coarse_body():
    """Solid triangles several fluid cells wide (m = 3 rings on N = 32)."""
    xy, tris = fi.ring_disk_mesh(3, 0.3, (0.5, 0.49))
    d = xy - np.array([0.5, 0.49])
    X0 = np.stack([d[:, 0] + 0.25 * d[:, 1], 0.9 * d[:, 1]], 1) + np.array([0.5, 0.49])
    return fi.FsiCase(N=32, rho_f=1.0, nu=0.5, kappa=20.0, dt=0.01, lid_u=0.0, ref_xy=xy, tris=tris,
                      u0=fi.initial_velocity(32, 3), X0=X0, precond=1, rtol=1e-12)


CASES = {"disk16": fi.disk16_case, "ragged24": _ragged, "coarse_body32": _coarse_body}


def _oracle(case):
    return fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, case.ref_xy, case.tris,
                            coupling="exact")


def _coupling_matches(g, case):
    rows, cols, vals = g.get_coupling()
    grid = fo.FluidGrid(case.N)
    C = fo.assemble_coupling_exact(grid, case.ref_xy, case.tris.astype(np.int64), case.X0)
    C = C.tocsc()[:, grid.interior_nodes].tocsr()
    G = sp.coo_matrix((vals, (rows, np.searchsorted(grid.interior_nodes, cols))), shape=C.shape).tocsr()
    assert abs(G - C).max() <= 1e-13 * abs(C).max()


@pytest.mark.parametrize("name", list(CASES))
def test_exact_coupling_matrix(fsi, name):
    case = CASES[name]()
    g = fsi.problem_from_case(case, coupling=1)
    g.assemble_step()
    _coupling_matches(g, case)
    with pytest.raises(fsi.FsiError):   # the exact rule locates no points
        g.get_points()
    g.close()


@pytest.mark.parametrize("name", list(CASES))
def test_exact_coupling_one_step_fp64(fsi, name):
    case = CASES[name]()
    g = fsi.problem_from_case(case, precision=0, precond=1, rtol=1e-12, coupling=1)
    info = g.step()
    assert info.rel_residual <= 1e-12
    u, p, X, lam = g.get_state()
    o = _oracle(case)
    uo, po, Xo, lamo = o.step(case.u0, case.X0)
    assert rel(u, uo) < 1e-7
    assert rel(p, po) < 1e-7
    assert rel(X - case.X0, Xo - case.X0) < 1e-7
    assert rel(lam, lamo) < 1e-7
    g.close()


def test_exact_coupling_bench_workload(fsi):
    """The N = 128 cavity in the bench's mixed configuration with the exact
    rule: C_f entry by entry, the operator and right-hand side, and a step
    whose residual in the oracle's operator meets 1e-8."""
    case = fi.cavity128_case()
    g = fsi.problem_from_case(case, precision=1, precond=bench.PRECOND, rtol=1e-8, max_it=bench.MAX_IT,
                              stokes_its=bench.STOKES_ITS, coupling=1, **bench.arm_settings(1))
    g.assemble_step()
    _coupling_matches(g, case)
    o = _oracle(case)
    K, rhs, _ = o.system(case.u0, case.X0)
    q = oracle_to_gpu_perm(o, g)
    x = np.random.default_rng(2).standard_normal(K.shape[0])
    assert rel(g.apply_operator(x[q], precision=0), (K @ x)[q]) < 1e-13
    assert rel(g.get_rhs(), rhs[q]) < 1e-13
    info = g.step()
    assert info.status == 0 and info.rel_residual <= 1e-8
    u, p, X, lam = g.get_state()
    assert o.relative_residual(case.u0, case.X0, u, p, X, lam) <= 1e-8 * (1 + 1e-6)
    g.close()
