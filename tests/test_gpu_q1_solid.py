"""The Q1 quadrilateral solid of the annulus test (Section 6) on the GPU
against the oracle's restatement: the rule points located bit for bit (same
rounding-fixed bilinear map, same half-open cell rule), C_f to 1e-13, the
operator and right-hand side to 1e-13, one time step to 1e-7 relative at a
1e-12 solve for every preconditioner, the mirrored full annulus, mixed
precision at the annulus workload size, and the parameter combinations the
Q1 solid refuses.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


def _oracle(case):
    return fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, case.ref_xy, case.tris)


def _sheared():
    """A quad mesh moved by a shear and rotation, on a ragged grid (N = 20),
    with a wall lid: rule points in many cells and on both sides of lines."""
    xy, quads = fi.annulus_mesh(3, 7, quads=True)
    xy = 0.15 + 0.8 * xy
    c, s = np.cos(0.35), np.sin(0.35)
    d = xy - 0.4
    X0 = np.stack([c * d[:, 0] - s * d[:, 1] + 0.2 * d[:, 1], s * d[:, 0] + c * d[:, 1]], 1) + 0.45
    return fi.FsiCase(N=20, rho_f=1.2, nu=0.05, kappa=25.0, dt=0.005, lid_u=1.0, ref_xy=xy, tris=quads,
                      u0=fi.initial_velocity(20, 5, lid_u=1.0), X0=X0, precond=1, rtol=1e-12)


CASES = {"annulus16": lambda: fi.annulus_case(16, quads=True), "sheared20": _sheared}


@pytest.mark.parametrize("name", list(CASES))
def test_points_bit_exact_and_coupling(fsi, name):
    case = CASES[name]()
    g = fsi.problem_from_case(case)
    g.assemble_step()
    cell, xi, eta = g.get_points()
    grid = fo.FluidGrid(case.N)
    C, (xq, ocell, oxi, oeta) = fo.assemble_coupling(grid, case.ref_xy, case.tris.astype(np.int64), case.X0)
    assert np.array_equal(cell, ocell)
    assert np.array_equal(xi, oxi) and np.array_equal(eta, oeta)
    rows, cols, vals = g.get_coupling()
    Ci = C.tocsc()[:, grid.interior_nodes].tocsr()
    G = sp.coo_matrix((vals, (rows, np.searchsorted(grid.interior_nodes, cols))), shape=Ci.shape).tocsr()
    assert abs(G - Ci).max() <= 1e-13 * abs(Ci).max()
    g.close()


@pytest.mark.parametrize("name", list(CASES))
def test_operator_and_rhs(fsi, name):
    case = CASES[name]()
    g = fsi.problem_from_case(case)
    g.assemble_step()
    o = _oracle(case)
    K, rhs, _ = o.system(case.u0, case.X0)
    q = oracle_to_gpu_perm(o, g)
    x = np.random.default_rng(3).standard_normal(K.shape[0])
    assert rel(g.apply_operator(x[q], precision=0), (K @ x)[q]) < 1e-13
    assert rel(g.get_rhs(), rhs[q]) < 1e-13
    g.close()


@pytest.mark.parametrize("precond", [0, 1, 2])
@pytest.mark.parametrize("name", list(CASES))
def test_one_step_fp64(fsi, name, precond):
    case = CASES[name]()
    g = fsi.problem_from_case(case, precision=0, precond=precond, rtol=1e-12)
    info = g.step()
    assert info.rel_residual <= 1e-12
    u, p, X, lam = g.get_state()
    uo, po, Xo, lamo = _oracle(case).step(case.u0, case.X0)
    assert rel(u, uo) < 1e-7
    assert rel(X - case.X0, Xo - case.X0) < 1e-7
    assert rel(lam, lamo) < 1e-7
    g.close()


def test_symmetric_annulus_q1(fsi):
    """The full annulus with Q1 elements (free-slip quarter by symmetry):
    oracle parity and mirror symmetry of the displacement."""
    from scipy.spatial import cKDTree
    case = fi.symmetric_annulus_case(8, quads=True)
    g = fsi.problem_from_case(case, precision=0, precond=1, rtol=1e-12)
    g.step()
    u, p, X, lam = g.get_state()
    uo, po, Xo, lamo = _oracle(case).step(case.u0, case.X0)
    assert rel(X - case.X0, Xo - case.X0) < 1e-7
    assert rel(lam, lamo) < 1e-7
    mirror = case.ref_xy.copy()
    mirror[:, 0] = 1.0 - mirror[:, 0]
    idx = cKDTree(case.ref_xy).query(mirror)[1]
    D = X - case.X0
    assert np.max(np.abs(D[idx, 0] + D[:, 0])) <= 1e-8 * np.max(np.abs(D))
    assert np.max(np.abs(D[idx, 1] - D[:, 1])) <= 1e-8 * np.max(np.abs(D))
    g.close()


def test_mixed_precision_annulus48(fsi):
    """The annulus workload size in the mixed arm: the step meets 1e-8 in the
    oracle's operator."""
    case = fi.annulus_case(48, quads=True)
    g = fsi.problem_from_case(case, precision=1, precond=2, rtol=1e-8, stokes_its=4, restart=60)
    info = g.step()
    assert info.status == 0 and info.rel_residual <= 1e-8
    u, p, X, lam = g.get_state()
    assert _oracle(case).relative_residual(case.u0, case.X0, u, p, X, lam) <= 1e-8 * (1 + 1e-6)
    g.close()


def test_q1_refusals_and_footprint(fsi):
    case = CASES["annulus16"]()
    with pytest.raises(fsi.FsiError):
        fsi.problem_from_case(case, coupling=1)
    with pytest.raises(fsi.FsiError):
        fsi.problem_from_case(case, solid_law=1, gamma=1.0, eta=1.0)
    prm = fsi.make_params(case.N, case.rho_f, case.nu, case.kappa, case.dt, solid_elem=1)
    assert fsi.footprint_bytes(prm, case.ref_xy.shape[0], case.tris.shape[0]) > 0
