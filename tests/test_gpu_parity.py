"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: point-location cells and local coordinates.  Floating point:
coupling entries and operator products to 1e-13 relative (same FP64
arithmetic, different summation order); one time step to 1e-7 relative L2
per block with a 1e-12 solve, and the GPU solution's residual in the
oracle's own operator below the requested tolerance.
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


def _deformed_case(N=24, m=9, seed=7):
    """A ragged case: N = 3 * 2^3, solid sheared and rotated, u_0 random, lid."""
    xy, tris = fi.ring_disk_mesh(m, 0.23, (0.47, 0.52))
    c, s = np.cos(0.3), np.sin(0.3)
    d = xy - np.array([0.47, 0.52])
    X0 = np.stack([c * d[:, 0] - s * d[:, 1] + 0.2 * d[:, 1], s * d[:, 0] + c * d[:, 1]], 1) + np.array([0.47, 0.52])
    return fi.FsiCase(N=N, rho_f=1.3, nu=0.05, kappa=30.0, dt=0.005, lid_u=1.0, ref_xy=xy, tris=tris,
                      u0=fi.initial_velocity(N, seed, lid_u=1.0), X0=X0, precond=1, rtol=1e-12)


# lidbody16: rule points in the top row of cells under a moving lid, so the
# wall columns of C_f enter the right-hand side (g2 = -(1/dt) C_s X^n - C_D u_D)
CASES = {"disk16": fi.disk16_case, "ragged24": _deformed_case, "lidbody16": fi.lid_body_case}


@pytest.mark.parametrize("name", list(CASES))
def test_point_location_is_bit_exact(fsi, name):
    case = CASES[name]()
    g = fsi.problem_from_case(case)
    g.assemble_step()
    cell, xi, eta = g.get_points()
    x = fo.quadrature_points(case.X0, case.tris.astype(np.int64))
    ocell, oxi, oeta = fo.locate_brute_force(x, case.N)
    assert np.array_equal(cell, ocell)
    assert np.array_equal(xi, oxi) and np.array_equal(eta, oeta)
    g.close()


@pytest.mark.parametrize("name", list(CASES))
def test_coupling_matrix(fsi, name):
    case = CASES[name]()
    g = fsi.problem_from_case(case)
    g.assemble_step()
    rows, cols, vals = g.get_coupling()
    o = _oracle(case)
    C, _ = fo.assemble_coupling(o.grid, case.ref_xy, case.tris.astype(np.int64), case.X0)
    C = C.tocsc()[:, o.grid.interior_nodes].tocsr()
    G = sp.coo_matrix((vals, (rows, np.searchsorted(o.grid.interior_nodes, cols))), shape=C.shape).tocsr()
    assert abs(G - C).max() <= 1e-13 * abs(C).max()
    g.close()


@pytest.mark.parametrize("name", list(CASES))
def test_operator_and_rhs(fsi, name):
    case = CASES[name]()
    for precision in (0, 1):
        g = fsi.problem_from_case(case, precision=precision)
        g.assemble_step()
        o = _oracle(case)
        K, rhs, _ = o.system(case.u0, case.X0)
        q = oracle_to_gpu_perm(o, g)
        rng = np.random.default_rng(3)
        x = rng.standard_normal(K.shape[0])
        y_ref = (K @ x)[q]
        y = g.apply_operator(x[q], precision=0)
        assert rel(y, y_ref) < 1e-13
        if precision == 1:
            y32 = g.apply_operator(x[q], precision=1)
            assert rel(y32, y_ref) < 1e-5
        b = g.get_rhs()
        assert rel(b, rhs[q]) < 1e-13
        g.close()


@pytest.mark.parametrize("precond,stokes_its", [(0, 1), (1, 1), (2, 1), (1, 4), (2, 8)])
@pytest.mark.parametrize("name", list(CASES))
def test_one_step_fp64_matches_oracle(fsi, name, precond, stokes_its):
    """Every preconditioner (block-diagonal, lower and upper block-triangular,
    with one V-cycle pair or inner Richardson steps on the Stokes block)
    gives the oracle's solution of Eq. (matrix)."""
    case = CASES[name]()
    g = fsi.problem_from_case(case, precision=0, precond=precond, rtol=1e-12, stokes_its=stokes_its)
    info = g.step()
    assert info.rel_residual <= 1e-12
    u, p, X, lam = g.get_state()
    o = _oracle(case)
    uo, po, Xo, lamo = o.step(case.u0, case.X0)
    assert rel(u, uo) < 1e-7
    assert rel(p, po) < 1e-7
    assert rel(X - case.X0, Xo - case.X0) < 1e-7
    assert rel(lam, lamo) < 1e-7
    assert o.relative_residual(case.u0, case.X0, u, p, X, lam) < 1e-10
    g.close()


@pytest.mark.parametrize("precond,stokes_its", [(1, 1), (2, 8)])
@pytest.mark.parametrize("name", list(CASES))
def test_one_step_mixed_precision(fsi, name, precond, stokes_its):
    """FP32 operators and preconditioner inside FP64 refinement reach the
    same 1e-8 residual; the error against the FP64 oracle is reported."""
    case = CASES[name]()
    g = fsi.problem_from_case(case, precision=1, rtol=1e-8, precond=precond, stokes_its=stokes_its)
    info = g.step()
    assert info.rel_residual <= 1e-8
    u, p, X, lam = g.get_state()
    o = _oracle(case)
    assert o.relative_residual(case.u0, case.X0, u, p, X, lam) < 1e-8
    uo, po, Xo, lamo = o.step(case.u0, case.X0)
    assert rel(u, uo) < 1e-5
    assert rel(lam, lamo) < 1e-5
    g.close()


def test_five_step_trajectory(fsi):
    case = fi.disk16_case()
    g = fsi.problem_from_case(case, precision=0, precond=1, rtol=1e-12)
    o = _oracle(case)
    u, X = case.u0, case.X0
    for _ in range(5):
        g.step()
        u, p, X, lam = o.step(u, X)
    ug, pg, Xg, lamg = g.get_state()
    assert rel(ug, u) < 1e-7
    assert rel(Xg - case.X0, X - case.X0) < 1e-7
    assert rel(lamg, lam) < 1e-7
    g.close()


@pytest.mark.parametrize("precond", [0, 1])
def test_quarter_annulus_one_step(fsi, precond):
    """The linear-solid test geometry of Section 6 (quarter annulus released
    from its stretched state; edges on the walls x = 0 and y = 0)."""
    case = fi.annulus_case(16)
    g = fsi.problem_from_case(case, precision=0, precond=precond, rtol=1e-12)
    info = g.step()
    assert info.rel_residual <= 1e-12
    u, p, X, lam = g.get_state()
    uo, po, Xo, lamo = _oracle(case).step(case.u0, case.X0)
    assert rel(u, uo) < 1e-7
    assert rel(X - case.X0, Xo - case.X0) < 1e-7
    assert rel(lam, lamo) < 1e-7
    g.close()


@pytest.mark.parametrize("N,mg_coarse", [(4, 0), (6, 0), (8, 0), (12, 0), (12, 8), (12, 4)])
def test_tiny_grids(fsi, N, mg_coarse):
    """Degenerate hierarchies: with the default coarsest grid (16 cells) every
    N here is a single level (the V-cycle is the dense inverse, no cluster
    suffix); N = 12 with mg_coarse 8 coarsens once (12, 6), with mg_coarse 4
    twice, to an odd grid (12, 6, 3)."""
    xy, tris = fi.ring_disk_mesh(3, 0.2, (0.5, 0.5))
    case = fi.FsiCase(N=N, rho_f=1.0, nu=0.5, kappa=10.0, dt=0.01, lid_u=1.0, ref_xy=xy, tris=tris,
                      u0=fi.initial_velocity(N, 11, lid_u=1.0), X0=xy.copy(), precond=1, rtol=1e-12)
    for precision, tol in ((0, 1e-7), (1, 1e-5)):
        g = fsi.problem_from_case(case, precision=precision, rtol=1e-12 if precision == 0 else 1e-9,
                                  mg_coarse=mg_coarse)
        info = g.step()
        assert info.status == 0
        u, p, X, lam = g.get_state()
        uo, po, Xo, lamo = _oracle(case).step(case.u0, case.X0)
        assert rel(u, uo) < tol
        assert rel(lam, lamo) < tol
        g.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-5)])
@pytest.mark.parametrize("name", ["disk16", "lidbody16"])
def test_coarsest_inverse_is_the_velocity_solve(fsi, name, precision, tol):
    """A 16-cell grid with mg_coarse = 16 is a one-level hierarchy: the
    V-cycle is the dense inverse that Gauss-Jordan builds on the device.  The
    velocity part of the preconditioner (precond 3, one Stokes step, v with
    velocity entries only, so the solid and multiplier parts are zero) is
    then A_II^-1 v_u, A_II the oracle's assembled velocity block (Section 5:
    the first block of A_11), solved here by scipy's sparse LU."""
    import scipy.sparse.linalg as spla
    case = CASES[name]()
    g = fsi.problem_from_case(case, precision=precision, precond=3, stokes_its=1, mg_coarse=16)
    g.assemble_step()
    o = _oracle(case)
    K, _, _ = o.system(case.u0, case.X0)
    q = oracle_to_gpu_perm(o, g)
    nu = g.n_u
    rng = np.random.default_rng(5)
    vo = np.zeros(K.shape[0])
    vo[:nu] = rng.standard_normal(nu)
    zo = np.zeros(K.shape[0])
    zo[:nu] = spla.spsolve(sp.csc_matrix(K)[:nu, :nu], vo[:nu])
    z = g.apply_preconditioner(vo[q], precision=precision)
    assert rel(z[:nu], zo[q][:nu]) < tol
    g.close()


def test_symmetric_annulus_one_step_is_mirror_symmetric(fsi):
    """The full annulus that carries the quarter problem's free-slip walls by
    symmetry: the GPU step matches the oracle and is mirror-symmetric."""
    from scipy.spatial import cKDTree
    case = fi.symmetric_annulus_case(8)
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
