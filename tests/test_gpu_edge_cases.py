"""Edge and degenerate cases through the C ABI: invalid and empty inputs are
refused on the host, a body leaving the fluid domain and NaN data end the
step with their status codes (no fault), solid vertices lying exactly on
fluid grid lines and on the wall are located and clipped like the oracle
does, and the body at rest stays at rest."""
import numpy as np
import pytest
import scipy.sparse as sp

import fsi_inputs as fi
from oracle import fsi_oracle as fo
from tests.gpu_helpers import rel

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


def test_invalid_parameters_and_empty_mesh_are_refused(fsi):
    case = fi.disk16_case()
    for kw in (dict(N=15), dict(N=18), dict(N=0)):          # odd, c > 8, empty grid
        prm = fsi.make_params(kw["N"], 1.0, 1.0, 10.0, 0.01)
        with pytest.raises(fsi.FsiError) as e:
            fsi.Problem(prm, case.ref_xy, case.tris)
        assert e.value.code == fsi.FSI_ERR_INVALID
    prm = fsi.make_params(16, 1.0, 1.0, 10.0, 0.01)
    with pytest.raises(fsi.FsiError) as e:                   # no triangles
        fsi.Problem(prm, case.ref_xy, np.zeros((0, 3), dtype=np.int32))
    assert e.value.code == fsi.FSI_ERR_INVALID
    with pytest.raises(fsi.FsiError) as e:                   # dt <= 0
        fsi.Problem(fsi.make_params(16, 1.0, 1.0, 10.0, 0.0), case.ref_xy, case.tris)
    assert e.value.code == fsi.FSI_ERR_INVALID


def test_budget_refusal_allocates_nothing(fsi):
    case = fi.cavity128_case()
    prm = fsi.make_params(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, precision=1)
    need = fsi.footprint_bytes(prm, case.ref_xy.shape[0], case.tris.shape[0])
    assert need > 0
    with pytest.raises(fsi.FsiError) as e:
        fsi.Problem(prm, case.ref_xy, case.tris, u0=case.u0, X0=case.X0, budget_bytes=need // 2)
    assert e.value.code == fsi.FSI_ERR_BUDGET


@pytest.mark.parametrize("coupling", [0, 1])
def test_body_outside_the_domain_reports_out_of_domain(fsi, coupling):
    case = fi.disk16_case()
    X0 = case.X0.copy()
    X0[:, 0] += 0.45                                        # the disk crosses x = 1
    g = fsi.Problem(fsi.make_params(case.N, 1.0, 1.0, 10.0, 0.01, coupling=coupling), case.ref_xy, case.tris,
                    u0=case.u0, X0=X0)
    with pytest.raises(fsi.FsiError) as e:
        g.step()
    assert e.value.code == fsi.FSI_ERR_OUT_OF_DOMAIN
    g.close()


def test_nan_velocity_reports_nan(fsi):
    case = fi.disk16_case()
    u0 = case.u0.copy()
    u0[len(u0) // 2] = np.nan
    g = fsi.Problem(fsi.make_params(case.N, 1.0, 1.0, 10.0, 0.01, precond=1), case.ref_xy, case.tris, u0=u0,
                    X0=case.X0)
    with pytest.raises(fsi.FsiError) as e:
        g.step()
    assert e.value.code == fsi.FSI_ERR_NAN
    g.close()


def test_vertices_on_grid_lines_and_wall(fsi):
    """The bar [0,0.4] x [0.45,0.55] on N = 20: every vertex row lies on a
    fluid grid line (y = 9/20, 11/20, x = k/20) and the left edge on the wall
    x = 0.  Point location is bit-exact, and both coupling rules match the
    oracle's, whose clipping meets these degenerate pieces too."""
    xy, tris = fi.bar_mesh(8, 2)
    case = fi.FsiCase(N=20, rho_f=1.0, nu=0.2, kappa=5.0, dt=0.002, lid_u=0.0, ref_xy=xy, tris=tris,
                      u0=fi.initial_velocity(20, 5), X0=xy.copy(), precond=1, rtol=1e-12)
    grid = fo.FluidGrid(20)
    t64 = tris.astype(np.int64)
    for coupling in (0, 1):
        g = fsi.problem_from_case(case, coupling=coupling)
        g.assemble_step()
        if coupling == 0:
            cell, xi, eta = g.get_points()
            ocell, oxi, oeta = fo.locate_brute_force(fo.quadrature_points(case.X0, t64), 20)
            assert np.array_equal(cell, ocell) and np.array_equal(xi, oxi) and np.array_equal(eta, oeta)
            C, _ = fo.assemble_coupling(grid, xy, t64, case.X0)
        else:
            C = fo.assemble_coupling_exact(grid, xy, t64, case.X0)
        rows, cols, vals = g.get_coupling()
        Ci = C.tocsc()[:, grid.interior_nodes].tocsr()
        G = sp.coo_matrix((vals, (rows, np.searchsorted(grid.interior_nodes, cols))), shape=Ci.shape).tocsr()
        assert abs(G - Ci).max() <= 1e-13 * abs(Ci).max()
        info = g.step()
        assert info.status == 0
        o = fo.OracleProblem(20, 1.0, 0.2, 5.0, 0.002, 0.0, xy, tris, coupling="exact" if coupling else "point")
        u, p, X, lam = g.get_state()
        uo, po, Xo, lamo = o.step(case.u0, case.X0)
        assert rel(u, uo) < 1e-7 and rel(lam, lamo) < 1e-7
        g.close()


def test_body_at_rest_stays_at_rest(fsi):
    """kappa = 0, fluid and walls at rest, X0 = s: the step leaves u = 0 and
    X = s (up to the solve's tolerance)."""
    xy, tris = fi.ring_disk_mesh(5, 0.2, (0.5, 0.5))
    case = fi.FsiCase(N=16, rho_f=1.0, nu=1.0, kappa=0.0, dt=0.01, lid_u=0.0, ref_xy=xy, tris=tris,
                      u0=fi.wall_velocity(16, 0.0), X0=xy.copy(), precond=1, rtol=1e-12)
    g = fsi.problem_from_case(case, precision=0)
    g.step()
    u, p, X, lam = g.get_state()
    assert np.max(np.abs(u)) < 1e-9
    assert np.max(np.abs(X - xy)) < 1e-9
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_iteration_cap_reports_not_converged(fsi, precision):
    """max_it = 2 Krylov iterations cannot reach a 1e-12 residual: the step
    ends with FSI_ERR_NOT_CONVERGED and reports the two iterations it took."""
    case = fi.disk16_case()
    g = fsi.problem_from_case(case, precision=precision, precond=1, rtol=1e-12, max_it=2)
    g.assemble_step()
    info = g.solve_step(check=False)
    assert info.status == fsi.FSI_ERR_NOT_CONVERGED
    assert info.iterations == 2 and info.rel_residual > 1e-12
    g.close()


@pytest.mark.parametrize("coupling", [0, 1])
def test_row_over_capacity_reports_capacity(fsi, coupling):
    """A coupling row holds the lattice nodes of the cells its triangles
    overlap in the reference configuration.  A body stretched 2.2 times about
    its centre (still inside the domain) makes the central node's row need
    far more: both coupling rules end the step with FSI_ERR_CAPACITY."""
    xy, tris = fi.ring_disk_mesh(2, 0.2, (0.5, 0.5))
    g = fsi.Problem(fsi.make_params(16, 1.0, 1.0, 10.0, 0.01, precond=1, coupling=coupling), xy, tris,
                    u0=fi.wall_velocity(16, 0.0), X0=xy)
    g.set_state(None, 0.5 + 2.2 * (xy - 0.5))
    g.assemble_step()
    info = g.solve_step(check=False)
    assert info.status == fsi.FSI_ERR_CAPACITY
    g.close()


def test_restart_and_stokes_steps_above_their_limits_are_refused(fsi):
    """restart > 250 (one Hessenberg column lives in shared memory), more
    than 16 inner Stokes steps and a coarsest grid above 32 cells are
    refused at creation, not clamped."""
    case = fi.disk16_case()
    for kw in (dict(restart=251), dict(stokes_its=17), dict(mg_coarse=33), dict(mg_coarse_p=33)):
        with pytest.raises(fsi.FsiError) as e:
            fsi.problem_from_case(case, **kw)
        assert e.value.code == fsi.FSI_ERR_INVALID
    fsi.problem_from_case(case, restart=250, stokes_its=16, mg_coarse=32, mg_coarse_p=32).close()
