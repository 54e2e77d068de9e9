"""The fused matrix-free multigrid levels (fsi_mgfused.cuh: two launches per
V-cycle level on the finest levels of the FP32 hierarchy) against the
per-level sparse kernels on the assembled level matrices (mg_fused = -1):
the same preconditioner of Section 5 (V-cycles with Chebyshev-Jacobi
smoothing inside the block preconditioner) up to FP32 rounding, with fewer
kernel nodes per Arnoldi step, for every block preconditioner, with and
without the cluster-resident coarse levels, and a solve with them reaches
the time step's tolerance in the oracle's own operator."""
import numpy as np
import pytest

import bench
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


def _ragged():
    xy, tris = fi.ring_disk_mesh(9, 0.23, (0.47, 0.52))
    return fi.FsiCase(N=24, rho_f=1.3, nu=0.05, kappa=30.0, dt=0.005, lid_u=1.0, ref_xy=xy, tris=tris,
                      u0=fi.initial_velocity(24, 7, lid_u=1.0), X0=xy.copy(), precond=2, rtol=1e-12)


def _ragged48():
    """N = 48 = 3 * 2^4: levels 48, 24 fused, 12 and 6 below (odd coarsening)."""
    xy, tris = fi.ring_disk_mesh(12, 0.21, (0.52, 0.47))
    return fi.FsiCase(N=48, rho_f=1.0, nu=0.02, kappa=300.0, dt=0.002, lid_u=1.0, ref_xy=xy, tris=tris,
                      u0=fi.initial_velocity(48, 9, lid_u=1.0), X0=xy.copy(), precond=2, rtol=1e-12)


CASES = {"disk16": fi.disk16_case, "ragged24": _ragged, "ragged48": _ragged48, "lidbody16": fi.lid_body_case,
         "cavity128": fi.cavity128_case, "ellipse256": lambda: fi.ellipse_case(256)}


@pytest.mark.parametrize("mg_cluster", [0, -1])
@pytest.mark.parametrize("precond,stokes_its", [(0, 1), (1, 1), (2, 1), (2, bench.STOKES_ITS), (3, 2)])
@pytest.mark.parametrize("name", list(CASES))
def test_fused_levels_match_per_level_kernels(fsi, name, precond, stokes_its, mg_cluster):
    case = CASES[name]()
    kw = dict(precision=1, precond=precond, stokes_its=stokes_its, restart=bench.RESTART, mg_cluster=mg_cluster)
    on = fsi.problem_from_case(case, mg_fused=0, **kw)
    off = fsi.problem_from_case(case, mg_fused=-1, **kw)
    on.assemble_step()
    off.assemble_step()
    # with the cluster off on both sides every level of 16 cells or more above
    # the coarsest takes two fused launches instead of the per-level kernels
    # (with mg_cluster = 0 the per-level side may hold its coarse levels in
    # one cluster launch, the fused side does not)
    # (a 16-cell problem is its own coarsest grid)
    if mg_cluster == -1 and case.N > 16:
        assert on.graph_kernel_counts()[3] < off.graph_kernel_counts()[3]
    rng = np.random.default_rng(17)
    for _ in range(2):
        v = rng.standard_normal(on.n)
        assert rel(on.apply_preconditioner(v, precision=1), off.apply_preconditioner(v, precision=1)) < 2e-5
        # the FP64 preconditioner does not use the fused kernels
        assert rel(on.apply_preconditioner(v, precision=0), off.apply_preconditioner(v, precision=0)) < 1e-12
    on.close()
    off.close()


@pytest.mark.parametrize("degree", [1, 3, 4])
def test_fused_levels_other_smoothing_degrees(fsi, degree):
    case = fi.cavity128_case()
    kw = dict(precision=1, precond=bench.PRECOND, stokes_its=2, restart=bench.RESTART, mg_degree=degree)
    on = fsi.problem_from_case(case, mg_fused=0, **kw)
    off = fsi.problem_from_case(case, mg_fused=-1, **kw)
    on.assemble_step()
    off.assemble_step()
    v = np.random.default_rng(3).standard_normal(on.n)
    assert rel(on.apply_preconditioner(v, precision=1), off.apply_preconditioner(v, precision=1)) < 2e-5
    on.close()
    off.close()


def test_fused_bench_step_meets_the_oracle_operator(fsi):
    """The bench workload's mixed step with the fused levels: the solution's
    residual in the oracle's FP64 operator is below the 1e-8 tolerance."""
    case = fi.cavity128_case()
    g = fsi.problem_from_case(case, precision=1, precond=bench.PRECOND, rtol=1e-8, max_it=bench.MAX_IT,
                              stokes_its=bench.STOKES_ITS, mg_fused=0, **bench.arm_settings(1))
    info = g.step()
    assert info.status == 0 and info.rel_residual <= 1e-8
    u, p, X, lam = g.get_state()
    o = fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, case.ref_xy, case.tris)
    assert o.relative_residual(case.u0, case.X0, u, p, X, lam) <= 1e-8 * (1 + 1e-6)
    g.close()
