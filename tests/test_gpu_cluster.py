"""The cluster-resident coarse multigrid levels (one thread-block-cluster
launch per V-cycle for the levels that fit in shared memory) against the
per-level kernels: the same preconditioner (Section 5: V-cycles with
Chebyshev-Jacobi smoothing inside the block preconditioner), so the two
applications agree to rounding, and the solve with the cluster path still
meets the oracle."""
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


CASES = {"disk16": fi.disk16_case, "ragged24": _ragged, "cavity128": fi.cavity128_case, "ellipse256": lambda: fi.ellipse_case(256)}


def _pair(fsi, case, precision, precond, stokes_its):
    # the per-level sparse kernels above the cluster (an FP32 hierarchy with
    # the fused matrix-free levels leaves the cluster out by default), and an
    # 8-cell coarsest grid (the default stops at 16 cells, and a 16-cell
    # problem then has no level for the cluster)
    kw = dict(precision=precision, precond=precond, stokes_its=stokes_its, restart=bench.RESTART, mg_fused=-1,
              mg_coarse=8)
    on = fsi.problem_from_case(case, mg_cluster=0, **kw)
    off = fsi.problem_from_case(case, mg_cluster=-1, **kw)
    on.assemble_step()
    off.assemble_step()
    return on, off


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_cluster_levels_match_per_level_kernels(fsi, name, precision):
    case = CASES[name]()
    on, off = _pair(fsi, case, precision, bench.PRECOND, bench.STOKES_ITS)
    # the cluster path is taken: fewer kernel nodes per Arnoldi step
    assert on.graph_kernel_counts()[3] < off.graph_kernel_counts()[3]
    rng = np.random.default_rng(11)
    for _ in range(2):
        v = rng.standard_normal(on.n)
        for p in sorted({0, precision}):
            z_on = on.apply_preconditioner(v, precision=p)
            z_off = off.apply_preconditioner(v, precision=p)
            assert rel(z_on, z_off) < (1e-12 if p == 0 else 2e-5)
    on.close()
    off.close()


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_cluster_solve_meets_oracle(fsi, precond):
    case = _ragged()
    g = fsi.problem_from_case(case, precision=0, precond=precond, rtol=1e-12, stokes_its=4, mg_cluster=0)
    info = g.step()
    assert info.rel_residual <= 1e-12
    u, p, X, lam = g.get_state()
    o = fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, case.ref_xy, case.tris)
    uo, po, Xo, lamo = o.step(case.u0, case.X0)
    assert rel(u, uo) < 1e-7
    assert rel(lam, lamo) < 1e-7
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["cavity128", "ellipse256"])
def test_autotuned_tiles_match_fixed_tiles(fsi, name, precision):
    """The autotuner only changes how the per-level SpMV splits a row over
    threads (the summation order): the preconditioner is the same to
    rounding."""
    case = CASES[name]()
    kw = dict(precision=precision, precond=bench.PRECOND, stokes_its=bench.STOKES_ITS, restart=bench.RESTART)
    tuned = fsi.problem_from_case(case, autotune=1, **kw)
    fixed = fsi.problem_from_case(case, autotune=0, **kw)
    tuned.assemble_step()
    fixed.assemble_step()
    v = np.random.default_rng(5).standard_normal(tuned.n)
    for p in sorted({0, precision}):
        assert rel(tuned.apply_preconditioner(v, precision=p), fixed.apply_preconditioner(v, precision=p)) < (
            1e-12 if p == 0 else 2e-5)
    tuned.close()
    fixed.close()
