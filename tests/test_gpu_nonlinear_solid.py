"""The nonlinear solid law of the bar test (Section 6: exponential strain
energy, each time step solved by Newton's method) on the GPU against the
oracle's Newton iteration on the same discrete problem.

Tight tolerances on both sides (linear solves to 1e-12, Newton to 1e-12)
make both converge to the same nonlinear solution: states agree to 1e-7
relative.  At the workload size the converged state's nonlinear residual is
checked in the oracle's operator instead.
"""
import numpy as np
import pytest

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


def _oracle(case, tol=1e-12):
    x = case.extra
    return fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, case.ref_xy, case.tris,
                            solid_law="exp", gamma=x["gamma"], eta=x["eta"], newton_tol=tol)


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_bar_one_step_fp64_matches_oracle(fsi, precond):
    case = fi.bar_case(N=16, nx=8, ny=2)
    g = fsi.problem_from_case(case, precision=0, precond=precond, rtol=1e-12, newton_tol=1e-12, stokes_its=4)
    info = g.step()
    assert info.status == 0 and info.newton_iterations >= 2
    u, p, X, lam = g.get_state()
    o = _oracle(case)
    uo, po, Xo, lamo = o.step(case.u0, case.X0)
    assert rel(u, uo) < 1e-7
    assert rel(p, po) < 1e-7
    assert rel(X - case.X0, Xo - case.X0) < 1e-7
    assert rel(lam, lamo) < 1e-7
    g.close()


def test_bar_three_step_trajectory(fsi):
    case = fi.bar_case(N=16, nx=8, ny=2)
    g = fsi.problem_from_case(case, precision=0, precond=1, rtol=1e-12, newton_tol=1e-12)
    o = _oracle(case)
    u, X = case.u0, case.X0
    for _ in range(3):
        g.step()
        u, p, X, lam = o.step(u, X)
    ug, pg, Xg, lamg = g.get_state()
    assert rel(ug, u) < 1e-7
    assert rel(Xg - case.X0, X - case.X0) < 1e-7
    assert rel(lamg, lam) < 1e-7
    g.close()


def test_bar_mixed_precision(fsi):
    """FP32 operators inside FP64 refinement, Newton to the default 1e-6: the
    state is a converged nonlinear solution to the solve's tolerance."""
    case = fi.bar_case(N=32, nx=16, ny=4)
    g = fsi.problem_from_case(case, precision=1, precond=2, rtol=1e-10, stokes_its=4, restart=60)
    info = g.step()
    assert info.status == 0 and 2 <= info.newton_iterations <= 6
    u, p, X, lam = g.get_state()
    o = _oracle(case, tol=1e-6)
    assert o.relative_residual(case.u0, case.X0, u, p, X, lam) < 1e-7
    uo, po, Xo, lamo = o.step(case.u0, case.X0)
    assert rel(X - case.X0, Xo - case.X0) < 1e-5
    g.close()


def test_nonlinear_law_rejects_unsupported_paths(fsi):
    case = fi.bar_case(N=16, nx=8, ny=2)
    g = fsi.problem_from_case(case, precision=0)
    with pytest.raises(fsi.FsiError):      # Newton needs the host between solves
        g.step_async()
    g.close()
    with pytest.raises(fsi.FsiError):      # the law needs gamma, eta > 0
        fsi.problem_from_case(case, precision=0, gamma=0.0)
