"""Batched and served instances give the same results as instances run
alone (every reduction in the library has a fixed order, so the results are
bit-identical), and admission by footprint refuses what does not fit."""
import numpy as np
import pytest

import fsi_inputs as fi

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


def _cases():
    out = []
    for i, (N, m, R) in enumerate(((16, 5, 0.2), (32, 8, 0.15), (24, 6, 0.25))):
        xy, tris = fi.ring_disk_mesh(m, R, (0.5, 0.48))
        out.append(fi.FsiCase(N=N, rho_f=1.0, nu=0.1 * (i + 1), kappa=10.0 ** (i + 1), dt=0.01, lid_u=1.0,
                              ref_xy=xy, tris=tris, u0=fi.initial_velocity(N, 77 + i, lid_u=1.0), X0=xy.copy(),
                              precond=2, rtol=1e-10))
    return out


def _alone(fsi, case, steps, **kw):
    p = fsi.problem_from_case(case, precision=1, **kw)
    for _ in range(steps):
        p.step()
    st = p.get_state()
    p.close()
    return st


def test_batch_step_equals_alone(fsi):
    cases = _cases()
    probs = [fsi.problem_from_case(c, precision=1) for c in cases]
    for _ in range(3):
        st, infos = fsi.step_batch(probs)
        assert st == 0 and all(i.status == 0 for i in infos)
    for c, p in zip(cases, probs):
        ref = _alone(fsi, c, 3)
        got = p.get_state()
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        p.close()


def test_served_mix_equals_alone(fsi):
    from paper_2301_10041_gb300.serve import Request, Server, gpu_ops
    cases = _cases()
    ops = gpu_ops(precision=1, restart=40, stokes_its=1, precond=2)
    budget = sum(sorted(ops.footprint(c) for c in cases)[-2:])   # two at a time at most
    srv = Server(ops, budget_bytes=budget)
    reqs = [Request(rid=i, arrival=0.0, case=c, steps=2 + i) for i, c in enumerate(cases)]
    wall = srv.run(reqs, realtime=False)
    rep = srv.report(wall)
    assert rep["requests_finished"] == 3 and rep["requests_rejected"] == 0
    for r in srv.finished:
        assert r.error is None
        ref = _alone(fsi, r.case, r.steps, restart=40)
        for a, b in zip(r.result, ref):
            assert np.array_equal(a, b)


def test_admission_budget_refuses(fsi):
    c = _cases()[0]
    prm = fsi.make_params(c.N, c.rho_f, c.nu, c.kappa, c.dt, c.lid_u, precond=2, precision=1)
    need = fsi.footprint_bytes(prm, c.ref_xy.shape[0], c.tris.shape[0])
    assert need > 0
    with pytest.raises(fsi.FsiError) as e:
        fsi.Problem(prm, c.ref_xy, c.tris, u0=c.u0, X0=c.X0, budget_bytes=need // 2)
    assert e.value.code == fsi.FSI_ERR_BUDGET
    p = fsi.Problem(prm, c.ref_xy, c.tris, u0=c.u0, X0=c.X0, budget_bytes=need)
    p.close()


def _mixed_elements():
    """A P1 disk and two Q1 annuli (quarter, no-slip; mirrored full annulus)."""
    return [_cases()[0], fi.annulus_case(16, quads=True), fi.symmetric_annulus_case(8, quads=True)]


def test_batch_mixed_elements_equals_alone(fsi):
    cases = _mixed_elements()
    probs = [fsi.problem_from_case(c, precision=1) for c in cases]
    for _ in range(2):
        st, infos = fsi.step_batch(probs)
        assert st == 0 and all(i.status == 0 for i in infos)
    for c, p in zip(cases, probs):
        ref = _alone(fsi, c, 2)
        for a, b in zip(p.get_state(), ref):
            assert np.array_equal(a, b)
        p.close()


def test_served_q1_requests_equal_alone(fsi):
    from paper_2301_10041_gb300.serve import Request, Server, gpu_ops
    cases = _mixed_elements()
    ops = gpu_ops(precision=1, restart=40, stokes_its=1, precond=2)
    srv = Server(ops, budget_bytes=sum(ops.footprint(c) for c in cases))
    reqs = [Request(rid=i, arrival=0.0, case=c, steps=2) for i, c in enumerate(cases)]
    srv.run(reqs, realtime=False)
    assert len(srv.finished) == 3
    for r in srv.finished:
        assert r.error is None
        ref = _alone(fsi, r.case, r.steps, restart=40, stokes_its=1, precond=2)
        for a, b in zip(r.result, ref):
            assert np.array_equal(a, b)
