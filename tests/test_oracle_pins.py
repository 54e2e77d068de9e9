"""Pins of the CPU oracle against facts fixed by the mathematics and the paper.

Each test checks the oracle against something other than itself: closed-form
integrals, invariants, published quadrature tables, manufactured-solution
convergence rates and brute-force special cases.  A dropped term, a wrong
sign, a transposed block or a wrong index in the oracle fails one of these.
"""
import math
import os

import numpy as np
import pytest

import fsi_inputs as fi
from oracle import fsi_oracle as fo

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- quadrature

def test_triangle_rule_matches_published_table():
    """Constants agree with Dunavant (1985) Table I (p = 4) to its 15 digits."""
    rows = np.loadtxt(os.path.join(HERE, "golden", "dunavant_deg4.txt"))
    lam, w = fo.triangle_rule()
    assert np.allclose(w[[0, 3]], rows[:, 0], atol=1e-15, rtol=0)
    # representatives: the point whose odd coordinate sits in lam0
    assert np.allclose(lam[[0, 3]], rows[:, 1:], atol=1e-15, rtol=0)
    assert abs(w.sum() - 1.0) < 1e-15


def test_triangle_rule_exact_to_degree_4():
    """Integral of lam1^i lam2^j over a triangle of area 1 is 2 i! j!/(i+j+2)!."""
    lam, w = fo.triangle_rule()
    for d in range(5):
        for i in range(d + 1):
            j = d - i
            exact = 2.0 * math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            q = np.sum(w * lam[:, 1] ** i * lam[:, 2] ** j)
            assert abs(q - exact) < 1e-15
    # and it is a degree-4 rule, not more
    q = np.sum(w * lam[:, 1] ** 5)
    assert abs(q - 2.0 * math.factorial(5) / math.factorial(7)) > 1e-6


def test_q2_basis_is_nodal_and_complete():
    nodes = np.array([0.0, 0.5, 1.0])
    assert np.allclose(fo.q2_1d(nodes), np.eye(3), atol=0)
    t = np.linspace(0, 1, 7)
    L = fo.q2_1d(t)
    assert np.allclose(L.sum(1), 1.0)
    assert np.allclose(L @ nodes, t)            # reproduces linears
    assert np.allclose(L @ nodes ** 2, t ** 2)  # and quadratics
    assert np.allclose(fo.q2_1d_deriv(t) @ nodes ** 2, 2 * t)


# ------------------------------------------------------------- fluid blocks

@pytest.fixture(scope="module")
def fluid8():
    g = fo.FluidGrid(8)
    M, K, B = fo.assemble_fluid(g, nu=0.7)
    return g, M, K, B


def _nodal(g, fx, fy):
    u = np.zeros(2 * g.n_nodes)
    u[0::2] = fx(g.node_xy[:, 0], g.node_xy[:, 1])
    u[1::2] = fy(g.node_xy[:, 0], g.node_xy[:, 1])
    return u


def test_mass_matrix_integrals(fluid8):
    g, M, K, B = fluid8
    one = _nodal(g, lambda x, y: 1 + 0 * x, lambda x, y: 0 * x)
    assert abs(one @ M @ one - 1.0) < 1e-13                # area of the unit square
    sq = _nodal(g, lambda x, y: x * x, lambda x, y: 0 * x)
    assert abs(one @ M @ sq - 1.0 / 3.0) < 1e-13           # int x^2
    xy = _nodal(g, lambda x, y: x * y, lambda x, y: 0 * x)
    assert abs(xy @ M @ xy - 1.0 / 9.0) < 1e-13            # int x^2 y^2
    assert abs(M - M.T).max() < 1e-15


def test_strain_energy_of_linear_fields(fluid8):
    """a(u, u) = nu int eps(u):eps(u) with eps the symmetric gradient, no factor 2."""
    g, M, K, B = fluid8
    nu = 0.7
    cases = [((lambda x, y: x, lambda x, y: y), 2 * nu),        # eps = I
             ((lambda x, y: y, lambda x, y: 0 * x), nu / 2),     # pure shear
             ((lambda x, y: x, lambda x, y: -y), 2 * nu),
             ((lambda x, y: 0 * x, lambda x, y: x), nu / 2)]
    for (fx, fy), val in cases:
        u = _nodal(g, fx, fy)
        assert abs(u @ K @ u - val) < 1e-12
    assert abs(K - K.T).max() < 1e-13


def test_rigid_motions_have_no_strain(fluid8):
    g, M, K, B = fluid8
    for fx, fy in ((lambda x, y: 1 + 0 * x, lambda x, y: 0 * x),
                   (lambda x, y: 0 * x, lambda x, y: 1 + 0 * y),
                   (lambda x, y: -y, lambda x, y: x)):
        assert np.abs(K @ _nodal(g, fx, fy)).max() < 1e-12


def test_divergence_matrix(fluid8):
    g, M, K, B = fluid8
    h = g.h
    # divergence-free quadratic field -> B u = 0 exactly
    u = _nodal(g, lambda x, y: x * x, lambda x, y: -2 * x * y)
    assert np.abs(B @ u).max() < 1e-14
    # div (x, 0) = 1: (B u)_k = int psi_k over the cell = (h^2, 0, 0)
    b = (B @ _nodal(g, lambda x, y: x, lambda x, y: 0 * x)).reshape(-1, 3)
    assert np.allclose(b, np.array([h * h, 0, 0])[None, :], atol=1e-15)
    # div (x^2, 0) = 2x: (2 xc h^2, h^3/6, 0)
    b = (B @ _nodal(g, lambda x, y: x * x, lambda x, y: 0 * x)).reshape(-1, 3)
    xc = (np.arange(g.N * g.N) % g.N + 0.5) * h
    assert np.allclose(b[:, 0], 2 * xc * h * h, atol=1e-15)
    assert np.allclose(b[:, 1], h ** 3 / 6, atol=1e-15)
    assert np.allclose(b[:, 2], 0, atol=1e-15)
    # div (0, y^2) = 2y: third coefficient h^3/6
    b = (B @ _nodal(g, lambda x, y: 0 * x, lambda x, y: y * y)).reshape(-1, 3)
    assert np.allclose(b[:, 2], h ** 3 / 6, atol=1e-15)
    assert np.allclose(b[:, 1], 0, atol=1e-15)


def _manufactured(nu, rho, dt):
    pi = math.pi
    s, c = np.sin, np.cos

    def u(x, y):
        return np.stack([2 * pi * s(pi * x) ** 2 * s(pi * y) * c(pi * y),
                         -2 * pi * s(pi * x) * c(pi * x) * s(pi * y) ** 2], 1)

    def gu(x, y):
        a = 2 * pi * pi
        ux_x = a * 2 * s(pi * x) * c(pi * x) * s(pi * y) * c(pi * y)
        ux_y = a * s(pi * x) ** 2 * (c(pi * y) ** 2 - s(pi * y) ** 2)
        uy_x = -a * (c(pi * x) ** 2 - s(pi * x) ** 2) * s(pi * y) ** 2
        uy_y = -a * s(pi * x) * c(pi * x) * 2 * s(pi * y) * c(pi * y)
        return np.stack([np.stack([ux_x, ux_y], 1), np.stack([uy_x, uy_y], 1)], 1)

    def p(x, y):
        return c(pi * x) * c(pi * y)

    def lap(x, y):
        # Laplacian of u, componentwise
        a = 2 * pi ** 3
        lx = a * (2 * c(2 * pi * x) * s(pi * y) * c(pi * y) - 4 * s(pi * x) ** 2 * s(pi * y) * c(pi * y))
        ly = -a * (2 * c(2 * pi * y) * s(pi * x) * c(pi * x) - 4 * s(pi * y) ** 2 * s(pi * x) * c(pi * x))
        return np.stack([lx, ly], 1)

    def f(x, y):
        # (rho/dt) u - div(nu eps(u)) + grad p, with div(eps(u)) = lap(u)/2 for div-free u
        gp = np.stack([-pi * s(pi * x) * c(pi * y), -pi * c(pi * x) * s(pi * y)], 1)
        return (rho / dt) * u(x, y) - 0.5 * nu * lap(x, y) + gp

    return u, gu, p, f


def test_stokes_manufactured_convergence_rates():
    """Q2/P1disc generalized Stokes: ||u-u_h|| = O(h^3), |u-u_h|_1 = O(h^2),
    ||p-p_h|| = O(h^2)."""
    u, gu, p, f = _manufactured(nu=1.0, rho=1.0, dt=0.1)
    errs = [fo.stokes_manufactured(N, 1.0, 1.0, 0.1, u, gu, p, f) for N in (4, 8, 16)]
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1, 0] > 2.8, rates
    assert rates[-1, 1] > 1.85, rates
    assert rates[-1, 2] > 1.85, rates


# ------------------------------------------------------------- solid blocks

def test_solid_mass_and_stiffness():
    xy, tris = fi.ring_disk_mesh(5, 0.3, (0.4, 0.6))
    C, A = fo.assemble_solid(xy, tris, kappa=3.0)
    one = np.ones(xy.shape[0])
    # polygon area of the outer ring by the shoelace formula
    ring = xy[-30:]
    area = 0.5 * abs(np.sum(ring[:, 0] * np.roll(ring[:, 1], -1) - np.roll(ring[:, 0], -1) * ring[:, 1]))
    assert abs(one @ C @ one - area) < 1e-14
    assert np.abs(A @ one).max() < 1e-12                   # constants have no gradient
    # kappa int |grad x|^2 = kappa * area
    x = xy[:, 0]
    assert abs(x @ A @ x - 3.0 * area) < 1e-12
    # mass entries by the (independent) degree-4 rule: exact for P1 x P1
    lam, w = fo.triangle_rule()
    area_t, _ = fo.p1_geometry(xy, tris)
    Cq = np.zeros((xy.shape[0],) * 2)
    for t in range(tris.shape[0]):
        for a in range(3):
            for b in range(3):
                Cq[tris[t, a], tris[t, b]] += area_t[t] * np.sum(w * lam[:, a] * lam[:, b])
    assert np.abs(C.toarray() - Cq).max() < 1e-15


# ------------------------------------------------------------ point location

def test_locate_matches_floor_rule_and_grid_lines():
    N = 7
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, size=(4000, 2))
    lines = np.arange(N + 1) / N
    x[:64, 0] = np.resize(lines, 64)
    x[64:128, 1] = np.resize(lines, 64)
    x[128] = (1.0, 1.0)
    x[129] = (0.0, 0.0)
    x[130] = (np.nextafter(1.0, 0), np.nextafter(0.0, 1))
    x[131] = (-1e-300, 0.5)
    x[132] = (0.5, 1.0 + 2 ** -52)
    x[133] = (np.nan, 0.5)
    cell, xi, eta = fo.locate_brute_force(x, N)
    t = x * N
    ok = (x >= 0).all(1) & (x <= 1).all(1)
    i = np.where(ok[:, None], np.minimum(np.floor(np.where(ok[:, None], t, 0)), N - 1), -1).astype(int)
    expect = np.where(ok, i[:, 1] * N + i[:, 0], -1)
    assert np.array_equal(cell, expect)
    assert cell[131] == -1 and cell[132] == -1 and cell[133] == -1
    assert cell[128] == N * N - 1 and cell[129] == 0
    m = cell >= 0
    assert np.array_equal(xi[m], (t[:, 0] - i[:, 0])[m])
    assert np.array_equal(eta[m], (t[:, 1] - i[:, 1])[m])
    assert (xi[m] >= 0).all() and (xi[m] <= 1).all()


# ------------------------------------------------------------------ coupling

def _deformed(xy, shear=0.3, rot=0.4, center=(0.5, 0.5)):
    c, s = math.cos(rot), math.sin(rot)
    x = xy[:, 0] - center[0]
    y = xy[:, 1] - center[1]
    X = np.stack([c * x - s * y + shear * y, s * x + c * y + 0.1 * x * x], 1)
    return X + np.array(center)


def test_coupling_partition_of_unity_and_reproduction():
    """C_f 1 = C_s 1 (partition of unity); C_f reproduces linear and quadratic
    fields exactly because the rule integrates degree <= 4."""
    N = 12
    g = fo.FluidGrid(N)
    xy, tris = fi.ring_disk_mesh(7, 0.22, (0.5, 0.5))
    X = _deformed(xy)
    C, (xq, cell, xi, eta) = fo.assemble_coupling(g, xy, tris, X)
    Cs, _ = fo.assemble_solid(xy, tris, 1.0)
    one = np.ones(g.n_nodes)
    rs = C @ one
    assert np.abs(rs - Cs @ np.ones(xy.shape[0])).max() < 1e-12 * np.abs(rs).max()
    # linear reproduction: (C x_nodal)_l = int chi_l X_x = (C_s X_x)_l
    for comp in range(2):
        lin = C @ g.node_xy[:, comp]
        assert np.abs(lin - Cs @ X[:, comp]).max() < 1e-13
    # quadratic: (C x^2)_l = int chi_l (X_x)^2 by the closed form
    # int_T lam_a lam_b lam_c = 2|T| a_! b_! c_!/(n+2)! over multiplicities
    area_t, _ = fo.p1_geometry(xy, tris)
    ref = np.zeros(xy.shape[0])
    for t in range(tris.shape[0]):
        v = tris[t]
        for a in range(3):
            s = 0.0
            for b in range(3):
                for c in range(3):
                    mult = np.bincount([a, b, c], minlength=3)
                    integ = 2 * area_t[t] * np.prod([math.factorial(k) for k in mult]) / math.factorial(5)
                    s += integ * X[v[b], 0] * X[v[c], 0]
            ref[v[a]] += s
    quad = C @ g.node_xy[:, 0] ** 2
    assert np.abs(quad - ref).max() < 1e-13


def test_coupling_rejects_points_outside():
    g = fo.FluidGrid(8)
    xy, tris = fi.ring_disk_mesh(3, 0.2, (0.5, 0.5))
    X = xy + np.array([0.45, 0.0])
    with pytest.raises(ValueError):
        fo.assemble_coupling(g, xy, tris, X)


# ------------------------------------------------------------------- one step

def test_step_residual_and_scipy_agreement():
    c = fi.disk16_case()
    prob = fo.OracleProblem(c.N, c.rho_f, c.nu, c.kappa, c.dt, c.lid_u, c.ref_xy, c.tris)
    Kmat, rhs, _ = prob.system(c.u0, c.X0)
    x = prob.solve_system(Kmat, rhs, c.X0)
    assert np.linalg.norm(rhs - Kmat @ x) / np.linalg.norm(rhs) < 1e-12
    # an unscaled, differently ordered library solve of the bordered system
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n_u, n_p, n_x = prob.sizes()
    e = np.zeros(Kmat.shape[0])
    e[n_u:n_u + n_p:3] = 1.0
    big = sp.bmat([[Kmat, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
    x2 = spla.spsolve(big, np.concatenate([rhs, [0.0]]))[:-1]
    assert np.linalg.norm(x - x2) / np.linalg.norm(x2) < 1e-9


def test_pressure_has_zero_mean_and_velocity_is_discretely_solenoidal():
    c = fi.disk16_case()
    prob, u, p, X, lam = fo.run_steps(c, 1)
    assert abs(p[:, 0].sum()) < 1e-10 * np.abs(p[:, 0]).max()
    div = prob.B @ u.reshape(-1)
    assert np.abs(div).max() < 1e-12 * np.abs(prob.B).max() * np.abs(u).max()


def test_discrete_energy_identity():
    """Testing Eq. (matrix) with (u^{n+1}, p, (X^{n+1}-X^n)/dt, -lambda) gives
    rho/(2dt)(|u1|_M^2 - |u0|_M^2 + |u1-u0|_M^2) + a(u1, u1)
      + kappa/(2dt)(|grad X1|^2 - |grad X0|^2 + |grad(X1-X0)|^2) = 0
    with walls at rest: the coupling and pressure terms cancel in pairs."""
    c = fi.disk16_case()
    prob, u1, p, X1, lam = fo.run_steps(c, 1)
    u0 = c.u0.reshape(-1)
    u1 = u1.reshape(-1)
    M, K, As = prob.M, prob.K, prob.As
    X0 = c.X0.reshape(-1)
    X1 = X1.reshape(-1)
    r, dt = prob.rho, prob.dt
    kin = r / (2 * dt) * (u1 @ M @ u1 - u0 @ M @ u0 + (u1 - u0) @ M @ (u1 - u0))
    visc = u1 @ K @ u1
    ela = 1.0 / (2 * dt) * (X1 @ As @ X1 - X0 @ As @ X0 + (X1 - X0) @ As @ (X1 - X0))
    scale = max(abs(kin), abs(visc), abs(ela), r / (2 * dt) * (u0 @ M @ u0))
    assert abs(kin + visc + ela) < 1e-9 * scale


def test_kappa_zero_body_at_rest_stays_at_rest():
    xy, tris = fi.ring_disk_mesh(4, 0.2, (0.5, 0.5))
    prob = fo.OracleProblem(8, 1.0, 0.5, 0.0, 0.01, 0.0, xy, tris)
    u, p, X, lam = prob.step(np.zeros((prob.grid.n_nodes, 2)), xy)
    assert np.abs(u).max() < 1e-13
    assert np.abs(X - xy).max() < 1e-14
    assert np.abs(lam).max() < 1e-10
    assert np.abs(p).max() < 1e-10


def test_lid_driven_cavity_conserves_no_mass_through_walls():
    """With the lid, B u^{n+1} = 0 for the full field (interior + wall data)."""
    xy, tris = fi.ring_disk_mesh(4, 0.2, (0.5, 0.5))
    prob = fo.OracleProblem(8, 1.0, 0.1, 50.0, 0.01, 1.0, xy, tris)
    u0 = fi.wall_velocity(8, 1.0)
    u, p, X, lam = prob.step(u0, xy)
    assert np.abs(prob.B @ u.reshape(-1)).max() < 1e-11 * np.abs(prob.B).max()
    top = (prob.grid.n1 - 1) * prob.grid.n1 + np.arange(1, prob.grid.n1 - 1)
    assert np.all(u[top, 0] == 1.0)


def _q2_field_at(u_nodal, N, pts):
    """The Q2 field with nodal values u_nodal [(2N+1)^2, 2] at points [n, 2]:
    cell by truncation (no point here lies on a grid line), then the
    tensor product of the three quadratic Lagrange polynomials on the local
    nodes 0, 1/2, 1 written as products of their roots."""
    n1 = 2 * N + 1
    t = pts * N
    c = np.minimum(np.floor(t).astype(np.int64), N - 1)
    s = t - c

    def lag(v):
        return np.stack([2.0 * (v - 0.5) * (v - 1.0), -4.0 * v * (v - 1.0), 2.0 * v * (v - 0.5)], 1)

    Lx, Ly = lag(s[:, 0]), lag(s[:, 1])
    out = np.zeros((pts.shape[0], 2))
    for b in range(3):
        for a in range(3):
            node = (2 * c[:, 1] + b) * n1 + (2 * c[:, 0] + a)
            out += (Lx[:, a] * Ly[:, b])[:, None] * u_nodal[node]
    return out


def test_constraint_row_with_lid_data_on_the_body():
    """The multiplier row of Eq. (matrix), with the Dirichlet data moved to
    the right-hand side (g2 = -(1/dt) C_s X^n - C_D u_D), says that the whole
    discrete velocity field, wall values included, matches the solid velocity
    on the body: (chi_l, u^{n+1}(X^n))_B = (1/dt) (chi_l, X^{n+1} - X^n)_B
    for every solid node l.  The left side is evaluated here without the
    oracle's coupling matrix: the published degree-4 rule (golden table) on
    each reference triangle, the body map by barycentric combination, and the
    nodal field interpolated in its Q2 cell.  The body's rule points fill the
    top row of cells under a moving lid, so the wall term C_D u_D is a large
    part of the row; a wrong sign or wall index in it breaks the identity."""
    c = fi.lid_body_case()
    prob, u1, p, X1, lam = fo.run_steps(c, 1)
    rows = np.loadtxt(os.path.join(HERE, "golden", "dunavant_deg4.txt"))
    bary, wts = [], []
    for w, l0, l1, l2 in rows:     # each orbit: the odd coordinate visits every vertex
        for k in range(3):
            bary.append(np.roll([l0, l1, l2], k))
            wts.append(w)
    bary, wts = np.array(bary), np.array(wts)
    tris = c.tris.astype(np.int64)
    P = c.X0[tris]                                     # [T, 3, 2] body at X^n
    R = c.ref_xy[tris]
    area = 0.5 * np.abs((R[:, 1, 0] - R[:, 0, 0]) * (R[:, 2, 1] - R[:, 0, 1])
                        - (R[:, 2, 0] - R[:, 0, 0]) * (R[:, 1, 1] - R[:, 0, 1]))
    pts = np.einsum("qk,tkd->tqd", bary, P).reshape(-1, 2)
    top = pts[:, 1] >= (c.N - 1) / c.N
    assert top.sum() > 0.2 * pts.shape[0]            # many rule points in the lid's row of cells
    n_s = c.ref_xy.shape[0]

    def rows_of(field):
        v = _q2_field_at(field, c.N, pts).reshape(tris.shape[0], 6, 2)
        out = np.zeros((n_s, 2))
        for k in range(3):
            np.add.at(out, tris[:, k], np.einsum("t,q,q,tqd->td", area, wts, bary[:, k], v))
        return out

    lhs = rows_of(u1)
    rhs = (1.0 / c.dt) * (prob.Cs_scalar @ (X1 - c.X0))
    lid_part = rows_of(fi.wall_velocity(c.N, c.lid_u))   # what the wall values contribute
    assert np.linalg.norm(lid_part) > 0.1 * np.linalg.norm(lhs)
    assert np.linalg.norm(lhs - rhs) < 1e-10 * np.linalg.norm(lhs)


# ------------------------------------------- exact coupling (mesh intersection)

def _duffy_rule(n: int):
    """Gauss product rule on the reference triangle {s1, s2 >= 0, s1 + s2 <= 1}
    through the collapsed map s = (u, v (1 - u)) with Jacobian (1 - u): an
    independent rule, exact for polynomials of degree <= 2n - 2 in s."""
    g, w = fo.gauss01(n)
    U, V = np.meshgrid(g, g, indexing="ij")
    W = np.outer(w, w) * (1.0 - U)
    return np.stack([U.ravel(), (V * (1.0 - U)).ravel()], 1), W.ravel()   # weights sum to 1/2


def test_radon_rule_exact_to_degree_5():
    """Integrals of s1^a s2^b over the reference triangle: a! b! / (a+b+2)!,
    exact for a + b <= 5 and not for every monomial of degree 6."""
    lam, w = fo.radon_rule()
    assert abs(w.sum() - 1.0) < 1e-15
    s1, s2 = lam[:, 1], lam[:, 2]
    for a in range(6):
        for b in range(6 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(0.5 * np.dot(w, s1 ** a * s2 ** b) - exact) < 1e-15
    errs = [abs(0.5 * np.dot(w, s1 ** a * s2 ** (6 - a))
                - math.factorial(a) * math.factorial(6 - a) / math.factorial(8)) for a in range(7)]
    assert max(errs) > 1e-6


def test_clipping_conserves_area_and_covers_the_triangle():
    """The pieces of a triangle cut by every cell of its bounding box
    (Sutherland-Hodgman) have areas that add up to the triangle's, for
    triangles with vertices on grid lines, inside one cell and across many."""
    rng = np.random.default_rng(4)
    N = 8
    h = 1.0 / N
    tris = [np.array([[0.1, 0.1], [0.9, 0.2], [0.3, 0.8]]),
            np.array([[0.25, 0.25], [0.5, 0.25], [0.25, 0.5]]),          # vertices on grid lines
            np.array([[0.51, 0.52], [0.56, 0.53], [0.52, 0.6]])]          # inside one cell
    tris += [rng.uniform(0.0, 1.0, (3, 2)) for _ in range(20)]
    for P in tris:
        d1, d2 = P[1] - P[0], P[2] - P[0]
        area = 0.5 * abs(d1[0] * d2[1] - d1[1] * d2[0])
        lo = np.minimum(np.floor(P.min(0) * N).astype(int), N - 1)
        hi = np.minimum(np.floor(P.max(0) * N).astype(int), N - 1)
        tot = 0.0
        for cy in range(lo[1], hi[1] + 1):
            for cx in range(lo[0], hi[0] + 1):
                poly = fo.clip_to_cell(P, cx * h, (cx + 1) * h, cy * h, (cy + 1) * h)
                for q in poly:   # every piece lies in its cell
                    assert cx * h - 1e-15 <= q[0] <= (cx + 1) * h + 1e-15
                    assert cy * h - 1e-15 <= q[1] <= (cy + 1) * h + 1e-15
                for i in range(1, len(poly) - 1):
                    e1, e2 = poly[i] - poly[0], poly[i + 1] - poly[0]
                    tot += 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        assert abs(tot - area) <= 1e-14 * max(area, 1e-3)


def _sheared_body(m=4, R=0.23, c=(0.47, 0.52)):
    xy, tris = fi.ring_disk_mesh(m, R, c)
    d = xy - np.array(c)
    co, si = np.cos(0.4), np.sin(0.4)
    X = np.stack([co * d[:, 0] - si * d[:, 1] + 0.3 * d[:, 1], si * d[:, 0] + co * d[:, 1]], 1) + np.array(c)
    return xy, tris.astype(np.int64), X


def test_exact_coupling_reproduces_biquadratic_fields():
    """For a biquadratic field p, the Q2 interpolant is p itself on every
    cell, so (C p_nodal)_l must equal the integral over B of chi_l p(X(s)),
    computed here on whole solid triangles by an independent product rule.
    The integrand has degree 5 (x^2 y^2 times a linear chi), so the exact
    rule passes and the degree-4 point rule does not."""
    xy, tris, X = _sheared_body(m=2)                      # large triangles across many cells
    rng = np.random.default_rng(9)
    c = rng.standard_normal((3, 3))                      # p = sum c_ab x^a y^b, a, b <= 2

    def p(pts):
        return sum(c[a, b] * pts[:, 0] ** a * pts[:, 1] ** b for a in range(3) for b in range(3))

    s, w = _duffy_rule(5)
    ref = np.zeros(xy.shape[0])
    for t in range(tris.shape[0]):
        A, Bv, Cv = xy[tris[t]]
        jac = abs((Bv - A)[0] * (Cv - A)[1] - (Bv - A)[1] * (Cv - A)[0])
        lam = np.stack([1.0 - s[:, 0] - s[:, 1], s[:, 0], s[:, 1]], 1)
        Xq = lam @ X[tris[t]]
        for k in range(3):
            ref[tris[t, k]] += jac * np.dot(w, lam[:, k] * p(Xq))
    for N in (6, 8, 16):
        grid = fo.FluidGrid(N)
        pn = p(grid.node_xy)
        Cx = fo.assemble_coupling_exact(grid, xy, tris, X)
        assert np.max(np.abs(Cx @ pn - ref)) <= 1e-13 * np.max(np.abs(ref))
        Cp, _ = fo.assemble_coupling(grid, xy, tris, X)
        assert np.max(np.abs(Cp @ pn - ref)) > 1e-10 * np.max(np.abs(ref))


def test_exact_coupling_partition_of_unity_and_agreement_with_point_rule():
    """Rows of the exact C sum to the rows of the solid mass matrix (the Q2
    basis sums to one); and as the solid mesh is refined on a fixed fluid
    grid (triangles ever more often inside a single cell, where the integrand
    is one polynomial), the point rule approaches the exact rule."""
    grid = fo.FluidGrid(8)
    errs = []
    for m in (3, 6, 12):
        xy, tris, X = _sheared_body(m=m)
        Cs, _ = fo.assemble_solid(xy, tris, 1.0)
        mass = np.asarray(Cs.sum(axis=1)).ravel()
        Cx = fo.assemble_coupling_exact(grid, xy, tris, X)
        assert np.max(np.abs(np.asarray(Cx.sum(axis=1)).ravel() - mass)) <= 1e-13 * mass.max()
        Cp, _ = fo.assemble_coupling(grid, xy, tris, X)
        u = np.cos(3.0 * grid.node_xy[:, 0]) * np.sin(2.0 * grid.node_xy[:, 1])   # a smooth nodal field
        errs.append(np.max(np.abs(Cx @ u - Cp @ u)) / np.max(np.abs(Cx @ u)))
    assert errs[2] < errs[1] < errs[0]


def test_exact_coupling_rejects_vertices_outside():
    xy, tris, X = _sheared_body()
    X = X.copy()
    X[0] = (1.01, 0.5)
    with pytest.raises(ValueError):
        fo.assemble_coupling_exact(fo.FluidGrid(8), xy, tris, X)


# ------------------------------------------------------- nonlinear solid law

def _bent_bar():
    case = fi.bar_case(N=16, nx=8, ny=2)
    return case, case.ref_xy, case.tris.astype(np.int64), case.X0


def test_exp_law_stress_is_the_energy_gradient():
    """S = d/dX of sum_E |E| W(F_E), by central differences of the energy."""
    _, xy, tris, X = _bent_bar()
    g, e = 1.333, 9.242
    area, _ = fo.p1_geometry(xy, tris)

    def energy(Xv):
        return float(np.dot(area, fo.exp_law_energy(fo.deformation_gradients(xy, tris, Xv), g, e)))

    S, _ = fo.solid_nonlinear(xy, tris, X, g, e)
    rng = np.random.default_rng(1)
    for _ in range(6):
        i, c = int(rng.integers(xy.shape[0])), int(rng.integers(2))
        hstep = 1e-6
        Xp, Xm = X.copy(), X.copy()
        Xp[i, c] += hstep
        Xm[i, c] -= hstep
        fd = (energy(Xp) - energy(Xm)) / (2 * hstep)
        assert abs(fd - S[i, c]) <= 1e-6 * max(1.0, abs(S[i, c]))


def test_exp_law_tangent_is_the_stress_derivative():
    """K_T = dS/dX, column by column by central differences of S."""
    _, xy, tris, X = _bent_bar()
    g, e = 1.333, 9.242
    _, K = fo.solid_nonlinear(xy, tris, X, g, e)
    K = K.toarray()
    for j in (0, 5, 11, 20):
        for c in range(2):
            hstep = 1e-6
            Xp, Xm = X.copy(), X.copy()
            Xp[j, c] += hstep
            Xm[j, c] -= hstep
            Sp, _ = fo.solid_nonlinear(xy, tris, Xp, g, e)
            Sm, _ = fo.solid_nonlinear(xy, tris, Xm, g, e)
            fd = ((Sp - Sm) / (2 * hstep)).reshape(-1)
            assert np.max(np.abs(fd - K[:, 2 * j + c])) <= 1e-5 * max(1.0, np.max(np.abs(K)))


def test_exp_law_tends_to_the_linear_law():
    """As eta -> 0, W -> gamma/(2 eta) + (gamma/2)(|F|^2 - 2): P -> gamma F,
    so S -> A_s X with kappa = gamma (the linear law of Eq. (matrix))."""
    _, xy, tris, X = _bent_bar()
    S, K = fo.solid_nonlinear(xy, tris, X, 1.333, 1e-9)
    _, As = fo.assemble_solid(xy, tris, 1.333)
    assert np.max(np.abs(S - As @ X)) <= 1e-7 * np.max(np.abs(S))
    assert abs(K - fo.kron2(As)).max() <= 1e-7 * abs(K).max()


def test_newton_converges_quadratically_on_the_bar():
    """Newton on the linearised block systems: the change of X falls at
    least quadratically until it reaches rounding, and the converged state
    has a small nonlinear residual in the oracle's operator."""
    case, xy, tris, X = _bent_bar()
    o = fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, xy, tris,
                         solid_law="exp", gamma=1.333, eta=9.242, newton_tol=1e-12)
    u, p, Xn, lam = o.step(case.u0, case.X0)
    h = o.newton_history
    assert len(h) >= 3
    for a, b in zip(h[:-2], h[1:-1]):
        assert b <= 100.0 * a * a or b <= 1e-11
    assert o.relative_residual(case.u0, case.X0, u, p, Xn, lam) < 1e-10


# ------------------------------------------------- Q1 solid (annulus test)

def _quad_areas(xy, quads):
    P = xy[quads]
    x, y = P[..., 0], P[..., 1]
    return 0.5 * np.sum(x * np.roll(y, -1, axis=1) - np.roll(x, -1, axis=1) * y, axis=1)


def test_q1_rule_is_the_gauss_legendre_product_rule():
    """Nodes and weights equal the library Gauss-Legendre rule mapped to
    [0,1]; the product rule integrates s^i t^j exactly for i, j <= 5."""
    s, t, st, w = fo.q1_rule()
    x, wx = np.polynomial.legendre.leggauss(3)
    g, wg = 0.5 * (x + 1.0), 0.5 * wx
    assert np.allclose(s, np.tile(g, 3), atol=1e-16, rtol=0)
    assert np.allclose(t, np.repeat(g, 3), atol=1e-16, rtol=0)
    assert np.allclose(w, np.tile(wg, 3) * np.repeat(wg, 3), atol=1e-16, rtol=0)
    assert np.array_equal(st, s * t)
    for i in range(6):
        for j in range(6):
            assert abs(np.sum(w * s ** i * t ** j) - 1.0 / ((i + 1) * (j + 1))) < 1e-15


def test_q1_element_matrices_on_a_square_match_closed_forms():
    """Square of side h: mass h^2/36 [4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4],
    stiffness kappa/6 [4 -1 -2 -1; -1 4 -1 -2; -2 -1 4 -1; -1 -2 -1 4]."""
    h, kappa = 0.125, 2.5
    xy = np.array([[0.3, 0.4], [0.3 + h, 0.4], [0.3 + h, 0.4 + h], [0.3, 0.4 + h]])
    quads = np.array([[0, 1, 2, 3]])
    C, A = fo.assemble_solid_q1(xy, quads, kappa)
    circ = lambda r: np.array([np.roll(r, k) for k in range(4)])
    assert np.abs(C.toarray() - h * h / 36.0 * circ([4.0, 2.0, 1.0, 2.0])).max() < 1e-17
    assert np.abs(A.toarray() - kappa / 6.0 * circ([4.0, -1.0, -2.0, -1.0])).max() < 1e-14


def test_q1_solid_matrices_on_curved_quadrilaterals():
    """Annulus quadrilaterals (no two edges parallel): total mass = polygon
    area, constants have no gradient, kappa int |grad f|^2 = kappa |G|^2 area
    for a linear f (its Q1 interpolant is f itself), and the mass entries
    equal an independent 6 x 6 Gauss product rule (the integrand is a
    polynomial of degree 3 in each reference variable)."""
    xy, quads = fi.annulus_mesh(3, 5, quads=True)
    kappa = 3.0
    C, A = fo.assemble_solid_q1(xy, quads, kappa)
    one = np.ones(xy.shape[0])
    area = _quad_areas(xy, quads).sum()
    assert abs(one @ C @ one - area) < 1e-15
    assert np.abs(A @ one).max() < 1e-13
    f = 0.7 * xy[:, 0] - 1.3 * xy[:, 1]
    assert abs(f @ A @ f - kappa * (0.7 ** 2 + 1.3 ** 2) * area) < 1e-13
    x6, w6 = np.polynomial.legendre.leggauss(6)
    g6, v6 = 0.5 * (x6 + 1), 0.5 * w6
    S, T = np.meshgrid(g6, g6, indexing="ij")
    W = np.outer(v6, v6)
    chi = np.stack([(1 - S) * (1 - T), S * (1 - T), S * T, (1 - S) * T])
    Cq = np.zeros((xy.shape[0],) * 2)
    for q in quads:
        P = xy[q]
        xs = (-(1 - T) * P[0, 0] + (1 - T) * P[1, 0] + T * P[2, 0] - T * P[3, 0])
        ys = (-(1 - T) * P[0, 1] + (1 - T) * P[1, 1] + T * P[2, 1] - T * P[3, 1])
        xt = (-(1 - S) * P[0, 0] - S * P[1, 0] + S * P[2, 0] + (1 - S) * P[3, 0])
        yt = (-(1 - S) * P[0, 1] - S * P[1, 1] + S * P[2, 1] + (1 - S) * P[3, 1])
        J = xs * yt - ys * xt
        for a in range(4):
            for b in range(4):
                Cq[q[a], q[b]] += np.sum(W * J * chi[a] * chi[b])
    assert np.abs(C.toarray() - Cq).max() < 1e-16


def test_q1_mapped_points_are_the_bilinear_map():
    """The rounding-fixed point formula is the bilinear map sum_a chi_a(s) P_a
    (to rounding), and the mirrored quadrilaterals keep a positive Jacobian."""
    xy, quads = fi.annulus_mesh(2, 4, quads=True)
    X = _deformed(xy)
    x = fo.quadrature_points_q1(X, quads).reshape(-1, 9, 2)
    s, t, _, _ = fo.q1_rule()
    chi, _, _ = fo.q1_shape(s, t)
    ref = np.einsum("qa,ead->eqd", chi, X[quads])
    assert np.abs(x - ref).max() < 4e-16
    mxy, mquads = fi.mirrored_annulus_mesh(2, 4, quads=True)
    det, _ = fo.q1_geometry(mxy, mquads)
    assert (det > 0).all()


def test_q1_coupling_partition_of_unity_and_reproduction():
    """C_f 1 = C_s 1; C_f reproduces linear fields (f o X is bilinear, equal
    to the Q1 interpolant of f at the moved nodes); for x^2 the integrand
    chi_l (X_x)^2 |det J| is of degree 4 in each reference variable, so the
    3 x 3 rule is exact: compare with an independent 6 x 6 Gauss rule."""
    N = 12
    g = fo.FluidGrid(N)
    xy, quads = fi.annulus_mesh(3, 6, quads=True)
    xy = 0.1 + 0.9 * xy
    X = _deformed(xy, center=(0.45, 0.45))
    C, (xq, cell, xi, eta) = fo.assemble_coupling(g, xy, quads, X)
    Cs, _ = fo.assemble_solid_q1(xy, quads, 1.0)
    rs = C @ np.ones(g.n_nodes)
    assert np.abs(rs - Cs @ np.ones(xy.shape[0])).max() < 1e-13 * np.abs(rs).max()
    for comp in range(2):
        assert np.abs(C @ g.node_xy[:, comp] - Cs @ X[:, comp]).max() < 1e-14
    x6, w6 = np.polynomial.legendre.leggauss(6)
    g6, v6 = 0.5 * (x6 + 1), 0.5 * w6
    S, T = np.meshgrid(g6, g6, indexing="ij")
    W = np.outer(v6, v6)
    chi = np.stack([(1 - S) * (1 - T), S * (1 - T), S * T, (1 - S) * T])
    ref = np.zeros(xy.shape[0])
    for q in quads:
        P = xy[q]
        xs = -(1 - T) * P[0, 0] + (1 - T) * P[1, 0] + T * P[2, 0] - T * P[3, 0]
        ys = -(1 - T) * P[0, 1] + (1 - T) * P[1, 1] + T * P[2, 1] - T * P[3, 1]
        xt = -(1 - S) * P[0, 0] - S * P[1, 0] + S * P[2, 0] + (1 - S) * P[3, 0]
        yt = -(1 - S) * P[0, 1] - S * P[1, 1] + S * P[2, 1] + (1 - S) * P[3, 1]
        Xx = sum(chi[a] * X[q[a], 0] for a in range(4))
        for a in range(4):
            ref[q[a]] += np.sum(W * (xs * yt - ys * xt) * chi[a] * Xx ** 2)
    assert np.abs(C @ g.node_xy[:, 0] ** 2 - ref).max() < 1e-14


def test_q1_step_residual_and_body_at_rest():
    """One step with a Q1 solid: the direct solve meets its residual and
    agrees with an unscaled library solve; with kappa = 0, u_0 = 0 and no
    lid the body at rest stays at rest."""
    c = fi.annulus_case(12, quads=True)
    prob = fo.OracleProblem(c.N, c.rho_f, c.nu, c.kappa, c.dt, c.lid_u, c.ref_xy, c.tris)
    Kmat, rhs, _ = prob.system(c.u0, c.X0)
    x = prob.solve_system(Kmat, rhs, c.X0)
    assert np.linalg.norm(rhs - Kmat @ x) / np.linalg.norm(rhs) < 1e-12
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n_u, n_p, n_x = prob.sizes()
    e = np.zeros(Kmat.shape[0])
    e[n_u:n_u + n_p:3] = 1.0
    big = sp.bmat([[Kmat, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
    x2 = spla.spsolve(big, np.concatenate([rhs, [0.0]]))[:-1]
    assert np.linalg.norm(x - x2) / np.linalg.norm(x2) < 1e-9
    rest = fo.OracleProblem(c.N, 1.0, 0.1, 0.0, 0.01, 0.0, c.ref_xy, c.tris)
    u, p, X, lam = rest.step(np.zeros_like(c.u0), c.ref_xy)
    assert np.abs(u).max() < 1e-13 and np.abs(X - c.ref_xy).max() < 1e-15
    with pytest.raises(ValueError):
        fo.OracleProblem(c.N, 1.0, 0.1, 1.0, 0.01, 0.0, c.ref_xy, c.tris, coupling="exact")


@pytest.mark.parametrize("quads", [False, True])
def test_mirrored_annulus_gives_free_slip_quarter(quads):
    """The reading behind the free-slip walls of the annulus test (Section 6):
    the full annulus, mirror-symmetric mesh and data, has a mirror-symmetric
    step, so its velocity has no normal component on the mirror lines x = 1/2
    and y = 1/2 (the quarter problem's free-slip walls) and the body's
    displacement is mirror-symmetric."""
    from scipy.spatial import cKDTree
    case = fi.symmetric_annulus_case(8, quads=quads)
    prob = fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, case.ref_xy, case.tris)
    u, p, X, lam = prob.step(case.u0, case.X0)
    n1 = 2 * case.N + 1
    U = u.reshape(n1, n1, 2)                        # [iy, ix, comp]
    scale = np.abs(U).max()
    assert scale > 0
    # mirror in x = 1/2: u_x odd, u_y even; in y = 1/2: u_x even, u_y odd
    assert np.abs(U[:, ::-1, 0] + U[:, :, 0]).max() <= 1e-10 * scale
    assert np.abs(U[:, ::-1, 1] - U[:, :, 1]).max() <= 1e-10 * scale
    assert np.abs(U[::-1, :, 0] - U[:, :, 0]).max() <= 1e-10 * scale
    assert np.abs(U[::-1, :, 1] + U[:, :, 1]).max() <= 1e-10 * scale
    # no flow through the mirror lines (the quarter's free-slip walls)
    assert np.abs(U[:, case.N, 0]).max() <= 1e-10 * scale
    assert np.abs(U[case.N, :, 1]).max() <= 1e-10 * scale
    D = X - case.X0
    tree = cKDTree(case.ref_xy)
    mx = case.ref_xy.copy()
    mx[:, 0] = 1.0 - mx[:, 0]
    ix = tree.query(mx)[1]
    assert np.abs(case.ref_xy[ix] - mx).max() < 1e-12
    dmax = np.abs(D).max()
    assert np.abs(D[ix, 0] + D[:, 0]).max() <= 1e-10 * dmax
    assert np.abs(D[ix, 1] - D[:, 1]).max() <= 1e-10 * dmax
