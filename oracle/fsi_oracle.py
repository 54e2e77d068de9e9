"""CPU oracle for one time step of the DLM fictitious-domain FSI method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The GPU library never calls it, and it shares no code with the GPU
path; the only common module is ``fsi_inputs`` (seeded meshes and initial
data, no arithmetic of the method).

It is a plain, slow, FP64 restatement of the paper's discrete problem
(Boffi, Credali, Gastaldi, Scacchi, "A parallel solver for FSI problems with
fictitious domain approach", arXiv:2301.10041):

* Problem 2 (Section 3): Navier-Stokes without convection, rho_s = rho_f, so
  the solid inertia term vanishes; a(u, v) = nu (eps(u), eps(v)) with
  eps(u) = (grad u + grad u^T)/2 and no factor 2.
* Section 4: backward Euler in time; the coupling terms use the old solid
  position X^n and the new velocity u^{n+1} (the matrix of Eq. (matrix)).
* Fluid: Q2 velocity / P1-discontinuous pressure on a uniform N x N grid of
  the unit square (Section 4); pressure basis per cell {1, (x-xc)/h, (y-yc)/h}.
* Solid and multiplier: one space S_h = Lambda_h (Section 4), so the duality
  pairing is the L2(B) product and C_s is its mass matrix: P1 on triangles,
  or Q1 on quadrilaterals (the annulus test of Section 6), integrated by a
  3 x 3 Gauss rule.
* P(F) = kappa F (Section 4, before Eq. (matrix)): A_s = kappa (grad chi_j,
  grad chi_i)_B per component.
* C_f(X^n)_{l j} = (chi_l, phi_j(X^n))_B is computed in one of two ways:
  by locating every solid quadrature point in the fluid grid (brute force
  over all cells) and evaluating the Q2 basis there, with a 6-point degree-4
  symmetric triangle rule (Dunavant 1985); or exactly, as the paper does
  (Section 4), by intersecting each mapped solid triangle with the fluid
  cells (Sutherland-Hodgman) and integrating on the pieces with a degree-5
  rule (``assemble_coupling_exact``).
* The block system of Eq. (matrix) is solved by a sparse direct solve with a
  bordering row that fixes the pressure mean (p in L^2_0, Problem 2).

Readings where the paper is silent or inconsistent are documented at the
function that applies them.  Every function below is a direct transcription
of a definition; nothing is blocked, fused or reordered.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# --------------------------------------------------------------------------
# Quadrature and reference basis functions
# --------------------------------------------------------------------------


def gauss01(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (nodes, weights)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def q2_1d(t):
    """1-D quadratic Lagrange basis on [0,1] with nodes 0, 1/2, 1 (Q2 factor)."""
    t = np.asarray(t, dtype=np.float64)
    return np.stack([(1.0 - t) * (1.0 - 2.0 * t), 4.0 * t * (1.0 - t), t * (2.0 * t - 1.0)], axis=-1)


def q2_1d_deriv(t):
    """Derivatives d/dt of ``q2_1d``."""
    t = np.asarray(t, dtype=np.float64)
    return np.stack([4.0 * t - 3.0, 4.0 - 8.0 * t, 4.0 * t - 1.0], axis=-1)


# Dunavant (1985) degree-4 symmetric rule, 6 points, weights normalised to 1.
# Orbit (a, a, 1-2a) for a = A1 (weight W1) and a = A2 (weight W2).
A1 = 0.44594849091596488632
A2 = 0.091576213509770743460
W1 = 0.22338158967801146570
W2 = 0.10995174365532186764


def triangle_rule():
    """Barycentric points (lam0, lam1, lam2) and weights of the 6-point rule.

    Point order: for each orbit a in (A1, A2) the vertex with the odd
    coordinate 1-2a cycles through lam0, lam1, lam2.
    """
    pts = []
    wts = []
    for a, w in ((A1, W1), (A2, W2)):
        b = 1.0 - 2.0 * a
        pts += [(b, a, a), (a, b, a), (a, a, b)]
        wts += [w, w, w]
    return np.array(pts), np.array(wts)


# --------------------------------------------------------------------------
# Fluid: node numbering and element matrices (Section 4, Eq. (matrix))
# --------------------------------------------------------------------------


class FluidGrid:
    """Uniform N x N grid of [0,1]^2 with Q2 nodes on a (2N+1)^2 lattice.

    Node id = iy * (2N+1) + ix; velocity dof = 2 * node + component.
    Cell id = cy * N + cx; pressure dof = 3 * cell + k with basis
    psi_0 = 1, psi_1 = (x - xc)/h, psi_2 = (y - yc)/h.
    """

    def __init__(self, N: int):
        self.N = N
        self.h = 1.0 / N
        self.n1 = 2 * N + 1
        self.n_nodes = self.n1 * self.n1
        cx, cy = np.meshgrid(np.arange(N), np.arange(N))
        cx = cx.ravel()
        cy = cy.ravel()
        # local node (a, b) of cell (cx, cy) is lattice node (2cx + a, 2cy + b); local id = 3b + a
        a = np.tile(np.arange(3), 3)
        b = np.repeat(np.arange(3), 3)
        self.cell_nodes = (2 * cy[:, None] + b[None, :]) * self.n1 + (2 * cx[:, None] + a[None, :])
        ix, iy = np.meshgrid(np.arange(self.n1), np.arange(self.n1))
        ix = ix.ravel()
        iy = iy.ravel()
        self.node_xy = np.stack([ix * (self.h / 2), iy * (self.h / 2)], axis=1)
        self.boundary = (ix == 0) | (iy == 0) | (ix == self.n1 - 1) | (iy == self.n1 - 1)
        self.interior_nodes = np.nonzero(~self.boundary)[0]
        bd = np.zeros(2 * self.n_nodes, dtype=bool)
        bd[0::2] = self.boundary
        bd[1::2] = self.boundary
        self.dof_boundary = bd
        self.interior_dofs = np.nonzero(~bd)[0]
        self.boundary_dofs = np.nonzero(bd)[0]


def fluid_element_matrices(h: float, nu: float):
    """Element matrices of one square cell of side h by 3x3 Gauss quadrature
    (exact for the polynomial integrands of Q2 x Q2 and Q2 x P1).

    Returns (M 18x18, K 18x18, B 3x18) in local dof order 2*(3b + a) + c:
    M_{ij} = (phi_j, phi_i), K_{ij} = nu (eps(phi_j), eps(phi_i)),
    B_{ki} = (div phi_i, psi_k)  (the definitions after Eq. (matrix)).
    """
    t, w = gauss01(3)
    M = np.zeros((18, 18))
    K = np.zeros((18, 18))
    B = np.zeros((3, 18))
    for qy in range(3):
        for qx in range(3):
            wt = w[qx] * w[qy] * h * h
            Lx, Ly = q2_1d(t[qx]), q2_1d(t[qy])
            dLx, dLy = q2_1d_deriv(t[qx]) / h, q2_1d_deriv(t[qy]) / h
            val = np.zeros(9)
            gx = np.zeros(9)
            gy = np.zeros(9)
            for b in range(3):
                for a in range(3):
                    loc = 3 * b + a
                    val[loc] = Lx[a] * Ly[b]
                    gx[loc] = dLx[a] * Ly[b]
                    gy[loc] = Lx[a] * dLy[b]
            # pressure basis at the point, cell centre at (h/2, h/2)
            psi = np.array([1.0, t[qx] - 0.5, t[qy] - 0.5])
            for i in range(9):
                for c in range(2):
                    I = 2 * i + c
                    # eps(phi_i e_c) as a 2x2 matrix
                    G = np.zeros((2, 2))
                    G[c, 0] = gx[i]
                    G[c, 1] = gy[i]
                    Ei = 0.5 * (G + G.T)
                    divi = G[0, 0] + G[1, 1]
                    B[:, I] += wt * divi * psi
                    for j in range(9):
                        for d in range(2):
                            J = 2 * j + d
                            H = np.zeros((2, 2))
                            H[d, 0] = gx[j]
                            H[d, 1] = gy[j]
                            Ej = 0.5 * (H + H.T)
                            K[I, J] += wt * nu * np.sum(Ei * Ej)
                            if c == d:
                                M[I, J] += wt * val[i] * val[j]
    return M, K, B


def assemble_fluid(grid: FluidGrid, nu: float):
    """Global M_f, K_f (2 n_nodes square) and B (3 N^2 x 2 n_nodes), all nodes."""
    M_e, K_e, B_e = fluid_element_matrices(grid.h, nu)
    nc = grid.N * grid.N
    dofs = np.empty((nc, 18), dtype=np.int64)
    dofs[:, 0::2] = 2 * grid.cell_nodes
    dofs[:, 1::2] = 2 * grid.cell_nodes + 1
    rows = np.repeat(dofs, 18, axis=1).ravel()
    cols = np.tile(dofs, (1, 18)).ravel()
    nd = 2 * grid.n_nodes
    M = sp.coo_matrix((np.tile(M_e.ravel(), nc), (rows, cols)), shape=(nd, nd)).tocsr()
    K = sp.coo_matrix((np.tile(K_e.ravel(), nc), (rows, cols)), shape=(nd, nd)).tocsr()
    prow = (3 * np.arange(nc)[:, None] + np.arange(3)[None, :])
    brows = np.repeat(prow, 18, axis=1).ravel()
    bcols = np.tile(dofs, (1, 3)).ravel()
    B = sp.coo_matrix((np.tile(B_e.ravel(), nc), (brows, bcols)), shape=(3 * nc, nd)).tocsr()
    return M, K, B


# --------------------------------------------------------------------------
# Solid: P1 matrices (Section 4; A_s and C_s after Eq. (matrix))
# --------------------------------------------------------------------------


def p1_geometry(xy: np.ndarray, tris: np.ndarray):
    """Signed areas and barycentric gradients of each triangle."""
    P0, P1, P2 = xy[tris[:, 0]], xy[tris[:, 1]], xy[tris[:, 2]]
    d1 = P1 - P0
    d2 = P2 - P0
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    area = 0.5 * det
    # grad lam1 = (d2_y, -d2_x)/det, grad lam2 = (-d1_y, d1_x)/det, grad lam0 = -(sum)
    g1 = np.stack([d2[:, 1], -d2[:, 0]], axis=1) / det[:, None]
    g2 = np.stack([-d1[:, 1], d1[:, 0]], axis=1) / det[:, None]
    g0 = -(g1 + g2)
    return area, np.stack([g0, g1, g2], axis=1)


def assemble_solid(ref_xy: np.ndarray, tris: np.ndarray, kappa: float):
    """Scalar P1 mass C (= C_s per component) and kappa * stiffness (= A_s per
    component), n_s x n_s, on the reference configuration B."""
    ns = ref_xy.shape[0]
    area, grads = p1_geometry(ref_xy, tris)
    if np.any(area <= 0):
        raise ValueError("solid triangles must be counter-clockwise and non-degenerate")
    rows = np.repeat(tris, 3, axis=1).ravel()
    cols = np.tile(tris, (1, 3)).ravel()
    mass_e = (area[:, None, None] / 12.0) * (np.ones((3, 3)) + np.eye(3))[None]
    stiff_e = kappa * area[:, None, None] * np.einsum("tad,tbd->tab", grads, grads)
    C = sp.coo_matrix((mass_e.ravel(), (rows, cols)), shape=(ns, ns)).tocsr()
    A = sp.coo_matrix((stiff_e.ravel(), (rows, cols)), shape=(ns, ns)).tocsr()
    return C, A


# --------------------------------------------------------------------------
# Solid: Q1 matrices (the quadrilateral solid of the annulus test, Section 6)
# --------------------------------------------------------------------------


def q1_rule():
    """3 x 3 Gauss-Legendre rule on the unit square [0,1]^2 from its closed
    form: 1-D nodes 1/2 and 1/2 -/+ sqrt(3/5)/2 with weights 4/9 and 5/18.
    Point q = 3 j + i sits at (s_i, t_j); returns (s, t, s*t, weight) per
    point, the product s*t rounded once in FP64 (the mapped-point formula of
    ``quadrature_points_q1`` uses it)."""
    r = 0.5 * np.sqrt(0.6)
    g = np.array([0.5 - r, 0.5, 0.5 + r])
    w1 = np.array([5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0])
    s = np.tile(g, 3)
    t = np.repeat(g, 3)
    w = np.tile(w1, 3) * np.repeat(w1, 3)
    return s, t, s * t, w


def q1_shape(s, t):
    """Bilinear shape functions of the vertices (0,0), (1,0), (1,1), (0,1)
    of the unit square, and their derivatives d/ds, d/dt; each [..., 4]."""
    s = np.asarray(s, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    chi = np.stack([(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], -1)
    ds = np.stack([-(1 - t), 1 - t, t, -t], -1)
    dt = np.stack([-(1 - s), -s, s, 1 - s], -1)
    return chi, ds, dt


def q1_geometry(xy: np.ndarray, quads: np.ndarray):
    """Jacobian determinant and physical shape-function gradients at the 9
    rule points of every quadrilateral (vertices counter-clockwise, the
    bilinear map of the unit square).  Returns det [n_el, 9] and grads
    [n_el, 9, 4, 2]."""
    s, t, _, _ = q1_rule()
    _, ds, dt = q1_shape(s, t)                              # [9, 4]
    P = xy[quads]                                           # [n_el, 4, 2]
    Js = np.einsum("qa,ead->eqd", ds, P)                    # dx/ds  [n_el, 9, 2]
    Jt = np.einsum("qa,ead->eqd", dt, P)                    # dx/dt
    det = Js[..., 0] * Jt[..., 1] - Js[..., 1] * Jt[..., 0]
    # grad chi = J^-T (dchi/ds, dchi/dt), J = [[Js_x, Jt_x], [Js_y, Jt_y]]
    gx = (Jt[..., 1, None] * ds[None] - Js[..., 1, None] * dt[None]) / det[..., None]
    gy = (-Jt[..., 0, None] * ds[None] + Js[..., 0, None] * dt[None]) / det[..., None]
    return det, np.stack([gx, gy], -1)


def assemble_solid_q1(ref_xy: np.ndarray, quads: np.ndarray, kappa: float):
    """Scalar Q1 mass C and kappa * stiffness A on the reference
    configuration, by the 3 x 3 Gauss rule on each quadrilateral.  The mass
    integrand (bilinear x bilinear x the bilinear |det J|) is integrated
    exactly; the stiffness integrand is rational on a general quadrilateral
    and the rule is the stated reading (exact on parallelograms)."""
    ns = ref_xy.shape[0]
    s, t, _, w = q1_rule()
    chi, _, _ = q1_shape(s, t)
    det, grads = q1_geometry(ref_xy, quads)
    if np.any(det <= 0):
        raise ValueError("solid quadrilaterals must be counter-clockwise and non-degenerate")
    wd = w[None, :] * det                                   # [n_el, 9]
    mass_e = np.einsum("eq,qa,qb->eab", wd, chi, chi)
    stiff_e = kappa * np.einsum("eq,eqad,eqbd->eab", wd, grads, grads)
    rows = np.repeat(quads, 4, axis=1).ravel()
    cols = np.tile(quads, (1, 4)).ravel()
    C = sp.coo_matrix((mass_e.ravel(), (rows, cols)), shape=(ns, ns)).tocsr()
    A = sp.coo_matrix((stiff_e.ravel(), (rows, cols)), shape=(ns, ns)).tocsr()
    return C, A


def solid_matrices(ref_xy: np.ndarray, elems: np.ndarray, kappa: float):
    """(C, A) of the solid space: P1 for triangles, Q1 for quadrilaterals."""
    if elems.shape[1] == 4:
        return assemble_solid_q1(ref_xy, elems, kappa)
    return assemble_solid(ref_xy, elems, kappa)


# --------------------------------------------------------------------------
# Coupling: point location and C_f(X^n) (Section 4, "coupling matrix")
# --------------------------------------------------------------------------

OUT_OF_DOMAIN = -1


def quadrature_points(X: np.ndarray, tris: np.ndarray):
    """Physical positions X^n(s_q) of all rule points, shape [n_tri*6, 2].

    Reading (the paper does not fix it): the mapped point is
    x = P0 + xi1 (P1 - P0) + xi2 (P2 - P0) with (xi1, xi2) = (lam1, lam2),
    evaluated left to right in round-to-nearest FP64 with no fused
    multiply-add, so that any implementation reproduces it bit for bit.
    Point id = 6 * triangle + q.
    """
    lam, _ = triangle_rule()
    P0 = X[tris[:, 0]][:, None, :]
    P1 = X[tris[:, 1]][:, None, :]
    P2 = X[tris[:, 2]][:, None, :]
    xi1 = lam[None, :, 1, None]
    xi2 = lam[None, :, 2, None]
    d1 = P1 - P0
    d2 = P2 - P0
    t1 = xi1 * d1
    t2 = xi2 * d2
    x = (P0 + t1) + t2
    return x.reshape(-1, 2)


def quadrature_points_q1(X: np.ndarray, quads: np.ndarray):
    """Physical positions X^n(s_q) of the 9 rule points of every
    quadrilateral, shape [n_el*9, 2], point id = 9 * element + q.

    Reading (the paper does not fix it): with d1 = P1 - P0, d3 = P3 - P0 and
    e = (P2 - P3) - d1, the bilinear map is evaluated as
    x = ((P0 + s d1) + t d3) + (s t) e, left to right in round-to-nearest FP64
    with no fused multiply-add, so that any implementation reproduces it bit
    for bit.
    """
    s, t, st, _ = q1_rule()
    P0 = X[quads[:, 0]][:, None, :]
    P1 = X[quads[:, 1]][:, None, :]
    P2 = X[quads[:, 2]][:, None, :]
    P3 = X[quads[:, 3]][:, None, :]
    d1 = P1 - P0
    d3 = P3 - P0
    e = (P2 - P3) - d1
    a = s[None, :, None] * d1
    b = t[None, :, None] * d3
    c = st[None, :, None] * e
    x = ((P0 + a) + b) + c
    return x.reshape(-1, 2)


def locate_brute_force(x: np.ndarray, N: int):
    """Cell (cx, cy) and local coordinates (xi, eta) of each point.

    Reading of the cell rule (the paper only says the fluid mesh is
    Cartesian): with t = fl(x * N), the point lies in cell i when
    i <= t < i + 1, except that t = N belongs to the last cell; points with
    x < 0 or x > 1 (or NaN) are outside the domain and get cell -1.  This
    routine tests every candidate cell index in turn (brute force over the
    grid lines) rather than taking a floor.
    Returns (cell_id int64, xi, eta) with cell_id = cy * N + cx.
    """
    n = x.shape[0]
    idx = np.full((n, 2), -1, dtype=np.int64)
    loc = np.zeros((n, 2))
    for c in range(2):
        t = x[:, c] * float(N)
        inside = (x[:, c] >= 0.0) & (x[:, c] <= 1.0)
        for i in range(N):
            hit = inside & (t >= float(i)) & ((t < float(i + 1)) | ((i == N - 1) & (t == float(N))))
            idx[hit, c] = i
        loc[:, c] = t - idx[:, c]
    cell = np.where((idx[:, 0] >= 0) & (idx[:, 1] >= 0), idx[:, 1] * N + idx[:, 0], OUT_OF_DOMAIN)
    loc[cell < 0] = 0.0
    return cell, loc[:, 0], loc[:, 1]


def assemble_coupling(grid: FluidGrid, ref_xy: np.ndarray, tris: np.ndarray, X: np.ndarray):
    """Scalar coupling matrix C (n_s x n_nodes) with
    C_{l j} = sum_T sum_q |T| w_q chi_l(s_q) phi_j(X^n(s_q))  ~  (chi_l, phi_j(X^n))_B,
    where |T| is the reference-triangle area (the integral is over B).
    C_f = C acting on each velocity component.  Raises on a point outside
    the fluid domain.  Also returns the point locations.
    With quadrilaterals (4 node ids per element) the solid space is Q1 and
    the rule is the 3 x 3 Gauss rule of ``q1_rule``:
    C_{l j} = sum_E sum_q w_q |det J_E(s_q)| chi_l(s_q) phi_j(X^n(s_q))."""
    if tris.shape[1] == 4:
        return assemble_coupling_q1(grid, ref_xy, tris, X)
    lam, w = triangle_rule()
    area, _ = p1_geometry(ref_xy, tris)
    x = quadrature_points(X, tris)
    cell, xi, eta = locate_brute_force(x, grid.N)
    if np.any(cell < 0):
        raise ValueError("solid quadrature point outside the fluid domain")
    ntri = tris.shape[0]
    Lx = q2_1d(xi)            # [npts, 3]
    Ly = q2_1d(eta)
    phi = (Ly[:, :, None] * Lx[:, None, :]).reshape(-1, 9)   # local id 3b + a
    fluid_nodes = grid.cell_nodes[cell]                     # [npts, 9]
    wq = (area[:, None] * w[None, :]).ravel()               # [npts]
    chi = np.tile(lam, (ntri, 1))                           # [npts, 3]
    solid_nodes = np.repeat(tris, 6, axis=0)                # [npts, 3]
    vals = wq[:, None, None] * chi[:, :, None] * phi[:, None, :]
    rows = np.repeat(solid_nodes[:, :, None], 9, axis=2)
    cols = np.repeat(fluid_nodes[:, None, :], 3, axis=1)
    C = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())),
                      shape=(ref_xy.shape[0], grid.n_nodes)).tocsr()
    return C, (x, cell, xi, eta)


def assemble_coupling_q1(grid: FluidGrid, ref_xy: np.ndarray, quads: np.ndarray, X: np.ndarray):
    """C_f for a Q1 solid (see ``assemble_coupling``): the reference-element
    weights w_q |det J_E(s_q)| come from the reference configuration B."""
    s, t, _, w = q1_rule()
    chi, _, _ = q1_shape(s, t)                               # [9, 4]
    det, _ = q1_geometry(ref_xy, quads)
    x = quadrature_points_q1(X, quads)
    cell, xi, eta = locate_brute_force(x, grid.N)
    if np.any(cell < 0):
        raise ValueError("solid quadrature point outside the fluid domain")
    nel = quads.shape[0]
    Lx = q2_1d(xi)
    Ly = q2_1d(eta)
    phi = (Ly[:, :, None] * Lx[:, None, :]).reshape(-1, 9)
    fluid_nodes = grid.cell_nodes[cell]
    wq = (w[None, :] * det).ravel()
    chis = np.tile(chi, (nel, 1))                            # [npts, 4]
    solid_nodes = np.repeat(quads, 9, axis=0)                # [npts, 4]
    vals = wq[:, None, None] * chis[:, :, None] * phi[:, None, :]
    rows = np.repeat(solid_nodes[:, :, None], 9, axis=2)
    cols = np.repeat(fluid_nodes[:, None, :], 4, axis=1)
    C = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())),
                      shape=(ref_xy.shape[0], grid.n_nodes)).tocsr()
    return C, (x, cell, xi, eta)


# --------------------------------------------------------------------------
# Exact coupling by mesh intersection (Section 4: the paper's own rule)
# --------------------------------------------------------------------------


def radon_rule():
    """Radon's 7-point symmetric rule on a triangle, exact for degree 5
    (Radon 1948; Stroud's T2:5-1), from its closed form: the centroid with
    weight 9/40 and the orbits (a, a, 1-2a), a = (6 -/+ sqrt 15)/21, with
    weights (155 -/+ sqrt 15)/1200.  Barycentric points, weights summing to 1."""
    r = np.sqrt(15.0)
    pts = [(1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)]
    wts = [9.0 / 40.0]
    for a, w in (((6.0 - r) / 21.0, (155.0 - r) / 1200.0), ((6.0 + r) / 21.0, (155.0 + r) / 1200.0)):
        b = 1.0 - 2.0 * a
        pts += [(b, a, a), (a, b, a), (a, a, b)]
        wts += [w, w, w]
    return np.array(pts), np.array(wts)


def clip_half_plane(poly, axis: int, value: float, keep_below: bool):
    """One Sutherland-Hodgman pass: the part of a convex polygon (list of
    2-vectors, in order) with x[axis] <= value (keep_below) or >= value.
    A crossing edge contributes its intersection point, whose clipped
    coordinate is set to `value` exactly."""
    out = []
    n = len(poly)
    for i in range(n):
        P, Q = poly[i], poly[(i + 1) % n]
        inP = P[axis] <= value if keep_below else P[axis] >= value
        inQ = Q[axis] <= value if keep_below else Q[axis] >= value
        if inP:
            out.append(P)
        if inP != inQ:
            t = (value - P[axis]) / (Q[axis] - P[axis])
            R = P + t * (Q - P)
            R[axis] = value
            out.append(R)
    return out


def clip_to_cell(P: np.ndarray, x0: float, x1: float, y0: float, y1: float):
    """Intersection of the triangle P (3 x 2) with the square [x0,x1] x
    [y0,y1] by four Sutherland-Hodgman passes (Section 4); [] if empty."""
    poly = [P[0].copy(), P[1].copy(), P[2].copy()]
    for axis, value, below in ((0, x0, False), (0, x1, True), (1, y0, False), (1, y1, True)):
        poly = clip_half_plane(poly, axis, value, below)
        if len(poly) < 3:
            return []
    return poly


def assemble_coupling_exact(grid: FluidGrid, ref_xy: np.ndarray, tris: np.ndarray, X: np.ndarray):
    """Scalar coupling matrix C (n_s x n_nodes), C_{l j} = (chi_l, phi_j(X^n))_B,
    integrated exactly as in Section 4.  On a solid triangle E the map X^n is
    affine, so the integral over E equals (|E| / |X(E)|) times the integral
    over the mapped triangle X(E) of lambda_l(x) phi_j(x), lambda_l the
    barycentric coordinate of X(E).  X(E) is intersected with every fluid cell
    its bounding box touches (Sutherland-Hodgman), each intersection polygon
    is split into triangles from its first vertex, and the integrand (linear
    times biquadratic: degree 5) is integrated by Radon's degree-5 rule.
    Raises on a vertex outside the fluid domain or a degenerate image."""
    N, h = grid.N, grid.h
    lam_q, w_q = radon_rule()
    area_ref, _ = p1_geometry(ref_xy, tris)
    rows, cols, vals = [], [], []
    for t in range(tris.shape[0]):
        P = np.asarray(X[tris[t]], dtype=np.float64)
        if np.any(P < 0.0) or np.any(P > 1.0):
            raise ValueError("mapped solid vertex outside the fluid domain")
        d1, d2 = P[1] - P[0], P[2] - P[0]
        det = d1[0] * d2[1] - d1[1] * d2[0]
        if det == 0.0:
            raise ValueError("degenerate mapped solid triangle")
        scale = area_ref[t] / (0.5 * abs(det))
        lo = np.minimum(np.floor(P.min(axis=0) * N).astype(np.int64), N - 1)
        hi = np.minimum(np.floor(P.max(axis=0) * N).astype(np.int64), N - 1)
        for cy in range(lo[1], hi[1] + 1):
            for cx in range(lo[0], hi[0] + 1):
                poly = clip_to_cell(P, cx * h, (cx + 1) * h, cy * h, (cy + 1) * h)
                acc = np.zeros((3, 9))
                for i in range(1, len(poly) - 1):
                    S = np.array([poly[0], poly[i], poly[i + 1]])
                    e1, e2 = S[1] - S[0], S[2] - S[0]
                    a_sub = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
                    if a_sub == 0.0:
                        continue
                    xq = lam_q @ S                                   # 7 x 2 points
                    r = xq - P[0]
                    l1 = (r[:, 0] * d2[1] - r[:, 1] * d2[0]) / det
                    l2 = (d1[0] * r[:, 1] - d1[1] * r[:, 0]) / det
                    lam = np.stack([1.0 - l1 - l2, l1, l2], axis=1)  # 7 x 3
                    phi = (q2_1d((xq[:, 1] - cy * h) / h)[:, :, None]
                           * q2_1d((xq[:, 0] - cx * h) / h)[:, None, :]).reshape(-1, 9)  # local id 3b + a
                    acc += a_sub * np.einsum("q,qa,qj->aj", w_q, lam, phi)
                if not acc.any():
                    continue
                rows.append(np.repeat(tris[t], 9))
                cols.append(np.tile(grid.cell_nodes[cy * N + cx], 3))
                vals.append((scale * acc).ravel())
    C = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ref_xy.shape[0], grid.n_nodes)).tocsr()
    return C


# --------------------------------------------------------------------------
# Nonlinear solid (Section 6, bar test): exponential strain energy
# --------------------------------------------------------------------------


def exp_law_energy(F, gamma: float, eta: float):
    """W(F) = (gamma / (2 eta)) exp(eta (tr(F^T F) - 2)) per element, F [t, 2, 2]."""
    n2 = np.einsum("tck,tck->t", F, F)
    return (gamma / (2.0 * eta)) * np.exp(eta * (n2 - 2.0))


def deformation_gradients(ref_xy: np.ndarray, tris: np.ndarray, X: np.ndarray):
    """F_E = dX/ds on every P1 triangle (constant): F[t, c, k] = sum_v X_{v,c} d chi_v / d s_k."""
    _, grads = p1_geometry(ref_xy, tris)                     # [t, 3, 2]
    return np.einsum("tvc,tvk->tck", X[tris], grads)


def solid_nonlinear(ref_xy: np.ndarray, tris: np.ndarray, X: np.ndarray, gamma: float, eta: float):
    """The solid term (P(F), grad Y)_B of Problem 3 for P = dW/dF =
    gamma exp(eta (|F|^2 - 2)) F, and its derivative in X.

    Returns S [n_s, 2] with S_i = sum_E |E| P(F_E) grad chi_i, and the
    tangent K_T = dS/dX as a sparse (2 n_s x 2 n_s) matrix in the order
    2*node + component:
      K_T[(i,d),(j,c)] = sum_E |E| e (delta_dc grad chi_j . grad chi_i
                                      + 2 eta (F grad chi_j)_c (F grad chi_i)_d),
    e = gamma exp(eta (|F|^2 - 2))."""
    area, grads = p1_geometry(ref_xy, tris)
    F = deformation_gradients(ref_xy, tris, X)
    e = gamma * np.exp(eta * (np.einsum("tck,tck->t", F, F) - 2.0))
    ns = ref_xy.shape[0]
    S = np.zeros((ns, 2))
    FG = np.einsum("tck,tvk->tvc", F, grads)                  # (F grad chi_v)_c
    np.add.at(S, tris, (area * e)[:, None, None] * FG)
    rows, cols, vals = [], [], []
    for v in range(3):
        for w in range(3):
            gg = np.einsum("tk,tk->t", grads[:, v], grads[:, w])
            for d in range(2):
                for c in range(2):
                    val = area * e * ((1.0 if d == c else 0.0) * gg + 2.0 * eta * FG[:, w, c] * FG[:, v, d])
                    rows.append(2 * tris[:, v] + d)
                    cols.append(2 * tris[:, w] + c)
                    vals.append(val)
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * ns, 2 * ns)).tocsr()
    return S, K


def kron2(A):
    """Scalar operator acting on both components of interleaved 2-vectors."""
    return sp.kron(A, sp.identity(2), format="csr")


# --------------------------------------------------------------------------
# One time step: the block system of Eq. (matrix)
# --------------------------------------------------------------------------


def nested_dissection(G, xy, leaf: int = 64):
    """Fill-reducing elimination order for the direct solve (George 1973,
    geometric variant): split the unknowns at the coordinate median along
    the longer extent, take as separator the unknowns of the first half
    that are connected to the second half, order both halves recursively
    and the separator last."""
    G = G.tocsr()

    def rec(idx):
        if idx.size <= leaf:
            return [idx]
        pts = xy[idx]
        ext = pts.max(0) - pts.min(0)
        d = 0 if ext[0] >= ext[1] else 1
        left = pts[:, d] <= np.median(pts[:, d])
        if left.all() or (~left).all():
            order = np.argsort(pts[:, d], kind="stable")
            left = np.zeros(idx.size, dtype=bool)
            left[order[: idx.size // 2]] = True
        sub = G[idx][:, idx]
        Li = np.nonzero(left)[0]
        Ri = np.nonzero(~left)[0]
        cross = sub[Li][:, Ri]
        sep = np.zeros(idx.size, dtype=bool)
        sep[Li[np.diff(cross.indptr) > 0]] = True
        return rec(idx[left & ~sep]) + rec(idx[~left]) + [idx[sep]]

    return np.concatenate(rec(np.arange(G.shape[0])))


class OracleProblem:
    """Constant matrices of one FSI instance (the paper's T_ass work)."""

    def __init__(self, N, rho_f, nu, kappa, dt, lid_u, ref_xy, tris, coupling: str = "point",
                 solid_law: str = "linear", gamma: float = 0.0, eta: float = 0.0, newton_tol: float = 1e-6,
                 newton_max: int = 30):
        """coupling: "point" (the degree-4 point rule with point location) or
        "exact" (mesh intersection, the paper's rule of Section 4).
        solid_law: "linear" (P = kappa F) or "exp" (the exponential strain
        energy of the bar test, Section 6, solved by Newton's method)."""
        self.N, self.rho, self.nu, self.kappa, self.dt, self.lid_u = N, rho_f, nu, kappa, dt, lid_u
        if coupling not in ("point", "exact"):
            raise ValueError("coupling")
        if solid_law not in ("linear", "exp"):
            raise ValueError("solid_law")
        self.coupling = coupling
        self.solid_law, self.gamma, self.eta = solid_law, gamma, eta
        self.newton_tol, self.newton_max = newton_tol, newton_max
        self.newton_history = []
        self.grid = FluidGrid(N)
        self.ref_xy = np.asarray(ref_xy, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        if self.tris.shape[1] == 4 and (coupling != "point" or solid_law != "linear"):
            raise ValueError("the Q1 solid takes the point rule and the linear law only")
        self.M, self.K, self.B = assemble_fluid(self.grid, nu)
        self.A = (rho_f / dt) * self.M + self.K
        Cs, As = solid_matrices(self.ref_xy, self.tris, kappa)
        self.Cs_scalar, self.As_scalar = Cs, As
        self.Cs = kron2(Cs)
        self.As = kron2(As)
        g = self.grid
        self.I = g.interior_dofs
        self.D = g.boundary_dofs
        # boundary data: walls at rest, lid (lid_u, 0) strictly between the top corners
        uD = np.zeros((g.n_nodes, 2))
        if lid_u != 0.0:
            top = (g.n1 - 1) * g.n1 + np.arange(1, g.n1 - 1)
            uD[top, 0] = lid_u
        self.u_wall = uD

    def system(self, u_nodal, X, X_iter=None):
        """Block matrix of Eq. (matrix) on interior velocity dofs and its
        right-hand side, for the state (u^n, X^n).

        Rows: [u_I; p; X; lambda], RHS (Dirichlet data u_D moved right):
          A_II u - B_I^T p + C_I^T lam = (rho/dt) M_{I,:} u^n - A_ID u_D
          -B_I u                        = B_D u_D
          A_s X - C_s lam               = 0
          C_I u - (1/dt) C_s X          = -(1/dt) C_s X^n - C_D u_D
        Reading: the constraint row uses u^{n+1}, as the matrix does (the
        printed Problem 3 writes u^n there; Section 4 text and the matrix
        both use u^{n+1}).
        """
        I, D = self.I, self.D
        if self.coupling == "exact":
            Cscal, loc = assemble_coupling_exact(self.grid, self.ref_xy, self.tris, X), None
        else:
            Cscal, loc = assemble_coupling(self.grid, self.ref_xy, self.tris, X)
        Cf = kron2(Cscal)
        uD = self.u_wall.reshape(-1)[D]
        un = np.asarray(u_nodal, dtype=np.float64).reshape(-1)
        Xn = np.asarray(X, dtype=np.float64).reshape(-1)
        A_II = self.A[I][:, I]
        A_ID = self.A[I][:, D]
        B_I = self.B[:, I]
        B_D = self.B[:, D]
        C_I = Cf[:, I]
        C_D = Cf[:, D]
        Z = None
        # solid row: linear law A_s X; exponential law linearised at the
        # Newton iterate X_k: K_T(X_k) X = K_T(X_k) X_k - S(X_k) + ...
        if self.solid_law == "exp":
            Xk = np.asarray(X if X_iter is None else X_iter, dtype=np.float64)
            S, KT = solid_nonlinear(self.ref_xy, self.tris, Xk, self.gamma, self.eta)
            Asolid = KT
            g3 = KT @ Xk.reshape(-1) - S.reshape(-1)
        else:
            Asolid = self.As
            g3 = np.zeros(Xn.size)
        Kmat = sp.bmat([[A_II, -B_I.T, Z, C_I.T],
                        [-B_I, Z, Z, Z],
                        [Z, Z, Asolid, -self.Cs],
                        [C_I, Z, -(1.0 / self.dt) * self.Cs, Z]], format="csr")
        g1 = (self.rho / self.dt) * (self.M[I] @ un) - A_ID @ uD
        g2 = B_D @ uD
        g4 = -(1.0 / self.dt) * (self.Cs @ Xn) - C_D @ uD
        rhs = np.concatenate([g1, g2, g3, g4])
        return Kmat, rhs, loc

    def sizes(self):
        n_u = self.I.size
        n_p = 3 * self.N * self.N
        n_x = 2 * self.ref_xy.shape[0]
        return n_u, n_p, n_x

    def unknown_coordinates(self, X):
        """A point in the plane for every unknown (used only to order the
        sparse elimination): velocity dofs at their node, pressure dofs at
        the cell centre, solid and multiplier dofs at the solid node X^n."""
        n_u, n_p, n_x = self.sizes()
        g = self.grid
        xy = np.zeros((n_u + n_p + 2 * n_x, 2))
        xy[:n_u] = g.node_xy[self.I // 2]
        cells = np.arange(self.N * self.N)
        cc = np.stack([(cells % self.N + 0.5) / self.N, (cells // self.N + 0.5) / self.N], 1)
        xy[n_u:n_u + n_p] = np.repeat(cc, 3, axis=0)
        Xs = np.repeat(np.asarray(X, dtype=np.float64).reshape(-1, 2), 2, axis=0)
        xy[n_u + n_p:n_u + n_p + n_x] = Xs
        xy[n_u + n_p + n_x:] = Xs
        return xy

    def solve_system(self, Kmat, rhs, X):
        """Sparse direct solve of Eq. (matrix) with the pressure mean fixed by
        a bordering Lagrange row (sum over cells of the constant pressure
        coefficient is zero, i.e. p in L^2_0 as in Problem 2).

        The solve is an LU factorisation with threshold partial pivoting
        (SuperLU).  Before it, rows and columns are scaled by positive
        diagonal matrices (this changes no solution, only the pivot sizes),
        and unknowns are ordered by a geometric nested dissection so that
        the factors stay sparse.  Neither step is part of the method.  One
        step of iterative refinement with the same factors follows (residual
        of the scaled bordered system in FP64, one more pair of triangular
        solves): it removes the error of pivot growth, which on badly scaled
        steps (a body at rest, whose large multiplier cancels against the
        pressure) leaves the plain LU answer several orders of magnitude
        above the rounding floor of the relative residual.
        """
        n_u, n_p, n_x = self.sizes()
        n = Kmat.shape[0]
        dt = self.dt
        # symmetric form: rows [1, 1, 1/dt, dt], multiplier unknown lambda = dt * mu
        r = np.ones(n)
        r[n_u + n_p:n_u + n_p + n_x] = 1.0 / dt
        r[n_u + n_p + n_x:] = dt
        cs = np.ones(n)
        cs[n_u + n_p + n_x:] = dt
        Ks = (sp.diags(r) @ Kmat @ sp.diags(cs)).tocsr()
        d = np.abs(Ks.diagonal())
        s = np.ones(n)
        s[d > 0] = 1.0 / np.sqrt(d[d > 0])
        Ka = abs(Ks).tocsr()
        for lo, hi in ((n_u, n_u + n_p), (n_u + n_p + n_x, n)):
            mx = (Ka[lo:hi] @ sp.diags(s)).max(axis=1).toarray().ravel()
            s[lo:hi] = 1.0 / np.maximum(mx, 1e-300)
        Kss = (sp.diags(s) @ Ks @ sp.diags(s)).tocsr()
        e = np.zeros(n)
        e[n_u:n_u + n_p:3] = 1.0
        ecol = sp.csr_matrix((e * s)[:, None])
        big = sp.bmat([[Kss, ecol], [ecol.T, None]], format="csr")
        G = abs(Kss)
        G = (G + G.T).tocsr()
        perm = np.concatenate([nested_dissection(G, self.unknown_coordinates(X)), [n]])
        P = big[perm][:, perm].tocsc()
        b = np.concatenate([s * r * rhs, [0.0]])[perm]
        lu = spla.splu(P, permc_spec="NATURAL", diag_pivot_thresh=0.01)
        yp = lu.solve(b)
        yp = yp + lu.solve(b - P @ yp)
        y = np.empty_like(yp)
        y[perm] = yp
        return cs * s * y[:n]

    def split(self, x):
        n_u, n_p, n_x = self.sizes()
        g = self.grid
        u = self.u_wall.reshape(-1).copy()
        u[self.I] = x[:n_u]
        p = x[n_u:n_u + n_p].reshape(-1, 3)
        X = x[n_u + n_p:n_u + n_p + n_x].reshape(-1, 2)
        lam = x[n_u + n_p + n_x:].reshape(-1, 2)
        return u.reshape(g.n_nodes, 2), p, X, lam

    def pack(self, u_nodal, p, X, lam):
        u = np.asarray(u_nodal).reshape(-1)[self.I]
        return np.concatenate([u, np.asarray(p).ravel(), np.asarray(X).ravel(), np.asarray(lam).ravel()])

    def step(self, u_nodal, X):
        """One backward-Euler step (Section 4): returns u^{n+1} (nodal, with
        wall values), p^{n+1} [N^2, 3], X^{n+1} [n_s, 2], lambda^{n+1} [n_s, 2]."""
        if self.solid_law == "linear":
            Kmat, rhs, _ = self.system(u_nodal, X)
            x = self.solve_system(Kmat, rhs, X)
            return self.split(x)
        # Newton's method on the nonlinear solid row (Section 4): each iterate
        # solves the block system linearised at X_k; stop when the change of X
        # is below newton_tol times the step's displacement (absolute floor
        # 1e-13)
        Xk = np.asarray(X, dtype=np.float64)
        self.newton_history = []
        for _ in range(self.newton_max):
            Kmat, rhs, _ = self.system(u_nodal, X, Xk)
            out = self.split(self.solve_system(Kmat, rhs, X))
            Xn1 = out[2]
            dX = np.max(np.abs(Xn1 - Xk))
            self.newton_history.append(dX)
            Xk = Xn1
            if dX <= max(self.newton_tol * np.max(np.abs(Xn1 - X)), 1e-13):
                return out
        raise RuntimeError("Newton did not converge")

    def relative_residual(self, u_nodal_old, X_old, u_new, p, X_new, lam):
        """||b - K x|| / ||b|| of a candidate solution in the oracle's operator
        (for the exponential law the system linearised at X_new, whose
        residual is the nonlinear one: S(X_new) - C_s lambda in the solid rows)."""
        Kmat, rhs, _ = self.system(u_nodal_old, X_old, X_new if self.solid_law == "exp" else None)
        x = self.pack(u_new, p, X_new, lam)
        return float(np.linalg.norm(rhs - Kmat @ x) / np.linalg.norm(rhs))


def run_steps(case, steps: int):
    """Advance ``steps`` time steps from the case's initial state."""
    prob = OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u,
                         case.ref_xy, case.tris)
    u = np.array(case.u0, dtype=np.float64)
    X = np.array(case.X0, dtype=np.float64)
    p = lam = None
    for _ in range(steps):
        u, p, X, lam = prob.step(u, X)
    return prob, u, p, X, lam


# --------------------------------------------------------------------------
# Generalized Stokes solve (fluid block alone), for manufactured solutions
# --------------------------------------------------------------------------


def stokes_manufactured(N: int, rho: float, nu: float, dt: float, u_exact, grad_exact, p_exact, f,
                        nq: int = 5):
    """Solve A_f u - B^T p = F, -B u = 0, p in L^2_0 with zero walls, where
    F_i = (f, phi_i) by an nq x nq Gauss rule per cell.  Returns the L2 error
    of u, the L2 error of grad u, and the L2 error of p."""
    grid = FluidGrid(N)
    M, K, B = assemble_fluid(grid, nu)
    A = (rho / dt) * M + K
    I = grid.interior_dofs
    h = grid.h
    t, w = gauss01(nq)
    F = np.zeros(2 * grid.n_nodes)
    cx = np.arange(grid.N * grid.N) % grid.N
    cy = np.arange(grid.N * grid.N) // grid.N
    for qy in range(nq):
        for qx in range(nq):
            xs = (cx + t[qx]) * h
            ys = (cy + t[qy]) * h
            fv = f(xs, ys)                                   # [nc, 2]
            phi = (q2_1d(t[qy])[:, None] * q2_1d(t[qx])[None, :]).ravel()
            wt = w[qx] * w[qy] * h * h
            for loc in range(9):
                np.add.at(F, 2 * grid.cell_nodes[:, loc], wt * phi[loc] * fv[:, 0])
                np.add.at(F, 2 * grid.cell_nodes[:, loc] + 1, wt * phi[loc] * fv[:, 1])
    nu_, np_ = I.size, 3 * grid.N * grid.N
    Kmat = sp.bmat([[A[I][:, I], -B[:, I].T], [-B[:, I], None]], format="csr")
    e = np.zeros(nu_ + np_)
    e[nu_::3] = 1.0
    ecol = sp.csr_matrix(e[:, None])
    big = sp.bmat([[Kmat, ecol], [ecol.T, None]], format="csc")
    sol = spla.spsolve(big, np.concatenate([F[I], np.zeros(np_), [0.0]]))
    u = np.zeros(2 * grid.n_nodes)
    u[I] = sol[:nu_]
    p = sol[nu_:nu_ + np_].reshape(-1, 3)
    # errors by the same Gauss rule
    eu = egu = ep = 0.0
    for qy in range(nq):
        for qx in range(nq):
            xs = (cx + t[qx]) * h
            ys = (cy + t[qy]) * h
            wt = w[qx] * w[qy] * h * h
            Lx, Ly = q2_1d(t[qx]), q2_1d(t[qy])
            dLx, dLy = q2_1d_deriv(t[qx]) / h, q2_1d_deriv(t[qy]) / h
            val = (Ly[:, None] * Lx[None, :]).ravel()
            gx = (Ly[:, None] * dLx[None, :]).ravel()
            gy = (dLy[:, None] * Lx[None, :]).ravel()
            ue = u_exact(xs, ys)
            ge = grad_exact(xs, ys)                          # [nc, 2(comp), 2(dir)]
            for c in range(2):
                uc = u[2 * grid.cell_nodes + c]               # [nc, 9]
                eu += wt * np.sum((uc @ val - ue[:, c]) ** 2)
                egu += wt * np.sum((uc @ gx - ge[:, c, 0]) ** 2 + (uc @ gy - ge[:, c, 1]) ** 2)
            ph = p[:, 0] + p[:, 1] * (t[qx] - 0.5) + p[:, 2] * (t[qy] - 0.5)
            ep += wt * np.sum((ph - p_exact(xs, ys)) ** 2)
    return np.sqrt(eu), np.sqrt(egu), np.sqrt(ep)
