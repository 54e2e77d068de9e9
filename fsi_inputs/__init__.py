"""Seeded synthetic inputs for the DLM fictitious-domain FSI step.

This module is shared by the CPU oracle (``oracle/``) and by the GPU path
(``paper_2301_10041_gb300``).  It holds no arithmetic of the method: it only
draws random numbers and lays out the geometry and initial data that both
sides receive as plain arrays.

* ``splitmix64`` is the counter-based generator of Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators" (OOPSLA 2014): value i of
  stream ``seed`` is the finaliser applied to ``seed + (i + 1) * golden``.
* ``ring_disk_mesh`` builds the concentric-ring P1 triangulation of a disk
  used for the immersed body: ring k (k = 1..m) sits at radius k R / m and
  carries 6k nodes; the strip between ring k-1 and ring k holds 6(2k-1)
  triangles, so the mesh has 1 + 3m(m+1) nodes and 6 m^2 triangles.
* ``ellipse_mesh`` maps the unit-disk ring mesh affinely onto an ellipse.
* ``initial_velocity`` draws u_0 uniform in [-1, 1] per interior velocity
  dof of the (2N+1)^2 Q2 node grid; boundary nodes carry the wall values.

Workload shapes follow the paper's experiments (Section 6: cavity-like unit
square, an elastic body at rest in the middle, 3e4 - 2e6 dofs).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx) -> np.ndarray:
    """Counter-based SplitMix64: uint64 value ``idx`` of stream ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, idx) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of ``splitmix64``."""
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _strip(inner: list[int], outer: list[int], tris: list[tuple[int, int, int]]) -> None:
    """Triangulate the annular strip between two closed rings of nodes.

    Nodes of each ring are equally spaced in angle starting at angle 0.  The
    two rings are merged in angular order (exact integer comparison of
    (j+1)/n_out against (i+1)/n_in); each step emits one counter-clockwise
    triangle, so the strip gets n_in + n_out triangles.
    """
    n_in, n_out = len(inner), len(outer)
    if n_in == 1:
        c = inner[0]
        for j in range(n_out):
            tris.append((c, outer[j], outer[(j + 1) % n_out]))
        return
    i = j = 0
    while i < n_in or j < n_out:
        adv_outer = j < n_out and (i == n_in or (j + 1) * n_in <= (i + 1) * n_out)
        if adv_outer:
            tris.append((inner[i % n_in], outer[j], outer[(j + 1) % n_out]))
            j += 1
        else:
            tris.append((inner[i], outer[j % n_out], inner[(i + 1) % n_in]))
            i += 1


def ring_disk_mesh(m: int, radius: float = 1.0, center=(0.0, 0.0)):
    """Concentric-ring triangulation of a disk; returns (xy[n,2], tris[t,3])."""
    if m < 1:
        raise ValueError("m must be >= 1")
    xy = [(0.0, 0.0)]
    rings = [[0]]
    for k in range(1, m + 1):
        n = 6 * k
        base = len(xy)
        r = radius * k / m
        for j in range(n):
            th = 2.0 * math.pi * j / n
            xy.append((r * math.cos(th), r * math.sin(th)))
        rings.append(list(range(base, base + n)))
    tris: list[tuple[int, int, int]] = []
    for k in range(1, m + 1):
        _strip(rings[k - 1], rings[k], tris)
    xy = np.asarray(xy, dtype=np.float64)
    xy[:, 0] += center[0]
    xy[:, 1] += center[1]
    return xy, np.asarray(tris, dtype=np.int32)


def ellipse_mesh(m: int, a: float, b: float, angle_deg: float, center=(0.5, 0.5)):
    """Ring mesh of the unit disk mapped onto an ellipse with semi-axes a, b
    rotated by ``angle_deg`` about ``center``."""
    xy, tris = ring_disk_mesh(m, 1.0)
    th = math.radians(angle_deg)
    c, s = math.cos(th), math.sin(th)
    x = a * xy[:, 0]
    y = b * xy[:, 1]
    out = np.empty_like(xy)
    out[:, 0] = center[0] + c * x - s * y
    out[:, 1] = center[1] + s * x + c * y
    return out, tris


def bar_mesh(nx: int, ny: int, x0: float = 0.0, x1: float = 0.4, y0: float = 0.45, y1: float = 0.55):
    """Structured P1 triangulation of the rectangle [x0,x1] x [y0,y1]
    ((nx+1)(ny+1) nodes, row-major from the bottom left; each grid square cut
    by the diagonal from its bottom-left corner, counter-clockwise)."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys)
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    tris = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, d = a + 1, a + nx + 2, a + nx + 1
            tris += [(a, b, c), (a, c, d)]
    return xy, np.array(tris, dtype=np.int32)


def bar_case(N: int = 32, nx: int = 16, ny: int = 4, bend: float = 0.05) -> FsiCase:
    """Nonlinear solid (the bar test of Section 6): the bar [0,0.4] x
    [0.45,0.55] with W(F) = (gamma/(2 eta)) exp(eta (tr F^T F - 2)),
    gamma = 1.333, eta = 9.242, rho = 1, nu = 0.2, dt = 0.002, walls and
    fluid at rest.  The paper pulls the bar down by a force of unstated size
    and releases it; here the bar starts bent down (X0 = s - bend (s_x/0.4)^2
    e_y, clamped at the left wall) and relaxes, which is the released phase."""
    xy, tris = bar_mesh(nx, ny)
    X0 = xy.copy()
    X0[:, 1] -= bend * (xy[:, 0] / 0.4) ** 2
    return FsiCase(N=N, rho_f=1.0, nu=0.2, kappa=0.0, dt=0.002, lid_u=0.0, ref_xy=xy, tris=tris,
                   u0=wall_velocity(N, 0.0), X0=X0, precond=1, rtol=1e-8, steps=1, name=f"bar_N{N}",
                   extra={"solid_law": "exp", "gamma": 1.333, "eta": 9.242})


def annulus_mesh(nr: int, nt: int, r0: float = 0.3, r1: float = 0.5, quads: bool = False):
    """Structured mesh of the quarter annulus {x, y >= 0, r0 <= |x| <= r1}:
    nodes (r_i cos t_j, r_i sin t_j) on nr radial and nt angular intervals,
    node id = j (nr+1) + i.  Each (r, t) cell is one quadrilateral
    (quads=True, the Q1 solid of the paper's test) or two triangles cut by a
    diagonal; counter-clockwise either way.  The edges t = 0 and t = pi/2 lie
    exactly on y = 0 and x = 0."""
    r = np.linspace(r0, r1, nr + 1)
    t = np.linspace(0.0, 0.5 * np.pi, nt + 1)
    R, T = np.meshgrid(r, t)
    xy = np.stack([R * np.cos(T), R * np.sin(T)], -1).reshape(-1, 2)
    xy[-(nr + 1):, 0] = 0.0          # t = pi/2 on the wall x = 0
    xy[:nr + 1, 1] = 0.0             # t = 0 on the wall y = 0
    tris = []
    for j in range(nt):
        for i in range(nr):
            a = j * (nr + 1) + i
            b, c, d = a + 1, a + nr + 2, a + nr + 1
            tris += [(a, b, c, d)] if quads else [(a, b, c), (a, c, d)]
    return xy, np.array(tris, dtype=np.int32)


def annulus_case(N: int = 48, quads: bool = False) -> FsiCase:
    """The linear-solid test of Section 6 (Table 1): the quarter annulus
    0.3 <= |s| <= 0.5 in the first quadrant, kappa = 10, rho = 1, nu = 0.1,
    dt = 0.01, fluid at rest, released from the stretched state
    X(s, 0) = (s1 / 1.4, 1.4 s2).  Solid mesh refined with the fluid grid
    (about one solid interval per fluid cell).  The paper lets fluid and body
    slide along the walls x = 0 and y = 0; here every wall is no-slip.
    quads=True takes the paper's Q1 solid (one quadrilateral per (r, t)
    cell) instead of P1 triangles."""
    nr = max(2, int(np.ceil(0.2 * N)))
    nt = max(4, int(np.ceil(0.2 * np.pi * N)))
    xy, tris = annulus_mesh(nr, nt, quads=quads)
    X0 = np.stack([xy[:, 0] / 1.4, 1.4 * xy[:, 1]], 1)
    return FsiCase(N=N, rho_f=1.0, nu=0.1, kappa=10.0, dt=0.01, lid_u=0.0, ref_xy=xy, tris=tris,
                   u0=wall_velocity(N, 0.0), X0=X0, precond=1, rtol=1e-8, steps=1,
                   name=f"annulus_{'q1' if quads else 'p1'}_N{N}")


def mirrored_annulus_mesh(nr: int, nt: int, r0: float = 0.3, r1: float = 0.5, quads: bool = False):
    """The full annulus r0 <= |x| <= r1 as the quarter mesh of annulus_mesh
    and its mirror images in x = 0 and y = 0 (orientation restored in the
    mirrored quadrants; nodes on the mirror lines shared), so that the mesh is
    exactly symmetric under both reflections."""
    qxy, qtris = annulus_mesh(nr, nt, r0, r1, quads=quads)
    index: dict = {}
    xy: list = []
    tris: list = []
    for sx, sy in ((1.0, 1.0), (-1.0, 1.0), (-1.0, -1.0), (1.0, -1.0)):
        ids = []
        for p in qxy:
            key = (sx * p[0] + 0.0, sy * p[1] + 0.0)   # + 0.0: one key for -0.0 and 0.0
            if key not in index:
                index[key] = len(xy)
                xy.append(key)
            ids.append(index[key])
        for el in qtris:
            t = tuple(ids[v] for v in el)
            tris.append(t if sx * sy > 0 else (t[0],) + t[:0:-1])   # reversed after the first vertex
    return np.array(xy), np.array(tris, dtype=np.int32)


def symmetric_annulus_case(Nq: int = 24, quads: bool = False) -> FsiCase:
    """The Table 1 test (see annulus_case) with the paper's free-slip walls
    x = 0 and y = 0, obtained by symmetry: the quarter problem on [0,1]^2 with
    free slip on x = 0, y = 0 and no slip on x = 1, y = 1 is the restriction
    of the full-annulus problem on [-1,1]^2 with no slip everywhere.  That
    problem, scaled into the unit square (x' = (x + 1)/2, so u' = u/2), is
    the same dynamics with nu' = nu/4 and kappa' = kappa/4 (pressure /4),
    rho and dt unchanged.  Nq is the quarter problem's grid; this grid is
    N = 2 Nq, with the solid mesh mirrored from the quarter mesh (Q1
    quadrilaterals with quads=True, else P1 triangles)."""
    nr = max(2, int(np.ceil(0.2 * Nq)))
    nt = max(4, int(np.ceil(0.2 * np.pi * Nq)))
    xy, tris = mirrored_annulus_mesh(nr, nt, quads=quads)
    X = np.stack([xy[:, 0] / 1.4, 1.4 * xy[:, 1]], 1)
    ref = 0.5 + 0.5 * xy
    X0 = 0.5 + 0.5 * X
    N = 2 * Nq
    return FsiCase(N=N, rho_f=1.0, nu=0.1 / 4.0, kappa=10.0 / 4.0, dt=0.01, lid_u=0.0, ref_xy=ref, tris=tris,
                   u0=wall_velocity(N, 0.0), X0=X0, precond=1, rtol=1e-8, steps=1,
                   name=f"annulus_sym_{'q1' if quads else 'p1'}_Nq{Nq}")


def node_grid_shape(N: int) -> int:
    """Number of Q2 nodes per side of the N x N cell grid."""
    return 2 * N + 1


def wall_velocity(N: int, lid_u: float) -> np.ndarray:
    """Nodal Dirichlet data on the (2N+1)^2 grid, shape [(2N+1)^2, 2].

    Walls are at rest; with a lid, the nodes of the top wall strictly between
    the two corners move with (lid_u, 0); the corners stay at rest.
    """
    n1 = 2 * N + 1
    u = np.zeros((n1 * n1, 2))
    if lid_u != 0.0:
        top = (n1 - 1) * n1 + np.arange(1, n1 - 1)
        u[top, 0] = lid_u
    return u


def initial_velocity(N: int, seed: int, lid_u: float = 0.0, amplitude: float = 1.0) -> np.ndarray:
    """u_0 on the (2N+1)^2 node grid, shape [(2N+1)^2, 2], node id = iy*(2N+1)+ix.

    Interior dofs are ``amplitude * (2U - 1)`` with U = uniform01(seed, dof id)
    and dof id = 2 * node id + component; boundary nodes take the wall values.
    """
    n1 = 2 * N + 1
    u = wall_velocity(N, lid_u)
    if amplitude != 0.0:
        ix, iy = np.meshgrid(np.arange(n1), np.arange(n1))
        ix = ix.ravel()
        iy = iy.ravel()
        interior = (ix > 0) & (ix < n1 - 1) & (iy > 0) & (iy < n1 - 1)
        nodes = np.nonzero(interior)[0]
        for c in range(2):
            dof = 2 * nodes.astype(np.uint64) + np.uint64(c)
            u[nodes, c] = amplitude * (2.0 * uniform01(seed, dof) - 1.0)
    return u


@dataclass
class FsiCase:
    """One FSI instance: parameters, solid mesh and initial state."""
    N: int
    rho_f: float
    nu: float
    kappa: float
    dt: float
    lid_u: float
    ref_xy: np.ndarray          # [n_s, 2] reference (= initial) solid node positions
    tris: np.ndarray            # [n_el, 3] P1 triangles or [n_el, 4] Q1 quadrilaterals, int32, counter-clockwise
    u0: np.ndarray              # [(2N+1)^2, 2] nodal velocity
    X0: np.ndarray              # [n_s, 2] initial solid node positions
    precond: int = 0            # 0 block-diagonal, 1 block-triangular
    rtol: float = 1e-8
    steps: int = 1
    name: str = ""
    extra: dict = field(default_factory=dict)


BASE_SEED = 2301


def disk16_case(seed: int = BASE_SEED + 0) -> FsiCase:
    """Plain FP64 single step: N=16, nu=1, rho=1, kappa=10, dt=0.01, disk
    R=0.2 at (0.5, 0.5) with m=6 (216 triangles), u_0 uniform[-1,1]."""
    N = 16
    xy, tris = ring_disk_mesh(6, 0.2, (0.5, 0.5))
    return FsiCase(N=N, rho_f=1.0, nu=1.0, kappa=10.0, dt=0.01, lid_u=0.0,
                   ref_xy=xy, tris=tris, u0=initial_velocity(N, seed), X0=xy.copy(),
                   precond=0, rtol=1e-10, steps=1, name="cavity16_disk216_fp64")


def cavity128_case(seed: int = BASE_SEED + 1, N: int = 128, m: int = 36) -> FsiCase:
    """Plain vs mixed precision: N=128, nu=0.01, kappa=1e3, dt=1e-3, lid 1,
    disk R=0.2 with m=36 (7776 triangles), body at rest, fluid at rest."""
    xy, tris = ring_disk_mesh(m, 0.2, (0.5, 0.5))
    return FsiCase(N=N, rho_f=1.0, nu=0.01, kappa=1e3, dt=1e-3, lid_u=1.0,
                   ref_xy=xy, tris=tris, u0=wall_velocity(N, 1.0), X0=xy.copy(),
                   precond=1, rtol=1e-8, steps=100,
                   name=f"cavity{N}_lid_disk{len(tris)}")


def lid_body_case(N: int = 16, m: int = 5, seed: int = BASE_SEED + 5) -> FsiCase:
    """A disk (R = 0.07 at (0.43, 0.925), m rings) whose rule points fall in
    the top row of cells, under a lid moving with velocity 1: the coupling
    rows see the lid's nodal values.  nu = 0.1, kappa = 30, dt = 0.01,
    u_0 = half-amplitude seeded field with the wall data."""
    xy, tris = ring_disk_mesh(m, 0.07, (0.43, 0.925))
    return FsiCase(N=N, rho_f=1.0, nu=0.1, kappa=30.0, dt=0.01, lid_u=1.0,
                   ref_xy=xy, tris=tris, u0=initial_velocity(N, seed, lid_u=1.0, amplitude=0.5), X0=xy.copy(),
                   precond=1, rtol=1e-12, steps=1, name=f"lid_body{N}")


def ellipse_case(N: int, seed: int = BASE_SEED + 2) -> FsiCase:
    """Size sweep member: ellipse 0.2/0.1 rotated 30 degrees, m = ceil(0.4 N),
    kappa=1e2, nu=1, rho=1, dt=0.01, walls at rest, fluid at rest."""
    m = int(math.ceil(0.4 * N))
    xy, tris = ellipse_mesh(m, 0.2, 0.1, 30.0)
    return FsiCase(N=N, rho_f=1.0, nu=1.0, kappa=1e2, dt=0.01, lid_u=0.0,
                   ref_xy=xy, tris=tris, u0=wall_velocity(N, 0.0), X0=xy.copy(),
                   precond=1, rtol=1e-8, steps=20, name=f"ellipse_N{N}")


def batch_instance(i: int, seed: int = BASE_SEED + 3) -> FsiCase:
    """Instance i of the batch of uneven problems: N ~ U{16,32,48,64,96},
    R ~ U[0.1,0.3], centre ~ U[0.35,0.65]^2, kappa log-uniform [1,1e4],
    nu log-uniform [1e-3,1], m = ceil(2 R N), walls at rest, u_0 seeded;
    dt = 1e-3 as in the 128x128 workload (the batch definition leaves it open)."""
    r = uniform01(seed, np.arange(8 * i, 8 * i + 8, dtype=np.uint64))
    N = (16, 32, 48, 64, 96)[min(int(r[0] * 5), 4)]
    R = 0.1 + 0.2 * r[1]
    cx, cy = 0.35 + 0.3 * r[2], 0.35 + 0.3 * r[3]
    kappa = 10.0 ** (4.0 * r[4])
    nu = 10.0 ** (-3.0 + 3.0 * r[5])
    m = int(math.ceil(2.0 * R * N))
    xy, tris = ring_disk_mesh(m, R, (cx, cy))
    return FsiCase(N=N, rho_f=1.0, nu=nu, kappa=kappa, dt=1e-3, lid_u=0.0,
                   ref_xy=xy, tris=tris, u0=initial_velocity(N, seed * 1000003 + i),
                   X0=xy.copy(), precond=1, rtol=1e-8, steps=50, name=f"batch{i}_N{N}")


def serve_trace(n_requests: int = 2000, rate: float = 200.0, seed: int = BASE_SEED + 4):
    """Served stream: Poisson arrivals (exponential gaps at ``rate``/s); each
    request is 50 steps of a cavity problem with N in {32,64,128,256}
    (p = .4/.3/.2/.1), disk or ellipse (p = 1/2), R ~ U[0.1,0.3],
    kappa log-uniform [1,1e4].  Returns a list of (arrival_s, FsiCase-args)."""
    out = []
    t = 0.0
    for i in range(n_requests):
        r = uniform01(seed, np.arange(8 * i, 8 * i + 8, dtype=np.uint64))
        t += -math.log(1.0 - r[0]) / rate
        u = r[1]
        N = 32 if u < 0.4 else 64 if u < 0.7 else 128 if u < 0.9 else 256
        R = 0.1 + 0.2 * r[3]
        kappa = 10.0 ** (4.0 * r[4])
        out.append((t, dict(N=N, ellipse=bool(r[2] < 0.5), R=R, kappa=kappa, index=i)))
    return out


def serve_case(spec: dict, seed: int = BASE_SEED + 4) -> FsiCase:
    N = spec["N"]
    R = spec["R"]
    m = int(math.ceil(2.0 * R * N))
    if spec["ellipse"]:
        xy, tris = ellipse_mesh(m, R, 0.5 * R, 30.0)
    else:
        xy, tris = ring_disk_mesh(m, R, (0.5, 0.5))
    return FsiCase(N=N, rho_f=1.0, nu=0.1, kappa=spec["kappa"], dt=1e-3, lid_u=1.0,
                   ref_xy=xy, tris=tris, u0=wall_velocity(N, 1.0), X0=xy.copy(),
                   precond=1, rtol=1e-8, steps=50, name=f"req{spec['index']}_N{N}")
