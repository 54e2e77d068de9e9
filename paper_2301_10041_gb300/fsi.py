"""ctypes binding of the C ABI in ``include/fsi.h`` (argument marshalling only).

Every function here forwards to the CUDA library ``_lib/libfsi_gb300.so``;
no step of the FSI solve runs in Python.  Importing this module does not
load the library; the first call does, and raises if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libfsi_gb300.so")

FSI_OK = 0
FSI_ERR_INVALID = -1
FSI_ERR_OOM = -2
FSI_ERR_BUDGET = -3
FSI_ERR_OUT_OF_DOMAIN = -4
FSI_ERR_NOT_CONVERGED = -5
FSI_ERR_BREAKDOWN = -6
FSI_ERR_NAN = -7
FSI_ERR_TIMEOUT = -8
FSI_ERR_CAPACITY = -9
FSI_ERR_CUDA = -10


class fsi_params(C.Structure):
    _fields_ = [("N", C.c_int), ("rho_f", C.c_double), ("nu", C.c_double), ("kappa", C.c_double),
                ("dt", C.c_double), ("lid_u", C.c_double), ("precond", C.c_int), ("precision", C.c_int),
                ("restart", C.c_int), ("rtol", C.c_double), ("max_it", C.c_int), ("mg_degree", C.c_int),
                ("cs_degree", C.c_int), ("inner_rtol", C.c_double), ("max_refine", C.c_int),
                ("stokes_its", C.c_int), ("stokes_omega", C.c_double), ("mg_cluster", C.c_int),
                ("coupling", C.c_int), ("solid_law", C.c_int), ("gamma", C.c_double), ("eta", C.c_double),
                ("newton_tol", C.c_double), ("newton_max", C.c_int), ("autotune", C.c_int),
                ("solid_elem", C.c_int), ("mg_fused", C.c_int),
                ("mg_coarse", C.c_int), ("mg_coarse_p", C.c_int)]


class fsi_solid_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_tris", C.c_int), ("ref_xy", C.POINTER(C.c_double)),
                ("tris", C.POINTER(C.c_int))]


class fsi_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("rel_residual", C.c_double), ("rel_residual_est", C.c_double), ("newton_iterations", C.c_int)]


EXPORTS = {
    "fsi_create_problem": (C.c_int, [C.POINTER(fsi_params), C.POINTER(fsi_solid_mesh), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.POINTER(C.c_void_p)]),
    "fsi_create_problem_budget": (C.c_int, [C.POINTER(fsi_params), C.POINTER(fsi_solid_mesh), C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
    "fsi_footprint_bytes": (C.c_size_t, [C.POINTER(fsi_params), C.c_int, C.c_int]),
    "fsi_assemble_step": (C.c_int, [C.c_void_p]),
    "fsi_solve_step": (C.c_int, [C.c_void_p, C.POINTER(fsi_solve_info)]),
    "fsi_advance": (C.c_int, [C.c_void_p]),
    "fsi_step": (C.c_int, [C.c_void_p, C.POINTER(fsi_solve_info)]),
    "fsi_step_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(fsi_solve_info)]),
    "fsi_step_async": (C.c_int, [C.c_void_p]),
    "fsi_step_poll": (C.c_int, [C.c_void_p, C.POINTER(fsi_solve_info)]),
    "fsi_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fsi_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "fsi_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                            C.POINTER(C.c_int)]),
    "fsi_get_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fsi_get_coupling": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p]),
    "fsi_apply_operator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "fsi_apply_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "fsi_interior_nodes": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fsi_get_rhs": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fsi_graph_kernel_counts": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fsi_time_kernel": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "fsi_kernel_flops": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "fsi_locate_bin_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fsi_destroy": (None, [C.c_void_p]),
    "fsi_status_str": (C.c_char_p, [C.c_int]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises OSError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"{path} is missing: run paper_2301_10041_gb300.build.build() first")
        lib = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class FsiError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load_library().fsi_status_str(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(N, rho_f, nu, kappa, dt, lid_u=0.0, precond=1, precision=0, restart=0, rtol=0.0, max_it=0,
                mg_degree=0, cs_degree=0, inner_rtol=0.0, max_refine=0, stokes_its=0,
                stokes_omega=0.0, mg_cluster=0, coupling=0, solid_law=0, gamma=0.0, eta=0.0, newton_tol=0.0,
                newton_max=0, autotune=0, solid_elem=0, mg_fused=0, mg_coarse=0, mg_coarse_p=0) -> fsi_params:
    return fsi_params(int(N), float(rho_f), float(nu), float(kappa), float(dt), float(lid_u), int(precond),
                      int(precision), int(restart), float(rtol), int(max_it), int(mg_degree), int(cs_degree),
                      float(inner_rtol), int(max_refine), int(stokes_its), float(stokes_omega), int(mg_cluster),
                      int(coupling), int(solid_law), float(gamma), float(eta), float(newton_tol), int(newton_max),
                      int(autotune), int(solid_elem), int(mg_fused), int(mg_coarse), int(mg_coarse_p))


def footprint_bytes(params: fsi_params, n_nodes: int, n_tris: int) -> int:
    return int(load_library().fsi_footprint_bytes(C.byref(params), int(n_nodes), int(n_tris)))


@dataclass
class SolveInfo:
    iterations: int
    refinements: int
    restarts: int
    status: int
    rel_residual: float
    rel_residual_est: float
    newton_iterations: int = 0


class Problem:
    """One FSI instance owned by the CUDA library (fsi_problem*)."""

    def __init__(self, params: fsi_params, ref_xy, tris, u0=None, X0=None, stream=None, budget_bytes: int = 0):
        lib = load_library()
        self.params = params
        self.ref_xy = _f64(ref_xy).reshape(-1, 2)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 4 if params.solid_elem == 1 else 3)
        mesh = fsi_solid_mesh(self.ref_xy.shape[0], self.tris.shape[0],
                              self.ref_xy.ctypes.data_as(C.POINTER(C.c_double)),
                              self.tris.ctypes.data_as(C.POINTER(C.c_int)))
        u0a = None if u0 is None else _f64(u0)
        X0a = None if X0 is None else _f64(X0)
        h = C.c_void_p()
        st = lib.fsi_create_problem_budget(C.byref(params), C.byref(mesh), _ptr(u0a), _ptr(X0a),
                                           C.c_void_p(stream) if stream else None, C.c_size_t(budget_bytes),
                                           C.byref(h))
        if st != FSI_OK:
            raise FsiError(st, "fsi_create_problem")
        self._h = h
        nu_, np_, nx_, nt_ = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        lib.fsi_sizes(h, C.byref(nu_), C.byref(np_), C.byref(nx_), C.byref(nt_))
        self.n_u, self.n_p, self.n_x, self.n = nu_.value, np_.value, nx_.value, nt_.value
        self.N = params.N
        self.n_nodes = self.ref_xy.shape[0]

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            load_library().fsi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where):
        if st != FSI_OK:
            raise FsiError(st, where)

    # -- the time step
    def assemble_step(self):
        self._check(load_library().fsi_assemble_step(self._h), "fsi_assemble_step")

    def solve_step(self, check: bool = True) -> SolveInfo:
        info = fsi_solve_info()
        st = load_library().fsi_solve_step(self._h, C.byref(info))
        if check:
            self._check(st, "fsi_solve_step")
        return SolveInfo(info.iterations, info.refinements, info.restarts, info.status, info.rel_residual,
                         info.rel_residual_est, info.newton_iterations)

    def advance(self):
        self._check(load_library().fsi_advance(self._h), "fsi_advance")

    def step(self) -> SolveInfo:
        self.assemble_step()
        info = self.solve_step()
        self.advance()
        return info

    def step_async(self):
        self._check(load_library().fsi_step_async(self._h), "fsi_step_async")

    def step_poll(self):
        """None while the queued step runs, else its SolveInfo."""
        info = fsi_solve_info()
        st = load_library().fsi_step_poll(self._h, C.byref(info))
        if st == 1:
            return None
        if st < 0:
            raise FsiError(st, "fsi_step_poll")
        return SolveInfo(info.iterations, info.refinements, info.restarts, info.status, info.rel_residual,
                         info.rel_residual_est, info.newton_iterations)

    # -- state
    def get_state(self):
        n1 = 2 * self.N + 1
        u = np.empty((n1 * n1, 2))
        p = np.empty((self.N * self.N, 3))
        X = np.empty((self.n_nodes, 2))
        lam = np.empty((self.n_nodes, 2))
        self._check(load_library().fsi_get_state(self._h, _ptr(u), _ptr(p), _ptr(X), _ptr(lam)), "fsi_get_state")
        return u, p, X, lam

    def set_state(self, u=None, X=None):
        ua = None if u is None else _f64(u)
        Xa = None if X is None else _f64(X)
        self._check(load_library().fsi_set_state(self._h, _ptr(ua), _ptr(Xa)), "fsi_set_state")

    # -- test hooks
    def get_points(self):
        npts = (9 if self.params.solid_elem == 1 else 6) * self.tris.shape[0]
        cell = np.empty(npts, dtype=np.int32)
        xi = np.empty(npts)
        eta = np.empty(npts)
        self._check(load_library().fsi_get_points(self._h, _ptr(cell), _ptr(xi), _ptr(eta)), "fsi_get_points")
        return cell, xi, eta

    def get_coupling(self):
        lib = load_library()
        nnz = C.c_int(0)
        self._check(lib.fsi_get_coupling(self._h, C.byref(nnz), None, None, None), "fsi_get_coupling")
        rows = np.empty(nnz.value, dtype=np.int32)
        cols = np.empty(nnz.value, dtype=np.int32)
        vals = np.empty(nnz.value)
        self._check(lib.fsi_get_coupling(self._h, C.byref(nnz), _ptr(rows), _ptr(cols), _ptr(vals)),
                    "fsi_get_coupling")
        return rows, cols, vals

    def apply_operator(self, x, precision: int = 0):
        x = _f64(x)
        y = np.empty(self.n)
        self._check(load_library().fsi_apply_operator(self._h, _ptr(x), _ptr(y), int(precision)),
                    "fsi_apply_operator")
        return y

    def apply_preconditioner(self, v, precision: int = 0):
        v = _f64(v)
        z = np.empty(self.n)
        self._check(load_library().fsi_apply_preconditioner(self._h, _ptr(v), _ptr(z), int(precision)),
                    "fsi_apply_preconditioner")
        return z

    def interior_nodes(self):
        ids = np.empty(self.n_u // 2, dtype=np.int32)
        self._check(load_library().fsi_interior_nodes(self._h, _ptr(ids)), "fsi_interior_nodes")
        return ids

    def graph_kernel_counts(self):
        c = np.zeros(5, dtype=np.int32)
        self._check(load_library().fsi_graph_kernel_counts(self._h, _ptr(c)), "fsi_graph_kernel_counts")
        return c

    def time_kernel(self, which: int, reps: int = 20):
        """(mean launch ms, algorithmic bytes per launch) of one kernel."""
        ms = C.c_double()
        by = C.c_double()
        self._check(load_library().fsi_time_kernel(self._h, int(which), int(reps), C.byref(ms), C.byref(by)),
                    "fsi_time_kernel")
        return ms.value, by.value

    def kernel_flops(self, which: int) -> float:
        """Algorithmic floating-point operations of one launch of kernel `which`."""
        f = C.c_double()
        self._check(load_library().fsi_kernel_flops(self._h, int(which), C.byref(f)), "fsi_kernel_flops")
        return f.value

    def get_rhs(self):
        b = np.empty(self.n)
        self._check(load_library().fsi_get_rhs(self._h, _ptr(b)), "fsi_get_rhs")
        return b


FSI_NOALLOC_MAX_CELLS = 262144


def locate_bin_noalloc(N: int, n_tris: int, tris_ptr: int, X_ptr: int, cell_ptr: int, xi_ptr: int, eta_ptr: int,
                       cell_start_ptr: int, cell_points_ptr: int, n_outside_ptr: int, stream: int = 0) -> int:
    """Allocation-free point location and binning (device pointers in and out;
    see fsi_locate_bin_noalloc in include/fsi.h).  Returns the status code."""
    return int(load_library().fsi_locate_bin_noalloc(
        int(N), int(n_tris), C.c_void_p(tris_ptr), C.c_void_p(X_ptr), C.c_void_p(cell_ptr), C.c_void_p(xi_ptr),
        C.c_void_p(eta_ptr), C.c_void_p(cell_start_ptr), C.c_void_p(cell_points_ptr), C.c_void_p(n_outside_ptr),
        C.c_void_p(stream) if stream else None))


def step_batch(problems) -> list:
    """One time step of every problem, all queued before any is waited for."""
    n = len(problems)
    handles = (C.c_void_p * n)(*[p._h for p in problems])
    infos = (fsi_solve_info * n)()
    st = load_library().fsi_step_batch(handles, n, infos)
    out = [SolveInfo(i.iterations, i.refinements, i.restarts, i.status, i.rel_residual, i.rel_residual_est)
           for i in infos]
    return st, out


def problem_from_case(case, precision: int = 0, precond=None, rtol=None, stream=None, **kw) -> Problem:
    """Build a Problem from an ``fsi_inputs.FsiCase`` (its ``extra`` may name
    the exponential solid law with gamma and eta; a mesh of quadrilaterals
    takes the Q1 solid)."""
    extra = getattr(case, "extra", None) or {}
    if np.asarray(case.tris).shape[1] == 4:
        kw.setdefault("solid_elem", 1)
    if extra.get("solid_law") == "exp":
        kw.setdefault("solid_law", 1)
        kw.setdefault("gamma", extra["gamma"])
        kw.setdefault("eta", extra["eta"])
    prm = make_params(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u,
                      precond=case.precond if precond is None else precond, precision=precision,
                      rtol=case.rtol if rtol is None else rtol, **kw)
    return Problem(prm, case.ref_xy, case.tris, u0=case.u0, X0=case.X0, stream=stream)
