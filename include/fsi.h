/*
 * fsi.h — C ABI of the GB300 (sm_103a) library for one time step of the
 * distributed-Lagrange-multiplier fictitious-domain FSI method of
 * Boffi, Credali, Gastaldi and Scacchi, "A parallel solver for FSI problems
 * with fictitious domain approach" (arXiv:2301.10041).
 *
 * Problem solved per step (Section 4, Problem 3 and Eq. (matrix)): for the
 * fluid velocity u (Q2, interior nodes of a uniform N x N grid of the unit
 * square), pressure p (P1 discontinuous, 3 coefficients per cell),
 * solid position X and multiplier lambda (both P1 on the solid mesh):
 *
 *     [ A_f      -B^T   0           C_f(X^n)^T ] [u^{n+1}]   [g1]
 *     [ -B        0     0           0          ] [p^{n+1}] = [g_p]
 *     [ 0         0     A_s         -C_s       ] [X^{n+1}]   [0 ]
 *     [ C_f(X^n)  0     -C_s/dt     0          ] [l^{n+1}]   [g2]
 *
 * with A_f = (rho_f/dt) M_f + K_f, K_f from nu (eps(u), eps(v)),
 * A_s = kappa (grad chi_j, grad chi_i)_B (P(F) = kappa F), C_s the P1 mass
 * matrix, g1 = (rho_f/dt) M_f u^n, g2 = -(1/dt) C_s X^n, Dirichlet wall data
 * moved to the right-hand side.  C_f(X^n) is re-assembled every step by
 * locating the 6 points of a degree-4 triangle rule of every solid triangle
 * in the fluid grid (Section 4 assembles it by exact intersection instead).
 * The system is solved by right-preconditioned flexible GMRES with the
 * paper's block-diagonal or block-triangular preconditioner (Section 5).
 *
 * Conventions for every entry point:
 *  - All arrays passed in are HOST arrays owned by the caller; they are
 *    copied and may be freed after the call returns.
 *  - The library owns every device buffer it allocates (cudaMalloc); one
 *    problem lives on the device that was current at fsi_create_problem.
 *  - Work is queued on the CUDA stream given at creation (NULL: the library
 *    creates and owns a non-blocking stream; the legacy default stream cannot
 *    be used because the step is captured in CUDA graphs).
 *    fsi_assemble_step and fsi_advance are asynchronous;
 *    fsi_solve_step, fsi_get_* and fsi_set_state synchronise the stream.
 *  - Every call returns an int status: FSI_OK (0) or a negative FSI_ERR_*
 *    code; no C++ exception crosses the boundary.  Errors found on the
 *    device during fsi_assemble_step (a point outside the domain, a row over
 *    capacity) are reported by the next synchronising call.
 *  - Node layouts: the fluid node lattice has (2N+1)^2 nodes, node id =
 *    iy*(2N+1) + ix at (ix/(2N), iy/(2N)); nodal velocity arrays are
 *    interleaved [u_x, u_y] per node.  Pressure arrays hold 3 doubles per
 *    cell (cell id = cy*N + cx) in the basis {1, (x-xc)/h, (y-yc)/h}, with
 *    zero mean over the domain.  Solid arrays are interleaved [x, y] per node.
 */
#ifndef FSI_GB300_H
#define FSI_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FSI_OK                  0
#define FSI_ERR_INVALID        -1  /* bad argument or parameter */
#define FSI_ERR_OOM            -2  /* cudaMalloc failed */
#define FSI_ERR_BUDGET         -3  /* footprint above the caller's byte budget */
#define FSI_ERR_OUT_OF_DOMAIN  -4  /* a solid quadrature point left [0,1]^2 */
#define FSI_ERR_NOT_CONVERGED  -5  /* max_it reached above rtol */
#define FSI_ERR_BREAKDOWN      -6  /* Krylov breakdown (zero new direction) */
#define FSI_ERR_NAN            -7  /* NaN/Inf in the residual */
#define FSI_ERR_TIMEOUT        -8  /* reserved: no call of this version returns it (no
                                      kernel of the library waits on a flag) */
#define FSI_ERR_CAPACITY       -9  /* a coupling row exceeded its storage */
#define FSI_ERR_CUDA          -10  /* a CUDA runtime call failed */

/* Parameters of one instance (Section 4 and Section 6 of the paper). */
typedef struct fsi_params {
    int    N;          /* fluid cells per side: even, N = c * 2^k with c <= 8 */
    double rho_f;      /* fluid (= solid) density, Problem 2: rho_s = rho_f */
    double nu;         /* viscosity, nu_f = nu_s (Section 3) */
    double kappa;      /* P(F) = kappa F (Section 4, before Eq. (matrix)) */
    double dt;         /* backward-Euler time step (Section 4) */
    double lid_u;      /* tangential velocity of the top wall, 0 = all walls at rest */
    int    precond;    /* 0 block-diagonal, 1 block lower-triangular (the two
                          preconditioners of Section 5), 2 block upper-triangular
                          [[A11, A12], [0, A22]] (solid block first), 3 as 2 with
                          the velocity and pressure parts of A11^-1 applied
                          side by side (block-diagonal Stokes approximation) */
    int    precision;  /* 0 FP64 everywhere; 1 FP32 operators and preconditioner
                          inside FGMRES, FP64 Gram-Schmidt, least squares and
                          iterative refinement */
    int    restart;    /* GMRES restart length, paper: 200 (Section 6); 0 = 200;
                          at most 250 (FSI_ERR_INVALID above) */
    double rtol;       /* relative residual target, paper: 1e-8 (Section 6); 0 = 1e-8 */
    int    max_it;     /* total Krylov iteration cap per step; 0 = 1000 */
    int    mg_degree;  /* Chebyshev degree of each multigrid smoothing; 0 = 2 */
    int    cs_degree;  /* Chebyshev iterations per solid mass solve; 0 = 16 */
    double inner_rtol; /* precision 1: inner FGMRES tolerance; 0 = 1e-5 */
    int    max_refine; /* precision 1: refinement steps cap; 0 = 30 */
    int    stokes_its; /* Richardson steps on the fluid (Stokes) block inside one
                          preconditioner application, each one V-cycle pair;
                          0 = 1 (the one-shot approximation); at most 16
                          (FSI_ERR_INVALID above) */
    double stokes_omega; /* damping of the Richardson corrections after the first; 0 = 1 */
    int    mg_cluster; /* 0: automatic -- the coarse multigrid levels whose operators
                          fit in the shared memory of one thread-block cluster
                          run as one cluster launch per V-cycle (same
                          arithmetic), except that an FP32 hierarchy with the
                          fused matrix-free levels (mg_fused = 0) keeps only
                          levels of at most 8 cells there; -1: no cluster; n > 0:
                          levels of at most n cells a side in the cluster */
    int    coupling;   /* C_f(X^n) quadrature: 0 = the degree-4 6-point rule at
                          points located in the fluid grid; 1 = exact, by
                          intersecting each mapped solid triangle with the
                          fluid cells (Sutherland-Hodgman) and integrating the
                          pieces with a degree-5 rule (Section 4) */
    int    solid_law;  /* 0: P(F) = kappa F (the linear law of Eq. (matrix));
                          1: the exponential strain energy of the bar test
                          (Section 6), W(F) = (gamma/(2 eta)) exp(eta (tr F^T F
                          - 2)), each time step solved by Newton's method */
    double gamma;      /* solid_law 1: gamma of W (the paper's test: 1.333) */
    double eta;        /* solid_law 1: eta of W (the paper's test: 9.242) */
    double newton_tol; /* solid_law 1: stop when max |X_{k+1} - X_k| <=
                          newton_tol * max |X_{k+1} - X^n| (floor 1e-13);
                          0 = 1e-6 */
    int    newton_max; /* solid_law 1: Newton iteration cap; 0 = 20 */
    int    autotune;   /* 0: one fixed tile shape (4 threads per block row) for
                          every multigrid level's SpMV; 1: the shape of each
                          level (4 or 8 threads per block row) is chosen at
                          creation by timing its Chebyshev smoothing step alone
                          on the device (cached per matrix shape and size for
                          the process) */
    int    solid_elem; /* solid (and multiplier) element: 0 = P1 triangles, 3
                          node ids per element; 1 = Q1 quadrilaterals (the
                          annulus test of Section 6), 4 node ids per element,
                          with A_s, C_s and the C_f point rule by the 3 x 3
                          Gauss rule on each element.  Q1 takes coupling 0 and
                          solid_law 0 only */
    int    mg_fused;   /* 0: the finest multigrid levels of the FP32 hierarchy
                          (down to the cluster-resident ones, at least 16 cells a
                          side) run matrix-free, each V-cycle level as two fused
                          launches (pre-smoothing + residual + restriction;
                          prolongation + post-smoothing); -1: the per-level
                          sparse kernels on every level */
    int    mg_coarse;  /* the coarsening stops at the first grid of at most
                          mg_coarse cells a side, whose operators are inverted
                          densely on the device when the problem is created
                          (Gauss-Jordan in FP64, one launch per unknown);
                          0 or less = 16 (a 16-cell grid: 1922 velocity unknowns, a
                          15 MB FP32 or 30 MB FP64 inverse, held in L2); at
                          most 32 (FSI_ERR_INVALID above) */
    int    mg_coarse_p; /* the same for the pressure-Laplacian hierarchy alone;
                          0 or less = mg_coarse; at most 32 (FSI_ERR_INVALID
                          above; a 32-cell grid has 3072 pressure unknowns,
                          a 38 MB FP32 inverse) */
} fsi_params;

/* Solid reference mesh (the body at t = 0): P1 triangles, or Q1
 * quadrilaterals with fsi_params.solid_elem = 1; vertices counter-clockwise. */
typedef struct fsi_solid_mesh {
    int           n_nodes;
    int           n_tris;  /* elements (triangles or quadrilaterals) */
    const double* ref_xy;  /* host, 2*n_nodes, interleaved (x, y) */
    const int*    tris;    /* host, 3*n_tris (triangles) or 4*n_tris
                              (quadrilaterals) node ids */
} fsi_solid_mesh;

/* Per-step report (the paper's its / T_coup / T_sol, Tables 1-4). */
typedef struct fsi_solve_info {
    int    iterations;       /* Krylov iterations (all refinements) */
    int    refinements;      /* outer refinement steps (precision 1), else 0 */
    int    restarts;         /* FGMRES restarts */
    int    status;           /* same as the return value */
    double rel_residual;     /* true ||b - A x|| / ||b|| in FP64 at exit */
    double rel_residual_est; /* last Krylov estimate */
    int    newton_iterations; /* solid_law 1: Newton iterations of the step (each
                                 one linear solve; iterations above sum over
                                 them); 0 for the linear law */
} fsi_solve_info;

typedef struct fsi_problem fsi_problem;  /* opaque; owns all device memory */

/* Build constant matrices (M_f, K_f, B, A_s, C_s, multigrid hierarchy) and
 * device state.  u0: host, 2*(2N+1)^2 nodal velocity (boundary entries are
 * replaced by the wall data); X0: host, 2*n_nodes initial solid positions.
 * cuda_stream: a cudaStream_t or NULL.  On success *out owns the problem. */
int fsi_create_problem(const fsi_params* params, const fsi_solid_mesh* mesh,
                       const double* u0, const double* X0, void* cuda_stream,
                       fsi_problem** out);

/* Bytes of device memory fsi_create_problem would allocate for these sizes
 * (n_tris: solid elements of the kind params->solid_elem names); 0 when the
 * parameters are invalid. */
size_t fsi_footprint_bytes(const fsi_params* params, int n_solid_nodes, int n_tris);

/* Same as fsi_create_problem, but fails with FSI_ERR_BUDGET (allocating
 * nothing) when fsi_footprint_bytes exceeds budget_bytes. */
int fsi_create_problem_budget(const fsi_params* params, const fsi_solid_mesh* mesh,
                              const double* u0, const double* X0, void* cuda_stream,
                              size_t budget_bytes, fsi_problem** out);

/* Steps S1-S4 on the device, asynchronous: locate the solid quadrature
 * points in the fluid grid, assemble C_f(X^n) and its transpose, build the
 * right-hand side (g1, g_p, 0, g2). */
int fsi_assemble_step(fsi_problem* p);

/* Steps S5-S8: FGMRES (precision 0) or FP64 iterative refinement around an
 * FP32-operator FGMRES (precision 1) until ||b - A x|| / ||b|| <= rtol,
 * warm-started from the current state.  Synchronises.  info may be NULL. */
int fsi_solve_step(fsi_problem* p, fsi_solve_info* info);

/* Step S9, asynchronous: (u^n, X^n) <- (u^{n+1}, X^{n+1}). */
int fsi_advance(fsi_problem* p);

/* assemble + solve + advance. */
int fsi_step(fsi_problem* p, fsi_solve_info* info);

/* Batched step of several instances: queues assemble + solve + advance of
 * every problem on its own stream (the library-owned streams of problems
 * created with NULL run concurrently on the device), then waits for all of
 * them.  infos (may be NULL) receives one report per problem.  Returns FSI_OK
 * or the first failing status.  Problems built with FSI_HOST_LOOP=1 are
 * rejected (FSI_ERR_INVALID). */
int fsi_step_batch(fsi_problem* const* problems, int count, fsi_solve_info* infos);

/* Asynchronous step for continuous batching: fsi_step_async queues
 * assemble + solve + advance on the problem's stream and returns at once;
 * fsi_step_poll returns 1 while that step is still running and 0 once it has
 * finished (filling info; info->status is the step's status), or a negative
 * FSI_ERR_* if the stream failed.  Poll before touching the problem again. */
int fsi_step_async(fsi_problem* p);
int fsi_step_poll(fsi_problem* p, fsi_solve_info* info);

/* Host copies of the current solution; any pointer may be NULL.
 * u: 2*(2N+1)^2 (wall values included), pr: 3*N^2, X and lam: 2*n_nodes. */
int fsi_get_state(fsi_problem* p, double* u, double* pr, double* X, double* lam);

/* Replace (u^n, X^n) and the warm start of u and X; u: 2*(2N+1)^2 nodal,
 * X: 2*n_nodes.  Either may be NULL (kept). */
int fsi_set_state(fsi_problem* p, const double* u, const double* X);

/* Sizes: n_u (interior velocity dofs), n_p, n_x (= 2*n_nodes), total n. */
int fsi_sizes(const fsi_problem* p, int* n_u, int* n_p, int* n_x, int* n_total);

/* Test hooks.  Point location of the last fsi_assemble_step: for point
 * id = 6*triangle + q (P1; 9*quadrilateral + q with a Q1 solid, q = 3 j + i
 * at Gauss nodes (s_i, t_j)), the fluid cell id (cy*N + cx, or -1 outside)
 * and the local coordinates (xi, eta) in [0,1]^2.  Arrays of 6*n_tris
 * (9*n_tris for Q1); may be NULL.
 * FSI_ERR_INVALID with coupling = 1 (the exact rule locates no points). */
int fsi_get_points(fsi_problem* p, int* cell, double* xi, double* eta);

/* Test hook: the scalar coupling matrix C of the last fsi_assemble_step in
 * coordinate form (C_f = C on each velocity component), interior fluid node
 * columns only (wall columns enter the right-hand side g2, see
 * fsi_get_rhs).  Call with rows == NULL to get the count
 * in *nnz; then with arrays of that size: solid node, lattice node id, value. */
int fsi_get_coupling(fsi_problem* p, int* nnz, int* rows, int* lattice_cols, double* vals);

/* Test hook: y = A x for the full block operator in the library's block
 * order [u_interior | p | X | lambda] on host arrays of length n_total;
 * precision 0 = FP64 operator, 1 = FP32 operator.  Node order of u follows
 * fsi_interior_nodes. */
int fsi_apply_operator(fsi_problem* p, const double* x, double* y, int precision);

/* Test hook: z = P^{-1} v, one application of the preconditioner. */
int fsi_apply_preconditioner(fsi_problem* p, const double* v, double* z, int precision);

/* Lattice node id of every interior velocity node, in the library's order
 * (n_u/2 entries). */
int fsi_interior_nodes(const fsi_problem* p, int* lattice_ids);

/* Kernel nodes in the captured graphs: counts[0] assembly (S1-S4),
 * counts[1] solve set-up, counts[2] one refinement/restart cycle outside
 * the Arnoldi loop, counts[3] one Arnoldi iteration (S5-S7), counts[4]
 * pressure normalisation.  Kernels per step = c0 + c1 + cycles*c2 +
 * iterations*c3 + c4 (cycles = refinements + 1). */
int fsi_graph_kernel_counts(const fsi_problem* p, int* counts);

/* Measurement hook: time `reps` launches of one kernel on the problem's
 * stream with CUDA events, each launch after a 256 MiB write that evicts
 * L2, on the current data of the problem.  which: 0 full operator in FP32
 * (precision 1 only), 1 full operator in FP64 (residual form), 2 finest
 * velocity Chebyshev smoothing step in FP32 (precision 1 only), 3 the same in
 * FP64; 4 and 5 (precision 1 only): one whole V-cycle on the velocity /
 * pressure-Laplacian hierarchy in FP32, with L2 left warm as inside a solve
 * (bytes: every level's vectors once, the stored matrices of the levels that
 * run the per-level kernels once per application, the dense coarsest inverse
 * once); 6 and 7: the cluster launch of that
 * hierarchy's coarse levels alone (FSI_ERR_INVALID when they run as
 * per-level kernels); 8: the C_f row assembly by located points (coupling
 * 0 only), 9: by mesh intersection (coupling 1 only), both on the current
 * X^n (L2 evicted; bytes = 0); 10 .. 13 (precision 1, fused finest levels
 * only, else FSI_ERR_INVALID): the fused matrix-free launch of the finest
 * level, velocity down (pre-smoothing, residual, restriction) and up
 * (prolongation, post-smoothing), pressure down and up, L2 evicted.
 * avg_ms: mean launch time; bytes: algorithmic bytes of one launch (stored
 * blocks and indices without padding, each vector once).  Allocates and
 * frees a 256 MiB scratch buffer. */
int fsi_time_kernel(fsi_problem* p, int which, int reps, double* avg_ms, double* bytes);

/* Measurement hook: algorithmic floating-point operations of one launch of
 * kernel `which` (10 .. 13 of fsi_time_kernel), or of one V-cycle (4, 5):
 * two per stored scalar entry of each operator and transfer application,
 * six per unknown per smoothing step, two per entry of the dense coarsest
 * inverse, without the work the tiles repeat on their overlaps.  Precision
 * 1 only (FSI_ERR_INVALID otherwise). */
int fsi_kernel_flops(fsi_problem* p, int which, double* flops);

/* Right-hand side of the last fsi_assemble_step in block order (n_total). */
int fsi_get_rhs(fsi_problem* p, double* b);

void fsi_destroy(fsi_problem* p);
const char* fsi_status_str(int status);

/* ---------------------------------------------------------------------------
 * Allocation-free point location and binning.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory when
 * they need the work done (code running while a stream is captured into a CUDA
 * graph, hosts that forbid allocation after start-up, plugins confined to
 * another framework's memory pool).  It performs steps S2-S3 on its own: it
 * locates the 6 degree-4 rule points of every triangle (point id =
 * 6*triangle + q, same arithmetic and cell rule as fsi_assemble_step) and
 * sorts them into per-cell lists.  It calls no cudaMalloc, cudaFree or other
 * allocating routine; its only scratch is a fixed array compiled into the
 * library, FSI_NOALLOC_MAX_CELLS counters wide, which every GPU that loads the
 * library holds until the process exits.
 *
 * All pointers are DEVICE pointers owned by the caller:
 *   tris  3*n_tris node ids;  X  2*n_nodes positions (x, y interleaved);
 *   cell, xi, eta  6*n_tris outputs (cell = cy*N + cx, or -1 outside [0,1]^2);
 *   cell_start  N*N + 1 outputs (CSR offsets), cell_points  6*n_tris outputs
 *   (point ids of each cell in increasing order; points outside are left out);
 *   n_outside  one int output: points found outside the domain.
 * Work is queued on cuda_stream (may be NULL: the current device's legacy
 * stream) on the device that stream belongs to, and the call returns without
 * waiting.  Returns FSI_ERR_INVALID, allocating and launching nothing, when a
 * pointer is NULL or N*N exceeds FSI_NOALLOC_MAX_CELLS (N <= 512).  The first
 * call on a device looks up the scratch array's device address and uploads the
 * rule table there (no allocation, but a synchronous copy); make that first
 * call before any stream capture: while it is still pending, a call on a
 * capturing stream returns FSI_ERR_INVALID and leaves the capture untouched.
 * An error left pending by an earlier CUDA call of the process is not
 * cleared: the call returns FSI_ERR_CUDA without launching.  Every call shares
 * the one scratch array and clears the part it uses before using it; calls
 * that overlap on the GPU race on it, so callers must serialise them.  The
 * per-cell lists are sorted by one thread per cell, in time quadratic in the
 * points of a cell (about 50 when the solid mesh size is half the fluid's). */
#define FSI_NOALLOC_MAX_CELLS 262144
int fsi_locate_bin_noalloc(int N, int n_tris, const int* tris, const double* X,
                           int* cell, double* xi, double* eta,
                           int* cell_start, int* cell_points, int* n_outside,
                           void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FSI_GB300_H */
