// Internal declarations shared by the host setup, the kernels and the
// solver of the GB300 FSI library.  Nothing here is part of the C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

namespace fsi {

// ---------------------------------------------------------------- host side
// Block-sparse matrix with BR x BC blocks; KRON blocks store one scalar s and
// act as s * I (BR == BC).  Rows are sorted by column.
struct HostBlockMatrix {
  int BR = 1, BC = 1, NV = 1;   // NV: values stored per block
  bool kron = false;
  int nrows = 0, ncols = 0;     // block rows / block columns
  std::vector<int> ptr, col;
  std::vector<double> val;      // NV per block, row-major inside a block
  size_t nnzb() const { return col.size(); }
};

// Type-blocked numbering of the interior Q2 nodes of an N x N grid:
// cell corners, then x-edge midpoints, then y-edge midpoints, then cell
// centres, each block in lattice order.  Rows of one block have the same
// stencil, so a 32-row slice needs little padding.
struct VNum {
  int N = 0, nV = 0, nX = 0, nY = 0, nC = 0, n = 0;
  explicit VNum(int N_ = 0);
  int id(int ix, int iy) const;                 // lattice -> internal, -1 on the wall
  void lattice(int k, int& ix, int& iy) const;  // internal -> lattice
};

struct FluidLevelHost {
  int N = 0;
  double h = 0;
  HostBlockMatrix A;      // A_f = (rho/dt) M + K, 2x2 blocks over interior nodes
  HostBlockMatrix L;      // pressure Laplacian B diag(M)^-1 B^T, 3x3 cell blocks
  HostBlockMatrix Pu, Ru; // velocity prolongation from / restriction to the coarser level (kron 2)
  HostBlockMatrix Pp, Rp; // pressure prolongation / restriction (3x3)
  HostBlockMatrix RAp;    // Rp L (coarse rows x fine columns, full blocks): the restricted
                          // pressure residual R (b - L x) = R b - (R L) x in one pass
  std::vector<double> dinvA, dinvL;  // Jacobi inverses (per scalar dof)
  double lmaxA = 0, lmaxL = 0;       // lambda_max of D^-1 A and D^-1 L
  // Matrix-free form of A and L on the uniform grid (levels with N >= 4).
  // A: one 2x2 block per (node type, lattice offset) -- every interior row of
  // a type has the same blocks, a wall neighbour's block is simply absent;
  // type = (ix & 1) | (iy & 1) << 1 (corner, x-edge, y-edge, centre).
  // L: one 3x3 block per (wall variant of the row cell, cell offset); the
  // variant v = 3 vy + vx with vx = 0 (cx = 0), 1 (inside), 2 (cx = N-1).
  // Both are the rows of the assembled matrices, bit for bit.
  bool mf = false;
  double stenA[4][5][5][4] = {};     // [type][dy+2][dx+2][2x2 row-major]
  double dinvAt[4][2] = {};          // D^-1 per type and component
  double stenL[9][3][3][9] = {};     // [variant][dy+1][dx+1][3x3 row-major]
  double dinvLv[9][3] = {};          // D^-1 per variant and pressure dof
  // the entries of -B and of -B^T (the same numbers): [pressure dof][node of
  // the cell, 3 y + x][velocity component]; one cell contributes to each
  // (cell, node) pair, so they are the assembled values
  double divB[3][9][2] = {};
};

struct SetupParams {
  int N; double rho, nu, kappa, dt, lid;
  int npe = 3;            // solid element: 3 = P1 triangle, 4 = Q1 quadrilateral
  int coarse_max = 8;     // coarsening stops at the first grid of at most this many cells a side
  int coarse_max_p = 0;   // the same for the pressure hierarchy (0: coarse_max)
};

struct HostSetup {
  // finest level operators of Eq. (matrix)
  HostBlockMatrix M;      // fluid mass (kron 2) over interior nodes
  HostBlockMatrix Bt;     // -B^T: node rows x cell columns, 2x3 blocks (sign folded in)
  HostBlockMatrix Bneg;   // -B: cell rows x node columns, 3x2 blocks (sign folded in)
  HostBlockMatrix Ssol;   // solid pair: per block (A_s, C_s) scalars, NV = 2
  HostBlockMatrix Cs;     // solid mass (kron 2)
  HostBlockMatrix As;     // solid stiffness (kron 2)
  std::vector<double> lift_u;  // -K_ID u_D on interior velocity rows
  std::vector<double> lift_p;  // B_D u_D on pressure rows
  std::vector<double> mp_inv;  // inverse P1disc mass diagonal, 3 per cell
  std::vector<double> cs_dinv; // inverse diagonal of the solid mass
  std::vector<FluidLevelHost> levels;  // 0 = finest
  int nlev_u = 0, nlev_p = 0;          // levels of the velocity / pressure hierarchy (the first ones)
  // the coarsest level as dense row-major matrices, inverted on the device
  // when a problem is created: A_f, and the pressure Laplacian made regular
  // by a rank-one term (L + t e e^T / |e|^2, whose inverse equals L^+ on
  // right-hand sides orthogonal to the constants e, up to e-components)
  std::vector<double> coarseA;
  std::vector<double> coarseL;
  int coarse_nA = 0, coarse_nL = 0;
  std::vector<int> interior_lattice;   // internal node -> lattice id (finest)
  std::vector<int> lattice_to_node;    // lattice id -> internal node or -1
  std::vector<double> wall_u;          // lattice nodal wall data, 2 per node
  // solid mesh data for the coupling assembly
  std::vector<double> tri_area;        // P1: reference areas
  std::vector<double> pt_w;            // Q1: w_q |det J_E(s_q)| per rule point (9 per element)
  std::vector<int> node_tri_ptr, node_tri;  // node -> (element*npe + local vertex)
  double cs_lo = 0.5, cs_hi = 2.0;     // an interval holding the spectrum of D^-1 C_s
};

void build_setup(const SetupParams& sp, int n_s, int n_tri, const double* ref_xy,
                 const int* tris, HostSetup& out);

// 6-point degree-4 symmetric triangle rule (Dunavant 1985): barycentric
// (lam0, lam1, lam2) and weights summing to 1, in the order used by the
// point-location kernel (point id = 6*triangle + q).
void triangle_rule(double lam[6][3], double w[6]);

// 3 x 3 Gauss-Legendre rule on the unit square: point q = 3 j + i at
// (s_i, t_j), its rounded product s t, and weights summing to 1.
void quad_rule(double s[9], double t[9], double st[9], double w[9]);

// Bilinear shape functions of the unit square's vertices (0,0), (1,0),
// (1,1), (0,1) at (s, t).
void q1_shape(double s, double t, double chi[4]);

// ------------------------------------------------------------- device side
template <class T>
struct Sell {            // sliced ELL of block rows, slice height 8
  static constexpr int kMaxRuns = 16;
  int nrows = 0;         // block rows
  int BR = 1, BC = 1, NV = 1;
  bool kron = false;
  const int* soff = nullptr;  // per slice: first slot
  const int* len = nullptr;   // per block row
  const int* col = nullptr;   // per slot (-1 in padding slots when nrun > 0)
  const T* val = nullptr;     // NV per slot
  // Slices of equal width come in a few runs on the structured fluid grid
  // (node types x wall rows).  With nrun > 0 a kernel computes the first slot
  // of slice s as run_off[k] + 8 (s - run_s[k]) run_w[k] for the run k that
  // holds s and scans run_w[k] slots, skipping column -1, so it reads neither
  // soff nor len (one dependent memory round trip less per launch).
  int nrun = 0;
  int tpr = 4;                 // threads per block row of the per-level SpMV (4 or 8, set by the autotuner)
  int run_s[kMaxRuns] = {};    // first slice of each run
  int run_w[kMaxRuns] = {};    // slots per row in the run
  int run_off[kMaxRuns] = {};  // first slot of the run
};

struct SellHost {        // SELL arrays before upload
  int nrows = 0, nslices = 0, BR = 1, BC = 1, NV = 1;
  bool kron = false;
  std::vector<int> soff, len, col;
  std::vector<double> val;
};
SellHost to_sell(const HostBlockMatrix& A);

}  // namespace fsi
