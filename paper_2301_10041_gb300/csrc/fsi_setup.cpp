// Host-side discretisation of the FSI step (the paper's T_ass work, done once
// per problem): Q2/P1disc fluid operators on the uniform grid and its
// multigrid hierarchy, P1 solid operators, and the sliced-ELL layout.
//
// Element matrices are written in closed form from 1-D integrals of the
// quadratic Lagrange basis on [0,1] (nodes 0, 1/2, 1); every cell is the
// same square, so one element matrix serves the whole grid.  The definitions
// are those after Eq. (matrix) of the paper:
//   M_ij = (phi_j, phi_i), K_ij = nu (eps(phi_j), eps(phi_i)),
//   B_ki = (div phi_i, psi_k), A_s = kappa (grad chi_j, grad chi_i)_B,
//   C_s = (chi_l, chi_j)_B.
#include "fsi_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

namespace fsi {

// ------------------------------------------------------------------ numbering
VNum::VNum(int N_) : N(N_) {
  if (N <= 0) return;
  nV = (N - 1) * (N - 1);
  nX = N * (N - 1);
  nY = (N - 1) * N;
  nC = N * N;
  n = nV + nX + nY + nC;
}

int VNum::id(int ix, int iy) const {
  if (ix <= 0 || iy <= 0 || ix >= 2 * N || iy >= 2 * N) return -1;
  const bool ox = ix & 1, oy = iy & 1;
  if (!ox && !oy) return (iy / 2 - 1) * (N - 1) + (ix / 2 - 1);
  if (ox && !oy) return nV + (iy / 2 - 1) * N + (ix - 1) / 2;
  if (!ox && oy) return nV + nX + ((iy - 1) / 2) * (N - 1) + (ix / 2 - 1);
  return nV + nX + nY + ((iy - 1) / 2) * N + (ix - 1) / 2;
}

void VNum::lattice(int k, int& ix, int& iy) const {
  if (k < nV) { ix = 2 * (k % (N - 1) + 1); iy = 2 * (k / (N - 1) + 1); return; }
  k -= nV;
  if (k < nX) { ix = 2 * (k % N) + 1; iy = 2 * (k / N + 1); return; }
  k -= nX;
  if (k < nY) { ix = 2 * (k % (N - 1) + 1); iy = 2 * (k / (N - 1)) + 1; return; }
  k -= nY;
  ix = 2 * (k % N) + 1; iy = 2 * (k / N) + 1;
}

// -------------------------------------------------------- 1-D Q2 integrals
// Basis on [0,1]: L0 = (1-t)(1-2t), L1 = 4t(1-t), L2 = t(2t-1).
static const double M1[3][3] = {{4 / 30.0, 2 / 30.0, -1 / 30.0},
                                {2 / 30.0, 16 / 30.0, 2 / 30.0},
                                {-1 / 30.0, 2 / 30.0, 4 / 30.0}};          // int L_a L_b
static const double K1[3][3] = {{7 / 3.0, -8 / 3.0, 1 / 3.0},
                                {-8 / 3.0, 16 / 3.0, -8 / 3.0},
                                {1 / 3.0, -8 / 3.0, 7 / 3.0}};             // int L_a' L_b'
static const double G1[3][3] = {{-0.5, -2 / 3.0, 1 / 6.0},
                                {2 / 3.0, 0.0, -2 / 3.0},
                                {-1 / 6.0, 2 / 3.0, 0.5}};                 // int L_a' L_b
static const double E1[3] = {-1.0, 0.0, 1.0};                            // int L_a'
static const double F1[3] = {1 / 3.0, -2 / 3.0, 1 / 3.0};                // int L_a' (t - 1/2)
static const double C0[3] = {1 / 6.0, 2 / 3.0, 1 / 6.0};                 // int L_a
static const double C1[3] = {-1 / 12.0, 0.0, 1 / 12.0};                  // int L_a (t - 1/2)

struct Elem {
  double A[9][9][2][2];  // test node, trial node, test comp, trial comp
  double K[9][9][2][2];  // viscous part only
  double M[9][9];        // scalar mass
  double B[3][9][2];     // pressure basis k, node, component: (d phi / dx_c, psi_k)
};

static void element(double h, double ma, double nu, Elem& e) {
  for (int al = 0; al < 9; ++al) {
    const int aa = al % 3, ab = al / 3;
    for (int be = 0; be < 9; ++be) {
      const int ba = be % 3, bb = be / 3;
      const double mass = h * h * M1[aa][ba] * M1[ab][bb];
      const double sxx = K1[aa][ba] * M1[ab][bb];
      const double syy = M1[aa][ba] * K1[ab][bb];
      const double sxy_ab = G1[aa][ba] * G1[bb][ab];  // int dx phi_al dy phi_be
      const double sxy_ba = G1[ba][aa] * G1[ab][bb];  // int dx phi_be dy phi_al
      e.M[al][be] = mass;
      e.K[al][be][0][0] = nu * (sxx + 0.5 * syy);
      e.K[al][be][1][1] = nu * (syy + 0.5 * sxx);
      e.K[al][be][0][1] = 0.5 * nu * sxy_ba;
      e.K[al][be][1][0] = 0.5 * nu * sxy_ab;
      for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2; ++d) e.A[al][be][c][d] = e.K[al][be][c][d] + (c == d ? ma * mass : 0.0);
    }
    e.B[0][al][0] = h * E1[aa] * C0[ab];
    e.B[1][al][0] = h * F1[aa] * C0[ab];
    e.B[2][al][0] = h * E1[aa] * C1[ab];
    e.B[0][al][1] = h * C0[aa] * E1[ab];
    e.B[1][al][1] = h * C1[aa] * E1[ab];
    e.B[2][al][1] = h * C0[aa] * F1[ab];
  }
}

// ----------------------------------------------------------- row accumulator
struct RowAcc {
  int NV;
  std::vector<int> cols;
  std::vector<double> vals;
  explicit RowAcc(int nv) : NV(nv) {}
  double* slot(int c) {
    for (size_t i = 0; i < cols.size(); ++i)
      if (cols[i] == c) return &vals[i * NV];
    cols.push_back(c);
    vals.resize(vals.size() + NV, 0.0);
    return &vals[(cols.size() - 1) * NV];
  }
  void flush(HostBlockMatrix& A) {
    std::vector<int> idx(cols.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return cols[a] < cols[b]; });
    for (int i : idx) {
      A.col.push_back(cols[i]);
      for (int v = 0; v < NV; ++v) A.val.push_back(vals[(size_t)i * NV + v]);
    }
    A.ptr.push_back((int)A.col.size());
    cols.clear();
    vals.clear();
  }
};

static void init_matrix(HostBlockMatrix& A, int BR, int BC, bool kron, int nrows, int ncols) {
  A.BR = BR; A.BC = BC; A.kron = kron; A.NV = kron ? 1 : BR * BC;
  A.nrows = nrows; A.ncols = ncols;
  A.ptr.assign(1, 0); A.col.clear(); A.val.clear();
}

// cells containing lattice coordinate i (1-D): even -> two cells, odd -> one
static int cells_of(int i, int N, int out[2]) {
  int n = 0;
  if (i & 1) { out[n++] = (i - 1) / 2; }
  else {
    if (i / 2 - 1 >= 0) out[n++] = i / 2 - 1;
    if (i / 2 < N) out[n++] = i / 2;
  }
  return n;
}

// Velocity operator A_f (2x2 blocks) of an N-cell grid with cell size h; also
// the kron-2 mass matrix and the Dirichlet lift -K_ID u_D when requested.
static void assemble_velocity(int N, double h, double ma, double nu, HostBlockMatrix& A,
                              HostBlockMatrix* M, const std::vector<double>* wall,
                              std::vector<double>* lift) {
  VNum vn(N);
  Elem e;
  element(h, ma, nu, e);
  init_matrix(A, 2, 2, false, vn.n, vn.n);
  if (M) init_matrix(*M, 2, 2, true, vn.n, vn.n);
  if (lift) lift->assign(2 * (size_t)vn.n, 0.0);
  const int n1 = 2 * N + 1;
  RowAcc ra(4), rm(1);
  for (int k = 0; k < vn.n; ++k) {
    int ix, iy;
    vn.lattice(k, ix, iy);
    int cxs[2], cys[2];
    const int ncx = cells_of(ix, N, cxs), ncy = cells_of(iy, N, cys);
    for (int a = 0; a < ncy; ++a)
      for (int b = 0; b < ncx; ++b) {
        const int cx = cxs[b], cy = cys[a];
        const int al = (iy - 2 * cy) * 3 + (ix - 2 * cx);
        for (int be = 0; be < 9; ++be) {
          const int jx = 2 * cx + be % 3, jy = 2 * cy + be / 3;
          const int c = vn.id(jx, jy);
          if (c >= 0) {
            double* s = ra.slot(c);
            s[0] += e.A[al][be][0][0]; s[1] += e.A[al][be][0][1];
            s[2] += e.A[al][be][1][0]; s[3] += e.A[al][be][1][1];
            if (M) rm.slot(c)[0] += e.M[al][be];
          } else if (lift && wall) {
            const double* ud = &(*wall)[2 * ((size_t)jy * n1 + jx)];
            for (int cc = 0; cc < 2; ++cc)
              (*lift)[2 * (size_t)k + cc] -= e.K[al][be][cc][0] * ud[0] + e.K[al][be][cc][1] * ud[1];
          }
        }
      }
    ra.flush(A);
    if (M) rm.flush(*M);
  }
}

// -B (cell rows, 3x2 blocks) and -B^T (node rows, 2x3 blocks), plus B_D u_D.
static void assemble_divergence(int N, double h, HostBlockMatrix& Bneg, HostBlockMatrix* Bt,
                                const std::vector<double>* wall, std::vector<double>* liftp) {
  VNum vn(N);
  Elem e;
  element(h, 0.0, 0.0, e);
  const int nc = N * N, n1 = 2 * N + 1;
  init_matrix(Bneg, 3, 2, false, nc, vn.n);
  if (liftp) liftp->assign(3 * (size_t)nc, 0.0);
  RowAcc acc(6);
  for (int c = 0; c < nc; ++c) {
    const int cx = c % N, cy = c / N;
    for (int be = 0; be < 9; ++be) {
      const int jx = 2 * cx + be % 3, jy = 2 * cy + be / 3;
      const int col = vn.id(jx, jy);
      if (col >= 0) {
        double* s = acc.slot(col);
        for (int k = 0; k < 3; ++k)
          for (int d = 0; d < 2; ++d) s[k * 2 + d] -= e.B[k][be][d];
      } else if (liftp && wall) {
        const double* ud = &(*wall)[2 * ((size_t)jy * n1 + jx)];
        for (int k = 0; k < 3; ++k) (*liftp)[3 * (size_t)c + k] += e.B[k][be][0] * ud[0] + e.B[k][be][1] * ud[1];
      }
    }
    acc.flush(Bneg);
  }
  if (Bt) {
    init_matrix(*Bt, 2, 3, false, vn.n, nc);
    RowAcc at(6);
    for (int k = 0; k < vn.n; ++k) {
      int ix, iy;
      vn.lattice(k, ix, iy);
      int cxs[2], cys[2];
      const int ncx = cells_of(ix, N, cxs), ncy = cells_of(iy, N, cys);
      for (int a = 0; a < ncy; ++a)
        for (int b = 0; b < ncx; ++b) {
          const int cx = cxs[b], cy = cys[a];
          const int al = (iy - 2 * cy) * 3 + (ix - 2 * cx);
          double* s = at.slot(cy * N + cx);
          for (int d = 0; d < 2; ++d)
            for (int kk = 0; kk < 3; ++kk) s[d * 3 + kk] -= e.B[kk][al][d];
        }
      at.flush(*Bt);
    }
  }
}

// Pressure Laplacian L = B diag(M)^-1 B^T on cell blocks (3x3).
static void assemble_pressure_laplacian(int N, double h, HostBlockMatrix& L) {
  VNum vn(N);
  Elem e;
  element(h, 0.0, 0.0, e);
  // diagonal of the scalar mass at each interior node
  std::vector<double> dm(vn.n, 0.0);
  for (int k = 0; k < vn.n; ++k) {
    int ix, iy;
    vn.lattice(k, ix, iy);
    int cxs[2], cys[2];
    const int ncx = cells_of(ix, N, cxs), ncy = cells_of(iy, N, cys);
    for (int a = 0; a < ncy; ++a)
      for (int b = 0; b < ncx; ++b) {
        const int al = (iy - 2 * cys[a]) * 3 + (ix - 2 * cxs[b]);
        dm[k] += e.M[al][al];
      }
  }
  const int nc = N * N;
  init_matrix(L, 3, 3, false, nc, nc);
  RowAcc acc(9);
  for (int c1 = 0; c1 < nc; ++c1) {
    const int cx1 = c1 % N, cy1 = c1 / N;
    for (int al1 = 0; al1 < 9; ++al1) {
      const int ix = 2 * cx1 + al1 % 3, iy = 2 * cy1 + al1 / 3;
      const int node = vn.id(ix, iy);
      if (node < 0) continue;
      const double wgt = 1.0 / dm[node];
      int cxs[2], cys[2];
      const int ncx = cells_of(ix, N, cxs), ncy = cells_of(iy, N, cys);
      for (int a = 0; a < ncy; ++a)
        for (int b = 0; b < ncx; ++b) {
          const int cx2 = cxs[b], cy2 = cys[a];
          const int al2 = (iy - 2 * cy2) * 3 + (ix - 2 * cx2);
          double* s = acc.slot(cy2 * N + cx2);
          for (int k1 = 0; k1 < 3; ++k1)
            for (int k2 = 0; k2 < 3; ++k2)
              s[k1 * 3 + k2] += wgt * (e.B[k1][al1][0] * e.B[k2][al2][0] + e.B[k1][al1][1] * e.B[k2][al2][1]);
        }
    }
    acc.flush(L);
  }
}

// Q2 prolongation from an Nc grid to a 2Nc grid (scalar weights, kron 2):
// the coarse quadratic evaluated at the fine nodes, 1-D weights
// L_a(t) at t in {0, 1/4, 1/2, 3/4, 1}.
static void assemble_prolong_u(int Nc, HostBlockMatrix& P) {
  const int Nf = 2 * Nc;
  VNum vf(Nf), vc(Nc);
  init_matrix(P, 2, 2, true, vf.n, vc.n);
  RowAcc acc(1);
  auto w1 = [](int f, int Nc_, int& cc, double w[3]) {
    cc = std::min(f / 4, Nc_ - 1);
    const int r = f - 4 * cc;  // 0..4
    static const double tab[5][3] = {{1, 0, 0}, {0.375, 0.75, -0.125}, {0, 1, 0},
                                     {-0.125, 0.75, 0.375}, {0, 0, 1}};
    for (int a = 0; a < 3; ++a) w[a] = tab[r][a];
  };
  for (int k = 0; k < vf.n; ++k) {
    int fx, fy;
    vf.lattice(k, fx, fy);
    int ccx, ccy;
    double wx[3], wy[3];
    w1(fx, Nc, ccx, wx);
    w1(fy, Nc, ccy, wy);
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        const double w = wx[a] * wy[b];
        if (w == 0.0) continue;
        const int c = vc.id(2 * ccx + a, 2 * ccy + b);
        if (c < 0) continue;
        acc.slot(c)[0] += w;
      }
    acc.flush(P);
  }
}

// P1disc prolongation: the coarse linear function restricted to each child.
static void assemble_prolong_p(int Nc, HostBlockMatrix& P) {
  const int Nf = 2 * Nc;
  init_matrix(P, 3, 3, false, Nf * Nf, Nc * Nc);
  for (int f = 0; f < Nf * Nf; ++f) {
    const int fx = f % Nf, fy = f / Nf;
    const double sx = (fx & 1) ? 0.25 : -0.25, sy = (fy & 1) ? 0.25 : -0.25;
    P.col.push_back((fy / 2) * Nc + fx / 2);
    const double blk[9] = {1, sx, sy, 0, 0.5, 0, 0, 0, 0.5};
    P.val.insert(P.val.end(), blk, blk + 9);
    P.ptr.push_back((int)P.col.size());
  }
}

static HostBlockMatrix transpose(const HostBlockMatrix& A) {
  HostBlockMatrix T;
  init_matrix(T, A.BC, A.BR, A.kron, A.ncols, A.nrows);
  std::vector<int> cnt(A.ncols + 1, 0);
  for (int c : A.col) cnt[c + 1]++;
  for (int i = 0; i < A.ncols; ++i) cnt[i + 1] += cnt[i];
  T.ptr = cnt;
  T.col.assign(A.col.size(), 0);
  T.val.assign(A.val.size(), 0.0);
  std::vector<int> pos(cnt.begin(), cnt.end() - 1);
  for (int r = 0; r < A.nrows; ++r)
    for (int j = A.ptr[r]; j < A.ptr[r + 1]; ++j) {
      const int c = A.col[j];
      const int dst = pos[c]++;
      T.col[dst] = r;
      for (int i = 0; i < A.BR; ++i)
        for (int jj = 0; jj < A.BC; ++jj) {
          if (A.kron) { if (i == 0 && jj == 0) T.val[dst] = A.val[j]; continue; }
          T.val[(size_t)dst * T.NV + jj * A.BR + i] = A.val[(size_t)j * A.NV + i * A.BC + jj];
        }
    }
  return T;
}

// C = R A for a block matrix R (B x B blocks, kron or full) and a square-block
// matrix A (B x B, full): full B x B blocks, rows sorted by column.
static HostBlockMatrix block_product(const HostBlockMatrix& R, const HostBlockMatrix& A) {
  const int B = A.BR;
  if (A.BC != B || A.kron || R.BR != B || R.BC != B || R.ncols != A.nrows)
    throw std::logic_error("block_product: shapes");
  HostBlockMatrix C;
  init_matrix(C, B, B, false, R.nrows, A.ncols);
  const int BB = B * B;
  std::vector<int> slot(A.ncols, -1), cols, order;
  std::vector<double> acc;
  for (int r = 0; r < R.nrows; ++r) {
    cols.clear();
    acc.clear();
    for (int j = R.ptr[r]; j < R.ptr[r + 1]; ++j) {
      const int k = R.col[j];
      for (int m = A.ptr[k]; m < A.ptr[k + 1]; ++m) {
        const int c = A.col[m];
        if (slot[c] < 0) {
          slot[c] = (int)cols.size();
          cols.push_back(c);
          acc.resize(acc.size() + BB, 0.0);
        }
        double* dst = &acc[(size_t)slot[c] * BB];
        const double* a = &A.val[(size_t)m * BB];
        for (int i = 0; i < B; ++i)
          for (int jj = 0; jj < B; ++jj) {
            double sum = 0.0;
            if (R.kron) {
              sum = R.val[j] * a[i * B + jj];
            } else {
              for (int q = 0; q < B; ++q) sum += R.val[(size_t)j * BB + i * B + q] * a[q * B + jj];
            }
            dst[i * B + jj] += sum;
          }
      }
    }
    order.resize(cols.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cols[x] < cols[y]; });
    for (int i : order) {
      C.col.push_back(cols[i]);
      for (int v = 0; v < BB; ++v) C.val.push_back(acc[(size_t)i * BB + v]);
      slot[cols[i]] = -1;
    }
    C.ptr.push_back((int)C.col.size());
  }
  return C;
}

static std::vector<double> block_diag_inverse_scalar(const HostBlockMatrix& A) {
  // inverse of the scalar diagonal (per dof) of a square block matrix
  std::vector<double> d((size_t)A.nrows * A.BR, 0.0);
  for (int r = 0; r < A.nrows; ++r)
    for (int j = A.ptr[r]; j < A.ptr[r + 1]; ++j)
      if (A.col[j] == r)
        for (int i = 0; i < A.BR; ++i)
          d[(size_t)r * A.BR + i] = A.kron ? A.val[j] : A.val[(size_t)j * A.NV + i * A.BC + i];
  for (auto& v : d) v = 1.0 / v;
  return d;
}

static void host_spmv(const HostBlockMatrix& A, const std::vector<double>& x, std::vector<double>& y) {
  y.assign((size_t)A.nrows * A.BR, 0.0);
  for (int r = 0; r < A.nrows; ++r)
    for (int j = A.ptr[r]; j < A.ptr[r + 1]; ++j) {
      const int c = A.col[j];
      for (int i = 0; i < A.BR; ++i)
        for (int k = 0; k < A.BC; ++k) {
          double v;
          if (A.kron) v = (i == k) ? A.val[j] : 0.0;
          else v = A.val[(size_t)j * A.NV + i * A.BC + k];
          y[(size_t)r * A.BR + i] += v * x[(size_t)c * A.BC + k];
        }
    }
}

// lambda_max of D^-1 A by power iteration (A symmetric, D its diagonal).
static double power_lmax(const HostBlockMatrix& A, const std::vector<double>& dinv, int iters) {
  const size_t n = (size_t)A.nrows * A.BR;
  std::vector<double> x(n), y;
  uint64_t s = 0x2301u;
  for (size_t i = 0; i < n; ++i) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    x[i] = (double)(s >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
  double lam = 0;
  for (int it = 0; it < iters; ++it) {
    // y = D^-1 A x; Rayleigh quotient in the D inner product
    host_spmv(A, x, y);
    double num = 0, den = 0;
    for (size_t i = 0; i < n; ++i) {
      num += x[i] * y[i];
      den += x[i] * x[i] / dinv[i];
    }
    lam = num / den;
    double nrm = 0;
    for (size_t i = 0; i < n; ++i) { y[i] *= dinv[i]; nrm += y[i] * y[i]; }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0)) break;
    for (size_t i = 0; i < n; ++i) x[i] = y[i] / nrm;
  }
  return lam;
}

static std::vector<double> dense_of(const HostBlockMatrix& A) {
  const int n = A.nrows * A.BR;
  std::vector<double> D((size_t)n * n, 0.0);
  for (int r = 0; r < A.nrows; ++r)
    for (int j = A.ptr[r]; j < A.ptr[r + 1]; ++j)
      for (int i = 0; i < A.BR; ++i)
        for (int k = 0; k < A.BC; ++k) {
          double v = A.kron ? (i == k ? A.val[j] : 0.0) : A.val[(size_t)j * A.NV + i * A.BC + k];
          D[(size_t)(r * A.BR + i) * n + A.col[j] * A.BC + k] += v;
        }
  return D;
}

void triangle_rule(double lam[6][3], double w[6]) {
  const double A1 = 0.44594849091596488632, W1 = 0.22338158967801146570;
  const double A2 = 0.091576213509770743460, W2 = 0.10995174365532186764;
  const double as[2] = {A1, A2}, ws[2] = {W1, W2};
  for (int o = 0; o < 2; ++o) {
    const double a = as[o], b = 1.0 - 2.0 * a;
    for (int r = 0; r < 3; ++r) {
      const int q = 3 * o + r;
      for (int v = 0; v < 3; ++v) lam[q][v] = (v == r) ? b : a;
      w[q] = ws[o];
    }
  }
}

void quad_rule(double s[9], double t[9], double st[9], double w[9]) {
  // 1-D Gauss-Legendre on [0,1]: 1/2 and 1/2 -/+ sqrt(3/5)/2, weights 4/9, 5/18
  const double r = 0.5 * std::sqrt(0.6);
  const double g[3] = {0.5 - r, 0.5, 0.5 + r};
  const double w1[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) {
      const int q = 3 * j + i;
      s[q] = g[i];
      t[q] = g[j];
      st[q] = g[i] * g[j];
      w[q] = w1[i] * w1[j];
    }
}

void q1_shape(double s, double t, double chi[4]) {
  chi[0] = (1.0 - s) * (1.0 - t);
  chi[1] = s * (1.0 - t);
  chi[2] = s * t;
  chi[3] = (1.0 - s) * t;
}

// Extreme eigenvalues of a symmetric 4 x 4 matrix by cyclic Jacobi rotations.
static void sym4_eig_range(double a[4][4], double& lo, double& hi) {
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < 4; ++p)
      for (int q = p + 1; q < 4; ++q) off += a[p][q] * a[p][q];
    if (off < 1e-30) break;
    for (int p = 0; p < 4; ++p)
      for (int q = p + 1; q < 4; ++q) {
        if (a[p][q] == 0.0) continue;
        const double th = 0.5 * (a[q][q] - a[p][p]) / a[p][q];
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < 4; ++k) {  // columns p, q
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - sn * akq;
          a[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < 4; ++k) {  // rows p, q
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - sn * aqk;
          a[q][k] = sn * apk + c * aqk;
        }
      }
  }
  lo = hi = a[0][0];
  for (int k = 1; k < 4; ++k) {
    lo = std::min(lo, a[k][k]);
    hi = std::max(hi, a[k][k]);
  }
}

// Matrix-free stencils of one level (cell size h), read from the rows of
// proxy grids assembled by the same routines: an 8-cell grid for A (the rows
// of the nodes at lattice (8 + ox, 8 + oy) have all their neighbours inside)
// and a 4-cell grid for L (cells 0, 1 and 3 give the three variants per
// axis).  The blocks are therefore the assembled values bit for bit.
static void matrix_free_stencils(double h, double ma, double nu, FluidLevelHost& L) {
  HostBlockMatrix A8, L4;
  assemble_velocity(8, h, ma, nu, A8, nullptr, nullptr, nullptr);
  VNum v8(8);
  for (int tau = 0; tau < 4; ++tau) {
    const int ix = 8 + (tau & 1), iy = 8 + (tau >> 1);
    const int row = v8.id(ix, iy);
    for (int k = A8.ptr[row]; k < A8.ptr[row + 1]; ++k) {
      int jx, jy;
      v8.lattice(A8.col[k], jx, jy);
      const int dx = jx - ix, dy = jy - iy;
      if (dx < -2 || dx > 2 || dy < -2 || dy > 2) throw std::logic_error("velocity stencil wider than 5x5");
      for (int q = 0; q < 4; ++q) L.stenA[tau][dy + 2][dx + 2][q] = A8.val[4 * (size_t)k + q];
      if (dx == 0 && dy == 0) {
        L.dinvAt[tau][0] = 1.0 / A8.val[4 * (size_t)k];
        L.dinvAt[tau][1] = 1.0 / A8.val[4 * (size_t)k + 3];
      }
    }
  }
  assemble_pressure_laplacian(4, h, L4);
  const int rep[3] = {0, 1, 3};
  for (int vy = 0; vy < 3; ++vy)
    for (int vx = 0; vx < 3; ++vx) {
      const int v = 3 * vy + vx, cx = rep[vx], cy = rep[vy], row = cy * 4 + cx;
      for (int k = L4.ptr[row]; k < L4.ptr[row + 1]; ++k) {
        const int c2 = L4.col[k], dx = c2 % 4 - cx, dy = c2 / 4 - cy;
        if (dx < -1 || dx > 1 || dy < -1 || dy > 1) throw std::logic_error("pressure stencil wider than 3x3");
        for (int q = 0; q < 9; ++q) L.stenL[v][dy + 1][dx + 1][q] = L4.val[9 * (size_t)k + q];
        if (dx == 0 && dy == 0)
          for (int i = 0; i < 3; ++i) L.dinvLv[v][i] = 1.0 / L4.val[9 * (size_t)k + 4 * i];
      }
    }
  Elem e;
  element(h, 0.0, 0.0, e);
  for (int k = 0; k < 3; ++k)
    for (int al = 0; al < 9; ++al)
      for (int d = 0; d < 2; ++d) L.divB[k][al][d] = 0.0 - e.B[k][al][d];
  L.mf = true;
}

void build_setup(const SetupParams& sp, int n_s, int n_tri, const double* ref_xy, const int* tris,
                 HostSetup& out) {
  const int N = sp.N;
  const double ma = sp.rho / sp.dt;
  const int n1 = 2 * N + 1;
  VNum vn(N);
  // wall data: top wall strictly between the corners moves with (lid, 0)
  out.wall_u.assign(2 * (size_t)n1 * n1, 0.0);
  if (sp.lid != 0.0)
    for (int ix = 1; ix < n1 - 1; ++ix) out.wall_u[2 * ((size_t)(n1 - 1) * n1 + ix)] = sp.lid;
  out.interior_lattice.resize(vn.n);
  out.lattice_to_node.assign((size_t)n1 * n1, -1);
  for (int k = 0; k < vn.n; ++k) {
    int ix, iy;
    vn.lattice(k, ix, iy);
    out.interior_lattice[k] = iy * n1 + ix;
    out.lattice_to_node[(size_t)iy * n1 + ix] = k;
  }
  // ---- multigrid hierarchy: N, N/2, ... while even and above coarse_max
  // cells a side; the coarsest is solved with its dense inverse (a grid of 16
  // cells has 2 * 31^2 = 1922 velocity unknowns)
  const int cu = sp.coarse_max, cp = sp.coarse_max_p > 0 ? sp.coarse_max_p : sp.coarse_max;
  std::vector<int> Ns{N};
  while (Ns.back() % 2 == 0 && Ns.back() > std::min(cu, cp)) Ns.push_back(Ns.back() / 2);
  // each hierarchy ends at its first grid of at most its coarse_max cells
  // (or at the last, odd, one)
  auto levels_to = [&](int c) {
    int l = 0;
    while (l + 1 < (int)Ns.size() && Ns[l] > c) ++l;
    return l + 1;
  };
  out.nlev_u = levels_to(cu);
  out.nlev_p = levels_to(cp);
  out.levels.resize(Ns.size());
  for (size_t l = 0; l < Ns.size(); ++l) {
    FluidLevelHost& L = out.levels[l];
    L.N = Ns[l];
    L.h = 1.0 / Ns[l];
    if (l == 0) {
      assemble_velocity(L.N, L.h, ma, sp.nu, L.A, &out.M, &out.wall_u, &out.lift_u);
      assemble_divergence(L.N, L.h, out.Bneg, &out.Bt, &out.wall_u, &out.lift_p);
    } else {
      assemble_velocity(L.N, L.h, ma, sp.nu, L.A, nullptr, nullptr, nullptr);
    }
    assemble_pressure_laplacian(L.N, L.h, L.L);
    L.dinvA = block_diag_inverse_scalar(L.A);
    L.dinvL = block_diag_inverse_scalar(L.L);
    if (L.N >= 4) matrix_free_stencils(L.h, ma, sp.nu, L);
    if (l + 1 < Ns.size()) {
      assemble_prolong_u(Ns[l + 1], L.Pu);
      L.Ru = transpose(L.Pu);
      assemble_prolong_p(Ns[l + 1], L.Pp);
      L.Rp = transpose(L.Pp);
      L.RAp = block_product(L.Rp, L.L);
    }
    // lambda_max on a proxy grid of at most 24 cells with the same cell size
    const int Np = std::min(L.N, 24);
    HostBlockMatrix Ap, Lp;
    assemble_velocity(Np, L.h, ma, sp.nu, Ap, nullptr, nullptr, nullptr);
    assemble_pressure_laplacian(Np, L.h, Lp);
    L.lmaxA = power_lmax(Ap, block_diag_inverse_scalar(Ap), 60);
    L.lmaxL = power_lmax(Lp, block_diag_inverse_scalar(Lp), 60);
  }
  {
    const FluidLevelHost& C = out.levels[out.nlev_u - 1];
    out.coarseA = dense_of(C.A);
    out.coarse_nA = C.A.nrows * 2;
    // the singular pressure Laplacian plus t e e^T / |e|^2 (t its mean
    // diagonal), e the constants (first dof of every cell)
    const FluidLevelHost& Cp = out.levels[out.nlev_p - 1];
    std::vector<double> Ld = dense_of(Cp.L);
    const int n = Cp.L.nrows * 3;
    out.coarse_nL = n;
    double t = 0;
    for (int i = 0; i < n; ++i) t += Ld[(size_t)i * n + i];
    t /= n;
    const double ee = (double)(n / 3);
    for (int i = 0; i < n; i += 3)
      for (int j = 0; j < n; j += 3) Ld[(size_t)i * n + j] += t / ee;
    out.coarseL.swap(Ld);
  }
  // inverse P1disc mass: diag(h^2, h^2/12, h^2/12) per cell
  {
    const double h2 = 1.0 / ((double)N * N);
    out.mp_inv.resize(3 * (size_t)N * N);
    for (size_t c = 0; c < (size_t)N * N; ++c) {
      out.mp_inv[3 * c] = 1.0 / h2;
      out.mp_inv[3 * c + 1] = 12.0 / h2;
      out.mp_inv[3 * c + 2] = 12.0 / h2;
    }
  }
  // ---- solid operators on the reference configuration (P1 or Q1)
  const int npe = sp.npe;
  out.node_tri_ptr.assign(n_s + 1, 0);
  for (int t = 0; t < n_tri; ++t)
    for (int a = 0; a < npe; ++a) out.node_tri_ptr[tris[npe * t + a] + 1]++;
  for (int i = 0; i < n_s; ++i) out.node_tri_ptr[i + 1] += out.node_tri_ptr[i];
  out.node_tri.assign(npe * (size_t)n_tri, 0);
  {
    std::vector<int> pos(out.node_tri_ptr.begin(), out.node_tri_ptr.end() - 1);
    for (int t = 0; t < n_tri; ++t)
      for (int a = 0; a < npe; ++a) out.node_tri[pos[tris[npe * t + a]]++] = npe * t + a;
  }
  HostBlockMatrix S;
  init_matrix(S, 2, 2, true, n_s, n_s);
  S.NV = 2;  // (A_s, C_s) per block
  std::vector<RowAcc> acc(n_s, RowAcc(2));
  if (npe == 4) {
    // Q1: 3 x 3 Gauss on each element, J = [dx/ds dx/dt] of the bilinear map;
    // the interval for D^-1 C_s from the element mass matrices (Wathen: the
    // Rayleigh quotient of (C_s, D) lies between the extreme eigenvalues of
    // the element pairs (M_E, diag M_E))
    double qs[9], qt[9], qst[9], qw[9];
    quad_rule(qs, qt, qst, qw);
    out.pt_w.resize(9 * (size_t)n_tri);
    out.cs_lo = 1e300;
    out.cs_hi = 0.0;
    for (int e = 0; e < n_tri; ++e) {
      const int* v = tris + 4 * (size_t)e;
      double P[4][2];
      for (int a = 0; a < 4; ++a) { P[a][0] = ref_xy[2 * v[a]]; P[a][1] = ref_xy[2 * v[a] + 1]; }
      double Me[4][4] = {};
      for (int q = 0; q < 9; ++q) {
        const double s_ = qs[q], t_ = qt[q];
        double chi[4];
        q1_shape(s_, t_, chi);
        const double ds[4] = {-(1.0 - t_), 1.0 - t_, t_, -t_};
        const double dt[4] = {-(1.0 - s_), -s_, s_, 1.0 - s_};
        double xs = 0, ys = 0, xt = 0, yt = 0;
        for (int a = 0; a < 4; ++a) {
          xs += ds[a] * P[a][0]; ys += ds[a] * P[a][1];
          xt += dt[a] * P[a][0]; yt += dt[a] * P[a][1];
        }
        const double det = xs * yt - ys * xt;
        if (!(det > 0)) throw std::invalid_argument("solid quadrilateral not counter-clockwise");
        const double wd = qw[q] * det;
        out.pt_w[9 * (size_t)e + q] = wd;
        double g[4][2];
        for (int a = 0; a < 4; ++a) {
          g[a][0] = (yt * ds[a] - ys * dt[a]) / det;
          g[a][1] = (-xt * ds[a] + xs * dt[a]) / det;
        }
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            double* sl = acc[v[a]].slot(v[b]);
            sl[0] += sp.kappa * wd * (g[a][0] * g[b][0] + g[a][1] * g[b][1]);
            sl[1] += wd * chi[a] * chi[b];
            Me[a][b] += wd * chi[a] * chi[b];
          }
      }
      double Ds[4];
      for (int a = 0; a < 4; ++a) Ds[a] = 1.0 / std::sqrt(Me[a][a]);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) Me[a][b] *= Ds[a] * Ds[b];
      double lo, hi;
      sym4_eig_range(Me, lo, hi);
      out.cs_lo = std::min(out.cs_lo, lo);
      out.cs_hi = std::max(out.cs_hi, hi);
    }
    for (int i = 0; i < n_s; ++i) acc[i].flush(S);
  }
  if (npe == 3) out.tri_area.resize(n_tri);
  for (int t = 0; t < (npe == 3 ? n_tri : 0); ++t) {
    const int v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
    const double x0 = ref_xy[2 * v[0]], y0 = ref_xy[2 * v[0] + 1];
    const double d1x = ref_xy[2 * v[1]] - x0, d1y = ref_xy[2 * v[1] + 1] - y0;
    const double d2x = ref_xy[2 * v[2]] - x0, d2y = ref_xy[2 * v[2] + 1] - y0;
    const double det = d1x * d2y - d1y * d2x;
    if (!(det > 0)) throw std::invalid_argument("solid triangle not counter-clockwise");
    const double area = 0.5 * det;
    out.tri_area[t] = area;
    double g[3][2];
    g[1][0] = d2y / det; g[1][1] = -d2x / det;
    g[2][0] = -d1y / det; g[2][1] = d1x / det;
    g[0][0] = -(g[1][0] + g[2][0]); g[0][1] = -(g[1][1] + g[2][1]);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double* s = acc[v[a]].slot(v[b]);
        s[0] += sp.kappa * area * (g[a][0] * g[b][0] + g[a][1] * g[b][1]);
        s[1] += area / 12.0 * (a == b ? 2.0 : 1.0);
      }
  }
  if (npe == 3)
    for (int i = 0; i < n_s; ++i) acc[i].flush(S);
  out.Ssol = S;
  out.Cs = S; out.Cs.NV = 1; out.Cs.val.resize(S.nnzb());
  out.As = S; out.As.NV = 1; out.As.val.resize(S.nnzb());
  for (size_t j = 0; j < S.nnzb(); ++j) { out.As.val[j] = S.val[2 * j]; out.Cs.val[j] = S.val[2 * j + 1]; }
  out.cs_dinv.resize(2 * (size_t)n_s);
  for (int r = 0; r < n_s; ++r)
    for (int j = S.ptr[r]; j < S.ptr[r + 1]; ++j)
      if (S.col[j] == r) out.cs_dinv[2 * r] = out.cs_dinv[2 * r + 1] = 1.0 / S.val[2 * j + 1];
}

SellHost to_sell(const HostBlockMatrix& A) {
  SellHost s;
  s.nrows = A.nrows; s.BR = A.BR; s.BC = A.BC; s.NV = A.NV; s.kron = A.kron;
  s.nslices = (A.nrows + 7) / 8;
  s.soff.assign(s.nslices + 1, 0);
  s.len.assign(A.nrows, 0);
  for (int r = 0; r < A.nrows; ++r) s.len[r] = A.ptr[r + 1] - A.ptr[r];
  for (int sl = 0; sl < s.nslices; ++sl) {
    int w = 0;
    for (int r = sl * 8; r < std::min(A.nrows, sl * 8 + 8); ++r) w = std::max(w, s.len[r]);
    s.soff[sl + 1] = s.soff[sl] + 8 * w;
  }
  const size_t nslot = (size_t)s.soff[s.nslices];
  s.col.assign(nslot, 0);
  s.val.assign(nslot * s.NV, 0.0);
  for (int r = 0; r < A.nrows; ++r) {
    const int sl = r / 8, lane = r % 8;
    for (int k = 0; k < s.len[r]; ++k) {
      const size_t slot = (size_t)s.soff[sl] + (size_t)k * 8 + lane;
      const int j = A.ptr[r] + k;
      s.col[slot] = A.col[j];
      for (int v = 0; v < s.NV; ++v) s.val[slot * s.NV + v] = A.val[(size_t)j * A.NV + v];
    }
  }
  return s;
}

}  // namespace fsi
