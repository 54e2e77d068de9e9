// Host-only checks of the library's setup code (fsi_setup.cpp), run by
// tests/test_setup_host.py without a GPU.
//
//   setup_harness products N
//     for every pressure level with a fused restriction, the product R L
//     applied to a random vector against R applied to L x (one line per
//     level: {"level": l, "rel_err": e});
//   setup_harness stencils N
//     every row of the assembled level operators against their matrix-free
//     stencils, and the finest -B and -B^T against the divergence table (one
//     line per level);
//   setup_harness levels N cu cp
//     the velocity and pressure hierarchies for coarsest-grid limits cu, cp;
//   setup_harness solid <mesh file> <kappa>
//     build the solid operators of a Q1 mesh (file: n_nodes n_el, then x y
//     per node, then 4 node ids per element) and print C_s and A_s as
//     triplets and the Chebyshev interval of D^-1 C_s, as one JSON object.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "fsi_internal.h"

using namespace fsi;

static void spmv(const HostBlockMatrix& A, const std::vector<double>& x, std::vector<double>& y) {
  y.assign((size_t)A.nrows * A.BR, 0.0);
  for (int r = 0; r < A.nrows; ++r)
    for (int j = A.ptr[r]; j < A.ptr[r + 1]; ++j) {
      const int c = A.col[j];
      for (int i = 0; i < A.BR; ++i)
        for (int k = 0; k < A.BC; ++k) {
          const double v = A.kron ? (i == k ? A.val[j] : 0.0) : A.val[(size_t)j * A.NV + i * A.BC + k];
          y[(size_t)r * A.BR + i] += v * x[(size_t)c * A.BC + k];
        }
    }
}

static int products(int N) {
  // a small solid inside the domain: the fluid hierarchy does not depend on it
  const double xy[6] = {0.4, 0.4, 0.6, 0.4, 0.5, 0.6};
  const int tris[3] = {0, 1, 2};
  SetupParams sp{N, 1.0, 0.1, 10.0, 0.01, 0.0};
  HostSetup hs;
  build_setup(sp, 3, 1, xy, tris, hs);
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (size_t l = 0; l + 1 < hs.levels.size(); ++l) {
    const FluidLevelHost& L = hs.levels[l];
    std::vector<double> x((size_t)L.L.ncols * L.L.BC), Lx, RLx, fused;
    for (double& v : x) v = U(rng);
    spmv(L.L, x, Lx);
    spmv(L.Rp, Lx, RLx);
    spmv(L.RAp, x, fused);
    double num = 0, den = 0;
    for (size_t i = 0; i < RLx.size(); ++i) {
      num += (fused[i] - RLx[i]) * (fused[i] - RLx[i]);
      den += RLx[i] * RLx[i];
    }
    std::printf("{\"level\": %zu, \"rows\": %d, \"rel_err\": %.3e}\n", l, L.RAp.nrows, std::sqrt(num / den));
  }
  return 0;
}

static void triplets(const char* name, const HostBlockMatrix& A) {
  std::printf("\"%s\": [", name);
  bool first = true;
  for (int r = 0; r < A.nrows; ++r)
    for (int j = A.ptr[r]; j < A.ptr[r + 1]; ++j) {
      std::printf("%s[%d, %d, %.17g]", first ? "" : ", ", r, A.col[j], A.val[j]);
      first = false;
    }
  std::printf("]");
}

static int solid(const char* path, double kappa) {
  FILE* f = std::fopen(path, "r");
  if (!f) return 2;
  int ns = 0, ne = 0;
  if (std::fscanf(f, "%d %d", &ns, &ne) != 2) return 2;
  std::vector<double> xy(2 * (size_t)ns);
  std::vector<int> el(4 * (size_t)ne);
  for (double& v : xy)
    if (std::fscanf(f, "%lf", &v) != 1) return 2;
  for (int& v : el)
    if (std::fscanf(f, "%d", &v) != 1) return 2;
  std::fclose(f);
  SetupParams sp{8, 1.0, 0.1, kappa, 0.01, 0.0};
  sp.npe = 4;
  HostSetup hs;
  build_setup(sp, ns, ne, xy.data(), el.data(), hs);
  std::printf("{");
  triplets("Cs", hs.Cs);
  std::printf(", ");
  triplets("As", hs.As);
  std::printf(", \"cs_lo\": %.17g, \"cs_hi\": %.17g}\n", hs.cs_lo, hs.cs_hi);
  return 0;
}

// Every row of the assembled A and L of every level against the matrix-free
// stencils of that level: same blocks bit for bit, and no stored block the
// stencil lacks.  One line per level: {"level", "N", "a_mismatch",
// "l_mismatch", "a_rows", "l_rows"}.
static int stencils(int N) {
  const double xy[6] = {0.4, 0.4, 0.6, 0.4, 0.5, 0.6};
  const int tris[3] = {0, 1, 2};
  SetupParams sp{N, 1.3, 0.07, 10.0, 0.004, 1.0};
  HostSetup hs;
  build_setup(sp, 3, 1, xy, tris, hs);
  for (size_t l = 0; l < hs.levels.size(); ++l) {
    const FluidLevelHost& L = hs.levels[l];
    if (!L.mf) continue;
    VNum vn(L.N);
    long a_bad = 0, l_bad = 0;
    for (int r = 0; r < L.A.nrows; ++r) {
      int ix, iy;
      vn.lattice(r, ix, iy);
      const int tau = (ix & 1) | ((iy & 1) << 1);
      int expect = 0;  // stencil blocks whose neighbour is interior
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          const double* c = L.stenA[tau][dy + 2][dx + 2];
          if ((c[0] != 0 || c[1] != 0 || c[2] != 0 || c[3] != 0) && vn.id(ix + dx, iy + dy) >= 0) ++expect;
        }
      if (L.A.ptr[r + 1] - L.A.ptr[r] != expect) ++a_bad;
      for (int j = L.A.ptr[r]; j < L.A.ptr[r + 1]; ++j) {
        int jx, jy;
        vn.lattice(L.A.col[j], jx, jy);
        const int dx = jx - ix, dy = jy - iy;
        bool ok = dx >= -2 && dx <= 2 && dy >= -2 && dy <= 2;
        for (int q = 0; ok && q < 4; ++q) ok = L.A.val[4 * (size_t)j + q] == L.stenA[tau][dy + 2][dx + 2][q];
        if (!ok) ++a_bad;
      }
      for (int i = 0; i < 2; ++i)
        if (L.dinvA[2 * (size_t)r + i] != L.dinvAt[tau][i]) ++a_bad;
    }
    for (int r = 0; r < L.L.nrows; ++r) {
      const int cx = r % L.N, cy = r / L.N;
      const int vx = cx == 0 ? 0 : (cx == L.N - 1 ? 2 : 1), vy = cy == 0 ? 0 : (cy == L.N - 1 ? 2 : 1);
      const int v = 3 * vy + vx;
      int expect = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          bool nz = false;
          for (int q = 0; q < 9; ++q) nz = nz || L.stenL[v][dy + 1][dx + 1][q] != 0;
          if (nz && cx + dx >= 0 && cx + dx < L.N && cy + dy >= 0 && cy + dy < L.N) ++expect;
        }
      if (L.L.ptr[r + 1] - L.L.ptr[r] != expect) ++l_bad;
      for (int j = L.L.ptr[r]; j < L.L.ptr[r + 1]; ++j) {
        const int c2 = L.L.col[j], dx = c2 % L.N - cx, dy = c2 / L.N - cy;
        bool ok = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
        for (int q = 0; ok && q < 9; ++q) ok = L.L.val[9 * (size_t)j + q] == L.stenL[v][dy + 1][dx + 1][q];
        if (!ok) ++l_bad;
      }
      for (int i = 0; i < 3; ++i)
        if (L.dinvL[3 * (size_t)r + i] != L.dinvLv[v][i]) ++l_bad;
    }
    // the finest level's divergence table against -B (cell rows) and -B^T
    // (node rows) of the finest grid, entry for entry
    long b_bad = 0;
    if (l == 0) {
      for (int c = 0; c < hs.Bneg.nrows; ++c) {
        const int cx = c % L.N, cy = c / L.N;
        for (int j = hs.Bneg.ptr[c]; j < hs.Bneg.ptr[c + 1]; ++j) {
          int jx, jy;
          vn.lattice(hs.Bneg.col[j], jx, jy);
          const int al = (jy - 2 * cy) * 3 + (jx - 2 * cx);
          for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 2; ++d)
              if (al < 0 || al > 8 || hs.Bneg.val[6 * (size_t)j + 2 * k + d] != L.divB[k][al][d]) ++b_bad;
        }
      }
      for (int r = 0; r < hs.Bt.nrows; ++r) {
        int ix, iy;
        vn.lattice(r, ix, iy);
        for (int j = hs.Bt.ptr[r]; j < hs.Bt.ptr[r + 1]; ++j) {
          const int c = hs.Bt.col[j], cx = c % L.N, cy = c / L.N;
          const int al = (iy - 2 * cy) * 3 + (ix - 2 * cx);
          for (int d = 0; d < 2; ++d)
            for (int k = 0; k < 3; ++k)
              if (al < 0 || al > 8 || hs.Bt.val[6 * (size_t)j + 3 * d + k] != L.divB[k][al][d]) ++b_bad;
        }
      }
    }
    std::printf("{\"level\": %zu, \"N\": %d, \"a_mismatch\": %ld, \"l_mismatch\": %ld, \"b_mismatch\": %ld, "
                "\"a_rows\": %d, \"l_rows\": %d}\n", l, L.N, a_bad, l_bad, b_bad, L.A.nrows, L.L.nrows);
  }
  return 0;
}

// The two hierarchies of grid N with coarse_max cu and coarse_max_p cp: the
// grid sides of all levels, the level counts of each hierarchy and the sizes
// of the dense coarsest matrices, as one JSON object.
static int levels(int N, int cu, int cp) {
  const double xy[6] = {0.4, 0.4, 0.6, 0.4, 0.5, 0.6};
  const int tris[3] = {0, 1, 2};
  SetupParams sp{N, 1.0, 0.1, 10.0, 0.01, 0.0};
  sp.coarse_max = cu;
  sp.coarse_max_p = cp;
  HostSetup hs;
  build_setup(sp, 3, 1, xy, tris, hs);
  std::printf("{\"Ns\": [");
  for (size_t l = 0; l < hs.levels.size(); ++l) std::printf("%s%d", l ? ", " : "", hs.levels[l].N);
  std::printf("], \"nlev_u\": %d, \"nlev_p\": %d, \"coarse_nA\": %d, \"coarse_nL\": %d, "
              "\"dense_A\": %zu, \"dense_L\": %zu}\n", hs.nlev_u, hs.nlev_p, hs.coarse_nA, hs.coarse_nL,
              hs.coarseA.size(), hs.coarseL.size());
  return 0;
}

int main(int argc, char** argv) {
  if (argc >= 3 && std::string(argv[1]) == "stencils") return stencils(std::atoi(argv[2]));
  if (argc >= 3 && std::string(argv[1]) == "products") return products(std::atoi(argv[2]));
  if (argc >= 5 && std::string(argv[1]) == "levels")
    return levels(std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]));
  if (argc >= 4 && std::string(argv[1]) == "solid") return solid(argv[2], std::atof(argv[3]));
  std::fprintf(stderr, "usage: setup_harness products N | solid mesh kappa\n");
  return 1;
}
