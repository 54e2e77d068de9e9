// Host emulation of the cluster-resident coarse V-cycle (k_vcycle_cluster in
// fsi_cluster.cuh), run by tests/test_cluster_host.py without a GPU.
//
// It builds the per-CTA shared-memory images with the library's own builder
// (fsi_cluster_host.h), replays the kernel's phases on the host with every
// shared-memory, remote (distributed shared memory) and global access checked
// against the buffer it may touch, and compares the result with a plain
// per-level V-cycle on the host matrices (restriction, dense coarsest
// inverse, prolongation, Chebyshev-Jacobi smoothing in the same order).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "fsi_cluster_host.h"
#include "fsi_internal.h"

using namespace fsi;

static long n_checks = 0;
#define REQ(c)                                                       \
  do {                                                               \
    ++n_checks;                                                      \
    if (!(c)) {                                                      \
      std::printf("BOUNDS FAIL: %s (line %d)\n", #c, __LINE__);      \
      std::exit(2);                                                  \
    }                                                                \
  } while (0)

struct HostArena {
  bool count_only = false;
  std::vector<std::vector<unsigned char>> keep;
  template <class T>
  T* upload(const std::vector<T>& h) {
    keep.emplace_back(h.size() * sizeof(T));
    std::memcpy(keep.back().data(), h.data(), h.size() * sizeof(T));
    return reinterpret_cast<T*>(keep.back().data());
  }
};

struct ChebCoef {
  double c0 = 0;
  std::vector<double> c1, c2;
};

// Chebyshev semi-iteration coefficients on [lo, hi] (three-term recurrence)
static ChebCoef cheb(double lo, double hi, int k) {
  ChebCoef c;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  c.c0 = 1.0 / theta;
  double rho_old = 1.0 / sigma;
  for (int i = 1; i < k; ++i) {
    const double rho = 1.0 / (2.0 * sigma - rho_old);
    c.c1.push_back(rho * rho_old);
    c.c2.push_back(2.0 * rho / delta);
    rho_old = rho;
  }
  return c;
}

template <class T>
struct HostMG {
  struct Lv { ChebCoef ch; };
  std::vector<Lv> lv;
  T* coarse_inv = nullptr;
  int coarse_n = 0;
  int coarse_ld = 0;
  int degree = 2;
  struct {
    bool on = false;
    int lc = 0;
    size_t smem = 0;
    ClArgs<T> args;
  } cl;
};

struct Emu {
  int cs;
  size_t smem;
  std::vector<std::vector<unsigned char>> sm;
  template <class T>
  T& at(int r, int off, long idx) {
    REQ(r >= 0 && r < cs && off >= 0 && idx >= 0);
    REQ((size_t)off + (size_t)(idx + 1) * sizeof(T) <= smem);
    return *reinterpret_cast<T*>(sm[r].data() + off + idx * sizeof(T));
  }
};

// one phase of cl_phase; reads of all CTAs happen before any write (the
// kernel separates phases by cluster barriers)
template <class T>
static void phase(Emu& e, const ClMat& M, int nrows, int nsl, int col_nrows, int col_nsl, int B, bool kron, int xsrc,
                  int xown, int y, int z, int d, int dinv, int xo, T alpha, T beta, T c1, T c2, int mode,
                  int cap_row, int cap_col) {
  struct W { int r, off; long idx; T v; };
  std::vector<W> writes;
  for (int r = 0; r < e.cs; ++r) {
    int s0, s1;
    cl_own(nsl, r, e.cs, s0, s1);
    const int nown = cl_own_rows(nrows, nsl, r, e.cs);
    for (int sl = 0; sl < s1 - s0; ++sl)
      for (int lane = 0; lane < kSliceRows; ++lane) {
        const int rl = sl * kSliceRows + lane;
        if (s0 * kSliceRows + rl >= nrows) continue;
        REQ(rl < nown && rl < cap_row);
        std::vector<T> acc(B, T(0));
        const int base = e.at<int>(r, M.soff, sl) + lane;
        const int n = e.at<int>(r, M.len, rl);
        for (int k = 0; k < n; ++k) {
          const int slot = base + kSliceRows * k;
          REQ(slot >= 0 && (size_t)M.col + (size_t)(slot + 1) * sizeof(int) <= (size_t)M.val);
          const int c = e.at<int>(r, M.col, slot);
          const int owner = c >> kClColBits, loc = c & kClColMask;
          REQ(owner >= 0 && owner < e.cs);
          REQ(loc < cl_own_rows(col_nrows, col_nsl, owner, e.cs) && loc < cap_col);
          for (int i = 0; i < B; ++i) {
            if (kron) {
              acc[i] += e.at<T>(r, M.val, slot) * e.at<T>(owner, xsrc, (long)loc * B + i);
            } else {
              for (int j = 0; j < B; ++j)
                acc[i] += e.at<T>(r, M.val, (long)slot * B * B + i * B + j) * e.at<T>(owner, xsrc, (long)loc * B + j);
            }
          }
        }
        for (int i = 0; i < B; ++i) {
          const int q = rl * B + i;
          if (mode == MODE_AXPBY) {
            T out = alpha * acc[i];
            if (z >= 0) out += beta * e.at<T>(r, z, q);
            writes.push_back({r, y, q, out});
          } else if (mode == MODE_CHEB || mode == MODE_CHEB0) {
            const T res = e.at<T>(r, z, q) - acc[i];
            T dn = c2 * e.at<T>(r, dinv, q) * res;
            if (mode == MODE_CHEB) dn = c1 * e.at<T>(r, d, q) + dn;
            writes.push_back({r, d, q, dn});
            writes.push_back({r, y, q, e.at<T>(r, xown, q) + dn});
          } else {
            T tt = alpha * acc[i];
            if (z >= 0) tt += beta * e.at<T>(r, z, q);
            writes.push_back({r, y, q, tt});
            const T dn = c2 * e.at<T>(r, dinv, q) * tt;
            writes.push_back({r, d, q, dn});
            writes.push_back({r, xo, q, dn});
          }
        }
      }
  }
  for (auto& w : writes) e.at<T>(w.r, w.off, w.idx) = w.v;
}

template <class T>
static std::vector<T> emulate(const ClArgs<T>& a, size_t smem, int B, bool tkron, const std::vector<T>& in_b,
                              size_t dense_elems) {
  Emu e{a.csize, smem, std::vector<std::vector<unsigned char>>(a.csize, std::vector<unsigned char>(smem, 0xCD))};
  REQ((size_t)a.blob_bytes <= smem && a.blob_bytes % 16 == 0 && a.blob_stride * 16 >= (size_t)a.blob_bytes);
  for (int r = 0; r < a.csize; ++r)
    std::memcpy(e.sm[r].data(), reinterpret_cast<const unsigned char*>(a.blob) + (size_t)r * a.blob_stride * 16,
                a.blob_bytes);
  const int last = a.nlev - 1;
  std::vector<int> cap(a.nlev);
  for (int l = 0; l < a.nlev; ++l) {
    int mx = 0;
    for (int r = 0; r < a.csize; ++r) mx = std::max(mx, cl_own_rows(a.lv[l].nrows, a.lv[l].nsl, r, a.csize));
    cap[l] = mx;
  }
  {
    const ClLevel<T>& L = a.lv[0];
    for (int r = 0; r < a.csize; ++r) {
      int s0, s1;
      cl_own(L.nsl, r, a.csize, s0, s1);
      const int n = cl_own_rows(L.nrows, L.nsl, r, a.csize) * B;
      for (int i = 0; i < n; ++i) {
        const size_t g = (size_t)s0 * kSliceRows * B + i;
        REQ(g < in_b.size());
        const T v = in_b[g];
        e.at<T>(r, L.b, i) = v;
        const T tv = L.c0 * e.at<T>(r, L.dinv, i) * v;
        e.at<T>(r, L.x, i) = tv;
        e.at<T>(r, L.d, i) = tv;
      }
    }
  }
  std::vector<int> cur(a.nlev), oth(a.nlev);
  for (int l = 0; l < last; ++l) {
    const ClLevel<T>& L = a.lv[l];
    cur[l] = L.x;
    oth[l] = L.x2;
    for (int i = 1; i < a.degree; ++i) {
      phase<T>(e, L.A, L.nrows, L.nsl, L.nrows, L.nsl, B, false, cur[l], cur[l], oth[l], L.b, L.d, L.dinv, -1, 0, 0,
               L.c1[i - 1], L.c2[i - 1], MODE_CHEB, cap[l], cap[l]);
      std::swap(cur[l], oth[l]);
    }
    phase<T>(e, L.A, L.nrows, L.nsl, L.nrows, L.nsl, B, false, cur[l], -1, L.r, L.b, -1, -1, -1, -1, 1, 0, 0,
             MODE_AXPBY, cap[l], cap[l]);
    const ClLevel<T>& C = a.lv[l + 1];
    if (l + 1 < last)
      phase<T>(e, C.R, C.nrows, C.nsl, L.nrows, L.nsl, B, tkron, L.r, -1, C.b, -1, C.d, C.dinv, C.x, 1, 0, 0, C.c0,
               MODE_INIT, cap[l + 1], cap[l]);
    else
      phase<T>(e, C.R, C.nrows, C.nsl, L.nrows, L.nsl, B, tkron, L.r, -1, C.b, -1, -1, -1, -1, 1, 0, 0, 0, MODE_AXPBY,
               cap[l + 1], cap[l]);
  }
  {
    const ClLevel<T>& C = a.lv[last];
    const int n = a.dense_n;
    REQ(n == C.nrows * B && (size_t)n * n == dense_elems);
    std::vector<std::vector<T>> g(a.csize, std::vector<T>(n));
    for (int r = 0; r < a.csize; ++r)
      for (int i = 0; i < n; ++i) {
        const int row = i / B, comp = i - row * B;
        const int c = e.at<int>(r, a.gmap, row);
        const int owner = c >> kClColBits, loc = c & kClColMask;
        REQ(owner < a.csize && loc < cl_own_rows(C.nrows, C.nsl, owner, a.csize));
        g[r][i] = e.at<T>(owner, C.b, (long)loc * B + comp);
        e.at<T>(r, a.gbuf, i) = g[r][i];
      }
    for (int r = 0; r < a.csize; ++r) {
      int s0, s1;
      cl_own(C.nsl, r, a.csize, s0, s1);
      const int nown = cl_own_rows(C.nrows, C.nsl, r, a.csize) * B;
      for (int i = 0; i < nown; ++i) {
        const size_t row = (size_t)s0 * kSliceRows * B + i;
        REQ(row < (size_t)n);
        T s = 0;
        for (int j = 0; j < n; ++j) s += a.dense_inv[row * a.dense_ld + j] * g[r][j];
        e.at<T>(r, C.x, i) = s;
      }
    }
    cur[last] = C.x;
  }
  for (int l = last - 1; l >= 0; --l) {
    const ClLevel<T>& L = a.lv[l];
    const ClLevel<T>& C = a.lv[l + 1];
    phase<T>(e, L.P, L.nrows, L.nsl, C.nrows, C.nsl, B, tkron, cur[l + 1], -1, cur[l], cur[l], -1, -1, -1, 1, 1, 0, 0,
             MODE_AXPBY, cap[l], cap[l + 1]);
    for (int i = 0; i < a.degree; ++i) {
      if (i == 0)
        phase<T>(e, L.A, L.nrows, L.nsl, L.nrows, L.nsl, B, false, cur[l], cur[l], oth[l], L.b, L.d, L.dinv, -1, 0, 0,
                 0, L.c0, MODE_CHEB0, cap[l], cap[l]);
      else
        phase<T>(e, L.A, L.nrows, L.nsl, L.nrows, L.nsl, B, false, cur[l], cur[l], oth[l], L.b, L.d, L.dinv, -1, 0, 0,
                 L.c1[i - 1], L.c2[i - 1], MODE_CHEB, cap[l], cap[l]);
      std::swap(cur[l], oth[l]);
    }
  }
  std::vector<T> out(in_b.size(), T(0));
  const ClLevel<T>& L = a.lv[0];
  for (int r = 0; r < a.csize; ++r) {
    int s0, s1;
    cl_own(L.nsl, r, a.csize, s0, s1);
    const int n = cl_own_rows(L.nrows, L.nsl, r, a.csize) * B;
    for (int i = 0; i < n; ++i) out[(size_t)s0 * kSliceRows * B + i] = e.at<T>(r, cur[0], i);
  }
  return out;
}

// ---- reference: the per-level V-cycle on the host matrices (FP64)
static std::vector<double> mv(const HostBlockMatrix& A, const std::vector<double>& x) {
  std::vector<double> y((size_t)A.nrows * A.BR, 0.0);
  for (int r = 0; r < A.nrows; ++r)
    for (int j = A.ptr[r]; j < A.ptr[r + 1]; ++j) {
      const int c = A.col[j];
      for (int i = 0; i < A.BR; ++i) {
        if (A.kron) {
          y[(size_t)r * A.BR + i] += A.val[j] * x[(size_t)c * A.BC + i];
        } else {
          for (int k = 0; k < A.BC; ++k)
            y[(size_t)r * A.BR + i] += A.val[(size_t)j * A.NV + i * A.BC + k] * x[(size_t)c * A.BC + k];
        }
      }
    }
  return y;
}

// Gauss-Jordan inverse with partial pivoting (row-major, n x n): the dense
// coarsest solve of the reference V-cycle and of the emulated cluster
static std::vector<double> host_inverse(std::vector<double> a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)p * n + k], a[(size_t)c * n + k]);
        std::swap(inv[(size_t)p * n + k], inv[(size_t)c * n + k]);
      }
    const double piv = 1.0 / a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) { a[(size_t)c * n + k] *= piv; inv[(size_t)c * n + k] *= piv; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  return inv;
}

static std::vector<double> ref_vcycle(const HostSetup& hs, bool pr, const std::vector<double>& D,
                                      const std::vector<ChebCoef>& ch, int degree, int l, const std::vector<double>& b) {
  const int last = (int)hs.levels.size() - 1;
  const int n = (int)b.size();
  if (l == last) {
    std::vector<double> x(n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) x[i] += D[(size_t)i * n + j] * b[j];
    return x;
  }
  const FluidLevelHost& H = hs.levels[l];
  const HostBlockMatrix& A = pr ? H.L : H.A;
  const std::vector<double>& dinv = pr ? H.dinvL : H.dinvA;
  std::vector<double> x(n), d(n);
  for (int i = 0; i < n; ++i) x[i] = d[i] = ch[l].c0 * dinv[i] * b[i];
  for (int i = 1; i < degree; ++i) {
    const auto Ax = mv(A, x);
    for (int q = 0; q < n; ++q) {
      d[q] = ch[l].c1[i - 1] * d[q] + ch[l].c2[i - 1] * dinv[q] * (b[q] - Ax[q]);
      x[q] += d[q];
    }
  }
  const auto Ax = mv(A, x);
  std::vector<double> r(n);
  for (int q = 0; q < n; ++q) r[q] = b[q] - Ax[q];
  const auto xc = ref_vcycle(hs, pr, D, ch, degree, l + 1, mv(pr ? H.Rp : H.Ru, r));
  const auto Px = mv(pr ? H.Pp : H.Pu, xc);
  for (int q = 0; q < n; ++q) x[q] += Px[q];
  for (int i = 0; i < degree; ++i) {
    const auto Ax2 = mv(A, x);
    for (int q = 0; q < n; ++q) {
      const double res = b[q] - Ax2[q];
      d[q] = (i == 0) ? ch[l].c0 * dinv[q] * res : ch[l].c1[i - 1] * d[q] + ch[l].c2[i - 1] * dinv[q] * res;
      x[q] += d[q];
    }
  }
  return x;
}

template <class T>
static int run_case(const HostSetup& hs, int N, bool pr, int cs, int degree, size_t cap, double tol) {
  const int nl = (int)hs.levels.size();
  HostMG<T> mg;
  mg.degree = degree;
  mg.lv.resize(nl);
  std::vector<ChebCoef> ch(nl);
  for (int l = 0; l < nl; ++l) {
    const double hi = 1.05 * (pr ? hs.levels[l].lmaxL : hs.levels[l].lmaxA);
    ch[l] = cheb(hi / (pr ? 8.0 : 6.0), hi, degree);
    mg.lv[l].ch = ch[l];
  }
  mg.coarse_n = pr ? hs.coarse_nL : hs.coarse_nA;
  mg.coarse_ld = mg.coarse_n;
  const std::vector<double> D = host_inverse(pr ? hs.coarseL : hs.coarseA, mg.coarse_n);
  std::vector<T> dense(D.begin(), D.end());
  mg.coarse_inv = dense.data();
  HostArena ar;
  if (!build_cluster<T>(ar, hs, pr, mg, cs, cap, [](size_t) { return true; })) {
    std::printf("N=%d %s cs=%d: no cluster suffix fits\n", N, pr ? "P" : "U", cs);
    return 0;
  }
  const int lc = mg.cl.lc;
  const int B = pr ? 3 : 2;
  const HostBlockMatrix& Alc = pr ? hs.levels[lc].L : hs.levels[lc].A;
  std::vector<double> b((size_t)Alc.nrows * B);
  std::mt19937_64 rng(N * 7 + pr);
  std::normal_distribution<double> nd;
  for (auto& v : b) v = nd(rng);
  std::vector<T> bt(b.begin(), b.end());
  const auto xe = emulate<T>(mg.cl.args, mg.cl.smem, B, !pr, bt, dense.size());
  const auto xr = ref_vcycle(hs, pr, D, ch, degree, lc, b);
  double num = 0, den = 0;
  for (size_t i = 0; i < xr.size(); ++i) {
    num += ((double)xe[i] - xr[i]) * ((double)xe[i] - xr[i]);
    den += xr[i] * xr[i];
  }
  const double rel = std::sqrt(num / den);
  std::printf("N=%d %s %s cs=%d degree=%d levels %d..%d smem=%zu rel=%.2e\n", N, pr ? "P" : "U",
              sizeof(T) == 8 ? "f64" : "f32", cs, degree, lc, nl - 1, mg.cl.smem, rel);
  return rel <= tol ? 0 : 1;
}

int main() {
  int failures = 0;
  const size_t cap = 227 * 1024;
  for (int N : {16, 24, 96, 128}) {
    SetupParams sp{N, 1.0, 0.01, 1e3, 1e-3, 1.0};
    const std::vector<double> xy = {0.4, 0.4, 0.6, 0.4, 0.5, 0.6};
    const std::vector<int> tris = {0, 1, 2};
    HostSetup hs;
    build_setup(sp, 3, 1, xy.data(), tris.data(), hs);
    for (int pr = 0; pr < 2; ++pr)
      for (int cs : {16, 8}) {
        failures += run_case<double>(hs, N, pr, cs, 2, 2 * cap, 1e-12);
        failures += run_case<float>(hs, N, pr, cs, 2, cap, 1e-5);
        if (N == 24) failures += run_case<double>(hs, N, pr, cs, 3, 2 * cap, 1e-12);
      }
  }
  std::printf("checks=%ld failures=%d\n", n_checks, failures);
  return failures ? 1 : 0;
}
