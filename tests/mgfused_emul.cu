// Host run of the fused matrix-free multigrid kernels (fsi_mgfused.cuh),
// called by tests/test_mgfused_host.py without a GPU.
//
// The kernel bodies are __host__ __device__: here every CTA of a launch is
// run by one host thread (the bodies' loops are strided over the CTA's
// threads and separated by barriers, so one thread computes the same
// values).  Each launch is compared with the same step written on the
// assembled level matrices of the library's host setup (A, L, and the
// transfer matrices P, R = P^T), in double precision:
//   down: x0 = c0 D^-1 b, K - 1 Chebyshev steps, r = b - A x, b_c = R r
//         (and the coarse smoother start x_c = d_c = c0_c D_c^-1 b_c);
//   up:   x = x_pre + P x_c, CHEB0 then K - 1 Chebyshev steps, with the
//         Richardson and Cahouet-Chabard epilogues.
// The FP64 instantiation must agree to 1e-12; the FP32 one to 1e-5 (the
// residual b - A x cancels: its FP32 rounding error is about 50 unit
// roundoffs of its size on these levels).
// Built with AddressSanitizer, every shared-memory frame is its own heap
// block of exactly the launch's size, so an access outside it aborts.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "fsi_internal.h"
#include "fsi_mgfused.cuh"

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

struct Coef {
  double c0 = 0;
  std::vector<double> c1, c2;
};

// Chebyshev three-term coefficients on [lo, hi]
static Coef cheb(double lo, double hi, int k) {
  Coef c;
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

static double rel(const std::vector<double>& a, const std::vector<double>& b) {
  double num = 0, den = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    num += (a[i] - b[i]) * (a[i] - b[i]);
    den += b[i] * b[i];
  }
  return std::sqrt(num / (den > 0 ? den : 1.0));
}

template <class T>
static std::vector<T> as(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}
template <class T>
static std::vector<double> back(const std::vector<T>& v) {
  return std::vector<double>(v.begin(), v.end());
}

// run every CTA of a grid (vthr threads per CTA on the device) by one host
// thread, each with its own exactly sized frame
template <class Body>
static void run_grid(int gx, int gy, int vthr, size_t smem, Body body) {
  for (int by = 0; by < gy; ++by)
    for (int bx = 0; bx < gx; ++bx) {
      std::vector<unsigned char>* buf = new std::vector<unsigned char>(smem);
      std::memset(buf->data(), 0xA5, smem);  // stale data: every read must be of a written entry
      const MfCta c{bx, by, 0, 1, vthr, buf->data()};
      body(c);
      delete buf;
    }
}

static int failures = 0;

static void report(const char* what, int N, int K, int level, double err, double tol) {
  const bool ok = err <= tol;
  if (!ok) ++failures;
  std::printf("{\"check\": \"%s\", \"N\": %d, \"K\": %d, \"level\": %d, \"rel_err\": %.3e, \"ok\": %s}\n", what, N, K,
              level, err, ok ? "true" : "false");
}

template <class T>
static void velocity(const HostSetup& hs, int l, int K, double tol, std::mt19937_64& rng) {
  const FluidLevelHost& H = hs.levels[l];
  const FluidLevelHost& Hc = hs.levels[l + 1];
  const int N = H.N, n = 2 * H.A.nrows, nc = 2 * Hc.A.nrows;
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<double> b(n), xpre(n), xc(nc), acc0(n), dinvc(nc);
  for (double& v : b) v = U(rng);
  for (double& v : xpre) v = U(rng);
  for (double& v : xc) v = U(rng);
  for (double& v : acc0) v = U(rng);
  const Coef ch = cheb(0.3, 2.1, K);
  MfVelArgs<T> a;
  a.op.N = N;
  for (int t = 0; t < 4; ++t) {
    for (int y = 0; y < 5; ++y)
      for (int x = 0; x < 5; ++x)
        for (int q = 0; q < 4; ++q) a.op.c[t][y][x][q] = (T)H.stenA[t][y][x][q];
    for (int c = 0; c < 2; ++c) a.op.dinv[t][c] = (T)H.dinvAt[t][c];
  }
  a.ch.k = K;
  a.ch.c0 = (T)ch.c0;
  for (int i = 0; i + 1 < K; ++i) { a.ch.c1[i] = (T)ch.c1[i]; a.ch.c2[i] = (T)ch.c2[i]; }
  // ---------------------------------------------------------------- down
  std::vector<T> bT = as<T>(b), xout(n, (T)7), bc(nc, (T)7), cix(nc, (T)7), cid(nc, (T)7);
  std::vector<T> dcT = as<T>(Hc.dinvA);
  const double c0c = 0.37;
  a.b = bT.data(); a.xout = xout.data(); a.bc = bc.data();
  a.ci.x = cix.data(); a.ci.d = cid.data(); a.ci.dinv = dcT.data(); a.ci.c0 = (T)c0c;
  mf_with_tile_u(N, [&](auto tc) {   // the tile the library uses on this level
    constexpr int TC = decltype(tc)::value;
    const int gd = (N + TC - 1) / TC;
    mf_with_degree(K, [&](auto kc) {
      constexpr int KD = decltype(kc)::value;
      run_grid(gd, gd, mf_threads_ud(TC), mfu_down_smem<T>(TC, KD), [&](const MfCta& c) { mfu_down_body<T, TC, KD>(a, c); });
    });
  });
  // reference: smoothing from x0 = c0 D^-1 b, then residual and restriction
  std::vector<double> x(n), d(n), Ax, r(n), Rr, xr;
  for (int i = 0; i < n; ++i) x[i] = d[i] = ch.c0 * H.dinvA[i] * b[i];
  for (int s = 1; s < K; ++s) {
    spmv(H.A, x, Ax);
    for (int i = 0; i < n; ++i) {
      d[i] = ch.c1[s - 1] * d[i] + ch.c2[s - 1] * H.dinvA[i] * (b[i] - Ax[i]);
      x[i] += d[i];
    }
  }
  spmv(H.A, x, Ax);
  for (int i = 0; i < n; ++i) r[i] = b[i] - Ax[i];
  spmv(H.Ru, r, Rr);
  report("velocity down: pre-smoothed iterate", N, K, l, rel(back(xout), x), tol);
  report("velocity down: restricted residual", N, K, l, rel(back(bc), Rr), tol);
  std::vector<double> ci_ref(nc);
  for (int i = 0; i < nc; ++i) ci_ref[i] = c0c * Hc.dinvA[i] * Rr[i];
  report("velocity down: coarse smoother start", N, K, l, std::max(rel(back(cix), ci_ref), rel(back(cid), ci_ref)),
         tol);
  // ------------------------------------------------------------------ up
  std::vector<T> xpT = as<T>(xpre), xcT = as<T>(xc), out(n, (T)7), accT = as<T>(acc0);
  MfVelArgs<T> u = a;
  u.ci = MfInit<T>();
  u.b = bT.data(); u.xpre = xpT.data(); u.xc = xcT.data(); u.xout = out.data(); u.bc = nullptr;
  u.fin.acc = accT.data(); u.fin.omega = (T)0.8;
  mf_with_tile_u(N, [&](auto tc) {
    constexpr int TC = decltype(tc)::value;
    const int gu = (2 * N + 2 * TC - 1) / (2 * TC);
    mf_with_degree(K, [&](auto kc) {
      constexpr int KD = decltype(kc)::value;
      run_grid(gu, gu, mf_threads_uu(TC), mfu_up_smem<T>(TC, KD), [&](const MfCta& c) { mfu_up_body<T, TC, KD>(u, c); });
    });
  });
  std::vector<double> Pxc;
  spmv(H.Pu, xc, Pxc);
  for (int i = 0; i < n; ++i) x[i] = xpre[i] + Pxc[i];
  for (int s = 0; s < K; ++s) {
    spmv(H.A, x, Ax);
    for (int i = 0; i < n; ++i) {
      const double res = b[i] - Ax[i];
      d[i] = (s == 0) ? ch.c0 * H.dinvA[i] * res : ch.c1[s - 1] * d[i] + ch.c2[s - 1] * H.dinvA[i] * res;
      x[i] += d[i];
    }
  }
  std::vector<double> acc_ref(n);
  for (int i = 0; i < n; ++i) acc_ref[i] = acc0[i] + 0.8 * x[i];
  report("velocity up: post-smoothed result", N, K, l, rel(back(out), x), tol);
  report("velocity up: Richardson update", N, K, l, rel(back(accT), acc_ref), tol);
  if (l != 0) return;
  // -------------------------------- down with the Stokes residual start
  // b = r - A zu - (-B^T) zp on the finest level, against the assembled
  // A_f and -B^T; then the same smoothing, residual and restriction
  const int np = 3 * N * N;
  std::vector<double> zu(n), zp(np);
  for (double& v : zu) v = U(rng);
  for (double& v : zp) v = U(rng);
  std::vector<double> Az, Btz, bres(n);
  spmv(H.A, zu, Az);
  spmv(hs.Bt, zp, Btz);
  for (int i = 0; i < n; ++i) bres[i] = b[i] - Az[i] - Btz[i];
  std::vector<T> zuT = as<T>(zu), zpT = as<T>(zp), bout(n, (T)7), xout2(n, (T)7), bc2(nc, (T)7);
  MfVelArgs<T> w = a;
  w.ci = MfInit<T>();
  w.b = bT.data(); w.xout = xout2.data(); w.bc = bc2.data();
  w.res.zu = zuT.data(); w.res.zp = zpT.data(); w.res.bout = bout.data();
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 9; ++q)
      for (int c = 0; c < 2; ++c) w.res.divB[k][q][c] = (T)H.divB[k][q][c];
  mf_with_tile_u(N, [&](auto tc) {
    constexpr int TC = decltype(tc)::value;
    const int gd = (N + TC - 1) / TC;
    mf_with_degree(K, [&](auto kc) {
      constexpr int KD = decltype(kc)::value;
      run_grid(gd, gd, mf_threads_ud(TC), mfu_down_smem<T>(TC, KD), [&](const MfCta& c) { mfu_down_body<T, TC, KD>(w, c); });
    });
  });
  for (int i = 0; i < n; ++i) x[i] = d[i] = ch.c0 * H.dinvA[i] * bres[i];
  for (int s = 1; s < K; ++s) {
    spmv(H.A, x, Ax);
    for (int i = 0; i < n; ++i) {
      d[i] = ch.c1[s - 1] * d[i] + ch.c2[s - 1] * H.dinvA[i] * (bres[i] - Ax[i]);
      x[i] += d[i];
    }
  }
  spmv(H.A, x, Ax);
  for (int i = 0; i < n; ++i) r[i] = bres[i] - Ax[i];
  spmv(H.Ru, r, Rr);
  report("velocity down, residual start: right-hand side", N, K, l, rel(back(bout), bres), tol);
  report("velocity down, residual start: pre-smoothed iterate", N, K, l, rel(back(xout2), x), tol);
  report("velocity down, residual start: restricted residual", N, K, l, rel(back(bc2), Rr), tol);
  // zu absent (the first Stokes application): b = r - (-B^T) zp
  std::vector<T> bout3(n, (T)7);
  w.res.zu = nullptr;
  w.res.bout = bout3.data();
  mf_with_tile_u(N, [&](auto tc) {
    constexpr int TC = decltype(tc)::value;
    const int gd = (N + TC - 1) / TC;
    mf_with_degree(K, [&](auto kc) {
      constexpr int KD = decltype(kc)::value;
      run_grid(gd, gd, mf_threads_ud(TC), mfu_down_smem<T>(TC, KD), [&](const MfCta& c) { mfu_down_body<T, TC, KD>(w, c); });
    });
  });
  for (int i = 0; i < n; ++i) bres[i] = b[i] - Btz[i];
  report("velocity down, pressure only: right-hand side", N, K, l, rel(back(bout3), bres), tol);
}

template <class T>
static void pressure(const HostSetup& hs, int l, int K, double tol, std::mt19937_64& rng) {
  const FluidLevelHost& H = hs.levels[l];
  const FluidLevelHost& Hc = hs.levels[l + 1];
  const int N = H.N, n = 3 * N * N, nc = 3 * Hc.N * Hc.N;
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<double> b(n), xpre(n), xc(nc), acc0(n), sv(n), smp(n);
  for (double& v : b) v = U(rng);
  for (double& v : xpre) v = U(rng);
  for (double& v : xc) v = U(rng);
  for (double& v : acc0) v = U(rng);
  for (double& v : sv) v = U(rng);
  for (double& v : smp) v = 1.5 + U(rng);
  const Coef ch = cheb(0.2, 2.4, K);
  std::vector<double> tab(kMfPresTab);
  for (int v = 0; v < 9; ++v)
    for (int y = 0; y < 3; ++y)
      for (int x = 0; x < 3; ++x)
        for (int q = 0; q < 9; ++q) tab[mf_pres_blk(v, y, x) + q] = H.stenL[v][y][x][q];
  for (int v = 0; v < 9; ++v)
    for (int k = 0; k < 3; ++k) tab[kMfPresDinv + 3 * v + k] = H.dinvLv[v][k];
  std::vector<T> tabT = as<T>(tab);
  MfPresArgs<T> a;
  a.N = N;
  a.tab = tabT.data();
  a.ch.k = K;
  a.ch.c0 = (T)ch.c0;
  for (int i = 0; i + 1 < K; ++i) { a.ch.c1[i] = (T)ch.c1[i]; a.ch.c2[i] = (T)ch.c2[i]; }
  std::vector<T> bT = as<T>(b), xout(n, (T)7), bc(nc, (T)7), cix(nc, (T)7), cid(nc, (T)7);
  std::vector<T> dcT = as<T>(Hc.dinvL);
  const double c0c = 0.41;
  a.b = bT.data(); a.xout = xout.data(); a.bc = bc.data();
  a.ci.x = cix.data(); a.ci.d = cid.data(); a.ci.dinv = dcT.data(); a.ci.c0 = (T)c0c;
  mf_with_tile_p(N, [&](auto tp) {
    constexpr int TP = decltype(tp)::value;
    const int gd = (N / 2 + TP - 1) / TP;
    mf_with_degree(K, [&](auto kc) {
      constexpr int KD = decltype(kc)::value;
      run_grid(gd, gd, mf_threads_p(TP), mfp_down_smem<T>(TP, KD), [&](const MfCta& c) { mfp_down_body<T, TP, KD>(a, c); });
    });
  });
  std::vector<double> x(n), d(n), Lx, r(n), Rr;
  for (int i = 0; i < n; ++i) x[i] = d[i] = ch.c0 * H.dinvL[i] * b[i];
  for (int s = 1; s < K; ++s) {
    spmv(H.L, x, Lx);
    for (int i = 0; i < n; ++i) {
      d[i] = ch.c1[s - 1] * d[i] + ch.c2[s - 1] * H.dinvL[i] * (b[i] - Lx[i]);
      x[i] += d[i];
    }
  }
  spmv(H.L, x, Lx);
  for (int i = 0; i < n; ++i) r[i] = b[i] - Lx[i];
  spmv(H.Rp, r, Rr);
  report("pressure down: pre-smoothed iterate", N, K, l, rel(back(xout), x), tol);
  report("pressure down: restricted residual", N, K, l, rel(back(bc), Rr), tol);
  std::vector<double> ci_ref(nc);
  for (int i = 0; i < nc; ++i) ci_ref[i] = c0c * Hc.dinvL[i] * Rr[i];
  report("pressure down: coarse smoother start", N, K, l, std::max(rel(back(cix), ci_ref), rel(back(cid), ci_ref)),
         tol);
  // up with the Cahouet-Chabard epilogue s = -(nu mp sv + (rho/dt) y), acc += omega s
  std::vector<T> xpT = as<T>(xpre), xcT = as<T>(xc), out(n, (T)7), accT = as<T>(acc0), svT = as<T>(sv),
                 smpT = as<T>(smp), sout(n, (T)7);
  MfPresArgs<T> u = a;
  u.ci = MfInit<T>();
  u.b = bT.data(); u.xpre = xpT.data(); u.xc = xcT.data(); u.xout = out.data(); u.bc = nullptr;
  u.fin.sv = svT.data(); u.fin.smp = smpT.data(); u.fin.sout = sout.data();
  u.fin.snu = (T)0.07; u.fin.srdt = (T)325.0; u.fin.acc = accT.data(); u.fin.omega = (T)0.9;
  mf_with_tile_p(N, [&](auto tp) {
    constexpr int TP = decltype(tp)::value;
    const int gu = (N + 2 * TP - 1) / (2 * TP);
    mf_with_degree(K, [&](auto kc) {
      constexpr int KD = decltype(kc)::value;
      run_grid(gu, gu, mf_threads_p(TP), mfp_up_smem<T>(TP, KD), [&](const MfCta& c) { mfp_up_body<T, TP, KD>(u, c); });
    });
  });
  std::vector<double> Pxc;
  spmv(H.Pp, xc, Pxc);
  for (int i = 0; i < n; ++i) x[i] = xpre[i] + Pxc[i];
  for (int s = 0; s < K; ++s) {
    spmv(H.L, x, Lx);
    for (int i = 0; i < n; ++i) {
      const double res = b[i] - Lx[i];
      d[i] = (s == 0) ? ch.c0 * H.dinvL[i] * res : ch.c1[s - 1] * d[i] + ch.c2[s - 1] * H.dinvL[i] * res;
      x[i] += d[i];
    }
  }
  std::vector<double> s_ref(n), acc_ref(n);
  for (int i = 0; i < n; ++i) {
    s_ref[i] = -(0.07 * smp[i] * sv[i] + 325.0 * x[i]);
    acc_ref[i] = acc0[i] + 0.9 * s_ref[i];
  }
  report("pressure up: post-smoothed result", N, K, l, rel(back(out), x), tol);
  report("pressure up: Cahouet-Chabard combination", N, K, l, rel(back(sout), s_ref), tol);
  report("pressure up: Richardson update", N, K, l, rel(back(accT), acc_ref), tol);
  if (l != 0) return;
  // -------------------------------- down with the Stokes residual start
  // b = r - (-B) zu on the finest level, against the assembled -B
  const int nu = 2 * hs.Bt.nrows;
  std::vector<double> zu(nu), Bz, bres(n);
  for (double& v : zu) v = U(rng);
  spmv(hs.Bneg, zu, Bz);
  for (int i = 0; i < n; ++i) bres[i] = b[i] - Bz[i];
  std::vector<T> zuT = as<T>(zu), bout(n, (T)7), xout2(n, (T)7), bc2(nc, (T)7);
  MfPresArgs<T> w = a;
  w.ci = MfInit<T>();
  w.b = bT.data(); w.xout = xout2.data(); w.bc = bc2.data();
  w.res.zu = zuT.data(); w.res.bout = bout.data();
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 9; ++q)
      for (int c = 0; c < 2; ++c) w.res.divB[k][q][c] = (T)H.divB[k][q][c];
  mf_with_tile_p(N, [&](auto tp) {
    constexpr int TP = decltype(tp)::value;
    const int gd = (N / 2 + TP - 1) / TP;
    mf_with_degree(K, [&](auto kc) {
      constexpr int KD = decltype(kc)::value;
      run_grid(gd, gd, mf_threads_p(TP), mfp_down_smem<T>(TP, KD), [&](const MfCta& c) { mfp_down_body<T, TP, KD>(w, c); });
    });
  });
  for (int i = 0; i < n; ++i) x[i] = d[i] = ch.c0 * H.dinvL[i] * bres[i];
  for (int s = 1; s < K; ++s) {
    spmv(H.L, x, Lx);
    for (int i = 0; i < n; ++i) {
      d[i] = ch.c1[s - 1] * d[i] + ch.c2[s - 1] * H.dinvL[i] * (bres[i] - Lx[i]);
      x[i] += d[i];
    }
  }
  spmv(H.L, x, Lx);
  for (int i = 0; i < n; ++i) r[i] = bres[i] - Lx[i];
  spmv(H.Rp, r, Rr);
  report("pressure down, residual start: right-hand side", N, K, l, rel(back(bout), bres), tol);
  report("pressure down, residual start: pre-smoothed iterate", N, K, l, rel(back(xout2), x), tol);
  report("pressure down, residual start: restricted residual", N, K, l, rel(back(bc2), Rr), tol);
}

int main(int argc, char** argv) {
  std::vector<int> grids{16, 24, 48, 128, 512};
  if (argc > 1) {
    grids.clear();
    for (int i = 1; i < argc; ++i) grids.push_back(std::atoi(argv[i]));
  }
  std::mt19937_64 rng(11);
  for (int N : grids) {
    const double xy[6] = {0.4, 0.4, 0.6, 0.4, 0.5, 0.6};
    const int tris[3] = {0, 1, 2};
    SetupParams sp{N, 1.3, 0.07, 10.0, 0.004, 1.0};
    HostSetup hs;
    build_setup(sp, 3, 1, xy, tris, hs);
    for (int l = 0; l + 1 < (int)hs.levels.size() && l < 2; ++l) {
      if (!hs.levels[l].mf) continue;
      for (int K = 1; K <= kMfMaxDeg; ++K) {
        if (N > 48 && K != 2) continue;  // the largest grids only at the default degree
        if (N > 128 && l > 0) continue;
        velocity<double>(hs, l, K, 1e-12, rng);
        pressure<double>(hs, l, K, 1e-12, rng);
        velocity<float>(hs, l, K, 1e-5, rng);
        pressure<float>(hs, l, K, 1e-5, rng);
      }
    }
  }
  std::printf("failures=%d\n", failures);
  return failures ? 1 : 0;
}
