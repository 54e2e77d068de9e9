// Nonlinear solid law (the bar test of Section 6): tangent stiffness and
// Newton right-hand side of the exponential strain energy
//   W(F) = (gamma / (2 eta)) exp(eta (tr F^T F - 2)),  P = dW/dF = e F,
//   e = gamma exp(eta (|F|^2 - 2)).
// With P1 elements F is constant on every triangle E.  The solid row of
// Problem 3 is S(X) - C_s lambda with S_i = sum_E |E| P(F_E) grad chi_i; one
// Newton iteration solves the block system with A_s replaced by the tangent
//   K_T[(i,d),(j,c)] = sum_E |E| e (delta_dc grad chi_j . grad chi_i
//                                   + 2 eta (F grad chi_j)_c (F grad chi_i)_d)
// and the solid right-hand side K_T X_k - S(X_k), which on an element is
// |E| 2 eta e |F|^2 F grad chi_i (F is linear in X).  Included by
// fsi_solver.cu only.
#pragma once
#include "fsi_kernels.cuh"

namespace fsi {

// One thread per solid node l: row l of K_T in the slots of the solid pair
// matrix (soff/len/col; 2x2 block per slot, FP64 and FP32), and the Newton
// right-hand side of the node's two solid rows.  Each thread writes only its
// own row, adding its triangles in a fixed order (deterministic).  A column
// missing from the row's pattern raises FLAG_CAPACITY; a non-finite e raises
// FLAG_NAN.
__global__ void k_solid_tangent(int nS, const int* __restrict__ ntp, const int* __restrict__ nt,
                                const int* __restrict__ tris, const double* __restrict__ area,
                                const double* __restrict__ tgrad, const double* __restrict__ X, double gamma,
                                double eta, const int* __restrict__ soff, const int* __restrict__ len,
                                const int* __restrict__ col, double* __restrict__ kt, float* __restrict__ kt32,
                                double* __restrict__ bX, int* __restrict__ flags) {
  pdl_begin();
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nS) return;
  const int base = soff[l >> 3] + (l & 7), n = len[l];
  for (int k = 0; k < n; ++k) {
    const size_t s = (size_t)base + ((size_t)k << 3);
#pragma unroll
    for (int q = 0; q < 4; ++q) kt[4 * s + q] = 0.0;
  }
  double b0 = 0.0, b1 = 0.0;
  bool bad = false;
  for (int e = ntp[l]; e < ntp[l + 1]; ++e) {
    const int t = nt[e] / 3, a = nt[e] - 3 * (nt[e] / 3);
    const double* g = tgrad + 6 * (size_t)t;   // grad chi_v = (g[2v], g[2v+1]) on the reference triangle
    double F[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    int vn[3];
    for (int v = 0; v < 3; ++v) {
      vn[v] = tris[3 * t + v];
      const double x0 = X[2 * vn[v]], x1 = X[2 * vn[v] + 1];
      F[0][0] += x0 * g[2 * v]; F[0][1] += x0 * g[2 * v + 1];
      F[1][0] += x1 * g[2 * v]; F[1][1] += x1 * g[2 * v + 1];
    }
    const double n2 = F[0][0] * F[0][0] + F[0][1] * F[0][1] + F[1][0] * F[1][0] + F[1][1] * F[1][1];
    const double ee = gamma * exp(eta * (n2 - 2.0));
    if (!isfinite(ee)) bad = true;
    const double A = area[t];
    double Fg[3][2];   // (F grad chi_v)_c
    for (int v = 0; v < 3; ++v) {
      Fg[v][0] = F[0][0] * g[2 * v] + F[0][1] * g[2 * v + 1];
      Fg[v][1] = F[1][0] * g[2 * v] + F[1][1] * g[2 * v + 1];
    }
    const double rb = A * 2.0 * eta * ee * n2;
    b0 += rb * Fg[a][0];
    b1 += rb * Fg[a][1];
    for (int w = 0; w < 3; ++w) {
      int slot = -1;
      for (int k = 0; k < n; ++k)
        if (col[base + (k << 3)] == vn[w]) { slot = base + (k << 3); break; }
      if (slot < 0) { bad = true; continue; }
      const double gg = g[2 * w] * g[2 * a] + g[2 * w + 1] * g[2 * a + 1];
      double* blk = kt + 4 * (size_t)slot;   // row-major 2x2: (d, c)
      for (int d = 0; d < 2; ++d)
        for (int c = 0; c < 2; ++c)
          blk[2 * d + c] += A * ee * ((d == c ? gg : 0.0) + 2.0 * eta * Fg[w][c] * Fg[a][d]);
    }
  }
  bX[2 * l] = b0;
  bX[2 * l + 1] = b1;
  for (int k = 0; k < n; ++k) {
    const size_t s = (size_t)base + ((size_t)k << 3);
#pragma unroll
    for (int q = 0; q < 4; ++q) kt32[4 * s + q] = (float)kt[4 * s + q];
  }
  if (bad) atomicOr(flags, FLAG_NAN);
}

}  // namespace fsi
