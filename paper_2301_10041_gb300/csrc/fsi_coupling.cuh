// Per-step coupling kernels (steps S2-S4): point location, assembly of
// C_f(X^n) by rows of solid nodes, and its transpose by a counting sort of
// the entries by fluid node.  Included by fsi_solver.cu only.
#pragma once
#include "fsi_kernels.cuh"

namespace fsi {

__constant__ double c_rule_lam[6][3];  // barycentric points of the degree-4 rule
__constant__ double c_rule_w[6];       // weights, summing to 1
__constant__ double c_q1_pt[9][3];     // Q1: (s, t, s t) of the 3 x 3 Gauss points
__constant__ double c_q1_chi[9][4];    // Q1: the four bilinear shape functions there

// Rule points per solid element: the 6-point triangle rule (P1) or the 3 x 3
// Gauss rule (Q1 quadrilaterals).
template <int NPE>
__host__ __device__ constexpr int rule_points() { return NPE == 3 ? 6 : 9; }

// S2: the mapped point, evaluated left to right with explicitly rounded FP64
// operations (no contraction):
//   P1: x_q = P0 + xi1 (P1 - P0) + xi2 (P2 - P0);
//   Q1: x_q = ((P0 + s d1) + t d3) + (s t) e with d1 = P1 - P0,
//       d3 = P3 - P0, e = (P2 - P3) - d1 (the bilinear map of the square);
// then the cell by the half-open rule on t = x * N (the last cell is closed
// at x = 1).
template <int NPE>
__global__ void k_locate(int n_pts, int N, const int* __restrict__ tris, const double* __restrict__ X,
                         int* __restrict__ cell, double* __restrict__ xi, double* __restrict__ eta,
                         int* __restrict__ flags) {
  pdl_begin();
  constexpr int NQ = rule_points<NPE>();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pts) return;
  const int t = p / NQ, q = p - NQ * (p / NQ);
  int v[NPE];
#pragma unroll
  for (int a = 0; a < NPE; ++a) v[a] = tris[NPE * t + a];
  const double fN = (double)N;
  double loc[2];
  int idx[2];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    double xc;
    if constexpr (NPE == 3) {
      const double l1 = c_rule_lam[q][1], l2 = c_rule_lam[q][2];
      const double P0 = X[2 * v[0] + c], P1 = X[2 * v[1] + c], P2 = X[2 * v[2] + c];
      const double d1 = __dsub_rn(P1, P0), d2 = __dsub_rn(P2, P0);
      xc = __dadd_rn(__dadd_rn(P0, __dmul_rn(l1, d1)), __dmul_rn(l2, d2));
    } else {
      const double P0 = X[2 * v[0] + c], P1 = X[2 * v[1] + c], P2 = X[2 * v[2] + c], P3 = X[2 * v[3] + c];
      const double d1 = __dsub_rn(P1, P0), d3 = __dsub_rn(P3, P0);
      const double e = __dsub_rn(__dsub_rn(P2, P3), d1);
      xc = __dadd_rn(__dadd_rn(__dadd_rn(P0, __dmul_rn(c_q1_pt[q][0], d1)), __dmul_rn(c_q1_pt[q][1], d3)),
                     __dmul_rn(c_q1_pt[q][2], e));
    }
    if (!(xc >= 0.0 && xc <= 1.0)) { ok = false; idx[c] = 0; loc[c] = 0.0; continue; }
    const double tc = __dmul_rn(xc, fN);
    int i = (int)floor(tc);
    if (i >= N) i = N - 1;
    idx[c] = i;
    loc[c] = __dsub_rn(tc, (double)i);
  }
  if (!ok) {
    cell[p] = -1; xi[p] = 0.0; eta[p] = 0.0;
    atomicOr(flags, FLAG_OUT_OF_DOMAIN);
    return;
  }
  cell[p] = idx[1] * N + idx[0];
  xi[p] = loc[0];
  eta[p] = loc[1];
}

// Compaction of a row window (wn x hn lattice nodes from (2 x0, 2 y0)) into
// the ELL row of solid node l (slot = (l/32)*32*cap + k*32 + l%32): interior
// columns in lattice order, wall columns into the right-hand-side lift (times
// the wall velocity).  Called by all 32 lanes of the row's warp.
__device__ __forceinline__ void cf_compact_row(const double* W, int l, int x0, int y0, int wn, int hn, int N,
                                               const int* __restrict__ l2n, const double* __restrict__ wall, int cap,
                                               int* __restrict__ len, int* __restrict__ col, double* __restrict__ val,
                                               float* __restrict__ val32, double* __restrict__ lift,
                                               int* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const size_t base = (size_t)(l >> 5) * 32 * cap + (l & 31);
  const int n1 = 2 * N + 1;
  int cnt = 0;
  double lx = 0.0, ly = 0.0;
  for (int k0 = 0; k0 < wn * hn; k0 += 32) {
    const int k = k0 + lane;
    double v = 0.0;
    int node = -1, lat = 0;
    if (k < wn * hn) {
      v = W[k];
      const int ix = 2 * x0 + k % wn, iy = 2 * y0 + k / wn;
      lat = iy * n1 + ix;
      node = l2n[lat];
    }
    const bool interior = (v != 0.0) && node >= 0;
    if (v != 0.0 && node < 0) { lx += v * wall[2 * lat]; ly += v * wall[2 * lat + 1]; }
    const unsigned m = __ballot_sync(0xffffffffu, interior);
    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
    if (interior) {
      if (pos < cap) {
        const size_t slot = base + ((size_t)pos << 5);
        col[slot] = node;
        val[slot] = v;
        val32[slot] = (float)v;
      }
    }
    cnt += __popc(m);
  }
  lx = warp_sum(lx);
  ly = warp_sum(ly);
  if (lane == 0) {
    if (cnt > cap) { atomicOr(flags, FLAG_CAPACITY); cnt = cap; }
    len[l] = cnt;
    lift[2 * l] = lx;
    lift[2 * l + 1] = ly;
  }
}

__device__ __forceinline__ double q2b(int a, double t) {
  return a == 0 ? (1.0 - t) * (1.0 - 2.0 * t) : (a == 1 ? 4.0 * t * (1.0 - t) : t * (2.0 * t - 1.0));
}

// S4: one warp per solid node l.  Row l of the scalar coupling matrix,
//   C_{l j} = sum_{E ni l} sum_q omega_{E,q} chi_l(q) phi_j(x_q),
// with omega = |T| w_q for a P1 triangle (area: one per triangle) and
// omega = w_q |det J_E(s_q)| for a Q1 quadrilateral (area: one per point, from
// the reference configuration), is accumulated in a shared-memory window
// over the fluid lattice nodes of the cells hit by the row's points, points
// taken in a fixed order (no atomics, deterministic); then the window is
// compacted into the ELL row.  Columns on the wall go to the right-hand side
// (times the wall velocity).
template <int NPE>
__global__ void __launch_bounds__(32 * kCfWarps) k_cf_rows(
    int nS, int N, const int* __restrict__ ntp, const int* __restrict__ nt, const double* __restrict__ area,
    const int* __restrict__ cell, const double* __restrict__ xi, const double* __restrict__ eta,
    const int* __restrict__ l2n, const double* __restrict__ wall, int cap, int* __restrict__ len,
    int* __restrict__ col, double* __restrict__ val, float* __restrict__ val32, double* __restrict__ lift,
    int* __restrict__ flags) {
  pdl_begin();
  __shared__ double win[kCfWarps][kCfWindow];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * kCfWarps + warp;
  if (l >= nS) return;
  double* W = win[warp];
  constexpr int NQ = rule_points<NPE>();
  const int e0 = ntp[l], e1 = ntp[l + 1];
  const int npt = NQ * (e1 - e0);
  // bounding box of the cells of the row's points
  int x0 = 1 << 30, y0 = 1 << 30, x1 = -1, y1 = -1;
  bool bad = false;
  for (int k = lane; k < npt; k += 32) {
    const int e = nt[e0 + k / NQ];
    const int p = NQ * (e / NPE) + (k % NQ);
    const int c = cell[p];
    if (c < 0) { bad = true; continue; }
    const int cx = c % N, cy = c / N;
    x0 = min(x0, cx); x1 = max(x1, cx); y0 = min(y0, cy); y1 = max(y1, cy);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  const int wn = 2 * (x1 - x0 + 1) + 1, hn = 2 * (y1 - y0 + 1) + 1;
  if (bad || x1 < 0 || wn * hn > kCfWindow) {
    if (lane == 0) {
      len[l] = 0;
      lift[2 * l] = 0.0; lift[2 * l + 1] = 0.0;
      if (!bad && x1 >= 0) atomicOr(flags, FLAG_CAPACITY);
    }
    return;
  }
  for (int k = lane; k < wn * hn; k += 32) W[k] = 0.0;
  __syncwarp();
  for (int k = 0; k < npt; ++k) {
    const int e = nt[e0 + k / NQ];
    const int t = e / NPE, a = e - NPE * (e / NPE), q = k % NQ;
    const int p = NQ * t + q;
    const int c = cell[p];
    const int cx = c % N, cy = c / N;
    if (lane < 9) {
      const int aa = lane % 3, bb = lane / 3;
      const double wq = (NPE == 3) ? area[t] * c_rule_w[q] * c_rule_lam[q][a] : area[p] * c_q1_chi[q][a];
      const double phi = q2b(aa, xi[p]) * q2b(bb, eta[p]);
      W[(2 * (cy - y0) + bb) * wn + 2 * (cx - x0) + aa] += wq * phi;
    }
    __syncwarp();
  }
  cf_compact_row(W, l, x0, y0, wn, hn, N, l2n, wall, cap, len, col, val, val32, lift, flags);
}

// ------------------------------------------- S4 exact: mesh intersection
__constant__ double c_radon_lam[7][3];  // Radon's degree-5 rule (barycentric points)
__constant__ double c_radon_w[7];       // its weights, summing to 1

// One Sutherland-Hodgman pass: the part of the convex polygon `in` (n
// vertices) with x[axis] <= v (below) or >= v; a crossing edge contributes its
// intersection point with the clipped coordinate set to v.  A triangle cut by
// the four sides of a square has at most 7 vertices; the output is capped at
// kClipMax all the same, so that rounding in a degenerate sliver can never
// write past the buffers.
constexpr int kClipMax = 8;
__device__ __forceinline__ int sh_clip(const double (*in)[2], int n, double (*out)[2], int axis, double v, bool below) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const double* P = in[i];
    const double* Q = in[(i + 1 == n) ? 0 : i + 1];
    const bool inP = below ? (P[axis] <= v) : (P[axis] >= v);
    const bool inQ = below ? (Q[axis] <= v) : (Q[axis] >= v);
    if (inP && m < kClipMax) {
      out[m][0] = P[0];
      out[m][1] = P[1];
      ++m;
    }
    if (inP != inQ && m < kClipMax) {
      const double t = (v - P[axis]) / (Q[axis] - P[axis]);
      out[m][0] = P[0] + t * (Q[0] - P[0]);
      out[m][1] = P[1] + t * (Q[1] - P[1]);
      out[m][axis] = v;
      ++m;
    }
  }
  return m;
}

// Contribution of one (mapped solid triangle, fluid cell) pair to row l:
// acc[3 bb + aa] = (|E| / |X(E)|) * integral over X(E) cut by the cell of
// lambda_a(x) phi_{aa,bb}(x), with the piece split from its first vertex into
// triangles and Radon's degree-5 rule on each (the integrand is linear times
// biquadratic).
__device__ __forceinline__ void exact_pair(const double (*P)[2], double det, double scale, int a, int cx, int cy,
                                           int N, double* acc) {
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  const double h = 1.0 / (double)N;
  double b0[kClipMax][2], b1[kClipMax][2];
  b0[0][0] = P[0][0]; b0[0][1] = P[0][1];
  b0[1][0] = P[1][0]; b0[1][1] = P[1][1];
  b0[2][0] = P[2][0]; b0[2][1] = P[2][1];
  int n = 3;
  n = sh_clip(b0, n, b1, 0, cx * h, false);
  if (n >= 3) n = sh_clip(b1, n, b0, 0, (cx + 1) * h, true);
  if (n >= 3) n = sh_clip(b0, n, b1, 1, cy * h, false);
  if (n >= 3) n = sh_clip(b1, n, b0, 1, (cy + 1) * h, true);
  if (n < 3) return;
  const double d1x = P[1][0] - P[0][0], d1y = P[1][1] - P[0][1];
  const double d2x = P[2][0] - P[0][0], d2y = P[2][1] - P[0][1];
  const double idet = 1.0 / det;       // one division per pair: the FP64 pipe is the bound
  const double fN = (double)N;
  for (int i = 1; i + 1 < n; ++i) {
    const double e1x = b0[i][0] - b0[0][0], e1y = b0[i][1] - b0[0][1];
    const double e2x = b0[i + 1][0] - b0[0][0], e2y = b0[i + 1][1] - b0[0][1];
    const double asub = 0.5 * fabs(e1x * e2y - e1y * e2x);
    if (asub == 0.0) continue;
    for (int q = 0; q < 7; ++q) {
      const double xq = c_radon_lam[q][0] * b0[0][0] + c_radon_lam[q][1] * b0[i][0] + c_radon_lam[q][2] * b0[i + 1][0];
      const double yq = c_radon_lam[q][0] * b0[0][1] + c_radon_lam[q][1] * b0[i][1] + c_radon_lam[q][2] * b0[i + 1][1];
      const double rx = xq - P[0][0], ry = yq - P[0][1];
      const double l1 = (rx * d2y - ry * d2x) * idet;
      const double l2 = (d1x * ry - d1y * rx) * idet;
      const double la = (a == 0) ? 1.0 - l1 - l2 : (a == 1 ? l1 : l2);
      const double xi = xq * fN - cx, eta = yq * fN - cy;
      const double wq = asub * c_radon_w[q] * la;
      double bx[3], by[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        bx[j] = q2b(j, xi);
        by[j] = q2b(j, eta);
      }
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) acc[3 * bb + aa] += wq * bx[aa] * by[bb];
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] *= scale;
}

// S4 with the paper's exact rule (Section 4): one warp per solid node l.
// Every (triangle of l, fluid cell of the triangle's bounding box) pair is one
// work item; the lanes take 32 items at a time, and their 9 contributions are
// added to the row window in item order (no atomics, deterministic), then
// compacted as in k_cf_rows.  A vertex outside [0,1]^2 raises
// FLAG_OUT_OF_DOMAIN; more than 32 triangles at a node or a window above
// kCfWindow lattice nodes raises FLAG_CAPACITY (the row is then left empty).
__global__ void __launch_bounds__(32 * kCfWarps) k_cf_rows_exact(
    int nS, int N, const int* __restrict__ ntp, const int* __restrict__ nt, const int* __restrict__ tris,
    const double* __restrict__ X, const double* __restrict__ area, const int* __restrict__ l2n,
    const double* __restrict__ wall, int cap, int* __restrict__ len, int* __restrict__ col,
    double* __restrict__ val, float* __restrict__ val32, double* __restrict__ lift, int* __restrict__ flags) {
  pdl_begin();
  __shared__ double win[kCfWarps][kCfWindow];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * kCfWarps + warp;
  if (l >= nS) return;
  double* W = win[warp];
  const int e0 = ntp[l], nk = ntp[l + 1] - e0;
  // lane k < nk holds triangle k of the row: mapped vertices, cell box, item count
  int t = 0, a = 0, cx0 = 0, cy0 = 0, bw = 0, cnt = 0;
  bool outside = false;
  if (lane < nk) {
    const int e = nt[e0 + lane];
    t = e / 3;
    a = e - 3 * t;
    double lo[2] = {2.0, 2.0}, hi[2] = {-1.0, -1.0};
    for (int v = 0; v < 3; ++v) {
      const int node = tris[3 * t + v];
      for (int c = 0; c < 2; ++c) {
        const double xc = X[2 * node + c];
        if (!(xc >= 0.0 && xc <= 1.0)) outside = true;
        lo[c] = fmin(lo[c], xc);
        hi[c] = fmax(hi[c], xc);
      }
    }
    if (!outside) {
      cx0 = min((int)floor(lo[0] * N), N - 1);
      cy0 = min((int)floor(lo[1] * N), N - 1);
      const int cx1 = min((int)floor(hi[0] * N), N - 1), cy1 = min((int)floor(hi[1] * N), N - 1);
      bw = cx1 - cx0 + 1;
      cnt = bw * (cy1 - cy0 + 1);
    }
  }
  const bool bad = __any_sync(0xffffffffu, outside);
  // window: union of the cell boxes
  int x0 = (lane < nk) ? cx0 : (1 << 30), y0 = (lane < nk) ? cy0 : (1 << 30);
  int x1 = (lane < nk && bw > 0) ? cx0 + bw - 1 : -1, y1 = (lane < nk && bw > 0) ? cy0 + cnt / bw - 1 : -1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
  }
  const int wn = 2 * (x1 - x0 + 1) + 1, hn = 2 * (y1 - y0 + 1) + 1;
  if (bad || nk > 32 || nk == 0 || x1 < 0 || wn * hn > kCfWindow) {
    if (lane == 0) {
      len[l] = 0;
      lift[2 * l] = 0.0;
      lift[2 * l + 1] = 0.0;
      if (bad) atomicOr(flags, FLAG_OUT_OF_DOMAIN);
      else if (nk > 0) atomicOr(flags, FLAG_CAPACITY);
    }
    return;
  }
  // exclusive prefix of the item counts over the row's triangles
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int excl = incl - cnt;
  const int nitems = __shfl_sync(0xffffffffu, incl, 31);
  for (int k = lane; k < wn * hn; k += 32) W[k] = 0.0;
  __syncwarp();
  for (int i0 = 0; i0 < nitems; i0 += 32) {
    const int i = i0 + lane;
    double acc[9];
    int cx = x0, cy = y0;
    {
      int k = 0;
      for (int kk = 1; kk < nk; ++kk)
        if (i >= __shfl_sync(0xffffffffu, excl, kk)) k = kk;
      // every lane takes part in the shuffles; lanes past the items compute nothing
      const int tk = __shfl_sync(0xffffffffu, t, k), ak = __shfl_sync(0xffffffffu, a, k);
      const int bx0 = __shfl_sync(0xffffffffu, cx0, k), by0 = __shfl_sync(0xffffffffu, cy0, k);
      const int bwk = __shfl_sync(0xffffffffu, bw, k), ek = __shfl_sync(0xffffffffu, excl, k);
      if (i < nitems) {
        const int j = i - ek;
        cx = bx0 + j % bwk;
        cy = by0 + j / bwk;
        double P[3][2];
        for (int v = 0; v < 3; ++v) {
          const int node = tris[3 * tk + v];
          P[v][0] = X[2 * node];
          P[v][1] = X[2 * node + 1];
        }
        const double det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[1][1] - P[0][1]) * (P[2][0] - P[0][0]);
        if (det != 0.0) {
          exact_pair(P, det, area[tk] / (0.5 * fabs(det)), ak, cx, cy, N, acc);
        } else {
#pragma unroll
          for (int q = 0; q < 9; ++q) acc[q] = 0.0;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = 0.0;
      }
    }
    const int ns = min(32, nitems - i0);
    for (int src = 0; src < ns; ++src) {
      const int scx = __shfl_sync(0xffffffffu, cx, src), scy = __shfl_sync(0xffffffffu, cy, src);
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const double tq = __shfl_sync(0xffffffffu, acc[q], src);
        if (lane == q) v = tq;
      }
      if (lane < 9) W[(2 * (scy - y0) + lane / 3) * wn + 2 * (scx - x0) + lane % 3] += v;
      __syncwarp();
    }
  }
  __syncwarp();
  cf_compact_row(W, l, x0, y0, wn, hn, N, l2n, wall, cap, len, col, val, val32, lift, flags);
}

// S3 (the "hash grid"): counting sort of the C_f entries by fluid node.
__global__ void k_cft_count(int nS, int cap, const int* __restrict__ len, const int* __restrict__ col,
                            int* __restrict__ cnt) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = i / cap, k = i - cap * (i / cap);
  if (l >= nS || k >= len[l]) return;
  atomicAdd(&cnt[col[(size_t)(l >> 5) * 32 * cap + ((size_t)k << 5) + (l & 31)]], 1);
}

constexpr int kScanBlock = 1024;

// exclusive scan of cnt[0..n) into out[0..n], three phases
__global__ void k_scan_partial(int n, const int* __restrict__ in, int* __restrict__ bsum) {
  pdl_begin();
  __shared__ int sm[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  int v = (i < n) ? in[i] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int s = sm[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
  }
}

__device__ __forceinline__ int block_excl_scan(int v, int* sm, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sm[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    sm[lane] = s;
  }
  __syncthreads();
  total = sm[(blockDim.x >> 5) - 1];
  const int before = (w > 0) ? sm[w - 1] : 0;
  const int r = before + inc - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_top(int nb, int* __restrict__ bsum) {
  pdl_begin();
  __shared__ int sm[32];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanBlock) {
    const int i = b0 + threadIdx.x;
    const int v = (i < nb) ? bsum[i] : 0;
    int total;
    const int e = block_excl_scan(v, sm, total);
    if (i < nb) bsum[i] = carry + e;
    carry += total;
  }
}

__global__ void k_scan_final(int n, const int* __restrict__ in, const int* __restrict__ bsum,
                             int* __restrict__ out, int* __restrict__ cursor) {
  pdl_begin();
  __shared__ int sm[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int v = (i < n) ? in[i] : 0;
  int total;
  const int e = block_excl_scan(v, sm, total) + bsum[blockIdx.x];
  if (i < n) { out[i] = e; cursor[i] = e; }
  if (i == n - 1) out[n] = e + v;
}

__global__ void k_cft_scatter(int nS, int cap, const int* __restrict__ len, const int* __restrict__ col,
                              const double* __restrict__ val, int* __restrict__ cursor, int* __restrict__ tcol,
                              double* __restrict__ tval) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = i / cap, k = i - cap * (i / cap);
  if (l >= nS || k >= len[l]) return;
  const size_t slot = (size_t)(l >> 5) * 32 * cap + ((size_t)k << 5) + (l & 31);
  const int pos = atomicAdd(&cursor[col[slot]], 1);
  tcol[pos] = l;
  tval[pos] = val[slot];
}

// sort each transposed row by solid node (the scatter order is not fixed)
__global__ void k_cft_sort(int nU, const int* __restrict__ ptr, int* __restrict__ tcol, double* __restrict__ tval,
                           float* __restrict__ tval32) {
  pdl_begin();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nU) return;
  const int a = ptr[r], b = ptr[r + 1];
  for (int i = a + 1; i < b; ++i) {
    const int c = tcol[i];
    const double v = tval[i];
    int j = i - 1;
    while (j >= a && tcol[j] > c) { tcol[j + 1] = tcol[j]; tval[j + 1] = tval[j]; --j; }
    tcol[j + 1] = c;
    tval[j + 1] = v;
  }
  for (int i = a; i < b; ++i) tval32[i] = (float)tval[i];
}

}  // namespace fsi
