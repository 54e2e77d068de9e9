// Matrix-free, temporally blocked kernels for the fine levels of the
// geometric multigrid V-cycle (Section 5: one V-cycle with Chebyshev-Jacobi
// smoothing approximates each inner fluid solve).
//
// On the uniform grid every level operator has constant coefficients: the
// Q2 velocity operator A = (rho/dt) M + K one 2x2 block per (node type,
// lattice offset), the pressure Laplacian L = B diag(M)^-1 B^T one 3x3 block
// per (wall variant, cell offset); the transfers are the fixed Q2 and P1disc
// interpolation weights.  So a level needs no stored matrix, and the work of
// one V-cycle level folds into two launches:
//
//   down: x0 = c0 D^-1 b, the remaining pre-smoothing Chebyshev steps, the
//         residual r = b - A x and its restriction R r to the next level;
//   up:   x + P x_coarse, then the post-smoothing Chebyshev steps, with the
//         caller's epilogue (Richardson update, Cahouet-Chabard combination).
//
// Each CTA owns a tile and computes every intermediate on the tile grown by
// the reach of the steps that follow (two lattice nodes per velocity sweep,
// one cell per pressure sweep, four lattice nodes for the Q2 restriction),
// in shared memory, so the steps of one launch need no grid-wide barrier.
// Neighbouring tiles repeat the arithmetic of their overlap in the same
// order, so every node gets the same value whichever tile computes it.
// Positions on the wall or outside the grid hold zero (absent unknowns).
//
// Each kernel is a thin wrapper around a __host__ __device__ body that takes
// the CTA's coordinates explicitly.  Every loop of a body is strided over the
// CTA's threads and the phases are separated by barriers, so a body run by
// one thread per CTA computes the same values; the host test of these
// kernels runs the bodies that way.
#pragma once
#include <cuda_runtime.h>

#include "fsi_internal.h"

namespace fsi {

#ifndef FSI_VEC2_DEFINED
#define FSI_VEC2_DEFINED
template <class T>
struct Vec2;
template <>
struct Vec2<float> { using type = float2; };
template <>
struct Vec2<double> { using type = double2; };
#endif

// the CTA a body works for: block coordinates, this thread, the thread count
// and the dynamic shared memory
struct MfCta {
  int bx, by, tid, nthr;
  unsigned char* sm;
};

#ifdef __CUDA_ARCH__
#define MF_SYNC() __syncthreads()
#else
#define MF_SYNC() ((void)0)
#endif

__host__ __device__ __forceinline__ int mf_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int mf_max(int a, int b) { return a > b ? a : b; }

constexpr int kMfThreads = 256;
constexpr int kMfMaxDeg = 4;   // Chebyshev degrees 1..4 (the default is 2)
constexpr int kMfTileU = 8;    // velocity down: coarse lattice nodes per tile side
constexpr int kMfTileUf = 16;  // velocity up: fine lattice nodes per tile side
constexpr int kMfTileP = 4;    // pressure down: coarse cells per tile side
constexpr int kMfTilePf = 8;   // pressure up: fine cells per tile side
constexpr int kMfPresTab = 9 * 9 * 9 + 9 * 3;  // pressure stencil table: blocks, then D^-1

template <class T>
struct MfCheb {
  int k = 2;                       // degree: 1 initial step + k - 1 Chebyshev steps per smoothing
  T c0 = 0;
  T c1[kMfMaxDeg] = {}, c2[kMfMaxDeg] = {};
};

// Q2 velocity level: blocks [type][dy+2][dx+2][2x2 row-major], type =
// (ix & 1) | (iy & 1) << 1; D^-1 per type and component.
template <class T>
struct MfVelOp {
  int N = 0;
  T c[4][5][5][4];
  T dinv[4][2];
};

// Coarse-level smoother start written by a down kernel when the next level
// runs the per-level sparse kernels: x = d = c0 D^-1 b.
template <class T>
struct MfInit {
  T* x = nullptr;
  T* d = nullptr;
  const T* dinv = nullptr;
  T c0 = 0;
};

// Epilogue of the last post-smoothing step (the caller's SpmvArgs fields):
// with sout, s = -(snu smp sv + srdt y) is written to sout; with acc,
// acc += omega * (s if sout else y).
template <class T>
struct MfFin {
  const T* sv = nullptr;
  const T* smp = nullptr;
  T* sout = nullptr;
  T snu = 0, srdt = 0;
  T* acc = nullptr;
  T omega = 1;
};

template <class T>
struct MfVelArgs {
  MfVelOp<T> op;
  MfCheb<T> ch;
  const T* b = nullptr;     // level right-hand side (node order, (x, y) per node)
  const T* xpre = nullptr;  // up: the pre-smoothed iterate
  const T* xc = nullptr;    // up: the coarse correction
  T* xout = nullptr;        // down: pre-smoothed iterate; up: result
  T* bc = nullptr;          // down: coarse right-hand side
  MfInit<T> ci;
  MfFin<T> fin;
};

template <class T>
struct MfPresArgs {
  int N = 0;
  const T* tab = nullptr;   // kMfPresTab values
  MfCheb<T> ch;
  const T* b = nullptr;     // 3 per cell
  const T* xpre = nullptr;
  const T* xc = nullptr;
  T* xout = nullptr;
  T* bc = nullptr;
  MfInit<T> ci;
  MfFin<T> fin;
};

// --------------------------------------------------------------- velocity
// interior Q2 node (1 <= ix, iy <= 2N-1) -> id in the type-blocked order
// (corners, x-edge midpoints, y-edge midpoints, centres; lattice order inside)
__host__ __device__ __forceinline__ int mf_vnode(int N, int ix, int iy) {
  const int nV = (N - 1) * (N - 1), nX = N * (N - 1);
  const int ox = ix & 1, oy = iy & 1;
  if (!ox && !oy) return (iy / 2 - 1) * (N - 1) + (ix / 2 - 1);
  if (ox && !oy) return nV + (iy / 2 - 1) * N + (ix - 1) / 2;
  if (!ox && oy) return nV + nX + ((iy - 1) / 2) * (N - 1) + (ix / 2 - 1);
  return nV + 2 * nX + ((iy - 1) / 2) * N + (ix - 1) / 2;
}

__host__ __device__ __forceinline__ bool mf_vinterior(int N, int ix, int iy) {
  return ix >= 1 && iy >= 1 && ix <= 2 * N - 1 && iy <= 2 * N - 1;
}

// A lattice frame in shared memory: origin (ox, oy) even, 4 parity planes
// (one per node type) of pw x ph entries; lattice (ox + 2 px + (t & 1),
// oy + 2 py + (t >> 1)) is entry (t ph + py) pw + px.
struct MfFrame {
  int ox, oy, pw, ph;
  __host__ __device__ __forceinline__ int plane() const { return pw * ph; }
};

// y += A v at the node of type TAU with plane coordinates (px, py)
template <class T, int TAU>
__host__ __device__ __forceinline__ void mf_vel_apply(const MfVelOp<T>& op, const typename Vec2<T>::type* __restrict__ v,
                                             const MfFrame& f, int px, int py, T& y0, T& y1) {
  constexpr int PX = TAU & 1, PY = TAU >> 1;
  constexpr int RX = PX ? 1 : 2, RY = PY ? 1 : 2;
#pragma unroll
  for (int dy = -RY; dy <= RY; ++dy) {
#pragma unroll
    for (int dx = -RX; dx <= RX; ++dx) {
      const int t2 = ((PX + dx) & 1) | (((PY + dy) & 1) << 1);
      const int qx = px + ((PX + dx) >> 1), qy = py + ((PY + dy) >> 1);
      const auto x = v[(t2 * f.ph + qy) * f.pw + qx];
      const T* c = op.c[TAU][dy + 2][dx + 2];
      y0 += c[0] * x.x + c[1] * x.y;
      y1 += c[2] * x.x + c[3] * x.y;
    }
  }
}

template <class T>
__host__ __device__ __forceinline__ void mf_vel_res(const MfVelOp<T>& op, int tau, const typename Vec2<T>::type* __restrict__ v,
                                           const MfFrame& f, int px, int py, T& y0, T& y1) {
  switch (tau) {
    case 0: mf_vel_apply<T, 0>(op, v, f, px, py, y0, y1); break;
    case 1: mf_vel_apply<T, 1>(op, v, f, px, py, y0, y1); break;
    case 2: mf_vel_apply<T, 2>(op, v, f, px, py, y0, y1); break;
    default: mf_vel_apply<T, 3>(op, v, f, px, py, y0, y1); break;
  }
}

// Visit every frame entry of the plane rectangle [q0, q1) (x and y) in all
// four planes; warps never straddle two planes, so the node type (and with
// it the stencil) is the same across a warp.
template <class F>
__host__ __device__ __forceinline__ void mf_vsweep(const MfCta& c, const MfFrame& f, int qx0, int qx1, int qy0,
                                                   int qy1, F&& fn) {
  const int nqx = qx1 - qx0, nq = nqx * (qy1 - qy0);
  const int nq32 = (nq + 31) & ~31;
  for (int i = c.tid; i < 4 * nq32; i += c.nthr) {
    const int tau = i / nq32, j = i - tau * nq32;
    if (j >= nq) continue;
    const int px = qx0 + j % nqx, py = qy0 + j / nqx;
    fn(tau, px, py, (tau * f.ph + py) * f.pw + px);
  }
}

// One Chebyshev step on the plane rectangle shrunk by `s` from the frame:
// first (CHEB0 / after init): dn = c2 D^-1 (b - A xo); otherwise
// dn = c1 do + c2 D^-1 (b - A xo); xn = xo + dn.  Outside the interior 0.
template <class T>
__host__ __device__ __forceinline__ void mf_vel_cheb(const MfCta& cta, const MfVelOp<T>& op, const MfFrame& f, int s,
                                            const typename Vec2<T>::type* __restrict__ B,
                                            const typename Vec2<T>::type* __restrict__ Xo,
                                            const typename Vec2<T>::type* __restrict__ Do,
                                            typename Vec2<T>::type* __restrict__ Xn,
                                            typename Vec2<T>::type* __restrict__ Dn, bool first, T c1, T c2) {
  using T2 = typename Vec2<T>::type;
  const int N = op.N;
  mf_vsweep(cta, f, s, f.pw - s, s, f.ph - s, [&](int tau, int px, int py, int e) {
    const int ix = f.ox + 2 * px + (tau & 1), iy = f.oy + 2 * py + (tau >> 1);
    T2 xn, dn;
    if (mf_vinterior(N, ix, iy)) {
      T a0 = 0, a1 = 0;
      mf_vel_res<T>(op, tau, Xo, f, px, py, a0, a1);
      const T2 b = B[e], xo = Xo[e];
      const T r0 = b.x - a0, r1 = b.y - a1;
      if (first) {
        dn.x = c2 * op.dinv[tau][0] * r0;
        dn.y = c2 * op.dinv[tau][1] * r1;
      } else {
        const T2 d = Do[e];
        dn.x = c1 * d.x + c2 * op.dinv[tau][0] * r0;
        dn.y = c1 * d.y + c2 * op.dinv[tau][1] * r1;
      }
      xn.x = xo.x + dn.x;
      xn.y = xo.y + dn.y;
    } else {
      xn.x = xn.y = dn.x = dn.y = 0;
    }
    Xn[e] = xn;
    Dn[e] = dn;
  });
}

// Q2 prolongation weights: a fine lattice coordinate f lies in coarse cell
// cc = min(f / 4, Nc - 1) at r = f - 4 cc; coarse node 2 cc + a gets the
// coarse quadratic's value there, mf_pw(r, a)
__host__ __device__ __forceinline__ float mf_pw(int r, int a) {
  switch (r) {
    case 0: return a == 0 ? 1.f : 0.f;
    case 1: return a == 0 ? 0.375f : (a == 1 ? 0.75f : -0.125f);
    case 2: return a == 1 ? 1.f : 0.f;
    case 3: return a == 0 ? -0.125f : (a == 1 ? 0.75f : 0.375f);
    default: return a == 2 ? 1.f : 0.f;
  }
}

// restriction weight of a fine node at offset d from 2X (coarse node X) in 1-D
__host__ __device__ __forceinline__ float mf_rw(int odd, int d) {
  const int a = d < 0 ? -d : d;
  if (odd) return a == 0 ? 1.f : (a == 1 ? 0.75f : 0.f);
  return a == 0 ? 1.f : (a == 1 ? 0.375f : (a == 3 ? -0.125f : 0.f));
}

// down: grid (ceil(N / kMfTileU))^2 over the coarse lattice [0, N)^2
template <class T>
__host__ __device__ void mfu_down_body(const MfVelArgs<T>& a, const MfCta& cta) {
  using T2 = typename Vec2<T>::type;
  unsigned char* mf_sm = cta.sm;
  const MfVelOp<T>& op = a.op;
  const int N = op.N, K = a.ch.k;
  const int CX0 = cta.bx * kMfTileU, CY0 = cta.by * kMfTileU;
  MfFrame f;
  f.ox = 2 * CX0 - 4 - 2 * K;
  f.oy = 2 * CY0 - 4 - 2 * K;
  f.pw = f.ph = (2 * kMfTileU + 8 + 4 * K) / 2;
  const int nf = 4 * f.plane();
  T2* B = reinterpret_cast<T2*>(mf_sm);
  T2 *Xc = B + nf, *Xn = B + 2 * nf, *Dc = B + 3 * nf, *Dn = B + 4 * nf;   // current / next iterate
  T2* R = B + 5 * nf;
  // b on the frame; x0 = d0 = c0 D^-1 b
  for (int e = cta.tid; e < nf; e += cta.nthr) {
    const int tau = e / f.plane(), j = e - tau * f.plane();
    const int ix = f.ox + 2 * (j % f.pw) + (tau & 1), iy = f.oy + 2 * (j / f.pw) + (tau >> 1);
    T2 v;
    v.x = v.y = 0;
    if (mf_vinterior(N, ix, iy)) v = *reinterpret_cast<const T2*>(a.b + 2 * (size_t)mf_vnode(N, ix, iy));
    B[e] = v;
    T2 x0;
    x0.x = a.ch.c0 * op.dinv[tau][0] * v.x;
    x0.y = a.ch.c0 * op.dinv[tau][1] * v.y;
    Xc[e] = x0;
    Dc[e] = x0;
  }
  MF_SYNC();
  for (int s = 1; s < K; ++s) {  // pre-smoothing steps 1 .. K-1 on the frame shrunk by s nodes per plane
    mf_vel_cheb<T>(cta, op, f, s, B, Xc, Dc, Xn, Dn, false, a.ch.c1[s - 1], a.ch.c2[s - 1]);
    T2* t = Xc; Xc = Xn; Xn = t;
    t = Dc; Dc = Dn; Dn = t;
    MF_SYNC();
  }
  // residual on the frame shrunk by K (plane units): the restriction's support
  mf_vsweep(cta, f, K, f.pw - K, K, f.ph - K, [&](int tau, int px, int py, int e) {
    const int ix = f.ox + 2 * px + (tau & 1), iy = f.oy + 2 * py + (tau >> 1);
    T2 r;
    r.x = r.y = 0;
    if (mf_vinterior(N, ix, iy)) {
      T a0 = 0, a1 = 0;
      mf_vel_res<T>(op, tau, Xc, f, px, py, a0, a1);
      r.x = B[e].x - a0;
      r.y = B[e].y - a1;
    }
    R[e] = r;
  });
  // the pre-smoothed iterate on the owned fine nodes [2 CX0, 2 CX0 + 2 tile)
  const int o = (4 + 2 * K) / 2;   // plane offset of the owned region in the frame
  for (int i = cta.tid; i < 4 * kMfTileU * kMfTileU; i += cta.nthr) {
    const int tau = i / (kMfTileU * kMfTileU), j = i - tau * kMfTileU * kMfTileU;
    const int px = o + j % kMfTileU, py = o + j / kMfTileU;
    const int ix = f.ox + 2 * px + (tau & 1), iy = f.oy + 2 * py + (tau >> 1);
    if (mf_vinterior(N, ix, iy))
      *reinterpret_cast<T2*>(a.xout + 2 * (size_t)mf_vnode(N, ix, iy)) = Xc[(tau * f.ph + py) * f.pw + px];
  }
  MF_SYNC();
  // restriction to the coarse nodes of the tile (coarse lattice interior 1 .. N - 1)
  const int Nc = N / 2;
  for (int i = cta.tid; i < kMfTileU * kMfTileU; i += cta.nthr) {
    const int X0 = CX0 + i % kMfTileU, Y0 = CY0 + i / kMfTileU;
    if (!mf_vinterior(Nc, X0, Y0)) continue;
    T s0 = 0, s1 = 0;
    const int rx = (X0 & 1) ? 1 : 3, ry = (Y0 & 1) ? 1 : 3;
    for (int dy = -ry; dy <= ry; ++dy) {
      const T wy = (T)mf_rw(Y0 & 1, dy);
      if (wy == (T)0) continue;
      for (int dx = -rx; dx <= rx; ++dx) {
        const T wx = (T)mf_rw(X0 & 1, dx);
        if (wx == (T)0) continue;
        const int ix = 2 * X0 + dx, iy = 2 * Y0 + dy;
        const T2 r = R[((((ix & 1) | ((iy & 1) << 1)) * f.ph + ((iy - f.oy) >> 1)) * f.pw) + ((ix - f.ox) >> 1)];
        const T w = wx * wy;
        s0 += w * r.x;
        s1 += w * r.y;
      }
    }
    const int id = mf_vnode(Nc, X0, Y0);
    a.bc[2 * id] = s0;
    a.bc[2 * id + 1] = s1;
    if (a.ci.x) {
      const T d0 = a.ci.c0 * a.ci.dinv[2 * id] * s0, d1 = a.ci.c0 * a.ci.dinv[2 * id + 1] * s1;
      a.ci.x[2 * id] = d0;
      a.ci.x[2 * id + 1] = d1;
      a.ci.d[2 * id] = d0;
      a.ci.d[2 * id + 1] = d1;
    }
  }
}

// up: grid (ceil(2N / kMfTileUf))^2 over the fine lattice [0, 2N)^2
template <class T>
__host__ __device__ void mfu_up_body(const MfVelArgs<T>& a, const MfCta& cta) {
  using T2 = typename Vec2<T>::type;
  unsigned char* mf_sm = cta.sm;
  const MfVelOp<T>& op = a.op;
  const int N = op.N, K = a.ch.k, Nc = N / 2;
  const int FX0 = cta.bx * kMfTileUf, FY0 = cta.by * kMfTileUf;
  MfFrame f;
  f.ox = FX0 - 2 * K;
  f.oy = FY0 - 2 * K;
  f.pw = f.ph = (kMfTileUf + 4 * K) / 2;
  // coarse lattice frame covering the prolongation taps of the fine frame
  MfFrame g;
  {
    const int lox = mf_max(f.ox, 0) >> 2, loy = mf_max(f.oy, 0) >> 2;
    const int hix = mf_min((f.ox + 2 * f.pw - 1) >> 2, Nc - 1), hiy = mf_min((f.oy + 2 * f.ph - 1) >> 2, Nc - 1);
    g.ox = 2 * lox;
    g.oy = 2 * loy;
    g.pw = hix - lox + 2;   // coarse lattice 2 lo .. 2 hi + 2, i.e. 2 (hi - lo) + 3 nodes
    g.ph = hiy - loy + 2;
  }
  const int nf = 4 * f.plane(), ng = 4 * g.plane();
  T2* B = reinterpret_cast<T2*>(mf_sm);
  T2 *Xc = B + nf, *Xn = B + 2 * nf, *Dc = B + 3 * nf, *Dn = B + 4 * nf;
  T2* XC = B + 5 * nf;
  for (int e = cta.tid; e < ng; e += cta.nthr) {
    const int tau = e / g.plane(), j = e - tau * g.plane();
    const int ix = g.ox + 2 * (j % g.pw) + (tau & 1), iy = g.oy + 2 * (j / g.pw) + (tau >> 1);
    T2 v;
    v.x = v.y = 0;
    if (mf_vinterior(Nc, ix, iy)) v = *reinterpret_cast<const T2*>(a.xc + 2 * (size_t)mf_vnode(Nc, ix, iy));
    XC[e] = v;
  }
  MF_SYNC();
  // b and x + P x_coarse on the frame
  for (int e = cta.tid; e < nf; e += cta.nthr) {
    const int tau = e / f.plane(), j = e - tau * f.plane();
    const int ix = f.ox + 2 * (j % f.pw) + (tau & 1), iy = f.oy + 2 * (j / f.pw) + (tau >> 1);
    T2 bv, xv;
    bv.x = bv.y = xv.x = xv.y = 0;
    if (mf_vinterior(N, ix, iy)) {
      const size_t id = mf_vnode(N, ix, iy);
      bv = *reinterpret_cast<const T2*>(a.b + 2 * id);
      xv = *reinterpret_cast<const T2*>(a.xpre + 2 * id);
      const int ccx = mf_min(ix >> 2, Nc - 1), ccy = mf_min(iy >> 2, Nc - 1);
      const int rx = ix - 4 * ccx, ry = iy - 4 * ccy;
      T p0 = 0, p1 = 0;
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        const T wy = (T)mf_pw(ry, bb);
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) {
          const T w = (T)mf_pw(rx, aa) * wy;
          const int X0 = 2 * ccx + aa, Y0 = 2 * ccy + bb;
          const T2 c = XC[((((X0 & 1) | ((Y0 & 1) << 1)) * g.ph + ((Y0 - g.oy) >> 1)) * g.pw) + ((X0 - g.ox) >> 1)];
          p0 += w * c.x;
          p1 += w * c.y;
        }
      }
      xv.x = p0 + xv.x;
      xv.y = p1 + xv.y;
    }
    B[e] = bv;
    Xc[e] = xv;
  }
  MF_SYNC();
  for (int s = 0; s < K; ++s) {  // post-smoothing: CHEB0, then CHEB steps, each on a frame 1 plane entry smaller
    const bool last = (s == K - 1);
    if (!last) {
      mf_vel_cheb<T>(cta, op, f, s + 1, B, Xc, Dc, Xn, Dn, s == 0,
                     s == 0 ? (T)0 : a.ch.c1[s - 1], s == 0 ? a.ch.c0 : a.ch.c2[s - 1]);
      T2* t = Xc; Xc = Xn; Xn = t;
      t = Dc; Dc = Dn; Dn = t;
      MF_SYNC();
      continue;
    }
    // last step on the owned tile: write the result and the epilogue
    const T c1 = s == 0 ? (T)0 : a.ch.c1[s - 1], c2 = s == 0 ? a.ch.c0 : a.ch.c2[s - 1];
    mf_vsweep(cta, f, K, f.pw - K, K, f.ph - K, [&](int tau, int px, int py, int e) {
      const int ix = f.ox + 2 * px + (tau & 1), iy = f.oy + 2 * py + (tau >> 1);
      if (!mf_vinterior(N, ix, iy)) return;
      T a0 = 0, a1 = 0;
      mf_vel_res<T>(op, tau, Xc, f, px, py, a0, a1);
      const T2 b = B[e], xo = Xc[e];
      const T r0 = b.x - a0, r1 = b.y - a1;
      T d0 = c2 * op.dinv[tau][0] * r0, d1 = c2 * op.dinv[tau][1] * r1;
      if (s > 0) {
        const T2 d = Dc[e];
        d0 = c1 * d.x + c2 * op.dinv[tau][0] * r0;
        d1 = c1 * d.y + c2 * op.dinv[tau][1] * r1;
      }
      const size_t id = mf_vnode(N, ix, iy);
      const T y0 = xo.x + d0, y1 = xo.y + d1;
      T2 y;
      y.x = y0;
      y.y = y1;
      *reinterpret_cast<T2*>(a.xout + 2 * id) = y;
      if (a.fin.acc) {
        a.fin.acc[2 * id] += a.fin.omega * y0;
        a.fin.acc[2 * id + 1] += a.fin.omega * y1;
      }
    });
  }
}

// --------------------------------------------------------------- pressure
// A cell frame in shared memory: origin (ox, oy), w x w cells, three planes
// (one per P1disc coefficient).
struct MfCells {
  int ox, oy, w;
  __host__ __device__ __forceinline__ int n() const { return w * w; }
};

template <class T>
__host__ __device__ __forceinline__ int mf_variant(int N, int cx, int cy) {
  const int vx = cx == 0 ? 0 : (cx == N - 1 ? 2 : 1), vy = cy == 0 ? 0 : (cy == N - 1 ? 2 : 1);
  return 3 * vy + vx;
}

// y = L v at cell (cx, cy) (frame entry e) with the stencil table in shared memory
template <class T>
__host__ __device__ __forceinline__ void mf_pres_apply(const T* __restrict__ tab, const T* __restrict__ v, const MfCells& f,
                                              int N, int cx, int cy, int e, T y[3]) {
  const T* base = tab + 81 * mf_variant<T>(N, cx, cy);
  const int n = f.n();
  y[0] = y[1] = y[2] = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int q = e + dy * f.w + dx;
      const T x0 = v[q], x1 = v[n + q], x2 = v[2 * n + q];
      const T* c = base + 9 * ((dy + 1) * 3 + dx + 1);
#pragma unroll
      for (int i = 0; i < 3; ++i) y[i] += c[3 * i] * x0 + c[3 * i + 1] * x1 + c[3 * i + 2] * x2;
    }
  }
}

template <class T>
__host__ __device__ __forceinline__ bool mf_cin(int N, int cx, int cy) {
  return cx >= 0 && cy >= 0 && cx < N && cy < N;
}

// one Chebyshev step on the cell frame shrunk by s cells
template <class T>
__host__ __device__ __forceinline__ void mf_pres_cheb(const MfCta& cta, const T* __restrict__ tab, int N,
                                                      const MfCells& f, int s,
                                             const T* __restrict__ B, const T* __restrict__ Xo,
                                             const T* __restrict__ Do, T* __restrict__ Xn, T* __restrict__ Dn,
                                             bool first, T c1, T c2) {
  const int m = f.w - 2 * s, n = f.n();
  const T* dv = tab + 729;
  for (int i = cta.tid; i < m * m; i += cta.nthr) {
    const int lx = s + i % m, ly = s + i / m, e = ly * f.w + lx;
    const int cx = f.ox + lx, cy = f.oy + ly;
    if (!mf_cin<T>(N, cx, cy)) {
      for (int k = 0; k < 3; ++k) Xn[k * n + e] = Dn[k * n + e] = 0;
      continue;
    }
    T y[3];
    mf_pres_apply<T>(tab, Xo, f, N, cx, cy, e, y);
    const int v = mf_variant<T>(N, cx, cy);
    for (int k = 0; k < 3; ++k) {
      const T r = B[k * n + e] - y[k];
      const T dn = first ? c2 * dv[3 * v + k] * r : c1 * Do[k * n + e] + c2 * dv[3 * v + k] * r;
      Dn[k * n + e] = dn;
      Xn[k * n + e] = Xo[k * n + e] + dn;
    }
  }
}

// down: grid (ceil(Nc / kMfTileP))^2 over the coarse cells
template <class T>
__host__ __device__ void mfp_down_body(const MfPresArgs<T>& a, const MfCta& cta) {
  unsigned char* mf_sm = cta.sm;
  const int N = a.N, K = a.ch.k, Nc = N / 2;
  const int CX0 = cta.bx * kMfTileP, CY0 = cta.by * kMfTileP;
  MfCells f;
  f.ox = 2 * CX0 - K;
  f.oy = 2 * CY0 - K;
  f.w = 2 * kMfTileP + 2 * K;
  const int n = f.n();
  T* tab = reinterpret_cast<T*>(mf_sm);
  T* B = tab + ((kMfPresTab + 3) & ~3);
  T *Xc = B + 3 * n, *Xn = B + 6 * n, *Dc = B + 9 * n, *Dn = B + 12 * n;
  for (int i = cta.tid; i < kMfPresTab; i += cta.nthr) tab[i] = a.tab[i];
  MF_SYNC();
  const T* dv = tab + 729;
  for (int e = cta.tid; e < n; e += cta.nthr) {
    const int cx = f.ox + e % f.w, cy = f.oy + e / f.w;
    const bool in = mf_cin<T>(N, cx, cy);
    const int v = in ? mf_variant<T>(N, cx, cy) : 0;
    for (int k = 0; k < 3; ++k) {
      const T bv = in ? a.b[3 * ((size_t)cy * N + cx) + k] : (T)0;
      B[k * n + e] = bv;
      const T x0 = a.ch.c0 * dv[3 * v + k] * bv;
      Xc[k * n + e] = x0;
      Dc[k * n + e] = x0;
    }
  }
  MF_SYNC();
  for (int s = 1; s < K; ++s) {
    mf_pres_cheb<T>(cta, tab, N, f, s, B, Xc, Dc, Xn, Dn, false, a.ch.c1[s - 1], a.ch.c2[s - 1]);
    T* t = Xc; Xc = Xn; Xn = t;
    t = Dc; Dc = Dn; Dn = t;
    MF_SYNC();
  }
  // residual on the owned cells (frame shrunk by K), kept in the free direction buffer
  T* R = Dn;
  {
    const int m = f.w - 2 * K;
    for (int i = cta.tid; i < m * m; i += cta.nthr) {
      const int lx = K + i % m, ly = K + i / m, e = ly * f.w + lx;
      const int cx = f.ox + lx, cy = f.oy + ly;
      if (!mf_cin<T>(N, cx, cy)) {
        for (int k = 0; k < 3; ++k) R[k * n + e] = 0;
        continue;
      }
      T y[3];
      mf_pres_apply<T>(tab, Xc, f, N, cx, cy, e, y);
      const size_t id = 3 * ((size_t)cy * N + cx);
      for (int k = 0; k < 3; ++k) {
        R[k * n + e] = B[k * n + e] - y[k];
        a.xout[id + k] = Xc[k * n + e];
      }
    }
  }
  MF_SYNC();
  // restriction R = P^T to the tile's coarse cells: the children's
  // coefficients with the transposed P1disc blocks [1 sx sy; 0 1/2 0; 0 0 1/2]
  for (int i = cta.tid; i < kMfTileP * kMfTileP; i += cta.nthr) {
    const int X0 = CX0 + i % kMfTileP, Y0 = CY0 + i / kMfTileP;
    if (X0 >= Nc || Y0 >= Nc) continue;
    T s0 = 0, s1 = 0, s2 = 0;
    for (int j = 0; j < 4; ++j) {
      const int cx = 2 * X0 + (j & 1), cy = 2 * Y0 + (j >> 1);
      const int e = (cy - f.oy) * f.w + (cx - f.ox);
      const T sx = (j & 1) ? (T)0.25 : (T)-0.25, sy = (j >> 1) ? (T)0.25 : (T)-0.25;
      const T r0 = R[e], r1 = R[n + e], r2 = R[2 * n + e];
      s0 += r0;
      s1 += sx * r0 + (T)0.5 * r1;
      s2 += sy * r0 + (T)0.5 * r2;
    }
    const size_t id = 3 * ((size_t)Y0 * Nc + X0);
    a.bc[id] = s0;
    a.bc[id + 1] = s1;
    a.bc[id + 2] = s2;
    if (a.ci.x) {
      const T v[3] = {s0, s1, s2};
      for (int k = 0; k < 3; ++k) {
        const T d = a.ci.c0 * a.ci.dinv[id + k] * v[k];
        a.ci.x[id + k] = d;
        a.ci.d[id + k] = d;
      }
    }
  }
}

// up: grid (ceil(N / kMfTilePf))^2 over the fine cells
template <class T>
__host__ __device__ void mfp_up_body(const MfPresArgs<T>& a, const MfCta& cta) {
  unsigned char* mf_sm = cta.sm;
  const int N = a.N, K = a.ch.k, Nc = N / 2;
  const int FX0 = cta.bx * kMfTilePf, FY0 = cta.by * kMfTilePf;
  MfCells f;
  f.ox = FX0 - K;
  f.oy = FY0 - K;
  f.w = kMfTilePf + 2 * K;
  const int n = f.n();
  T* tab = reinterpret_cast<T*>(mf_sm);
  T* B = tab + ((kMfPresTab + 3) & ~3);
  T *Xc = B + 3 * n, *Xn = B + 6 * n, *Dc = B + 9 * n, *Dn = B + 12 * n;
  for (int i = cta.tid; i < kMfPresTab; i += cta.nthr) tab[i] = a.tab[i];
  // b and x + P x_coarse (each fine cell from its parent: [1 sx sy; 0 1/2 0; 0 0 1/2])
  for (int e = cta.tid; e < n; e += cta.nthr) {
    const int cx = f.ox + e % f.w, cy = f.oy + e / f.w;
    T bv[3] = {0, 0, 0}, xv[3] = {0, 0, 0};
    if (mf_cin<T>(N, cx, cy)) {
      const size_t id = 3 * ((size_t)cy * N + cx), pc = 3 * ((size_t)(cy >> 1) * Nc + (cx >> 1));
      const T sx = (cx & 1) ? (T)0.25 : (T)-0.25, sy = (cy & 1) ? (T)0.25 : (T)-0.25;
      const T c0 = a.xc[pc], c1 = a.xc[pc + 1], c2 = a.xc[pc + 2];
      const T p[3] = {c0 + sx * c1 + sy * c2, (T)0.5 * c1, (T)0.5 * c2};
      for (int k = 0; k < 3; ++k) {
        bv[k] = a.b[id + k];
        xv[k] = p[k] + a.xpre[id + k];
      }
    }
    for (int k = 0; k < 3; ++k) {
      B[k * n + e] = bv[k];
      Xc[k * n + e] = xv[k];
    }
  }
  MF_SYNC();
  const T* dv = tab + 729;
  for (int s = 0; s < K - 1; ++s) {
    mf_pres_cheb<T>(cta, tab, N, f, s + 1, B, Xc, Dc, Xn, Dn, s == 0,
                    s == 0 ? (T)0 : a.ch.c1[s - 1], s == 0 ? a.ch.c0 : a.ch.c2[s - 1]);
    T* t = Xc; Xc = Xn; Xn = t;
    t = Dc; Dc = Dn; Dn = t;
    MF_SYNC();
  }
  // last step on the owned cells, with the epilogue
  const int s = K - 1;
  const T c1 = s == 0 ? (T)0 : a.ch.c1[s - 1], c2 = s == 0 ? a.ch.c0 : a.ch.c2[s - 1];
  const int m = f.w - 2 * K;
  for (int i = cta.tid; i < m * m; i += cta.nthr) {
    const int lx = K + i % m, ly = K + i / m, e = ly * f.w + lx;
    const int cx = f.ox + lx, cy = f.oy + ly;
    if (!mf_cin<T>(N, cx, cy)) continue;
    T y[3];
    mf_pres_apply<T>(tab, Xc, f, N, cx, cy, e, y);
    const int v = mf_variant<T>(N, cx, cy);
    const size_t id = 3 * ((size_t)cy * N + cx);
    for (int k = 0; k < 3; ++k) {
      const T r = B[k * n + e] - y[k];
      const T dn = (s == 0) ? c2 * dv[3 * v + k] * r : c1 * Dc[k * n + e] + c2 * dv[3 * v + k] * r;
      const T yv = Xc[k * n + e] + dn;
      a.xout[id + k] = yv;
      T ov = yv;
      if (a.fin.sout) {
        ov = -(a.fin.snu * a.fin.smp[id + k] * a.fin.sv[id + k] + a.fin.srdt * yv);
        a.fin.sout[id + k] = ov;
      }
      if (a.fin.acc) a.fin.acc[id + k] += a.fin.omega * ov;
    }
  }
}

#ifdef __CUDACC__
// The kernels: one CTA of kMfThreads threads per tile.
#define FSI_MF_KERNEL(name, body, Args)                                      \
  template <class T>                                                         \
  __global__ void __launch_bounds__(kMfThreads) name(const __grid_constant__ Args<T> a) { \
    asm volatile("griddepcontrol.wait;" ::: "memory");                       \
    extern __shared__ __align__(16) unsigned char mf_smem[];                 \
    const MfCta c{(int)blockIdx.x, (int)blockIdx.y, (int)threadIdx.x, (int)blockDim.x, mf_smem}; \
    body<T>(a, c);                                                           \
  }
FSI_MF_KERNEL(k_mfu_down, mfu_down_body, MfVelArgs)
FSI_MF_KERNEL(k_mfu_up, mfu_up_body, MfVelArgs)
FSI_MF_KERNEL(k_mfp_down, mfp_down_body, MfPresArgs)
FSI_MF_KERNEL(k_mfp_up, mfp_up_body, MfPresArgs)
#undef FSI_MF_KERNEL
#endif

// shared memory of one launch (bytes)
template <class T>
inline size_t mfu_down_smem(int K) {
  const int w = 2 * kMfTileU + 8 + 4 * K;
  return 6 * (size_t)w * w * 2 * sizeof(T);
}
template <class T>
inline size_t mfu_up_smem(int K) {
  const int w = kMfTileUf + 4 * K;
  const int gw = 2 * ((w + 3) / 4 + 2);   // coarse frame side (upper bound)
  return (5 * (size_t)w * w + (size_t)gw * gw) * 2 * sizeof(T);
}
template <class T>
inline size_t mfp_down_smem(int K) {
  const int w = 2 * kMfTileP + 2 * K;
  return (((kMfPresTab + 3) & ~3) + 15 * (size_t)w * w) * sizeof(T);
}
template <class T>
inline size_t mfp_up_smem(int K) {
  const int w = kMfTilePf + 2 * K;
  return (((kMfPresTab + 3) & ~3) + 15 * (size_t)w * w) * sizeof(T);
}

}  // namespace fsi
