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
// Work is spread without integer division: a sweep gives each row of a
// rectangle to a group of 8, 16 or 32 lanes, and the velocity sweeps take
// the four node types as four blocks of rows padded so that a warp never
// straddles two of them; the type (and with it the whole stencil) is then a
// compile-time constant of the code a warp runs.
//
// Each kernel is a thin wrapper around a __host__ __device__ body that takes
// the CTA's coordinates explicitly.  A body loops over the "virtual threads"
// of the launch it is written for, strided by the threads that actually run
// it, and its phases are separated by barriers, so a body run by one thread
// per CTA computes the same values; the host test of these kernels runs the
// bodies that way.
#pragma once
#include <cstdlib>
#include <cuda_runtime.h>

#include <type_traits>

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

// the CTA a body works for: block coordinates, this thread, the threads that
// run the body (1 on the host), the threads of the launch (the body's
// virtual threads) and the dynamic shared memory
struct MfCta {
  int bx, by, tid, nthr, vthr;
  unsigned char* sm;
};

#ifdef __CUDA_ARCH__
#define MF_SYNC() __syncthreads()
#else
#define MF_SYNC() ((void)0)
#endif

__host__ __device__ __forceinline__ int mf_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int mf_max(int a, int b) { return a > b ? a : b; }

constexpr int kMfMaxDeg = 4;      // Chebyshev degrees 1..4 (the default is 2)
// pressure stencil table: per wall variant 9 blocks of 3x3, each padded to
// 12 values (16-byte aligned: three 16-byte loads per block), then D^-1
// (3 per variant)
constexpr int kMfPresBlk = 12;
constexpr int kMfPresVar = 9 * kMfPresBlk;
constexpr int kMfPresDinv = 9 * kMfPresVar;
constexpr int kMfPresTab = kMfPresDinv + 9 * 3;
// table index of block (dy + 1, dx + 1) = (y, x) of variant v
constexpr int mf_pres_blk(int v, int y, int x) { return kMfPresVar * v + kMfPresBlk * (3 * y + x); }

// Tile sizes by level: velocity down TC coarse lattice nodes a side (up:
// 2 TC fine lattice nodes), pressure down TP coarse cells (up: 2 TP fine
// cells).  A launch's time on these grids is mostly its fixed cost (launch,
// one global round trip, the barriers between its phases), not the work of
// the overlaps the tiles repeat: on the 128 x 128 cavity, tiles shrunk to
// keep 256 CTAs on every level measured slower (9.8 against 10.7 steps/s)
// than one tile size for all levels.  From 512 cells on, the larger tiles
// repeat less of their neighbours' work.
__host__ __device__ __forceinline__ int mf_tile_u(int N) { return N >= 512 ? 16 : 8; }
__host__ __device__ __forceinline__ int mf_tile_p(int N) { return N >= 512 ? 8 : 4; }
// Threads of a velocity launch.  A launch's time on these grids is one CTA's
// chain of phases, and the threads' share of a phase sets it.  The stencil
// sweeps give each thread two plane rows (mf_vsweep2), so 512 threads cover
// the smoothing and residual sweeps of an 8-node tile once; the loads and
// sweeps of whole frames take two rounds.  The 16-node tiles of the large
// grids use 512 as well (1024 measured slower there).  Down frames have
// TC + 8 plane entries a side (four planes), up frames TC + 4; a warp takes
// two rows of up to 16 entries, four rows of up to 8.
constexpr int mf_threads_ud(int tc) { return tc >= 16 ? 512 : (tc == 8 ? 512 : (tc == 4 ? 768 : 640)); }
constexpr int mf_threads_uu(int tc) { return tc >= 16 ? 512 : (tc == 8 ? 512 : (tc == 4 ? 256 : 192)); }
constexpr int mf_threads_p(int tp) { return tp >= 4 ? 256 : 128; }

// Call f(integral_constant<degree>) for a Chebyshev degree 1 .. kMfMaxDeg
// (the frame sizes and the step loops of the kernels are compile-time).
template <class F>
inline void mf_with_degree(int K, F&& f) {
  switch (K) {
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    case 3: f(std::integral_constant<int, 3>()); break;
    default: f(std::integral_constant<int, 4>()); break;
  }
}

// Call f(integral_constant<tile>) with the tile of the level.
template <class F>
inline void mf_with_tile_u(int N, F&& f) {
  switch (mf_tile_u(N)) {
    case 16: f(std::integral_constant<int, 16>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    default: f(std::integral_constant<int, 2>()); break;
  }
}
template <class F>
inline void mf_with_tile_p(int N, F&& f) {
  switch (mf_tile_p(N)) {
    case 8: f(std::integral_constant<int, 8>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    default: f(std::integral_constant<int, 1>()); break;
  }
}

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

// Residual start of a finest-level down launch inside a Richardson step on
// the Stokes block (Section 5): the level's right-hand side is the Stokes
// residual of the current iterate, computed on the tile's frame from the
// input b (the Richardson input r), the velocity iterate zu and the pressure
// iterate zp (either null: zero):
//   velocity: b - A_f zu - (-B^T) zp,   pressure: b - (-B) zu.
// Its owned part goes to bout, which the up launch reads as its b.
template <class T>
struct MfRes {
  const T* zu = nullptr;
  const T* zp = nullptr;
  T* bout = nullptr;
  T divB[3][9][2];          // entries of -B and -B^T: [pressure dof][node of the cell][component]
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
  MfRes<T> res;             // down: residual start when res.zu or res.zp
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
  MfRes<T> res;             // down: residual start when res.zu (res.zp unused)
};

// Quadratic Lagrange basis on [0, 1] (nodes 0, 1/2, 1) at t; exact in
// binary floating point at the quarter points the transfers use.
__host__ __device__ __forceinline__ float mf_l0(float t) { return (1.f - t) * (1.f - 2.f * t); }
__host__ __device__ __forceinline__ float mf_l1(float t) { return 4.f * t * (1.f - t); }
__host__ __device__ __forceinline__ float mf_l2(float t) { return t * (2.f * t - 1.f); }

// ------------------------------------------------------------------ sweeps
// fn(x, y) for every (x, y) in [0, nx) x [0, ny): groups of cw = 2^sh lanes
// (the smallest of 8, 16, 32 that holds a row) take one row each.
template <class F>
__host__ __device__ __forceinline__ void mf_rows(const MfCta& c, int nx, int ny, F&& fn) {
  const int sh = nx <= 8 ? 3 : (nx <= 16 ? 4 : 5);
  const int cw = 1 << sh, rpw = 32 >> sh, step = (c.vthr >> 5) * rpw;
  for (int t = c.tid; t < c.vthr; t += c.nthr) {
    const int lane = t & 31;
    for (int y = (t >> 5) * rpw + (lane >> sh); y < ny; y += step)
      for (int x = lane & (cw - 1); x < nx; x += cw) fn(x, y);
  }
}

// fn(type, px, py) over the plane rectangle [qx0, qx1) x [qy0, qy1) of all
// four planes, the type as std::integral_constant: each plane's rows are
// padded to a multiple of the rows a warp takes, so a warp stays in one plane.
template <class F>
__host__ __device__ __forceinline__ void mf_vsweep(const MfCta& c, int qx0, int qx1, int qy0, int qy1, F&& fn) {
  const int nqx = qx1 - qx0, nqy = qy1 - qy0;
  const int sh = nqx <= 8 ? 3 : (nqx <= 16 ? 4 : 5);
  const int cw = 1 << sh, rsh = 5 - sh, rpw = 1 << rsh;
  const int nyp = ((nqy + rpw - 1) >> rsh) << rsh;
  const int nrow = 4 * nyp, step = (c.vthr >> 5) * rpw;
  for (int t = c.tid; t < c.vthr; t += c.nthr) {
    const int lane = t & 31;
    for (int yy = (t >> 5) * rpw + (lane >> sh); yy < nrow; yy += step) {
      const int tau = (yy >= nyp) + (yy >= 2 * nyp) + (yy >= 3 * nyp);
      const int y = yy - tau * nyp;
      if (y >= nqy) continue;
      for (int x = lane & (cw - 1); x < nqx; x += cw) {
        switch (tau) {
          case 0: fn(std::integral_constant<int, 0>(), qx0 + x, qy0 + y); break;
          case 1: fn(std::integral_constant<int, 1>(), qx0 + x, qy0 + y); break;
          case 2: fn(std::integral_constant<int, 2>(), qx0 + x, qy0 + y); break;
          default: fn(std::integral_constant<int, 3>(), qx0 + x, qy0 + y); break;
        }
      }
    }
  }
}

// fn(type, px, py) over the same rectangle, a thread taking the two
// entries (px, py) and (px, py + 1) of a plane: fn computes both, so that
// the stencil taps the two share (two of three plane rows) and their
// coefficients are loaded once.  The row count of the rectangle is even
// (every frame side and shrink used here keeps it so).
template <class F>
__host__ __device__ __forceinline__ void mf_vsweep2(const MfCta& c, int qx0, int qx1, int qy0, int qy1, F&& fn) {
  const int nqx = qx1 - qx0, npr = (qy1 - qy0) >> 1;
#ifndef __CUDA_ARCH__
  if ((qy1 - qy0) & 1) std::abort();
#endif
  const int sh = nqx <= 8 ? 3 : (nqx <= 16 ? 4 : 5);
  const int cw = 1 << sh, rsh = 5 - sh, rpw = 1 << rsh;
  const int nyp = ((npr + rpw - 1) >> rsh) << rsh;
  const int nrow = 4 * nyp, step = (c.vthr >> 5) * rpw;
  for (int t = c.tid; t < c.vthr; t += c.nthr) {
    const int lane = t & 31;
    for (int yy = (t >> 5) * rpw + (lane >> sh); yy < nrow; yy += step) {
      const int tau = (yy >= nyp) + (yy >= 2 * nyp) + (yy >= 3 * nyp);
      const int y = yy - tau * nyp;
      if (y >= npr) continue;
      for (int x = lane & (cw - 1); x < nqx; x += cw) {
        switch (tau) {
          case 0: fn(std::integral_constant<int, 0>(), qx0 + x, qy0 + 2 * y); break;
          case 1: fn(std::integral_constant<int, 1>(), qx0 + x, qy0 + 2 * y); break;
          case 2: fn(std::integral_constant<int, 2>(), qx0 + x, qy0 + 2 * y); break;
          default: fn(std::integral_constant<int, 3>(), qx0 + x, qy0 + 2 * y); break;
        }
      }
    }
  }
}

// --------------------------------------------------------------- velocity
// interior Q2 node (1 <= ix, iy <= 2N-1) -> id in the type-blocked order
// (corners, x-edge midpoints, y-edge midpoints, centres; lattice order inside)
template <int TAU>
__host__ __device__ __forceinline__ int mf_vnode_t(int N, int ix, int iy) {
  const int nV = (N - 1) * (N - 1), nX = N * (N - 1);
  if (TAU == 0) return ((iy >> 1) - 1) * (N - 1) + ((ix >> 1) - 1);
  if (TAU == 1) return nV + ((iy >> 1) - 1) * N + (ix >> 1);
  if (TAU == 2) return nV + nX + (iy >> 1) * (N - 1) + ((ix >> 1) - 1);
  return nV + 2 * nX + (iy >> 1) * N + (ix >> 1);
}

__host__ __device__ __forceinline__ int mf_vnode(int N, int ix, int iy) {
  switch ((ix & 1) | ((iy & 1) << 1)) {
    case 0: return mf_vnode_t<0>(N, ix, iy);
    case 1: return mf_vnode_t<1>(N, ix, iy);
    case 2: return mf_vnode_t<2>(N, ix, iy);
    default: return mf_vnode_t<3>(N, ix, iy);
  }
}

__host__ __device__ __forceinline__ bool mf_vinterior(int N, int ix, int iy) {
  return ix >= 1 && iy >= 1 && ix <= 2 * N - 1 && iy <= 2 * N - 1;
}

// a b + c in one rounding on the device (a multiply-add the stencil sums are
// chains of); the host emulation rounds twice
template <class T>
__host__ __device__ __forceinline__ T mf_fma(T a, T b, T c) {
#ifdef __CUDA_ARCH__
  return fma(a, b, c);
#else
  return a * b + c;
#endif
}

// A lattice frame in shared memory: origin (ox, oy) even, 4 parity planes
// (one per node type) of pw x ph entries; lattice (ox + 2 px + (t & 1),
// oy + 2 py + (t >> 1)) is entry (t ph + py) pw + px.  MfFrame has run-time
// sides; MfFrameT<PW, PH> compile-time ones, so that every stencil tap is a
// constant offset from the node's entry.
struct MfFrame {
  int ox, oy, pw, ph;
  __host__ __device__ __forceinline__ int plane() const { return pw * ph; }
  __host__ __device__ __forceinline__ int at(int t, int px, int py) const { return (t * ph + py) * pw + px; }
  __host__ __device__ __forceinline__ int at_lattice(int ix, int iy) const {
    return at((ix & 1) | ((iy & 1) << 1), (ix - ox) >> 1, (iy - oy) >> 1);
  }
};
template <int PW, int PH>
struct MfFrameT {
  int ox, oy;
  static constexpr int pw = PW, ph = PH;
  __host__ __device__ static constexpr int plane() { return PW * PH; }
  __host__ __device__ static constexpr int at(int t, int px, int py) { return (t * PH + py) * PW + px; }
  __host__ __device__ __forceinline__ int at_lattice(int ix, int iy) const {
    return at((ix & 1) | ((iy & 1) << 1), (ix - ox) >> 1, (iy - oy) >> 1);
  }
};

// y = A v at the node of type TAU with plane coordinates (px, py) of frame
// f; the neighbours of even and odd rows go to two accumulator pairs (two
// shorter dependency chains of multiply-adds), added at the end
template <class T, int TAU, class F>
__host__ __device__ __forceinline__ void mf_vel_apply(const MfVelOp<T>& op, const typename Vec2<T>::type* __restrict__ v,
                                                      const F& f, int px, int py, T& y0, T& y1) {
  constexpr int PX = TAU & 1, PY = TAU >> 1;
  constexpr int RX = PX ? 1 : 2, RY = PY ? 1 : 2;
  T a0 = 0, a1 = 0, b0 = 0, b1 = 0;
  const typename Vec2<T>::type* __restrict__ w = v + f.at(0, px, py);
#pragma unroll
  for (int dy = -RY; dy <= RY; ++dy) {
#pragma unroll
    for (int dx = -RX; dx <= RX; ++dx) {
      const int t2 = ((PX + dx) & 1) | (((PY + dy) & 1) << 1);
      const auto x = w[(t2 * f.ph + ((PY + dy) >> 1)) * f.pw + ((PX + dx) >> 1)];
      const T* c = op.c[TAU][dy + 2][dx + 2];
      if ((dy & 1) == 0) {
        a0 = mf_fma(c[1], x.y, mf_fma(c[0], x.x, a0));
        a1 = mf_fma(c[3], x.y, mf_fma(c[2], x.x, a1));
      } else {
        b0 = mf_fma(c[1], x.y, mf_fma(c[0], x.x, b0));
        b1 = mf_fma(c[3], x.y, mf_fma(c[2], x.x, b1));
      }
    }
  }
  y0 = a0 + b0;
  y1 = a1 + b1;
}

// One Chebyshev step on the plane rectangle shrunk by `s` from the frame:
// first (CHEB0 / after init): dn = c2 D^-1 (b - A xo); otherwise
// dn = c1 do + c2 D^-1 (b - A xo); xn = xo + dn.  Outside the interior 0.
template <class T, class F>
__host__ __device__ __forceinline__ void mf_vel_cheb(const MfCta& cta, const MfVelOp<T>& op, const F& f, int s,
                                                     const typename Vec2<T>::type* __restrict__ B,
                                                     const typename Vec2<T>::type* __restrict__ Xo,
                                                     const typename Vec2<T>::type* __restrict__ Do,
                                                     typename Vec2<T>::type* __restrict__ Xn,
                                                     typename Vec2<T>::type* __restrict__ Dn, bool first, T c1, T c2) {
  using T2 = typename Vec2<T>::type;
  const int N = op.N;
  // two plane rows per thread: A applied at both (the reads stay inside the
  // frame since s >= 1; outside the interior the result is not used)
  mf_vsweep2(cta, s, f.pw - s, s, f.ph - s, [&](auto tc, int px, int py) {
    constexpr int TAU = decltype(tc)::value;
    T a[2][2];
    mf_vel_apply<T, TAU>(op, Xo, f, px, py, a[0][0], a[0][1]);
    mf_vel_apply<T, TAU>(op, Xo, f, px, py + 1, a[1][0], a[1][1]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int qy = py + k;
      const int ix = f.ox + 2 * px + (TAU & 1), iy = f.oy + 2 * qy + (TAU >> 1);
      const int e = f.at(TAU, px, qy);
      T2 xn, dn;
      if (mf_vinterior(N, ix, iy)) {
        const T2 b = B[e], xo = Xo[e];
        const T r0 = b.x - a[k][0], r1 = b.y - a[k][1];
        if (first) {
          dn.x = c2 * op.dinv[TAU][0] * r0;
          dn.y = c2 * op.dinv[TAU][1] * r1;
        } else {
          const T2 d = Do[e];
          dn.x = c1 * d.x + c2 * op.dinv[TAU][0] * r0;
          dn.y = c1 * d.y + c2 * op.dinv[TAU][1] * r1;
        }
        xn.x = xo.x + dn.x;
        xn.y = xo.y + dn.y;
      } else {
        xn.x = xn.y = dn.x = dn.y = 0;
      }
      Xn[e] = xn;
      Dn[e] = dn;
    }
  });
}

// y += (-B^T zp) at the interior node (ix, iy) of type TAU: the sum over the
// node's cells (one or two per direction: an odd lattice index lies inside a
// cell, at local node 1; an even one on the edge between two, at local node 2
// of the lower and 0 of the upper), lower cells first.  zp holds the three
// values of cell (cx, cy) at 3 ((cy - cy0) stride + cx - cx0): the global
// vector (0, 0, N) or a copy of the cells around a frame.
template <class T, int TAU>
__host__ __device__ __forceinline__ void mf_vel_btp(const MfRes<T>& r, const T* __restrict__ zp, int cx0, int cy0,
                                                    int stride, int ix, int iy, T& y0, T& y1) {
  constexpr int PX = TAU & 1, PY = TAU >> 1;
#pragma unroll
  for (int j = 0; j < (PY ? 1 : 2); ++j) {
#pragma unroll
    for (int i = 0; i < (PX ? 1 : 2); ++i) {
      const int aa = PX ? 1 : (i == 0 ? 2 : 0), ab = PY ? 1 : (j == 0 ? 2 : 0);
      const int cx = (ix - aa) >> 1, cy = (iy - ab) >> 1, al = 3 * ab + aa;
      const T* __restrict__ p = zp + 3 * ((size_t)(cy - cy0) * stride + (cx - cx0));
      const T p0 = p[0], p1 = p[1], p2 = p[2];
      y0 += r.divB[0][al][0] * p0 + r.divB[1][al][0] * p1 + r.divB[2][al][0] * p2;
      y1 += r.divB[0][al][1] * p0 + r.divB[1][al][1] * p1 + r.divB[2][al][1] * p2;
    }
  }
}

// down: grid (ceil(N / TC))^2 over the coarse lattice [0, N)^2
template <class T, int TC, int K>
__host__ __device__ void mfu_down_body(const MfVelArgs<T>& a, const MfCta& cta) {
  using T2 = typename Vec2<T>::type;
  const MfVelOp<T>& op = a.op;
  const int N = op.N;
  const int CX0 = cta.bx * TC, CY0 = cta.by * TC;
  constexpr int PW = TC + 4 + 2 * K;   // (2 TC + 8 + 4 K) lattice nodes a side
  MfFrameT<PW, PW> f;
  f.ox = 2 * CX0 - 4 - 2 * K;
  f.oy = 2 * CY0 - 4 - 2 * K;
  constexpr int nf = 4 * PW * PW;
  T2* B = reinterpret_cast<T2*>(cta.sm);
  T2 *Xc = B + nf, *Xn = B + 2 * nf, *Dc = B + 3 * nf, *Dn = B + 4 * nf;   // current / next iterate
  T2* R = B + 5 * nf;
  const int o = 2 + K;   // owned fine nodes: plane entries [o, o + TC) of the frame
  const MfRes<T>& rs = a.res;
  // residual start: the velocity iterate on the frame grown by one plane
  // entry (two lattice nodes, the reach of A), in Dn and R, which are
  // contiguous and unused until the smoothing (2 nf = 8 pw^2 entries, at
  // least 4 (pw + 2)^2 since pw >= 8)
  MfFrameT<PW + 2, PW + 2> g;
  g.ox = f.ox - 2;
  g.oy = f.oy - 2;
  T2* Z = Dn;
  static_assert(TC + 4 + 2 * K >= 8, "the grown frame must fit in Dn and R");
  // With zu, the frame's b and the pressure of the cells around the frame
  // (cells f.ox / 2 - 1 .. f.ox / 2 + PW - 1, PW + 1 a side, after Z when they
  // fit) come in the same phase, so the launch makes one global round trip
  // before its first barrier.
  constexpr int ZPW = PW + 1;
  constexpr bool zp_frame = 4 * (PW + 2) * (PW + 2) * 2 + 3 * ZPW * ZPW <= 2 * nf * 2;
  T* ZP = reinterpret_cast<T*>(Z + 4 * (PW + 2) * (PW + 2));
  const int zcx0 = (f.ox >> 1) - 1, zcy0 = (f.oy >> 1) - 1;
  const bool zp_smem = zp_frame && rs.zu && rs.zp;
  if (rs.zu) {
    mf_vsweep(cta, 0, g.pw, 0, g.ph, [&](auto tc, int px, int py) {
      constexpr int TAU = decltype(tc)::value;
      const int ix = g.ox + 2 * px + (TAU & 1), iy = g.oy + 2 * py + (TAU >> 1);
      T2 v;
      v.x = v.y = 0;
      if (mf_vinterior(N, ix, iy)) v = *reinterpret_cast<const T2*>(rs.zu + 2 * (size_t)mf_vnode_t<TAU>(N, ix, iy));
      Z[g.at(TAU, px, py)] = v;
    });
    mf_vsweep(cta, 0, f.pw, 0, f.ph, [&](auto tc, int px, int py) {
      constexpr int TAU = decltype(tc)::value;
      const int ix = f.ox + 2 * px + (TAU & 1), iy = f.oy + 2 * py + (TAU >> 1);
      T2 v;
      v.x = v.y = 0;
      if (mf_vinterior(N, ix, iy)) v = *reinterpret_cast<const T2*>(a.b + 2 * (size_t)mf_vnode_t<TAU>(N, ix, iy));
      B[f.at(TAU, px, py)] = v;
    });
    if (zp_smem)
      mf_rows(cta, ZPW, ZPW, [&](int i, int j) {
        const int cx = zcx0 + i, cy = zcy0 + j;
        const bool in = cx >= 0 && cy >= 0 && cx < N && cy < N;
#pragma unroll
        for (int k = 0; k < 3; ++k) ZP[3 * (j * ZPW + i) + k] = in ? rs.zp[3 * ((size_t)cy * N + cx) + k] : (T)0;
      });
    MF_SYNC();
  }
  // b on the frame (with the residual start: b - A zu - (-B^T) zp, its owned
  // part to rs.bout); x0 = d0 = c0 D^-1 b
  mf_vsweep(cta, 0, f.pw, 0, f.ph, [&](auto tc, int px, int py) {
    constexpr int TAU = decltype(tc)::value;
    const int ix = f.ox + 2 * px + (TAU & 1), iy = f.oy + 2 * py + (TAU >> 1);
    const int e = f.at(TAU, px, py);
    T2 v;
    v.x = v.y = 0;
    if (mf_vinterior(N, ix, iy)) {
      const size_t id = 2 * (size_t)mf_vnode_t<TAU>(N, ix, iy);
      v = rs.zu ? B[e] : *reinterpret_cast<const T2*>(a.b + id);
      if (rs.zu || rs.zp) {
        T y0 = 0, y1 = 0;
        if (rs.zu) mf_vel_apply<T, TAU>(op, Z, g, px + 1, py + 1, y0, y1);
        if (zp_smem) mf_vel_btp<T, TAU>(rs, ZP, zcx0, zcy0, ZPW, ix, iy, y0, y1);
        else if (rs.zp) mf_vel_btp<T, TAU>(rs, rs.zp, 0, 0, N, ix, iy, y0, y1);
        v.x -= y0;
        v.y -= y1;
        if (px >= o && px < o + TC && py >= o && py < o + TC) *reinterpret_cast<T2*>(rs.bout + id) = v;
      }
    }
    B[e] = v;
    T2 x0;
    x0.x = a.ch.c0 * op.dinv[TAU][0] * v.x;
    x0.y = a.ch.c0 * op.dinv[TAU][1] * v.y;
    Xc[e] = x0;
    Dc[e] = x0;
  });
  MF_SYNC();
  for (int s = 1; s < K; ++s) {  // pre-smoothing steps 1 .. K-1 on the frame shrunk by s nodes per plane
    mf_vel_cheb<T>(cta, op, f, s, B, Xc, Dc, Xn, Dn, false, a.ch.c1[s - 1], a.ch.c2[s - 1]);
    T2* t = Xc; Xc = Xn; Xn = t;
    t = Dc; Dc = Dn; Dn = t;
    MF_SYNC();
  }
  // residual on the frame shrunk by K (plane units): the restriction's
  // support; the pre-smoothed iterate on the owned fine nodes [2 CX0, 2 CX0
  // + 2 tile), plane entries [o, o + tile), goes out in the same sweep
  mf_vsweep2(cta, K, f.pw - K, K, f.ph - K, [&](auto tc, int px, int py) {
    constexpr int TAU = decltype(tc)::value;
    T ap[2][2];
    mf_vel_apply<T, TAU>(op, Xc, f, px, py, ap[0][0], ap[0][1]);
    mf_vel_apply<T, TAU>(op, Xc, f, px, py + 1, ap[1][0], ap[1][1]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int qy = py + k;
      const int ix = f.ox + 2 * px + (TAU & 1), iy = f.oy + 2 * qy + (TAU >> 1);
      const int e = f.at(TAU, px, qy);
      T2 r;
      r.x = r.y = 0;
      if (mf_vinterior(N, ix, iy)) {
        r.x = B[e].x - ap[k][0];
        r.y = B[e].y - ap[k][1];
        if (px >= o && px < o + TC && qy >= o && qy < o + TC)
          *reinterpret_cast<T2*>(a.xout + 2 * (size_t)mf_vnode_t<TAU>(N, ix, iy)) = Xc[e];
      }
      R[e] = r;
    }
  });
  MF_SYNC();
  // restriction to the coarse nodes of the tile (coarse lattice interior
  // 1 .. N - 1).  The weight of a fine node at (2X + dx, 2Y + dy) is the
  // product of 1-D weights, each the coarse quadratic of its node there:
  // L0(|d| / 4) at a cell corner, L1((d + 2) / 4) at an edge or cell midpoint
  // (|d| <= 1).  So the sum is taken in two passes, along x into the free
  // buffer Xn (fine rows 2 CY0 - 3 .. 2 CY0 + 2 TC + 1 by coarse columns),
  // then along y.
  const int Nc = N / 2;
  constexpr int RR = 2 * TC + 5;
  T2* Rx = Xn;
  mf_rows(cta, TC, RR, [&](int i, int j) {
    const int X0 = CX0 + i, iy = 2 * CY0 - 3 + j;
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int dx = -3; dx <= 3; ++dx) {
      const float tx = (X0 & 1) ? 0.25f * (float)(dx + 2) : 0.25f * (float)(dx < 0 ? -dx : dx);
      const T wx = (X0 & 1) ? ((dx >= -1 && dx <= 1) ? (T)mf_l1(tx) : (T)0) : (T)mf_l0(tx);
      if (wx == (T)0) continue;
      const T2 r = R[f.at_lattice(2 * X0 + dx, iy)];
      s0 += wx * r.x;
      s1 += wx * r.y;
    }
    T2 v;
    v.x = s0;
    v.y = s1;
    Rx[j * TC + i] = v;
  });
  MF_SYNC();
  mf_rows(cta, TC, TC, [&](int i, int j) {
    const int X0 = CX0 + i, Y0 = CY0 + j;
    if (!mf_vinterior(Nc, X0, Y0)) return;
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int dy = -3; dy <= 3; ++dy) {
      const float ty = (Y0 & 1) ? 0.25f * (float)(dy + 2) : 0.25f * (float)(dy < 0 ? -dy : dy);
      const T wy = (Y0 & 1) ? ((dy >= -1 && dy <= 1) ? (T)mf_l1(ty) : (T)0) : (T)mf_l0(ty);
      if (wy == (T)0) continue;
      const T2 r = Rx[(2 * j + 3 + dy) * TC + i];   // fine row 2 Y0 + dy
      s0 += wy * r.x;
      s1 += wy * r.y;
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
  });
}

// up: grid (ceil(2N / (2 TC)))^2 over the fine lattice [0, 2N)^2
template <class T, int TC, int K>
__host__ __device__ void mfu_up_body(const MfVelArgs<T>& a, const MfCta& cta) {
  using T2 = typename Vec2<T>::type;
  constexpr int TF = 2 * TC;
  const MfVelOp<T>& op = a.op;
  const int N = op.N, Nc = N / 2;
  const int FX0 = cta.bx * TF, FY0 = cta.by * TF;
  constexpr int PW = TC + 2 * K;   // (TF + 4 K) lattice nodes a side
  MfFrameT<PW, PW> f;
  f.ox = FX0 - 2 * K;
  f.oy = FY0 - 2 * K;
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
  constexpr int nf = 4 * PW * PW;
  T2* B = reinterpret_cast<T2*>(cta.sm);
  T2 *Xc = B + nf, *Xn = B + 2 * nf, *Dc = B + 3 * nf, *Dn = B + 4 * nf;
  T2* XC = B + 5 * nf;
  mf_vsweep(cta, 0, g.pw, 0, g.ph, [&](auto tc, int px, int py) {
    constexpr int TAU = decltype(tc)::value;
    const int ix = g.ox + 2 * px + (TAU & 1), iy = g.oy + 2 * py + (TAU >> 1);
    T2 v;
    v.x = v.y = 0;
    if (mf_vinterior(Nc, ix, iy)) v = *reinterpret_cast<const T2*>(a.xc + 2 * (size_t)mf_vnode_t<TAU>(Nc, ix, iy));
    XC[g.at(TAU, px, py)] = v;
  });
  MF_SYNC();
  // b and x + P x_coarse on the frame: the coarse quadratic of the coarse
  // cell cc = min(ix / 4, Nc - 1) at t = (ix - 4 cc) / 4 in each direction
  mf_vsweep(cta, 0, f.pw, 0, f.ph, [&](auto tc, int px, int py) {
    constexpr int TAU = decltype(tc)::value;
    const int ix = f.ox + 2 * px + (TAU & 1), iy = f.oy + 2 * py + (TAU >> 1);
    T2 bv, xv;
    bv.x = bv.y = xv.x = xv.y = 0;
    if (mf_vinterior(N, ix, iy)) {
      const size_t id = mf_vnode_t<TAU>(N, ix, iy);
      bv = *reinterpret_cast<const T2*>(a.b + 2 * id);
      xv = *reinterpret_cast<const T2*>(a.xpre + 2 * id);
      const int ccx = mf_min(ix >> 2, Nc - 1), ccy = mf_min(iy >> 2, Nc - 1);
      const float tx = 0.25f * (float)(ix - 4 * ccx), ty = 0.25f * (float)(iy - 4 * ccy);
      const T wx[3] = {(T)mf_l0(tx), (T)mf_l1(tx), (T)mf_l2(tx)};
      const T wy[3] = {(T)mf_l0(ty), (T)mf_l1(ty), (T)mf_l2(ty)};
      T p0 = 0, p1 = 0;
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) {
          const T w = wx[aa] * wy[bb];
          const T2 c = XC[g.at_lattice(2 * ccx + aa, 2 * ccy + bb)];
          p0 += w * c.x;
          p1 += w * c.y;
        }
      }
      xv.x = p0 + xv.x;
      xv.y = p1 + xv.y;
    }
    const int e = f.at(TAU, px, py);
    B[e] = bv;
    Xc[e] = xv;
  });
  MF_SYNC();
  // The Richardson update of the last step reads the iterate it adds to.
  // With K >= 2 those reads go out in the phase before the last step, into
  // the coarse frame's buffer (free after the prolongation; the owned tile,
  // TC x TC entries per plane, fits in it for the 8-node tile), so the last
  // step makes no global round trip of its own.
  constexpr int GW = 2 * ((2 * TC + 4 * K + 3) / 4 + 2);
  constexpr bool acc_pre = K >= 2 && 4 * TC * TC <= GW * GW;
  T2* ACC = XC;
  for (int s = 0; s + 1 < K; ++s) {  // post-smoothing: CHEB0, then CHEB steps, each on a frame 1 plane entry smaller
    if (acc_pre && s + 2 == K && a.fin.acc)
      mf_vsweep(cta, K, f.pw - K, K, f.ph - K, [&](auto tc, int px, int py) {
        constexpr int TAU = decltype(tc)::value;
        const int ix = f.ox + 2 * px + (TAU & 1), iy = f.oy + 2 * py + (TAU >> 1);
        if (!mf_vinterior(N, ix, iy)) return;
        const size_t id = mf_vnode_t<TAU>(N, ix, iy);
        ACC[(TAU * TC + py - K) * TC + px - K] = *reinterpret_cast<const T2*>(a.fin.acc + 2 * id);
      });
    mf_vel_cheb<T>(cta, op, f, s + 1, B, Xc, Dc, Xn, Dn, s == 0,
                   s == 0 ? (T)0 : a.ch.c1[s - 1], s == 0 ? a.ch.c0 : a.ch.c2[s - 1]);
    T2* t = Xc; Xc = Xn; Xn = t;
    t = Dc; Dc = Dn; Dn = t;
    MF_SYNC();
  }
  // last step on the owned tile: write the result and the epilogue
  const int s = K - 1;
  const T c1 = s == 0 ? (T)0 : a.ch.c1[s - 1], c2 = s == 0 ? a.ch.c0 : a.ch.c2[s - 1];
  mf_vsweep2(cta, K, f.pw - K, K, f.ph - K, [&](auto tc, int px, int py) {
    constexpr int TAU = decltype(tc)::value;
    T ap[2][2];
    mf_vel_apply<T, TAU>(op, Xc, f, px, py, ap[0][0], ap[0][1]);
    mf_vel_apply<T, TAU>(op, Xc, f, px, py + 1, ap[1][0], ap[1][1]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int qy = py + k;
      const int ix = f.ox + 2 * px + (TAU & 1), iy = f.oy + 2 * qy + (TAU >> 1);
      if (!mf_vinterior(N, ix, iy)) continue;
      const int e = f.at(TAU, px, qy);
      const T2 b = B[e], xo = Xc[e];
      const T r0 = b.x - ap[k][0], r1 = b.y - ap[k][1];
      T d0 = c2 * op.dinv[TAU][0] * r0, d1 = c2 * op.dinv[TAU][1] * r1;
      if (s > 0) {
        const T2 d = Dc[e];
        d0 = c1 * d.x + c2 * op.dinv[TAU][0] * r0;
        d1 = c1 * d.y + c2 * op.dinv[TAU][1] * r1;
      }
      const size_t id = mf_vnode_t<TAU>(N, ix, iy);
      const T y0 = xo.x + d0, y1 = xo.y + d1;
      T2 y;
      y.x = y0;
      y.y = y1;
      *reinterpret_cast<T2*>(a.xout + 2 * id) = y;
      if (a.fin.acc) {
        T2 z;
        if (acc_pre) z = ACC[(TAU * TC + qy - K) * TC + px - K];
        else z = *reinterpret_cast<const T2*>(a.fin.acc + 2 * id);
        z.x += a.fin.omega * y0;
        z.y += a.fin.omega * y1;
        *reinterpret_cast<T2*>(a.fin.acc + 2 * id) = z;
      }
    }
  });
}

// --------------------------------------------------------------- pressure
// A cell frame in shared memory: origin (ox, oy), w x w cells, three planes
// (one per P1disc coefficient).
struct MfCells {
  int ox, oy, w;
  __host__ __device__ __forceinline__ int n() const { return w * w; }
};

__host__ __device__ __forceinline__ int mf_variant(int N, int cx, int cy) {
  const int vx = cx == 0 ? 0 : (cx == N - 1 ? 2 : 1), vy = cy == 0 ? 0 : (cy == N - 1 ? 2 : 1);
  return 3 * vy + vx;
}

__host__ __device__ __forceinline__ bool mf_cin(int N, int cx, int cy) {
  return cx >= 0 && cy >= 0 && cx < N && cy < N;
}

// the 12 values of a padded pressure block from shared memory (16-byte aligned)
template <class T>
__host__ __device__ __forceinline__ void mf_load12(const T* __restrict__ p, T c[12]);
template <>
__host__ __device__ __forceinline__ void mf_load12<float>(const float* __restrict__ p, float c[12]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 v = reinterpret_cast<const float4*>(p)[k];
    c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
  }
}
template <>
__host__ __device__ __forceinline__ void mf_load12<double>(const double* __restrict__ p, double c[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 v = reinterpret_cast<const double2*>(p)[k];
    c[2 * k] = v.x; c[2 * k + 1] = v.y;
  }
}

// y = L v at cell (cx, cy) (frame entry e) with the stencil table in shared
// memory; the three cell rows go to separate partial sums
template <class T>
__host__ __device__ __forceinline__ void mf_pres_apply(const T* __restrict__ tab, const T* __restrict__ v,
                                                       const MfCells& f, int N, int cx, int cy, int e, T y[3]) {
  const T* base = tab + kMfPresVar * mf_variant(N, cx, cy);
  const int n = f.n();
  T p[3][3];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int i = 0; i < 3; ++i) p[dy + 1][i] = 0;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int q = e + dy * f.w + dx;
      const T x0 = v[q], x1 = v[n + q], x2 = v[2 * n + q];
      T c[kMfPresBlk];
      mf_load12<T>(base + kMfPresBlk * ((dy + 1) * 3 + dx + 1), c);
#pragma unroll
      for (int i = 0; i < 3; ++i) p[dy + 1][i] = mf_fma(c[3 * i + 2], x2, mf_fma(c[3 * i + 1], x1, mf_fma(c[3 * i], x0, p[dy + 1][i])));
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = (p[0][i] + p[1][i]) + p[2][i];
}

// one Chebyshev step on the cell frame shrunk by s cells
template <class T>
__host__ __device__ __forceinline__ void mf_pres_cheb(const MfCta& cta, const T* __restrict__ tab, int N,
                                                      const MfCells& f, int s, const T* __restrict__ B,
                                                      const T* __restrict__ Xo, const T* __restrict__ Do,
                                                      T* __restrict__ Xn, T* __restrict__ Dn, bool first, T c1, T c2) {
  const int m = f.w - 2 * s, n = f.n();
  const T* dv = tab + kMfPresDinv;
  mf_rows(cta, m, m, [&](int i, int j) {
    const int lx = s + i, ly = s + j, e = ly * f.w + lx;
    const int cx = f.ox + lx, cy = f.oy + ly;
    if (!mf_cin(N, cx, cy)) {
      for (int k = 0; k < 3; ++k) Xn[k * n + e] = Dn[k * n + e] = 0;
      return;
    }
    T y[3];
    mf_pres_apply<T>(tab, Xo, f, N, cx, cy, e, y);
    const int v = mf_variant(N, cx, cy);
    for (int k = 0; k < 3; ++k) {
      const T r = B[k * n + e] - y[k];
      const T dn = first ? c2 * dv[3 * v + k] * r : c1 * Do[k * n + e] + c2 * dv[3 * v + k] * r;
      Dn[k * n + e] = dn;
      Xn[k * n + e] = Xo[k * n + e] + dn;
    }
  });
}

// b -= (-B zu) at cell (cx, cy): its nine Q2 nodes, the interior ones
template <class T>
__host__ __device__ __forceinline__ void mf_pres_bu(const MfRes<T>& r, int N, int cx, int cy, T b[3]) {
#pragma unroll
  for (int be = 0; be < 9; ++be) {
    const int jx = 2 * cx + be % 3, jy = 2 * cy + be / 3;
    if (!mf_vinterior(N, jx, jy)) continue;
    const size_t id = 2 * (size_t)mf_vnode(N, jx, jy);
    const T u0 = r.zu[id], u1 = r.zu[id + 1];
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] -= r.divB[k][be][0] * u0 + r.divB[k][be][1] * u1;
  }
}

// down: grid (ceil(Nc / TP))^2 over the coarse cells
template <class T, int TP, int K>
__host__ __device__ void mfp_down_body(const MfPresArgs<T>& a, const MfCta& cta) {
  const int N = a.N, Nc = N / 2;
  const int CX0 = cta.bx * TP, CY0 = cta.by * TP;
  MfCells f;
  f.ox = 2 * CX0 - K;
  f.oy = 2 * CY0 - K;
  f.w = 2 * TP + 2 * K;
  const int n = f.n();
  T* tab = reinterpret_cast<T*>(cta.sm);
  T* B = tab + ((kMfPresTab + 3) & ~3);
  T *Xc = B + 3 * n, *Xn = B + 6 * n, *Dc = B + 9 * n, *Dn = B + 12 * n;
  // the table to shared memory in the same phase as the frame's b: the
  // smoother start takes D^-1 from the global table (one round trip for all)
  for (int t = cta.tid; t < kMfPresTab; t += cta.nthr) tab[t] = a.tab[t];
  const T* dv = a.tab + kMfPresDinv;
  // b on the frame (with the residual start: b - (-B) zu, its owned part, the
  // cells [K, K + 2 TP) of the frame, to res.bout); x0 = d0 = c0 D^-1 b
  mf_rows(cta, f.w, f.w, [&](int i, int j) {
    const int e = j * f.w + i, cx = f.ox + i, cy = f.oy + j;
    const bool in = mf_cin(N, cx, cy);
    const int v = in ? mf_variant(N, cx, cy) : 0;
    T bv[3] = {0, 0, 0};
    if (in) {
      const size_t id = 3 * ((size_t)cy * N + cx);
      for (int k = 0; k < 3; ++k) bv[k] = a.b[id + k];
      if (a.res.zu) {
        mf_pres_bu<T>(a.res, N, cx, cy, bv);
        if (i >= K && i < K + 2 * TP && j >= K && j < K + 2 * TP)
          for (int k = 0; k < 3; ++k) a.res.bout[id + k] = bv[k];
      }
    }
    for (int k = 0; k < 3; ++k) {
      B[k * n + e] = bv[k];
      const T x0 = a.ch.c0 * dv[3 * v + k] * bv[k];
      Xc[k * n + e] = x0;
      Dc[k * n + e] = x0;
    }
  });
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
    mf_rows(cta, m, m, [&](int i, int j) {
      const int lx = K + i, ly = K + j, e = ly * f.w + lx;
      const int cx = f.ox + lx, cy = f.oy + ly;
      if (!mf_cin(N, cx, cy)) {
        for (int k = 0; k < 3; ++k) R[k * n + e] = 0;
        return;
      }
      T y[3];
      mf_pres_apply<T>(tab, Xc, f, N, cx, cy, e, y);
      const size_t id = 3 * ((size_t)cy * N + cx);
      for (int k = 0; k < 3; ++k) {
        R[k * n + e] = B[k * n + e] - y[k];
        a.xout[id + k] = Xc[k * n + e];
      }
    });
  }
  MF_SYNC();
  // restriction R = P^T to the tile's coarse cells: the children's
  // coefficients with the transposed P1disc blocks [1 sx sy; 0 1/2 0; 0 0 1/2]
  mf_rows(cta, TP, TP, [&](int i, int j) {
    const int X0 = CX0 + i, Y0 = CY0 + j;
    if (X0 >= Nc || Y0 >= Nc) return;
    T s0 = 0, s1 = 0, s2 = 0;
    for (int q = 0; q < 4; ++q) {
      const int cx = 2 * X0 + (q & 1), cy = 2 * Y0 + (q >> 1);
      const int e = (cy - f.oy) * f.w + (cx - f.ox);
      const T sx = (q & 1) ? (T)0.25 : (T)-0.25, sy = (q >> 1) ? (T)0.25 : (T)-0.25;
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
  });
}

// up: grid (ceil(N / (2 TP)))^2 over the fine cells
template <class T, int TP, int K>
__host__ __device__ void mfp_up_body(const MfPresArgs<T>& a, const MfCta& cta) {
  constexpr int TPF = 2 * TP;
  const int N = a.N, Nc = N / 2;
  const int FX0 = cta.bx * TPF, FY0 = cta.by * TPF;
  MfCells f;
  f.ox = FX0 - K;
  f.oy = FY0 - K;
  f.w = TPF + 2 * K;
  const int n = f.n();
  T* tab = reinterpret_cast<T*>(cta.sm);
  T* B = tab + ((kMfPresTab + 3) & ~3);
  T *Xc = B + 3 * n, *Xn = B + 6 * n, *Dc = B + 9 * n, *Dn = B + 12 * n;
  // the epilogue's operands on the owned cells (sv, smp, acc: 3 per cell
  // each), read in the first phase so that the last step makes no global
  // round trip of its own
  constexpr int M = TPF;                     // owned cells a side (f.w - 2 K)
  T* E = B + 15 * n;
  for (int t = cta.tid; t < kMfPresTab; t += cta.nthr) tab[t] = a.tab[t];
  // b and x + P x_coarse (each fine cell from its parent: [1 sx sy; 0 1/2 0; 0 0 1/2])
  mf_rows(cta, f.w, f.w, [&](int i, int j) {
    const int e = j * f.w + i, cx = f.ox + i, cy = f.oy + j;
    T bv[3] = {0, 0, 0}, xv[3] = {0, 0, 0};
    if (mf_cin(N, cx, cy)) {
      const size_t id = 3 * ((size_t)cy * N + cx), pc = 3 * ((size_t)(cy >> 1) * Nc + (cx >> 1));
      const T sx = (cx & 1) ? (T)0.25 : (T)-0.25, sy = (cy & 1) ? (T)0.25 : (T)-0.25;
      const T c0 = a.xc[pc], c1 = a.xc[pc + 1], c2 = a.xc[pc + 2];
      const T p[3] = {c0 + sx * c1 + sy * c2, (T)0.5 * c1, (T)0.5 * c2};
      for (int k = 0; k < 3; ++k) {
        bv[k] = a.b[id + k];
        xv[k] = p[k] + a.xpre[id + k];
      }
      if (i >= K && i < K + M && j >= K && j < K + M) {
        T* eo = E + 9 * ((j - K) * M + (i - K));
        for (int k = 0; k < 3; ++k) {
          if (a.fin.sout) {
            eo[k] = a.fin.sv[id + k];
            eo[3 + k] = a.fin.smp[id + k];
          }
          if (a.fin.acc) eo[6 + k] = a.fin.acc[id + k];
        }
      }
    }
    for (int k = 0; k < 3; ++k) {
      B[k * n + e] = bv[k];
      Xc[k * n + e] = xv[k];
    }
  });
  MF_SYNC();
  const T* dv = tab + kMfPresDinv;
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
  mf_rows(cta, m, m, [&](int i, int j) {
    const int lx = K + i, ly = K + j, e = ly * f.w + lx;
    const int cx = f.ox + lx, cy = f.oy + ly;
    if (!mf_cin(N, cx, cy)) return;
    T y[3];
    mf_pres_apply<T>(tab, Xc, f, N, cx, cy, e, y);
    const int v = mf_variant(N, cx, cy);
    const size_t id = 3 * ((size_t)cy * N + cx);
    const T* eo = E + 9 * (j * M + i);
    for (int k = 0; k < 3; ++k) {
      const T r = B[k * n + e] - y[k];
      const T dn = (s == 0) ? c2 * dv[3 * v + k] * r : c1 * Dc[k * n + e] + c2 * dv[3 * v + k] * r;
      const T yv = Xc[k * n + e] + dn;
      a.xout[id + k] = yv;
      T ov = yv;
      if (a.fin.sout) {
        ov = -(a.fin.snu * eo[3 + k] * eo[k] + a.fin.srdt * yv);
        a.fin.sout[id + k] = ov;
      }
      if (a.fin.acc) a.fin.acc[id + k] = eo[6 + k] + a.fin.omega * ov;
    }
  });
}

#ifdef __CUDACC__
// The kernels: one CTA per tile, NT threads.
#define FSI_MF_KERNEL(name, body, Args)                                                      \
  template <class T, int TILE, int K, int NT>                                                \
  __global__ void __launch_bounds__(NT) name(const __grid_constant__ Args<T> a) {            \
    asm volatile("griddepcontrol.wait;" ::: "memory");                                       \
    extern __shared__ __align__(16) unsigned char mf_smem[];                                 \
    const MfCta c{(int)blockIdx.x, (int)blockIdx.y, (int)threadIdx.x, (int)blockDim.x, NT,   \
                  mf_smem};                                                                  \
    body<T, TILE, K>(a, c);                                                                  \
  }
FSI_MF_KERNEL(k_mfu_down, mfu_down_body, MfVelArgs)
FSI_MF_KERNEL(k_mfu_up, mfu_up_body, MfVelArgs)
FSI_MF_KERNEL(k_mfp_down, mfp_down_body, MfPresArgs)
FSI_MF_KERNEL(k_mfp_up, mfp_up_body, MfPresArgs)
#undef FSI_MF_KERNEL
#endif

// shared memory of one launch (bytes) for tile tc (velocity: coarse lattice
// nodes; pressure: coarse cells) and Chebyshev degree K
template <class T>
inline size_t mfu_down_smem(int tc, int K) {
  const int w = 2 * tc + 8 + 4 * K;
  return 6 * (size_t)w * w * 2 * sizeof(T);
}
template <class T>
inline size_t mfu_up_smem(int tc, int K) {
  const int w = 2 * tc + 4 * K;
  const int gw = 2 * ((w + 3) / 4 + 2);   // coarse frame side (upper bound)
  return (5 * (size_t)w * w + (size_t)gw * gw) * 2 * sizeof(T);
}
template <class T>
inline size_t mfp_down_smem(int tp, int K) {
  const int w = 2 * tp + 2 * K;
  return (((kMfPresTab + 3) & ~3) + 15 * (size_t)w * w) * sizeof(T);
}
template <class T>
inline size_t mfp_up_smem(int tp, int K) {
  const int w = 2 * tp + 2 * K;
  return (((kMfPresTab + 3) & ~3) + 15 * (size_t)w * w + 9 * (size_t)(2 * tp) * (2 * tp)) * sizeof(T);
}

}  // namespace fsi
