// Device kernels of the FSI step and their launch descriptors.  Included by
// fsi_solver.cu only (one translation unit holds all device code).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "fsi_internal.h"

namespace fsi {

// Programmatic dependent launch: kernels are launched so that the next one
// may be scheduled while the previous one finishes.  Every kernel first waits
// until all the grids it depends on have completed and their writes are
// visible, before it reads anything (pdl_begin); the SpMV kernels let their
// dependents launch once their loads are done (pdl_trigger), so that the
// next kernel's CTAs arrive during the tail rather than competing for the SMs
// from the start.  Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// device error flags (OR-ed into Ctl::flags)
enum : int {
  FLAG_OUT_OF_DOMAIN = 1,
  FLAG_CAPACITY = 2,
  FLAG_NAN = 4,
  FLAG_BREAKDOWN = 8,
};

// Krylov control block, one per problem, in device memory.
struct Ctl {
  int j;            // Arnoldi index inside the current cycle
  int its;          // iterations of this solve
  int cycles;       // cycles (restarts / refinements) of this solve
  int flags;        // FLAG_* bits
  int converged;    // 1 once ||b - A x|| <= target (true FP64 residual)
  int stop;         // 1 once the solve must end (converged, cap, error)
  int max_it;
  int m;            // restart length
  int pad0, pad1;
  double beta;      // true residual norm at the start of the current cycle
  double bnorm;     // ||b||
  double target;    // rtol * ||b||
  double cycle_tol; // stop the cycle when |g_{j+1}| <= cycle_tol
  double inner_rtol;
  double res;       // current Krylov residual estimate
  double last_true; // true relative residual at the last cycle start
  double scale;     // 1 / ||w|| for the next basis vector
  double pmean;     // mean of the constant pressure coefficients
  int aflags;       // FLAG_* bits raised by the assembly (S2-S4)
  int cyc_active;   // 1 while the Arnoldi loop of the current cycle continues
  int refine;       // 1 when the current Gram-Schmidt step needs a second pass
  int max_cycles;   // cap on restart / refinement cycles of one solve
  int refines;      // second passes taken in this solve
  double wnorm2;    // ||w||^2 before orthogonalisation
  unsigned int counter[8];  // last-block counters for reductions
};

constexpr int kRedThreads = 256;
constexpr int kCfWindow = 1024;   // fluid lattice nodes in one C_f row window
constexpr int kCfWarps = 4;       // warps per CTA in the C_f row kernel

// --------------------------------------------------------- sliced ELL SpMV
// MODE_AXPBY : y = alpha A x + beta z            (z may alias y)
// MODE_CHEB  : d = c1 d + c2 dinv (z - A x); y = x + d      (z = b)
// MODE_CHEB0 : d = c2 dinv (z - A x);        y = x + d
// MODE_INIT  : t = alpha A x + beta z; y = t; d = xo = c2 dinv t
enum { MODE_AXPBY = 0, MODE_CHEB = 1, MODE_CHEB0 = 2, MODE_INIT = 3 };

template <class T>
struct SpmvArgs {
  const T* x = nullptr;
  T* y = nullptr;
  const T* z = nullptr;
  T alpha = 1, beta = 0;
  T* d = nullptr;
  const T* dinv = nullptr;
  T* xo = nullptr;
  T c1 = 0, c2 = 0;
  // MODE_CHEB / MODE_CHEB0 extras (the last smoothing step of a V-cycle):
  // with sout, s = -(snu * smp * sv + srdt * y) is written to sout (the
  // Cahouet-Chabard combination of the Schur approximation); with acc,
  // acc += omega * (s if sout else y) (a Richardson update)
  const T* sv = nullptr;
  const T* smp = nullptr;
  T* sout = nullptr;
  T snu = 0, srdt = 0;
  T* acc = nullptr;
  T omega = 1;
};

// Sliced ELL with slice height 8 ("SELL-8"): slot(s, k, r) = soff[s] + 8k + r.
// One warp owns one slice and gives each block row 4 threads: lane = 8 t + r,
// thread t takes the entries k = t, t + 4, ...  For a fixed round the warp
// reads 32 consecutive slots (coalesced), and 4x more threads are in flight
// than with one thread per row.  Partial sums meet through two shuffles.
constexpr int kSliceRows = 8;
constexpr int kRowThreads = 4;

#ifndef FSI_VEC2_DEFINED
#define FSI_VEC2_DEFINED
template <class T>
struct Vec2;
template <>
struct Vec2<float> { using type = float2; };
template <>
struct Vec2<double> { using type = double2; };
#endif

template <class T, int NV>
__device__ __forceinline__ void load_block(const T* __restrict__ p, T* v) {
  if constexpr (NV == 4 && sizeof(T) == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (NV % 2 == 0) {
    using V2 = typename Vec2<T>::type;
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) {
      const V2 q = __ldg(reinterpret_cast<const V2*>(p) + i);
      v[2 * i] = q.x; v[2 * i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = __ldg(p + i);
  }
}

template <class TX, class TA, int BC>
__device__ __forceinline__ void load_x(const TX* __restrict__ x, int c, TA* xv) {
  if constexpr (BC == 2) {
    using V2 = typename Vec2<TX>::type;
    const V2 q = *reinterpret_cast<const V2*>(x + 2 * (size_t)c);
    xv[0] = (TA)q.x; xv[1] = (TA)q.y;
  } else {
#pragma unroll
    for (int j = 0; j < BC; ++j) xv[j] = (TA)x[(size_t)c * BC + j];
  }
}

// accumulate this thread's share of block row `row` of A (BR x BC blocks) times x.
// Entries are taken two at a time: both column indices are loaded first,
// then both value blocks and gathered x blocks, so that several independent
// loads are in flight per thread before the first FMA (two, not more, keeps
// the kernels at 32 registers and full occupancy).
template <class TA, class TX, int BR, int BC, bool KRON, int NV, int TPR = kRowThreads>
__device__ __forceinline__ void sell_row(const Sell<TA>& A, int row, int t, const TX* __restrict__ x, TA* acc) {
  int base, n;
  if (A.nrun > 0) {  // slice offset from the run table (kernel parameters, no memory load)
    const int s = row >> 3;
    int k = 0;
#pragma unroll
    for (int q = 1; q < Sell<TA>::kMaxRuns; ++q)
      if (q < A.nrun && s >= A.run_s[q]) k = q;
    n = A.run_w[k];
    base = A.run_off[k] + (s - A.run_s[k]) * kSliceRows * n + (row & 7);
  } else {
    base = A.soff[row >> 3] + (row & 7);
    n = A.len[row];
  }
  constexpr int U = 2;
  for (int k0 = t; k0 < n; k0 += U * TPR) {
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * TPR;
      c[u] = (k < n) ? __ldg(A.col + base + (k << 3)) : -1;
    }
    TA xv[U][BC];
    TA v[U][KRON ? 1 : NV];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int slot = base + ((k0 + u * TPR) << 3);
      if (c[u] >= 0) {
        load_x<TX, TA, BC>(x, c[u], xv[u]);
        if constexpr (KRON) v[u][0] = __ldg(A.val + slot);
        else load_block<TA, NV>(A.val + (size_t)slot * NV, v[u]);
      } else {
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[u][j] = 0;
#pragma unroll
        for (int j = 0; j < (KRON ? 1 : NV); ++j) v[u][j] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if constexpr (KRON) {
#pragma unroll
        for (int i = 0; i < BR; ++i) acc[i] += v[u][0] * xv[u][i];
      } else {
#pragma unroll
        for (int i = 0; i < BR; ++i)
#pragma unroll
          for (int j = 0; j < BC; ++j) acc[i] += v[u][i * BC + j] * xv[u][j];
      }
    }
  }
}

// sum of a row's partial sums over its TPR threads (lane = (32/TPR) t + r)
template <class T, int BR, int TPR = kRowThreads>
__device__ __forceinline__ void row_reduce(T* acc) {
#pragma unroll
  for (int i = 0; i < BR; ++i) {
#pragma unroll
    for (int o = 32 / TPR; o < 32; o <<= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
  }
}

// The per-level SpMV (k_sell) takes TPR threads per block row (4 or 8, the
// tile shape the autotuner picks per matrix): a warp holds 32 / TPR rows.
template <class T, int BR, int BC, bool KRON, int NV, int MODE, int TPR>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 16 : 8) k_sell(Sell<T> A, SpmvArgs<T> a) {
  pdl_begin();
  constexpr int RPW = 32 / TPR;  // block rows per warp
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RPW + (lane % RPW);
  const int t = lane / RPW;
  const bool live = row < A.nrows;
  // The row's epilogue operands (z, d, dinv, x) do not depend on A x.  For
  // square blocks (the multigrid level operators) thread t of the row loads
  // one of them (t = 0: z, 1: d, 2: dinv, 3: x) before the product, so that
  // their memory latency overlaps it, and they reach thread 0 by shuffles
  // after the reduction; other shapes load them after it (more registers
  // would spill).  Only thread 0 of the row writes y[r] and d[r], and x is not
  // written in these modes, so the early reads see the same values.
  constexpr bool PRE = (BR == BC);
  const T* pre_src = nullptr;
  if (t == 0) pre_src = a.z;
  else if (t == 1 && MODE == MODE_CHEB) pre_src = a.d;
  else if (t == 2 && MODE != MODE_AXPBY) pre_src = a.dinv;
  else if (t == 3 && (MODE == MODE_CHEB || MODE == MODE_CHEB0)) pre_src = a.x;
  T pre[BR];
#pragma unroll
  for (int i = 0; i < BR; ++i) pre[i] = (PRE && live && pre_src) ? pre_src[row * BR + i] : (T)0;
  T acc[BR];
#pragma unroll
  for (int i = 0; i < BR; ++i) acc[i] = 0;
  if (live) sell_row<T, T, BR, BC, KRON, NV, TPR>(A, row, t, a.x, acc);
  row_reduce<T, BR, TPR>(acc);
  pdl_trigger();
  T zr[BR], dr[BR], vr[BR], xr[BR];
  if constexpr (PRE) {
    const int r0 = lane % RPW;  // lane of the row's thread 0; thread k is at r0 + k RPW
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      zr[i] = __shfl_sync(0xffffffffu, pre[i], r0);
      dr[i] = __shfl_sync(0xffffffffu, pre[i], r0 + RPW);
      vr[i] = __shfl_sync(0xffffffffu, pre[i], r0 + 2 * RPW);
      xr[i] = __shfl_sync(0xffffffffu, pre[i], r0 + 3 * RPW);
    }
  }
  if (!live || t != 0) return;
  if constexpr (!PRE) {
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      const int r = row * BR + i;
      zr[i] = a.z ? a.z[r] : (T)0;
      dr[i] = (MODE == MODE_CHEB) ? a.d[r] : (T)0;
      vr[i] = (MODE != MODE_AXPBY) ? a.dinv[r] : (T)0;
      xr[i] = (MODE == MODE_CHEB || MODE == MODE_CHEB0) ? a.x[r] : (T)0;
    }
  }
#pragma unroll
  for (int i = 0; i < BR; ++i) {
    const int r = row * BR + i;
    if (MODE == MODE_AXPBY) {
      T out = a.alpha * acc[i];
      if (a.z) out += a.beta * zr[i];
      a.y[r] = out;
    } else if (MODE == MODE_CHEB || MODE == MODE_CHEB0) {
      const T res = zr[i] - acc[i];
      const T dn = (MODE == MODE_CHEB) ? a.c1 * dr[i] + a.c2 * vr[i] * res : a.c2 * vr[i] * res;
      a.d[r] = dn;
      const T yv = xr[i] + dn;
      a.y[r] = yv;
      T ov = yv;
      if (a.sout) {
        ov = -(a.snu * a.smp[r] * a.sv[r] + a.srdt * yv);
        a.sout[r] = ov;
      }
      if (a.acc) a.acc[r] += a.omega * ov;
    } else {  // MODE_INIT
      T tt = a.alpha * acc[i];
      if (a.z) tt += a.beta * zr[i];
      a.y[r] = tt;
      const T dn = a.c2 * vr[i] * tt;
      a.d[r] = dn;
      a.xo[r] = dn;
    }
  }
}

// Fused residual and restriction of one multigrid level, on the coarse rows:
//   y = R b - (R A) x  (= R (b - A x); R A is formed once on the host),
// so the fine residual is neither launched nor stored.  MODE_INIT also starts
// the coarse level's smoother: d = xo = c2 dinv y.  Used on the pressure
// levels, whose R A is small (16 blocks per coarse row).
template <class T, int B, bool RKRON, int RNV, int MODE, int TPR>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 16 : 8) k_resrestrict(Sell<T> R, Sell<T> RA, SpmvArgs<T> a) {
  pdl_begin();
  constexpr int RPW = 32 / TPR;
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RPW + (lane % RPW);
  const int t = lane / RPW;
  const bool live = row < R.nrows;
  T acc[B];
#pragma unroll
  for (int i = 0; i < B; ++i) acc[i] = 0;
  if (live) {
    sell_row<T, T, B, B, false, B * B, TPR>(RA, row, t, a.x, acc);  // (R A) x
#pragma unroll
    for (int i = 0; i < B; ++i) acc[i] = -acc[i];
    sell_row<T, T, B, B, RKRON, RNV, TPR>(R, row, t, a.z, acc);     // + R b
  }
  row_reduce<T, B, TPR>(acc);
  pdl_trigger();
  if (!live || t != 0) return;
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const int r = row * B + i;
    a.y[r] = acc[i];
    if (MODE == MODE_INIT) {
      const T dn = a.c2 * a.dinv[r] * acc[i];
      a.d[r] = dn;
      a.xo[r] = dn;
    }
  }
}

// --------------------------------------------------- full-system operator
// y = alpha * A x + beta * z for the block operator of Eq. (matrix) in the
// layout [u (2 nU) | p (3 nP) | X (2 nS) | lambda (2 nS)].  One launch covers
// the three row segments; each CTA (4 warps, 32 block rows) lies in one.
template <class TA>
struct FullOp {
  int nU = 0, nP = 0, nS = 0;
  int gU = 0, gP = 0, gS = 0;        // CTAs per segment
  Sell<TA> Af, Bt, Bneg, Ssol;        // constant blocks (signs folded in)
  const int* cft_ptr = nullptr;       // C_f^T as CSR over interior nodes
  const int* cft_col = nullptr;
  const TA* cft_val = nullptr;
  const int* cf_len = nullptr;        // C_f as ELL over solid nodes, cap per row
  const int* cf_col = nullptr;
  const TA* cf_val = nullptr;
  int cf_cap = 0;
  TA inv_dt = 0;
  const TA* kt = nullptr;             // nonlinear solid: 2x2 tangent blocks in the Ssol slots
};

template <class TA, class TX, class TY>
__global__ void __launch_bounds__(128, sizeof(TA) == 4 ? 16 : 8) k_fullmv(FullOp<TA> op, const TX* __restrict__ x, TY* __restrict__ y,
                                                const TY* __restrict__ z, TY alpha, TY beta) {
  pdl_begin();
  const int lane = threadIdx.x & 31, t = lane >> 3;
  const int b = blockIdx.x;
  const int wrow = (threadIdx.x >> 5) * kSliceRows + (lane & 7);
  const size_t offP = 2 * (size_t)op.nU, offX = offP + 3 * (size_t)op.nP, offL = offX + 2 * (size_t)op.nS;
  if (b < op.gU) {
    const int r = b * 32 + wrow;
    const bool live = r < op.nU;
    TA a[2] = {0, 0};
    if (live) {
      sell_row<TA, TX, 2, 2, false, 4>(op.Af, r, t, x, a);
      sell_row<TA, TX, 2, 3, false, 6>(op.Bt, r, t, x + offP, a);
      for (int k = op.cft_ptr[r] + t; k < op.cft_ptr[r + 1]; k += kRowThreads) {
        const int c = op.cft_col[k];
        const TA v = op.cft_val[k];
        TA lv[2];
        load_x<TX, TA, 2>(x + offL, c, lv);
        a[0] += v * lv[0];
        a[1] += v * lv[1];
      }
    }
    row_reduce<TA, 2>(a);
    if (!live || t != 0) return;
    TY o0 = alpha * (TY)a[0], o1 = alpha * (TY)a[1];
    if (z) { o0 += beta * z[2 * r]; o1 += beta * z[2 * r + 1]; }
    y[2 * r] = o0;
    y[2 * r + 1] = o1;
  } else if (b < op.gU + op.gP) {
    const int r = (b - op.gU) * 32 + wrow;
    const bool live = r < op.nP;
    TA a[3] = {0, 0, 0};
    if (live) sell_row<TA, TX, 3, 2, false, 6>(op.Bneg, r, t, x, a);
    row_reduce<TA, 3>(a);
    if (!live || t != 0) return;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      TY o = alpha * (TY)a[i];
      if (z) o += beta * z[offP + 3 * r + i];
      y[offP + 3 * r + i] = o;
    }
  } else {
    const int r = (b - op.gU - op.gP) * 32 + wrow;
    const bool live = r < op.nS;
    TA a[4] = {0, 0, 0, 0};
    if (live) {
      const int base = op.Ssol.soff[r >> 3] + (r & 7), n = op.Ssol.len[r];
      for (int k = t; k < n; k += kRowThreads) {
        const int slot = base + (k << 3);
        const int c = __ldg(op.Ssol.col + slot);
        const TA as = __ldg(op.Ssol.val + 2 * (size_t)slot), cs = __ldg(op.Ssol.val + 2 * (size_t)slot + 1);
        TA Xv[2], Lv[2];
        load_x<TX, TA, 2>(x + offX, c, Xv);
        load_x<TX, TA, 2>(x + offL, c, Lv);
        if (op.kt) {  // tangent of the nonlinear law: a 2x2 block per slot
          const TA* kb = op.kt + 4 * (size_t)slot;
          a[0] += kb[0] * Xv[0] + kb[1] * Xv[1] - cs * Lv[0];
          a[1] += kb[2] * Xv[0] + kb[3] * Xv[1] - cs * Lv[1];
        } else {
          a[0] += as * Xv[0] - cs * Lv[0];
          a[1] += as * Xv[1] - cs * Lv[1];
        }
        a[2] -= op.inv_dt * cs * Xv[0];
        a[3] -= op.inv_dt * cs * Xv[1];
      }
      const size_t cbase = (size_t)(r >> 5) * 32 * op.cf_cap + (r & 31);
      const int nc = op.cf_len[r];
      for (int k = t; k < nc; k += kRowThreads) {
        const size_t slot = cbase + ((size_t)k << 5);
        const int c = op.cf_col[slot];
        const TA v = op.cf_val[slot];
        TA uv[2];
        load_x<TX, TA, 2>(x, c, uv);
        a[2] += v * uv[0];
        a[3] += v * uv[1];
      }
    }
    row_reduce<TA, 4>(a);
    if (!live || t != 0) return;
    TY o[4] = {alpha * (TY)a[0], alpha * (TY)a[1], alpha * (TY)a[2], alpha * (TY)a[3]};
    if (z) {
      o[0] += beta * z[offX + 2 * r]; o[1] += beta * z[offX + 2 * r + 1];
      o[2] += beta * z[offL + 2 * r]; o[3] += beta * z[offL + 2 * r + 1];
    }
    y[offX + 2 * r] = o[0]; y[offX + 2 * r + 1] = o[1];
    y[offL + 2 * r] = o[2]; y[offL + 2 * r + 1] = o[3];
  }
}

// Residual of the fluid (Stokes) block A_11 = [[A_f, -B^T], [-B, 0]]:
// t_u = r_u - (A_f z_u - B^T z_p), t_p = r_p + B z_u.  Vectors hold
// [u (2 nU) | p (3 nP)] at offset 0; same CTA layout as k_fullmv's first two
// segments.  With pd given, the pressure rows also start the pressure
// V-cycle on t_p: pb = t_p, pd = px = pc0 pdinv t_p.
template <class T>
__global__ void __launch_bounds__(128) k_stokes_res(FullOp<T> op, const T* __restrict__ z, const T* __restrict__ ru,
                                                    const T* __restrict__ rp, T* __restrict__ t,
                                                    const T* __restrict__ pdinv, T pc0, T* __restrict__ pb,
                                                    T* __restrict__ pd, T* __restrict__ px) {
  pdl_begin();
  const int lane = threadIdx.x & 31, tt = lane >> 3;
  const int b = blockIdx.x;
  const int wrow = (threadIdx.x >> 5) * kSliceRows + (lane & 7);
  const size_t offP = 2 * (size_t)op.nU;
  if (b < op.gU) {
    const int r = b * 32 + wrow;
    const bool live = r < op.nU;
    T a[2] = {0, 0};
    if (live) {
      sell_row<T, T, 2, 2, false, 4>(op.Af, r, tt, z, a);
      sell_row<T, T, 2, 3, false, 6>(op.Bt, r, tt, z + offP, a);
    }
    row_reduce<T, 2>(a);
    pdl_trigger();
    if (!live || tt != 0) return;
    t[2 * r] = ru[2 * r] - a[0];
    t[2 * r + 1] = ru[2 * r + 1] - a[1];
  } else {
    const int r = (b - op.gU) * 32 + wrow;
    const bool live = r < op.nP;
    T a[3] = {0, 0, 0};
    if (live) sell_row<T, T, 3, 2, false, 6>(op.Bneg, r, tt, z, a);
    row_reduce<T, 3>(a);
    pdl_trigger();
    if (!live || tt != 0) return;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T tv = rp[3 * r + i] - a[i];
      t[offP + 3 * r + i] = tv;
      if (pd) {  // first Chebyshev step of the pressure V-cycle on this residual
        pb[3 * r + i] = tv;
        const T v = pc0 * pdinv[3 * r + i] * tv;
        pd[3 * r + i] = v;
        px[3 * r + i] = v;
      }
    }
  }
}

template <class T>
__global__ void k_axpy(size_t n, T a, const T* __restrict__ x, T* __restrict__ y) {
  pdl_begin();
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// C_f (ELL over solid nodes, kron 2) times a velocity vector:
// y = alpha C_f u + beta z on 2 nS entries; MODE_INIT also sets d = xo = c2 dinv y.
template <class T>
__global__ void k_cf_apply(int nS, int cap, const int* __restrict__ len, const int* __restrict__ col,
                           const T* __restrict__ val, SpmvArgs<T> a, int mode) {
  pdl_begin();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nS) return;
  const size_t cbase = (size_t)(r >> 5) * 32 * cap + (r & 31);
  T a0 = 0, a1 = 0;
  for (int k = 0; k < len[r]; ++k) {
    const size_t slot = cbase + ((size_t)k << 5);
    const int c = col[slot];
    const T v = val[slot];
    a0 += v * a.x[2 * c];
    a1 += v * a.x[2 * c + 1];
  }
  T t0 = a.alpha * a0, t1 = a.alpha * a1;
  if (a.z) { t0 += a.beta * a.z[2 * r]; t1 += a.beta * a.z[2 * r + 1]; }
  a.y[2 * r] = t0;
  a.y[2 * r + 1] = t1;
  if (mode == MODE_INIT) {
    const T d0 = a.c2 * a.dinv[2 * r] * t0, d1 = a.c2 * a.dinv[2 * r + 1] * t1;
    a.d[2 * r] = d0; a.d[2 * r + 1] = d1;
    a.xo[2 * r] = d0; a.xo[2 * r + 1] = d1;
  }
}

// ------------------------------------------------------------ small dense
// y = A x for a dense row-major n x n matrix (coarsest multigrid level):
// one warp per row, lanes over the columns, 8 rows per CTA
// 16-byte vector of T
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  __device__ static float dot(float4 a, float4 b, float s) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
  }
};
template <>
struct Vec16<double> {
  using type = double2;
  __device__ static double dot(double2 a, double2 b, double s) { return fma(a.y, b.y, fma(a.x, b.x, s)); }
};

// y = A x with the dense inverse of the coarsest level: one warp per row,
// rows of ld entries (16-byte multiples, zero padding), x padded to ld with
// zeros; 16-byte loads, eight per lane in flight, so that a row of a few
// thousand entries takes one or two L2 round trips.
template <class T>
__global__ void k_dense_mv(int n, int ld, const T* __restrict__ A, const T* __restrict__ x, T* __restrict__ y) {
  pdl_begin();
  using V = typename Vec16<T>::type;
  constexpr int W = 16 / (int)sizeof(T), U = 8;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const V* __restrict__ a = reinterpret_cast<const V*>(A + (size_t)i * ld);
  const V* xv = reinterpret_cast<const V*>(x);
  const int nv = ld / W;
  T acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = 0;
  for (int j0 = lane; j0 < nv; j0 += 32 * U) {
    V av[U], bv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + 32 * u;
      if (j < nv) {
        av[u] = __ldg(a + j);
        bv[u] = xv[j];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + 32 * u < nv) acc[u] = Vec16<T>::dot(av[u], bv[u], acc[u]);
  }
  T s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[i] = s;
}

// ------------------------------------------------ coarsest-level inverse
// Gauss-Jordan elimination in place on a symmetric positive definite matrix
// (the coarsest A_f, or the pressure Laplacian made regular): launch k
// exchanges unknown k with equation k.  With p the pivot M_kk before the
// launch, entry (i, j) becomes
//   1 / p                   for i = j = k,
//   M_kj / p                for i = k, j != k,
//   -M_ik / p               for j = k, i != k,
//   M_ij - M_ik M_kj / p    otherwise,
// and after the launches for k = 0 .. n-1 the matrix holds its inverse.  The
// pivots of a positive definite matrix stay positive, so no rows are
// exchanged.  Row k and column k come from copies (rin, cin) written by the
// previous launch, so the entries of one launch are independent; the launch
// writes its row k+1 and column k+1 to (rout, cout) for the next one.
__global__ void k_gj_step(int n, int ld, int k, double* __restrict__ M, const double* __restrict__ rin,
                          const double* __restrict__ cin, double* __restrict__ rout, double* __restrict__ cout) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const double ip = 1.0 / rin[k];
  double v;
  if (i == k)
    v = (j == k) ? ip : rin[j] * ip;
  else if (j == k)
    v = -cin[i] * ip;
  else
    v = M[(size_t)i * ld + j] - cin[i] * (rin[j] * ip);
  M[(size_t)i * ld + j] = v;
  if (i == k + 1) rout[j] = v;
  if (j == k + 1) cout[i] = v;
}

// row 0 and column 0 of M for the first k_gj_step
__global__ void k_gj_first(int n, int ld, const double* __restrict__ M, double* __restrict__ r, double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = M[i];
  c[i] = M[(size_t)i * ld];
}

// out = (T) in, n rows; rows of ldi (in) and ldo (out) entries, the padding
// of out zero
template <class T>
__global__ void k_dense_round(int n, const double* __restrict__ in, int ldi, T* __restrict__ out, int ldo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= ldo) return;
  out[(size_t)i * ldo + j] = j < n ? (T)in[(size_t)i * ldi + j] : (T)0;
}

// ----------------------------------------------------------- vector kernels
template <class T>
__global__ void k_cheb_first(int n, const T* __restrict__ b, const T* __restrict__ dinv, T c, T* __restrict__ d,
                             T* __restrict__ x, T scale, T* __restrict__ bout) {
  pdl_begin();
  // b' = scale * b (stored in bout when given); d = x = c dinv b'
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T bs = scale * b[i];
  if (bout) bout[i] = bs;
  const T v = c * dinv[i] * bs;
  d[i] = v;
  x[i] = v;
}

template <class TI, class TO>
__global__ void k_convert(size_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  pdl_begin();
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (TO)in[i];
}

template <class T>
__global__ void k_copy(size_t n, const T* __restrict__ in, T* __restrict__ out) {
  pdl_begin();
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

// Schur complement approximation (Cahouet-Chabard):
// z_p = -(nu Mp^-1 v_p + (rho/dt) s_p)
template <class T>
__global__ void k_schur(int n, const T* __restrict__ vp, const T* __restrict__ sp, const T* __restrict__ mpinv,
                        T nu, T rdt, T* __restrict__ zp) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  zp[i] = -(nu * mpinv[i] * vp[i] + rdt * sp[i]);
}

// ---------------------------------------------------- deterministic reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum, result valid in thread 0 (fixed tree -> deterministic)
__device__ __forceinline__ double block_sum(double v, double* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double r = 0;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// returns true in the last block to finish (after its partial is visible)
__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

}  // namespace fsi
