// Device kernels of the FSI step and their launch descriptors.  Included by
// fsi_solver.cu only (one translation unit holds all device code).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "fsi_internal.h"

namespace fsi {

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
  int pad2;
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
};

template <class T>
__device__ __forceinline__ void load_vals(const T* p, T* v, int nv) {
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (i < nv) v[i] = p[i];
}

template <class T, int BR, int BC, bool KRON, int NV, int MODE>
__global__ void __launch_bounds__(128) k_sell(int nrows, const int* __restrict__ soff,
                                              const int* __restrict__ len, const int* __restrict__ col,
                                              const T* __restrict__ val, SpmvArgs<T> a) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int s = r >> 5, lane = r & 31;
  const int base = soff[s] + lane;
  const int n = len[r];
  T acc[BR];
#pragma unroll
  for (int i = 0; i < BR; ++i) acc[i] = 0;
  const T* __restrict__ x = a.x;
  for (int k = 0; k < n; ++k) {
    const int slot = base + (k << 5);
    const int c = __ldg(col + slot);
    if (KRON) {
      const T v = __ldg(val + slot);
#pragma unroll
      for (int i = 0; i < BR; ++i) acc[i] += v * x[c * BC + i];
    } else {
      T v[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = __ldg(val + (size_t)slot * NV + i);
      T xv[BC];
#pragma unroll
      for (int jj = 0; jj < BC; ++jj) xv[jj] = x[c * BC + jj];
#pragma unroll
      for (int i = 0; i < BR; ++i)
#pragma unroll
        for (int jj = 0; jj < BC; ++jj) acc[i] += v[i * BC + jj] * xv[jj];
    }
  }
#pragma unroll
  for (int i = 0; i < BR; ++i) {
    const int row = r * BR + i;
    if (MODE == MODE_AXPBY) {
      T out = a.alpha * acc[i];
      if (a.z) out += a.beta * a.z[row];
      a.y[row] = out;
    } else if (MODE == MODE_CHEB) {
      const T res = a.z[row] - acc[i];
      const T dn = a.c1 * a.d[row] + a.c2 * a.dinv[row] * res;
      a.d[row] = dn;
      a.y[row] = x[row] + dn;
    } else if (MODE == MODE_CHEB0) {
      const T res = a.z[row] - acc[i];
      const T dn = a.c2 * a.dinv[row] * res;
      a.d[row] = dn;
      a.y[row] = x[row] + dn;
    } else {  // MODE_INIT
      T t = a.alpha * acc[i];
      if (a.z) t += a.beta * a.z[row];
      a.y[row] = t;
      const T dn = a.c2 * a.dinv[row] * t;
      a.d[row] = dn;
      a.xo[row] = dn;
    }
  }
}

// --------------------------------------------------- full-system operator
// y = alpha * A x + beta * z for the block operator of Eq. (matrix) in the
// layout [u (2 nU) | p (3 nP) | X (2 nS) | lambda (2 nS)].
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
};

template <class TA, class TX, class TY>
__global__ void __launch_bounds__(128) k_fullmv(FullOp<TA> op, const TX* __restrict__ x, TY* __restrict__ y,
                                                const TY* __restrict__ z, TY alpha, TY beta) {
  const int b = blockIdx.x;
  const size_t offP = 2 * (size_t)op.nU, offX = offP + 3 * (size_t)op.nP, offL = offX + 2 * (size_t)op.nS;
  if (b < op.gU) {
    const int r = b * blockDim.x + threadIdx.x;
    if (r >= op.nU) return;
    TA a0 = 0, a1 = 0;
    {
      const int base = op.Af.soff[r >> 5] + (r & 31), n = op.Af.len[r];
      for (int k = 0; k < n; ++k) {
        const int slot = base + (k << 5);
        const int c = __ldg(op.Af.col + slot);
        const TA* v = op.Af.val + (size_t)slot * 4;
        const TA x0 = (TA)x[2 * c], x1 = (TA)x[2 * c + 1];
        a0 += __ldg(v) * x0 + __ldg(v + 1) * x1;
        a1 += __ldg(v + 2) * x0 + __ldg(v + 3) * x1;
      }
    }
    {
      const int base = op.Bt.soff[r >> 5] + (r & 31), n = op.Bt.len[r];
      for (int k = 0; k < n; ++k) {
        const int slot = base + (k << 5);
        const int c = __ldg(op.Bt.col + slot);
        const TA* v = op.Bt.val + (size_t)slot * 6;
        const TA p0 = (TA)x[offP + 3 * c], p1 = (TA)x[offP + 3 * c + 1], p2 = (TA)x[offP + 3 * c + 2];
        a0 += __ldg(v) * p0 + __ldg(v + 1) * p1 + __ldg(v + 2) * p2;
        a1 += __ldg(v + 3) * p0 + __ldg(v + 4) * p1 + __ldg(v + 5) * p2;
      }
    }
    for (int k = op.cft_ptr[r]; k < op.cft_ptr[r + 1]; ++k) {
      const int c = op.cft_col[k];
      const TA v = op.cft_val[k];
      a0 += v * (TA)x[offL + 2 * c];
      a1 += v * (TA)x[offL + 2 * c + 1];
    }
    TY o0 = alpha * (TY)a0, o1 = alpha * (TY)a1;
    if (z) { o0 += beta * z[2 * r]; o1 += beta * z[2 * r + 1]; }
    y[2 * r] = o0;
    y[2 * r + 1] = o1;
  } else if (b < op.gU + op.gP) {
    const int r = (b - op.gU) * blockDim.x + threadIdx.x;
    if (r >= op.nP) return;
    TA a[3] = {0, 0, 0};
    const int base = op.Bneg.soff[r >> 5] + (r & 31), n = op.Bneg.len[r];
    for (int k = 0; k < n; ++k) {
      const int slot = base + (k << 5);
      const int c = __ldg(op.Bneg.col + slot);
      const TA* v = op.Bneg.val + (size_t)slot * 6;
      const TA x0 = (TA)x[2 * c], x1 = (TA)x[2 * c + 1];
#pragma unroll
      for (int i = 0; i < 3; ++i) a[i] += __ldg(v + 2 * i) * x0 + __ldg(v + 2 * i + 1) * x1;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      TY o = alpha * (TY)a[i];
      if (z) o += beta * z[offP + 3 * r + i];
      y[offP + 3 * r + i] = o;
    }
  } else {
    const int r = (b - op.gU - op.gP) * blockDim.x + threadIdx.x;
    if (r >= op.nS) return;
    TA ax0 = 0, ax1 = 0, al0 = 0, al1 = 0;
    const int base = op.Ssol.soff[r >> 5] + (r & 31), n = op.Ssol.len[r];
    for (int k = 0; k < n; ++k) {
      const int slot = base + (k << 5);
      const int c = __ldg(op.Ssol.col + slot);
      const TA as = __ldg(op.Ssol.val + 2 * (size_t)slot), cs = __ldg(op.Ssol.val + 2 * (size_t)slot + 1);
      const TA X0 = (TA)x[offX + 2 * c], X1 = (TA)x[offX + 2 * c + 1];
      const TA L0 = (TA)x[offL + 2 * c], L1 = (TA)x[offL + 2 * c + 1];
      ax0 += as * X0 - cs * L0;
      ax1 += as * X1 - cs * L1;
      al0 -= op.inv_dt * cs * X0;
      al1 -= op.inv_dt * cs * X1;
    }
    const size_t cbase = (size_t)(r >> 5) * 32 * op.cf_cap + (r & 31);
    const int nc = op.cf_len[r];
    for (int k = 0; k < nc; ++k) {
      const size_t slot = cbase + ((size_t)k << 5);
      const int c = op.cf_col[slot];
      const TA v = op.cf_val[slot];
      al0 += v * (TA)x[2 * c];
      al1 += v * (TA)x[2 * c + 1];
    }
    TY o[4] = {alpha * (TY)ax0, alpha * (TY)ax1, alpha * (TY)al0, alpha * (TY)al1};
    if (z) {
      o[0] += beta * z[offX + 2 * r]; o[1] += beta * z[offX + 2 * r + 1];
      o[2] += beta * z[offL + 2 * r]; o[3] += beta * z[offL + 2 * r + 1];
    }
    y[offX + 2 * r] = o[0]; y[offX + 2 * r + 1] = o[1];
    y[offL + 2 * r] = o[2]; y[offL + 2 * r + 1] = o[3];
  }
}

// C_f (ELL over solid nodes, kron 2) times a velocity vector:
// y = alpha C_f u + beta z on 2 nS entries; MODE_INIT also sets d = xo = c2 dinv y.
template <class T>
__global__ void k_cf_apply(int nS, int cap, const int* __restrict__ len, const int* __restrict__ col,
                           const T* __restrict__ val, SpmvArgs<T> a, int mode) {
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
// y = A x for a dense row-major n x n matrix (coarsest multigrid level).
template <class T>
__global__ void k_dense_mv(int n, const T* __restrict__ A, const T* __restrict__ x, T* __restrict__ y) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T s = 0;
    for (int j = 0; j < n; ++j) s += A[(size_t)i * n + j] * x[j];
    y[i] = s;
  }
}

// ----------------------------------------------------------- vector kernels
template <class T>
__global__ void k_cheb_first(int n, const T* __restrict__ b, const T* __restrict__ dinv, T c, T* __restrict__ d,
                             T* __restrict__ x, T scale, T* __restrict__ bout) {
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
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (TO)in[i];
}

template <class T>
__global__ void k_copy(size_t n, const T* __restrict__ in, T* __restrict__ out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

// Schur complement approximation (Cahouet-Chabard):
// z_p = -(nu Mp^-1 v_p + (rho/dt) s_p)
template <class T>
__global__ void k_schur(int n, const T* __restrict__ vp, const T* __restrict__ sp, const T* __restrict__ mpinv,
                        T nu, T rdt, T* __restrict__ zp) {
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
