// Cluster-resident coarse levels of the geometric multigrid V-cycle.
//
// The coarse part of a V-cycle (Section 5: one V-cycle with Chebyshev-Jacobi
// smoothing approximates each inner fluid solve) is a chain of tiny,
// dependent sparse products; as separate launches each one costs a kernel
// node and three dependent memory round trips.  Here the levels whose
// operators fit in the shared memory of one thread-block cluster run as ONE
// launch: every CTA of the cluster copies its slice of the level operators
// (sliced ELL, its own block rows) into shared memory once, keeps its part of
// every level vector in shared memory, gathers the vector entries of other
// CTAs through distributed shared memory, and separates dependent phases by
// hardware cluster barriers.  The arithmetic of each phase is the same as in
// the per-level kernels (k_sell modes CHEB, CHEB0, AXPBY, INIT).
#pragma once
#include <cooperative_groups.h>

#include "fsi_kernels.cuh"

namespace fsi {

namespace cg = cooperative_groups;

constexpr int kClMaxLevels = 6;
constexpr int kClMaxDeg = 8;
constexpr int kClThreads = 1024;
constexpr int kClColBits = 20;   // packed column: (owner CTA << 20) | block row inside the owner
constexpr int kClColMask = (1 << kClColBits) - 1;

// One sliced-ELL matrix as held by one CTA: byte offsets of its arrays in the
// CTA's shared memory.  Slot (s, k, r) = soff[s] + 8k + r over the CTA's own
// slices; len per own block row; col packed as above.
struct ClMat {
  int soff = -1, len = -1, col = -1, val = -1;
};

template <class T>
struct ClLevel {
  int nrows = 0, nsl = 0;  // block rows and 8-row slices of the whole level
  ClMat A;                 // level operator (absent on the coarsest level)
  ClMat P;                 // prolongation from the next coarser level (rows here)
  ClMat R;                 // restriction from the next finer level (rows here)
  int dinv = -1;           // byte offsets of per-unknown arrays over the CTA's rows
  int x = -1, x2 = -1, b = -1, r = -1, d = -1;
  T c0 = 0, c1[kClMaxDeg] = {}, c2[kClMaxDeg] = {};
};

template <class T>
struct ClArgs {
  int nlev = 0;            // cluster levels; the last one is solved by the dense inverse
  int degree = 2;          // Chebyshev steps per smoothing
  int csize = 16;          // CTAs per cluster
  int blob_bytes = 0;      // bytes of operator data per CTA (multiple of 16)
  size_t blob_stride = 0;  // in uint4 between consecutive CTAs' data
  const uint4* blob = nullptr;
  int gmap = -1;           // coarsest level: packed owner of every block row
  int gbuf = -1;           // coarsest level: gathered right-hand side
  const T* dense_inv = nullptr;
  int dense_n = 0;
  int dense_ld = 0;        // entries per row of dense_inv (>= dense_n)
  const T* in_b = nullptr; // right-hand side of the top cluster level (global)
  T* out_x = nullptr;      // its V-cycle result (global)
  ClLevel<T> lv[kClMaxLevels];
};

// slices [s0, s1) of a level owned by CTA `rank` (the host packs columns with
// the same rule)
__host__ __device__ inline void cl_own(int nsl, int rank, int csize, int& s0, int& s1) {
  s0 = (int)(((long long)nsl * rank) / csize);
  s1 = (int)(((long long)nsl * (rank + 1)) / csize);
}

template <class T>
__device__ __forceinline__ T* cl_ptr(unsigned char* sm, int off) {
  return reinterpret_cast<T*>(sm + off);
}

// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cl_map(unsigned saddr, unsigned rank) {
  unsigned r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// BC consecutive values at a shared::cluster address (ordered after the
// preceding cluster barrier, which is itself a volatile asm with a memory
// clobber)
template <class T, int BC>
__device__ __forceinline__ void cl_load(unsigned addr, T* v) {
  if constexpr (sizeof(T) == 4 && BC == 2) {
    float a, b;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "r"(addr));
    v[0] = a; v[1] = b;
  } else if constexpr (sizeof(T) == 8 && BC == 2) {
    double a, b;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "r"(addr));
    v[0] = a; v[1] = b;
  } else {
#pragma unroll
    for (int j = 0; j < BC; ++j) {
      if constexpr (sizeof(T) == 4) {
        float a;
        asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(a) : "r"(addr + 4u * j));
        v[j] = a;
      } else {
        double a;
        asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(a) : "r"(addr + 8u * j));
        v[j] = a;
      }
    }
  }
}

template <class T, int NV>
__device__ __forceinline__ void cl_block(const T* __restrict__ p, T* v) {
  if constexpr (NV == 4 && sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = p[i];
  }
}

// One phase: for every own block row of M, acc = M x (x gathered from the
// owners' shared memory), then the epilogue of MODE on own rows:
//   AXPBY: y = alpha acc + beta z          CHEB : d = c1 d + c2 dinv (z - acc); y = xown + d
//   CHEB0: d = c2 dinv (z - acc); y = xown + d
//   INIT : y = alpha acc + beta z; d = xo = c2 dinv y
// Vector arguments are byte offsets (-1 = absent); they are the same in
// every CTA of the cluster.
template <class T, int BR, int BC, bool KRON, int NV, int MODE>
__device__ __forceinline__ void cl_phase(unsigned char* sm, const cg::cluster_group& cl, const ClMat& M, int nrows,
                                         int nsl, int rank, int csize, int xsrc, int xown, int y, int z, int d,
                                         int dinv, int xo, T alpha, T beta, T c1, T c2) {
  int s0, s1;
  cl_own(nsl, rank, csize, s0, s1);
  const int nloc = s1 - s0;
  const int* __restrict__ soff = cl_ptr<const int>(sm, M.soff);
  const int* __restrict__ len = cl_ptr<const int>(sm, M.len);
  const int* __restrict__ col = cl_ptr<const int>(sm, M.col);
  const T* __restrict__ val = cl_ptr<const T>(sm, M.val);
  const unsigned xs = (unsigned)__cvta_generic_to_shared(sm + xsrc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int t = lane >> 3;
  constexpr int U = 4;   // entries in flight per thread (one round for most rows)
  for (int sl = warp; sl < nloc; sl += nw) {
    const int rl = sl * kSliceRows + (lane & 7);
    const bool live = s0 * kSliceRows + rl < nrows;
    T acc[BR];
#pragma unroll
    for (int i = 0; i < BR; ++i) acc[i] = 0;
    if (live) {
      const int base = soff[sl] + (lane & 7);
      const int n = len[rl];
      for (int k0 = t; k0 < n; k0 += U * kRowThreads) {
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u * kRowThreads;
          c[u] = (k < n) ? col[base + (k << 3)] : -1;
        }
        T xv[U][BC];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (c[u] >= 0) {
            const unsigned addr = cl_map(xs + (unsigned)((c[u] & kClColMask) * BC * (int)sizeof(T)),
                                         (unsigned)(c[u] >> kClColBits));
            cl_load<T, BC>(addr, xv[u]);
          } else {
#pragma unroll
            for (int j = 0; j < BC; ++j) xv[u][j] = 0;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (c[u] < 0) continue;
          const int slot = base + ((k0 + u * kRowThreads) << 3);
          if constexpr (KRON) {
            const T v = val[slot];
#pragma unroll
            for (int i = 0; i < BR; ++i) acc[i] += v * xv[u][i];
          } else {
            T v[NV];
            cl_block<T, NV>(val + (size_t)slot * NV, v);
#pragma unroll
            for (int i = 0; i < BR; ++i)
#pragma unroll
              for (int j = 0; j < BC; ++j) acc[i] += v[i * BC + j] * xv[u][j];
          }
        }
      }
    }
    row_reduce<T, BR>(acc);
    if (!live || t != 0) continue;
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      const int q = rl * BR + i;
      if (MODE == MODE_AXPBY) {
        T out = alpha * acc[i];
        if (z >= 0) out += beta * cl_ptr<T>(sm, z)[q];
        cl_ptr<T>(sm, y)[q] = out;
      } else if (MODE == MODE_CHEB || MODE == MODE_CHEB0) {
        const T res = cl_ptr<T>(sm, z)[q] - acc[i];
        T dn = c2 * cl_ptr<T>(sm, dinv)[q] * res;
        if (MODE == MODE_CHEB) dn = c1 * cl_ptr<T>(sm, d)[q] + dn;
        cl_ptr<T>(sm, d)[q] = dn;
        cl_ptr<T>(sm, y)[q] = cl_ptr<T>(sm, xown)[q] + dn;
      } else {  // MODE_INIT
        T tt = alpha * acc[i];
        if (z >= 0) tt += beta * cl_ptr<T>(sm, z)[q];
        cl_ptr<T>(sm, y)[q] = tt;
        const T dn = c2 * cl_ptr<T>(sm, dinv)[q] * tt;
        cl_ptr<T>(sm, d)[q] = dn;
        cl_ptr<T>(sm, xo)[q] = dn;
      }
    }
  }
}

// The V-cycle from the top cluster level down to the dense coarsest level and
// back, in the order of the per-level host code: on each level (degree - 1)
// Chebyshev steps from x = d = c0 D^-1 b, residual, restriction (which
// initialises the coarser smoother), the coarser cycle, prolongation and
// correction, then `degree` Chebyshev steps.  B: unknowns per block row (2
// velocity, 3 pressure); TKRON: transfers act on components alike (Q2
// velocity) instead of as full B x B blocks (P1disc pressure).
template <class T, int B, bool TKRON>
__global__ void __launch_bounds__(kClThreads, 1) k_vcycle_cluster(const __grid_constant__ ClArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cs = a.csize;
  constexpr int TNV = TKRON ? 1 : B * B;
  const ClLevel<T>& L0 = a.lv[0];
  int t0, t1;
  cl_own(L0.nsl, rank, cs, t0, t1);
  const int r0 = t0 * kSliceRows, r1 = min(t1 * kSliceRows, L0.nrows);
  const int n0 = max(r1 - r0, 0) * B;  // own unknowns of the top level
  {  // stage this CTA's operators and its part of the top-level right-hand
     // side: every copy is issued before the single wait, so all are in flight
    const uint4* __restrict__ src = a.blob + (size_t)rank * a.blob_stride;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(sm);
    const int n16 = a.blob_bytes >> 4;
    for (int i = threadIdx.x; i < n16; i += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * (unsigned)i), "l"(src + i) : "memory");
    const unsigned bdst = (unsigned)__cvta_generic_to_shared(sm + L0.b);
    const T* bsrc = a.in_b + (size_t)r0 * B;
    for (int i = threadIdx.x; i < n0; i += blockDim.x)
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(bdst + (unsigned)(i * sizeof(T))), "l"(bsrc + i),
                   "n"(sizeof(T)) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  __syncthreads();
  {  // top level: x = d = c0 D^-1 b on own rows
    const T* b = cl_ptr<const T>(sm, L0.b);
    T* x = cl_ptr<T>(sm, L0.x);
    T* d = cl_ptr<T>(sm, L0.d);
    const T* dinv = cl_ptr<const T>(sm, L0.dinv);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
      const T tv = L0.c0 * dinv[i] * b[i];
      x[i] = tv;
      d[i] = tv;
    }
  }
  cl.sync();
  int cur[kClMaxLevels], oth[kClMaxLevels];
  const int last = a.nlev - 1;
  for (int l = 0; l < last; ++l) {
    const ClLevel<T>& L = a.lv[l];
    cur[l] = L.x;
    oth[l] = L.x2;
    for (int i = 1; i < a.degree; ++i) {
      cl_phase<T, B, B, false, B * B, MODE_CHEB>(sm, cl, L.A, L.nrows, L.nsl, rank, cs, cur[l], cur[l], oth[l], L.b,
                                                   L.d, L.dinv, -1, T(0), T(0), L.c1[i - 1], L.c2[i - 1]);
      const int tmp = cur[l]; cur[l] = oth[l]; oth[l] = tmp;
      cl.sync();
    }
    cl_phase<T, B, B, false, B * B, MODE_AXPBY>(sm, cl, L.A, L.nrows, L.nsl, rank, cs, cur[l], -1, L.r, L.b, -1, -1,
                                                  -1, T(-1), T(1), T(0), T(0));
    cl.sync();
    const ClLevel<T>& C = a.lv[l + 1];
    if (l + 1 < last)
      cl_phase<T, B, B, TKRON, TNV, MODE_INIT>(sm, cl, C.R, C.nrows, C.nsl, rank, cs, L.r, -1, C.b, -1, C.d, C.dinv,
                                               C.x, T(1), T(0), T(0), C.c0);
    else
      cl_phase<T, B, B, TKRON, TNV, MODE_AXPBY>(sm, cl, C.R, C.nrows, C.nsl, rank, cs, L.r, -1, C.b, -1, -1, -1, -1,
                                                T(1), T(0), T(0), T(0));
    cl.sync();
  }
  {  // coarsest level: gather its right-hand side, own rows of (dense inverse) b
    const ClLevel<T>& C = a.lv[last];
    const int n = a.dense_n;
    const int* __restrict__ gmap = cl_ptr<const int>(sm, a.gmap);
    T* g = cl_ptr<T>(sm, a.gbuf);
    T* cb = cl_ptr<T>(sm, C.b);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int row = i / B, comp = i - row * B;
      const int c = gmap[row];
      const T* src = cl.map_shared_rank(cb, (unsigned)(c >> kClColBits));
      g[i] = src[(size_t)(c & kClColMask) * B + comp];
    }
    __syncthreads();
    int s0, s1;
    cl_own(C.nsl, rank, cs, s0, s1);
    const int rc0 = s0 * kSliceRows, rc1 = min(s1 * kSliceRows, C.nrows);
    const int nown = max(rc1 - rc0, 0) * B;
    T* x = cl_ptr<T>(sm, C.x);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < nown; i += nw) {
      const T* __restrict__ arow = a.dense_inv + (size_t)(rc0 * B + i) * a.dense_ld;
      // eight independent loads in flight per lane, one L2 round trip for
      // rows of up to 256 entries
      T acc8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc8[u] = 0;
      for (int j0 = lane; j0 < n; j0 += 256) {
        T av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) av[u] = (j0 + 32 * u < n) ? __ldg(arow + j0 + 32 * u) : (T)0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j0 + 32 * u < n) acc8[u] += av[u] * g[j0 + 32 * u];
      }
      T sum = ((acc8[0] + acc8[1]) + (acc8[2] + acc8[3])) + ((acc8[4] + acc8[5]) + (acc8[6] + acc8[7]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
      if (lane == 0) x[i] = sum;
    }
    cur[last] = C.x;
  }
  cl.sync();
  for (int l = last - 1; l >= 0; --l) {
    const ClLevel<T>& L = a.lv[l];
    cl_phase<T, B, B, TKRON, TNV, MODE_AXPBY>(sm, cl, L.P, L.nrows, L.nsl, rank, cs, cur[l + 1], -1, cur[l], cur[l], -1,
                                              -1, -1, T(1), T(1), T(0), T(0));
    cl.sync();
    for (int i = 0; i < a.degree; ++i) {
      if (i == 0)
        cl_phase<T, B, B, false, B * B, MODE_CHEB0>(sm, cl, L.A, L.nrows, L.nsl, rank, cs, cur[l], cur[l], oth[l],
                                                      L.b, L.d, L.dinv, -1, T(0), T(0), T(0), L.c0);
      else
        cl_phase<T, B, B, false, B * B, MODE_CHEB>(sm, cl, L.A, L.nrows, L.nsl, rank, cs, cur[l], cur[l], oth[l], L.b,
                                                     L.d, L.dinv, -1, T(0), T(0), L.c1[i - 1], L.c2[i - 1]);
      const int tmp = cur[l]; cur[l] = oth[l]; oth[l] = tmp;
      cl.sync();
    }
  }
  {  // the top level's result to global memory (no remote access follows the last barrier)
    const T* x = cl_ptr<const T>(sm, cur[0]);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) a.out_x[(size_t)r0 * B + i] = x[i];
  }
}

}  // namespace fsi
