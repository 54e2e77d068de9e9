// GB300 (sm_103a) solver for one time step of the DLM fictitious-domain FSI
// method (Boffi, Credali, Gastaldi, Scacchi, arXiv:2301.10041), and the C ABI
// declared in include/fsi.h.
//
// Per step (Section 4): S1 right-hand side, S2 point location, S3 binning of
// the coupling entries by fluid node, S4 C_f(X^n) and its transpose, S5 the
// block operator of Eq. (matrix), S6 the block-diagonal / block-triangular
// preconditioner of Section 5, S7 flexible GMRES (CGS2, Givens on device,
// the whole Arnoldi loop inside one CUDA graph WHILE node), S8 FP64 iterative
// refinement around FP32 operators, S9 advance.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/fsi.h"
#include "fsi_cluster.cuh"
#include "fsi_cluster_host.h"
#include "fsi_coupling.cuh"
#include "fsi_internal.h"
#include "fsi_kernels.cuh"
#include "fsi_mgfused.cuh"
#include "fsi_solid.cuh"

namespace fsi {

struct CudaError : std::runtime_error {
  cudaError_t code;
  explicit CudaError(cudaError_t c, const char* what) : std::runtime_error(what), code(c) {}
};
#define CK(x)                                                                 \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) throw CudaError(e_, #x);                           \
  } while (0)

static inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Every kernel of the library (but the cluster V-cycle) is launched through
// here.  The launches carry programmatic stream serialisation, so a kernel may
// be scheduled while its predecessor on the stream finishes; each kernel
// waits for its producers (griddepcontrol.wait, in pdl_begin() or the fused
// kernels' wrapper) before it touches memory.  With the fused multigrid
// levels this measured faster than plain launches (12.5 against 11.6 steps/s
// mixed, 3.71 against 3.54 FP64, on the 128 x 128 cavity); with the per-level
// sparse kernels alone it had measured slower.  FSI_PDL=0 in the environment
// turns it off.
static bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("FSI_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <typename... KArgs, typename... Args>
static void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                   Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(std::forward<Args>(args))...);
  if (e != cudaSuccess) throw CudaError(e, "cudaLaunchKernelEx");
}


// ------------------------------------------------------------ device memory
struct Arena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  bool count_only = false;
  template <class T>
  T* alloc(size_t n) {
    const size_t b = std::max<size_t>(n, 1) * sizeof(T);
    bytes += (b + 255) & ~(size_t)255;
    if (count_only) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, b) != cudaSuccess) throw std::bad_alloc();
    ptrs.push_back(p);
    return (T*)p;
  }
  template <class T>
  T* upload(const std::vector<T>& h) {
    T* d = alloc<T>(h.size());
    if (d && !h.empty()) CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

template <class T>
static Sell<T> upload_sell(Arena& ar, const SellHost& s) {
  Sell<T> d;
  d.nrows = s.nrows; d.BR = s.BR; d.BC = s.BC; d.NV = s.NV; d.kron = s.kron;
  d.soff = ar.upload(s.soff);
  d.len = ar.upload(s.len);
  // runs of equal slice width (structured-grid matrices have at most 15)
  std::vector<int> rs, rw, ro;
  for (int sl = 0; sl < s.nslices; ++sl) {
    const int w = (s.soff[sl + 1] - s.soff[sl]) / kSliceRows;
    if (rw.empty() || w != rw.back()) {
      rs.push_back(sl);
      rw.push_back(w);
      ro.push_back(s.soff[sl]);
    }
  }
  std::vector<int> col = s.col;
  if (!rs.empty() && rs.size() <= (size_t)Sell<T>::kMaxRuns) {
    d.nrun = (int)rs.size();
    for (int k = 0; k < d.nrun; ++k) {
      d.run_s[k] = rs[k];
      d.run_w[k] = rw[k];
      d.run_off[k] = ro[k];
    }
    for (int r = 0; r < s.nrows; ++r) {  // mark the padding slots
      const int sl = r / kSliceRows, lane = r % kSliceRows;
      const int w = (s.soff[sl + 1] - s.soff[sl]) / kSliceRows;
      for (int k = s.len[r]; k < w; ++k) col[(size_t)s.soff[sl] + (size_t)k * kSliceRows + lane] = -1;
    }
  }
  d.col = ar.upload(col);
  std::vector<T> v(s.val.begin(), s.val.end());
  d.val = ar.upload(v);
  return d;
}

template <class T>
static T* upload_as(Arena& ar, const std::vector<double>& h) {
  std::vector<T> v(h.begin(), h.end());
  return ar.upload(v);
}

// ------------------------------------------------------------- SpMV launch
template <class T, int BR, int BC, bool KRON, int NV, int TPR>
static void sell_launch_tpr(const Sell<T>& A, int mode, const SpmvArgs<T>& a, cudaStream_t s) {
  const unsigned g = nblk(A.nrows, 4 * (32 / TPR));  // 4 warps x 32/TPR block rows
  switch (mode) {
    case MODE_AXPBY: launch(k_sell<T, BR, BC, KRON, NV, MODE_AXPBY, TPR>, g, 128, 0, s, A, a); break;
    case MODE_CHEB: launch(k_sell<T, BR, BC, KRON, NV, MODE_CHEB, TPR>, g, 128, 0, s, A, a); break;
    case MODE_CHEB0: launch(k_sell<T, BR, BC, KRON, NV, MODE_CHEB0, TPR>, g, 128, 0, s, A, a); break;
    default: launch(k_sell<T, BR, BC, KRON, NV, MODE_INIT, TPR>, g, 128, 0, s, A, a); break;
  }
}

template <class T, int BR, int BC, bool KRON, int NV>
static void sell_launch_shape(const Sell<T>& A, int mode, const SpmvArgs<T>& a, cudaStream_t s) {
  if (A.tpr == 8) return sell_launch_tpr<T, BR, BC, KRON, NV, 8>(A, mode, a, s);
  sell_launch_tpr<T, BR, BC, KRON, NV, 4>(A, mode, a, s);
}

// Fused residual + restriction (k_resrestrict) of the pressure levels: full
// 3x3 restriction blocks, R L with full blocks.
template <class T, int B, bool RKRON, int RNV, int TPR>
static void resrestrict_shape(const Sell<T>& R, const Sell<T>& RA, int mode, const SpmvArgs<T>& a, cudaStream_t s) {
  const unsigned g = nblk(R.nrows, 4 * (32 / TPR));
  if (mode == MODE_INIT) launch(k_resrestrict<T, B, RKRON, RNV, MODE_INIT, TPR>, g, 128, 0, s, R, RA, a);
  else launch(k_resrestrict<T, B, RKRON, RNV, MODE_AXPBY, TPR>, g, 128, 0, s, R, RA, a);
}

template <class T>
static void resrestrict_launch(const Sell<T>& R, const Sell<T>& RA, int mode, const SpmvArgs<T>& a, cudaStream_t s) {
  if (R.nrows == 0) return;
  if (!R.kron && R.BR == 3 && RA.BR == 3) return resrestrict_shape<T, 3, false, 9, 4>(R, RA, mode, a, s);
  throw std::logic_error("unsupported restriction shape");
}

template <class T>
static void sell_launch(const Sell<T>& A, int mode, const SpmvArgs<T>& a, cudaStream_t s) {
  if (A.nrows == 0) return;
  if (A.kron && A.BR == 2) return sell_launch_shape<T, 2, 2, true, 1>(A, mode, a, s);
  if (A.BR == 2 && A.BC == 2) return sell_launch_shape<T, 2, 2, false, 4>(A, mode, a, s);
  if (A.BR == 2 && A.BC == 3) return sell_launch_shape<T, 2, 3, false, 6>(A, mode, a, s);
  if (A.BR == 3 && A.BC == 2) return sell_launch_shape<T, 3, 2, false, 6>(A, mode, a, s);
  if (A.BR == 3 && A.BC == 3) return sell_launch_shape<T, 3, 3, false, 9>(A, mode, a, s);
  throw std::logic_error("unsupported block shape");
}

template <class T>
static SpmvArgs<T> axpby(const T* x, T* y, const T* z, T alpha, T beta) {
  SpmvArgs<T> a;
  a.x = x; a.y = y; a.z = z; a.alpha = alpha; a.beta = beta;
  return a;
}

// ------------------------------------------------------------- autotuner
// Tile shape of the per-level SpMV: 4 or 8 threads per block row, chosen per
// matrix by timing both on the device in the form a V-cycle runs it (the
// Chebyshev-Jacobi smoothing step, 20 dependent launches captured in a CUDA
// graph and replayed once warm: the conditions inside a solve); 8 is kept
// only when at least 5 % faster.
// Results are cached per (device, block shape, rows, slots, precision) for
// the life of the process, so instances of one size tune once and problems
// created in one process take the same shapes (the same rounding).
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int, int, int, int>, int> g_tune;

template <class T>
static void autotune_sell(Sell<T>& A, int nslots) {
  if (A.nrows == 0 || A.BR != A.BC) return;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, A.BR, A.BC, (int)A.kron, A.nrows, nslots, (int)sizeof(T));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      A.tpr = it->second;
      return;
    }
  }
  const size_t nx = (size_t)A.nrows * A.BR;
  T* buf = nullptr;   // x, y, b, d, dinv
  CK(cudaMalloc(&buf, 5 * nx * sizeof(T)));
  CK(cudaMemset(buf, 0, 5 * nx * sizeof(T)));
  T* x = buf;
  T* y = buf + nx;
  cudaStream_t s;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float t[2] = {0.f, 0.f};
  SpmvArgs<T> axy;
  axy.z = buf + 2 * nx; axy.d = buf + 3 * nx; axy.dinv = buf + 4 * nx;
  axy.c1 = (T)0.5; axy.c2 = (T)0.5;
  SpmvArgs<T> ayx = axy;
  axy.x = x; axy.y = y;
  ayx.x = y; ayx.y = x;
  for (int v = 0; v < 2; ++v) {
    // 20 dependent launches (x -> y -> x ...) in a CUDA graph, as in a solve
    Sell<T> B = A;
    B.tpr = v == 0 ? 4 : 8;
    cudaGraph_t gr;
    cudaGraphExec_t ge;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < 20; ++r) sell_launch(B, MODE_CHEB, (r & 1) ? ayx : axy, s);
    CK(cudaStreamEndCapture(s, &gr));
    CK(cudaGraphInstantiate(&ge, gr, 0));
    CK(cudaGraphLaunch(ge, s));
    CK(cudaEventRecord(e0, s));
    CK(cudaGraphLaunch(ge, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&t[v], e0, e1));
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(gr);
  }
  A.tpr = (t[1] < 0.95f * t[0]) ? 8 : 4;
  if (const char* v = getenv("FSI_TUNE_VERBOSE"); v && v[0] == '1')
    fprintf(stderr, "fsi autotune: %dx%d blocks, %d rows, %s: 4 threads/row %.2f us, 8 threads/row %.2f us -> %d\n",
            A.BR, A.BC, A.nrows, sizeof(T) == 4 ? "fp32" : "fp64", t[0] * 50.f, t[1] * 50.f, A.tpr);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(buf);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = A.tpr;
}

// ---------------------------------------------------------------- multigrid
struct Cheb {
  double c0;                 // first step: d = c0 dinv r
  std::vector<double> c1, c2;  // steps 1..k-1
};

static Cheb cheb_coeffs(double lo, double hi, int k) {
  Cheb c;
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
struct MGLevel {
  Sell<T> A, P, R;  // P: prolongation from the next coarser level, R: restriction to it
  Sell<T> RA;       // pressure levels: R L, so that R (b - L x) = R b - (R L) x takes one pass
  T* dinv = nullptr;
  T *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr, *d = nullptr;
  int n = 0;        // scalar unknowns
  int N = 0;        // cells per side
  Cheb ch;
  // the level's stencils for the fused matrix-free kernels (fsi_mgfused.cuh),
  // and whether the V-cycle runs them on this level
  bool mf = false;
  MfVelOp<T> mfu;        // velocity hierarchy
  T* mftab = nullptr;    // pressure hierarchy: kMfPresTab values
  T divB[3][9][2] = {};  // entries of -B and -B^T on this level (residual start)
};

// Coarse levels run as one thread-block-cluster launch per V-cycle
// (fsi_cluster.cuh): levels lc .. last.
template <class T>
struct ClusterMG {
  bool on = false;
  int lc = 0;
  size_t smem = 0;
  ClArgs<T> args;
};

template <class T>
struct MG {
  std::vector<MGLevel<T>> lv;
  T* coarse_inv = nullptr;   // dense inverse of the coarsest level, rows of coarse_ld entries
  int coarse_n = 0;
  int coarse_ld = 0;         // coarse_n rounded up to 16 bytes (the row padding is zero)
  int degree = 2;
  bool pressure = false;
  ClusterMG<T> cl;
};

constexpr double kChebRatioU = 6.0;   // smoothing interval [hi/ratio, hi]
constexpr double kChebRatioP = 8.0;

// Dense inverse of the coarsest level in place on the device (FP64, rows of
// ld entries, the padding zero): Gauss-Jordan elimination, one launch per
// pivot (k_gj_step).  M holds the dense matrix on entry.
static void dense_inverse_device(Arena& ar, double* M, int n, int ld, cudaStream_t s) {
  double* rc = ar.alloc<double>(4 * (size_t)n);   // row and column copies, two pairs
  if (ar.count_only) return;
  double *r0 = rc, *c0 = rc + n, *r1 = rc + 2 * n, *c1 = rc + 3 * n;
  k_gj_first<<<nblk(n, 256), 256, 0, s>>>(n, ld, M, r0, c0);
  CK(cudaGetLastError());
  const dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  for (int k = 0; k < n; ++k) {
    k_gj_step<<<grd, blk, 0, s>>>(n, ld, k, M, r0, c0, r1, c1);
    std::swap(r0, r1);
    std::swap(c0, c1);
  }
  CK(cudaGetLastError());
}

// 16-byte row length of the dense coarsest inverse, in entries
template <class T>
static int dense_ld(int n) {
  constexpr int w = 16 / (int)sizeof(T);
  return (n + w - 1) / w * w;
}

// The coarsest level's dense inverse: the FP64 hierarchy inverts the
// assembled matrix in place; the FP32 one rounds the FP64 inverse (inv64,
// rows of ld64 entries).  The FP64 hierarchy is built first.
template <class T>
static void build_coarse_inverse(Arena& ar, const HostSetup& hs, bool pressure, MG<T>& mg, const double* inv64,
                                 int ld64, cudaStream_t s) {
  const int n = pressure ? hs.coarse_nL : hs.coarse_nA;
  mg.coarse_n = n;
  mg.coarse_ld = dense_ld<T>(n);
  const int ld = mg.coarse_ld;
  mg.coarse_inv = ar.alloc<T>((size_t)n * ld);
  if constexpr (std::is_same<T, double>::value) {
    if (!ar.count_only) {
      const std::vector<double>& D = pressure ? hs.coarseL : hs.coarseA;
      CK(cudaMemsetAsync(mg.coarse_inv, 0, (size_t)n * ld * sizeof(double), s));
      CK(cudaMemcpy2DAsync(mg.coarse_inv, (size_t)ld * sizeof(double), D.data(), (size_t)n * sizeof(double),
                           (size_t)n * sizeof(double), n, cudaMemcpyHostToDevice, s));
    }
    dense_inverse_device(ar, mg.coarse_inv, n, ld, s);
  } else if (!ar.count_only) {
    if (!inv64) throw std::logic_error("the FP64 coarse inverse is built first");
    k_dense_round<T><<<dim3((ld + 255) / 256, n), 256, 0, s>>>(n, inv64, ld64, mg.coarse_inv, ld);
    CK(cudaGetLastError());
  }
  // the coarsest right-hand side, padded to ld with zeros, for the dense product
  MGLevel<T>& C = mg.lv.back();
  C.b = ar.alloc<T>(ld);
  if (!ar.count_only) {
    CK(cudaMemsetAsync(C.b, 0, (size_t)ld * sizeof(T), s));
    CK(cudaStreamSynchronize(s));
  }
}

template <class T>
static void build_mg(Arena& ar, const HostSetup& hs, bool pressure, int degree, MG<T>& mg, bool tune,
                     cudaStream_t s, const double* inv64 = nullptr, int ld64 = 0) {
  const int nl = pressure ? hs.nlev_p : hs.nlev_u;
  mg.degree = degree;
  mg.pressure = pressure;
  mg.lv.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const FluidLevelHost& H = hs.levels[l];
    MGLevel<T>& L = mg.lv[l];
    const HostBlockMatrix& A = pressure ? H.L : H.A;
    const SellHost sa = to_sell(A);
    L.A = upload_sell<T>(ar, sa);
    if (tune && !ar.count_only) autotune_sell<T>(L.A, sa.soff[sa.nslices]);
    L.n = A.nrows * A.BR;
    L.N = H.N;
    L.dinv = upload_as<T>(ar, pressure ? H.dinvL : H.dinvA);
    if (l + 1 < nl) {
      L.P = upload_sell<T>(ar, to_sell(pressure ? H.Pp : H.Pu));
      L.R = upload_sell<T>(ar, to_sell(pressure ? H.Rp : H.Ru));
      if (pressure) L.RA = upload_sell<T>(ar, to_sell(H.RAp));
    }
    L.x = ar.alloc<T>(L.n); L.x2 = ar.alloc<T>(L.n);
    if (l + 1 < nl) L.b = ar.alloc<T>(L.n);   // the coarsest: build_coarse_inverse
    if (!pressure) L.r = ar.alloc<T>(L.n);
    L.d = ar.alloc<T>(L.n);
    const double hi = 1.05 * (pressure ? H.lmaxL : H.lmaxA);
    L.ch = cheb_coeffs(hi / (pressure ? kChebRatioP : kChebRatioU), hi, degree);
    if (H.mf)
      for (int k = 0; k < 3; ++k)
        for (int q = 0; q < 9; ++q)
          for (int d = 0; d < 2; ++d) L.divB[k][q][d] = (T)H.divB[k][q][d];
    if (H.mf && !pressure) {
      L.mfu.N = H.N;
      for (int t = 0; t < 4; ++t) {
        for (int y = 0; y < 5; ++y)
          for (int x = 0; x < 5; ++x)
            for (int q = 0; q < 4; ++q) L.mfu.c[t][y][x][q] = (T)H.stenA[t][y][x][q];
        for (int c = 0; c < 2; ++c) L.mfu.dinv[t][c] = (T)H.dinvAt[t][c];
      }
    } else if (H.mf) {
      std::vector<double> tab(kMfPresTab);
      for (int v = 0; v < 9; ++v)
        for (int y = 0; y < 3; ++y)
          for (int x = 0; x < 3; ++x)
            for (int q = 0; q < 9; ++q) tab[mf_pres_blk(v, y, x) + q] = H.stenL[v][y][x][q];
      for (int v = 0; v < 9; ++v)
        for (int k = 0; k < 3; ++k) tab[kMfPresDinv + 3 * v + k] = H.dinvLv[v][k];
      L.mftab = upload_as<T>(ar, tab);
    }
  }
  build_coarse_inverse<T>(ar, hs, pressure, mg, inv64, ld64, s);
}

// ------------------------------------------- cluster-resident coarse levels
constexpr size_t kClSmemCap = 227 * 1024;   // dynamic shared memory per CTA

// The shared-memory limit is a property of the kernel, shared by every
// problem alive in the process: always raise it to the cap.
template <class T, int B, bool TKRON>
static void cluster_kernel_setup() {
  auto kern = k_vcycle_cluster<T, B, TKRON>;
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmemCap));
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
}

template <class T, int B, bool TKRON>
static int cluster_fits(size_t smem, int csize) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_vcycle_cluster<T, B, TKRON>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Cluster of 16 CTAs (non-portable size) when the device schedules one,
// else 8; nothing when neither fits (the per-level kernels run instead).
template <class T>
static void setup_cluster(Arena& ar, const HostSetup& hs, MG<T>& mg, bool pressure, int max_n) {
  int lc_min = 0;   // with max_n > 0 the cluster's finest level has at most max_n cells a side
  if (max_n > 0)
    while (lc_min + 1 < (int)mg.lv.size() && hs.levels[lc_min].N > max_n) ++lc_min;
  for (int cs : {16, 8}) {
    auto viable = [&](size_t smem) {
      if (ar.count_only) return true;
      if (pressure) {
        cluster_kernel_setup<T, 3, false>();
        return cluster_fits<T, 3, false>(smem, cs) > 0;
      }
      cluster_kernel_setup<T, 2, true>();
      return cluster_fits<T, 2, true>(smem, cs) > 0;
    };
    if (build_cluster<T>(ar, hs, pressure, mg, cs, kClSmemCap, viable, lc_min)) return;
  }
}

template <class T>
static void cluster_launch(MG<T>& mg, const T* in_b, T* out_x, cudaStream_t s) {
  ClArgs<T> a = mg.cl.args;
  a.in_b = in_b;
  a.out_x = out_x;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.csize);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = mg.cl.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = a.csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = mg.pressure ? cudaLaunchKernelEx(&cfg, k_vcycle_cluster<T, 3, false>, a)
                                    : cudaLaunchKernelEx(&cfg, k_vcycle_cluster<T, 2, true>, a);
  if (e != cudaSuccess) throw CudaError(e, "cudaLaunchKernelEx (cluster V-cycle)");
}

// The finest levels, down to the first one that runs inside the cluster
// launch (or is the coarsest, or is below 16 cells a side), take the fused
// matrix-free kernels when the hierarchy is FP32 and the smoothing degree is
// at most kMfMaxDeg.
template <class T>
static void select_mf(MG<T>& mg, const HostSetup& hs, int mg_fused, bool count_only) {
  const int last = (int)mg.lv.size() - 1;
  if (mg_fused == -1 || !std::is_same<T, float>::value || mg.degree > kMfMaxDeg) return;
  bool any = false;
  for (int l = 0; l < last; ++l) {
    if (mg.cl.on && l >= mg.cl.lc) break;
    if (!hs.levels[l].mf || hs.levels[l].N < 16) break;
    mg.lv[l].mf = true;
    any = true;
  }
  if (any && !count_only) {
    static std::once_flag once;
    std::call_once(once, [] {
      auto vel = [](auto tc) {
        for (int K = 1; K <= kMfMaxDeg; ++K)
          mf_with_degree(K, [&](auto kc) {
            constexpr int TC = decltype(tc)::value, KD = decltype(kc)::value;
            constexpr int ND = mf_threads_ud(TC), NU = mf_threads_uu(TC);
            CK(cudaFuncSetAttribute(k_mfu_down<float, TC, KD, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mfu_down_smem<float>(TC, KD)));
            CK(cudaFuncSetAttribute(k_mfu_up<float, TC, KD, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mfu_up_smem<float>(TC, KD)));
          });
      };
      auto pres = [](auto tp) {
        for (int K = 1; K <= kMfMaxDeg; ++K)
          mf_with_degree(K, [&](auto kc) {
            constexpr int TP = decltype(tp)::value, KD = decltype(kc)::value, NT = mf_threads_p(TP);
            CK(cudaFuncSetAttribute(k_mfp_down<float, TP, KD, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mfp_down_smem<float>(TP, KD)));
            CK(cudaFuncSetAttribute(k_mfp_up<float, TP, KD, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)mfp_up_smem<float>(TP, KD)));
          });
      };
      for (int N : {16, 64, 128, 512}) mf_with_tile_u(N, vel);   // every tile the maps choose
      for (int N : {16, 64, 128, 512}) mf_with_tile_p(N, pres);
    });
  }
}

template <class T>
static MfCheb<T> mf_cheb(const MGLevel<T>& L, int degree) {
  MfCheb<T> c;
  c.k = degree;
  c.c0 = (T)L.ch.c0;
  for (int i = 0; i + 1 < degree; ++i) {
    c.c1[i] = (T)L.ch.c1[i];
    c.c2[i] = (T)L.ch.c2[i];
  }
  return c;
}

template <class T>
static T* vcycle(MG<T>& mg, int l, cudaStream_t s, T* out, const SpmvArgs<T>* fin = nullptr, bool* fused = nullptr);

// The down launch of fused level l: pre-smoothing from x0 = c0 D^-1 b, the
// residual and its restriction; the pre-smoothed iterate goes to L.x2, the
// coarse right-hand side to C.b (and the coarse smoother start when the next
// level runs the per-level sparse kernels).
template <class T>
static void mf_down_launch(MG<T>& mg, int l, const T* b, cudaStream_t s, const MfRes<T>* res = nullptr) {
  const int last = (int)mg.lv.size() - 1;
  MGLevel<T>& L = mg.lv[l];
  MGLevel<T>& C = mg.lv[l + 1];
  const bool c_cluster = mg.cl.on && l + 1 == mg.cl.lc;
  const bool c_sell = !C.mf && !c_cluster && l + 1 != last;
  const int N = L.N, K = mg.degree;
  MfInit<T> ci;
  if (c_sell) { ci.x = C.x; ci.d = C.d; ci.dinv = C.dinv; ci.c0 = (T)C.ch.c0; }
  MfRes<T> r;
  if (res) {
    r = *res;
    std::memcpy(r.divB, L.divB, sizeof(r.divB));
  }
  if (mg.pressure) {
    MfPresArgs<T> a;
    a.N = N; a.tab = L.mftab; a.ch = mf_cheb(L, K);
    a.b = b; a.xout = L.x2; a.bc = C.b; a.ci = ci; a.res = r;
    mf_with_tile_p(N, [&](auto tp) {
      mf_with_degree(K, [&](auto kc) {
        constexpr int TP = decltype(tp)::value, KD = decltype(kc)::value, NT = mf_threads_p(TP);
        const unsigned g = nblk(N / 2, TP);
        launch(k_mfp_down<T, TP, KD, NT>, dim3(g, g), NT, mfp_down_smem<T>(TP, KD), s, a);
      });
    });
  } else {
    MfVelArgs<T> a;
    a.op = L.mfu; a.ch = mf_cheb(L, K);
    a.b = b; a.xout = L.x2; a.bc = C.b; a.ci = ci; a.res = r;
    mf_with_tile_u(N, [&](auto tc) {
      mf_with_degree(K, [&](auto kc) {
        constexpr int TC = decltype(tc)::value, KD = decltype(kc)::value, NT = mf_threads_ud(TC);
        const unsigned g = nblk(N, TC);
        launch(k_mfu_down<T, TC, KD, NT>, dim3(g, g), NT, mfu_down_smem<T>(TC, KD), s, a);
      });
    });
  }
}

// The up launch of fused level l: x = L.x2 + P xc, post-smoothing, result to
// dst (never L.x2), with the epilogue fin.
template <class T>
static void mf_up_launch(MG<T>& mg, int l, const T* b, const T* xc, T* dst, const MfFin<T>* fin, cudaStream_t s) {
  MGLevel<T>& L = mg.lv[l];
  if (dst == L.x2) throw std::logic_error("mf_up_launch: the result may not overwrite the pre-smoothed iterate");
  const int N = L.N, K = mg.degree;
  if (mg.pressure) {
    MfPresArgs<T> a;
    a.N = N; a.tab = L.mftab; a.ch = mf_cheb(L, K);
    a.b = b; a.xpre = L.x2; a.xc = xc; a.xout = dst;
    if (fin) a.fin = *fin;
    mf_with_tile_p(N, [&](auto tp) {
      mf_with_degree(K, [&](auto kc) {
        constexpr int TP = decltype(tp)::value, KD = decltype(kc)::value, NT = mf_threads_p(TP);
        const unsigned g = nblk(N, 2 * TP);
        launch(k_mfp_up<T, TP, KD, NT>, dim3(g, g), NT, mfp_up_smem<T>(TP, KD), s, a);
      });
    });
  } else {
    MfVelArgs<T> a;
    a.op = L.mfu; a.ch = mf_cheb(L, K);
    a.b = b; a.xpre = L.x2; a.xc = xc; a.xout = dst;
    if (fin) a.fin = *fin;
    mf_with_tile_u(N, [&](auto tc) {
      mf_with_degree(K, [&](auto kc) {
        constexpr int TC = decltype(tc)::value, KD = decltype(kc)::value, NT = mf_threads_uu(TC);
        const unsigned g = nblk(2 * N, 2 * TC);
        launch(k_mfu_up<T, TC, KD, NT>, dim3(g, g), NT, mfu_up_smem<T>(TC, KD), s, a);
      });
    });
  }
}

// One V-cycle from fused level l (mg.lv[l].mf) with right-hand side b: the
// down launch, the coarser levels, the up launch.  The result goes to `out`,
// else to L.x.  With res, the down launch starts from the Stokes residual
// (MfRes) and the up launch reads the right-hand side it wrote to res->bout.
template <class T>
static T* vcycle_mf(MG<T>& mg, int l, const T* b, cudaStream_t s, T* out, const MfFin<T>* fin,
                    const MfRes<T>* res = nullptr) {
  MGLevel<T>& L = mg.lv[l];
  MGLevel<T>& C = mg.lv[l + 1];
  T* dst = out ? out : L.x;
  mf_down_launch<T>(mg, l, b, s, res);
  T* xc = C.mf ? vcycle_mf<T>(mg, l + 1, C.b, s, nullptr, nullptr) : vcycle<T>(mg, l + 1, s, (T*)nullptr);
  mf_up_launch<T>(mg, l, res ? res->bout : b, xc, dst, fin, s);
  return dst;
}

// Algorithmic work of the fused launches of level l (not counting the work
// the tiles repeat on their overlaps): bytes of the vectors read and written
// once, and floating-point operations of the K operator applications (two per
// stored scalar entry), the transfer (two per entry of R or P) and the
// Chebyshev and epilogue updates (about six per unknown per step).
struct MfWork {
  double bytes = 0, flops = 0;
};
static MfWork mf_work(const HostSetup& hs, int l, bool pressure, bool up, int K, size_t tsize) {
  const FluidLevelHost& H = hs.levels[l];
  const FluidLevelHost& Hc = hs.levels[l + 1];
  const HostBlockMatrix& A = pressure ? H.L : H.A;
  const HostBlockMatrix& Tr = pressure ? (up ? H.Pp : H.Rp) : (up ? H.Pu : H.Ru);
  const double n = (double)A.nrows * A.BR, nc = pressure ? 3.0 * Hc.N * Hc.N : 2.0 * Hc.A.nrows;
  const double a_entries = (double)A.nnzb() * A.BR * A.BC;
  const double t_entries = (double)Tr.nnzb() * (Tr.kron ? Tr.BR : Tr.BR * Tr.BC);
  MfWork w;
  w.flops = K * 2.0 * a_entries + 2.0 * t_entries + 6.0 * K * n;
  w.bytes = up ? (3.0 * n + nc) * tsize : (2.0 * n + nc) * tsize;
  return w;
}

// Algorithmic work of one V-cycle of hierarchy mg from its finest level:
// the fused levels' launches (mf_work), the per-level sparse kernels of the
// other levels above the coarsest (2K applications of the stored level
// matrix and one residual, the transfers, a few vectors each), and the
// dense coarsest product (the inverse read once).
template <class T>
static MfWork vcycle_work(const HostSetup& hs, const MG<T>& mg, bool pressure) {
  MfWork w;
  const int last = (int)mg.lv.size() - 1, K = mg.degree;
  const double ts = sizeof(T);
  for (int l = 0; l < last; ++l) {
    if (mg.lv[l].mf) {
      for (bool up : {false, true}) {
        const MfWork m = mf_work(hs, l, pressure, up, K, sizeof(T));
        w.bytes += m.bytes;
        w.flops += m.flops;
      }
      continue;
    }
    const FluidLevelHost& H = hs.levels[l];
    const HostBlockMatrix& A = pressure ? H.L : H.A;
    const HostBlockMatrix& R = pressure ? H.Rp : H.Ru;
    const HostBlockMatrix& Pm = pressure ? H.Pp : H.Pu;
    const double n = (double)A.nrows * A.BR;
    const double a_bytes = (double)A.nnzb() * (A.NV * ts + 4.0);
    const double t_bytes = (double)(R.nnzb() * (R.NV * ts + 4.0) + Pm.nnzb() * (Pm.NV * ts + 4.0));
    const double a_flops = 2.0 * A.nnzb() * A.BR * A.BC;
    w.bytes += (2 * K + 1) * (a_bytes + 4.0 * n * ts) + t_bytes;
    w.flops += (2 * K + 1) * a_flops + 2.0 * (R.nnzb() + Pm.nnzb()) * (R.kron ? R.BR : R.BR * R.BC);
  }
  const double nc = mg.coarse_n;
  w.bytes += nc * mg.coarse_ld * ts + 2.0 * nc * ts;
  w.flops += 2.0 * nc * nc;
  return w;
}

template <class T>
static MfFin<T> mf_fin(const SpmvArgs<T>& f) {
  MfFin<T> m;
  m.sv = f.sv; m.smp = f.smp; m.sout = f.sout; m.snu = f.snu; m.srdt = f.srdt; m.acc = f.acc; m.omega = f.omega;
  return m;
}

// Level l input: L.b, with L.x = L.d = c0 dinv b already set (l < last).
// Result of the level is written to `out` (if given) or returned.  Levels
// from mg.cl.lc down run as one cluster launch when mg.cl.on.
// `fin`, when given, adds its Schur / accumulate epilogue (SpmvArgs sv ..
// omega) to the last smoothing step of level l; *fused tells whether it was
// applied (not when level l is solved by the cluster launch or densely).
template <class T>
static T* vcycle(MG<T>& mg, int l, cudaStream_t s, T* out, const SpmvArgs<T>* fin, bool* fused) {
  const int last = (int)mg.lv.size() - 1;
  MGLevel<T>& L = mg.lv[l];
  if (fused) *fused = false;
  if (L.mf) {  // fused levels need only L.b
    MfFin<T> mfin;
    if (fin) mfin = mf_fin(*fin);
    if (fused) *fused = fin != nullptr;
    return vcycle_mf<T>(mg, l, L.b, s, out, fin ? &mfin : nullptr);
  }
  if (mg.cl.on && l == mg.cl.lc) {
    T* dst = out ? out : L.x;
    cluster_launch<T>(mg, L.b, dst, s);
    return dst;
  }
  if (l == last) {
    launch(k_dense_mv<T>, nblk(mg.coarse_n, 8), 256, 0, s, mg.coarse_n, mg.coarse_ld, (const T*)mg.coarse_inv,
           (const T*)L.b, out ? out : L.x);
    return out ? out : L.x;
  }
  T* xc = L.x;
  T* xn = L.x2;
  const int k = mg.degree;
  for (int i = 1; i < k; ++i) {  // pre-smoothing, zero initial guess
    SpmvArgs<T> a;
    a.x = xc; a.y = xn; a.z = L.b; a.d = L.d; a.dinv = L.dinv;
    a.c1 = (T)L.ch.c1[i - 1]; a.c2 = (T)L.ch.c2[i - 1];
    sell_launch(L.A, MODE_CHEB, a, s);
    std::swap(xc, xn);
  }
  MGLevel<T>& C = mg.lv[l + 1];
  if (L.RA.nrows == 0) {  // residual, then its restriction
    sell_launch(L.A, MODE_AXPBY, axpby<T>(xc, L.r, L.b, (T)-1, (T)1), s);
    if (l + 1 == last || (mg.cl.on && l + 1 == mg.cl.lc)) {
      sell_launch(L.R, MODE_AXPBY, axpby<T>(L.r, C.b, nullptr, (T)1, (T)0), s);
    } else {
      SpmvArgs<T> a = axpby<T>(L.r, C.b, nullptr, (T)1, (T)0);
      a.d = C.d; a.dinv = C.dinv; a.xo = C.x; a.c2 = (T)C.ch.c0;
      sell_launch(L.R, MODE_INIT, a, s);
    }
  } else {  // the coarse right-hand side R (b - A x) = R b - (R A) x in one launch
    SpmvArgs<T> ra;
    ra.x = xc; ra.z = L.b; ra.y = C.b;
    if (l + 1 == last || (mg.cl.on && l + 1 == mg.cl.lc)) {
      resrestrict_launch(L.R, L.RA, MODE_AXPBY, ra, s);
    } else {
      ra.d = C.d; ra.dinv = C.dinv; ra.xo = C.x; ra.c2 = (T)C.ch.c0;
      resrestrict_launch(L.R, L.RA, MODE_INIT, ra, s);
    }
  }
  T* xcoarse = vcycle<T>(mg, l + 1, s, (T*)nullptr);
  sell_launch(L.P, MODE_AXPBY, axpby<T>(xcoarse, xc, xc, (T)1, (T)1), s);
  for (int i = 0; i < k; ++i) {  // post-smoothing
    SpmvArgs<T> a;
    T* dst = (i == k - 1 && out) ? out : xn;
    if (i == k - 1 && fin) {
      a.sv = fin->sv; a.smp = fin->smp; a.sout = fin->sout; a.snu = fin->snu; a.srdt = fin->srdt;
      a.acc = fin->acc; a.omega = fin->omega;
      if (fused) *fused = true;
    }
    a.x = xc; a.y = dst; a.z = L.b; a.d = L.d; a.dinv = L.dinv;
    if (i == 0) { a.c2 = (T)L.ch.c0; sell_launch(L.A, MODE_CHEB0, a, s); }
    else { a.c1 = (T)L.ch.c1[i - 1]; a.c2 = (T)L.ch.c2[i - 1]; sell_launch(L.A, MODE_CHEB, a, s); }
    if (dst == out) return out;
    std::swap(xc, xn);
  }
  return xc;
}

// ----------------------------------------------------------- preconditioner
template <class T>
struct Prec {
  MG<T> mgU, mgP;
  FullOp<T> op;          // operator in this precision (shares structure arrays)
  Sell<T> Cs, As;
  T* mpinv = nullptr;    // inverse P1disc mass diagonal
  T* csdinv = nullptr;   // inverse diagonal of the solid mass
  T* vin = nullptr;      // preconditioner input (n)
  T* zw = nullptr;       // preconditioner output (n)
  T *sb = nullptr, *sx = nullptr, *sx2 = nullptr, *sd = nullptr;  // solid work (2 nS)
  Cheb chs;              // Chebyshev for D^-1 C_s on Wathen's interval ([1/2, 2] for P1)
  int cs_k = 16;
  // inner Richardson on the Stokes block: velocity right-hand side, residual
  // and correction, each [u (2 nU) | p (3 nP)]
  T *ru = nullptr, *t = nullptr, *dz = nullptr;
  int stokes_its = 1;
  T stokes_omega = 1;
  Sell<T> KT;            // nonlinear solid: the tangent as 2x2 blocks (pattern of the solid pair matrix)
};

struct Problem;
template <class T> static void precond_launch(Problem& P, Prec<T>& pr, cudaStream_t s);

// -------------------------------------------------------------- the problem
struct Problem {
  fsi_params prm{};
  int N = 0, nU = 0, nP = 0, nS = 0, nTri = 0, nPts = 0;
  size_t n = 0, offP = 0, offX = 0, offL = 0;
  cudaStream_t stream = nullptr, s2 = nullptr, s3 = nullptr, s4 = nullptr, s5 = nullptr;  // capture helpers
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork2 = nullptr, ev_join2 = nullptr;
  bool own_stream = false;
  int device = 0;
  Arena ar;
  HostSetup hs;
  // operators
  FullOp<double> op64;
  FullOp<float> op32;
  Sell<double> M64, Cs64;
  // coupling
  int* tris = nullptr; double* area = nullptr; int* ntp = nullptr; int* nt = nullptr;
  int* l2n = nullptr; double* wall = nullptr;
  int* cell = nullptr; double* xi = nullptr; double* eta = nullptr;
  int cf_cap = 64;
  // nonlinear solid: reference gradients of the P1 basis per triangle (3 x 2),
  // tangent blocks in the slots of the solid pair matrix (4 per slot)
  double* tgrad = nullptr;
  double* kt64 = nullptr;
  float* kt32 = nullptr;
  int* cf_len = nullptr; int* cf_col = nullptr; double* cf_val = nullptr; float* cf_val32 = nullptr;
  double* cflift = nullptr;
  int* cft_ptr = nullptr; int* cft_col = nullptr; double* cft_val = nullptr; float* cft_val32 = nullptr;
  int* cft_cnt = nullptr; int* cft_cur = nullptr; int* scan_bsum = nullptr;
  // state
  double *x = nullptr, *b = nullptr, *uold = nullptr, *Xold = nullptr, *lift_u = nullptr, *w = nullptr;
  // Krylov
  int m = 200;
  double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *part = nullptr;
  void* Z = nullptr;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;   // pinned mirror
  int red_blocks = 0;
  // preconditioners
  Prec<double> p64;
  Prec<float> p32;
  // graphs
  cudaGraphExec_t g_assemble = nullptr, g_begin = nullptr, g_cycle = nullptr, g_finish = nullptr;
  cudaGraph_t gr_assemble = nullptr, gr_begin = nullptr, gr_cycle = nullptr, gr_finish = nullptr;
  // host-driven Arnoldi loop (FSI_HOST_LOOP=1): no conditional nodes, so that
  // per-kernel profilers can see the kernels; same kernels, one sync per iteration
  bool host_loop = false;
  cudaGraphExec_t g_cstart = nullptr, g_body = nullptr, g_cend = nullptr;
  cudaGraph_t gr_cstart = nullptr, gr_body = nullptr, gr_cend = nullptr;
  bool assembled = false;
  int kn_assemble = 0, kn_begin = 0, kn_cycle = 0, kn_body = 0, kn_finish = 0;  // kernel nodes per graph
};

// ------------------------------------------------------- solid block A_22^-1
// Exact up to the two C_s solves (Chebyshev-Jacobi on [1/2, 2], Wathen's
// bounds for the Jacobi-scaled P1 mass matrix):
//   X = -dt C_s^-1 r_l,   lambda = C_s^-1 (A_s X - r_X),
// with r_l = v_l - C_f z_u for the block-triangular preconditioner.
template <class T>
static void solid_launch(Problem& P, Prec<T>& pr, cudaStream_t s) {
  const int n2 = 2 * P.nS;
  if (n2 == 0) return;
  const T* vX = pr.vin + P.offX;
  const T* vL = pr.vin + P.offL;
  T* zX = pr.zw + P.offX;
  T* zL = pr.zw + P.offL;
  const T dt = (T)P.prm.dt;
  auto cheb_rest = [&](T* out) {
    T* xc = pr.sx;
    T* xn = pr.sx2;
    if (pr.cs_k == 1) { launch(k_copy<T>, nblk(n2, 256), 256, 0, s, n2, pr.sx, out); return; }
    for (int i = 1; i < pr.cs_k; ++i) {
      SpmvArgs<T> a;
      T* dst = (i == pr.cs_k - 1) ? out : xn;
      a.x = xc; a.y = dst; a.z = pr.sb; a.d = pr.sd; a.dinv = pr.csdinv;
      a.c1 = (T)pr.chs.c1[i - 1]; a.c2 = (T)pr.chs.c2[i - 1];
      sell_launch(pr.Cs, MODE_CHEB, a, s);
      std::swap(xc, xn);
    }
  };
  if (P.prm.precond == 1) {  // lower block-triangular: r_l = v_l - C_f z_u
    SpmvArgs<T> a;
    a.x = pr.zw; a.y = pr.sb; a.z = vL; a.alpha = dt; a.beta = -dt;
    a.d = pr.sd; a.dinv = pr.csdinv; a.xo = pr.sx; a.c2 = (T)pr.chs.c0;
    launch(k_cf_apply<T>, nblk(P.nS, 128), 128, 0, s, P.nS, P.cf_cap, P.cf_len, P.cf_col, pr.op.cf_val, a, MODE_INIT);
  } else {
    launch(k_cheb_first<T>, nblk(n2, 256), 256, 0, s, n2, vL, pr.csdinv, (T)pr.chs.c0, pr.sd, pr.sx, -dt, pr.sb);
  }
  cheb_rest(zX);
  SpmvArgs<T> a2;
  a2.x = zX; a2.y = pr.sb; a2.z = vX; a2.alpha = 1; a2.beta = -1;
  a2.d = pr.sd; a2.dinv = pr.csdinv; a2.xo = pr.sx; a2.c2 = (T)pr.chs.c0;
  sell_launch(P.prm.solid_law == 1 ? pr.KT : pr.As, MODE_INIT, a2, s);
  cheb_rest(zL);
}

// C_f^T applied to the multiplier part: y_u = z_u - C_f^T lambda (CSR over interior nodes)
template <class T>
__global__ void k_cft_sub(int nU, const int* __restrict__ ptr, const int* __restrict__ col, const T* __restrict__ val,
                          const T* __restrict__ lam, const T* __restrict__ zu, T* __restrict__ y) {
  pdl_begin();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nU) return;
  T a0 = zu[2 * r], a1 = zu[2 * r + 1];
  for (int k = ptr[r]; k < ptr[r + 1]; ++k) {
    const T v = val[k];
    const int c = col[k];
    a0 -= v * lam[2 * c];
    a1 -= v * lam[2 * c + 1];
  }
  y[2 * r] = a0;
  y[2 * r + 1] = a1;
}

// Pressure part of one application of the upper block-triangular Stokes
// approximation [[A_f, -B^T], [0, -S]]^-1: p = -S^-1 in_p with the
// Cahouet-Chabard Schur approximation S^-1 ~ nu M_p^-1 + (rho/dt) L_p^-1
// (one V-cycle on the pressure Laplacian L_p = B diag(M_f)^-1 B^T).
//
// With started = true the caller has already set L0.b = in_p and
// L0.x = L0.d = c0 D^-1 in_p (k_stokes_res does it); with acc, also
// acc += omega * out_p.  Both the Schur combination and the update ride on
// the last smoothing kernel of the finest pressure level when it is a
// per-level kernel.  With zu (fused finest level only) the input is the
// residual in_p - (-B) zu, formed by the finest down launch.
template <class T>
static void stokes_pressure(Problem& P, Prec<T>& pr, const T* in_p, T* out_p, cudaStream_t s, bool started = false,
                            T* acc = nullptr, T omega = 1, const T* zu = nullptr) {
  const int n3 = 3 * P.nP;
  MGLevel<T>& L0p = pr.mgP.lv[0];
  SpmvArgs<T> fin;
  fin.sv = in_p; fin.smp = pr.mpinv; fin.sout = out_p;
  fin.snu = (T)P.prm.nu; fin.srdt = (T)(P.prm.rho_f / P.prm.dt);
  fin.acc = acc; fin.omega = omega;
  if (L0p.mf) {  // the fused finest level reads in_p itself and applies the epilogue
    if (zu) {   // the Schur combination takes the residual the down launch wrote
      MfRes<T> r;
      r.zu = zu;
      r.bout = L0p.b;
      fin.sv = L0p.b;
      const MfFin<T> mfin = mf_fin(fin);
      vcycle_mf<T>(pr.mgP, 0, in_p, s, nullptr, &mfin, &r);
      return;
    }
    const MfFin<T> mfin = mf_fin(fin);
    vcycle_mf<T>(pr.mgP, 0, in_p, s, nullptr, &mfin);
    return;
  }
  if (zu) throw std::logic_error("stokes_pressure: the residual start needs the fused finest level");
  if (!started)
    launch(k_cheb_first<T>, nblk(n3, 256), 256, 0, s, n3, in_p, L0p.dinv, (T)L0p.ch.c0, L0p.d, L0p.x, (T)1, L0p.b);
  bool fused = false;
  T* sp = vcycle<T>(pr.mgP, 0, s, (T*)nullptr, &fin, &fused);
  if (!fused) {
    launch(k_schur<T>, nblk(n3, 256), 256, 0, s, n3, in_p, sp, pr.mpinv, (T)P.prm.nu, (T)(P.prm.rho_f / P.prm.dt),
           out_p);
    if (acc) launch(k_axpy<T>, nblk(n3, 256), 256, 0, s, (size_t)n3, omega, (const T*)out_p, acc);
  }
}

// Velocity part: u = A_f^-1 (in_u + B^T p) by one V-cycle with
// Chebyshev-Jacobi smoothing on the Q2 hierarchy (p = nullptr: u = A_f^-1 in_u).
// With acc, also acc += omega * out_u (on the last smoothing kernel when the
// finest level is a per-level kernel).  With zu (fused finest level only)
// the input is the residual in_u - A_f zu + B^T p.  On the fused level the
// finest down launch forms the input itself.
template <class T>
static void stokes_velocity(Problem& P, Prec<T>& pr, const T* in_u, const T* p, T* out_u, cudaStream_t s,
                            T* acc = nullptr, T omega = 1, const T* zu = nullptr) {
  MGLevel<T>& L0u = pr.mgU.lv[0];
  if (L0u.mf) {  // the fused finest level starts its smoother itself
    MfFin<T> mfin;
    mfin.acc = acc; mfin.omega = omega;
    if (p || zu) {
      MfRes<T> r;
      r.zu = zu;
      r.zp = p;
      r.bout = L0u.b;
      vcycle_mf<T>(pr.mgU, 0, in_u, s, out_u, acc ? &mfin : nullptr, &r);
    } else {
      vcycle_mf<T>(pr.mgU, 0, in_u, s, out_u, acc ? &mfin : nullptr);
    }
    return;
  }
  if (zu) throw std::logic_error("stokes_velocity: the residual start needs the fused finest level");
  if (p) {
    SpmvArgs<T> a;
    a.x = p; a.y = L0u.b; a.z = in_u; a.alpha = -1; a.beta = 1;
    a.d = L0u.d; a.dinv = L0u.dinv; a.xo = L0u.x; a.c2 = (T)L0u.ch.c0;
    sell_launch(pr.op.Bt, MODE_INIT, a, s);
  } else {
    const int n2 = 2 * P.nU;
    launch(k_cheb_first<T>, nblk(n2, 256), 256, 0, s, n2, in_u, L0u.dinv, (T)L0u.ch.c0, L0u.d, L0u.x, (T)1, L0u.b);
  }
  SpmvArgs<T> fin;
  fin.acc = acc; fin.omega = omega;
  bool fused = false;
  vcycle(pr.mgU, 0, s, out_u, acc ? &fin : (const SpmvArgs<T>*)nullptr, &fused);
  if (acc && !fused) {
    const size_t n2 = 2 * (size_t)P.nU;
    launch(k_axpy<T>, nblk(n2, 256), 256, 0, s, n2, omega, (const T*)out_u, acc);
  }
}

// One application of the Stokes approximation to (in_u, in_p): the pressure
// part, then the velocity part with B^T p.  With split = true the pressure
// part runs on stream s4 beside the velocity part and the B^T p term is
// dropped (block-diagonal).
template <class T>
static void stokes_apply(Problem& P, Prec<T>& pr, const T* in_u, const T* in_p, T* out_u, T* out_p, cudaStream_t s,
                         bool split) {
  if (split) {
    CK(cudaEventRecord(P.ev_fork2, s));
    CK(cudaStreamWaitEvent(P.s4, P.ev_fork2, 0));
    stokes_pressure(P, pr, in_p, out_p, P.s4);
    CK(cudaEventRecord(P.ev_join2, P.s4));
    stokes_velocity(P, pr, in_u, (const T*)nullptr, out_u, s);
    CK(cudaStreamWaitEvent(s, P.ev_join2, 0));
  } else {
    stokes_pressure(P, pr, in_p, out_p, s);
    stokes_velocity(P, pr, in_u, (const T*)out_p, out_u, s);
  }
}

// One application z = P^-1 v of the block preconditioner (Section 5), input
// pr.vin, output pr.zw.
//   precond 0: diag(A_11, A_22)                      (block-diagonal)
//   precond 1: [[A_11, 0], [A_21, A_22]]             (block lower-triangular)
//   precond 2: [[A_11, A_12], [0, A_22]]             (block upper-triangular:
//              the solid block first, then the fluid with v_u - C_f^T z_l)
//   precond 3: as 2, velocity and pressure parts of A_11^-1 side by side.
// A_11^-1 is stokes_its steps of Richardson on the Stokes block, each step one
// application of stokes_apply (one step = the plain one-shot approximation).
template <class T>
static void precond_launch(Problem& P, Prec<T>& pr, cudaStream_t s) {
  const int pc = P.prm.precond;
  T* vp = pr.vin + P.offP;
  T* zp = pr.zw + P.offP;
  const bool split = (pc == 3);
  // the solid block does not depend on the fluid for precond 0, 2 and 3: run
  // it on a parallel branch (its kernels are small and latency-bound)
  if (pc != 1) {
    CK(cudaEventRecord(P.ev_fork, s));
    CK(cudaStreamWaitEvent(P.s3, P.ev_fork, 0));
    solid_launch(P, pr, P.s3);
    CK(cudaEventRecord(P.ev_join, P.s3));
  }
  const T* vu = pr.vin;
  if (pc == 2) {
    // the pressure part of the first Stokes application needs only v_p: it
    // runs beside the solid branch, and only the velocity part waits for z_l
    stokes_pressure(P, pr, vp, zp, s);
    CK(cudaStreamWaitEvent(s, P.ev_join, 0));
    launch(k_cft_sub<T>, nblk(P.nU, 128), 128, 0, s, P.nU, P.cft_ptr, P.cft_col, pr.op.cft_val, pr.zw + P.offL, pr.vin,
                                                  pr.ru);
    vu = pr.ru;
    stokes_velocity(P, pr, vu, (const T*)zp, pr.zw, s);
  } else {
    if (pc == 3) {
      CK(cudaStreamWaitEvent(s, P.ev_join, 0));
      launch(k_cft_sub<T>, nblk(P.nU, 128), 128, 0, s, P.nU, P.cft_ptr, P.cft_col, pr.op.cft_val, pr.zw + P.offL,
             pr.vin, pr.ru);
      vu = pr.ru;
    }
    stokes_apply(P, pr, vu, vp, pr.zw, zp, s, split);
  }
  const size_t nf = 2 * (size_t)P.nU + 3 * (size_t)P.nP;
  MGLevel<T>& L0p = pr.mgP.lv[0];
  for (int it = 1; it < pr.stokes_its; ++it) {
    if (split) {
      launch(k_stokes_res<T>, pr.op.gU + pr.op.gP, 128, 0, s, pr.op, pr.zw, vu, vp, pr.t, (const T*)nullptr, (T)0,
             (T*)nullptr, (T*)nullptr, (T*)nullptr);
      stokes_apply(P, pr, pr.t, pr.t + P.offP, pr.dz, pr.dz + P.offP, s, split);
      launch(k_axpy<T>, nblk(nf, 256), 256, 0, s, nf, pr.stokes_omega, pr.dz, pr.zw);
    } else if (L0p.mf && pr.mgU.lv[0].mf && (double)pr.stokes_omega == 1.0) {
      // the Stokes residual formed inside the finest down launches: the
      // pressure correction from v_p - (-B) z_u, added to z_p; then, since
      // z_p then holds the corrected pressure (omega = 1), the velocity
      // correction from v_u - A_f z_u - (-B^T) z_p, which is the upper
      // triangular step's right-hand side t_u - (-B^T) dz_p
      stokes_pressure(P, pr, vp, pr.dz + P.offP, s, false, pr.zw + P.offP, pr.stokes_omega, (const T*)pr.zw);
      stokes_velocity(P, pr, vu, (const T*)(pr.zw + P.offP), pr.dz, s, pr.zw, pr.stokes_omega, (const T*)pr.zw);
    } else {
      // residual (starting the pressure smoother), then the pressure and
      // velocity corrections, each added to z by its own last kernel
      if (L0p.mf)
        launch(k_stokes_res<T>, pr.op.gU + pr.op.gP, 128, 0, s, pr.op, pr.zw, vu, vp, pr.t, (const T*)nullptr, (T)0,
               (T*)nullptr, (T*)nullptr, (T*)nullptr);
      else
        launch(k_stokes_res<T>, pr.op.gU + pr.op.gP, 128, 0, s, pr.op, pr.zw, vu, vp, pr.t, (const T*)L0p.dinv,
               (T)L0p.ch.c0, L0p.b, L0p.d, L0p.x);
      stokes_pressure(P, pr, pr.t + P.offP, pr.dz + P.offP, s, true, pr.zw + P.offP, pr.stokes_omega);
      stokes_velocity(P, pr, pr.t, (const T*)(pr.dz + P.offP), pr.dz, s, pr.zw, pr.stokes_omega);
    }
  }
  if (pc == 1) solid_launch(P, pr, s);
  if (pc == 0) CK(cudaStreamWaitEvent(s, P.ev_join, 0));
}

// --------------------------------------------------------- Krylov kernels
// Reductions over the n unknowns use a fixed grid of nb CTAs of 256 threads,
// CTA b owning rows [512 b, 512 b + 512); per-CTA partials are summed in a
// fixed order, so every result is deterministic.  On GB300 these kernels are
// bound by the FP64 pipe (2 DFMA per clock per SM), so the multi-dot gives
// each warp whole vectors and each lane 16 rows of a vector: 16 DFMA against
// the 8 DADD of its partial sums and warp shuffle.
constexpr int kChunk = 512;

__device__ void mdot_warps(const double* __restrict__ V, size_t ld, int cnt, const double* __restrict__ ws, int r0,
                           int nrow, double* __restrict__ part, int nb) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wp; i < cnt; i += nw) {
    const double* __restrict__ v = V + (size_t)i * ld + r0;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if (nrow == kChunk) {
#pragma unroll
      for (int q = 0; q < kChunk / 128; ++q) {
        const int r = lane + 128 * q;
        a0 += v[r] * ws[r];
        a1 += v[r + 32] * ws[r + 32];
        a2 += v[r + 64] * ws[r + 64];
        a3 += v[r + 96] * ws[r + 96];
      }
    } else {
      for (int r = lane; r < nrow; r += 32) a0 += v[r] * ws[r];
    }
    const double sa = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) part[(size_t)i * nb + blockIdx.x] = sa;
  }
}

__device__ void finalize_warps(const double* __restrict__ part, int nb, int cnt, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wp; i < cnt; i += nw) {
    double acc = 0;
    for (int b = lane; b < nb; b += 32) acc += part[(size_t)i * nb + b];
    acc = warp_sum(acc);
    if (lane == 0) out[i] = acc;
  }
}

// w[r] - sum_i V[i][r] h[i] with four independent partial sums
__device__ __forceinline__ double gs_update(const double* __restrict__ V, size_t ld, int cnt, const double* hs,
                                            double w, int r) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int i = 0;
  for (; i + 3 < cnt; i += 4) {
    s0 += V[(size_t)i * ld + r] * hs[i];
    s1 += V[(size_t)(i + 1) * ld + r] * hs[i + 1];
    s2 += V[(size_t)(i + 2) * ld + r] * hs[i + 2];
    s3 += V[(size_t)(i + 3) * ld + r] * hs[i + 3];
  }
  for (; i < cnt; ++i) s0 += V[(size_t)i * ld + r] * hs[i];
  return w - ((s0 + s1) + (s2 + s3));
}

struct KrylovArgs {
  int n;
  int chunk;
  size_t ld;
  const double* V;
  double* w;
  double* part;
  int pstride;   // unused by the partial layout part[i * nb + block]
  double* h1;
  double* h2;
  double* H;
  double* cs;
  double* sn;
  double* g;
  Ctl* ctl;
  cudaGraphConditionalHandle cond;        // Arnoldi loop
  cudaGraphConditionalHandle cond_outer;  // restart / refinement loop
};

// Classical Gram-Schmidt with one refinement pass when needed (Daniel,
// Gragg, Kaufman and Stewart 1976; the "refine if needed" rule of PETSc's
// GMRES): pass 1 forms h1 = V^T w and ||w||; pass 2 updates w -= V h1 and
// forms ||w||; if the norm fell below ||w|| / sqrt(2), passes 3-4 repeat the
// projection (h2 = V^T w, w -= V h2).  Passes 3-4 return at once otherwise.

// Hessenberg column j, Givens rotation, residual estimate and the stop
// decision of the Arnoldi loop (one thread)
__device__ void arnoldi_finish(const KrylovArgs& k, double s2) {
  Ctl* c = k.ctl;
  const int j = c->j, m1 = c->m + 1;
  double* Hc = k.H + (size_t)j * m1;
  for (int i = 0; i <= j; ++i) Hc[i] = k.h1[i] + (c->refine ? k.h2[i] : 0.0);
  const double nrm = sqrt(s2);
  Hc[j + 1] = nrm;
  for (int i = 0; i < j; ++i) {
    const double a = Hc[i], b = Hc[i + 1];
    Hc[i] = k.cs[i] * a + k.sn[i] * b;
    Hc[i + 1] = -k.sn[i] * a + k.cs[i] * b;
  }
  const double a = Hc[j], b = Hc[j + 1];
  const double r = hypot(a, b);
  const double cc = (r > 0) ? a / r : 1.0, ss = (r > 0) ? b / r : 0.0;
  k.cs[j] = cc; k.sn[j] = ss;
  Hc[j] = r; Hc[j + 1] = 0.0;
  k.g[j + 1] = -ss * k.g[j];
  k.g[j] = cc * k.g[j];
  const double res = fabs(k.g[j + 1]);
  c->its += 1;
  c->res = res;
  bool stop = false;
  if (!(res == res) || !(nrm == nrm)) { c->flags |= FLAG_NAN; stop = true; c->j = j; }
  else if (r == 0.0) { c->flags |= FLAG_BREAKDOWN; stop = true; c->j = j; }
  else {
    c->j = j + 1;
    if (res <= c->cycle_tol || j + 1 >= c->m || c->its >= c->max_it || nrm == 0.0) stop = true;
  }
  c->scale = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  c->cyc_active = stop ? 0 : 1;
  if (k.cond) cudaGraphSetConditional(k.cond, stop ? 0u : 1u);
}

// pass 1: h1 = V[0..j]^T w and ||w||^2 (w is stored as vector j+1 of the dots)
__global__ void __launch_bounds__(kRedThreads) k_gs1(KrylovArgs k) {
  pdl_begin();
  __shared__ double ws[kChunk];
  __shared__ double sm[32];
  const int cnt = k.ctl->j + 1;
  const int r0 = blockIdx.x * kChunk, r1 = min(k.n, r0 + kChunk);
  double acc = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double v = k.w[r];
    ws[r - r0] = v;
    acc += v * v;
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) k.part[(size_t)cnt * gridDim.x + blockIdx.x] = acc;
  __syncthreads();
  mdot_warps(k.V, k.ld, cnt, ws, r0, r1 - r0, k.part, gridDim.x);
  if (last_block(&k.ctl->counter[0])) {
    finalize_warps(k.part, gridDim.x, cnt + 1, k.h1);
    __syncthreads();
    if (threadIdx.x == 0) {
      k.ctl->wnorm2 = k.h1[cnt];
      k.ctl->counter[0] = 0;
    }
  }
}

// pass 2: w -= V h1 and ||w||^2; finish the step or ask for refinement
__global__ void __launch_bounds__(kRedThreads) k_gs2(KrylovArgs k) {
  pdl_begin();
  __shared__ double hs[256];
  __shared__ double sm[32];
  const int cnt = k.ctl->j + 1;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) hs[i] = k.h1[i];
  __syncthreads();
  const int r0 = blockIdx.x * kChunk, r1 = min(k.n, r0 + kChunk);
  double acc = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double v = gs_update(k.V, k.ld, cnt, hs, k.w[r], r);
    k.w[r] = v;
    acc += v * v;
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) k.part[blockIdx.x] = acc;
  if (last_block(&k.ctl->counter[1])) {
    double a = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a += k.part[b];
    const double s2 = block_sum(a, sm);
    if (threadIdx.x == 0) {
      Ctl* c = k.ctl;
      c->counter[1] = 0;
      c->refine = (s2 < 0.5 * c->wnorm2) ? 1 : 0;
      if (c->refine) c->refines += 1;
      else arnoldi_finish(k, s2);
    }
  }
}

// pass 3 (refinement only): h2 = V^T w
__global__ void __launch_bounds__(kRedThreads) k_gs3(KrylovArgs k) {
  pdl_begin();
  __shared__ double ws[kChunk];
  if (!k.ctl->refine) return;
  const int cnt = k.ctl->j + 1;
  const int r0 = blockIdx.x * kChunk, r1 = min(k.n, r0 + kChunk);
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) ws[r - r0] = k.w[r];
  __syncthreads();
  mdot_warps(k.V, k.ld, cnt, ws, r0, r1 - r0, k.part, gridDim.x);
  if (last_block(&k.ctl->counter[2])) {
    finalize_warps(k.part, gridDim.x, cnt, k.h2);
    if (threadIdx.x == 0) k.ctl->counter[2] = 0;
  }
}

// pass 4 (refinement only): w -= V h2, ||w||^2, finish the step
__global__ void __launch_bounds__(kRedThreads) k_gs4(KrylovArgs k) {
  pdl_begin();
  __shared__ double hs[256];
  __shared__ double sm[32];
  if (!k.ctl->refine) return;
  const int cnt = k.ctl->j + 1;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) hs[i] = k.h2[i];
  __syncthreads();
  const int r0 = blockIdx.x * kChunk, r1 = min(k.n, r0 + kChunk);
  double acc = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double v = gs_update(k.V, k.ld, cnt, hs, k.w[r], r);
    k.w[r] = v;
    acc += v * v;
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) k.part[blockIdx.x] = acc;
  if (last_block(&k.ctl->counter[6])) {
    double a = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a += k.part[b];
    const double s2 = block_sum(a, sm);
    if (threadIdx.x == 0) {
      k.ctl->counter[6] = 0;
      arnoldi_finish(k, s2);
    }
  }
}

// V[j] = w * scale (j already advanced)
__global__ void k_gs_scale(int n, double* __restrict__ V, size_t ld, const double* __restrict__ w, const Ctl* ctl) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  V[(size_t)ctl->j * ld + i] = w[i] * ctl->scale;
}

// start of a cycle: beta = ||w|| with w = b - A x already formed
__global__ void __launch_bounds__(kRedThreads) k_cycle_start(KrylovArgs k) {
  pdl_begin();
  __shared__ double sm[32];
  const int r0 = blockIdx.x * k.chunk, r1 = min(k.n, r0 + k.chunk);
  double acc = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) acc += k.w[r] * k.w[r];
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) k.part[blockIdx.x] = acc;
  if (last_block(&k.ctl->counter[3])) {
    double a = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a += k.part[b];
    const double s2 = block_sum(a, sm);
    if (threadIdx.x == 0) {
      Ctl* c = k.ctl;
      c->counter[3] = 0;
      const double beta = sqrt(s2);
      c->beta = beta;
      c->j = 0;
      c->cycles += 1;
      k.g[0] = beta;
      c->last_true = (c->bnorm > 0) ? beta / c->bnorm : beta;
      bool stop = false;
      if (!(beta == beta)) { c->flags |= FLAG_NAN; stop = true; }
      c->converged = (beta <= c->target) ? 1 : 0;
      if (c->converged || c->its >= c->max_it || c->cycles > c->max_cycles ||
          (c->flags & (FLAG_NAN | FLAG_BREAKDOWN)) || c->aflags)
        stop = true;
      c->stop = stop ? 1 : 0;
      c->cycle_tol = fmax(c->inner_rtol * beta, c->target);
      c->scale = (beta > 0) ? 1.0 / beta : 0.0;
      c->res = beta;
      c->cyc_active = stop ? 0 : 1;
      if (k.cond) cudaGraphSetConditional(k.cond, stop ? 0u : 1u);
      if (k.cond_outer) cudaGraphSetConditional(k.cond_outer, stop ? 0u : 1u);
    }
  }
}

__global__ void k_scale0(int n, double* __restrict__ V, const double* __restrict__ w, const Ctl* ctl) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  V[i] = w[i] * ctl->scale;
}

// ||b||, the target, and reset of the per-solve counters
__global__ void __launch_bounds__(kRedThreads) k_solve_begin(KrylovArgs k, const double* __restrict__ b, double rtol,
                                                             double inner_rtol, int max_it, int m, int max_cycles) {
  pdl_begin();
  __shared__ double sm[32];
  const int r0 = blockIdx.x * k.chunk, r1 = min(k.n, r0 + k.chunk);
  double acc = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) acc += b[r] * b[r];
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) k.part[blockIdx.x] = acc;
  if (last_block(&k.ctl->counter[4])) {
    double a = 0;
    for (int bb = threadIdx.x; bb < (int)gridDim.x; bb += blockDim.x) a += k.part[bb];
    const double s2 = block_sum(a, sm);
    if (threadIdx.x == 0) {
      Ctl* c = k.ctl;
      c->counter[4] = 0;
      c->bnorm = sqrt(s2);
      c->target = rtol * c->bnorm;
      c->inner_rtol = inner_rtol;
      c->its = 0; c->cycles = 0; c->j = 0; c->flags = 0; c->refines = 0; c->refine = 0;
      c->converged = 0; c->stop = 0;
      c->max_it = max_it; c->m = m; c->max_cycles = max_cycles;
    }
  }
}

// least squares on the rotated Hessenberg matrix: y = R^-1 g (one thread)
__global__ void k_lsq(const double* __restrict__ H, const double* __restrict__ g, double* __restrict__ y,
                      const Ctl* ctl) {
  pdl_begin();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int kk = ctl->j, m1 = ctl->m + 1;
  for (int i = kk - 1; i >= 0; --i) {
    double v = g[i];
    for (int l = i + 1; l < kk; ++l) v -= H[(size_t)l * m1 + i] * y[l];
    y[i] = v / H[(size_t)i * m1 + i];
  }
}

// x += Z y (right preconditioning: the update lives in span{Z})
template <class T>
__global__ void k_xupdate(int n, double* __restrict__ x, const T* __restrict__ Z, size_t ld,
                          const double* __restrict__ y, const Ctl* ctl) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int kk = ctl->j;
  double v = x[i];
  for (int l = 0; l < kk; ++l) v += (double)Z[(size_t)l * ld + i] * y[l];
  x[i] = v;
}

template <class T>
__global__ void k_prec_in(int n, const double* __restrict__ V, size_t ld, const Ctl* ctl, T* __restrict__ vin) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) vin[i] = (T)V[(size_t)ctl->j * ld + i];
}

template <class T>
__global__ void k_prec_out(int n, const T* __restrict__ zw, T* __restrict__ Z, size_t ld, const Ctl* ctl) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Z[(size_t)ctl->j * ld + i] = zw[i];
}

// zero mean of the constant pressure coefficients (p in L^2_0)
__global__ void __launch_bounds__(kRedThreads) k_pmean(int nP, double* __restrict__ p, double* __restrict__ part,
                                                       Ctl* ctl) {
  pdl_begin();
  __shared__ double sm[32];
  double acc = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nP; c += gridDim.x * blockDim.x) acc += p[3 * (size_t)c];
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  if (last_block(&ctl->counter[5])) {
    if (threadIdx.x == 0) {
      double s = 0;
      for (int b = 0; b < (int)gridDim.x; ++b) s += part[b];
      ctl->counter[5] = 0;
      ctl->pmean = s / nP;
    }
  }
}

__global__ void k_psub(int nP, double* __restrict__ p, const Ctl* ctl) {
  pdl_begin();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nP) p[3 * (size_t)c] -= ctl->pmean;
}

// ------------------------------------------------------------------ setup
static void check_params(const fsi_params& p, int n_nodes, int n_tris) {
  if (p.N < 2 || p.N > 4096 || (p.N & 1)) throw std::invalid_argument("N must be even, 2..4096");
  int Nc = p.N;
  while (Nc % 2 == 0 && Nc > 4) Nc /= 2;
  if (Nc > 8) throw std::invalid_argument("N must be c * 2^k with c <= 8");
  if (!(p.dt > 0) || !(p.rho_f > 0) || !(p.nu > 0) || !(p.kappa >= 0)) throw std::invalid_argument("bad material");
  if (p.precond < 0 || p.precond > 3) throw std::invalid_argument("precond");
  if (p.precision != 0 && p.precision != 1) throw std::invalid_argument("precision");
  if (p.solid_elem != 0 && p.solid_elem != 1) throw std::invalid_argument("solid_elem");
  if (n_nodes < (p.solid_elem == 1 ? 4 : 3) || n_tris < 1) throw std::invalid_argument("solid mesh");
  if (p.solid_elem == 1 && (p.coupling != 0 || p.solid_law != 0))
    throw std::invalid_argument("the Q1 solid takes the point rule and the linear law");
  if (p.mg_cluster < -1) throw std::invalid_argument("mg_cluster");
  if (p.mg_fused != 0 && p.mg_fused != -1) throw std::invalid_argument("mg_fused");
  if (p.mg_coarse > 32) throw std::invalid_argument("mg_coarse must be at most 32");
  if (p.mg_coarse_p > 32) throw std::invalid_argument("mg_coarse_p must be at most 32");
  if (p.coupling != 0 && p.coupling != 1) throw std::invalid_argument("coupling");
  if (p.solid_law != 0 && p.solid_law != 1) throw std::invalid_argument("solid_law");
  if (p.autotune != 0 && p.autotune != 1) throw std::invalid_argument("autotune");
  if (p.solid_law == 1 && !(p.gamma > 0 && p.eta > 0)) throw std::invalid_argument("gamma, eta");
  // the Givens kernels hold one Hessenberg column in shared memory (256 doubles)
  if (p.restart > 250) throw std::invalid_argument("restart must be <= 250");
  if (p.stokes_its > 16) throw std::invalid_argument("stokes_its must be <= 16");
}

// Node ids per solid element and rule points per element (P1: the 6-point
// triangle rule; Q1: 3 x 3 Gauss).
static int elem_nodes(const fsi_params& p) { return p.solid_elem == 1 ? 4 : 3; }
static int elem_points(const fsi_params& p) { return p.solid_elem == 1 ? 9 : 6; }

static fsi_params with_defaults(fsi_params p) {
  if (p.restart <= 0) p.restart = 200;
  if (!(p.rtol > 0)) p.rtol = 1e-8;
  if (p.max_it <= 0) p.max_it = 1000;
  if (p.mg_degree <= 0) p.mg_degree = 2;
  // Q1: D^-1 C_s has a wider interval ([1/4, 9/4] on squares against [1/2, 2]
  // for P1), so about 1.6 x the Chebyshev steps for the same reduction
  if (p.cs_degree <= 0) p.cs_degree = (p.precision == 1) ? (p.solid_elem == 1 ? 20 : 12) : (p.solid_elem == 1 ? 26 : 16);
  if (!(p.inner_rtol > 0)) p.inner_rtol = 1e-5;
  if (p.max_refine <= 0) p.max_refine = 30;
  if (p.stokes_its <= 0) p.stokes_its = 1;
  if (!(p.stokes_omega > 0)) p.stokes_omega = 1.0;
  if (!(p.newton_tol > 0)) p.newton_tol = 1e-6;
  if (p.newton_max <= 0) p.newton_max = 20;
  // coarsest grid 16 cells: one dense product (a 15 MB FP32 inverse, held in
  // L2) in place of the 16-cell level's two launches and the 8-cell solve
  if (p.mg_coarse <= 0) p.mg_coarse = 16;
  if (p.mg_coarse_p <= 0) p.mg_coarse_p = p.mg_coarse;
  return p;
}

template <class T>
static void build_prec(Problem& P, Prec<T>& pr, const FullOp<T>& op, bool alloc_all) {
  (void)alloc_all;
  Arena& ar = P.ar;
  const bool f64 = std::is_same<T, double>::value;
  build_mg<T>(ar, P.hs, false, P.prm.mg_degree, pr.mgU, P.prm.autotune == 1, P.stream,
              f64 ? nullptr : P.p64.mgU.coarse_inv, P.p64.mgU.coarse_ld);
  build_mg<T>(ar, P.hs, true, P.prm.mg_degree, pr.mgP, P.prm.autotune == 1, P.stream,
              f64 ? nullptr : P.p64.mgP.coarse_inv, P.p64.mgP.coarse_ld);
  // With the fused matrix-free levels (FP32, every level of 16 cells or more)
  // the automatic choice leaves the cluster out: two fused launches per level
  // measured faster than the cluster launch of the same levels on GB300
  // (10.8 against 9.7 steps/s on the 128 x 128 cavity).
  int cl_max = P.prm.mg_cluster;
  if (cl_max == 0 && std::is_same<T, float>::value && P.prm.mg_fused == 0) cl_max = 8;
  if (cl_max >= 0) {
    setup_cluster<T>(ar, P.hs, pr.mgU, false, cl_max);
    setup_cluster<T>(ar, P.hs, pr.mgP, true, cl_max);
  }
  select_mf<T>(pr.mgU, P.hs, P.prm.mg_fused, ar.count_only);
  select_mf<T>(pr.mgP, P.hs, P.prm.mg_fused, ar.count_only);
  pr.op = op;
  pr.Cs = upload_sell<T>(ar, to_sell(P.hs.Cs));
  pr.As = upload_sell<T>(ar, to_sell(P.hs.As));
  if (P.prm.solid_law == 1) {
    pr.KT.nrows = P.nS; pr.KT.BR = 2; pr.KT.BC = 2; pr.KT.NV = 4; pr.KT.kron = false;
    pr.KT.soff = op.Ssol.soff; pr.KT.len = op.Ssol.len; pr.KT.col = op.Ssol.col;
    if constexpr (std::is_same<T, double>::value) pr.KT.val = P.kt64;
    else pr.KT.val = P.kt32;
  }
  pr.mpinv = upload_as<T>(ar, P.hs.mp_inv);
  pr.csdinv = upload_as<T>(ar, P.hs.cs_dinv);
  pr.vin = ar.alloc<T>(P.n);
  pr.zw = ar.alloc<T>(P.n);
  const size_t n2 = 2 * (size_t)P.nS;
  pr.sb = ar.alloc<T>(n2); pr.sx = ar.alloc<T>(n2); pr.sx2 = ar.alloc<T>(n2); pr.sd = ar.alloc<T>(n2);
  pr.cs_k = P.prm.cs_degree;
  pr.chs = cheb_coeffs(P.hs.cs_lo, P.hs.cs_hi, pr.cs_k);
  const size_t nf = 2 * (size_t)P.nU + 3 * (size_t)P.nP;
  pr.ru = ar.alloc<T>(2 * (size_t)P.nU);
  pr.t = ar.alloc<T>(nf);
  pr.dz = ar.alloc<T>(nf);
  pr.stokes_its = P.prm.stokes_its;
  pr.stokes_omega = (T)P.prm.stokes_omega;
}

template <class T>
static FullOp<T> make_op(Problem& P, const T* cfv, const T* cftv) {
  Arena& ar = P.ar;
  FullOp<T> op;
  op.nU = P.nU; op.nP = P.nP; op.nS = P.nS;
  op.gU = nblk(P.nU, 32); op.gP = nblk(P.nP, 32); op.gS = nblk(P.nS, 32);
  op.Af = upload_sell<T>(ar, to_sell(P.hs.levels[0].A));
  op.Bt = upload_sell<T>(ar, to_sell(P.hs.Bt));
  op.Bneg = upload_sell<T>(ar, to_sell(P.hs.Bneg));
  op.Ssol = upload_sell<T>(ar, to_sell(P.hs.Ssol));
  op.cft_ptr = P.cft_ptr; op.cft_col = P.cft_col; op.cft_val = cftv;
  op.cf_len = P.cf_len; op.cf_col = P.cf_col; op.cf_val = cfv; op.cf_cap = P.cf_cap;
  op.inv_dt = (T)(1.0 / P.prm.dt);
  if (P.prm.solid_law == 1) {
    if constexpr (std::is_same<T, double>::value) op.kt = P.kt64;
    else op.kt = P.kt32;
  }
  return op;
}

static KrylovArgs krylov_args(Problem& P, cudaGraphConditionalHandle h) {
  KrylovArgs k{};
  k.n = (int)P.n;
  k.chunk = kChunk;
  k.ld = P.n;
  k.V = P.V;
  k.w = P.w;
  k.part = P.part;
  k.pstride = P.m + 1;
  k.h1 = P.y + (P.m + 2);       // scratch after y (m+2 entries each)
  k.h2 = P.y + 2 * (P.m + 2);
  k.H = P.H; k.cs = P.cs; k.sn = P.sn; k.g = P.g;
  k.ctl = P.ctl;
  k.cond = h;
  return k;
}

// S2 + S4 by the point rule: locate the rule points, then the C_f rows.
static void point_rule_launch(Problem& P, cudaStream_t s) {
  if (elem_nodes(P.prm) == 4) {
    launch(k_locate<4>, nblk(P.nPts, 256), 256, 0, s, P.nPts, P.N, P.tris, P.Xold, P.cell, P.xi, P.eta,
           &P.ctl->aflags);
    launch(k_cf_rows<4>, nblk(P.nS, kCfWarps), 32 * kCfWarps, 0, s, P.nS, P.N, P.ntp, P.nt, P.area, P.cell, P.xi,
           P.eta, P.l2n, P.wall, P.cf_cap, P.cf_len, P.cf_col, P.cf_val, P.cf_val32, P.cflift, &P.ctl->aflags);
  } else {
    launch(k_locate<3>, nblk(P.nPts, 256), 256, 0, s, P.nPts, P.N, P.tris, P.Xold, P.cell, P.xi, P.eta,
           &P.ctl->aflags);
    launch(k_cf_rows<3>, nblk(P.nS, kCfWarps), 32 * kCfWarps, 0, s, P.nS, P.N, P.ntp, P.nt, P.area, P.cell, P.xi,
           P.eta, P.l2n, P.wall, P.cf_cap, P.cf_len, P.cf_col, P.cf_val, P.cf_val32, P.cflift, &P.ctl->aflags);
  }
}

static void assemble_launch(Problem& P, cudaStream_t s) {
  CK(cudaMemsetAsync(&P.ctl->aflags, 0, sizeof(int), s));
  if (P.prm.coupling == 1) {  // the paper's exact rule: mesh intersection
    launch(k_cf_rows_exact, nblk(P.nS, kCfWarps), 32 * kCfWarps, 0, s, P.nS, P.N, P.ntp, P.nt, P.tris, P.Xold, P.area,
           P.l2n, P.wall, P.cf_cap, P.cf_len, P.cf_col, P.cf_val, P.cf_val32, P.cflift, &P.ctl->aflags);
  } else {                    // located points of the point rule
    point_rule_launch(P, s);
  }
  CK(cudaMemsetAsync(P.cft_cnt, 0, sizeof(int) * P.nU, s));
  const size_t nslot = (size_t)P.nS * P.cf_cap;
  launch(k_cft_count, nblk(nslot, 256), 256, 0, s, P.nS, P.cf_cap, P.cf_len, P.cf_col, P.cft_cnt);
  const int nb = (int)nblk(P.nU, kScanBlock);
  launch(k_scan_partial, nb, kScanBlock, 0, s, P.nU, P.cft_cnt, P.scan_bsum);
  launch(k_scan_top, 1, kScanBlock, 0, s, nb, P.scan_bsum);
  launch(k_scan_final, nb, kScanBlock, 0, s, P.nU, P.cft_cnt, P.scan_bsum, P.cft_ptr, P.cft_cur);
  launch(k_cft_scatter, nblk(nslot, 256), 256, 0, s, P.nS, P.cf_cap, P.cf_len, P.cf_col, P.cf_val, P.cft_cur,
                                                 P.cft_col, P.cft_val);
  launch(k_cft_sort, nblk(P.nU, 128), 128, 0, s, P.nU, P.cft_ptr, P.cft_col, P.cft_val, P.cft_val32);
  // S1: g1 = (rho/dt) M u^n - K_ID u_D ;  g2 = -(1/dt) C_s X^n - C_D u_D
  sell_launch(P.M64, MODE_AXPBY, axpby<double>(P.uold, P.b, P.lift_u, P.prm.rho_f / P.prm.dt, 1.0), s);
  sell_launch(P.Cs64, MODE_AXPBY, axpby<double>(P.Xold, P.b + P.offL, P.cflift, -1.0 / P.prm.dt, -1.0), s);
}

template <class T>
static void iteration_launch(Problem& P, Prec<T>& pr, const KrylovArgs& k, cudaStream_t s) {
  const unsigned gn = nblk(P.n, 256);
  launch(k_prec_in<T>, gn, 256, 0, s, (int)P.n, P.V, P.n, P.ctl, pr.vin);
  precond_launch(P, pr, s);
  launch(k_prec_out<T>, gn, 256, 0, s, (int)P.n, pr.zw, (T*)P.Z, P.n, P.ctl);
  launch(k_fullmv<T, T, double>, pr.op.gU + pr.op.gP + pr.op.gS, 128, 0, s, pr.op, pr.zw, P.w, nullptr, 1.0, 0.0);
  launch(k_gs1, P.red_blocks, kRedThreads, 0, s, k);
  launch(k_gs2, P.red_blocks, kRedThreads, 0, s, k);
  launch(k_gs3, P.red_blocks, kRedThreads, 0, s, k);
  launch(k_gs4, P.red_blocks, kRedThreads, 0, s, k);
  launch(k_gs_scale, gn, 256, 0, s, (int)P.n, P.V, P.n, P.w, P.ctl);
}

static void cycle_start_launch(Problem& P, const KrylovArgs& k, cudaStream_t s) {
  launch(k_fullmv<double, double, double>, P.op64.gU + P.op64.gP + P.op64.gS, 128, 0, s, P.op64, P.x, P.w, P.b, -1.0, 1.0);
  launch(k_cycle_start, P.red_blocks, kRedThreads, 0, s, k);
  launch(k_scale0, nblk(P.n, 256), 256, 0, s, (int)P.n, P.V, P.w, P.ctl);
}

template <class T>
static void cycle_end_launch(Problem& P, cudaStream_t s) {
  launch(k_lsq, 1, 32, 0, s, P.H, P.g, P.y, P.ctl);
  launch(k_xupdate<T>, nblk(P.n, 256), 256, 0, s, (int)P.n, P.x, (const T*)P.Z, P.n, P.y, P.ctl);
}

static int count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  CK(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CK(cudaGraphGetNodes(g, nodes.data(), &n));
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// The whole solve as one graph: an outer WHILE node over restart/refinement
// cycles whose body computes the true FP64 residual (k_cycle_start sets both
// conditions), runs the Arnoldi loop as an inner WHILE node (k_gs2/k_gs4 set
// its condition) and updates x.  No host round trip inside a solve.
template <class T>
static void build_cycle_graph(Problem& P, Prec<T>& pr) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h_out;
  CK(cudaGraphConditionalHandleCreate(&h_out, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams op = {};
  op.type = cudaGraphNodeTypeConditional;
  op.conditional.handle = h_out;
  op.conditional.type = cudaGraphCondTypeWhile;
  op.conditional.size = 1;
  cudaGraphNode_t onode;
  CK(cudaGraphAddNode(&onode, g, nullptr, nullptr, 0, &op));
  cudaGraph_t obody = op.conditional.phGraph_out[0];
  cudaStream_t s = P.s2;
  CK(cudaStreamBeginCaptureToGraph(s, obody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaGraphConditionalHandle h_in;
  CK(cudaGraphConditionalHandleCreate(&h_in, obody, 0, 0));
  KrylovArgs k = krylov_args(P, h_in);
  k.cond_outer = h_out;
  cycle_start_launch(P, k, s);
  cudaStreamCaptureStatus st;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &ndeps));
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = h_in;
  ip.conditional.type = cudaGraphCondTypeWhile;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  CK(cudaGraphAddNode(&inode, cg, deps, nullptr, ndeps, &ip));
  CK(cudaStreamUpdateCaptureDependencies(s, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t ibody = ip.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(P.s5, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  KrylovArgs ki = k;
  ki.cond_outer = 0;
  iteration_launch(P, pr, ki, P.s5);
  CK(cudaStreamEndCapture(P.s5, &ibody));
  P.kn_body = count_kernel_nodes(ibody);
  cycle_end_launch<T>(P, s);
  CK(cudaStreamEndCapture(s, &obody));
  P.kn_cycle = count_kernel_nodes(obody);
  P.gr_cycle = g;
  CK(cudaGraphInstantiate(&P.g_cycle, P.gr_cycle, 0));
}

template <class T>
static void build_host_loop_graphs(Problem& P, Prec<T>& pr) {
  cudaStream_t s = P.stream;
  KrylovArgs k = krylov_args(P, 0);
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cycle_start_launch(P, k, s);
  CK(cudaStreamEndCapture(s, &P.gr_cstart));
  CK(cudaGraphInstantiate(&P.g_cstart, P.gr_cstart, 0));
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  iteration_launch(P, pr, k, s);
  CK(cudaStreamEndCapture(s, &P.gr_body));
  CK(cudaGraphInstantiate(&P.g_body, P.gr_body, 0));
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cycle_end_launch<T>(P, s);
  CK(cudaStreamEndCapture(s, &P.gr_cend));
  CK(cudaGraphInstantiate(&P.g_cend, P.gr_cend, 0));
  P.kn_body = count_kernel_nodes(P.gr_body);
}

static void build_graphs(Problem& P) {
  cudaStream_t s = P.stream;
  // assemble
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  assemble_launch(P, s);
  CK(cudaStreamEndCapture(s, &P.gr_assemble));
  CK(cudaGraphInstantiate(&P.g_assemble, P.gr_assemble, 0));
  // begin: ||b|| and counters
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  {
    KrylovArgs k = krylov_args(P, 0);
    const double inner = (P.prm.precision == 1) ? P.prm.inner_rtol : 0.0;
    const int max_cycles = (P.prm.precision == 1) ? P.prm.max_refine + 1 : (1 << 30);
    launch(k_solve_begin, P.red_blocks, kRedThreads, 0, s, k, P.b, P.prm.rtol, inner, P.prm.max_it, P.m, max_cycles);
  }
  CK(cudaStreamEndCapture(s, &P.gr_begin));
  CK(cudaGraphInstantiate(&P.g_begin, P.gr_begin, 0));
  // cycle
  const char* hl = getenv("FSI_HOST_LOOP");
  P.host_loop = hl && hl[0] == '1';
  if (P.host_loop) {
    if (P.prm.precision == 1) build_host_loop_graphs<float>(P, P.p32);
    else build_host_loop_graphs<double>(P, P.p64);
  } else {
    if (P.prm.precision == 1) build_cycle_graph<float>(P, P.p32);
    else build_cycle_graph<double>(P, P.p64);
  }
  // finish: zero-mean pressure
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  launch(k_pmean, std::min(64, (int)nblk(P.nP, kRedThreads)), kRedThreads, 0, s, P.nP, P.x + P.offP, P.part, P.ctl);
  launch(k_psub, nblk(P.nP, 256), 256, 0, s, P.nP, P.x + P.offP, P.ctl);
  CK(cudaStreamEndCapture(s, &P.gr_finish));
  CK(cudaGraphInstantiate(&P.g_finish, P.gr_finish, 0));
  P.kn_assemble = count_kernel_nodes(P.gr_assemble);
  P.kn_begin = count_kernel_nodes(P.gr_begin);
  if (P.host_loop) P.kn_cycle = count_kernel_nodes(P.gr_cstart) + count_kernel_nodes(P.gr_cend);
  P.kn_finish = count_kernel_nodes(P.gr_finish);
}

static void allocate_problem(Problem& P, const double* ref_xy, const int* tris_h) {
  Arena& ar = P.ar;
  const HostSetup& hs = P.hs;
  const int npe = elem_nodes(P.prm);
  P.tris = ar.upload(std::vector<int>(tris_h, tris_h + npe * (size_t)P.nTri));
  P.area = ar.upload(npe == 4 ? hs.pt_w : hs.tri_area);
  P.ntp = ar.upload(hs.node_tri_ptr);
  P.nt = ar.upload(hs.node_tri);
  P.l2n = ar.upload(hs.lattice_to_node);
  P.wall = ar.upload(hs.wall_u);
  P.cell = ar.alloc<int>(P.nPts);
  P.xi = ar.alloc<double>(P.nPts);
  P.eta = ar.alloc<double>(P.nPts);
  // capacity of a coupling row: the fluid lattice nodes of the cells that the
  // triangles around one solid node overlap in the reference configuration
  // (at least 64, at most the assembly window); a row that outgrows it later
  // raises FSI_ERR_CAPACITY
  {
    int need = 64;
    for (int l = 0; l < P.nS; ++l) {
      double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
      for (int k = hs.node_tri_ptr[l]; k < hs.node_tri_ptr[l + 1]; ++k) {
        const int t = hs.node_tri[k] / npe;
        for (int v = 0; v < npe; ++v)
          for (int c = 0; c < 2; ++c) {
            const double x = ref_xy[2 * (size_t)tris_h[npe * (size_t)t + v] + c];
            lo[c] = std::min(lo[c], x);
            hi[c] = std::max(hi[c], x);
          }
      }
      if (hi[0] < lo[0]) continue;
      const int cw = (int)std::floor(hi[0] * P.N) - (int)std::floor(lo[0] * P.N) + 1;
      const int ch = (int)std::floor(hi[1] * P.N) - (int)std::floor(lo[1] * P.N) + 1;
      need = std::max(need, (2 * cw + 1) * (2 * ch + 1));
    }
    P.cf_cap = std::min(need, kCfWindow);
  }
  if (P.prm.solid_law == 1) {
    std::vector<double> tg(6 * (size_t)P.nTri);
    for (int t = 0; t < P.nTri; ++t) {
      const double* p0 = ref_xy + 2 * (size_t)tris_h[3 * t];
      const double* p1 = ref_xy + 2 * (size_t)tris_h[3 * t + 1];
      const double* p2 = ref_xy + 2 * (size_t)tris_h[3 * t + 2];
      const double d1x = p1[0] - p0[0], d1y = p1[1] - p0[1], d2x = p2[0] - p0[0], d2y = p2[1] - p0[1];
      const double det = d1x * d2y - d1y * d2x;
      const double g1x = d2y / det, g1y = -d2x / det, g2x = -d1y / det, g2y = d1x / det;
      const double v[6] = {-(g1x + g2x), -(g1y + g2y), g1x, g1y, g2x, g2y};
      for (int q = 0; q < 6; ++q) tg[6 * (size_t)t + q] = v[q];
    }
    P.tgrad = ar.upload(tg);
    const SellHost ss = to_sell(hs.Ssol);
    const size_t nslot = (size_t)ss.soff[ss.nslices];
    P.kt64 = ar.alloc<double>(4 * nslot);
    P.kt32 = ar.alloc<float>(4 * nslot);
  }
  const size_t cfslots = (size_t)nblk(P.nS, 32) * 32 * P.cf_cap;
  P.cf_len = ar.alloc<int>(P.nS);
  P.cf_col = ar.alloc<int>(cfslots);
  P.cf_val = ar.alloc<double>(cfslots);
  P.cf_val32 = ar.alloc<float>(cfslots);
  P.cflift = ar.alloc<double>(2 * (size_t)P.nS);
  const size_t tcap = (size_t)P.nS * P.cf_cap;
  P.cft_ptr = ar.alloc<int>(P.nU + 1);
  P.cft_col = ar.alloc<int>(tcap);
  P.cft_val = ar.alloc<double>(tcap);
  P.cft_val32 = ar.alloc<float>(tcap);
  P.cft_cnt = ar.alloc<int>(P.nU);
  P.cft_cur = ar.alloc<int>(P.nU);
  P.scan_bsum = ar.alloc<int>(nblk(P.nU, kScanBlock) + 1);
  P.x = ar.alloc<double>(P.n);
  P.b = ar.alloc<double>(P.n);
  P.w = ar.alloc<double>(P.n);
  P.uold = ar.alloc<double>(2 * (size_t)P.nU);
  P.Xold = ar.alloc<double>(2 * (size_t)P.nS);
  P.lift_u = ar.upload(hs.lift_u);
  P.M64 = upload_sell<double>(ar, to_sell(hs.M));
  P.Cs64 = upload_sell<double>(ar, to_sell(hs.Cs));
  const int m = P.m;
  P.V = ar.alloc<double>((size_t)(m + 1) * P.n);
  if (P.prm.precision == 1) P.Z = ar.alloc<float>((size_t)m * P.n);
  else P.Z = ar.alloc<double>((size_t)m * P.n);
  P.H = ar.alloc<double>((size_t)(m + 1) * m);
  P.cs = ar.alloc<double>(m + 1);
  P.sn = ar.alloc<double>(m + 1);
  P.g = ar.alloc<double>(m + 2);
  P.y = ar.alloc<double>(3 * (size_t)(m + 2));
  P.red_blocks = (int)((P.n + kChunk - 1) / kChunk);
  P.part = ar.alloc<double>((size_t)std::max(P.red_blocks, 64) * (m + 2));
  P.ctl = ar.alloc<Ctl>(1);
  P.op64 = make_op<double>(P, P.cf_val, P.cft_val);
  build_prec<double>(P, P.p64, P.op64, true);
  if (P.prm.precision == 1) {
    P.op32 = make_op<float>(P, P.cf_val32, P.cft_val32);
    build_prec<float>(P, P.p32, P.op32, true);
  }
  (void)ref_xy;
}


// ----------------------------------------------------------- timing hook
template <class T>
static double sell_bytes(const HostBlockMatrix& A) {
  return (double)A.nnzb() * (A.NV * sizeof(T) + sizeof(int));  // stored blocks: values + column index
}

template <class T>
static double fullop_bytes(Problem& P, double cfnnz, size_t xbytes, size_t ybytes) {
  const HostSetup& hs = P.hs;
  double b = sell_bytes<T>(hs.levels[0].A) + sell_bytes<T>(hs.Bt) + sell_bytes<T>(hs.Bneg) + sell_bytes<T>(hs.Ssol);
  b += 2.0 * cfnnz * (sizeof(T) + sizeof(int)) + (P.nU + 1) * 4.0 + P.nS * 4.0;
  b += (double)P.n * (xbytes + ybytes);
  return b;
}

__global__ void k_flush(size_t n, uint4* __restrict__ buf, unsigned v) {
  pdl_begin();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    buf[i] = make_uint4(v, v, v, v);
}

}  // namespace fsi

// ================================================================== C ABI
using namespace fsi;

struct fsi_problem {
  Problem P;
};

static int map_exception() {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return FSI_ERR_OOM;
  } catch (const std::invalid_argument&) {
    return FSI_ERR_INVALID;
  } catch (const CudaError& e) {
    if (e.code == cudaErrorMemoryAllocation) return FSI_ERR_OOM;
    return FSI_ERR_CUDA;
  } catch (...) {
    return FSI_ERR_CUDA;
  }
}

static void upload_state(Problem& P, const double* u, const double* X) {
  const int n1 = 2 * P.N + 1;
  if (u) {
    std::vector<double> ui(2 * (size_t)P.nU);
    for (int k = 0; k < P.nU; ++k) {
      const int lat = P.hs.interior_lattice[k];
      ui[2 * k] = u[2 * (size_t)lat];
      ui[2 * k + 1] = u[2 * (size_t)lat + 1];
    }
    CK(cudaMemcpyAsync(P.uold, ui.data(), ui.size() * 8, cudaMemcpyHostToDevice, P.stream));
    CK(cudaMemcpyAsync(P.x, ui.data(), ui.size() * 8, cudaMemcpyHostToDevice, P.stream));
    CK(cudaStreamSynchronize(P.stream));
  }
  if (X) {
    CK(cudaMemcpyAsync(P.Xold, X, 2 * (size_t)P.nS * 8, cudaMemcpyHostToDevice, P.stream));
    CK(cudaMemcpyAsync(P.x + P.offX, X, 2 * (size_t)P.nS * 8, cudaMemcpyHostToDevice, P.stream));
    CK(cudaStreamSynchronize(P.stream));
  }
  (void)n1;
}

static size_t footprint_impl(const fsi_params& prm0, int n_nodes, int n_tris, const double* ref_xy,
                             const int* tris) {
  fsi_params prm = with_defaults(prm0);
  check_params(prm, n_nodes, n_tris);
  Problem P;
  P.prm = prm;
  P.ar.count_only = true;
  P.N = prm.N;
  VNum vn(prm.N);
  P.nU = vn.n; P.nP = prm.N * prm.N; P.nS = n_nodes; P.nTri = n_tris; P.nPts = elem_points(prm) * n_tris;
  P.offP = 2 * (size_t)P.nU; P.offX = P.offP + 3 * (size_t)P.nP; P.offL = P.offX + 2 * (size_t)P.nS;
  P.n = P.offL + 2 * (size_t)P.nS;
  P.m = prm.restart;
  SetupParams sp{prm.N, prm.rho_f, prm.nu, prm.kappa, prm.dt, prm.lid_u};
  sp.npe = elem_nodes(prm);
  sp.coarse_max = prm.mg_coarse;
  sp.coarse_max_p = prm.mg_coarse_p;
  build_setup(sp, n_nodes, n_tris, ref_xy, tris, P.hs);
  allocate_problem(P, ref_xy, tris);
  return P.ar.bytes;
}

extern "C" {

size_t fsi_footprint_bytes(const fsi_params* params, int n_solid_nodes, int n_tris) {
  if (!params || n_solid_nodes < 3 || n_tris < 1) return 0;
  try {
    // a synthetic solid with the same counts: matrix sizes depend on counts only
    // up to the solid adjacency, which is bounded by a small ring patch
    std::vector<double> xy(2 * (size_t)n_solid_nodes);
    std::vector<int> tr(3 * (size_t)n_tris);
    for (int i = 0; i < n_solid_nodes; ++i) { xy[2 * i] = 0.5 + 1e-3 * (i % 7); xy[2 * i + 1] = 0.5 + 1e-3 * (i / 7 % 7); }
    for (int t = 0; t < n_tris; ++t) { tr[3 * t] = 0; tr[3 * t + 1] = 1 + t % (n_solid_nodes - 2); tr[3 * t + 2] = 2 + t % (n_solid_nodes - 2); }
    // solid matrices only need a valid orientation; use a fan of unit triangles
    for (int i = 0; i < n_solid_nodes; ++i) {
      const double a = 6.283185307179586 * i / n_solid_nodes;
      xy[2 * i] = 0.5 + 0.1 * std::cos(a);
      xy[2 * i + 1] = 0.5 + 0.1 * std::sin(a);
    }
    xy[0] = 0.5; xy[1] = 0.5;
    if (params->solid_elem == 1) {
      if (n_solid_nodes < 4) return 0;  // a quadrilateral needs 4 nodes
      tr.assign(4 * (size_t)n_tris, 0);
      if (n_solid_nodes < 8) {
        // a ladder of m quadrilaterals-wide strip: nodes j (bottom) and m + j (top)
        const int m = n_solid_nodes / 2;
        for (int j = 0; j < m; ++j) {
          xy[2 * j] = xy[2 * (m + j)] = 0.3 + 0.4 * j / (m - 1);
          xy[2 * j + 1] = 0.45;
          xy[2 * (m + j) + 1] = 0.55;
        }
        for (int t = 0; t < n_tris; ++t) {
          const int j = t % (m - 1);
          tr[4 * t] = j; tr[4 * t + 1] = j + 1; tr[4 * t + 2] = m + j + 1; tr[4 * t + 3] = m + j;
        }
        return footprint_impl(*params, n_solid_nodes, n_tris, xy.data(), tr.data());
      }
      // quadrilaterals (centre, three consecutive ring nodes): convex and
      // counter-clockwise while three ring steps span less than half a turn
      for (int t = 0; t < n_tris; ++t) {
        const int a = 1 + t % (n_solid_nodes - 1);
        const int b = 1 + (a % (n_solid_nodes - 1));
        const int c = 1 + (b % (n_solid_nodes - 1));
        tr[4 * t] = 0; tr[4 * t + 1] = a; tr[4 * t + 2] = b; tr[4 * t + 3] = c;
      }
      return footprint_impl(*params, n_solid_nodes, n_tris, xy.data(), tr.data());
    }
    if (n_solid_nodes < 5) {
      // too few ring nodes for a fan (its closing triangle would span half a
      // turn): one triangle, or a strip of two-triangle cells (nodes j bottom,
      // m + j top), counter-clockwise
      const int m = n_solid_nodes / 2;
      if (n_solid_nodes == 3) {
        const double p3[6] = {0.45, 0.45, 0.55, 0.45, 0.5, 0.55};
        for (int i = 0; i < 6; ++i) xy[i] = p3[i];
      } else {
        for (int j = 0; j < m; ++j) {
          xy[2 * j] = xy[2 * (m + j)] = 0.3 + 0.4 * j / (m - 1);
          xy[2 * j + 1] = 0.45;
          xy[2 * (m + j) + 1] = 0.55;
        }
      }
      for (int t = 0; t < n_tris; ++t) {
        if (n_solid_nodes == 3) { tr[3 * t] = 0; tr[3 * t + 1] = 1; tr[3 * t + 2] = 2; continue; }
        const int c = t % (2 * (m - 1)), j = c / 2;
        if (c % 2 == 0) { tr[3 * t] = j; tr[3 * t + 1] = j + 1; tr[3 * t + 2] = m + j + 1; }
        else { tr[3 * t] = j; tr[3 * t + 1] = m + j + 1; tr[3 * t + 2] = m + j; }
      }
      return footprint_impl(*params, n_solid_nodes, n_tris, xy.data(), tr.data());
    }
    for (int t = 0; t < n_tris; ++t) {
      const int a = 1 + t % (n_solid_nodes - 1);
      const int b = 1 + (a % (n_solid_nodes - 1));
      tr[3 * t] = 0; tr[3 * t + 1] = a; tr[3 * t + 2] = b;
    }
    return footprint_impl(*params, n_solid_nodes, n_tris, xy.data(), tr.data());
  } catch (...) {
    return 0;
  }
}

int fsi_create_problem_budget(const fsi_params* params, const fsi_solid_mesh* mesh, const double* u0,
                              const double* X0, void* cuda_stream, size_t budget_bytes, fsi_problem** out) {
  if (!params || !mesh || !out || !mesh->ref_xy || !mesh->tris) return FSI_ERR_INVALID;
  *out = nullptr;
  fsi_problem* h = nullptr;
  try {
    fsi_params prm = with_defaults(*params);
    check_params(prm, mesh->n_nodes, mesh->n_tris);
    for (size_t i = 0; i < (size_t)elem_nodes(prm) * mesh->n_tris; ++i)
      if (mesh->tris[i] < 0 || mesh->tris[i] >= mesh->n_nodes) return FSI_ERR_INVALID;
    if (budget_bytes > 0) {
      const size_t need = footprint_impl(prm, mesh->n_nodes, mesh->n_tris, mesh->ref_xy, mesh->tris);
      if (need > budget_bytes) return FSI_ERR_BUDGET;
    }
    h = new fsi_problem();
    Problem& P = h->P;
    P.prm = prm;
    CK(cudaGetDevice(&P.device));
    if (cuda_stream) {
      P.stream = (cudaStream_t)cuda_stream;
    } else {
      CK(cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking));
      P.own_stream = true;
    }
    CK(cudaStreamCreateWithFlags(&P.s2, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&P.s3, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&P.s4, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&P.s5, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&P.ev_join2, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&P.ev_fork2, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&P.ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&P.ev_join, cudaEventDisableTiming));
    P.N = prm.N;
    VNum vn(prm.N);
    P.nU = vn.n; P.nP = prm.N * prm.N; P.nS = mesh->n_nodes; P.nTri = mesh->n_tris; P.nPts = elem_points(prm) * mesh->n_tris;
    P.offP = 2 * (size_t)P.nU; P.offX = P.offP + 3 * (size_t)P.nP; P.offL = P.offX + 2 * (size_t)P.nS;
    P.n = P.offL + 2 * (size_t)P.nS;
    P.m = prm.restart;
    SetupParams sp{prm.N, prm.rho_f, prm.nu, prm.kappa, prm.dt, prm.lid_u};
    sp.npe = elem_nodes(prm);
    sp.coarse_max = prm.mg_coarse;
  sp.coarse_max_p = prm.mg_coarse_p;
    build_setup(sp, P.nS, P.nTri, mesh->ref_xy, mesh->tris, P.hs);
    {
      double lam[6][3], w[6];
      triangle_rule(lam, w);
      CK(cudaMemcpyToSymbol(c_rule_lam, lam, sizeof(lam)));
      CK(cudaMemcpyToSymbol(c_rule_w, w, sizeof(w)));
      // Radon's 7-point rule (exact to degree 5) from its closed form: the
      // centroid, weight 9/40; orbits (a, a, 1-2a), a = (6 -/+ sqrt 15)/21,
      // weights (155 -/+ sqrt 15)/1200
      double rl[7][3], rw[7];
      const double r15 = std::sqrt(15.0);
      rl[0][0] = rl[0][1] = rl[0][2] = 1.0 / 3.0;
      rw[0] = 9.0 / 40.0;
      const double oa[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
      const double ow[2] = {(155.0 - r15) / 1200.0, (155.0 + r15) / 1200.0};
      for (int o = 0; o < 2; ++o)
        for (int k = 0; k < 3; ++k) {
          for (int c = 0; c < 3; ++c) rl[1 + 3 * o + k][c] = (c == k) ? 1.0 - 2.0 * oa[o] : oa[o];
          rw[1 + 3 * o + k] = ow[o];
        }
      CK(cudaMemcpyToSymbol(c_radon_lam, rl, sizeof(rl)));
      CK(cudaMemcpyToSymbol(c_radon_w, rw, sizeof(rw)));
      // Q1: (s, t, s t) of the 3 x 3 Gauss points and the shape functions there
      double qs[9], qt[9], qst[9], qw[9], qp[9][3], qc[9][4];
      quad_rule(qs, qt, qst, qw);
      for (int q = 0; q < 9; ++q) {
        qp[q][0] = qs[q]; qp[q][1] = qt[q]; qp[q][2] = qst[q];
        q1_shape(qs[q], qt[q], qc[q]);
      }
      CK(cudaMemcpyToSymbol(c_q1_pt, qp, sizeof(qp)));
      CK(cudaMemcpyToSymbol(c_q1_chi, qc, sizeof(qc)));
    }
    allocate_problem(P, mesh->ref_xy, mesh->tris);
    CK(cudaMemset(P.ctl, 0, sizeof(Ctl)));
    CK(cudaMemset(P.cf_len, 0, sizeof(int) * P.nS));
    CK(cudaMemset(P.cft_ptr, 0, sizeof(int) * (P.nU + 1)));
    CK(cudaMemset(P.cflift, 0, sizeof(double) * 2 * P.nS));
    CK(cudaMemset(P.x, 0, P.n * 8));
    CK(cudaMemset(P.b, 0, P.n * 8));
    CK(cudaMemcpy(P.b + P.offP, P.hs.lift_p.data(), P.hs.lift_p.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMallocHost((void**)&P.ctl_host, sizeof(Ctl)));
    std::vector<double> u(2 * (size_t)(2 * P.N + 1) * (2 * P.N + 1));
    if (u0) std::copy(u0, u0 + u.size(), u.begin());
    upload_state(P, u.data(), X0 ? X0 : mesh->ref_xy);
    build_graphs(P);
    CK(cudaDeviceSynchronize());
    *out = h;
    return FSI_OK;
  } catch (...) {
    const int code = map_exception();
    if (h) fsi_destroy(h);
    return code;
  }
}

int fsi_create_problem(const fsi_params* params, const fsi_solid_mesh* mesh, const double* u0, const double* X0,
                       void* cuda_stream, fsi_problem** out) {
  return fsi_create_problem_budget(params, mesh, u0, X0, cuda_stream, 0, out);
}

int fsi_assemble_step(fsi_problem* h) {
  if (!h) return FSI_ERR_INVALID;
  try {
    CK(cudaGraphLaunch(h->P.g_assemble, h->P.stream));
    h->P.assembled = true;
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

static int status_from_ctl(const Ctl& c) {
  if (c.aflags & FLAG_OUT_OF_DOMAIN) return FSI_ERR_OUT_OF_DOMAIN;
  if (c.aflags & FLAG_CAPACITY) return FSI_ERR_CAPACITY;
  if (c.flags & FLAG_NAN) return FSI_ERR_NAN;
  if (c.flags & FLAG_BREAKDOWN) return FSI_ERR_BREAKDOWN;
  if (!c.converged) return FSI_ERR_NOT_CONVERGED;
  return FSI_OK;
}

static int fill_info(const Problem& P, fsi_solve_info* info) {
  const Ctl& c = *P.ctl_host;
  const int st = status_from_ctl(c);
  if (info) {
    info->iterations = c.its;
    info->restarts = std::max(0, c.cycles - 2);
    info->refinements = (P.prm.precision == 1) ? std::max(0, c.cycles - 1) : 0;
    info->status = st;
    info->rel_residual = c.last_true;
    info->rel_residual_est = (c.bnorm > 0) ? c.res / c.bnorm : c.res;
  }
  return st;
}

// queue S5-S8 (and the pressure normalisation) without waiting
static void enqueue_solve(Problem& P) {
  if (!P.assembled) CK(cudaGraphLaunch(P.g_assemble, P.stream));
  P.assembled = false;
  CK(cudaGraphLaunch(P.g_begin, P.stream));
  CK(cudaGraphLaunch(P.g_cycle, P.stream));
  CK(cudaGraphLaunch(P.g_finish, P.stream));
  CK(cudaMemcpyAsync(P.ctl_host, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P.stream));
}

static void enqueue_advance(Problem& P) {
  CK(cudaMemcpyAsync(P.uold, P.x, 2 * (size_t)P.nU * 8, cudaMemcpyDeviceToDevice, P.stream));
  CK(cudaMemcpyAsync(P.Xold, P.x + P.offX, 2 * (size_t)P.nS * 8, cudaMemcpyDeviceToDevice, P.stream));
}

// One linear solve of the assembled block system (S5-S8) from the current
// iterate P.x.
static int solve_linear(Problem& P, fsi_solve_info* info) {
  {
    if (!P.host_loop) {
      enqueue_solve(P);
      CK(cudaStreamSynchronize(P.stream));
      return fill_info(P, info);
    }
    if (!P.assembled) CK(cudaGraphLaunch(P.g_assemble, P.stream));
    P.assembled = false;
    CK(cudaGraphLaunch(P.g_begin, P.stream));
    const int max_cycles = (P.prm.precision == 1) ? P.prm.max_refine + 1 : 1000000;
    Ctl& c = *P.ctl_host;
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
      CK(cudaGraphLaunch(P.g_cstart, P.stream));
      CK(cudaMemcpyAsync(P.ctl_host, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P.stream));
      CK(cudaStreamSynchronize(P.stream));
      while (c.cyc_active) {
        CK(cudaGraphLaunch(P.g_body, P.stream));
        CK(cudaMemcpyAsync(P.ctl_host, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P.stream));
        CK(cudaStreamSynchronize(P.stream));
      }
      CK(cudaGraphLaunch(P.g_cend, P.stream));
      CK(cudaMemcpyAsync(P.ctl_host, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P.stream));
      CK(cudaStreamSynchronize(P.stream));
      if (c.stop || c.aflags) break;
    }
    CK(cudaGraphLaunch(P.g_finish, P.stream));
    CK(cudaMemcpyAsync(P.ctl_host, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    return fill_info(P, info);
  }
}

// Newton's method for the nonlinear solid law (Section 4: a nonlinear P(F)
// is handled by a Newton iteration): from X_0 = X^n, each iteration puts the
// tangent K_T(X_k) in place of A_s and K_T X_k - S(X_k) in the solid rows of
// the right-hand side, and solves the block system from the current iterate.
// Stops when max |X_{k+1} - X_k| <= newton_tol * max |X_{k+1} - X^n| (floor
// 1e-13).
static int solve_newton(Problem& P, fsi_solve_info* info) {
  const size_t n2 = 2 * (size_t)P.nS;
  std::vector<double> xk(n2), xn(n2), xo(n2);
  CK(cudaMemcpyAsync(P.x + P.offX, P.Xold, n2 * 8, cudaMemcpyDeviceToDevice, P.stream));
  CK(cudaMemcpyAsync(xo.data(), P.Xold, n2 * 8, cudaMemcpyDeviceToHost, P.stream));
  CK(cudaStreamSynchronize(P.stream));
  xk = xo;
  int total_its = 0, st = FSI_OK;
  fsi_solve_info last{};
  for (int it = 0; it < P.prm.newton_max; ++it) {
    launch(k_solid_tangent, nblk(P.nS, 128), 128, 0, P.stream, P.nS, P.ntp, P.nt, P.tris, P.area, P.tgrad,
           (const double*)(P.x + P.offX), P.prm.gamma, P.prm.eta, P.op64.Ssol.soff, P.op64.Ssol.len,
           P.op64.Ssol.col, P.kt64, P.kt32, P.b + P.offX, &P.ctl->aflags);
    st = solve_linear(P, &last);
    total_its += last.iterations;
    if (st != FSI_OK) break;
    CK(cudaMemcpyAsync(xn.data(), P.x + P.offX, n2 * 8, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    double dx = 0.0, disp = 0.0;
    for (size_t i = 0; i < n2; ++i) {
      dx = std::max(dx, std::fabs(xn[i] - xk[i]));
      disp = std::max(disp, std::fabs(xn[i] - xo[i]));
    }
    xk.swap(xn);
    last.newton_iterations = it + 1;
    if (dx <= std::max(P.prm.newton_tol * disp, 1e-13)) break;
    if (it + 1 == P.prm.newton_max) st = FSI_ERR_NOT_CONVERGED;
    P.assembled = true;  // C_f(X^n) and the linear right-hand side stay as assembled
  }
  P.assembled = false;
  last.iterations = total_its;
  last.status = st;
  if (info) *info = last;
  return st;
}

int fsi_solve_step(fsi_problem* h, fsi_solve_info* info) {
  if (!h) return FSI_ERR_INVALID;
  Problem& P = h->P;
  try {
    if (info) info->newton_iterations = 0;
    if (P.prm.solid_law == 1) return solve_newton(P, info);
    return solve_linear(P, info);
  } catch (...) {
    return map_exception();
  }
}

int fsi_step_async(fsi_problem* h) {
  if (!h || h->P.host_loop || h->P.prm.solid_law != 0) return FSI_ERR_INVALID;
  Problem& P = h->P;
  try {
    P.assembled = false;
    enqueue_solve(P);
    enqueue_advance(P);
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_step_poll(fsi_problem* h, fsi_solve_info* info) {
  if (!h) return FSI_ERR_INVALID;
  Problem& P = h->P;
  const cudaError_t q = cudaStreamQuery(P.stream);
  if (q == cudaErrorNotReady) return 1;
  if (q != cudaSuccess) return FSI_ERR_CUDA;
  fill_info(P, info);
  return 0;
}

int fsi_step_batch(fsi_problem* const* problems, int count, fsi_solve_info* infos) {
  if (!problems || count < 0) return FSI_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (!problems[i] || problems[i]->P.host_loop || problems[i]->P.prm.solid_law != 0) return FSI_ERR_INVALID;
  int first_err = FSI_OK;
  try {
    // queue every instance's whole step on its own stream, then wait for all
    for (int i = 0; i < count; ++i) {
      Problem& P = problems[i]->P;
      P.assembled = false;
      enqueue_solve(P);
      enqueue_advance(P);
    }
    for (int i = 0; i < count; ++i) {
      Problem& P = problems[i]->P;
      CK(cudaStreamSynchronize(P.stream));
      const int st = fill_info(P, infos ? &infos[i] : nullptr);
      if (st != FSI_OK && first_err == FSI_OK) first_err = st;
    }
    return first_err;
  } catch (...) {
    return map_exception();
  }
}

int fsi_advance(fsi_problem* h) {
  if (!h) return FSI_ERR_INVALID;
  Problem& P = h->P;
  try {
    CK(cudaMemcpyAsync(P.uold, P.x, 2 * (size_t)P.nU * 8, cudaMemcpyDeviceToDevice, P.stream));
    CK(cudaMemcpyAsync(P.Xold, P.x + P.offX, 2 * (size_t)P.nS * 8, cudaMemcpyDeviceToDevice, P.stream));
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_step(fsi_problem* h, fsi_solve_info* info) {
  int st = fsi_assemble_step(h);
  if (st != FSI_OK) return st;
  st = fsi_solve_step(h, info);
  if (st != FSI_OK) return st;
  return fsi_advance(h);
}

int fsi_get_state(fsi_problem* h, double* u, double* pr, double* X, double* lam) {
  if (!h) return FSI_ERR_INVALID;
  Problem& P = h->P;
  try {
    std::vector<double> x(P.n);
    CK(cudaMemcpyAsync(x.data(), P.x, P.n * 8, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    if (u) {
      const size_t nl = (size_t)(2 * P.N + 1) * (2 * P.N + 1);
      std::copy(P.hs.wall_u.begin(), P.hs.wall_u.begin() + 2 * nl, u);
      for (int k = 0; k < P.nU; ++k) {
        const int lat = P.hs.interior_lattice[k];
        u[2 * (size_t)lat] = x[2 * (size_t)k];
        u[2 * (size_t)lat + 1] = x[2 * (size_t)k + 1];
      }
    }
    if (pr) std::copy(x.begin() + P.offP, x.begin() + P.offX, pr);
    if (X) std::copy(x.begin() + P.offX, x.begin() + P.offL, X);
    if (lam) std::copy(x.begin() + P.offL, x.end(), lam);
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_set_state(fsi_problem* h, const double* u, const double* X) {
  if (!h) return FSI_ERR_INVALID;
  try {
    upload_state(h->P, u, X);
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_sizes(const fsi_problem* h, int* n_u, int* n_p, int* n_x, int* n_total) {
  if (!h) return FSI_ERR_INVALID;
  const Problem& P = h->P;
  if (n_u) *n_u = 2 * P.nU;
  if (n_p) *n_p = 3 * P.nP;
  if (n_x) *n_x = 2 * P.nS;
  if (n_total) *n_total = (int)P.n;
  return FSI_OK;
}

int fsi_get_points(fsi_problem* h, int* cell, double* xi, double* eta) {
  if (!h) return FSI_ERR_INVALID;
  Problem& P = h->P;
  if (P.prm.coupling != 0) return FSI_ERR_INVALID;  // the exact rule locates no points
  try {
    if (cell) CK(cudaMemcpyAsync(cell, P.cell, (size_t)P.nPts * 4, cudaMemcpyDeviceToHost, P.stream));
    if (xi) CK(cudaMemcpyAsync(xi, P.xi, (size_t)P.nPts * 8, cudaMemcpyDeviceToHost, P.stream));
    if (eta) CK(cudaMemcpyAsync(eta, P.eta, (size_t)P.nPts * 8, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_get_coupling(fsi_problem* h, int* nnz, int* rows, int* lattice_cols, double* vals) {
  if (!h || !nnz) return FSI_ERR_INVALID;
  Problem& P = h->P;
  try {
    const size_t nslot = (size_t)nblk(P.nS, 32) * 32 * P.cf_cap;
    std::vector<int> len(P.nS), col(nslot);
    std::vector<double> val(nslot);
    CK(cudaMemcpyAsync(len.data(), P.cf_len, (size_t)P.nS * 4, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaMemcpyAsync(col.data(), P.cf_col, nslot * 4, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaMemcpyAsync(val.data(), P.cf_val, nslot * 8, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    int total = 0;
    for (int l = 0; l < P.nS; ++l) total += len[l];
    if (!rows) { *nnz = total; return FSI_OK; }
    if (*nnz < total) return FSI_ERR_INVALID;
    int q = 0;
    for (int l = 0; l < P.nS; ++l)
      for (int k = 0; k < len[l]; ++k) {
        const size_t slot = (size_t)(l >> 5) * 32 * P.cf_cap + (size_t)k * 32 + (l & 31);
        rows[q] = l;
        if (lattice_cols) lattice_cols[q] = P.hs.interior_lattice[col[slot]];
        if (vals) vals[q] = val[slot];
        ++q;
      }
    *nnz = total;
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_apply_operator(fsi_problem* h, const double* xh, double* yh, int precision) {
  if (!h || !xh || !yh) return FSI_ERR_INVALID;
  Problem& P = h->P;
  if (precision == 1 && P.prm.precision != 1) return FSI_ERR_INVALID;
  try {
    double* tmp = P.V;  // first basis vector as scratch
    CK(cudaMemcpyAsync(tmp, xh, P.n * 8, cudaMemcpyHostToDevice, P.stream));
    if (precision == 1) {
      launch(k_convert<double, float>, nblk(P.n, 256), 256, 0, P.stream, P.n, tmp, P.p32.vin);
      launch(k_fullmv<float, float, double>, P.op32.gU + P.op32.gP + P.op32.gS, 128, 0, P.stream, P.op32, P.p32.vin, P.w,
                                                                                            nullptr, 1.0, 0.0);
    } else {
      launch(k_fullmv<double, double, double>, P.op64.gU + P.op64.gP + P.op64.gS, 128, 0, P.stream, P.op64, tmp, P.w,
                                                                                               nullptr, 1.0, 0.0);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(yh, P.w, P.n * 8, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_apply_preconditioner(fsi_problem* h, const double* vh, double* zh, int precision) {
  if (!h || !vh || !zh) return FSI_ERR_INVALID;
  Problem& P = h->P;
  if (precision == 1 && P.prm.precision != 1) return FSI_ERR_INVALID;
  try {
    double* tmp = P.V;
    CK(cudaMemcpyAsync(tmp, vh, P.n * 8, cudaMemcpyHostToDevice, P.stream));
    if (precision == 1) {
      launch(k_convert<double, float>, nblk(P.n, 256), 256, 0, P.stream, P.n, tmp, P.p32.vin);
      precond_launch(P, P.p32, P.stream);
      launch(k_convert<float, double>, nblk(P.n, 256), 256, 0, P.stream, P.n, P.p32.zw, P.w);
    } else {
      launch(k_copy<double>, nblk(P.n, 256), 256, 0, P.stream, P.n, tmp, P.p64.vin);
      precond_launch(P, P.p64, P.stream);
      launch(k_copy<double>, nblk(P.n, 256), 256, 0, P.stream, P.n, P.p64.zw, P.w);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(zh, P.w, P.n * 8, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_graph_kernel_counts(const fsi_problem* h, int* counts) {
  if (!h || !counts) return FSI_ERR_INVALID;
  const Problem& P = h->P;
  counts[0] = P.kn_assemble; counts[1] = P.kn_begin; counts[2] = P.kn_cycle;
  counts[3] = P.kn_body; counts[4] = P.kn_finish;
  return FSI_OK;
}

int fsi_time_kernel(fsi_problem* h, int which, int reps, double* avg_ms, double* bytes) {
  if (!h || !avg_ms || !bytes || reps <= 0) return FSI_ERR_INVALID;
  Problem& P = h->P;
  if ((which == 0 || which == 2 || (which >= 4 && which <= 7) || (which >= 10 && which <= 13)) &&
      P.prm.precision != 1)
    return FSI_ERR_INVALID;
  if (which == 8 && P.prm.coupling != 0) return FSI_ERR_INVALID;  // would overwrite the exact rows
  if (which == 9 && P.prm.coupling != 1) return FSI_ERR_INVALID;
  if (which == 3 && P.p64.mgU.lv.empty()) return FSI_ERR_INVALID;  // no FP64 hierarchy in mixed mode
  try {
    // total C_f entries of the last assembly
    std::vector<int> len(P.nS);
    CK(cudaMemcpy(len.data(), P.cf_len, (size_t)P.nS * 4, cudaMemcpyDeviceToHost));
    double cfnnz = 0;
    for (int v : len) cfnnz += v;
    const size_t flush_n = (size_t)(256u << 20) / sizeof(uint4);
    uint4* fl = nullptr;
    CK(cudaMalloc(&fl, flush_n * sizeof(uint4)));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double total = 0;
    cudaStream_t s = P.stream;
    const HostBlockMatrix& A0 = P.hs.levels[0].A;
    for (int r = 0; r < reps + 1; ++r) {
      if (which < 4 || which >= 10) launch(k_flush, 2 * 152, 512, 0, s, flush_n, fl, (unsigned)r);
      CK(cudaEventRecord(e0, s));
      switch (which) {
        case 0:  // full operator, FP32 (mixed inner iteration)
          launch(k_fullmv<float, float, double>, P.op32.gU + P.op32.gP + P.op32.gS, 128, 0, s, P.op32, P.p32.zw, P.w,
                                                                                          nullptr, 1.0, 0.0);
          *bytes = fullop_bytes<float>(P, cfnnz, sizeof(float), sizeof(double));
          break;
        case 1:  // full operator, FP64 (residual / FP64 iteration)
          launch(k_fullmv<double, double, double>, P.op64.gU + P.op64.gP + P.op64.gS, 128, 0, s, P.op64, P.x, P.w, P.b,
                                                                                            -1.0, 1.0);
          *bytes = fullop_bytes<double>(P, cfnnz, 16, 8);
          break;
        case 2: {  // finest velocity Chebyshev step, FP32
          MGLevel<float>& L = P.p32.mgU.lv[0];
          SpmvArgs<float> a;
          a.x = L.x; a.y = L.x2; a.z = L.b; a.d = L.d; a.dinv = L.dinv; a.c1 = 0.5f; a.c2 = 0.5f;
          sell_launch(L.A, MODE_CHEB, a, s);
          *bytes = sell_bytes<float>(A0) + 6.0 * L.n * sizeof(float);
          break;
        }
        case 3: {  // finest velocity Chebyshev step, FP64
          MGLevel<double>& L = P.p64.mgU.lv[0];
          SpmvArgs<double> a;
          a.x = L.x; a.y = L.x2; a.z = L.b; a.d = L.d; a.dinv = L.dinv; a.c1 = 0.5; a.c2 = 0.5;
          sell_launch(L.A, MODE_CHEB, a, s);
          *bytes = sell_bytes<double>(A0) + 6.0 * L.n * sizeof(double);
          break;
        }
        case 4:    // one V-cycle on the Q2 velocity hierarchy, FP32
        case 5: {  // one V-cycle on the pressure Laplacian hierarchy, FP32
          MG<float>& mg = (which == 4) ? P.p32.mgU : P.p32.mgP;
          vcycle<float>(mg, 0, s, mg.lv[0].mf ? mg.lv[0].x : mg.lv[0].x2);
          *bytes = vcycle_work<float>(P.hs, mg, which == 5).bytes;
          break;
        }
        case 8:    // C_f rows by the point rule at located points (S2 + S4)
          point_rule_launch(P, s);
          *bytes = 0;
          break;
        case 9:    // C_f rows by the exact rule (mesh intersection)
          launch(k_cf_rows_exact, nblk(P.nS, kCfWarps), 32 * kCfWarps, 0, s, P.nS, P.N, P.ntp, P.nt, P.tris, P.Xold,
                 P.area, P.l2n, P.wall, P.cf_cap, P.cf_len, P.cf_col, P.cf_val, P.cf_val32, P.cflift, &P.ctl->aflags);
          *bytes = 0;
          break;
        case 10:   // fused finest-level launches, FP32: velocity down / up,
        case 11:   // pressure down / up (the level's current vectors)
        case 12:
        case 13: {
          MG<float>& mg = (which <= 11) ? P.p32.mgU : P.p32.mgP;
          MGLevel<float>& L = mg.lv[0];
          if (!L.mf) {
            cudaFree(fl);
            return FSI_ERR_INVALID;
          }
          MGLevel<float>& C = mg.lv[1];
          const bool up = (which & 1) != 0;
          if (up) mf_up_launch<float>(mg, 0, L.b, C.x, L.x, nullptr, s);
          else mf_down_launch<float>(mg, 0, L.b, s);
          *bytes = mf_work(P.hs, 0, which >= 12, up, mg.degree, sizeof(float)).bytes;
          break;
        }
        case 6:    // the cluster launch of the velocity coarse levels alone, FP32
        case 7: {  // the same for the pressure Laplacian
          MG<float>& mg = (which == 6) ? P.p32.mgU : P.p32.mgP;
          if (!mg.cl.on) {
            cudaFree(fl);
            return FSI_ERR_INVALID;
          }
          MGLevel<float>& L = mg.lv[mg.cl.lc];
          cluster_launch<float>(mg, L.b, L.x, s);
          *bytes = 0;
          break;
        }
        default:
          cudaFree(fl);
          return FSI_ERR_INVALID;
      }
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0) total += ms;  // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(fl);
    *avg_ms = total / reps;
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

int fsi_kernel_flops(fsi_problem* h, int which, double* flops) {
  if (!h || !flops) return FSI_ERR_INVALID;
  Problem& P = h->P;
  if (P.prm.precision != 1) return FSI_ERR_INVALID;
  if (which == 4 || which == 5) {
    *flops = vcycle_work<float>(P.hs, which == 4 ? P.p32.mgU : P.p32.mgP, which == 5).flops;
    return FSI_OK;
  }
  if (which < 10 || which > 13) return FSI_ERR_INVALID;
  const MG<float>& mg = (which <= 11) ? P.p32.mgU : P.p32.mgP;
  if (mg.lv.empty() || !mg.lv[0].mf) return FSI_ERR_INVALID;
  *flops = mf_work(P.hs, 0, which >= 12, (which & 1) != 0, mg.degree, sizeof(float)).flops;
  return FSI_OK;
}

int fsi_interior_nodes(const fsi_problem* h, int* lattice_ids) {
  if (!h || !lattice_ids) return FSI_ERR_INVALID;
  std::copy(h->P.hs.interior_lattice.begin(), h->P.hs.interior_lattice.end(), lattice_ids);
  return FSI_OK;
}

int fsi_get_rhs(fsi_problem* h, double* bh) {
  if (!h || !bh) return FSI_ERR_INVALID;
  Problem& P = h->P;
  try {
    CK(cudaMemcpyAsync(bh, P.b, P.n * 8, cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    return FSI_OK;
  } catch (...) {
    return map_exception();
  }
}

void fsi_destroy(fsi_problem* h) {
  if (!h) return;
  Problem& P = h->P;
  cudaGraphExec_t ex[7] = {P.g_assemble, P.g_begin, P.g_cycle, P.g_finish, P.g_cstart, P.g_body, P.g_cend};
  cudaGraph_t gr[7] = {P.gr_assemble, P.gr_begin, P.gr_cycle, P.gr_finish, P.gr_cstart, P.gr_body, P.gr_cend};
  if (P.stream) cudaStreamSynchronize(P.stream);
  for (auto e : ex) if (e) cudaGraphExecDestroy(e);
  for (auto g : gr) if (g) cudaGraphDestroy(g);
  P.ar.release();
  if (P.ctl_host) cudaFreeHost(P.ctl_host);
  if (P.s2) cudaStreamDestroy(P.s2);
  if (P.s3) cudaStreamDestroy(P.s3);
  if (P.s4) cudaStreamDestroy(P.s4);
  if (P.s5) cudaStreamDestroy(P.s5);
  if (P.ev_join2) cudaEventDestroy(P.ev_join2);
  if (P.ev_fork2) cudaEventDestroy(P.ev_fork2);
  if (P.ev_fork) cudaEventDestroy(P.ev_fork);
  if (P.ev_join) cudaEventDestroy(P.ev_join);
  if (P.own_stream && P.stream) cudaStreamDestroy(P.stream);
  delete h;
}

const char* fsi_status_str(int s) {
  switch (s) {
    case FSI_OK: return "ok";
    case FSI_ERR_INVALID: return "invalid argument";
    case FSI_ERR_OOM: return "device out of memory";
    case FSI_ERR_BUDGET: return "footprint above budget";
    case FSI_ERR_OUT_OF_DOMAIN: return "solid point outside the fluid domain";
    case FSI_ERR_NOT_CONVERGED: return "not converged";
    case FSI_ERR_BREAKDOWN: return "Krylov breakdown";
    case FSI_ERR_NAN: return "NaN or Inf in the residual";
    case FSI_ERR_TIMEOUT: return "bounded device wait ran out";
    case FSI_ERR_CAPACITY: return "coupling row over capacity";
    case FSI_ERR_CUDA: return "CUDA error";
    default: return "unknown status";
  }
}

}  // extern "C"
