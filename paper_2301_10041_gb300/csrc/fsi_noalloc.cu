// Point location and binning of the solid quadrature points by fluid cell,
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need this work done:
// code that runs while a CUDA stream is being captured into a graph,
// real-time or embedded hosts that forbid allocation after start-up, or plugins
// that live inside another framework's memory pool.  This entry point gives
// them the location of every point (cell, local coordinates) and the
// cell -> points lists with no allocation at all: the caller passes every
// input and output buffer, and the only scratch is a fixed array compiled
// into the library (see FSI_NOALLOC_MAX_CELLS in include/fsi.h).
//
// The scratch array lives in device memory of every GPU that loads the
// library, for as long as the process runs.  All calls share it and it keeps
// what the previous call left, so each call first clears the counters it
// needs.  Two calls that overlap on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/fsi.h"
#include "fsi_internal.h"

namespace {

constexpr int kNaBlock = 1024;
constexpr int kNaMaxBlocks = (FSI_NOALLOC_MAX_CELLS + kNaBlock - 1) / kNaBlock;

struct NoAllocScratch {
  int count[FSI_NOALLOC_MAX_CELLS];   // points per cell
  int cursor[FSI_NOALLOC_MAX_CELLS];  // fill position per cell
  int bsum[kNaMaxBlocks + 1];         // block sums of the scan
  int outside;                        // points outside [0,1]^2
};

static __device__ __align__(256) NoAllocScratch g_scratch;

__constant__ double c_na_lam[6][3];

// Set-up once per device (first call on that device, with that device
// current): the device address of the scratch array and the quadrature table
// in constant memory.  Host threads that make their first calls at the same
// time take turns on the mutex.
constexpr int kMaxDevices = 64;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mu;

bool setup_done(int dev) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  return g_scratch_ptr[dev] != nullptr;
}

int device_setup(int dev, NoAllocScratch** out) {
  if (dev < 0 || dev >= kMaxDevices) return FSI_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FSI_ERR_CUDA;
    double lam[6][3], w[6];
    fsi::triangle_rule(lam, w);
    if (cudaMemcpyToSymbol(c_na_lam, lam, sizeof(lam)) != cudaSuccess) return FSI_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return FSI_OK;
}

__global__ void k_na_clear(NoAllocScratch* s, int ncells) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncells) s->count[i] = 0;
  if (i == 0) s->outside = 0;
}

// same arithmetic as the library's point location: x = P0 + xi1 (P1 - P0) +
// xi2 (P2 - P0) in explicitly rounded FP64, half-open cells on t = x * N
__global__ void k_na_locate(int n_pts, int N, const int* __restrict__ tris, const double* __restrict__ X,
                            int* __restrict__ cell, double* __restrict__ xi, double* __restrict__ eta,
                            NoAllocScratch* s) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pts) return;
  const int t = p / 6, q = p - 6 * (p / 6);
  const int v0 = tris[3 * t], v1 = tris[3 * t + 1], v2 = tris[3 * t + 2];
  const double l1 = c_na_lam[q][1], l2 = c_na_lam[q][2];
  double loc[2];
  int idx[2];
  bool ok = true;
  for (int c = 0; c < 2; ++c) {
    const double P0 = X[2 * v0 + c], P1 = X[2 * v1 + c], P2 = X[2 * v2 + c];
    const double x = __dadd_rn(__dadd_rn(P0, __dmul_rn(l1, __dsub_rn(P1, P0))), __dmul_rn(l2, __dsub_rn(P2, P0)));
    if (!(x >= 0.0 && x <= 1.0)) { ok = false; idx[c] = 0; loc[c] = 0.0; continue; }
    const double tc = __dmul_rn(x, (double)N);
    int i = (int)floor(tc);
    if (i >= N) i = N - 1;
    idx[c] = i;
    loc[c] = __dsub_rn(tc, (double)i);
  }
  if (!ok) {
    cell[p] = -1; xi[p] = 0.0; eta[p] = 0.0;
    atomicAdd(&s->outside, 1);
    return;
  }
  const int c = idx[1] * N + idx[0];
  cell[p] = c;
  xi[p] = loc[0];
  eta[p] = loc[1];
  atomicAdd(&s->count[c], 1);
}

__device__ int na_block_excl_scan(int v, int* sm, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sm[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    sm[lane] = s;
  }
  __syncthreads();
  total = sm[(blockDim.x >> 5) - 1];
  const int r = ((w > 0) ? sm[w - 1] : 0) + inc - v;
  __syncthreads();
  return r;
}

__global__ void k_na_scan_blocks(int n, NoAllocScratch* s) {
  __shared__ int sm[32];
  const int i = blockIdx.x * kNaBlock + threadIdx.x;
  int total;
  na_block_excl_scan(i < n ? s->count[i] : 0, sm, total);
  if (threadIdx.x == 0) s->bsum[blockIdx.x] = total;
}

__global__ void k_na_scan_top(int nb, NoAllocScratch* s) {
  __shared__ int sm[32];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kNaBlock) {
    const int i = b0 + threadIdx.x;
    int total;
    const int e = na_block_excl_scan(i < nb ? s->bsum[i] : 0, sm, total);
    if (i < nb) s->bsum[i] = carry + e;
    carry += total;
  }
}

__global__ void k_na_scan_final(int n, NoAllocScratch* s, int* __restrict__ cell_start) {
  __shared__ int sm[32];
  const int i = blockIdx.x * kNaBlock + threadIdx.x;
  const int v = i < n ? s->count[i] : 0;
  int total;
  const int e = na_block_excl_scan(v, sm, total) + s->bsum[blockIdx.x];
  if (i < n) { cell_start[i] = e; s->cursor[i] = e; }
  if (i == n - 1) cell_start[n] = e + v;
}

__global__ void k_na_scatter(int n_pts, const int* __restrict__ cell, int* __restrict__ cell_points,
                             NoAllocScratch* s) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pts) return;
  const int c = cell[p];
  if (c < 0) return;
  cell_points[atomicAdd(&s->cursor[c], 1)] = p;
}

// the scatter order inside a cell is not fixed: sort each list by point id
// (insertion sort, one thread per cell: quadratic in the points of one cell,
// about 50 when the solid mesh size is half the fluid mesh size)
__global__ void k_na_sort(int ncells, const int* __restrict__ cell_start, int* __restrict__ cell_points) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int a = cell_start[c], b = cell_start[c + 1];
  for (int i = a + 1; i < b; ++i) {
    const int v = cell_points[i];
    int j = i - 1;
    while (j >= a && cell_points[j] > v) { cell_points[j + 1] = cell_points[j]; --j; }
    cell_points[j + 1] = v;
  }
}

__global__ void k_na_outside(const NoAllocScratch* s, int* out) { *out = s->outside; }

unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int run_locate_bin(int dev, int N, int n_tris, const int* tris, const double* X, int* cell, double* xi,
                   double* eta, int* cell_start, int* cell_points, int* n_outside, cudaStream_t stream);

}  // namespace

extern "C" int fsi_locate_bin_noalloc(int N, int n_tris, const int* tris, const double* X, int* cell, double* xi,
                                      double* eta, int* cell_start, int* cell_points, int* n_outside,
                                      void* cuda_stream) {
  if (N < 1 || n_tris < 1 || !tris || !X || !cell || !xi || !eta || !cell_start || !cell_points || !n_outside)
    return FSI_ERR_INVALID;
  const long long ncells = (long long)N * N;
  if (ncells > FSI_NOALLOC_MAX_CELLS) return FSI_ERR_INVALID;  // N*N above the compiled-in scratch
  if (6LL * n_tris > 0x7fffffffLL) return FSI_ERR_INVALID;
  // an error left pending by an earlier, unrelated call stays for its owner
  // to read: this call neither clears it nor claims it as its own
  if (cudaPeekAtLastError() != cudaSuccess) return FSI_ERR_CUDA;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  int cur = 0, dev = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return FSI_ERR_CUDA;
  dev = cur;
  if (stream && cudaStreamGetDevice(stream, &dev) != cudaSuccess) return FSI_ERR_INVALID;
  if (dev < 0 || dev >= kMaxDevices) return FSI_ERR_INVALID;
  if (!setup_done(dev)) {
    // the set-up copies synchronously, which would invalidate a capture in
    // progress: refuse instead, leaving the capture untouched
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return FSI_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return FSI_ERR_INVALID;
  }
  if (dev != cur && cudaSetDevice(dev) != cudaSuccess) return FSI_ERR_CUDA;
  const int rc = run_locate_bin(dev, N, n_tris, tris, X, cell, xi, eta, cell_start, cell_points, n_outside, stream);
  if (dev != cur && cudaSetDevice(cur) != cudaSuccess) return FSI_ERR_CUDA;
  return rc;
}

namespace {

// the work of one call on device `dev` (current)
int run_locate_bin(int dev, int N, int n_tris, const int* tris, const double* X, int* cell, double* xi,
                   double* eta, int* cell_start, int* cell_points, int* n_outside, cudaStream_t stream) {
  const long long ncells = (long long)N * N;
  NoAllocScratch* s = nullptr;
  const int st = device_setup(dev, &s);
  if (st != FSI_OK) return st;
  const int n_pts = 6 * n_tris;
  const int nc = (int)ncells;
  const unsigned nblocks = nb(nc, kNaBlock);
  k_na_clear<<<nb(nc, 256), 256, 0, stream>>>(s, nc);
  k_na_locate<<<nb(n_pts, 256), 256, 0, stream>>>(n_pts, N, tris, X, cell, xi, eta, s);
  k_na_scan_blocks<<<nblocks, kNaBlock, 0, stream>>>(nc, s);
  k_na_scan_top<<<1, kNaBlock, 0, stream>>>((int)nblocks, s);
  k_na_scan_final<<<nblocks, kNaBlock, 0, stream>>>(nc, s, cell_start);
  k_na_scatter<<<nb(n_pts, 256), 256, 0, stream>>>(n_pts, cell, cell_points, s);
  k_na_sort<<<nb(nc, 128), 128, 0, stream>>>(nc, cell_start, cell_points);
  k_na_outside<<<1, 1, 0, stream>>>(s, n_outside);
  if (cudaGetLastError() != cudaSuccess) return FSI_ERR_CUDA;
  return FSI_OK;
}

}  // namespace
