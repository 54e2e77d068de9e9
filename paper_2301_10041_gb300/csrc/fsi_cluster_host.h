// Host side of the cluster-resident coarse multigrid levels: partition of
// every level's block rows over the CTAs of one cluster, the per-CTA shared
// memory images of the level operators (sliced ELL with packed columns), and
// the shared-memory layout of the level vectors.
//
// Included after the definitions of Arena (upload, count_only), Cheb and
// MG<T> (lv[l].ch, coarse_inv, coarse_n, coarse_ld, degree, cl), by the solver and by
// the CPU test harness that emulates the cluster kernel.
#pragma once
#include <algorithm>
#include <cstring>
#include <vector>

#include "fsi_cluster.cuh"
#include "fsi_internal.h"

namespace fsi {

// Per-CTA images of the cluster levels.  Every array starts at the same
// offset in every CTA's image (the largest CTA part decides), so one set of
// offsets describes all of them.
struct ClImages {
  std::vector<std::vector<unsigned char>> img;
  explicit ClImages(int cs) : img(cs) {}
  int add(const std::vector<std::vector<unsigned char>>& parts) {
    size_t off = 0;
    for (auto& v : img) off = std::max(off, v.size());
    off = (off + 15) & ~(size_t)15;
    for (size_t r = 0; r < img.size(); ++r) {
      img[r].resize(off);
      img[r].insert(img[r].end(), parts[r].begin(), parts[r].end());
    }
    return (int)off;
  }
  size_t size() const {
    size_t m = 0;
    for (auto& v : img) m = std::max(m, v.size());
    return (m + 15) & ~(size_t)15;
  }
};

template <class V>
inline std::vector<unsigned char> cl_bytes(const std::vector<V>& v) {
  std::vector<unsigned char> b(v.size() * sizeof(V));
  if (!v.empty()) std::memcpy(b.data(), v.data(), b.size());
  return b;
}

// packed column of block column c of a level with nsl slices: owner CTA and
// block row inside the owner
inline int cl_pack(int c, int nsl, int cs) {
  const int s = c / kSliceRows;
  int r = (int)(((long long)s * cs) / nsl);
  int s0, s1;
  for (;;) {  // the owner rule cl_own, searched from the proportional guess
    cl_own(nsl, r, cs, s0, s1);
    if (s < s0) --r;
    else if (s >= s1) ++r;
    else break;
  }
  return (r << kClColBits) | (c - s0 * kSliceRows);
}

inline int cl_own_rows(int nrows, int nsl, int r, int cs) {
  int s0, s1;
  cl_own(nsl, r, cs, s0, s1);
  return std::max(0, std::min(s1 * kSliceRows, nrows) - s0 * kSliceRows);
}

// Add one matrix (rows on its own level, columns on a level of col_nsl
// slices) to the images; returns its offsets.
template <class T>
inline ClMat cl_add_matrix(ClImages& im, const SellHost& S, int col_nsl, int cs) {
  std::vector<std::vector<unsigned char>> soff(cs), len(cs), col(cs), val(cs);
  for (int r = 0; r < cs; ++r) {
    int s0, s1;
    cl_own(S.nslices, r, cs, s0, s1);
    const int a = S.soff[s0], e = S.soff[s1];
    std::vector<int> so, ln, cc;
    std::vector<T> vv;
    for (int s = s0; s < s1; ++s) so.push_back(S.soff[s] - a);
    for (int row = s0 * kSliceRows; row < std::min(s1 * kSliceRows, S.nrows); ++row) ln.push_back(S.len[row]);
    for (int q = a; q < e; ++q) cc.push_back(S.col[q] >= 0 ? cl_pack(S.col[q], col_nsl, cs) : 0);
    for (size_t q = (size_t)a * S.NV; q < (size_t)e * S.NV; ++q) vv.push_back((T)S.val[q]);
    soff[r] = cl_bytes(so); len[r] = cl_bytes(ln); col[r] = cl_bytes(cc); val[r] = cl_bytes(vv);
  }
  ClMat m;
  m.soff = im.add(soff);
  m.len = im.add(len);
  m.col = im.add(col);
  m.val = im.add(val);
  return m;
}

// Build the cluster image of levels lc..last, taking the finest lc whose
// operators and vectors fit in `cap` bytes of shared memory per CTA and that
// viable(smem) accepts; false when no suffix of two or more levels
// qualifies.  On success mg.cl holds the launch arguments (without in_b and
// out_x) and the images are uploaded through the arena.
template <class T, class ArenaT, class MGT, class Viable>
bool build_cluster(ArenaT& ar, const HostSetup& hs, bool pressure, MGT& mg, int cs, size_t cap, Viable viable,
                   int lc_min = 0) {
  const int last = (int)mg.lv.size() - 1;
  const int B = pressure ? 3 : 2;
  if (last < 1 || mg.degree > kClMaxDeg) return false;
  for (int lc = std::max(lc_min, last + 1 - kClMaxLevels); lc < last; ++lc) {
    ClImages im(cs);
    ClArgs<T> a;
    a.nlev = last - lc + 1;
    a.degree = mg.degree;
    a.csize = cs;
    for (int l = lc; l <= last; ++l) {
      const FluidLevelHost& H = hs.levels[l];
      ClLevel<T>& C = a.lv[l - lc];
      const HostBlockMatrix& A = pressure ? H.L : H.A;
      C.nrows = A.nrows;
      C.nsl = (A.nrows + kSliceRows - 1) / kSliceRows;
      if (l < last) {
        C.A = cl_add_matrix<T>(im, to_sell(A), C.nsl, cs);
        const HostBlockMatrix& Pm = pressure ? H.Pp : H.Pu;
        const HostBlockMatrix& Ac = pressure ? hs.levels[l + 1].L : hs.levels[l + 1].A;
        C.P = cl_add_matrix<T>(im, to_sell(Pm), (Ac.nrows + kSliceRows - 1) / kSliceRows, cs);
        const std::vector<double>& dv = pressure ? H.dinvL : H.dinvA;
        std::vector<std::vector<unsigned char>> parts(cs);
        for (int r = 0; r < cs; ++r) {
          int s0, s1;
          cl_own(C.nsl, r, cs, s0, s1);
          const int nr = cl_own_rows(C.nrows, C.nsl, r, cs);
          std::vector<T> v((size_t)nr * B);
          for (int i = 0; i < nr * B; ++i) v[i] = (T)dv[(size_t)s0 * kSliceRows * B + i];
          parts[r] = cl_bytes(v);
        }
        C.dinv = im.add(parts);
        const auto& ch = mg.lv[l].ch;
        C.c0 = (T)ch.c0;
        for (size_t i = 0; i < ch.c1.size() && i < (size_t)kClMaxDeg; ++i) {
          C.c1[i] = (T)ch.c1[i];
          C.c2[i] = (T)ch.c2[i];
        }
      }
      if (l > lc) {
        const FluidLevelHost& F = hs.levels[l - 1];
        const HostBlockMatrix& Rm = pressure ? F.Rp : F.Ru;
        const HostBlockMatrix& Af = pressure ? F.L : F.A;
        C.R = cl_add_matrix<T>(im, to_sell(Rm), (Af.nrows + kSliceRows - 1) / kSliceRows, cs);
      }
      if (l == last) {
        std::vector<std::vector<unsigned char>> parts(cs);
        std::vector<int> g(C.nrows);
        for (int row = 0; row < C.nrows; ++row) g[row] = cl_pack(row, C.nsl, cs);
        for (int r = 0; r < cs; ++r) parts[r] = cl_bytes(g);
        a.gmap = im.add(parts);
      }
    }
    const size_t blob = im.size();
    // level vectors follow the operator images (they are not copied in)
    size_t off = blob;
    auto vec = [&](size_t n) {
      off = (off + 15) & ~(size_t)15;
      const int o = (int)off;
      off += n * sizeof(T);
      return o;
    };
    for (int l = lc; l <= last; ++l) {
      ClLevel<T>& C = a.lv[l - lc];
      int mx = 0;
      for (int r = 0; r < cs; ++r) mx = std::max(mx, cl_own_rows(C.nrows, C.nsl, r, cs));
      const size_t n = (size_t)mx * B;
      C.x = vec(n); C.x2 = vec(n); C.b = vec(n); C.r = vec(n); C.d = vec(n);
    }
    a.dense_n = mg.coarse_n;
    a.dense_ld = mg.coarse_ld;
    a.gbuf = vec((size_t)a.dense_n);
    const size_t smem = (off + 15) & ~(size_t)15;
    if (smem > cap || !viable(smem)) continue;
    // upload the images, CTA after CTA
    const size_t stride = blob;
    std::vector<unsigned char> all(stride * cs, 0);
    for (int r = 0; r < cs; ++r) std::memcpy(all.data() + stride * r, im.img[r].data(), im.img[r].size());
    const unsigned char* d = ar.upload(all);
    a.blob = reinterpret_cast<const uint4*>(d);
    a.blob_bytes = (int)blob;
    a.blob_stride = stride / 16;
    a.dense_inv = mg.coarse_inv;
    mg.cl.on = true;
    mg.cl.lc = lc;
    mg.cl.smem = smem;
    mg.cl.args = a;
    return true;
  }
  return false;
}

}  // namespace fsi
