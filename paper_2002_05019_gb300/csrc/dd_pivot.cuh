// Restricted Bunch-Kaufman pivoting inside a diagonal block (Section II: the
// auxiliary matrix is factored by a block LDL^T whose diagonal blocks use
// Bunch-Kaufman pivoting restricted to the block, so the block structure
// found by the symbolic factorization never changes).
//
// Pivot choice (Bunch and Kaufman 1977, partial pivoting for symmetric
// indefinite matrices), at column j of the trailing part of an nb x nb block,
// with |z| the complex modulus and alpha = (1 + sqrt 17) / 8:
//   lambda = max_{i > j} |a_ij|   (rows of the block only), attained first at r;
//   1x1 at j                       if |a_jj| >= alpha lambda (or lambda = 0),
//   1x1 at j                       else if |a_jj| sigma >= alpha lambda^2,
//                                  sigma = max_{i >= j, i != r} |a_ir|;
//   1x1 at j after j <-> r         else if |a_rr| >= alpha sigma;
//   2x2 on (j, j+1) after j+1 <-> r otherwise.
// Ties go to the lowest index.  The last column of a block has lambda = 0.
//
// Storage of a factored diagonal tile that pivots (64 x 64, row-major in the
// front): unit lower factor below the diagonal with 0 at (j+1, j) of every
// 2x2 block, the diagonal of D on the diagonal, and the off-diagonal entry of
// each 2x2 block of D at (j, j+1) above the diagonal (0 at every other
// (c, c+1)).  perm[c] (one byte per position) is the tile-local index, in the
// order before the step, of the unknown at pivot position c.  With these the
// tile step reads  P_k S_kk P_k^T = L_kk D_k L_kk^T  and the panel below is
// L_ik = S_ik P_k^T L_kk^{-T} D_k^{-1}; the rows of earlier panels are not
// interchanged, so the solves apply P_k to the tile's right-hand side after
// the contributions of earlier tiles (forward) and P_k^T before publishing it
// (backward).
#pragma once
#include "dd_complex.cuh"

namespace ddk {

constexpr double kBkAlpha = 0.6403882032022076;   // (1 + sqrt(17)) / 8

__device__ __forceinline__ int pv_tri(int i, int c) { return (i * (i + 1)) / 2 + c; }

__device__ __forceinline__ double cabsd(double2 a) { return sqrt(a.x * a.x + a.y * a.y); }
__device__ __forceinline__ double cabsd(float2 a) { return sqrt((double)a.x * a.x + (double)a.y * a.y); }

// Pivot choice at column j of a packed-lower nb x nb block; called by one full
// warp.  Returns the pivot size s and the index exchanged with j + s - 1 (or -1).
template <typename C>
__device__ void bk_choose(const C* a, int j, int nb, int& s, int& q) {
  const int lane = threadIdx.x & 31;
  double lam = -1.0;
  int r = nb;
  for (int i = j + 1 + lane; i < nb; i += 32) {
    const double v = cabsd(a[pv_tri(i, j)]);
    if (v > lam) { lam = v; r = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double lo = __shfl_xor_sync(0xffffffffu, lam, o);
    const int ro = __shfl_xor_sync(0xffffffffu, r, o);
    if (lo > lam || (lo == lam && ro < r)) { lam = lo; r = ro; }
  }
  const double ajj = cabsd(a[pv_tri(j, j)]);
  s = 1;
  q = -1;
  if (r >= nb || !(lam > 0.0) || ajj >= kBkAlpha * lam) return;
  double sig = 0.0;
  for (int i = j + lane; i < nb; i += 32)
    if (i != r) sig = fmax(sig, cabsd(i < r ? a[pv_tri(r, i)] : a[pv_tri(i, r)]));
  for (int o = 16; o > 0; o >>= 1) sig = fmax(sig, __shfl_xor_sync(0xffffffffu, sig, o));
  if (ajj * sig >= kBkAlpha * lam * lam) return;
  if (cabsd(a[pv_tri(r, r)]) >= kBkAlpha * sig) {
    q = r;
    return;
  }
  s = 2;
  q = (r == j + 1) ? -1 : r;
}

// Symmetric interchange of rows and columns p < q of a packed-lower nb x nb
// block, including the already factored columns left of p.
template <typename C>
__device__ void sym_swap(C* a, int p, int q, int nb) {
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    int x = -1, y = -1;
    if (c < p) { x = pv_tri(p, c); y = pv_tri(q, c); }
    else if (c == p) { x = pv_tri(p, p); y = pv_tri(q, q); }
    else if (c < q) { x = pv_tri(c, p); y = pv_tri(q, c); }
    else if (c > q) { x = pv_tri(c, p); y = pv_tri(c, q); }
    if (x >= 0) {
      const C t = a[x];
      a[x] = a[y];
      a[y] = t;
    }
  }
}

// In-place LDL^T with restricted Bunch-Kaufman pivoting of a packed-lower
// nb x nb block in shared memory, by all threads of the block (nthreads a
// multiple of nb, at least 32).  On return: a holds L (unit, not stored) below
// the diagonal with 0 at (j+1, j) of each 2x2 pivot, D on the diagonal;
// dsup[c] the 2x2 off-diagonal of D at (c, c+1) or 0; perm[c] the original
// block index at position c.  w0, w1: nb scratch entries each.  Counts the
// interchanges and 2x2 pivots in *n_swap, *n_2x2 (shared counters).
template <typename C>
__device__ void ldlt_bk(C* a, int nb, int* perm, C* dsup, C* w0, C* w1, int* n_swap, int* n_2x2) {
  __shared__ int s_step, s_q;
  const int tpr = blockDim.x / nb, row = threadIdx.x / tpr, sub = threadIdx.x % tpr;
  if (threadIdx.x < nb) {
    perm[threadIdx.x] = threadIdx.x;
    dsup[threadIdx.x] = czero<C>();
  }
  __syncthreads();
  for (int j = 0; j < nb;) {
    if (threadIdx.x < 32) {
      int s, q;
      bk_choose(a, j, nb, s, q);
      if (threadIdx.x == 0) {
        s_step = s;
        s_q = q;
      }
    }
    __syncthreads();
    const int s = s_step, q = s_q;
    if (q >= 0) {
      const int p = j + s - 1;
      sym_swap(a, p, q, nb);
      if (threadIdx.x == 0) {
        const int t = perm[p];
        perm[p] = perm[q];
        perm[q] = t;
        ++*n_swap;
      }
      __syncthreads();
    }
    if (s == 1) {
      const C rinv = cdiv(cmake<C>(1, 0), a[pv_tri(j, j)]);
      if (sub == 0 && row > j && row < nb) {
        const C v = a[pv_tri(row, j)];
        w0[row] = v;
        a[pv_tri(row, j)] = cmul(v, rinv);
      }
      __syncthreads();
      if (row > j && row < nb) {
        const C l = a[pv_tri(row, j)];
        for (int c = j + 1 + sub; c <= row; c += tpr) a[pv_tri(row, c)] = cfms(l, w0[c], a[pv_tri(row, c)]);
      }
      __syncthreads();
    } else {
      // D block [d0 b; b d1] and its inverse [g0 g1; g1 g2]
      const C d0 = a[pv_tri(j, j)], b = a[pv_tri(j + 1, j)], d1 = a[pv_tri(j + 1, j + 1)];
      const C idet = cdiv(cmake<C>(1, 0), csub(cmul(d0, d1), cmul(b, b)));
      const C g0 = cmul(d1, idet), g2 = cmul(d0, idet);
      const C g1 = cmake<C>(-(b.x * idet.x - b.y * idet.y), -(b.x * idet.y + b.y * idet.x));
      if (sub == 0 && row > j + 1 && row < nb) {
        const C v0 = a[pv_tri(row, j)], v1 = a[pv_tri(row, j + 1)];
        w0[row] = v0;
        w1[row] = v1;
        a[pv_tri(row, j)] = cfma(v1, g1, cmul(v0, g0));
        a[pv_tri(row, j + 1)] = cfma(v1, g2, cmul(v0, g1));
      }
      __syncthreads();
      if (row > j + 1 && row < nb) {
        const C l0 = a[pv_tri(row, j)], l1 = a[pv_tri(row, j + 1)];
        for (int c = j + 2 + sub; c <= row; c += tpr)
          a[pv_tri(row, c)] = cfms(l1, w1[c], cfms(l0, w0[c], a[pv_tri(row, c)]));
      }
      if (threadIdx.x == 0) {
        dsup[j] = b;
        ++*n_2x2;
      }
      __syncthreads();
      if (threadIdx.x == 0) a[pv_tri(j + 1, j)] = czero<C>();
      __syncthreads();
    }
    j += s;
  }
}

// Coefficients of D_k^{-1} for pivot position p of a factored tile (see the
// storage note above; D points at the tile's (0, 0) entry in the front):
// (D^{-1} x)_p = g0 x_p + g1 x_q.
template <typename S>
__device__ __forceinline__ void dinv_col(const S* D, int64_t ld, int p, S& g0, S& g1, int& q) {
  constexpr int T = 64;
  const double2 dp = cconv<double2>(D[(int64_t)p * ld + p]);
  const S up = p + 1 < T ? D[(int64_t)p * ld + p + 1] : czero<S>();
  const S lo = p > 0 ? D[(int64_t)(p - 1) * ld + p] : czero<S>();
  const bool first = up.x != 0 || up.y != 0, second = !first && (lo.x != 0 || lo.y != 0);
  if (!first && !second) {
    g0 = cconv<S>(cdiv(make_double2(1.0, 0.0), dp));
    g1 = czero<S>();
    q = p;
    return;
  }
  q = first ? p + 1 : p - 1;
  const double2 dq = cconv<double2>(D[(int64_t)q * ld + q]);
  const double2 b = cconv<double2>(first ? up : lo);
  const double2 idet = cdiv(make_double2(1.0, 0.0), csub(cmul(dp, dq), cmul(b, b)));
  g0 = cconv<S>(cmul(dq, idet));
  const double2 nb = cmul(b, idet);
  g1 = cconv<S>(make_double2(-nb.x, -nb.y));
}

}  // namespace ddk
