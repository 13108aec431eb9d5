// Batched partial LDL^T of dense fronts (Section II: many independent domain
// factorizations, and the block LDL^T of the auxiliary matrix).
//
// One blocked right-looking step k of the elimination of every front in a
// batch is three launches over a host-built task list:
//   k_diag    (front)        : A_kk = L_kk D_k L_kk^T, 64 x 64, in shared memory
//   k_trsm    (front, i)     : L_ik = A_ik L_kk^{-T} D_k^{-1}
//   k_update  (front, i, j)  : A_ij -= L_ik D_k L_jk^T   (k < j <= i)
// Complex symmetric: plain transposes, no conjugation.  Fronts are stored
// row-major (lower triangle), interleaved complex, double2 (FP64 form) or
// float2 (mixed form).
#include <algorithm>
#include <type_traits>

#include "dd_complex.cuh"
#include "dd_dfloat.cuh"
#include "dd_internal.h"
#include "dd_pivot.cuh"
#include "dd_tc.cuh"

namespace ddk {

namespace {

constexpr int T = DD_TILE;

__device__ __forceinline__ int tri(int i, int c) { return (i * (i + 1)) / 2 + c; }

using tc::split_tf32;
using tc::swz128;
__device__ __forceinline__ void put_img(unsigned char* base, int row, int k, float v) {
  *reinterpret_cast<float*>(base + swz128(row, k)) = v;
}

template <typename S>
__device__ __forceinline__ void write_images(unsigned char*, const FrontDev&, int, int, S, S, bool) {}
// mixed form: the operand images of the tensor-core update.  Unpivoted
// fronts: one image of M_ik = L_ik D_k^(1/2) serves as both operands
// (L_i D L_j^T = M_i M_j^T); fronts that pivot (2 x 2 blocks in D): the A image
// of L_ik and the B image of W_ik = L_ik D_k.  Both images use the A layout.
template <>
__device__ __forceinline__ void write_images<float2>(unsigned char* ws, const FrontDev& F, int ti, int rc, float2 va,
                                                     float2 vb, bool dual) {
  const int r = rc >> 6, p = rc & 63;              // row of the tile, K index
  const int a = p >> 5, kk = p & 31;
  const int ra = (r >> 4) * 32 + (r & 15);         // piece row of the real part (imaginary: + 16)
  unsigned char* Ab = ws + F.ws_off + (int64_t)ti * DD_TC_ATILE;
  float h, l;
  split_tf32(va.x, h, l);
  put_img(Ab + (0 * 2 + a) * DD_TC_ATOM, ra, kk, h);
  put_img(Ab + (1 * 2 + a) * DD_TC_ATOM, ra, kk, l);
  split_tf32(va.y, h, l);
  put_img(Ab + (0 * 2 + a) * DD_TC_ATOM, ra + 16, kk, h);
  put_img(Ab + (1 * 2 + a) * DD_TC_ATOM, ra + 16, kk, l);
  if (!dual) return;
  unsigned char* Bb = ws + F.ws_boff + (int64_t)ti * DD_TC_BTILE;
  split_tf32(vb.x, h, l);
  put_img(Bb + (0 * 2 + a) * DD_TC_ATOM, ra, kk, h);
  put_img(Bb + (1 * 2 + a) * DD_TC_ATOM, ra, kk, l);
  split_tf32(vb.y, h, l);
  put_img(Bb + (0 * 2 + a) * DD_TC_ATOM, ra + 16, kk, h);
  put_img(Bb + (1 * 2 + a) * DD_TC_ATOM, ra + 16, kk, l);
}

// a square root w of z, w^2 = z (principal branch: for Re z >= 0,
// w = (t, Im z / 2t), else (|Im z| / 2t, sign(Im z) t), t = sqrt((|z| + |Re z|) / 2))
__device__ __forceinline__ float2 csqrt_f(float2 z) {
  const float t = sqrtf(0.5f * (hypotf(z.x, z.y) + fabsf(z.x)));
  if (t == 0.f) return make_float2(0.f, 0.f);
  if (z.x >= 0.f) return make_float2(t, 0.5f * z.y / t);
  return make_float2(0.5f * fabsf(z.y) / t, copysignf(t, z.y));
}

__device__ void status_pivot(DevStatus* st, int front, int row) {
  if (atomicCAS(&st->code, 0, 3) == 0) {
    st->front = front;
    st->row = row;
  }
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_pos(unsigned long long* p, double v) {
  atomicMin(p, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// leaf front initialisation: permuted A_i (lower part), identity padding, B_i
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_leaf_init(S* pool, const FrontDev* fr, const LeafDev* lv, const int32_t* rowptr,
                            const int32_t* colind, const double2* val, const int32_t* iperm,
                            const int32_t* b_row, const int32_t* b_local, const int8_t* b_sign) {
  const LeafDev L = lv[blockIdx.x];
  const FrontDev F = fr[L.front];
  if (F.kind != 0) return;   // a sparse domain: its fronts are filled by k_sparse_init
  S* A = pool + F.off;
  const int32_t* rp = rowptr + L.rowptr_off;
  const int32_t* ip = iperm + L.perm_off;
  const int32_t* ci = colind + L.csr_off;
  const double2* va = val + L.csr_off;
  for (int r = threadIdx.x; r < L.n; r += blockDim.x) {
    const int pr = ip[r];
    for (int q = rp[r]; q < rp[r + 1]; ++q) {
      const int pc = ip[ci[q]];
      if (pr >= pc) A[(int64_t)pr * F.ld + pc] = cconv<S>(va[q]);
    }
  }
  for (int r = F.ne + threadIdx.x; r < F.ne_pad; r += blockDim.x)
    A[(int64_t)r * F.ld + r] = cmake<S>(1, 0);
  for (int q = threadIdx.x; q < L.nb; q += blockDim.x) {
    const int row = F.ne_pad + b_row[L.b_off + q];
    const int col = ip[b_local[L.b_off + q]];
    A[(int64_t)row * F.ld + col] = cmake<S>((float)b_sign[L.b_off + q], 0);
  }
}

// fronts of sparse domains: every A_i entry, B_i entry and padding diagonal
// goes to its precomputed pool position (src >= 0: a CSR value; -1: +1; -2: -1)
template <typename S>
__global__ void k_sparse_init(S* pool, const int64_t* dst, const int32_t* src, int64_t n, const double2* val) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = src[e];
    pool[dst[e]] = q >= 0 ? cconv<S>(val[q]) : cmake<S>(q == -1 ? 1 : -1, 0);
  }
}

template <typename S>
__global__ void k_node_init(S* pool, const FrontDev* fr, const int32_t* ids) {
  const FrontDev F = fr[ids[blockIdx.x]];
  S* A = pool + F.off;
  for (int r = F.ne + threadIdx.x; r < F.ne_pad; r += blockDim.x)
    A[(int64_t)r * F.ld + r] = cmake<S>(1, 0);
}

// ---------------------------------------------------------------------------
// diagonal tile: unpivoted LDL^T of a 64 x 64 block in shared memory (packed
// lower triangle), computed in precision C (FP64 for the auxiliary pivot
// blocks of the mixed form)
// ---------------------------------------------------------------------------
// writes the pivot data of a factored tile that pivoted: the 2x2 off-diagonals
// of D above the diagonal (0 elsewhere on the superdiagonal) and the permutation
template <typename S, typename C>
__device__ void store_pivots(S* base, int64_t ld, const int* perm, const C* dsup, uint8_t* piv_tile) {
  if (threadIdx.x < T - 1) base[(int64_t)threadIdx.x * ld + threadIdx.x + 1] = cconv<S>(dsup[threadIdx.x]);
  if (threadIdx.x < T) piv_tile[threadIdx.x] = (uint8_t)perm[threadIdx.x];
}

// pivot statistics of column c of a factored tile: |d| (1x1) or sqrt|det| (2x2)
template <typename A, typename C>
__device__ void pivot_stats(const A* a, const C* dsup, bool pv, int c, int f, int row, DevStatus* st) {
  double m2 = cabs2d(a[tri(c, c)]);
  if (pv) {
    const int p0 = (c + 1 < T && (dsup[c].x != 0 || dsup[c].y != 0)) ? c
                   : (c > 0 && (dsup[c - 1].x != 0 || dsup[c - 1].y != 0)) ? c - 1 : -1;
    if (p0 >= 0) {
      const double2 d0 = cconv<double2>(a[tri(p0, p0)]), d1 = cconv<double2>(a[tri(p0 + 1, p0 + 1)]);
      const double2 b = cconv<double2>(dsup[p0]);
      m2 = sqrt(cabs2d(csub(cmul(d0, d1), cmul(b, b))));
    }
  }
  if (!(m2 > 0.0) || !isfinite(m2)) status_pivot(st, f, row);
  const double m = sqrt(m2);
  if (isfinite(m)) {
    atomic_max_pos(&st->max_abs_d, m);
    atomic_min_pos(&st->min_abs_d, m);
  }
}

// ---------------------------------------------------------------------------
// diagonal tile: LDL^T of a 64 x 64 block in shared memory (packed lower
// triangle), computed in precision C (FP64 for the auxiliary pivot blocks of
// the mixed form); unpivoted, or with restricted Bunch-Kaufman pivoting for
// the fronts that pivot
// ---------------------------------------------------------------------------
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_diag(S* pool, const FrontDev* fr, const int32_t* fids, int k,
                                              DevStatus* st, uint8_t* piv) {
  __shared__ C a[T * (T + 1) / 2];
  __shared__ C w[T];        // column j before scaling: w_c = d_j * l_cj
  __shared__ C w1[T];       // second column of a 2x2 pivot
  __shared__ C dsup[T];
  __shared__ int perm[T];
  __shared__ int cnt[2];
  __shared__ C rinv;        // 1 / d_j
  const int f = fids[blockIdx.x];
  const FrontDev F = fr[f];
  const bool pv = piv != nullptr && F.piv != 0;
  S* base = pool + F.off + (int64_t)(k * T) * F.ld + k * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int i = idx / T, c = idx % T;
    if (c <= i) a[tri(i, c)] = cconv<C>(base[(int64_t)i * F.ld + c]);
  }
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  if (pv) {
    ldlt_bk<C>(a, T, perm, dsup, w, w1, &cnt[0], &cnt[1]);
  } else {
    if (threadIdx.x == 0) rinv = cdiv(cmake<C>(1, 0), a[0]);
    __syncthreads();
    const int row = threadIdx.x >> 2, sub = threadIdx.x & 3;   // 4 threads per row
    for (int j = 0; j < T; ++j) {
      // l_ij = a_ij / d_j, keeping the unscaled value for the update
      if (sub == 0 && row > j) {
        const C v = a[tri(row, j)];
        w[row] = v;
        a[tri(row, j)] = cmul(v, rinv);
      }
      __syncthreads();
      // a_ic -= l_ij * (d_j l_cj) for j < c <= i
      if (row > j) {
        const C l = a[tri(row, j)];
        for (int c = j + 1 + sub; c <= row; c += 4) a[tri(row, c)] = cfms(l, w[c], a[tri(row, c)]);
        if (row == j + 1 && sub == 0) rinv = cdiv(cmake<C>(1, 0), a[tri(j + 1, j + 1)]);
      }
      __syncthreads();
    }
  }
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int i = idx / T, c = idx % T;
    if (c <= i) base[(int64_t)i * F.ld + c] = cconv<S>(a[tri(i, c)]);
  }
  if (pv) {
    store_pivots<S, C>(base, F.ld, perm, dsup, piv + ((int64_t)F.tile_off + k) * T);
    if (threadIdx.x == 0 && (cnt[0] | cnt[1])) {
      atomicAdd(&st->n_swap, (unsigned long long)cnt[0]);
      atomicAdd(&st->n_2x2, (unsigned long long)cnt[1]);
    }
  }
  if (threadIdx.x < T) {
    const int r = k * T + threadIdx.x;
    if (r < F.ne) pivot_stats(a, dsup, pv, threadIdx.x, f, r, st);
  }
}

// ---------------------------------------------------------------------------
// mixed form diagonal tile: the 64 x 64 tile is factored as 2 x 2 blocks of
// 32; the two 32 x 32 pivot blocks in precision C (FP64 for the auxiliary
// matrix, FP32 for the domains), everything else in FP32 as products with the
// inverses of the unit-lower pivot blocks:
//   L11 D1 L11^T = A11            (pivot block 1, precision C)
//   N11 = L11^{-1}
//   X21 = A21 N11^T,  L21 = X21 D1^{-1},  A22 -= L21 X21^T
//   L22 D2 L22^T = A22            (pivot block 2, precision C)
//   N22 = L22^{-1},   N21 = -N22 (L21 N11)
// N = [N11 0; N21 N22] = L_kk^{-1} is stored (FP32) for the panel kernel and
// the substitutions.  GB300's FP64 rate is about 1/64 of its FP32 rate, so
// the FP64 work is kept to the two pivot blocks and spread evenly over all
// threads.
// ---------------------------------------------------------------------------
constexpr int PB = 32;

// 1 / d: one real division (the pivot magnitudes of these matrices are far
// from the limits of the exponent range, so |d|^2 cannot overflow in FP64)
__device__ __forceinline__ double2 crcp(double2 d) {
  const double s = 1.0 / (d.x * d.x + d.y * d.y);
  return make_double2(d.x * s, -d.y * s);
}
// FP32 pivots: |d|^2 stays in range for pivots between about 1e-19 and 1e19
__device__ __forceinline__ float2 crcp(float2 d) {
  const float s = 1.f / (d.x * d.x + d.y * d.y);
  return make_float2(d.x * s, -d.y * s);
}

// element e of a column-descending enumeration of the update set of a 32 x 32
// block: columns c = 31, 30, ..., 1, rows r = c..31 within each, so the
// elements with c > j are exactly e < (31 - j)(32 - j) / 2
__device__ __forceinline__ uint16_t pb_elem(int e) {
  int k = 0;
  while ((k + 1) * (k + 2) / 2 <= e) ++k;
  const int c = PB - 1 - k, r = c + (e - k * (k + 1) / 2);
  return (uint16_t)((r << 8) | c);
}

// one complex value of lane `src` to the whole warp
__device__ __forceinline__ float2 shfl_c(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ double2 shfl_c(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ dfc shfl_c(dfc v, int src) {
  dfc r;
  r.x.hi = __shfl_sync(0xffffffffu, v.x.hi, src);
  r.x.lo = __shfl_sync(0xffffffffu, v.x.lo, src);
  r.y.hi = __shfl_sync(0xffffffffu, v.y.hi, src);
  r.y.lo = __shfl_sync(0xffffffffu, v.y.lo, src);
  return r;
}

// Unpivoted LDL^T of pivot block jb of the tile in precision C, and the FP32
// inverse N = L^{-1} of its unit-lower factor built alongside (N <- E_j N for
// the elimination E_j of column j: rows r > j of N lose l_rj times row j).
// Right-looking with a look-ahead of one column, one barrier per column:
// while warps 1-7 apply column j to the columns c >= j + 2 (and to N), warp 0
// applies it to column j + 1 alone, lane r holding row r, and factors that
// column at once (the pivot reaches every lane by shuffles, each lane forms
// the reciprocal itself and scales its entry), so the chain from one pivot to
// the next is one update, one reciprocal and one scaling inside a warp.  The
// unscaled column (w) and its FP32 scaled copy (lcol) are double-buffered:
// warps 1-7 read column j's while warp 0 writes column j + 1's.  Each thread
// of warps 1-7 owns at most three trailing elements (a column-descending
// enumeration: the elements with c > j + 1 are e < (30 - j)(31 - j) / 2) and
// the row r = t / 7 of N at columns t % 7 + 7 m (t = tid - 32).
template <typename C>
__device__ void factor_pivot32(float2* a, int jb, C* ap, C* w, float2* lcol, float2* li) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kW = 224;   // threads of warps 1-7
  int er[3], ec[3], erc[3], er0[3];
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const int e = (tid - 32) + h * kW;
    const bool has = warp > 0 && e < PB * (PB - 1) / 2;
    const uint16_t rc = has ? pb_elem(e) : (uint16_t)0;
    er[h] = rc >> 8;
    ec[h] = has ? (rc & 255) : -1;   // -1: no element
    erc[h] = tri(er[h], ec[h] < 0 ? 0 : ec[h]);
    er0[h] = tri(er[h], 0);
  }
  const int nt = tid - 32, nr = nt / 7, nq = nt - 7 * (nt / 7);   // N row and first column (warps 1-7)
  const int nbase = tri(jb + nr, jb);                                 // N[nr][q] at li[nbase + q]
  for (int idx = tid; idx < PB * PB; idx += blockDim.x) {
    const int i = idx / PB, c = idx % PB;
    if (c <= i) {
      ap[tri(i, c)] = cconv<C>(a[tri(jb + i, jb + c)]);
      li[tri(jb + i, jb + c)] = make_float2(c == i ? 1.f : 0.f, 0.f);
    }
  }
  __syncthreads();
  if (warp == 0) {   // column 0
    const C rv = crcp(ap[0]);
    if (lane > 0) {
      const C v = ap[tri(lane, 0)];
      const C l = cmul(v, rv);
      w[lane] = v;
      ap[tri(lane, 0)] = l;
      lcol[lane] = cconv<float2>(l);
    }
  }
  __syncthreads();
  for (int j = 0; j < PB - 1; ++j) {
    const int cur = (j & 1) * PB, nxt = PB - cur;   // buffers of columns j and j + 1
    if (warp == 0) {
      // column j + 1: update by column j, then the pivot and the scaled column
      C v = ap[tri(lane, 0)];   // placeholder for lanes above the column
      if (lane > j) v = cfms(ap[tri(lane, j)], w[cur + j + 1], ap[tri(lane, j + 1)]);
      const C d = shfl_c(v, j + 1);
      if (lane == j + 1) ap[tri(lane, lane)] = v;
      if (lane > j + 1) {
        const C l = cmul(v, crcp(d));
        w[nxt + lane] = v;
        ap[tri(lane, j + 1)] = l;
        lcol[nxt + lane] = cconv<float2>(l);
      }
    } else {
#pragma unroll
      for (int h = 0; h < 3; ++h)
        if (ec[h] > j + 1) ap[erc[h]] = cfms(ap[er0[h] + j], w[cur + ec[h]], ap[erc[h]]);
      if (nr > j && nr < PB) {
        const float2 l = lcol[cur + nr];
        const int jrow = tri(jb + j, jb);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          const int q = nq + 7 * m;
          if (q <= j) li[nbase + q] = cfms(l, li[jrow + q], li[nbase + q]);
        }
      }
    }
    __syncthreads();
  }
  // the last column of N: rows r > 30 lose l_{r,30} times row 30 -- done in
  // the loop; write the factor back
  for (int idx = tid; idx < PB * PB; idx += blockDim.x) {
    const int i = idx / PB, c = idx % PB;
    if (c <= i) a[tri(jb + i, jb + c)] = cconv<float2>(ap[tri(i, c)]);
  }
  __syncthreads();
}

// the same with restricted Bunch-Kaufman pivoting inside the 32 x 32 block;
// perm and dsup receive the block-local permutation and 2x2 off-diagonals
template <typename C>
__device__ void factor_pivot32_bk(float2* a, int jb, C* ap, C* w, C* w1, int* perm, C* dsup, int* cnt) {
  for (int idx = threadIdx.x; idx < PB * PB; idx += blockDim.x) {
    const int i = idx / PB, c = idx % PB;
    if (c <= i) ap[tri(i, c)] = cconv<C>(a[tri(jb + i, jb + c)]);
  }
  __syncthreads();
  ldlt_bk<C>(ap, PB, perm, dsup, w, w1, &cnt[0], &cnt[1]);
  for (int idx = threadIdx.x; idx < PB * PB; idx += blockDim.x) {
    const int i = idx / PB, c = idx % PB;
    if (c <= i) a[tri(jb + i, jb + c)] = cconv<float2>(ap[tri(i, c)]);
  }
  __syncthreads();
}

// the pivoting factorization where the precision supports it (FP32, FP64); the
// double-float form serves unpivoted fronts only and never calls it
template <typename C, typename CB>
__device__ void factor_pivot32_any_bk(float2* a, int jb, C* ap, C* w, CB* w1, int* perm, CB* dsup, int* cnt) {
  if constexpr (std::is_same<C, CB>::value) factor_pivot32_bk<C>(a, jb, ap, w, w1, perm, dsup, cnt);
}

// N = L^{-1} of the unit-lower 32 x 32 block jb of the tile, into the same
// positions of the packed 64 x 64 li: 8 lanes per column, rows in order
__device__ void inv_unit_lower32(const float2* a, int jb, float2* li) {
  const int col = threadIdx.x >> 3, part = threadIdx.x & 7;
  if (part == 0) li[tri(jb + col, jb + col)] = make_float2(1.f, 0.f);
  __syncwarp();
  const int col0 = (threadIdx.x >> 5) * 4;   // first column of this warp: the loop bound is warp-uniform
  for (int i = col0 + 1; i < PB; ++i) {
    float2 acc = make_float2(0.f, 0.f);
    if (i > col)
      for (int q = col + part; q < i; q += 8) acc = cfma(a[tri(jb + i, jb + q)], li[tri(jb + q, jb + col)], acc);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (part == 0 && i > col) li[tri(jb + i, jb + col)] = make_float2(-acc.x, -acc.y);
    __syncwarp();
  }
}

template <typename C>
__global__ void __launch_bounds__(256, 3) k_diag_mx(float2* pool, const FrontDev* fr, const int32_t* fids, int k,
                                                 DevStatus* st, float2* linv, uint8_t* piv, int sel) {
  __shared__ float2 a[T * (T + 1) / 2];
  __shared__ float2 li[T * (T + 1) / 2];   // L_kk^{-1}, packed lower
  // the precision-C pivot block, and between the two block factorizations the
  // 32 x 33 FP32 work block X21 (later L21 N11): the same bytes
  constexpr int kApBytes = sizeof(C) * (PB * (PB + 1) / 2), kX21Bytes = sizeof(float2) * PB * (PB + 1);
  __shared__ __align__(16) unsigned char ap_raw[kApBytes > kX21Bytes ? kApBytes : kX21Bytes];
  C* ap = reinterpret_cast<C*>(ap_raw);
  float2 (*x21)[PB + 1] = reinterpret_cast<float2 (*)[PB + 1]>(ap_raw);
  __shared__ C w[2 * PB];         // unscaled pivot columns (two buffers)
  __shared__ float2 lcol[2 * PB];  // the scaled columns, FP32, for N (two buffers)
  __shared__ float2 d1inv[PB];   // D1^{-1}: (D1^{-1} x)_c = d1inv[c] x_c + g1[c] x_{q1[c]}
  // restricted Bunch-Kaufman (fronts that pivot): 2x2 column, permutation, 2x2
  // off-diagonals; in precision C, or FP64 (unused) for the double-float form,
  // which serves unpivoted fronts only
  constexpr bool kBK = !std::is_same<C, dfc>::value;
  using CB = typename std::conditional<kBK, C, double2>::type;
  __shared__ CB w1[PB];
  __shared__ float2 g1[PB];
  __shared__ int q1[PB];
  __shared__ int perm[T];
  __shared__ CB dsup[T];
  __shared__ int cnt[2];
  const int f = fids[blockIdx.x];
  const FrontDev F = fr[f];
  // sel 1: separator fronts of the auxiliary matrix only, 2: domain fronts only
  if ((sel == 1 && F.kind != 1) || (sel == 2 && F.kind == 1)) return;
  const bool pv = kBK && piv != nullptr && F.piv != 0;
  float2* base = pool + F.off + (int64_t)(k * T) * F.ld + k * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int i = idx / T, c = idx % T;
    if (c <= i) a[tri(i, c)] = base[(int64_t)i * F.ld + c];
  }
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  if (pv) factor_pivot32_any_bk<C, CB>(a, 0, ap, w, w1, perm, dsup, cnt);
  else factor_pivot32<C>(a, 0, ap, w, lcol, li);
  // D1^{-1} (from the precision-C factor while ap still holds it) and N11
  if (threadIdx.x < PB) {
    const int c = threadIdx.x;
    const bool first = pv && c + 1 < PB && (dsup[c].x != 0 || dsup[c].y != 0);
    const bool second = pv && !first && c > 0 && (dsup[c - 1].x != 0 || dsup[c - 1].y != 0);
    if (!first && !second) {
      d1inv[c] = cconv<float2>(crcp(ap[tri(c, c)]));
      g1[c] = make_float2(0.f, 0.f);
      q1[c] = c;
    } else {
      // block inverse of [d0 b; b d1]
      const int p0 = first ? c : c - 1;
      const double2 d0 = cconv<double2>(ap[tri(p0, p0)]), dd = cconv<double2>(ap[tri(p0 + 1, p0 + 1)]);
      const double2 b = cconv<double2>(dsup[p0]);
      const double2 idet = cdiv(make_double2(1.0, 0.0), csub(cmul(d0, dd), cmul(b, b)));
      d1inv[c] = cconv<float2>(cmul(first ? dd : d0, idet));
      const double2 nb = cmul(b, idet);
      g1[c] = make_float2((float)-nb.x, (float)-nb.y);
      q1[c] = first ? c + 1 : c - 1;
    }
  }
  if (pv) inv_unit_lower32(a, 0, li);   // the unpivoted path formed N11 with the factor
  __syncthreads();   // ap (the precision-C block) is dead from here until pivot block 2
  {
    // X21 = A21 P1^T N11^T: x21[r][c] = sum_{q <= c} A21[r][perm q] N11[c][q];
    // the thread's four columns c = cg + 8 h advance together (four independent
    // chains), each summed in increasing q
    const int r = threadIdx.x >> 3, cg = threadIdx.x & 7;
    float2 acc[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) acc[h] = make_float2(0.f, 0.f);
    for (int q = 0; q < PB; ++q) {
      const float2 av = a[tri(PB + r, pv ? perm[q] : q)];
#pragma unroll
      for (int h = 0; h < 4; ++h)
        if (q <= cg + 8 * h) acc[h] = cfma(av, li[tri(cg + 8 * h, q)], acc[h]);
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) x21[r][cg + 8 * h] = acc[h];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < PB * PB; idx += blockDim.x) {
    const int rr = idx / PB, c = idx % PB;
    a[tri(PB + rr, c)] = cfma(x21[rr][q1[c]], g1[c], cmul(x21[rr][c], d1inv[c]));   // L21 = X21 D1^{-1}
  }
  __syncthreads();
  // A22 -= L21 X21^T (lower part): rows i0 + 8 k of column c, the four
  // chains advancing together, each in increasing q
  {
    static_assert(PB * PB == 4 * 256, "four A22 elements per thread");
    const int c = threadIdx.x % PB, i0 = threadIdx.x / PB;
    float2 acc[4];
#pragma unroll
    for (int k4 = 0; k4 < 4; ++k4) {
      const int i = i0 + 8 * k4;
      acc[k4] = c <= i ? a[tri(PB + i, PB + c)] : make_float2(0.f, 0.f);
    }
    for (int q = 0; q < PB; ++q) {
      const float2 xv = x21[c][q];
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4)
        if (c <= i0 + 8 * k4) acc[k4] = cfms(a[tri(PB + i0 + 8 * k4, q)], xv, acc[k4]);
    }
#pragma unroll
    for (int k4 = 0; k4 < 4; ++k4)
      if (c <= i0 + 8 * k4) a[tri(PB + i0 + 8 * k4, PB + c)] = acc[k4];
  }
  __syncthreads();
  if (pv) {
    factor_pivot32_any_bk<C, CB>(a, PB, ap, w, w1, perm + PB, dsup + PB, cnt);
    // rows of L21 follow the interchanges of the second pivot block
    for (int idx = threadIdx.x; idx < PB * PB; idx += blockDim.x) {
      const int rr = idx / PB, c = idx % PB;
      x21[rr][c] = a[tri(PB + rr, c)];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < PB * PB; idx += blockDim.x) {
      const int rr = idx / PB, c = idx % PB;
      a[tri(PB + rr, c)] = x21[perm[PB + rr]][c];
    }
    __syncthreads();
    if (threadIdx.x < PB) perm[PB + threadIdx.x] += PB;
  } else {
    factor_pivot32<C>(a, PB, ap, w, lcol, li);
  }
  // N22 (formed with the factor when unpivoted), then N21 = -N22 (L21 N11) through x21 = L21 N11
  if (pv) inv_unit_lower32(a, PB, li);
  {
    // x21 = L21 N11 (four column chains together, each in increasing q)
    const int r = threadIdx.x >> 3, cg = threadIdx.x & 7;
    float2 acc[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) acc[h] = make_float2(0.f, 0.f);
    for (int q = cg; q < PB; ++q) {
      const float2 av = a[tri(PB + r, q)];
#pragma unroll
      for (int h = 0; h < 4; ++h)
        if (q >= cg + 8 * h) acc[h] = cfma(av, li[tri(q, cg + 8 * h)], acc[h]);
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) x21[r][cg + 8 * h] = acc[h];
  }
  __syncthreads();
  {
    // N21 = -N22 x21
    const int r = threadIdx.x >> 3, cg = threadIdx.x & 7;
    float2 acc[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) acc[h] = make_float2(0.f, 0.f);
    for (int q = 0; q <= r; ++q) {
      const float2 lv = li[tri(PB + r, PB + q)];
#pragma unroll
      for (int h = 0; h < 4; ++h) acc[h] = cfma(lv, x21[q][cg + 8 * h], acc[h]);
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) li[tri(PB + r, cg + 8 * h)] = make_float2(-acc[h].x, -acc[h].y);
  }
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int i = idx / T, c = idx % T;
    if (c <= i) base[(int64_t)i * F.ld + c] = a[tri(i, c)];
  }
  if (pv) {
    __syncthreads();
    store_pivots<float2, CB>(base, F.ld, perm, dsup, piv + ((int64_t)F.tile_off + k) * T);
    if (threadIdx.x == 0 && (cnt[0] | cnt[1])) {
      atomicAdd(&st->n_swap, (unsigned long long)cnt[0]);
      atomicAdd(&st->n_2x2, (unsigned long long)cnt[1]);
    }
  }
  __syncthreads();
  float2* out = linv + ((int64_t)F.tile_off + k) * T * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int i = idx / T, c = idx % T;
    out[idx] = c <= i ? li[tri(i, c)] : make_float2(0.f, 0.f);
  }
  if (threadIdx.x < T) {
    const int r = k * T + threadIdx.x;
    if (r < F.ne) pivot_stats(a, dsup, pv, threadIdx.x, f, r, st);
  }
}

// mixed form panel: X = A_ik P_k^T L_kk^{-T} as a product with the stored
// inverse, L_ik = X D_k^{-1}; 4 x 4 register blocking like the trailing update
__global__ void __launch_bounds__(256) k_trsm_mx(float2* pool, const FrontDev* fr, const Task* tasks, int k,
                                                 DevStatus* st, const float2* linv, unsigned char* ws,
                                                 const uint8_t* piv) {
  constexpr int KC = 32;
  // A and B chunks; after the product the same storage holds X (64 x 65) when D has 2x2 blocks
  __shared__ float2 sraw[2 * KC * (T + 1)];
  float2 (*As)[T + 1] = reinterpret_cast<float2 (*)[T + 1]>(sraw);
  float2 (*Bs)[T + 1] = As + KC;
  float2 (*Xs)[T + 1] = As;
  __shared__ float2 rinv[T];
  __shared__ float2 rsq[T];      // unpivoted: a square root of 1 / d_p (image scaling D^(-1/2))
  __shared__ float2 g1[T];
  __shared__ int qc[T];
  __shared__ int perm[T];
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const bool pv = piv != nullptr && F.piv != 0;
  const int64_t ld = F.ld;
  float2* Aik = pool + F.off + (int64_t)(t.i * T) * ld + k * T;
  const float2* Dk = pool + F.off + (int64_t)(k * T) * ld + k * T;
  const float2* Li = linv + ((int64_t)F.tile_off + k) * T * T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  if (threadIdx.x < T) {
    const int p = threadIdx.x;
    if (pv) {
      float2 g0, gg;
      int q;
      dinv_col(Dk, ld, p, g0, gg, q);
      rinv[p] = g0;
      g1[p] = gg;
      qc[p] = q;
      perm[p] = piv[((int64_t)F.tile_off + k) * T + p];
    } else {
      rinv[p] = cdiv(make_float2(1.f, 0.f), Dk[(int64_t)p * (ld + 1)]);
      rsq[p] = csqrt_f(rinv[p]);
      perm[p] = p;
    }
  }
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
  for (int kc = 0; kc < T; kc += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < T * KC; idx += blockDim.x) {
      const int r = idx / KC, kk = idx % KC;
      As[kk][r] = Aik[(int64_t)r * ld + perm[kc + kk]];
      Bs[kk][r] = Li[r * T + kc + kk];   // Linv[p][q], p = r
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      float2 av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cfma(av[r], bv[c], acc[r][c]);
    }
  }
  __syncthreads();
  if (pv) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) Xs[ty + 16 * r][tx + 16 * c] = acc[r][c];
    __syncthreads();
  }
  // growth statistic in FP32 (the FP64 pipe is ~1/64 of FP32 on this part): max |l d|^2
  float mx = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int rr = ty + 16 * r, p = tx + 16 * c;
      const float2 x = acc[r][c];
      mx = fmaxf(mx, x.x * x.x + x.y * x.y);
      const float2 lv = pv ? cfma(Xs[rr][qc[p]], g1[p], cmul(x, rinv[p])) : cmul(x, rinv[p]);
      Aik[(int64_t)rr * ld + p] = lv;
      // unpivoted: M = X D^(-1/2) = L D^(1/2) serves as both operand images
      if (ws) write_images<float2>(ws, F, t.i - k - 1, rr * T + p, pv ? lv : cmul(x, rsq[p]), x, pv);
    }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f && isfinite(mx)) atomic_max_pos(&st->max_abs_l, sqrt((double)mx));
}

// mixed form panel on the tensor cores: X = A_ik P_k^T L_kk^{-T} as a 3xTF32
// tcgen05 product with the stored inverse (M = 128: real and imaginary rows
// of A_ik, N = 128: real and imaginary rows of L_kk^{-1}, K = 64 in two
// halves of 32, so that the 64 KB of operand images let three CTAs share an
// SM), the accumulator in TMEM; then L_ik = X D_k^{-1} and the operand
// images of the trailing update, as k_trsm_mx.  256 threads; warps 0-3 drain TMEM.
constexpr int kTrsmTcSmem = tc::kImage + 1024;   // A and B images of one K half (later X), 1024-aligned
__global__ void __launch_bounds__(256, 3) k_trsm_tc(float2* pool, const FrontDev* fr, const Task* tasks, int k,
                                                    DevStatus* st, const float2* linv, unsigned char* ws,
                                                    const uint8_t* piv) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* smem = tc_raw + ((1024u - (tc::smem_u32(tc_raw) & 1023u)) & 1023u);
  unsigned char* imgA = smem;
  unsigned char* imgB = smem + tc::kImage / 2;
  float2 (*Xs)[T + 1] = reinterpret_cast<float2 (*)[T + 1]>(smem);   // after the product
  __shared__ float2 rinv[T];
  __shared__ float2 rsq[T];      // unpivoted: a square root of 1 / d_p (image scaling D^(-1/2))
  __shared__ float2 g1[T];
  __shared__ int qc[T];
  __shared__ int perm[T];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int ok_s;
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const bool pv = piv != nullptr && F.piv != 0;
  const int64_t ld = F.ld;
  float2* Aik = pool + F.off + (int64_t)(t.i * T) * ld + k * T;
  const float2* Dk = pool + F.off + (int64_t)(k * T) * ld + k * T;
  const float2* Li = linv + ((int64_t)F.tile_off + k) * T * T;
  const int warp = threadIdx.x >> 5;
  const uint32_t b = tc::smem_u32(&bar);
  if (threadIdx.x == 0) {
    tc::mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x < T) {
    const int p = threadIdx.x;
    if (pv) {
      float2 g0, gg;
      int q;
      dinv_col(Dk, ld, p, g0, gg, q);
      rinv[p] = g0;
      g1[p] = gg;
      qc[p] = q;
      perm[p] = piv[((int64_t)F.tile_off + k) * T + p];
    } else {
      rinv[p] = cdiv(make_float2(1.f, 0.f), Dk[(int64_t)p * (ld + 1)]);
      rsq[p] = csqrt_f(rinv[p]);
      perm[p] = p;
    }
  }
  __syncthreads();
  const uint32_t tmem = tmem_slot;
  // operand images of K half h: A = A_ik P_k^T (rows r, K index q), B = L_kk^{-1} (rows p, K index q)
  if (threadIdx.x == 0) ok_s = 1;
  for (int h = 0; h < 2; ++h) {
    for (int idx = threadIdx.x; idx < T * (T / 2); idx += blockDim.x) {
      const int r = idx / (T / 2), q = idx % (T / 2);
      tc::put_a<1>(imgA, r, q, Aik[(int64_t)r * ld + perm[h * 32 + q]]);
      tc::put_b<1>(imgB, r, q, Li[r * T + h * 32 + q]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (threadIdx.x == 0) {
      if (ok_s) {
        tc::mma_tile<1>(tmem, tc::smem_u32(imgA), tc::smem_u32(imgB), h > 0);
        tc::mma_commit(b);
        ok_s = tc::mbar_wait(b, h) ? 1 : 0;
      }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  const bool ok = ok_s != 0;
  if (ok && warp < 4) tc::read_tile(tmem, [&](int r, int c, float2 v) { Xs[r][c] = v; });
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  if (!ok) {
    if (threadIdx.x == 0 && atomicCAS(&st->code, 0, 8) == 0) {
      st->front = t.f;
      st->row = k;
    }
    return;
  }
  // L_ik = X D_k^{-1}; growth statistic in FP32: max |l d|^2
  float mx = 0.f;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int rr = idx / T, p = idx % T;
    const float2 x = Xs[rr][p];
    mx = fmaxf(mx, x.x * x.x + x.y * x.y);
    const float2 lv = pv ? cfma(Xs[rr][qc[p]], g1[p], cmul(x, rinv[p])) : cmul(x, rinv[p]);
    Aik[(int64_t)rr * ld + p] = lv;
    // unpivoted: M = X D^(-1/2) = L D^(1/2) serves as both operand images
    if (ws) write_images<float2>(ws, F, t.i - k - 1, idx, pv ? lv : cmul(x, rsq[p]), x, pv);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f && isfinite(mx)) atomic_max_pos(&st->max_abs_l, sqrt((double)mx));
}

// ---------------------------------------------------------------------------
// panel: X = A_ik L_kk^{-T} (= L_ik D_k), then L_ik = X D_k^{-1}
// dynamic shared memory: Lt[64][64] (Lt[j][p] = L_kk[p][j]) + X[64][65] + d[64]
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(256) k_trsm(S* pool, const FrontDev* fr, const Task* tasks, int k,
                                              DevStatus* st, unsigned char* ws, const uint8_t* piv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* Lt = reinterpret_cast<S*>(smem_raw);  // Lt[j * T + p] = L_kk[p][j]
  S* X = Lt + T * T;                       // X[p * (T + 1) + r] = row r, column p
  S* rinv = X + T * (T + 1);               // 1 / d_p, or the first coefficient of D^{-1} (2x2 blocks)
  __shared__ S g1[T];                      // D^{-1} with 2x2 blocks: L_p = X_p rinv_p + X_q g1_p
  __shared__ int qc[T], perm[T];
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const bool pv = piv != nullptr && F.piv != 0;
  const S* Lkk = pool + F.off + (int64_t)(k * T) * F.ld + k * T;
  S* Aik = pool + F.off + (int64_t)(t.i * T) * F.ld + k * T;
  if (threadIdx.x < T) {
    const int p = threadIdx.x;
    if (pv) {
      S g0, gg;
      int q;
      dinv_col(Lkk, F.ld, p, g0, gg, q);
      rinv[p] = g0;
      g1[p] = gg;
      qc[p] = q;
      perm[p] = piv[((int64_t)F.tile_off + k) * T + p];
    } else {
      rinv[p] = cdiv(cmake<S>(1, 0), Lkk[(int64_t)p * F.ld + p]);
      perm[p] = p;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int p = idx / T, j = idx % T;  // coalesced reads along rows (A_ik P_k^T: permuted columns)
    Lt[j * T + p] = (j < p) ? Lkk[(int64_t)p * F.ld + j] : czero<S>();
    X[j * (T + 1) + p] = Aik[(int64_t)p * F.ld + perm[j]];
  }
  __syncthreads();
  // X L_kk^T = A_ik, column by column: X[:, p] -= X[:, j] L_kk[p][j] for p > j
  const int r = threadIdx.x & (T - 1), g = threadIdx.x >> 6;  // 4 column groups
  for (int j = 0; j < T - 1; ++j) {
    const S xj = X[j * (T + 1) + r];
    for (int p = j + 1 + ((g - j - 1) & 3); p < T; p += 4) X[p * (T + 1) + r] = cfms(xj, Lt[j * T + p], X[p * (T + 1) + r]);
    __syncthreads();
  }
  double mx = 0.0;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int rr = idx / T, p = idx % T;
    const S x = X[p * (T + 1) + rr];
    mx = fmax(mx, cabs2d(x));
    const S lv = pv ? cfma(X[qc[p] * (T + 1) + rr], g1[p], cmul(x, rinv[p])) : cmul(x, rinv[p]);
    Aik[(int64_t)rr * F.ld + p] = lv;
    if (ws) write_images<S>(ws, F, t.i - k - 1, idx, lv, x, true);
  }
  // block max of |L D| for the growth statistic
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0 && isfinite(mx)) atomic_max_pos(&st->max_abs_l, sqrt(mx));
}

// ---------------------------------------------------------------------------
// trailing update C_ij -= L_ik D_k L_jk^T, one 64 x 64 tile per CTA, 256
// threads with a 4 x 4 register block each (rows ty + 16 r, cols tx + 16 c)
// ---------------------------------------------------------------------------
template <typename S, int KC>
__global__ void __launch_bounds__(256) k_update(S* pool, const FrontDev* fr, const Task* tasks, int k) {
  __shared__ S As[KC][T + 1];
  __shared__ S Bs[KC][T + 1];
  __shared__ S dk[T];
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const int64_t ld = F.ld;
  const S* Li = pool + F.off + (int64_t)(t.i * T) * ld + k * T;
  const S* Lj = pool + F.off + (int64_t)(t.j * T) * ld + k * T;
  S* Cij = pool + F.off + (int64_t)(t.i * T) * ld + t.j * T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  // W_jk = L_jk D_k: D_k diagonal, or with 2x2 blocks (c, q) when the front pivots,
  // whose off-diagonal entry sits above the diagonal of the factored tile
  __shared__ S db[T];
  __shared__ int dq[T];
  if (threadIdx.x < T) {
    const int c = threadIdx.x;
    const S* Dk = pool + F.off + (int64_t)(k * T) * ld + k * T;
    dk[c] = Dk[(int64_t)c * (ld + 1)];
    int q = c;
    S b = czero<S>();
    if (F.piv) {
      const S up = c + 1 < T ? Dk[(int64_t)c * ld + c + 1] : czero<S>();
      const S lo = c > 0 ? Dk[(int64_t)(c - 1) * ld + c] : czero<S>();
      if (up.x != 0 || up.y != 0) { q = c + 1; b = up; }
      else if (lo.x != 0 || lo.y != 0) { q = c - 1; b = lo; }
    }
    dq[c] = q;
    db[c] = b;
  }
  S acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = czero<S>();
  for (int kc = 0; kc < T; kc += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < T * KC; idx += blockDim.x) {
      const int r = idx / KC, kk = idx % KC;
      As[kk][r] = Li[(int64_t)r * ld + kc + kk];
      const S w = cmul(Lj[(int64_t)r * ld + kc + kk], dk[kc + kk]);
      Bs[kk][r] = F.piv ? cfma(Lj[(int64_t)r * ld + dq[kc + kk]], db[kc + kk], w) : w;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      S a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cfma(a[r], b[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      S* p = Cij + (int64_t)(ty + 16 * r) * ld + tx + 16 * c;
      *p = csub(*p, acc[r][c]);
    }
}

// ---------------------------------------------------------------------------
// extend-add of one child's trailing block into its parent front.  Within one
// launch every destination entry is written by at most one thread (the map is
// injective), and the two children are added in two launches in a fixed
// order, so the assembly is deterministic without atomics.
// ---------------------------------------------------------------------------
// one warp per row of the child's trailing block (lower triangle), eight rows
// per CTA: each warp reads its row contiguously and adds it into the parent
// rows given by the map (grid.y covers the largest child of the level)
template <typename S>
__global__ void __launch_bounds__(256) k_extend_add(S* pool, const FrontDev* fr, const int32_t* nodes, int slot,
                                                    const int32_t* maps) {
  const FrontDev P = fr[nodes[blockIdx.x]];
  const int c = P.child[slot];
  if (c < 0 || P.kind == 1) return;   // separator fronts are assembled by k_assemble
  const FrontDev Cf = fr[c];
  const int a = blockIdx.y * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= Cf.nu) return;
  const int32_t* map = maps + P.map_off[slot];
  const S* src = pool + Cf.off + (int64_t)(Cf.ne_pad + a) * Cf.ld + Cf.ne_pad;
  S* dst = pool + P.off;
  const int ra = map[a];
  for (int b = lane; b <= a; b += 32) {
    const int rb = map[b];
    const S v = src[b];
    const int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
    S* p = dst + (int64_t)hi * P.ld + lo;
    *p = cadd(*p, v);
  }
}

// two consecutive complex entries, one 16-byte store for complex64
template <typename S>
__device__ __forceinline__ void store_pair(S* p, S a, S b) {
  p[0] = a;
  p[1] = b;
}
template <>
__device__ __forceinline__ void store_pair<float2>(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}

// Assembly of a separator front by pulling (Section II: the auxiliary
// matrix's blocks are sums of the children's Schur complements): entry (i, j)
// of the lower-triangular tiles is the sum over the children of their
// trailing-block entry at the inverse-mapped rows (child 0 first, then child 1,
// the order of the extend-add), 1 on the padding diagonal, 0 elsewhere.  The
// maps are increasing, so j <= i reads the children's lower triangles.  A warp
// per row, rows of 8 per CTA, grid-strided over the front.
template <typename S>
__global__ void __launch_bounds__(256) k_assemble(S* pool, const FrontDev* fr, const int32_t* nodes,
                                                  const int32_t* imaps) {
  const FrontDev P = fr[nodes[blockIdx.x]];
  if (P.kind != 1) return;
  const int lane = threadIdx.x & 31;
  for (int i = blockIdx.y * 8 + (threadIdx.x >> 5); i < P.ld; i += gridDim.y * 8) {
    const S* src[2] = {nullptr, nullptr};
    const int32_t* inv[2] = {nullptr, nullptr};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int c = P.child[s];
      if (c < 0) continue;
      const int32_t* m = imaps + P.imap_off[s];
      const int mi = m[i];
      if (mi < 0) continue;
      const FrontDev C = fr[c];
      inv[s] = m;
      src[s] = pool + C.off + (int64_t)(C.ne_pad + mi) * C.ld + C.ne_pad;
    }
    S* dst = pool + P.off + (int64_t)i * P.ld;
    const int jend = min(P.ld, (i / T + 1) * T);
    const bool pad = i >= P.ne && i < P.ne_pad;
    // two columns per lane (jend is a multiple of 64, rows and map offsets
    // start on multiples of 64 entries, so the pairs are aligned)
    for (int j = 2 * lane; j < jend; j += 64) {
      S v0 = czero<S>(), v1 = czero<S>();
      if (j <= i) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
          if (src[s]) {
            const int2 mj = *reinterpret_cast<const int2*>(inv[s] + j);
            if (mj.x >= 0) v0 = cadd(v0, src[s][mj.x]);
            if (j + 1 <= i && mj.y >= 0) v1 = cadd(v1, src[s][mj.y]);
          }
        if (pad && j == i) v0 = cmake<S>(1, 0);
        if (pad && j + 1 == i) v1 = cmake<S>(1, 0);
      }
      store_pair(dst + j, v0, v1);
    }
  }
}

// tile row t of front f: rows [64 t, 64 t + 64), columns [0, 64 (t + 1)), in
// 16-byte stores (front offsets and row strides are multiples of 64 entries)
__global__ void __launch_bounds__(256) k_zero_lower(unsigned char* pool, int elem, const FrontDev* fr,
                                                    const int2* tiles) {
  const int2 ft = tiles[blockIdx.x];
  const FrontDev F = fr[ft.x];
  const int64_t row_bytes = (int64_t)F.ld * elem;
  const int vec = (ft.y + 1) * T * elem / 16;
  unsigned char* base = pool + ((int64_t)F.off + (int64_t)ft.y * T * F.ld) * elem;
  for (int64_t idx = threadIdx.x; idx < (int64_t)T * vec; idx += blockDim.x) {
    const int r = (int)(idx / vec), v = (int)(idx % vec);
    reinterpret_cast<uint4*>(base + r * row_bytes)[v] = make_uint4(0u, 0u, 0u, 0u);
  }
}

template <typename S> constexpr int trsm_smem() { return (T * T + T * (T + 1) + T) * (int)sizeof(S); }

template <typename S>
void set_trsm_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_trsm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, trsm_smem<S>());
    done = true;
  }
}

}  // namespace

void launch_zero(void* p, size_t bytes, cudaStream_t s) {
  if (bytes) cudaMemsetAsync(p, 0, bytes, s);
}

void launch_zero_lower(void* pool, int elem, const FrontDev* fronts, const int2* tiles, int64_t n, cudaStream_t s) {
  if (n > 0) k_zero_lower<<<(unsigned)n, 256, 0, s>>>((unsigned char*)pool, elem, fronts, tiles);
}

void launch_assemble(int prec, void* pool, const FrontDev* fronts, const int32_t* node_ids, int n,
                     const int32_t* imaps, int max_ld, cudaStream_t s) {
  if (n <= 0 || max_ld <= 0) return;
  dim3 grid(n, std::min((max_ld + 7) / 8, 32768));
  if (prec == 0) k_assemble<double2><<<grid, 256, 0, s>>>((double2*)pool, fronts, node_ids, imaps);
  else k_assemble<float2><<<grid, 256, 0, s>>>((float2*)pool, fronts, node_ids, imaps);
}

void launch_leaf_init(int prec, void* pool, const FrontDev* fronts, const LeafDev* leaves, int n_leaves,
                      const int32_t* rowptr, const int32_t* colind, const double2* val, const int32_t* iperm,
                      const int32_t* b_row, const int32_t* b_local, const int8_t* b_sign, cudaStream_t s) {
  if (n_leaves <= 0) return;
  if (prec == 0)
    k_leaf_init<double2><<<n_leaves, 256, 0, s>>>((double2*)pool, fronts, leaves, rowptr, colind, val, iperm,
                                                  b_row, b_local, b_sign);
  else
    k_leaf_init<float2><<<n_leaves, 256, 0, s>>>((float2*)pool, fronts, leaves, rowptr, colind, val, iperm,
                                                 b_row, b_local, b_sign);
}

void launch_sparse_init(int prec, void* pool, const int64_t* dst, const int32_t* src, int64_t n, const double2* val,
                        cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (prec == 0) k_sparse_init<double2><<<grid, 256, 0, s>>>((double2*)pool, dst, src, n, val);
  else k_sparse_init<float2><<<grid, 256, 0, s>>>((float2*)pool, dst, src, n, val);
}

void launch_node_init(int prec, void* pool, const FrontDev* fronts, const int32_t* ids, int n, cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0) k_node_init<double2><<<n, 64, 0, s>>>((double2*)pool, fronts, ids);
  else k_node_init<float2><<<n, 64, 0, s>>>((float2*)pool, fronts, ids);
}

// FP64 form (the mixed form uses launch_diag_mx); prec and diag_fp64 must be 0
void launch_diag(int prec, int diag_fp64, void* pool, const FrontDev* fronts, const int32_t* fids, int n, int k,
                 DevStatus* st, cudaStream_t s, uint8_t* piv) {
  if (n <= 0 || prec != 0 || diag_fp64 != 0) return;
  k_diag<double2, double2><<<n, 256, 0, s>>>((double2*)pool, fronts, fids, k, st, piv);
}

void launch_diag_mx(int diag_fp64, void* pool, const FrontDev* fronts, const int32_t* fids, int n, int k,
                    DevStatus* st, void* linv, cudaStream_t s, uint8_t* piv) {
  if (n <= 0) return;
  // diag_fp64: 0 FP32 pivot blocks, 1 FP64, 2 by front: FP64 for the auxiliary
  // matrix's separator fronts, FP32 for domain fronts (two launches).  The
  // unpivoted FP64 blocks run in double-float arithmetic (about 48 bits, on
  // the FP32 pipes); restricted Bunch-Kaufman pivoting keeps true FP64.
  if ((diag_fp64 == 1 || diag_fp64 == 2) && piv)
    k_diag_mx<double2><<<n, 256, 0, s>>>((float2*)pool, fronts, fids, k, st, (float2*)linv, piv, diag_fp64 == 2 ? 1 : 0);
  if ((diag_fp64 == 1 || diag_fp64 == 2) && !piv)
    k_diag_mx<dfc><<<n, 256, 0, s>>>((float2*)pool, fronts, fids, k, st, (float2*)linv, piv, diag_fp64 == 2 ? 1 : 0);
  if (diag_fp64 == 0 || diag_fp64 == 2)
    k_diag_mx<float2><<<n, 256, 0, s>>>((float2*)pool, fronts, fids, k, st, (float2*)linv, piv, diag_fp64 == 2 ? 2 : 0);
}

void launch_diag_tile(int prec, void* pool, const FrontDev* front, const int32_t* fid, DevStatus* st, void* linv,
                      cudaStream_t s) {
  if (prec == 0) k_diag_mx<float2><<<1, 256, 0, s>>>((float2*)pool, front, fid, 0, st, (float2*)linv, nullptr, 0);
  if (prec == 1) k_diag_mx<dfc><<<1, 256, 0, s>>>((float2*)pool, front, fid, 0, st, (float2*)linv, nullptr, 0);
  if (prec == 2) k_diag_mx<double2><<<1, 256, 0, s>>>((float2*)pool, front, fid, 0, st, (float2*)linv, nullptr, 0);
}

void launch_trsm_mx(void* pool, const FrontDev* fronts, const Task* tasks, int n, int k, DevStatus* st,
                    const void* linv, unsigned char* ws, cudaStream_t s, const uint8_t* piv, int tensor) {
  if (n <= 0) return;
  if (tensor) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_trsm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsmTcSmem);
      attr = true;
    }
    k_trsm_tc<<<n, 256, kTrsmTcSmem, s>>>((float2*)pool, fronts, tasks, k, st, (const float2*)linv, ws, piv);
  } else {
    k_trsm_mx<<<n, 256, 0, s>>>((float2*)pool, fronts, tasks, k, st, (const float2*)linv, ws, piv);
  }
}

void launch_trsm(int prec, void* pool, const FrontDev* fronts, const Task* tasks, int n, int k, DevStatus* st,
                 cudaStream_t s, unsigned char* ws, const uint8_t* piv) {
  if (n <= 0 || prec != 0) return;   // FP64 form (the mixed form uses launch_trsm_mx)
  set_trsm_attr<double2>();
  k_trsm<double2><<<n, 256, trsm_smem<double2>(), s>>>((double2*)pool, fronts, tasks, k, st, ws, piv);
}

void launch_update(int prec, void* pool, const FrontDev* fronts, const Task* tasks, int n, int k, cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0) k_update<double2, 16><<<n, 256, 0, s>>>((double2*)pool, fronts, tasks, k);
  else k_update<float2, 32><<<n, 256, 0, s>>>((float2*)pool, fronts, tasks, k);
}

void launch_extend_add(int prec, void* pool, const FrontDev* fronts, const int32_t* node_ids, int n, int slot,
                       const int32_t* maps, int max_nu, cudaStream_t s) {
  if (n <= 0 || max_nu <= 0) return;
  dim3 grid(n, (max_nu + 7) / 8);
  if (prec == 0) k_extend_add<double2><<<grid, 256, 0, s>>>((double2*)pool, fronts, node_ids, slot, maps);
  else k_extend_add<float2><<<grid, 256, 0, s>>>((float2*)pool, fronts, node_ids, slot, maps);
}

}  // namespace ddk
