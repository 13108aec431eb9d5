// Forward / backward substitution over the front tree (Section II: after the
// auxiliary solve, the primal unknowns of every domain, or of a chosen subset,
// follow from many small independent substitutions), and the
// FP64 residual of the arrowhead system used by iterative refinement.
//
// Right-hand sides live in a per-front block z (ld rows x nrhs, row-major).
// Forward (leaves to root): z <- L^{-1} z over the eliminated rows, the
// update rows receive the Schur part of the right-hand side, which is
// extend-added into the parent; then z <- D^{-1} z on the eliminated rows.
// Backward (root to leaves): the update rows take the already known ancestor
// duals, and z <- L^{-T} (z - L_upd^T x_upd) over the eliminated rows.
#include "dd_complex.cuh"
#include "dd_internal.h"
#include "dd_pivot.cuh"
#include "dd_tc.cuh"

namespace ddk {

namespace {

constexpr int T = DD_TILE;
constexpr int SOLVE_THREADS = 256;

template <typename S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

template <typename S>
__global__ void k_rhs_leaf(S* rpool, const FrontDev* fr, const LeafDev* lv, const int32_t* perm, const double2* f,
                           int64_t ldf, int nrhs) {
  const LeafDev L = lv[blockIdx.x];
  const FrontDev F = fr[L.front];
  if (F.kind != 0) return;   // a sparse domain: its fronts load f by row id (k_rhs_node)
  S* z = rpool + F.roff * nrhs;
  const int32_t* pm = perm + L.perm_off;
  for (int64_t e = threadIdx.x; e < (int64_t)F.ld * nrhs; e += blockDim.x) {
    const int r = (int)(e / nrhs), j = (int)(e % nrhs);
    z[e] = r < L.n ? cconv<S>(f[L.vec_off + pm[r] + j * ldf]) : czero<S>();
  }
}

// the right-hand side of a separator front (its own rows: the dual load g,
// zero when g is NULL) or of a sparse-domain front (its own rows: the primal
// loads f, row id n_dual + stacked row); update rows start at zero
template <typename S>
__global__ void k_rhs_node(S* rpool, const FrontDev* fr, const int32_t* ids, const int32_t* sep, const double2* g,
                           int64_t ldg, const double2* f, int64_t ldf, int n_dual, int nrhs) {
  const FrontDev F = fr[ids[blockIdx.x]];
  if (F.kind == 0) return;
  S* z = rpool + F.roff * nrhs;
  for (int64_t e = threadIdx.x; e < (int64_t)F.ld * nrhs; e += blockDim.x) {
    const int r = (int)(e / nrhs), j = (int)(e % nrhs);
    S v = czero<S>();
    if (r < F.ne) {
      const int id = sep[F.sep_off + r];
      if (F.kind == 2) v = cconv<S>(f[(id - n_dual) + j * ldf]);
      else if (g != nullptr) v = cconv<S>(g[id + j * ldg]);
    }
    z[e] = v;
  }
}

template <typename S>
__global__ void k_rhs_extend_add(S* rpool, const FrontDev* fr, const int32_t* ids, int slot, const int32_t* maps,
                                 int nrhs) {
  const FrontDev P = fr[ids[blockIdx.x]];
  const int c = P.child[slot];
  if (c < 0) return;
  const FrontDev C = fr[c];
  const int32_t* map = maps + P.map_off[slot];
  const S* src = rpool + (C.roff + C.ne_pad) * nrhs;
  S* dst = rpool + P.roff * nrhs;
  for (int64_t e = threadIdx.x; e < (int64_t)C.nu * nrhs; e += blockDim.x) {
    const int a = (int)(e / nrhs), j = (int)(e % nrhs);
    S* p = dst + (int64_t)map[a] * nrhs + j;
    *p = cadd(*p, src[e]);
  }
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *flag >= epoch.  Bounded: after 2^24 polls (about a second) the
// wait gives up, records DD_ERR_TIMEOUT (8) in the status word and returns
// false; the caller then returns without publishing its own flag.
__device__ bool wait_ready(const int32_t* flag, int epoch, DevStatus* st, int front, int tile) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int it = 0;
    ok = 1;
    while (ld_acquire(flag) < epoch) {
      if (++it > (1 << 24)) {
        if (atomicCAS(&st->code, 0, 8) == 0) {
          st->front = front;
          st->row = tile;
        }
        ok = 0;
        break;
      }
      if (it > 4096) __nanosleep(64);   // spin first: most waits are short
    }
  }
  __syncthreads();
  const int r = ok;
  __syncthreads();
  return r != 0;
}

// packed lower triangle (with diagonal) of a 64 x 64 tile
__device__ __forceinline__ int tri(int r, int c) { return (r * (r + 1)) / 2 + c; }

template <typename S>
__device__ __forceinline__ S ldcg(const S* p);
template <>
__device__ __forceinline__ double2 ldcg<double2>(const double2* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ float2 ldcg<float2>(const float2* p) { return __ldcg(p); }

// Forward substitution, one CTA per (front, row tile i).  Rows of tile i
// accumulate L_ik z_k for every eliminated tile k < i as soon as tile k is
// final (its ready flag), then tile i is solved with the unit-lower diagonal
// block.  Tasks are ordered by tile index, so a CTA only waits on CTAs with a
// smaller block index.  Update tiles (i >= ne_pad / 64) only accumulate.
//
// Everything that does not depend on the tiles waited for is read before the
// waits -- the tile's diagonal block (L_ii^{-1} when given) into shared memory,
// the tile's own right-hand side and (FP32 form) the L block of the next tile
// into registers -- so after each wait only the 64 values of the finished tile
// are read, all issued before the products: the separator fronts' substitution
// is a chain of dependent tiles, and its step time is this latency.
template <typename S>
__global__ void __launch_bounds__(SOLVE_THREADS) k_forward(const S* pool, S* rpool, const FrontDev* fr,
                                                           const Task* tasks, int nrhs, int32_t* flags, int epoch,
                                                           DevStatus* st, const S* linv, const uint8_t* piv) {
  __shared__ S Lt[T * (T + 1) / 2];
  __shared__ S zi[T];
  __shared__ int perm[T];
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const S* L = pool + F.off;
  S* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int i = t.i, r0 = i * T;
  const int kmax = i < nte ? i : nte;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  int32_t* flg = flags + F.tile_off;
  constexpr int RW = T / (SOLVE_THREADS / 32);  // rows per warp
  constexpr bool kAhead = sizeof(S) == 8;
  const S* Li = (linv != nullptr && i < nte) ? linv + ((int64_t)F.tile_off + i) * T * T : nullptr;
  // restricted Bunch-Kaufman: the tile's right-hand side is permuted (P_i) before its solve
  const bool pv = piv != nullptr && F.piv != 0 && i < nte;
  if (pv && threadIdx.x < T) perm[threadIdx.x] = piv[((int64_t)F.tile_off + i) * T + threadIdx.x];
  if (i < nte) {
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
      const int rr = idx / T, c = idx % T;
      if (c <= rr) Lt[tri(rr, c)] = Li != nullptr ? Li[rr * T + c] : L[(r0 + rr) * ld + r0 + c];
    }
  }
  for (int j = 0; j < nrhs; ++j) {
    S acc[RW], own[RW], lnext[2][RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      acc[q] = czero<S>();
      own[q] = ldcg(z + (int64_t)(r0 + warp * RW + q) * nrhs + j);
    }
    if (kAhead && kmax > 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < RW; ++q) lnext[h][q] = L[(r0 + warp * RW + q) * ld + lane + 32 * h];
    }
    for (int k = 0; k < kmax; ++k) {
      if (j == 0 && !wait_ready(flg + k, epoch, st, t.f, k)) return;
      const int c0 = k * T;
      S zc[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) zc[h] = ldcg(z + (int64_t)(c0 + lane + 32 * h) * nrhs + j);
      if (kAhead) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int q = 0; q < RW; ++q) acc[q] = cfma(lnext[h][q], zc[h], acc[q]);
        if (k + 1 < kmax) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < RW; ++q) lnext[h][q] = L[(r0 + warp * RW + q) * ld + c0 + T + lane + 32 * h];
        }
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int q = 0; q < RW; ++q) acc[q] = cfma(L[(r0 + warp * RW + q) * ld + c0 + lane + 32 * h], zc[h], acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const S v = warp_sum(acc[q]);
      if (lane == 0) zi[warp * RW + q] = csub(own[q], v);
    }
    __syncthreads();
    if (pv) {
      S v;
      if (threadIdx.x < T) v = zi[perm[threadIdx.x]];
      __syncthreads();
      if (threadIdx.x < T) zi[threadIdx.x] = v;
      __syncthreads();
    }
    if (i < nte && Li != nullptr) {
      // z_i = L_ii^{-1} z_i: 4 lanes per row, 16 terms each
      const int row = threadIdx.x >> 2, part = threadIdx.x & 3;
      S acc = czero<S>();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int c = part * 16 + q;
        if (c <= row) acc = cfma(Lt[tri(row, c)], zi[c], acc);
      }
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      __syncthreads();
      if (part == 0) zi[row] = acc;
      __syncthreads();
    } else if (i < nte) {
      if (warp == 0) {
        S v0 = zi[lane], v1 = zi[lane + 32];
        for (int c = 0; c < T; ++c) {
          const S src = (c < 32) ? v0 : v1;
          S xc;
          xc.x = __shfl_sync(0xffffffffu, src.x, c & 31);
          xc.y = __shfl_sync(0xffffffffu, src.y, c & 31);
          if (lane > c) v0 = cfms(Lt[tri(lane, c)], xc, v0);
          if (lane + 32 > c) v1 = cfms(Lt[tri(lane + 32, c)], xc, v1);
        }
        zi[lane] = v0;
        zi[lane + 32] = v1;
      }
      __syncthreads();
    }
    if (threadIdx.x < T) z[(int64_t)(r0 + threadIdx.x) * nrhs + j] = zi[threadIdx.x];
    __syncthreads();
  }
  if (i < nte) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(flg + i, epoch);
    }
  }
}

// Update-row part of the backward substitution of separator fronts,
// w_j = L_uj^T x_u for every tile task of a launch, with the nu update rows of
// a task split over nsplit CTAs (grid n_tasks x nsplit): a front's first tile
// needs its w before the chain of dependent tiles can start, and one CTA per
// tile reads its rows at a small fraction of the bandwidth.  Partial sums go to
// out[((task * nsplit + split) * nrhs + column) * 64 + c]; the backward kernel
// adds them in split order, so the result does not depend on timing.
template <typename S>
__global__ void __launch_bounds__(SOLVE_THREADS) k_bwd_upd(const S* pool, const FrontDev* fr, const Task* tasks,
                                                           int nrhs, const int32_t* upd, const S* lam,
                                                           int64_t ld_lam, int nsplit, S* out) {
  constexpr int NG = SOLVE_THREADS / T;
  __shared__ S xu[SOLVE_THREADS];
  __shared__ S part[SOLVE_THREADS];
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const int split = blockIdx.y;
  const int rows = (F.nu + nsplit - 1) / nsplit;
  const int u_begin = min(F.nu, split * rows), u_end = min(F.nu, u_begin + rows);
  const int col = threadIdx.x % T, grp = threadIdx.x / T;
  const S* L = pool + F.off + (int64_t)F.ne_pad * F.ld + t.i * T + col;
  for (int jj = 0; jj < nrhs; ++jj) {
    S acc = czero<S>();
    for (int u0 = u_begin; u0 < u_end; u0 += SOLVE_THREADS) {
      const int nuc = min(SOLVE_THREADS, u_end - u0);
      __syncthreads();
      if (threadIdx.x < nuc) xu[threadIdx.x] = lam[upd[F.upd_off + u0 + threadIdx.x] + jj * ld_lam];
      __syncthreads();
#pragma unroll 8
      for (int u = grp; u < nuc; u += NG) acc = cfma(L[(int64_t)(u0 + u) * F.ld], xu[u], acc);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < T) {
      S sum = part[threadIdx.x];
#pragma unroll
      for (int g = 1; g < NG; ++g) sum = cadd(sum, part[g * T + threadIdx.x]);
      out[(((int64_t)blockIdx.x * nsplit + split) * nrhs + jj) * T + threadIdx.x] = sum;
    }
    __syncthreads();
  }
}

// Backward substitution, one CTA per (front, eliminated column tile j), tasks
// ordered by decreasing j.  y_j = D_j^{-1} z_j - L_uj^T x_u (update rows: the
// already solved ancestor duals) - sum_{i>j} L_ij^T x_i (as tiles i finish),
// then x_j = L_jj^{-T} y_j.  Node fronts publish x into lam.
//
// CHAIN (launches whose tiles all fit on the GPU at once: separator fronts,
// whose substitution is a chain of dependent tiles): everything independent
// of the awaited tiles -- the diagonal block or its inverse, the pivots, z_j,
// the destination indices and (FP32 form) the next L block -- is read before
// the waits, and each dependency's solution is loaded before its products.
// The other launches (leaves, bandwidth-bound) keep the registers low.
template <typename S, bool CHAIN>
__global__ void __launch_bounds__(SOLVE_THREADS) k_backward(const S* pool, S* rpool, const FrontDev* fr,
                                                            const Task* tasks, int nrhs, const int32_t* upd,
                                                            const int32_t* sep, S* lam, int64_t ld_lam,
                                                            int32_t* flags, int epoch, DevStatus* st, const S* linv,
                                                            const uint8_t* piv, const S* upart, int nsplit) {
  __shared__ S Lt[T * (T + 1) / 2];
  __shared__ S part[SOLVE_THREADS];
  __shared__ S yj[T];
  __shared__ S dv[T];            // the pivots d when Lt holds L_jj^{-1}
  constexpr int kUChunk = sizeof(S) == 8 ? 512 : 256;
  __shared__ S xu[kUChunk];      // gathered ancestor duals of the update rows; then each awaited tile's x_i (non-read-ahead form)
  __shared__ S g0s[T], g1s[T];   // D_j^{-1} coefficients when the tile pivoted
  __shared__ int qs[T], perm[T];
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const S* L = pool + F.off;
  S* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int j = t.i, c0 = j * T;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int col = threadIdx.x % T, grp = threadIdx.x / T;  // 64 columns x 4 row groups
  constexpr int NG = SOLVE_THREADS / T;
  constexpr int NQ = T / NG;   // rows of a tile per thread
  constexpr bool kAhead = CHAIN && sizeof(S) == 8;
  int32_t* flg = flags + F.tile_off;
  const S* Li = linv != nullptr ? linv + ((int64_t)F.tile_off + j) * T * T : nullptr;
  if (Li == nullptr || CHAIN) {
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
      const int rr = idx / T, c = idx % T;
      if (c <= rr) Lt[tri(rr, c)] = Li != nullptr ? Li[rr * T + c] : L[(c0 + rr) * ld + c0 + c];
    }
  }
  if (Li != nullptr && threadIdx.x < T) dv[threadIdx.x] = L[(c0 + threadIdx.x) * (ld + 1)];
  const bool pv = piv != nullptr && F.piv != 0;
  if (pv && threadIdx.x < T) {
    S g0, g1;
    int q;
    dinv_col(L + (int64_t)c0 * ld + c0, ld, threadIdx.x, g0, g1, q);
    g0s[threadIdx.x] = g0;
    g1s[threadIdx.x] = g1;
    qs[threadIdx.x] = q;
    perm[threadIdx.x] = piv[((int64_t)F.tile_off + j) * T + threadIdx.x];
  }
  // where x_j goes: its row of z and (node fronts) its dual index
  int xrow = 0, xdual = -1;
  if (threadIdx.x < T) {
    xrow = c0 + (pv ? perm[threadIdx.x] : threadIdx.x);
    if (F.kind != 0 && xrow < F.ne) xdual = sep[F.sep_off + xrow];
  }
  for (int jj = 0; jj < nrhs; ++jj) {
    S zc = czero<S>(), zq = czero<S>();
    if (CHAIN && threadIdx.x < T) {
      zc = ldcg(z + (int64_t)(c0 + threadIdx.x) * nrhs + jj);
      if (pv) zq = ldcg(z + (int64_t)(c0 + qs[threadIdx.x]) * nrhs + jj);
    }
    S lnext[NQ];
    if (kAhead && j + 1 < nte) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) lnext[q] = L[((nte - 1) * T + grp + NG * q) * ld + c0 + col];
    }
    // update rows: L_uj^T x_u, either summed from the partials of k_bwd_upd (in
    // split order) or formed here from the ancestor duals x_u, final since
    // earlier launches (plain loads), gathered into shared memory a chunk at a time
    S acc = czero<S>();
    if (CHAIN && upart != nullptr) {
      if (grp == 0)
        for (int q = 0; q < nsplit; ++q)
          acc = cadd(acc, upart[(((int64_t)blockIdx.x * nsplit + q) * nrhs + jj) * T + col]);
    }
    for (int u0 = 0; !(CHAIN && upart != nullptr) && u0 < F.nu; u0 += kUChunk) {
      const int nuc = min(kUChunk, F.nu - u0);
      __syncthreads();
#pragma unroll 2
      for (int e = threadIdx.x; e < nuc; e += SOLVE_THREADS) xu[e] = lam[upd[F.upd_off + u0 + e] + jj * ld_lam];
      __syncthreads();
      const S* Lu = L + (int64_t)(F.ne_pad + u0) * ld + c0 + col;
#pragma unroll 8
      for (int u = grp; u < nuc; u += NG) acc = cfma(Lu[(int64_t)u * ld], xu[u], acc);
    }
    for (int i = nte - 1; i > j; --i) {
      if (jj == 0 && !wait_ready(flg + i, epoch, st, t.f, i)) return;
      if (kAhead) {
        S xr[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) xr[q] = ldcg(z + (int64_t)(i * T + grp + NG * q) * nrhs + jj);
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc = cfma(lnext[q], xr[q], acc);
        if (i - 1 > j) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) lnext[q] = L[((i - 1) * T + grp + NG * q) * ld + c0 + col];
        }
      } else {
        // x_i through shared memory (one load per thread), so that the L loads
        // of the product are plain and all in flight together
        if (jj > 0) __syncthreads();
        if (threadIdx.x < T) xu[threadIdx.x] = ldcg(z + (int64_t)(i * T + threadIdx.x) * nrhs + jj);
        __syncthreads();
        const S* Li_ = L + (int64_t)(i * T + grp) * ld + c0 + col;
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc = cfma(Li_[(int64_t)q * NG * ld], xu[grp + NG * q], acc);
      }
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < T) {
      S sum = part[threadIdx.x];
#pragma unroll
      for (int g = 1; g < NG; ++g) sum = cadd(sum, part[g * T + threadIdx.x]);
      if (!CHAIN) {
        zc = ldcg(z + (int64_t)(c0 + threadIdx.x) * nrhs + jj);
        if (pv) zq = ldcg(z + (int64_t)(c0 + qs[threadIdx.x]) * nrhs + jj);
      }
      if (pv) {
        yj[threadIdx.x] = csub(cfma(zq, g1s[threadIdx.x], cmul(zc, g0s[threadIdx.x])), sum);
      } else {
        yj[threadIdx.x] = csub(cdiv(zc, Li != nullptr ? dv[threadIdx.x] : Lt[tri(threadIdx.x, threadIdx.x)]), sum);
      }
    }
    __syncthreads();
    if (Li != nullptr) {
      // x_j = L_jj^{-T} y_j: x[c] = sum_{r >= c} Linv[r][c] y[r], 4 lanes per column
      const int col2 = threadIdx.x >> 2, part = threadIdx.x & 3;
      S acc = czero<S>();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int r = part * 16 + q;
        if (r >= col2) acc = cfma(CHAIN ? Lt[tri(r, col2)] : Li[r * T + col2], yj[r], acc);
      }
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      __syncthreads();
      if (part == 0) yj[col2] = acc;
    } else if (warp == 0) {
      S v0 = yj[lane], v1 = yj[lane + 32];
      for (int c = T - 1; c >= 0; --c) {
        const S src = (c < 32) ? v0 : v1;
        S xc;
        xc.x = __shfl_sync(0xffffffffu, src.x, c & 31);
        xc.y = __shfl_sync(0xffffffffu, src.y, c & 31);
        if (lane < c) v0 = cfms(Lt[tri(c, lane)], xc, v0);
        if (lane + 32 < c) v1 = cfms(Lt[tri(c, lane + 32)], xc, v1);
      }
      yj[lane] = v0;
      yj[lane + 32] = v1;
    }
    __syncthreads();
    if (threadIdx.x < T) {   // x_j = P_j^T (L_jj^{-T} y_j)
      z[(int64_t)xrow * nrhs + jj] = yj[threadIdx.x];
      if (xdual >= 0) lam[xdual + jj * ld_lam] = yj[threadIdx.x];
    }
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flg + j, epoch);
  }
}

// ---------------------------------------------------------------------------
// Many right-hand sides (mixed form, up to 64 columns per pass): the same
// tile-parallel substitution, but every tile of L read from memory is applied
// to all columns at once as a 64 x 64 x nrhs product (4 x 4 register blocks),
// and the in-tile solves are products with the stored tile inverses.
// ---------------------------------------------------------------------------
constexpr int MR_KC = 32;

struct MrSmem {
  float2 As[MR_KC][T + 1];   // A chunk, k-major
  float2 Bs[MR_KC][T + 1];   // B chunk, k-major (columns = right-hand sides)
  float2 X[T][T + 1];        // tile block of right-hand sides
};

__device__ __forceinline__ void mr_fma(const MrSmem& sm, float2 (&acc)[4][4], int tx, int ty) {
#pragma unroll 4
  for (int kk = 0; kk < MR_KC; ++kk) {
    float2 a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = sm.As[kk][ty + 16 * r];
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = sm.Bs[kk][tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = cfma(a[r], b[c], acc[r][c]);
  }
}

// forward: Z_i = L_ii^{-1} (B_i - sum_k L_ik Z_k) for eliminated tiles; update tiles only subtract
__global__ void __launch_bounds__(256) k_forward_mr(const float2* pool, float2* rpool, const FrontDev* fr,
                                                    const Task* tasks, int nrhs, int32_t* flags, int epoch,
                                                    DevStatus* st, const float2* linv, const uint8_t* piv) {
  extern __shared__ __align__(16) unsigned char mr_raw[];
  MrSmem& sm = *reinterpret_cast<MrSmem*>(mr_raw);
  __shared__ int ip[T];   // inverse of the tile's pivot permutation (identity if it did not pivot)
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const float2* L = pool + F.off;
  float2* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int i = t.i, r0 = i * T;
  const int kmax = i < nte ? i : nte;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  int32_t* flg = flags + F.tile_off;
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
  for (int k = 0; k < kmax; ++k) {
    if (!wait_ready(flg + k, epoch, st, t.f, k)) return;
    for (int kc = 0; kc < T; kc += MR_KC) {
      for (int idx = threadIdx.x; idx < T * MR_KC; idx += blockDim.x) {
        const int rr = idx / MR_KC, kk = idx % MR_KC;
        sm.As[kk][rr] = L[(r0 + rr) * ld + k * T + kc + kk];
        const int col = rr;   // reuse the index: Bs[kk][col] = Z_k[kc + kk][col]
        sm.Bs[kk][col] = col < nrhs ? ldcg(z + (int64_t)(k * T + kc + kk) * nrhs + col) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      mr_fma(sm, acc, tx, ty);
      __syncthreads();
    }
  }
  // X = P_i (B_i - acc)
  if (threadIdx.x < T) {
    const bool pv = piv != nullptr && F.piv != 0 && i < nte;
    const int c = threadIdx.x;
    ip[pv ? piv[((int64_t)F.tile_off + i) * T + c] : c] = c;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int rr = ty + 16 * r, col = tx + 16 * c;
      const float2 b = col < nrhs ? ldcg(z + (int64_t)(r0 + rr) * nrhs + col) : make_float2(0.f, 0.f);
      sm.X[ip[rr]][col] = csub(b, acc[r][c]);
    }
  __syncthreads();
  if (i < nte) {
    // Z_i = Linv_ii X
    const float2* Li = linv + ((int64_t)F.tile_off + i) * T * T;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
    for (int kc = 0; kc < T; kc += MR_KC) {
      for (int idx = threadIdx.x; idx < T * MR_KC; idx += blockDim.x) {
        const int rr = idx / MR_KC, kk = idx % MR_KC;
        sm.As[kk][rr] = Li[rr * T + kc + kk];
        sm.Bs[kk][rr] = sm.X[kc + kk][rr];
      }
      __syncthreads();
      mr_fma(sm, acc, tx, ty);
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) sm.X[ty + 16 * r][tx + 16 * c] = acc[r][c];
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < T * nrhs; idx += blockDim.x) {
    const int rr = idx / nrhs, col = idx % nrhs;
    z[(int64_t)(r0 + rr) * nrhs + col] = sm.X[rr][col];
  }
  if (i < nte) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(flg + i, epoch);
    }
  }
}

// backward: X_j = L_jj^{-T} (D_j^{-1} Z_j - L_uj^T X_u - sum_{i>j} L_ij^T X_i)
__global__ void __launch_bounds__(256) k_backward_mr(const float2* pool, float2* rpool, const FrontDev* fr,
                                                     const Task* tasks, int nrhs, const int32_t* upd,
                                                     const int32_t* sep, float2* lam, int64_t ld_lam, int32_t* flags,
                                                     int epoch, DevStatus* st, const float2* linv,
                                                     const uint8_t* piv) {
  extern __shared__ __align__(16) unsigned char mr_raw[];
  MrSmem& sm = *reinterpret_cast<MrSmem*>(mr_raw);
  __shared__ float2 dinv[T];
  __shared__ float2 g1s[T];   // D_j^{-1} with 2x2 blocks: y_c = dinv_c z_c + g1_c z_q
  __shared__ int qs[T], perm[T];
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const float2* L = pool + F.off;
  float2* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int j = t.i, c0 = j * T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  int32_t* flg = flags + F.tile_off;
  const bool pv = piv != nullptr && F.piv != 0;
  if (threadIdx.x < T) {
    if (pv) {
      float2 g0, g1;
      int q;
      dinv_col(L + (int64_t)c0 * ld + c0, ld, threadIdx.x, g0, g1, q);
      dinv[threadIdx.x] = g0;
      g1s[threadIdx.x] = g1;
      qs[threadIdx.x] = q;
      perm[threadIdx.x] = piv[((int64_t)F.tile_off + j) * T + threadIdx.x];
    } else {
      dinv[threadIdx.x] = cdiv(make_float2(1.f, 0.f), L[(c0 + threadIdx.x) * (ld + 1)]);
      g1s[threadIdx.x] = make_float2(0.f, 0.f);
      qs[threadIdx.x] = threadIdx.x;
      perm[threadIdx.x] = threadIdx.x;
    }
  }
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
  // update rows: acc += L_uj^T X_u with X_u the known ancestor duals
  for (int u0 = 0; u0 < F.nu; u0 += MR_KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < T * MR_KC; idx += blockDim.x) {
      const int kk = idx / T, cc = idx % T;   // row kk of the chunk, column cc
      const int u = u0 + kk;
      sm.As[kk][cc] = u < F.nu ? L[(F.ne_pad + u) * ld + c0 + cc] : make_float2(0.f, 0.f);
      sm.Bs[kk][cc] = (u < F.nu && cc < nrhs) ? lam[upd[F.upd_off + u] + cc * ld_lam] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    mr_fma(sm, acc, tx, ty);
  }
  for (int i = nte - 1; i > j; --i) {
    if (!wait_ready(flg + i, epoch, st, t.f, i)) return;
    for (int kc = 0; kc < T; kc += MR_KC) {
      for (int idx = threadIdx.x; idx < T * MR_KC; idx += blockDim.x) {
        const int kk = idx / T, cc = idx % T;
        const int r = i * T + kc + kk;
        sm.As[kk][cc] = L[r * ld + c0 + cc];
        sm.Bs[kk][cc] = cc < nrhs ? ldcg(z + (int64_t)r * nrhs + cc) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      mr_fma(sm, acc, tx, ty);
      __syncthreads();
    }
  }
  __syncthreads();
  // Y = D^{-1} Z_j - acc  (rows = columns c of the tile)
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int cc = ty + 16 * r, col = tx + 16 * c;
      float2 y = make_float2(0.f, 0.f);
      if (col < nrhs) {
        y = cmul(ldcg(z + (int64_t)(c0 + cc) * nrhs + col), dinv[cc]);
        if (pv) y = cfma(ldcg(z + (int64_t)(c0 + qs[cc]) * nrhs + col), g1s[cc], y);
      }
      sm.X[cc][col] = csub(y, acc[r][c]);
    }
  __syncthreads();
  // X_j = Linv^T Y: acc[c][col] = sum_r Linv[r][c] Y[r][col]
  const float2* Li = linv + ((int64_t)F.tile_off + j) * T * T;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
  for (int kc = 0; kc < T; kc += MR_KC) {
    for (int idx = threadIdx.x; idx < T * MR_KC; idx += blockDim.x) {
      const int kk = idx / T, cc = idx % T;
      sm.As[kk][cc] = Li[(kc + kk) * T + cc];
      sm.Bs[kk][cc] = sm.X[kc + kk][cc];
    }
    __syncthreads();
    mr_fma(sm, acc, tx, ty);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) sm.X[ty + 16 * r][tx + 16 * c] = acc[r][c];
  __syncthreads();
  for (int idx = threadIdx.x; idx < T * nrhs; idx += blockDim.x) {
    const int cc = idx / nrhs, col = idx % nrhs;
    const float2 v = sm.X[cc][col];
    const int r = c0 + perm[cc];   // X_j = P_j^T (L_jj^{-T} Y)
    z[(int64_t)r * nrhs + col] = v;
    if (F.kind != 0 && r < F.ne) lam[sep[F.sep_off + r] + col * ld_lam] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flg + j, epoch);
  }
}

// ---------------------------------------------------------------------------
// Many right-hand sides on the tensor cores (mixed form, 4..64 columns): the
// same substitutions as k_forward_mr / k_backward_mr, every 64 x 64 x 64
// complex tile product a tcgen05 3xTF32 MMA (M = 128: real and imaginary rows
// of the left factor, N = 128: real and imaginary parts of the 64 columns,
// K = 64) accumulated in TMEM.  The CTA's 256 threads stage both operand
// images (tf32 hi / lo), thread 0 issues the MMAs, and all wait (bounded) on
// their completion; warps 0-3 drain TMEM into shared memory.
// ---------------------------------------------------------------------------
struct TcSolveSmem {
  unsigned char img[2 * tc::kImage];   // A and B operand images
  float2 X[T][T + 1];                  // the tile block of right-hand sides
};
constexpr int kTcSolveSmem = (int)sizeof(TcSolveSmem) + 1024;

struct TcCtx {
  unsigned char* imgA;
  unsigned char* imgB;
  uint32_t tmem, bar, phase;
  bool acc;   // the accumulator holds a product
};

// acc (+)= A B^T with A(r, q) = fa(r, q), B(c, q) = fb(c, q) (r, c, q < 64).
// A_QFAST / B_QFAST: the loop order that reads global memory contiguously.
// Returns false when the wait for the MMAs gave up (status recorded).
template <bool A_QFAST, bool B_QFAST, typename FA, typename FB>
__device__ bool tc_product(TcCtx& c, FA fa, FB fb, DevStatus* st, int front, int tile) {
  __shared__ int ok_s;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = A_QFAST ? idx / T : idx % T, q = A_QFAST ? idx % T : idx / T;
    tc::put_a(c.imgA, r, q, fa(r, q));
  }
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int n = B_QFAST ? idx / T : idx % T, q = B_QFAST ? idx % T : idx / T;
    tc::put_b(c.imgB, n, q, fb(n, q));
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (threadIdx.x == 0) {
    tc::mma_tile(c.tmem, tc::smem_u32(c.imgA), tc::smem_u32(c.imgB), c.acc);
    tc::mma_commit(c.bar);
    ok_s = tc::mbar_wait(c.bar, c.phase) ? 1 : 0;
    if (!ok_s && atomicCAS(&st->code, 0, 8) == 0) {
      st->front = front;
      st->row = tile;
    }
  }
  c.phase ^= 1;
  c.acc = true;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok_s != 0;
}

__device__ __forceinline__ void tc_setup(TcCtx& c, unsigned char* raw, uint64_t* bar, uint32_t* slot) {
  unsigned char* base = raw + ((1024u - (tc::smem_u32(raw) & 1023u)) & 1023u);
  c.imgA = base;
  c.imgB = base + tc::kImage;
  c.bar = tc::smem_u32(bar);
  c.phase = 0;
  c.acc = false;
  if (threadIdx.x == 0) {
    tc::mbar_init(c.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(slot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  c.tmem = *slot;
}

__device__ __forceinline__ void tc_release(const TcCtx& c) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"(128));
}

// forward: Z_i = L_ii^{-1} P_i (B_i - sum_k L_ik Z_k) for eliminated tiles; update tiles only subtract
__global__ void __launch_bounds__(256, 1) k_forward_tc(const float2* pool, float2* rpool, const FrontDev* fr,
                                                       const Task* tasks, int nrhs, int32_t* flags, int epoch,
                                                       DevStatus* st, const float2* linv, const uint8_t* piv) {
  extern __shared__ __align__(1024) unsigned char tcs_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  __shared__ int ip[T];
  TcCtx c;
  tc_setup(c, tcs_raw, &bar, &slot);
  float2 (*X)[T + 1] = reinterpret_cast<TcSolveSmem*>(c.imgA)->X;
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const float2* L = pool + F.off;
  float2* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int i = t.i, r0 = i * T;
  const int kmax = i < nte ? i : nte;
  int32_t* flg = flags + F.tile_off;
  bool ok = true;
  for (int k = 0; k < kmax && ok; ++k) {
    if (!wait_ready(flg + k, epoch, st, t.f, k)) {
      ok = false;
      break;
    }
    ok = tc_product<true, false>(
        c, [&](int r, int q) { return L[(int64_t)(r0 + r) * ld + k * T + q]; },
        [&](int n, int q) { return n < nrhs ? ldcg(z + (int64_t)(k * T + q) * nrhs + n) : make_float2(0.f, 0.f); }, st,
        t.f, k);
  }
  if (threadIdx.x < T) {
    const bool pv = piv != nullptr && F.piv != 0 && i < nte;
    const int cc = threadIdx.x;
    ip[pv ? piv[((int64_t)F.tile_off + i) * T + cc] : cc] = cc;
  }
  __syncthreads();
  // X = P_i (B_i - acc)
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int rr = idx / T, col = idx % T;
    X[ip[rr]][col] = col < nrhs ? ldcg(z + (int64_t)(r0 + rr) * nrhs + col) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (ok && c.acc && threadIdx.x < 128)
    tc::read_tile(c.tmem, [&](int r, int col, float2 v) { X[ip[r]][col] = csub(X[ip[r]][col], v); });
  __syncthreads();
  if (ok && i < nte) {
    // Z_i = Linv_ii X
    const float2* Li = linv + ((int64_t)F.tile_off + i) * T * T;
    c.acc = false;
    ok = tc_product<true, false>(c, [&](int r, int q) { return Li[r * T + q]; },
                                 [&](int n, int q) { return X[q][n]; }, st, t.f, i);
    if (ok && threadIdx.x < 128) tc::read_tile(c.tmem, [&](int r, int col, float2 v) { X[r][col] = v; });
    __syncthreads();
  }
  tc_release(c);
  if (!ok) return;
  for (int idx = threadIdx.x; idx < T * nrhs; idx += blockDim.x) {
    const int rr = idx / nrhs, col = idx % nrhs;
    z[(int64_t)(r0 + rr) * nrhs + col] = X[rr][col];
  }
  if (i < nte) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(flg + i, epoch);
    }
  }
}

// backward: X_j = P_j^T L_jj^{-T} (D_j^{-1} Z_j - L_uj^T X_u - sum_{i>j} L_ij^T X_i)
__global__ void __launch_bounds__(256, 1) k_backward_tc(const float2* pool, float2* rpool, const FrontDev* fr,
                                                        const Task* tasks, int nrhs, const int32_t* upd,
                                                        const int32_t* sep, float2* lam, int64_t ld_lam,
                                                        int32_t* flags, int epoch, DevStatus* st, const float2* linv,
                                                        const uint8_t* piv) {
  extern __shared__ __align__(1024) unsigned char tcs_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  __shared__ float2 dinv[T];
  __shared__ float2 g1s[T];   // D_j^{-1} with 2x2 blocks: y_c = dinv_c z_c + g1_c z_q
  __shared__ int qs[T], perm[T];
  TcCtx c;
  tc_setup(c, tcs_raw, &bar, &slot);
  float2 (*X)[T + 1] = reinterpret_cast<TcSolveSmem*>(c.imgA)->X;
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const float2* L = pool + F.off;
  float2* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int j = t.i, c0 = j * T;
  int32_t* flg = flags + F.tile_off;
  const bool pv = piv != nullptr && F.piv != 0;
  if (threadIdx.x < T) {
    if (pv) {
      float2 g0, g1;
      int q;
      dinv_col(L + (int64_t)c0 * ld + c0, ld, threadIdx.x, g0, g1, q);
      dinv[threadIdx.x] = g0;
      g1s[threadIdx.x] = g1;
      qs[threadIdx.x] = q;
      perm[threadIdx.x] = piv[((int64_t)F.tile_off + j) * T + threadIdx.x];
    } else {
      dinv[threadIdx.x] = cdiv(make_float2(1.f, 0.f), L[(c0 + threadIdx.x) * (ld + 1)]);
      g1s[threadIdx.x] = make_float2(0.f, 0.f);
      qs[threadIdx.x] = threadIdx.x;
      perm[threadIdx.x] = threadIdx.x;
    }
  }
  __syncthreads();
  bool ok = true;
  // update rows: acc += L_uj^T X_u with X_u the known ancestor values, 64 rows at a time
  for (int u0 = 0; u0 < F.nu && ok; u0 += T) {
    ok = tc_product<false, true>(
        c,
        [&](int r, int q) {
          return u0 + q < F.nu ? L[(int64_t)(F.ne_pad + u0 + q) * ld + c0 + r] : make_float2(0.f, 0.f);
        },
        [&](int n, int q) {
          return (u0 + q < F.nu && n < nrhs) ? lam[upd[F.upd_off + u0 + q] + n * ld_lam] : make_float2(0.f, 0.f);
        },
        st, t.f, j);
  }
  for (int i = nte - 1; i > j && ok; --i) {
    if (!wait_ready(flg + i, epoch, st, t.f, i)) {
      ok = false;
      break;
    }
    ok = tc_product<false, false>(
        c, [&](int r, int q) { return L[(int64_t)(i * T + q) * ld + c0 + r]; },
        [&](int n, int q) { return n < nrhs ? ldcg(z + (int64_t)(i * T + q) * nrhs + n) : make_float2(0.f, 0.f); }, st,
        t.f, i);
  }
  // Y = D^{-1} Z_j - acc
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int cc = idx / T, col = idx % T;
    float2 y = make_float2(0.f, 0.f);
    if (col < nrhs) {
      y = cmul(ldcg(z + (int64_t)(c0 + cc) * nrhs + col), dinv[cc]);
      if (pv) y = cfma(ldcg(z + (int64_t)(c0 + qs[cc]) * nrhs + col), g1s[cc], y);
    }
    X[cc][col] = y;
  }
  __syncthreads();
  if (ok && c.acc && threadIdx.x < 128)
    tc::read_tile(c.tmem, [&](int r, int col, float2 v) { X[r][col] = csub(X[r][col], v); });
  __syncthreads();
  if (ok) {
    // X_j = Linv^T Y: out[cc][col] = sum_r Linv[r][cc] Y[r][col]
    const float2* Li = linv + ((int64_t)F.tile_off + j) * T * T;
    c.acc = false;
    ok = tc_product<false, false>(c, [&](int r, int q) { return Li[q * T + r]; },
                                  [&](int n, int q) { return X[q][n]; }, st, t.f, j);
    if (ok && threadIdx.x < 128) tc::read_tile(c.tmem, [&](int r, int col, float2 v) { X[r][col] = v; });
    __syncthreads();
  }
  tc_release(c);
  if (!ok) return;
  for (int idx = threadIdx.x; idx < T * nrhs; idx += blockDim.x) {
    const int cc = idx / nrhs, col = idx % nrhs;
    const float2 v = X[cc][col];
    const int r = c0 + perm[cc];   // X_j = P_j^T (L_jj^{-T} Y)
    z[(int64_t)r * nrhs + col] = v;
    if (F.kind != 0 && r < F.ne) lam[sep[F.sep_off + r] + col * ld_lam] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flg + j, epoch);
  }
}

// diagnostic: a bounded wait on a flag that nothing sets
__global__ void k_wait_probe(const int32_t* flag, DevStatus* st) { wait_ready(flag, 1, st, -1, -1); }

template <typename S>
__global__ void k_leaf_out(const S* rpool, const FrontDev* fr, const LeafDev* lv, const int32_t* perm, double2* u,
                           int64_t ldu, int nrhs, int accumulate, const S* lam, int64_t ld_lam, int n_dual) {
  const LeafDev L = lv[blockIdx.x];
  const FrontDev F = fr[L.front];
  if (F.kind == 2) {
    // a sparse domain: the backward substitution left u_i in the row-id vector
    for (int64_t e = threadIdx.x; e < (int64_t)L.n * nrhs; e += blockDim.x) {
      const int r = (int)(e % L.n), j = (int)(e / L.n);
      double2* p = u + L.vec_off + r + j * ldu;
      const double2 v = cconv<double2>(lam[n_dual + L.vec_off + r + j * ld_lam]);
      *p = accumulate ? cadd(*p, v) : v;
    }
    return;
  }
  const S* z = rpool + F.roff * nrhs;
  const int32_t* pm = perm + L.perm_off;
  for (int64_t e = threadIdx.x; e < (int64_t)L.n * nrhs; e += blockDim.x) {
    const int r = (int)(e / nrhs), j = (int)(e % nrhs);
    double2* p = u + L.vec_off + pm[r] + j * ldu;
    const double2 v = cconv<double2>(z[e]);
    *p = accumulate ? cadd(*p, v) : v;
  }
}

template <typename S>
__global__ void k_lam_out(const S* w, int64_t ldw, int n_dual, int nrhs, double2* lam, int64_t ldl, int accumulate) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n_dual * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(e % n_dual), j = (int)(e / n_dual);
    const double2 v = cconv<double2>(w[d + j * ldw]);
    double2* p = lam + d + j * ldl;
    *p = accumulate ? cadd(*p, v) : v;
  }
}

// r_i = f_i - A_i u_i - B_i^T lambda in FP64 (row-sorted B entries per domain)
__global__ void k_residual(const LeafDev* lv, const int32_t* rowptr, const int32_t* colind, const double2* val,
                           const int32_t* bl_ptr, const int32_t* bl_dual, const int8_t* bl_sign, const double2* f,
                           int64_t ldf, const double2* u, int64_t ldu, const double2* lam, int64_t ldl, double2* r,
                           int64_t ldr, int nrhs) {
  const LeafDev L = lv[blockIdx.x];
  const int32_t* rp = rowptr + L.rowptr_off;
  const int32_t* ci = colind + L.csr_off;
  const double2* va = val + L.csr_off;
  const int32_t* bp = bl_ptr + L.rowptr_off;
  for (int64_t e = threadIdx.x; e < (int64_t)L.n * nrhs; e += blockDim.x) {
    const int row = (int)(e % L.n), j = (int)(e / L.n);
    double2 acc = f[L.vec_off + row + j * ldf];
    for (int q = rp[row]; q < rp[row + 1]; ++q) acc = cfms(va[q], u[L.vec_off + ci[q] + j * ldu], acc);
    for (int q = bp[row]; q < bp[row + 1]; ++q) {
      const double2 lv_ = lam[bl_dual[L.b_off + q] + j * ldl];
      const double sg = (double)bl_sign[L.b_off + q];
      acc.x -= sg * lv_.x;
      acc.y -= sg * lv_.y;
    }
    r[L.vec_off + row + j * ldr] = acc;
  }
}

// r_lambda = -B u (g = 0), one dual per thread in a fixed entry order
__global__ void k_dual_residual(int n_dual, const int32_t* bt_ptr, const int64_t* bt_row, const int8_t* bt_sign,
                                const double2* u, int64_t ldu, double2* rl, int64_t ldrl, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n_dual * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(e % n_dual), j = (int)(e / n_dual);
    double2 acc = make_double2(0.0, 0.0);
    for (int q = bt_ptr[d]; q < bt_ptr[d + 1]; ++q) {
      const double2 v = u[bt_row[q] + j * ldu];
      const double sg = (double)bt_sign[q];
      acc.x -= sg * v.x;
      acc.y -= sg * v.y;
    }
    rl[d + j * ldrl] = acc;
  }
}

// per-column sums of |x|^2: column j of x (n rows, ld n) reduced by gridDim.x blocks into out[j * gridDim.x + b]
__global__ void k_sumsq_cols(const double2* x, int64_t n, double* out) {
  __shared__ double sh[256];
  const double2* xc = x + (int64_t)blockIdx.y * n;
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s += xc[e].x * xc[e].x + xc[e].y * xc[e].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void k_sumsq(const double2* x, int64_t n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s += x[e].x * x[e].x + x[e].y * x[e].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

}  // namespace

void launch_rhs_leaf(int prec, void* rpool, const FrontDev* fronts, const LeafDev* leaves, int n_leaves,
                     const int32_t* perm, const double2* f, int64_t ldf, int nrhs, cudaStream_t s) {
  if (n_leaves <= 0) return;
  if (prec == 0) k_rhs_leaf<double2><<<n_leaves, 256, 0, s>>>((double2*)rpool, fronts, leaves, perm, f, ldf, nrhs);
  else k_rhs_leaf<float2><<<n_leaves, 256, 0, s>>>((float2*)rpool, fronts, leaves, perm, f, ldf, nrhs);
}

void launch_rhs_node(int prec, void* rpool, const FrontDev* fronts, const int32_t* ids, int n, const int32_t* sep,
                     const double2* g, int64_t ldg, const double2* f, int64_t ldf, int n_dual, int nrhs,
                     cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0)
    k_rhs_node<double2><<<n, 256, 0, s>>>((double2*)rpool, fronts, ids, sep, g, ldg, f, ldf, n_dual, nrhs);
  else
    k_rhs_node<float2><<<n, 256, 0, s>>>((float2*)rpool, fronts, ids, sep, g, ldg, f, ldf, n_dual, nrhs);
}

void launch_rhs_extend_add(int prec, void* rpool, const FrontDev* fronts, const int32_t* ids, int n, int slot,
                           const int32_t* maps, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0) k_rhs_extend_add<double2><<<n, 256, 0, s>>>((double2*)rpool, fronts, ids, slot, maps, nrhs);
  else k_rhs_extend_add<float2><<<n, 256, 0, s>>>((float2*)rpool, fronts, ids, slot, maps, nrhs);
}

// A substitution launch whose tiles all fit on the GPU at once is a chain of
// dependent tiles (separator fronts): it takes the read-ahead (CHAIN) form.
template <typename K>
bool fits_one_wave(K kernel, int n) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, SOLVE_THREADS, 0);
  return n <= sms * per_sm;
}

void launch_forward(int prec, const void* pool, void* rpool, const FrontDev* fronts, const Task* tasks, int n,
                    int nrhs, int32_t* flags, int epoch, DevStatus* st, cudaStream_t s, const void* linv,
                    const uint8_t* piv, int tensor) {
  if (n <= 0) return;
  if (prec == 1 && linv != nullptr && nrhs >= 4 && nrhs <= T && tensor) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSolveSmem);
      attr = true;
    }
    k_forward_tc<<<n, 256, kTcSolveSmem, s>>>((const float2*)pool, (float2*)rpool, fronts, tasks, nrhs, flags, epoch,
                                              st, (const float2*)linv, piv);
    return;
  }
  if (prec == 1 && linv != nullptr && nrhs >= 4 && nrhs <= T) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_forward_mr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MrSmem));
      attr = true;
    }
    k_forward_mr<<<n, 256, sizeof(MrSmem), s>>>((const float2*)pool, (float2*)rpool, fronts, tasks, nrhs, flags, epoch, st,
                                   (const float2*)linv, piv);
    return;
  }
  if (prec == 0)
    k_forward<double2><<<n, SOLVE_THREADS, 0, s>>>((const double2*)pool, (double2*)rpool, fronts, tasks, nrhs, flags,
                                                   epoch, st, nullptr, piv);
  else
    k_forward<float2><<<n, SOLVE_THREADS, 0, s>>>((const float2*)pool, (float2*)rpool, fronts, tasks, nrhs, flags,
                                                  epoch, st, (const float2*)linv, piv);
}

int launch_backward(int prec, const void* pool, void* rpool, const FrontDev* fronts, const Task* tasks, int n,
                    int nrhs, const int32_t* upd, const int32_t* sep, void* lam_work, int64_t ld_lam,
                    int32_t* flags, int epoch, DevStatus* st, cudaStream_t s, const void* linv,
                    const uint8_t* piv, void* upart, int nsplit, int tensor) {
  if (n <= 0) return 0;
  if (prec == 1 && linv != nullptr && nrhs >= 4 && nrhs <= T && tensor) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_backward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSolveSmem);
      attr = true;
    }
    k_backward_tc<<<n, 256, kTcSolveSmem, s>>>((const float2*)pool, (float2*)rpool, fronts, tasks, nrhs, upd, sep,
                                               (float2*)lam_work, ld_lam, flags, epoch, st, (const float2*)linv, piv);
    return 1;
  }
  if (prec == 1 && linv != nullptr && nrhs >= 4 && nrhs <= T) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_backward_mr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MrSmem));
      attr = true;
    }
    k_backward_mr<<<n, 256, sizeof(MrSmem), s>>>((const float2*)pool, (float2*)rpool, fronts, tasks, nrhs, upd, sep,
                                    (float2*)lam_work, ld_lam, flags, epoch, st, (const float2*)linv, piv);
    return 1;
  }
  const bool chain = prec == 0 ? fits_one_wave(k_backward<double2, true>, n) : fits_one_wave(k_backward<float2, true>, n);
  // the split update-row product serves the chain form only
  if (!chain || upart == nullptr || nsplit < 1) {
    upart = nullptr;
    nsplit = 0;
  }
  if (prec == 0) {
    const double2* up = (const double2*)upart;
    if (upart)
      k_bwd_upd<double2><<<dim3(n, nsplit), SOLVE_THREADS, 0, s>>>((const double2*)pool, fronts, tasks, nrhs, upd,
                                                                   (const double2*)lam_work, ld_lam, nsplit,
                                                                   (double2*)upart);
    if (chain)
      k_backward<double2, true><<<n, SOLVE_THREADS, 0, s>>>((const double2*)pool, (double2*)rpool, fronts, tasks, nrhs,
                                                           upd, sep, (double2*)lam_work, ld_lam, flags, epoch, st,
                                                           nullptr, piv, up, nsplit);
    else
      k_backward<double2, false><<<n, SOLVE_THREADS, 0, s>>>((const double2*)pool, (double2*)rpool, fronts, tasks,
                                                            nrhs, upd, sep, (double2*)lam_work, ld_lam, flags, epoch,
                                                            st, nullptr, piv, nullptr, 0);
  } else {
    const float2* up = (const float2*)upart;
    if (upart)
      k_bwd_upd<float2><<<dim3(n, nsplit), SOLVE_THREADS, 0, s>>>((const float2*)pool, fronts, tasks, nrhs, upd,
                                                                  (const float2*)lam_work, ld_lam, nsplit,
                                                                  (float2*)upart);
    if (chain)
      k_backward<float2, true><<<n, SOLVE_THREADS, 0, s>>>((const float2*)pool, (float2*)rpool, fronts, tasks, nrhs,
                                                          upd, sep, (float2*)lam_work, ld_lam, flags, epoch, st,
                                                          (const float2*)linv, piv, up, nsplit);
    else
      k_backward<float2, false><<<n, SOLVE_THREADS, 0, s>>>((const float2*)pool, (float2*)rpool, fronts, tasks, nrhs,
                                                           upd, sep, (float2*)lam_work, ld_lam, flags, epoch, st,
                                                           (const float2*)linv, piv, nullptr, 0);
  }
  return upart ? 2 : 1;
}

void launch_leaf_out(int prec, const void* rpool, const FrontDev* fronts, const LeafDev* leaves, int n_leaves,
                     const int32_t* perm, double2* u, int64_t ldu, int nrhs, int accumulate, cudaStream_t s,
                     const void* lam, int64_t ld_lam, int n_dual) {
  if (n_leaves <= 0) return;
  if (prec == 0)
    k_leaf_out<double2><<<n_leaves, 256, 0, s>>>((const double2*)rpool, fronts, leaves, perm, u, ldu, nrhs, accumulate,
                                                 (const double2*)lam, ld_lam, n_dual);
  else
    k_leaf_out<float2><<<n_leaves, 256, 0, s>>>((const float2*)rpool, fronts, leaves, perm, u, ldu, nrhs, accumulate,
                                                (const float2*)lam, ld_lam, n_dual);
}

void launch_lam_out(int prec, const void* lam_work, int64_t ld_work, int n_dual, int nrhs, double2* lam, int64_t ldl,
                    int accumulate, cudaStream_t s) {
  if (n_dual <= 0) return;
  const int blocks = (int)((((int64_t)n_dual * nrhs) + 255) / 256 < 4096 ? (((int64_t)n_dual * nrhs) + 255) / 256 : 4096);
  if (prec == 0)
    k_lam_out<double2><<<blocks, 256, 0, s>>>((const double2*)lam_work, ld_work, n_dual, nrhs, lam, ldl, accumulate);
  else
    k_lam_out<float2><<<blocks, 256, 0, s>>>((const float2*)lam_work, ld_work, n_dual, nrhs, lam, ldl, accumulate);
}

void launch_residual(const LeafDev* leaves, int n_leaves, const int32_t* rowptr, const int32_t* colind,
                     const double2* val, const int32_t* bl_ptr, const int32_t* bl_dual, const int8_t* bl_sign,
                     const double2* f, int64_t ldf, const double2* u, int64_t ldu, const double2* lam, int64_t ldl,
                     double2* r, int64_t ldr, int nrhs, cudaStream_t s) {
  if (n_leaves <= 0) return;
  k_residual<<<n_leaves, 256, 0, s>>>(leaves, rowptr, colind, val, bl_ptr, bl_dual, bl_sign, f, ldf, u, ldu, lam, ldl,
                                      r, ldr, nrhs);
}

void launch_dual_residual(int n_dual, const int32_t* bt_ptr, const int64_t* bt_row, const int8_t* bt_sign,
                          const double2* u, int64_t ldu, double2* rl, int64_t ldrl, int nrhs, cudaStream_t s) {
  if (n_dual <= 0) return;
  const int64_t work = (int64_t)n_dual * nrhs;
  const int blocks = (int)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
  k_dual_residual<<<blocks, 256, 0, s>>>(n_dual, bt_ptr, bt_row, bt_sign, u, ldu, rl, ldrl, nrhs);
}

void launch_wait_probe(const int32_t* flag, DevStatus* st, cudaStream_t s) { k_wait_probe<<<1, 32, 0, s>>>(flag, st); }

void launch_sumsq_cols(const double2* x, int64_t n, int ncols, int blocks, double* out, cudaStream_t s) {
  if (ncols <= 0) return;
  k_sumsq_cols<<<dim3(blocks, ncols), 256, 0, s>>>(x, n, out);
}

int launch_sumsq(const double2* x, int64_t n, double* out, int max_blocks, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  k_sumsq<<<blocks, 256, 0, s>>>(x, n, out);
  return blocks;
}

}  // namespace ddk
