// Forward / backward substitution over the front tree (Section II: "the
// solution of all ... primal unknowns are recovered ... via many smaller size
// sparse forward backward substitutions", after the auxiliary solve), and the
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
  S* z = rpool + F.roff * nrhs;
  const int32_t* pm = perm + L.perm_off;
  for (int64_t e = threadIdx.x; e < (int64_t)F.ld * nrhs; e += blockDim.x) {
    const int r = (int)(e / nrhs), j = (int)(e % nrhs);
    z[e] = r < L.n ? cconv<S>(f[L.vec_off + pm[r] + j * ldf]) : czero<S>();
  }
}

template <typename S>
__global__ void k_rhs_node(S* rpool, const FrontDev* fr, const int32_t* ids, const int32_t* sep, const double2* g,
                           int64_t ldg, int nrhs) {
  const FrontDev F = fr[ids[blockIdx.x]];
  S* z = rpool + F.roff * nrhs;
  for (int64_t e = threadIdx.x; e < (int64_t)F.ld * nrhs; e += blockDim.x) {
    const int r = (int)(e / nrhs), j = (int)(e % nrhs);
    z[e] = (g != nullptr && r < F.ne) ? cconv<S>(g[sep[F.sep_off + r] + j * ldg]) : czero<S>();
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

// forward substitution + diagonal scaling of one front per CTA
template <typename S>
__global__ void __launch_bounds__(SOLVE_THREADS) k_forward(const S* pool, S* rpool, const FrontDev* fr,
                                                           const int32_t* fids, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* Lt = reinterpret_cast<S*>(smem_raw);  // [T][T+1] diagonal tile
  const FrontDev F = fr[fids[blockIdx.x]];
  const S* L = pool + F.off;
  S* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int j = 0; j < nrhs; ++j) {
    for (int t = 0; t < nte; ++t) {
      const int r0 = t * T;
      // rows of tile t: subtract the contributions of all earlier (final) rows
      for (int rr = warp; rr < T; rr += nw) {
        const int r = r0 + rr;
        S acc = czero<S>();
        for (int c = lane; c < r0; c += 32) acc = cfma(L[r * ld + c], z[(int64_t)c * nrhs + j], acc);
        acc = warp_sum(acc);
        if (lane == 0) z[(int64_t)r * nrhs + j] = csub(z[(int64_t)r * nrhs + j], acc);
      }
      for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
        const int rr = idx / T, c = idx % T;
        Lt[rr * (T + 1) + c] = L[(r0 + rr) * ld + r0 + c];
      }
      __syncthreads();
      // unit lower solve inside the tile: lane owns rows lane and lane + 32
      if (warp == 0) {
        S v0 = z[(int64_t)(r0 + lane) * nrhs + j];
        S v1 = z[(int64_t)(r0 + lane + 32) * nrhs + j];
        for (int c = 0; c < T; ++c) {
          const int owner = c & 31;
          S xc;
          const S src = (c < 32) ? v0 : v1;
          xc.x = __shfl_sync(0xffffffffu, src.x, owner);
          xc.y = __shfl_sync(0xffffffffu, src.y, owner);
          if (lane > c) v0 = cfms(Lt[lane * (T + 1) + c], xc, v0);
          if (lane + 32 > c) v1 = cfms(Lt[(lane + 32) * (T + 1) + c], xc, v1);
        }
        z[(int64_t)(r0 + lane) * nrhs + j] = v0;
        z[(int64_t)(r0 + lane + 32) * nrhs + j] = v1;
      }
      __syncthreads();
    }
    // update rows: z_u -= L_ue z_e
    for (int rr = warp; rr < F.nu; rr += nw) {
      const int r = F.ne_pad + rr;
      S acc = czero<S>();
      for (int c = lane; c < F.ne_pad; c += 32) acc = cfma(L[r * ld + c], z[(int64_t)c * nrhs + j], acc);
      acc = warp_sum(acc);
      if (lane == 0) z[(int64_t)r * nrhs + j] = csub(z[(int64_t)r * nrhs + j], acc);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < F.ne_pad; r += blockDim.x)
      z[(int64_t)r * nrhs + j] = cdiv(z[(int64_t)r * nrhs + j], L[r * (ld + 1)]);
    __syncthreads();
  }
}

// backward substitution of one front per CTA; node fronts publish their
// separator solution into lam (dual id order)
template <typename S>
__global__ void __launch_bounds__(SOLVE_THREADS) k_backward(const S* pool, S* rpool, const FrontDev* fr,
                                                            const int32_t* fids, int nrhs, const int32_t* upd,
                                                            const int32_t* sep, S* lam, int64_t ld_lam) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* Lt = reinterpret_cast<S*>(smem_raw);
  const FrontDev F = fr[fids[blockIdx.x]];
  const S* L = pool + F.off;
  S* z = rpool + F.roff * nrhs;
  const int64_t ld = F.ld;
  const int nte = F.ne_pad / T;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int j = 0; j < nrhs; ++j) {
    // known ancestor duals on the update rows
    for (int rr = threadIdx.x; rr < F.nu; rr += blockDim.x)
      z[(int64_t)(F.ne_pad + rr) * nrhs + j] = lam[upd[F.upd_off + rr] + j * ld_lam];
    __syncthreads();
    for (int c = threadIdx.x; c < F.ne_pad; c += blockDim.x) {
      S acc = czero<S>();
      for (int rr = 0; rr < F.nu; ++rr)
        acc = cfma(L[(F.ne_pad + rr) * ld + c], z[(int64_t)(F.ne_pad + rr) * nrhs + j], acc);
      z[(int64_t)c * nrhs + j] = csub(z[(int64_t)c * nrhs + j], acc);
    }
    __syncthreads();
    for (int t = nte - 1; t >= 0; --t) {
      const int r0 = t * T;
      for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
        const int rr = idx / T, c = idx % T;
        Lt[rr * (T + 1) + c] = L[(r0 + rr) * ld + r0 + c];
      }
      __syncthreads();
      if (warp == 0) {
        S v0 = z[(int64_t)(r0 + lane) * nrhs + j];
        S v1 = z[(int64_t)(r0 + lane + 32) * nrhs + j];
        for (int c = T - 1; c >= 0; --c) {
          const int owner = c & 31;
          S xc;
          const S src = (c < 32) ? v0 : v1;
          xc.x = __shfl_sync(0xffffffffu, src.x, owner);
          xc.y = __shfl_sync(0xffffffffu, src.y, owner);
          if (lane < c) v0 = cfms(Lt[c * (T + 1) + lane], xc, v0);
          if (lane + 32 < c) v1 = cfms(Lt[c * (T + 1) + lane + 32], xc, v1);
        }
        z[(int64_t)(r0 + lane) * nrhs + j] = v0;
        z[(int64_t)(r0 + lane + 32) * nrhs + j] = v1;
      }
      __syncthreads();
      for (int c = threadIdx.x; c < r0; c += blockDim.x) {
        S acc = czero<S>();
        for (int rr = 0; rr < T; ++rr) acc = cfma(L[(r0 + rr) * ld + c], z[(int64_t)(r0 + rr) * nrhs + j], acc);
        z[(int64_t)c * nrhs + j] = csub(z[(int64_t)c * nrhs + j], acc);
      }
      __syncthreads();
    }
    if (F.kind == 1)
      for (int r = threadIdx.x; r < F.ne; r += blockDim.x) lam[sep[F.sep_off + r] + j * ld_lam] = z[(int64_t)r * nrhs + j];
    __syncthreads();
  }
}

template <typename S>
__global__ void k_leaf_out(const S* rpool, const FrontDev* fr, const LeafDev* lv, const int32_t* perm, double2* u,
                           int64_t ldu, int nrhs, int accumulate) {
  const LeafDev L = lv[blockIdx.x];
  const FrontDev F = fr[L.front];
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

template <typename S> constexpr int tile_smem() { return T * (T + 1) * (int)sizeof(S); }

template <typename S>
void set_solve_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_forward<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_smem<S>());
    cudaFuncSetAttribute(k_backward<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_smem<S>());
    done = true;
  }
}

}  // namespace

void launch_rhs_leaf(int prec, void* rpool, const FrontDev* fronts, const LeafDev* leaves, int n_leaves,
                     const int32_t* perm, const double2* f, int64_t ldf, int nrhs, cudaStream_t s) {
  if (n_leaves <= 0) return;
  if (prec == 0) k_rhs_leaf<double2><<<n_leaves, 256, 0, s>>>((double2*)rpool, fronts, leaves, perm, f, ldf, nrhs);
  else k_rhs_leaf<float2><<<n_leaves, 256, 0, s>>>((float2*)rpool, fronts, leaves, perm, f, ldf, nrhs);
}

void launch_rhs_node(int prec, void* rpool, const FrontDev* fronts, const int32_t* ids, int n, const int32_t* sep,
                     const double2* g, int64_t ldg, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0) k_rhs_node<double2><<<n, 256, 0, s>>>((double2*)rpool, fronts, ids, sep, g, ldg, nrhs);
  else k_rhs_node<float2><<<n, 256, 0, s>>>((float2*)rpool, fronts, ids, sep, g, ldg, nrhs);
}

void launch_rhs_extend_add(int prec, void* rpool, const FrontDev* fronts, const int32_t* ids, int n, int slot,
                           const int32_t* maps, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0) k_rhs_extend_add<double2><<<n, 256, 0, s>>>((double2*)rpool, fronts, ids, slot, maps, nrhs);
  else k_rhs_extend_add<float2><<<n, 256, 0, s>>>((float2*)rpool, fronts, ids, slot, maps, nrhs);
}

void launch_forward(int prec, const void* pool, void* rpool, const FrontDev* fronts, const int32_t* fids, int n,
                    int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0) {
    set_solve_attr<double2>();
    k_forward<double2><<<n, SOLVE_THREADS, tile_smem<double2>(), s>>>((const double2*)pool, (double2*)rpool, fronts,
                                                                       fids, nrhs);
  } else {
    set_solve_attr<float2>();
    k_forward<float2><<<n, SOLVE_THREADS, tile_smem<float2>(), s>>>((const float2*)pool, (float2*)rpool, fronts,
                                                                     fids, nrhs);
  }
}

void launch_backward(int prec, const void* pool, void* rpool, const FrontDev* fronts, const int32_t* fids, int n,
                     int nrhs, const int32_t* upd, const int32_t* sep, void* lam_work, int64_t ld_lam,
                     cudaStream_t s) {
  if (n <= 0) return;
  if (prec == 0) {
    set_solve_attr<double2>();
    k_backward<double2><<<n, SOLVE_THREADS, tile_smem<double2>(), s>>>(
        (const double2*)pool, (double2*)rpool, fronts, fids, nrhs, upd, sep, (double2*)lam_work, ld_lam);
  } else {
    set_solve_attr<float2>();
    k_backward<float2><<<n, SOLVE_THREADS, tile_smem<float2>(), s>>>(
        (const float2*)pool, (float2*)rpool, fronts, fids, nrhs, upd, sep, (float2*)lam_work, ld_lam);
  }
}

void launch_leaf_out(int prec, const void* rpool, const FrontDev* fronts, const LeafDev* leaves, int n_leaves,
                     const int32_t* perm, double2* u, int64_t ldu, int nrhs, int accumulate, cudaStream_t s) {
  if (n_leaves <= 0) return;
  if (prec == 0)
    k_leaf_out<double2><<<n_leaves, 256, 0, s>>>((const double2*)rpool, fronts, leaves, perm, u, ldu, nrhs, accumulate);
  else
    k_leaf_out<float2><<<n_leaves, 256, 0, s>>>((const float2*)rpool, fronts, leaves, perm, u, ldu, nrhs, accumulate);
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

int launch_sumsq(const double2* x, int64_t n, double* out, int max_blocks, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  k_sumsq<<<blocks, 256, 0, s>>>(x, n, out);
  return blocks;
}

}  // namespace ddk
