// Tensor-core trailing update of the mixed form (Section II: the dense block
// updates of the domain and auxiliary-matrix factorizations run as level-3
// BLAS; here on the 5th-generation tensor cores).
//
// A task is a block of up to 2 x 2 tiles (128 x 128 complex) of
//   C -= sum_p L_ip D_p L_jp^T
// (row tiles i, i + 1, column tiles j, j + 1) over one or two panels
// p = k, k + 1 (K = 64 or 128), computed with tcgen05.mma kind::tf32,
// M = 128, N = 256, one MMA chain per row tile into its own TMEM accumulator:
//   * the complex product as one real GEMM per row tile: the A operand stacks
//     the real and imaginary rows of L (for each group of 16 rows, Re rows
//     then Im rows, so both parts of a row of C sit in the same TMEM
//     sub-partition), the B operand the real and imaginary rows of W = L D of
//     both column tiles; the accumulator holds [Re L; Im L] [Re W | Im W]^T
//     and the epilogue forms Re = Re L Re W - Im L Im W,
//     Im = Re L Im W + Im L Re W with lane shuffles;
//   * 3xTF32 split for FP32-class accuracy: X Y^T ~ Xh Yh^T + Xh Yl^T + Xl Yh^T;
//   * operands are the pre-split, 64B-swizzled K-major images written by the
//     panel kernel, streamed into shared memory by bulk asynchronous copies
//     (TMA engine) completing on mbarriers, one 64 KB stage per 16-wide K
//     atom (both row tiles' L and both column tiles' W), three in flight.
// Two row tiles share each B stage, so a stage carries 4 tile products for
// 64 KB where a one-row task carries 2 for 48 KB: the operand stream out of
// L2, which bounds this kernel, shrinks by a third per flop.  C is read and
// written once per task (a red.global.add per element).  Every wait is
// bounded: on timeout the CTA records DD_ERR_TIMEOUT, its roles stop, and it
// frees its TMEM and returns.
#include "dd_complex.cuh"
#include "dd_internal.h"
#include "dd_tc.cuh"

namespace ddk {

namespace {

using tc::bulk_g2s;
using tc::mbar_arrive;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::smem_u32;
using tc::tmem_ld32;

constexpr int T = DD_TILE;

// shared-memory matrix descriptor: K-major, 64B swizzle, 8-row groups 512 B apart
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)4 << 61;            // 64B swizzle
  return d;
}
constexpr uint32_t kIdesc256 = tc::idesc_tf32(256), kIdesc128 = tc::idesc_tf32(128);

// Task .pad bits: 0 / 1 column tile j / j + 1 is present (with bit 1 clear the
// MMAs use N = 128 and only tile j's operand is loaded), 2 / 3 panel k / k + 1
// contributes, 4 row tile i + 1 is present, 6..9 tile (i, j), (i, j + 1),
// (i + 1, j), (i + 1, j + 1) is stored (a lower-triangle tile of C).
constexpr int kPiece = DD_TC_ATOM;               // 128 rows x 16 K: 8 KB
constexpr int kStageA = 2 * kPiece;              // hi, lo of one row tile: 16 KB
constexpr int kStageB = 2 * 2 * kPiece;          // hi, lo x two column tiles: 32 KB
constexpr int kStage = 2 * kStageA + kStageB;    // 64 KB per K atom
constexpr int kStages = 3;
constexpr int kEpiWarps = 8;                     // two per TMEM sub-partition: one per row tile
constexpr int kStg = 16 * 33;                    // per epilogue warp: 16 rows x 32 complex, padded
constexpr int kSmemP = kStages * kStage + kEpiWarps * kStg * 8 + 512;   // + alignment slack
constexpr int kThreads = 64 + 32 * kEpiWarps;    // producer warp, MMA warp, epilogue warps
constexpr int kSlotCols = 256;                   // fp32 columns per row tile's accumulator

constexpr int kRing = 8;   // group ids handed from the producer to the MMA and epilogue roles

struct PipeBars {
  uint64_t full[kStages], empty[kStages], acc_full, acc_empty;
  uint64_t g_full[kRing], g_empty[kRing];
};

// Claims the group of ring slot `it` for a consumer role: lane 0 waits for the
// producer, the warp learns the group id (-1: no more groups) or a timeout.
__device__ __forceinline__ bool ring_take(uint32_t b_gfull0, uint32_t b_gempty0, const int* gring, int it, int& g) {
  const int slot = it % kRing, lane = threadIdx.x & 31;
  bool ok = true;
  g = -1;
  if (lane == 0) {
    ok = mbar_wait(b_gfull0 + 8 * slot, (it / kRing) & 1);
    if (ok) g = gring[slot];
  }
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  g = __shfl_sync(0xffffffffu, g, 0);
  if (lane == 0 && ok) mbar_arrive(b_gempty0 + 8 * slot);
  return ok;
}

// Epilogue (warps 2-9): warp w drains the accumulator of row tile i + s,
// s = (w - 2) / 4, TMEM lanes 32 (w % 4) .. + 31, i.e. rows 16 (w % 4) ..
// + 15 of that tile, lanes < 16 their real parts, lanes >= 16 their imaginary
// parts.  Per 32-column chunk of a column tile: both parts are combined across
// the half-warps with shuffles (lanes < 16 form columns 0-15, lanes >= 16
// columns 16-31), transposed through shared memory, and reduced into C
// row-contiguously (two rows of 256 B per warp access).
__device__ __forceinline__ void epilogue_role(float2* pool, const FrontDev* fr, const Task* tasks, const int2* groups,
                                              uint32_t tmem, float2* stage_c, uint32_t b_gfull0, uint32_t b_gempty0,
                                              const int* gring, uint32_t b_accf, uint32_t b_acce, volatile int& fail) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = warp & 3, slot = (warp - 2) >> 2;
  const bool im = lane >= 16;
  const int rl = lane & 15;                 // row within the warp's 16 rows
  float2* stg = stage_c + (warp - 2) * kStg;
  int tl = 0;
  for (int it = 0;; ++it) {
    int g;
    if (!ring_take(b_gfull0, b_gempty0, gring, it, g)) { fail = 1; break; }
    if (g < 0) break;
    bool stop = false;
    for (int q = groups[g].x; q < groups[g].x + groups[g].y; ++q, ++tl) {
      const Task t = tasks[q];
      const FrontDev F = fr[t.f];
      bool ok = !fail;
      if (ok && lane == 0) ok = mbar_wait(b_accf, tl & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) { fail = 1; stop = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      float2* crow = pool + F.off + (int64_t)((t.i + slot) * T + sub * 16) * F.ld;
#pragma unroll 1
      for (int ct = 0; ct < 2; ++ct) {
        if (!(t.pad & (1 << (6 + 2 * slot + ct)))) continue;
#pragma unroll 1
        for (int hf = 0; hf < 2; ++hf) {
          uint32_t xr[32], xi[32];   // this lane's row times [Re W] and [Im W], 32 columns
          const uint32_t ta = tmem + slot * kSlotCols + ((uint32_t)(sub * 32) << 16) + ct * 128 + hf * 32;
          tmem_ld32(ta, xr);
          tmem_ld32(ta + 64, xi);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          // lanes < 16 (Re L) keep columns 0-15 and send 16-31; lanes >= 16 (Im L) the reverse
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const float sr = __uint_as_float(im ? xr[c] : xr[16 + c]);
            const float si = __uint_as_float(im ? xi[c] : xi[16 + c]);
            const float pr = __shfl_xor_sync(0xffffffffu, sr, 16);
            const float pi = __shfl_xor_sync(0xffffffffu, si, 16);
            // own part of this lane's columns and the partner's
            const float orr = __uint_as_float(im ? xr[16 + c] : xr[c]);
            const float oii = __uint_as_float(im ? xi[16 + c] : xi[c]);
            // Re = ReL.ReW - ImL.ImW, Im = ReL.ImW + ImL.ReW
            const float re = im ? pr - oii : orr - pi;
            const float imv = im ? pi + orr : oii + pr;
            stg[rl * 33 + (im ? 16 : 0) + c] = make_float2(-re, -imv);
          }
          __syncwarp();
          const int rsub = lane >> 4, cpair = (lane & 15) * 2;
#pragma unroll 4
          for (int rr = 0; rr < 8; ++rr) {
            const int r = 2 * rr + rsub;
            const float2 v0 = stg[r * 33 + cpair], v1 = stg[r * 33 + cpair + 1];
            float* dst = reinterpret_cast<float*>(crow + (int64_t)r * F.ld + (t.j + ct) * T + hf * 32 + cpair);
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(v0.x), "f"(v0.y), "f"(v1.x),
                         "f"(v1.y)
                         : "memory");
          }
          __syncwarp();
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(b_acce);
    }
    if (stop) break;
  }
}

// Persistent, warp-specialised: warp 0 lane 0 claims task groups (runs of <= 8
// tasks of one row-tile pair, in list order, through an atomic counter) and
// streams the operand pieces of each task through a three-stage ring; warp 1
// lane 0 issues the MMAs (per row tile, into its 256-column TMEM
// accumulator); warps 2-9 drain the accumulators into C.
__global__ void __launch_bounds__(kThreads, 1) k_update_tc(float2* pool, const FrontDev* fr, const Task* tasks,
                                                           const int2* groups, int n_groups, int k,
                                                           const unsigned char* ws0, const unsigned char* ws1,
                                                           DevStatus* st, int* counter) {
  extern __shared__ __align__(512) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((512u - (smem_u32(smem_raw) & 511u)) & 511u);   // 64B-swizzle atoms: 512 B
  float2* stage_c = reinterpret_cast<float2*>(smem + kStages * kStage);
  __shared__ __align__(8) PipeBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int fail;
  __shared__ int gring[kRing];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_full0 = smem_u32(&bars.full[0]), b_empty0 = smem_u32(&bars.empty[0]);
  const uint32_t b_accf = smem_u32(&bars.acc_full), b_acce = smem_u32(&bars.acc_empty);
  const uint32_t b_gfull0 = smem_u32(&bars.g_full[0]), b_gempty0 = smem_u32(&bars.g_empty[0]);
  if (tid == 0) {
    fail = 0;
    for (int i = 0; i < kStages; ++i) {
      mbar_init(b_full0 + 8 * i, 1);
      mbar_init(b_empty0 + 8 * i, 1);
    }
    mbar_init(b_accf, 1);
    mbar_init(b_acce, kEpiWarps);   // one arrival per epilogue warp
    for (int i = 0; i < kRing; ++i) {
      mbar_init(b_gfull0 + 8 * i, 1);
      mbar_init(b_gempty0 + 8 * i, 1 + kEpiWarps);  // the MMA issuer and the epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * kSlotCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer ----------------
    int u = 0;
    for (int it = 0; !fail; ++it) {
      const int slot = it % kRing;
      if (!mbar_wait(b_gempty0 + 8 * slot, ((it / kRing) & 1) ^ 1)) { fail = 1; break; }
      const int g = atomicAdd(counter, 1);
      gring[slot] = g < n_groups ? g : -1;
      mbar_arrive(b_gfull0 + 8 * slot);
      if (g >= n_groups) break;
      for (int q = groups[g].x; q < groups[g].x + groups[g].y && !fail; ++q) {
        const Task t = tasks[q];
        const FrontDev F = fr[t.f];
        const int ncol = (t.pad & 2) ? 2 : 1;
        const int nrow = (t.pad & 16) ? 2 : 1;
        const int bytes = nrow * kStageA + ncol * 2 * kPiece;
        for (int pp = 0; pp < 2 && !fail; ++pp) {
          if (!(t.pad & (4 << pp))) continue;
          const int p = k + pp;
          const unsigned char* w = pp ? ws1 : ws0;
          const unsigned char* gA = w + F.ws_off + (int64_t)(t.i - p - 1) * DD_TC_ATILE;
          const unsigned char* gB = w + F.ws_boff + (int64_t)(t.j - p - 1) * DD_TC_BTILE;
          for (int a = 0; a < DD_TC_NATOM; ++a, ++u) {
            const int sidx = u % kStages;
            if (!mbar_wait(b_empty0 + 8 * sidx, ((u / kStages) & 1) ^ 1)) { fail = 1; break; }
            const uint32_t fb = b_full0 + 8 * sidx;
            unsigned char* stg = smem + sidx * kStage;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes) : "memory");
            for (int r = 0; r < nrow; ++r)
              for (int sp = 0; sp < 2; ++sp)
                bulk_g2s(smem_u32(stg + r * kStageA + sp * kPiece),
                         gA + (int64_t)r * DD_TC_ATILE + (sp * DD_TC_NATOM + a) * kPiece, kPiece, fb);
            for (int sp = 0; sp < 2; ++sp)
              for (int c = 0; c < ncol; ++c)
                bulk_g2s(smem_u32(stg + 2 * kStageA + sp * 2 * kPiece + c * kPiece),
                         gB + (int64_t)c * DD_TC_BTILE + (sp * DD_TC_NATOM + a) * kPiece, kPiece, fb);
          }
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int u = 0, tl = 0;
    const uint32_t s0 = smem_u32(smem);
    for (int it = 0; !fail; ++it) {
      const int slot = it % kRing;
      if (!mbar_wait(b_gfull0 + 8 * slot, (it / kRing) & 1)) { fail = 1; break; }
      const int g = gring[slot];
      mbar_arrive(b_gempty0 + 8 * slot);
      if (g < 0) break;
      for (int q = groups[g].x; q < groups[g].x + groups[g].y && !fail; ++q, ++tl) {
        const Task t = tasks[q];
        // the accumulators are free once the epilogue drained the previous task
        if (!mbar_wait(b_acce, (tl & 1) ^ 1)) { fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t idesc = (t.pad & 2) ? kIdesc256 : kIdesc128;
        const int nrow = (t.pad & 16) ? 2 : 1;
        uint32_t acc_on = 0;
        for (int pp = 0; pp < 2 && !fail; ++pp) {
          if (!(t.pad & (4 << pp))) continue;
          for (int a = 0; a < DD_TC_NATOM; ++a, ++u) {
            const int sidx = u % kStages;
            if (!mbar_wait(b_full0 + 8 * sidx, (u / kStages) & 1)) { fail = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = s0 + sidx * kStage, b0 = a0 + 2 * kStageA;
            for (int r = 0; r < nrow; ++r) {
              const uint32_t dacc = tmem + r * kSlotCols;
#pragma unroll
              for (int s8 = 0; s8 < DD_TC_KATOM / 8; ++s8)   // K = 8 per MMA: 32 B into the 64 B rows
#pragma unroll
                for (int sp = 0; sp < 3; ++sp) {   // split pairs (hi, hi), (hi, lo), (lo, hi)
                  const int as = sp == 2 ? 1 : 0, bs = sp == 1 ? 1 : 0;
                  const uint64_t ad = desc_sw64(a0 + r * kStageA + as * kPiece + s8 * 32);
                  const uint64_t bd = desc_sw64(b0 + bs * 2 * kPiece + s8 * 32);
                  tc::mma_tf32(dacc, ad, bd, idesc, (acc_on || s8 || sp) ? 1u : 0u);
                }
            }
            acc_on = 1;
            mma_commit(b_empty0 + 8 * sidx);   // the stage is free once these MMAs have read it
          }
        }
        if (fail) break;
        mma_commit(b_accf);
      }
    }
  } else if (warp >= 2) {
    epilogue_role(pool, fr, tasks, groups, tmem, stage_c, b_gfull0, b_gempty0, gring, b_accf, b_acce, fail);
  }
  __syncthreads();
  if (fail && tid == 0) {
    if (atomicCAS(&st->code, 0, 8) == 0) {
      st->front = -1;
      st->row = k;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kSlotCols));
}

}  // namespace

void launch_update_tc(void* pool, const FrontDev* fronts, const Task* tasks, const int2* groups, int n, int k,
                      const unsigned char* ws0, const unsigned char* ws1, DevStatus* st, cudaStream_t s,
                      int reserve_sms, int* counter) {
  if (n <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemP);
  }
  const int avail = sms - reserve_sms > 1 ? sms - reserve_sms : 1;
  const int grid = n < avail ? n : avail;
  k_update_tc<<<grid, kThreads, kSmemP, s>>>((float2*)pool, fronts, tasks, groups, n, k, ws0, ws1, st, counter);
}

}  // namespace ddk
