// Tensor-core trailing update of the mixed form (Section II: the dense block
// updates of the domain and auxiliary-matrix factorizations run as level-3
// BLAS; here on the 5th-generation tensor cores).
//
// A task is a 64 x 128 complex block of  C -= sum_p L_ip D_p L_jp^T  (row tile
// i, column tiles j and j + 1) over one or two panels p = k, k + 1 (K = 64 or
// 128), computed with tcgen05.mma kind::tf32, M = 128, N = 256:
//   * the complex product as one real GEMM: the A operand stacks the real and
//     imaginary rows of L (for each group of 16 rows, Re rows then Im rows, so
//     both parts of a row of C sit in the same TMEM sub-partition), the B
//     operand the real and imaginary rows of W = L D of both column tiles in
//     the same layout; the accumulator holds [Re L; Im L] [Re W | Im W]^T and
//     the epilogue forms Re = Re L Re W - Im L Im W, Im = Re L Im W + Im L Re W
//     with lane shuffles.  For unpivoted fronts both operands are one image of
//     M = L D^(1/2) (L_i D L_j^T = M_i M_j^T), so the panel writes half the
//     image bytes;
//   * 3xTF32 split for FP32-class accuracy: X Y^T ~ Xh Yh^T + Xh Yl^T + Xl Yh^T;
//   * operands are the pre-split, 128B-swizzled K-major images written by the
//     panel kernel, streamed into shared memory by bulk asynchronous copies
//     (TMA engine) completing on mbarriers, one 96 KB stage per 32-wide K atom;
//     the accumulator lives in TMEM (two of 128 lanes x 256 fp32 columns).
// C is read and written once per task, so pairing two panels per task halves
// the trailing-matrix traffic.  Every wait is bounded: on timeout the CTA
// records DD_ERR_TIMEOUT, its roles stop, and it frees its TMEM and returns.
#include "dd_complex.cuh"
#include "dd_internal.h"

namespace ddk {

namespace {

constexpr int T = DD_TILE;
constexpr int kWaitPolls = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128B swizzle
  return d;
}

// instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = n
constexpr uint32_t idesc_tf32(uint32_t n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
constexpr uint32_t kIdesc256 = idesc_tf32(256), kIdesc128 = idesc_tf32(128);

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (int it = 0; it < kWaitPolls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
}

// Persistent, warp-specialised: warp 0 lane 0 claims task groups (runs of <= 8
// tasks of one row tile, in list order, through an atomic counter) and streams
// the operand pieces of each task through a two-stage ring; warp 1 lane 0
// issues the MMAs into one of two TMEM accumulators; warps 2-5 drain the other
// accumulator into C.  Task .pad: bit 0 / 1 store column tile j / j + 1 (with
// bit 1 clear the MMAs use N = 128 and only tile j's operand is loaded),
// bits 2..5 panel k .. k + 3 contributes (its images in ws.p[0 .. 3]).
constexpr int kStageA = 2 * DD_TC_ATOM;          // hi, lo pieces of the row tile: 32 KB
constexpr int kStageB = 2 * 2 * DD_TC_ATOM;      // hi, lo x two column tiles: 64 KB
constexpr int kStage = kStageA + kStageB;        // 96 KB per K atom
constexpr int kStages = 2;
constexpr int kStg = 16 * 33;                    // per epilogue warp: 16 rows x 32 complex, padded
constexpr int kSmemP = kStages * kStage + 4 * kStg * 8 + 1024;
constexpr int kAccCols = 256;                    // fp32 columns per accumulator; two accumulators

constexpr int kRing = 8;   // group ids handed from the producer to the MMA and epilogue roles

struct PipeBars {
  uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
  uint64_t g_full[kRing], g_empty[kRing];
};

__device__ __forceinline__ void mbar_init(uint32_t b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, int bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

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

// Epilogue (warps 2-5): warp s owns TMEM lanes 32 s .. 32 s + 31, i.e. rows
// 16 s .. 16 s + 15 of the row tile, lanes < 16 their real parts, lanes >= 16
// their imaginary parts.  Per 32-column chunk of a column tile: both parts are
// combined across the half-warps with shuffles (lanes < 16 form columns 0-15,
// lanes >= 16 columns 16-31), transposed through shared memory, and reduced
// into C row-contiguously (two rows of 256 B per warp access).
__device__ __forceinline__ void epilogue_role(float2* pool, const FrontDev* fr, const Task* tasks, const int2* groups,
                                              uint32_t tmem, float2* stage_c, uint32_t b_gfull0, uint32_t b_gempty0,
                                              const int* gring, uint32_t b_accf0, uint32_t b_acce0,
                                              volatile int& fail) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = warp & 3;
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
      const int ab = tl & 1;
      bool ok = !fail;
      if (ok && lane == 0) ok = mbar_wait(b_accf0 + 8 * ab, (tl >> 1) & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) { fail = 1; stop = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      float2* crow = pool + F.off + (int64_t)(t.i * T + sub * 16) * F.ld;
#pragma unroll 1
      for (int ct = 0; ct < 2; ++ct) {
        if (!(t.pad & (1 << ct))) continue;
#pragma unroll 1
        for (int hf = 0; hf < 2; ++hf) {
          // B rows in the A layout: per 16 rows of W, 16 real columns then 16
          // imaginary ones, so columns 64 hf .. 64 hf + 63 of the tile hold
          // W rows 32 hf .. 32 hf + 31 as (Re 0-15, Im 0-15, Re 16-31, Im 16-31)
          uint32_t u[32], v[32];
          const uint32_t ta = tmem + ab * kAccCols + ((uint32_t)(sub * 32) << 16) + ct * 128 + hf * 64;
          tmem_ld32(ta, u);
          tmem_ld32(ta + 32, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          uint32_t xr[32], xi[32];   // this lane's row times [Re W] and [Im W], 32 columns
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            xr[c] = u[c];
            xi[c] = u[16 + c];
            xr[16 + c] = v[c];
            xi[16 + c] = v[16 + c];
          }
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
      if (lane == 0) mbar_arrive(b_acce0 + 8 * ab);
    }
    if (stop) break;
  }
}

__global__ void __launch_bounds__(192, 1) k_update_tc(float2* pool, const FrontDev* fr, const Task* tasks,
                                                      const int2* groups, int n_groups, int k,
                                                      const PanelImages ws,
                                                      DevStatus* st, int* counter) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float2* stage_c = reinterpret_cast<float2*>(smem + kStages * kStage);
  __shared__ __align__(8) PipeBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int fail;
  __shared__ int gring[kRing];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_full0 = smem_u32(&bars.full[0]), b_empty0 = smem_u32(&bars.empty[0]);
  const uint32_t b_accf0 = smem_u32(&bars.acc_full[0]), b_acce0 = smem_u32(&bars.acc_empty[0]);
  const uint32_t b_gfull0 = smem_u32(&bars.g_full[0]), b_gempty0 = smem_u32(&bars.g_empty[0]);
  if (tid == 0) {
    fail = 0;
    for (int i = 0; i < kStages; ++i) {
      mbar_init(b_full0 + 8 * i, 1);
      mbar_init(b_empty0 + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_accf0 + 8 * i, 1);
      mbar_init(b_acce0 + 8 * i, 4);   // one arrival per epilogue warp
    }
    for (int i = 0; i < kRing; ++i) {
      mbar_init(b_gfull0 + 8 * i, 1);
      mbar_init(b_gempty0 + 8 * i, 5);  // the MMA issuer and the four epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * kAccCols));
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
        const int bytes = kStageA + ncol * 2 * DD_TC_ATOM;
        for (int pp = 0; pp < 4 && !fail; ++pp) {
          if (!(t.pad & (4 << pp))) continue;
          const int p = k + pp;
          const unsigned char* w = ws.p[pp];
          const unsigned char* gA = w + F.ws_off + (int64_t)(t.i - p - 1) * DD_TC_ATILE;
          // unpivoted fronts: the one image of M = L D^(1/2) is both operands
          const unsigned char* gB = w + (F.piv ? F.ws_boff : F.ws_off) + (int64_t)(t.j - p - 1) * DD_TC_BTILE;
          for (int a = 0; a < 2; ++a, ++u) {
            const int sidx = u % kStages;
            if (!mbar_wait(b_empty0 + 8 * sidx, ((u / kStages) & 1) ^ 1)) { fail = 1; break; }
            const uint32_t fb = b_full0 + 8 * sidx;
            unsigned char* stg = smem + sidx * kStage;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes) : "memory");
            for (int sp = 0; sp < 2; ++sp)
              bulk_g2s(smem_u32(stg + sp * DD_TC_ATOM), gA + (sp * 2 + a) * DD_TC_ATOM, DD_TC_ATOM, fb);
            for (int sp = 0; sp < 2; ++sp)
              for (int c = 0; c < ncol; ++c)
                bulk_g2s(smem_u32(stg + kStageA + sp * 2 * DD_TC_ATOM + c * DD_TC_ATOM),
                         gB + (int64_t)c * DD_TC_BTILE + (sp * 2 + a) * DD_TC_ATOM, DD_TC_ATOM, fb);
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
        const int ab = tl & 1;
        if (!mbar_wait(b_acce0 + 8 * ab, ((tl >> 1) & 1) ^ 1)) { fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dacc = tmem + ab * kAccCols;
        const uint32_t idesc = (t.pad & 2) ? kIdesc256 : kIdesc128;
        uint32_t acc_on = 0;
        for (int pp = 0; pp < 4 && !fail; ++pp) {
          if (!(t.pad & (4 << pp))) continue;
          for (int a = 0; a < 2; ++a, ++u) {
            const int sidx = u % kStages;
            if (!mbar_wait(b_full0 + 8 * sidx, (u / kStages) & 1)) { fail = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = s0 + sidx * kStage, b0 = a0 + kStageA;
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
              for (int sp = 0; sp < 3; ++sp) {   // split pairs (hi, hi), (hi, lo), (lo, hi)
                const int as = sp == 2 ? 1 : 0, bs = sp == 1 ? 1 : 0;
                const uint64_t ad = desc_sw128(a0 + as * DD_TC_ATOM + s4 * 32);
                const uint64_t bd = desc_sw128(b0 + bs * 2 * DD_TC_ATOM + s4 * 32);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc_on));
                acc_on = 1;
              }
            mma_commit(b_empty0 + 8 * sidx);   // the stage is free once these MMAs have read it
          }
        }
        if (fail) break;
        mma_commit(b_accf0 + 8 * ab);
      }
    }
  } else if (warp >= 2) {
    epilogue_role(pool, fr, tasks, groups, tmem, stage_c, b_gfull0, b_gempty0, gring, b_accf0, b_acce0, fail);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAccCols));
}

}  // namespace

void launch_update_tc(void* pool, const FrontDev* fronts, const Task* tasks, const int2* groups, int n, int k,
                      const PanelImages& ws, DevStatus* st, cudaStream_t s,
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
  k_update_tc<<<grid, 192, kSmemP, s>>>((float2*)pool, fronts, tasks, groups, n, k, ws, st, counter);
}

}  // namespace ddk
