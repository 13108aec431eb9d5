// Tensor-core trailing update of the mixed form (Section II: the dense block
// updates of the domain and auxiliary-matrix factorizations run as level-3
// BLAS; here on the 5th-generation tensor cores).
//
// A task is a 128 x 64 complex block of  C -= L_ik D_k L_jk^T  (rows of the
// tiles i0 and i0+1, column tile j), computed with tcgen05.mma kind::tf32:
//   * complex product as real GEMMs (N = 64) into a [Re | Im] accumulator:
//       acc[:, 0:64]   = Lr Wr^T - Li Wi^T,   acc[:, 64:128] = Lr Wi^T + Li Wr^T,
//     the minus sign through the instruction's negate-A bit;
//   * 3xTF32 split for FP32 accuracy: X Y^T ~ Xh Yh^T + Xh Yl^T + Xl Yh^T;
//   * operands are the pre-split, 128B-swizzled K-major images written by the
//     panel kernel, brought into shared memory by bulk asynchronous copies
//     (TMA engine) completing on an mbarrier; the accumulator lives in TMEM
//     (128 lanes x 128 fp32 columns) and is read back with tcgen05.ld.
// Every wait is bounded: on timeout the CTA records DD_ERR_TIMEOUT, its roles
// stop, and it frees its TMEM and returns.
#include "dd_complex.cuh"
#include "dd_internal.h"

namespace ddk {

namespace {

constexpr int T = DD_TILE;
constexpr int kA = DD_TC_ABLOCK;   // 128 KB
constexpr int kB = DD_TC_BTILE;    // 96 KB
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

// instruction descriptor: D f32, A/B tf32, both K-major, N = 64, M = 128; bit 13 negates A
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescNegA = kIdesc | (1u << 13);

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

// Persistent, warp-specialised form: grid <= one CTA per SM, each CTA takes a
// contiguous chunk of the task list, so consecutive tasks share their 128-row
// A block.  Warp 0 lane 0 loads the A block (128 KB, resident while it is
// reused) and streams the B tiles through a three-stage ring (one K-atom of B,
// 32 KB, per stage); warp 1 lane 0 issues the MMAs into one of two TMEM
// accumulators; warps 2-5 drain the other accumulator into C.
constexpr int kStageB = 2 * 2 * DD_TC_HALF;      // 2 splits x [Wr][Wi] of one atom = 32 KB
constexpr int kBStages = 2;
constexpr int kStg = 32 * 17;                            // per epilogue warp: 32 x 16 complex, padded rows
constexpr int kSmemP = kA + kBStages * kStageB + 4 * kStg * 8 + 1024;  // 128 + 64 + 17 KB + alignment

constexpr int kRing = 8;   // group ids handed from the producer to the MMA and epilogue roles

struct PipeBars {
  uint64_t a_full, a_empty, b_full[kBStages], b_empty[kBStages], acc_full[2], acc_empty[2];
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

// Epilogue role (warps 2-5): drain each task's TMEM accumulator into C
// (C -= acc), row by row through a per-warp shared-memory transpose so that a
// warp's reductions cover two full 256-byte row segments of C.
__device__ __forceinline__ void epilogue_role(float2* pool, const FrontDev* fr, const Task* tasks, const int2* groups,
                                              uint32_t tmem, float2* stage_c, uint32_t b_gfull0, uint32_t b_gempty0,
                                              const int* gring, uint32_t b_accf0, uint32_t b_acce0,
                                              volatile int& fail) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // ---------------- epilogue: C -= acc ----------------
    const int sub = warp & 3;                 // TMEM sub-partition of this warp
    const int row = sub * 32 + lane;
    int tl = 0;
    bool stop = false;
    for (int it = 0; !stop; ++it) {
      const int slot = it % kRing;
      int g = -1;
      bool okg = true;
      if (lane == 0) {
        okg = mbar_wait(b_gfull0 + 8 * slot, (it / kRing) & 1);
        if (okg) g = gring[slot];
      }
      okg = __shfl_sync(0xffffffffu, okg ? 1 : 0, 0) != 0;
      g = __shfl_sync(0xffffffffu, g, 0);
      if (lane == 0 && okg) mbar_arrive(b_gempty0 + 8 * slot);
      if (!okg) { fail = 1; break; }
      if (g < 0) break;
    for (int q = groups[g].x; q < groups[g].x + groups[g].y; ++q, ++tl) {
      const Task t = tasks[q];
      const FrontDev F = fr[t.f];
      const int ab = tl & 1;
      bool ok = !fail;
      if (ok && lane == 0) ok = mbar_wait(b_accf0 + 8 * ab, (tl >> 1) & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) { fail = 1; stop = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      // rows sub*32 .. sub*32+31 all lie in one 64-row tile: one store flag per warp
      const bool store = (sub < 2) ? (t.pad & 1) : (t.pad & 2);
      float2* stg = stage_c + (warp - 2) * kStg;
      float2* cblk = pool + F.off + (int64_t)(t.i * T + sub * 32) * F.ld + t.j * T;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        uint32_t vr[32], vi[32];
        const uint32_t ta = tmem + ab * 128 + ((uint32_t)(sub * 32) << 16) + h * 32;
        tmem_ld32(ta, vr);
        tmem_ld32(ta + 64, vi);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (store) {
          // thread = row -> shared memory -> four rows x 16 columns per warp access, so the
          // reductions into C are row-contiguous (128 B per row)
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
            for (int c = 0; c < 16; ++c)
              stg[lane * 17 + c] = make_float2(-__uint_as_float(vr[hh * 16 + c]), -__uint_as_float(vi[hh * 16 + c]));
            __syncwarp();
            const int rsub = lane >> 3, cpair = (lane & 7) * 2;
#pragma unroll 4
            for (int rr = 0; rr < 8; ++rr) {
              const int r = 4 * rr + rsub;
              const float2 v0 = stg[r * 17 + cpair], v1 = stg[r * 17 + cpair + 1];
              float* dst = reinterpret_cast<float*>(cblk + (int64_t)r * F.ld + h * 32 + hh * 16 + cpair);
              asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(v0.x), "f"(v0.y),
                           "f"(v1.x), "f"(v1.y)
                           : "memory");
            }
            __syncwarp();
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(b_acce0 + 8 * ab);
    }
    }
  }

__global__ void __launch_bounds__(192, 1) k_update_tc(float2* pool, const FrontDev* fr, const Task* tasks,
                                                      const int2* groups, int n_groups, int k,
                                                      const unsigned char* ws, DevStatus* st, int* counter) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;               // resident A block (planes x atoms, 16 KB each)
  unsigned char* sB = smem + kA;          // B ring: stage s at sB + s * kStageB
  float2* stage_c = reinterpret_cast<float2*>(smem + kA + kBStages * kStageB);   // epilogue transposes
  __shared__ __align__(8) PipeBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int fail;
  __shared__ int gring[kRing];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_afull = smem_u32(&bars.a_full), b_aempty = smem_u32(&bars.a_empty);
  const uint32_t b_full0 = smem_u32(&bars.b_full[0]), b_empty0 = smem_u32(&bars.b_empty[0]);
  const uint32_t b_accf0 = smem_u32(&bars.acc_full[0]), b_acce0 = smem_u32(&bars.acc_empty[0]);
  // groups (runs of <= 8 tasks that share one A block) are claimed dynamically
  // from a global counter in list order, so the groups in flight at any time are
  // consecutive ones of a few fronts (their B tiles are shared through L2) and
  // faster SMs simply take more of them
  const uint32_t b_gfull0 = smem_u32(&bars.g_full[0]), b_gempty0 = smem_u32(&bars.g_empty[0]);
  if (tid == 0) {
    fail = 0;
    mbar_init(b_afull, 1);
    mbar_init(b_aempty, 1);
    for (int i = 0; i < kBStages; ++i) {
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
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer ----------------
    int m = 0, u = 0;
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
      if (q == groups[g].x) {   // new A block
        if (m > 0 && !mbar_wait(b_aempty, (m - 1) & 1)) { fail = 1; break; }
        const unsigned char* gA = ws + F.ws_off + (int64_t)((t.i - k - 1) >> 1) * kA;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b_afull), "r"(kA) : "memory");
        for (int c = 0; c < kA / DD_TC_ATOM; ++c)
          bulk_g2s(smem_u32(sA + c * DD_TC_ATOM), gA + c * DD_TC_ATOM, DD_TC_ATOM, b_afull);
        ++m;
      }
      const unsigned char* gB = ws + F.ws_boff + (int64_t)(t.j - k - 1) * kB;
      for (int a = 0; a < 2; ++a, ++u) {
        const int sidx = u % kBStages;
        if (!mbar_wait(b_empty0 + 8 * sidx, ((u / kBStages) & 1) ^ 1)) { fail = 1; break; }
        const uint32_t fb = b_full0 + 8 * sidx;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStageB) : "memory");
        for (int sp = 0; sp < 2; ++sp)
          bulk_g2s(smem_u32(sB + sidx * kStageB + sp * 2 * DD_TC_HALF), gB + (sp * 2 + a) * 2 * DD_TC_HALF,
                   2 * DD_TC_HALF, fb);
      }
    }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int m = 0, u = 0, tl = 0;
    const uint32_t a0 = smem_u32(sA), bring = smem_u32(sB);
    for (int it = 0; !fail; ++it) {
      const int slot = it % kRing;
      if (!mbar_wait(b_gfull0 + 8 * slot, (it / kRing) & 1)) { fail = 1; break; }
      const int g = gring[slot];
      mbar_arrive(b_gempty0 + 8 * slot);
      if (g < 0) break;
    for (int q = groups[g].x; q < groups[g].x + groups[g].y && !fail; ++q, ++tl) {
      const Task t = tasks[q];
      if (q == groups[g].x) {
        if (!mbar_wait(b_afull, m & 1)) { fail = 1; break; }
        ++m;
      }
      const int ab = tl & 1;
      if (!mbar_wait(b_acce0 + 8 * ab, ((tl >> 1) & 1) ^ 1)) { fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t dacc = tmem + ab * 128;
      uint32_t init_re = 0, init_im = 0;   // accumulator halves already written for this task
      for (int a = 0; a < 2; ++a, ++u) {
        const int sidx = u % kBStages;
        if (!mbar_wait(b_full0 + 8 * sidx, (u / kBStages) & 1)) { fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t b0 = bring + sidx * kStageB;
        for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
          for (int sp = 0; sp < 3; ++sp) {     // split pairs (hi, hi), (hi, lo), (lo, hi)
            const int as = sp == 2 ? 1 : 0, bsp = sp == 1 ? 1 : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              // (Re L, Re W) -> Re, (Im L, Im W, negated) -> Re, (Re L, Im W) -> Im, (Im L, Re W) -> Im
              const int ar = q & 1, bw = (q == 1 || q == 2) ? 1 : 0, dh = q >> 1;
              const uint64_t ad = desc_sw128(a0 + ((ar * 2 + as) * 2 + a) * DD_TC_ATOM + s4 * 32);
              const uint64_t bd = desc_sw128(b0 + (bsp * 2 + bw) * DD_TC_HALF + s4 * 32);
              const uint32_t en = dh ? init_im : init_re;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc + dh * 64),
                  "l"(ad), "l"(bd), "r"(q == 1 ? kIdescNegA : kIdesc), "r"(en));
              if (dh) init_im = 1; else init_re = 1;
            }
          }
        mma_commit(b_empty0 + 8 * sidx);   // the B stage is free once these MMAs have read it
      }
      if (fail) break;
      mma_commit(b_accf0 + 8 * ab);
      // the A block is free once the last task that uses it has been issued
      if (q + 1 == groups[g].x + groups[g].y) mma_commit(b_aempty);   // last task of the group
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
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// Two-panel form: the trailing update of panels k and k + 1 in one pass,
// C -= [L_ik L_i,k+1] [W_jk W_j,k+1]^T with K = 128, so C is read and written
// once for two panel steps.  Operands are streamed: per K-atom a 96 KB stage
// holds the four A planes of the 128-row block (two 8 KB tile pieces each)
// and the B planes of the column tile; two stages.  Task .pad: bits 0 / 1
// store the rows of tile i0 / i0 + 1, bit 2 / 3 the panel k / k + 1
// contributes (a panel whose rows or column are structurally zero is skipped).
constexpr int kStage2 = 4 * DD_TC_ATOM + 2 * 2 * DD_TC_HALF;   // 96 KB
constexpr int kStages2 = 2;
constexpr int kSmemP2 = kStages2 * kStage2 + 4 * kStg * 8 + 1024;

__global__ void __launch_bounds__(192, 1) k_update_tc2(float2* pool, const FrontDev* fr, const Task* tasks,
                                                       const int2* groups, int n_groups, int k,
                                                       const unsigned char* ws0, const unsigned char* ws1,
                                                       DevStatus* st, int* counter) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float2* stage_c = reinterpret_cast<float2*>(smem + kStages2 * kStage2);
  __shared__ __align__(8) PipeBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int fail;
  __shared__ int gring[kRing];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_full0 = smem_u32(&bars.b_full[0]), b_empty0 = smem_u32(&bars.b_empty[0]);
  const uint32_t b_accf0 = smem_u32(&bars.acc_full[0]), b_acce0 = smem_u32(&bars.acc_empty[0]);
  const uint32_t b_gfull0 = smem_u32(&bars.g_full[0]), b_gempty0 = smem_u32(&bars.g_empty[0]);
  static_assert(kStages2 <= kBStages, "stage barriers");
  if (tid == 0) {
    fail = 0;
    for (int i = 0; i < kStages2; ++i) {
      mbar_init(b_full0 + 8 * i, 1);
      mbar_init(b_empty0 + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_accf0 + 8 * i, 1);
      mbar_init(b_acce0 + 8 * i, 4);
    }
    for (int i = 0; i < kRing; ++i) {
      mbar_init(b_gfull0 + 8 * i, 1);
      mbar_init(b_gempty0 + 8 * i, 5);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_slot)));
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
        const int nh = ((t.pad & 1) ? 1 : 0) + ((t.pad & 2) ? 1 : 0);
        const int bytes = nh * 4 * DD_TC_HALF + 2 * 2 * DD_TC_HALF;
        for (int pp = 0; pp < 2 && !fail; ++pp) {
          if (!(t.pad & (4 << pp))) continue;
          const int p = k + pp;
          const unsigned char* w = pp ? ws1 : ws0;
          const unsigned char* gB = w + F.ws_boff + (int64_t)(t.j - p - 1) * kB;
          for (int a = 0; a < 2; ++a, ++u) {
            const int sidx = u % kStages2;
            if (!mbar_wait(b_empty0 + 8 * sidx, ((u / kStages2) & 1) ^ 1)) { fail = 1; break; }
            const uint32_t fb = b_full0 + 8 * sidx;
            unsigned char* stg = smem + sidx * kStage2;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes) : "memory");
            for (int hh = 0; hh < 2; ++hh) {
              if (!(t.pad & (1 << hh))) continue;   // rows not stored: their smem rows stay stale
              const int ti = t.i + hh - p - 1;       // trailing-tile index of this row tile in panel p
              const unsigned char* gA = w + F.ws_off + (int64_t)(ti >> 1) * kA + (ti & 1) * DD_TC_HALF;
              for (int pl = 0; pl < 4; ++pl)
                bulk_g2s(smem_u32(stg + pl * DD_TC_ATOM + hh * DD_TC_HALF), gA + (pl * 2 + a) * DD_TC_ATOM,
                         DD_TC_HALF, fb);
            }
            for (int sp = 0; sp < 2; ++sp)
              bulk_g2s(smem_u32(stg + 4 * DD_TC_ATOM + sp * 2 * DD_TC_HALF), gB + (sp * 2 + a) * 2 * DD_TC_HALF,
                       2 * DD_TC_HALF, fb);
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
        const uint32_t dacc = tmem + ab * 128;
        uint32_t init_re = 0, init_im = 0;
        for (int pp = 0; pp < 2 && !fail; ++pp) {
          if (!(t.pad & (4 << pp))) continue;
          for (int a = 0; a < 2; ++a, ++u) {
            const int sidx = u % kStages2;
            if (!mbar_wait(b_full0 + 8 * sidx, (u / kStages2) & 1)) { fail = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = s0 + sidx * kStage2, b0 = a0 + 4 * DD_TC_ATOM;
            for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
              for (int sp = 0; sp < 3; ++sp) {   // split pairs (hi, hi), (hi, lo), (lo, hi)
                const int as = sp == 2 ? 1 : 0, bsp = sp == 1 ? 1 : 0;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                  const int ar = qq & 1, bw = (qq == 1 || qq == 2) ? 1 : 0, dh = qq >> 1;
                  const uint64_t ad = desc_sw128(a0 + (ar * 2 + as) * DD_TC_ATOM + s4 * 32);
                  const uint64_t bd = desc_sw128(b0 + (bsp * 2 + bw) * DD_TC_HALF + s4 * 32);
                  const uint32_t en = dh ? init_im : init_re;
                  asm volatile(
                      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc + dh * 64),
                      "l"(ad), "l"(bd), "r"(qq == 1 ? kIdescNegA : kIdesc), "r"(en));
                  if (dh) init_im = 1; else init_re = 1;
                }
              }
            mma_commit(b_empty0 + 8 * sidx);
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
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

}  // namespace

void launch_update_tc(void* pool, const FrontDev* fronts, const Task* tasks, const int2* groups, int n, int k,
                      const unsigned char* ws, DevStatus* st, cudaStream_t s, int reserve_sms, int* counter) {
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

void launch_update_tc2(void* pool, const FrontDev* fronts, const Task* tasks, const int2* groups, int n, int k,
                       const unsigned char* ws0, const unsigned char* ws1, DevStatus* st, cudaStream_t s,
                       int reserve_sms, int* counter) {
  if (n <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    cudaFuncSetAttribute(k_update_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemP2);
  }
  const int avail = sms - reserve_sms > 1 ? sms - reserve_sms : 1;
  const int grid = n < avail ? n : avail;
  k_update_tc2<<<grid, 192, kSmemP2, s>>>((float2*)pool, fronts, tasks, groups, n, k, ws0, ws1, st, counter);
}

}  // namespace ddk
