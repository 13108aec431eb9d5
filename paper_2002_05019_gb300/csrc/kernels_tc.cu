// Tensor-core trailing update of the mixed form (Section II: the dense block
// updates of the domain and auxiliary-matrix factorizations run as level-3
// BLAS; here on the 5th-generation tensor cores).
//
// One CTA computes a 128 x 64 complex block of  C -= L_ik D_k L_jk^T  (rows of
// the tiles i0 and i0+1, column tile j) with tcgen05.mma kind::tf32:
//   * complex product as one real GEMM with a [Re | Im] accumulator:
//       acc[:, 0:64]   = Lr Wr^T - Li Wi^T,   acc[:, 64:128] = Lr Wi^T + Li Wr^T
//     = Lr [Wr; Wi]^T + Li [-Wi; Wr]^T  (B operands of N = 128 rows);
//   * 3xTF32 split for FP32 accuracy: X Y^T ~ Xh Yh^T + Xh Yl^T + Xl Yh^T;
//   * operands are the pre-split, 128B-swizzled K-major images written by the
//     panel kernel, brought into shared memory by bulk asynchronous copies
//     (TMA engine) completing on an mbarrier; the accumulator lives in TMEM
//     (128 lanes x 128 fp32 columns) and is read back with tcgen05.ld.
// Every wait is bounded: on timeout the CTA records DD_ERR_TIMEOUT, waits once
// more (bounded) for its copies, frees its TMEM and returns.
#include "dd_complex.cuh"
#include "dd_internal.h"

namespace ddk {

namespace {

constexpr int T = DD_TILE;
constexpr int kA = DD_TC_ABLOCK;   // 128 KB
constexpr int kB = DD_TC_BTILE;    // 96 KB
constexpr int kSmem = kA + kB + 1024;
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

// instruction descriptor: D f32, A/B tf32, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

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

__global__ void __launch_bounds__(128, 1) k_update_tc(float2* pool, const FrontDev* fr, const Task* tasks, int k,
                                                      const unsigned char* ws, DevStatus* st) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;
  unsigned char* sB = smem + kA;
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ int ok_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Task t = tasks[blockIdx.x];
  const FrontDev F = fr[t.f];
  const uint32_t mb_load = smem_u32(&bar_load), mb_mma = smem_u32(&bar_mma);
  const unsigned char* gA = ws + F.ws_off + (int64_t)((t.i - k - 1) >> 1) * kA;
  const unsigned char* gB = ws + F.ws_boff + (int64_t)(t.j - k - 1) * kB;

  if (tid == 0) {
    ok_sh = 1;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_load));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_mma));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb_load), "r"(kA + kB) : "memory");
    for (int c = 0; c < kA / DD_TC_ATOM; ++c)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sA + c * DD_TC_ATOM)),
                   "l"(gA + c * DD_TC_ATOM), "r"(DD_TC_ATOM), "r"(mb_load)
                   : "memory");
    for (int c = 0; c < kB / DD_TC_HALF; ++c)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sB + c * DD_TC_HALF)),
                   "l"(gB + c * DD_TC_HALF), "r"(DD_TC_HALF), "r"(mb_load)
                   : "memory");
    if (!mbar_wait(mb_load, 0)) {
      ok_sh = 0;
      mbar_wait(mb_load, 0);  // second bounded wait for the copies in flight
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      // (A plane, B split, B variant): variant 1 = [Wr; Wi] (+8 KB), 0 = [-Wi; Wr]
      const int pl[6] = {0, 0, 1, 2, 2, 3};
      const int bs[6] = {0, 1, 0, 0, 1, 0};
      const int bv[6] = {1, 1, 1, 0, 0, 0};
      uint32_t acc = 0;
      for (int a = 0; a < 2; ++a)
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const uint64_t ad = desc_sw128(a0 + (pl[q] * 2 + a) * DD_TC_ATOM + s * 32);
            const uint64_t bd = desc_sw128(b0 + ((bs[q] * 2 + a) * 3 + bv[q]) * DD_TC_HALF + s * 32);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
            acc = 1;
          }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb_mma)
                   : "memory");
      if (!mbar_wait(mb_mma, 0)) ok_sh = 0;
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok_sh) {
    // epilogue: warp w owns rows 32w..32w+31 (its TMEM lanes)
    const int row = warp * 32 + lane;
    const bool store = (row < T) ? (t.pad & 1) : (t.pad & 2);
    float2* crow = pool + F.off + (int64_t)(t.i * T + row) * F.ld + t.j * T;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      uint32_t vr[32], vi[32];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + h * 32;
      tmem_ld32(ta, vr);
      tmem_ld32(ta + 64, vi);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (store) {
        float4* c4 = reinterpret_cast<float4*>(crow + h * 32);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float4 v = c4[q];
          v.x -= __uint_as_float(vr[2 * q]);
          v.y -= __uint_as_float(vi[2 * q]);
          v.z -= __uint_as_float(vr[2 * q + 1]);
          v.w -= __uint_as_float(vi[2 * q + 1]);
          c4[q] = v;
        }
      }
    }
  } else if (tid == 0) {
    if (atomicCAS(&st->code, 0, 8) == 0) {
      st->front = t.f;
      st->row = t.i * T;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

}  // namespace

void launch_update_tc(void* pool, const FrontDev* fronts, const Task* tasks, int n, int k, const unsigned char* ws,
                      DevStatus* st, cudaStream_t s) {
  if (n <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    attr = true;
  }
  k_update_tc<<<n, 128, kSmem, s>>>((float2*)pool, fronts, tasks, k, ws, st);
}

}  // namespace ddk
