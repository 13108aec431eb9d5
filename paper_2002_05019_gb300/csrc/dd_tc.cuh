// Building blocks of the tcgen05 (5th-generation tensor core) kernels of the
// mixed form: shared-memory matrix and instruction descriptors, mbarrier and
// TMEM access, the tf32 hi/lo split, and the operand image layout.
//
// Complex products run as real GEMMs: an A operand of 128 rows holds the real
// and imaginary parts of 64 complex rows (per group of 16 rows, their real
// parts then their imaginary parts, so that both parts of a row of the result
// sit in the same TMEM sub-partition); a B operand of 128 rows per 64 complex
// rows holds their 64 real parts then their 64 imaginary parts.  The
// accumulator of row p (Re / Im of complex row r), column n (Re / Im of
// complex column c) is then recombined into Re = ReA.ReB - ImA.ImB and
// Im = ReA.ImB + ImA.ReB.  Operands are K-major, 128B-swizzled, in atoms of
// 32 tf32 values (128 B a row); 3xTF32 products (hi.hi + hi.lo + lo.hi) give
// FP32-class accuracy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ddk {
namespace tc {

constexpr int kWaitPolls = 1 << 24;   // bounded waits: about a second of polling

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
__device__ __forceinline__ void mma_tf32(uint32_t dacc, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc_on) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc_on));
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

// byte offset of element (row, k), k in 0..31, in a 128B-swizzled K-major atom
// (8-row groups of 1024 B; the 16-byte chunk index is XORed with row % 8)
__device__ __forceinline__ int swz128(int row, int k) {
  return (row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 2) ^ (row & 7))) << 4) + (k & 3) * 4;
}
// x = hi + lo with hi, lo representable in tf32 (round to nearest, ties away)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  const float r = x - __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
  hi = __uint_as_float(h);
  lo = __uint_as_float(l);
}

// Operand image of 64 complex rows and NA atoms of 32 K (K = 32 NA): pieces of
// 128 rows x 32 K (16 KB), piece (split s, atom a) at (s NA + a) 16 KB.
constexpr int kAtom = 16384;
constexpr int kImage = 4 * kAtom;   // NA = 2: the full K = 64 of a tile
template <int NA>
__device__ __forceinline__ void put_split(unsigned char* img, int row, int k, float v) {
  float h, l;
  split_tf32(v, h, l);
  const int a = k >> 5, kk = k & 31;
  *reinterpret_cast<float*>(img + (0 * NA + a) * kAtom + swz128(row, kk)) = h;
  *reinterpret_cast<float*>(img + (1 * NA + a) * kAtom + swz128(row, kk)) = l;
}
// A operand: complex row r (0..63), K index k
template <int NA = 2>
__device__ __forceinline__ void put_a(unsigned char* img, int r, int k, float2 v) {
  const int ra = (r >> 4) * 32 + (r & 15);
  put_split<NA>(img, ra, k, v.x);
  put_split<NA>(img, ra + 16, k, v.y);
}
// B operand: complex row n (0..63), K index k
template <int NA = 2>
__device__ __forceinline__ void put_b(unsigned char* img, int n, int k, float2 v) {
  put_split<NA>(img, n, k, v.x);
  put_split<NA>(img, n + 64, k, v.y);
}

// Issues acc (+)= A B^T for two images of NA atoms (M = 128, N = 128,
// K = 32 NA tf32, 3xTF32: 12 NA MMAs) from one thread.
template <int NA = 2>
__device__ __forceinline__ void mma_tile(uint32_t dacc, uint32_t sA, uint32_t sB, bool accumulate) {
  constexpr uint32_t idesc = idesc_tf32(128);
  uint32_t on = accumulate ? 1u : 0u;
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
      for (int sp = 0; sp < 3; ++sp) {   // split pairs (hi, hi), (hi, lo), (lo, hi)
        const int as = sp == 2 ? 1 : 0, bs = sp == 1 ? 1 : 0;
        mma_tf32(dacc, desc_sw128(sA + (as * NA + a) * kAtom + s4 * 32),
                 desc_sw128(sB + (bs * NA + a) * kAtom + s4 * 32), idesc, on);
        on = 1;
      }
}

// Reads the complex 64 x 64 result of mma_tile from TMEM (warps 0-3 of the
// CTA, warp w holding complex rows 16 w .. 16 w + 15) and passes each element
// to store(row, col, value).
template <typename F>
__device__ __forceinline__ void read_tile(uint32_t tmem, F&& store) {
  const int warp = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
  const bool im = lane >= 16;
  const int row = warp * 16 + (lane & 15);
#pragma unroll 1
  for (int hf = 0; hf < 2; ++hf) {
    uint32_t xr[32], xi[32];   // this lane's row times [Re B] and [Im B], 32 columns
    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + hf * 32;
    tmem_ld32(ta, xr);
    tmem_ld32(ta + 64, xi);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    // lanes < 16 (Re A) keep columns 0-15 and send 16-31; lanes >= 16 (Im A) the reverse
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float sr = __uint_as_float(im ? xr[c] : xr[16 + c]);
      const float si = __uint_as_float(im ? xi[c] : xi[16 + c]);
      const float pr = __shfl_xor_sync(0xffffffffu, sr, 16);
      const float pi = __shfl_xor_sync(0xffffffffu, si, 16);
      const float orr = __uint_as_float(im ? xr[16 + c] : xr[c]);
      const float oii = __uint_as_float(im ? xi[16 + c] : xi[c]);
      const float re = im ? pr - oii : orr - pi;
      const float imv = im ? pi + orr : oii + pr;
      store(row, hf * 32 + (im ? 16 : 0) + c, make_float2(re, imv));
    }
  }
}

}  // namespace tc
}  // namespace ddk
