// Tensor-core products for the n = 64 combinations of the mixed-precision
// path: the FP32 products of the combination rule (Sec. IV-A, eq. lqt_comb)
// as tcgen05.mma kind::tf32 on the SM's tensor core, with the accumulator in
// tensor memory.
//
// Precision: an FP32 operand x is split into three TF32 pieces, x = hi + mid +
// lo, hi = x rounded to TF32's 10 mantissa bits, mid = (x - hi) rounded the
// same way, lo = x - hi - mid (every difference exact in FP32; |mid| <=
// 2^-11 |x|, |lo| <= 2^-22 |x|), and the product is accumulated in FP32 from
// the six terms down to 2^-22: hi hi, hi mid, mid hi, hi lo, lo hi, mid mid.
// The pieces' own TF32 truncation then sits near 2^-33 |x|, below the FP32
// accumulation's rounding, so the result carries FP32 accuracy (measured ~2e-6
// relative with two pieces, which was not enough for the 1e-4 target over a
// whole scan).
//
// Data path of one 64 x 64 x 64 product D = A B (one CTA of 256 threads):
//  * every thread converts its share of A and B (from FP64 storage) once and
//    writes the three pieces into shared memory in the tensor core's K-major,
//    unswizzled layout: 8-row x 16-byte core matrices, 128 contiguous bytes
//    each, 1024 B apart along K and 128 B apart along M (A) or N (B, stored
//    transposed, N x K).  The MMA's M is 128: rows 64..127 of A are read
//    from the next 1024 bytes (the next K chunk, or for the last chunk of
//    the last A piece the first B piece) and only produce rows 64..127 of D,
//    which nothing reads, so A needs no zero padding;
//  * one thread issues 8 x 6 MMAs of M = 128, N = 64, K = 8, K step s into its
//    own 64 TMEM columns (all 512 of the SM's: one CTA per SM), and commits
//    them to an mbarrier; every thread waits on it with an iteration limit (on
//    time-out: a status bit, then one more bounded wait);
//  * warps 0, 1 and 4, 5 read the 64 result rows back with tcgen05.ld (warp w
//    reaches TMEM lanes 32 (w mod 4) .. +31), 32 columns each, adding the 8
//    step accumulators with FP32 adds on the CUDA cores.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {
namespace tc {

constexpr int kTeam = 256;
constexpr int kSteps = 8;             // K = 64 in MMAs of K = 8
constexpr int kCols = 64 * kSteps;    // TMEM columns: one 64-column accumulator per K step
// shared memory: A's three pieces, then B's (64 x 64 floats each), from a
// 1024-byte boundary (the MMA composes a core matrix's row addresses into the
// low address bits, so the operands must start 128-byte aligned; the dynamic
// region itself is only guaranteed 16-byte alignment).  B follows A, so the
// unused rows 64..127 of the last A piece's last K chunk stay inside the
// region.
constexpr int kAFloats = 64 * 64, kBFloats = 64 * 64;
constexpr size_t kSmemBytes = (3 * kAFloats + 3 * kBFloats) * sizeof(float) + 1024;
constexpr unsigned kWaitLimit = 1u << 24;

struct Ctx {
  uint32_t tmem;                // base address of the accumulator
  unsigned long long* bar;      // completion barrier of the MMAs
  unsigned phase;               // its next phase parity
  float* a[3];  // A's pieces hi, mid, lo
  float* b[3];  // B's pieces
};

__device__ __forceinline__ unsigned s32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (M/N-direction) byte offsets between core matrices, descriptor
// version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Allocates the accumulator (warp 0) and sets up the barrier; every thread of
// the CTA calls it once, before any product.  `tmem_slot`, `bar`: this CTA's shared words; `smem`: kSmemBytes
// of dynamic shared memory, declared with no more than 16-byte alignment (with
// relocatable device code the dynamic region starts wherever the static
// variables end; a larger declared alignment would let the compiler fold the
// run-time alignment below away).
__device__ __forceinline__ void init(Ctx& c, uint32_t* tmem_slot, unsigned long long* bar, void* smem) {
  const int tid = threadIdx.x;
  c.a[0] = (float*)((char*)smem + ((1024u - (s32(smem) & 1023u)) & 1023u));
  c.a[1] = c.a[0] + kAFloats;
  c.a[2] = c.a[1] + kAFloats;
  c.b[0] = c.a[2] + kAFloats;
  c.b[1] = c.b[0] + kBFloats;
  c.b[2] = c.b[1] + kBFloats;
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(tmem_slot)),
                 "n"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  c.tmem = *tmem_slot;
  c.bar = bar;
  c.phase = 0;
}

// Releases the accumulator; every thread of the CTA calls it once, last.
__device__ __forceinline__ void release(Ctx& c) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "n"(kCols) : "memory");
}

// x rounded to TF32 (10 mantissa bits; ties away from zero on the
// magnitude), as an FP32 value
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split3(double v, float& hi, float& mid, float& lo) {
  const float x = (float)v;
  hi = tf32_rn(x);
  const float r = x - hi;
  mid = tf32_rn(r);
  lo = r - mid;
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

// out(i, j, sum_l a(i, l) b(l, j)) for i, j < 64 (FP32 accuracy on the tensor
// core).  a, b return the FP64 operands; out receives floats.  Every thread of
// the CTA calls it (it synchronises the CTA).  Operands are all read before
// any result is written, so out may overwrite an operand.
template <class FA, class FB, class FO>
__device__ __forceinline__ void gemm64(Ctx& c, FA a, FB b, FO out) {
  const int tid = threadIdx.x;
  // stage: consecutive threads fill consecutive floats of the core matrices
  for (int e = tid; e < 64 * 64; e += kTeam) {
    // e = ((kc * 8 + g) * 8 + r) * 4 + kk: K chunk kc (4 floats), row group g,
    // row r within it; A row m = 8 g + r, and B^T (N x K) the same with n = m
    const int kk = e & 3, r = (e >> 2) & 7, mg = (e >> 5) & 7, kc = e >> 8;
    const int m = mg * 8 + r, k = kc * 4 + kk;
    float p0, p1, p2;
    split3(a(m, k), p0, p1, p2);
    c.a[0][e] = p0;
    c.a[1][e] = p1;
    c.a[2][e] = p2;
    split3(b(k, m), p0, p1, p2);
    c.b[0][e] = p0;
    c.b[1][e] = p1;
    c.b[2][e] = p2;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0) {
    constexpr uint32_t id = idesc_tf32(128, 64);
    // pieces (i, j) with i + j <= 2, smallest first, each K step into its own
    // accumulator: chained in one accumulator the 48 MMAs left ~1e-6 relative
    // error (the tensor core's accumulation rounds each partial sum); with one
    // accumulator per K step, the large hi hi term joining its step's small
    // terms last, and the 8 steps added with IEEE FP32 adds at the read-back,
    // the product is within ~1.2e-7 relative, FP32's own accuracy
    const int pa[6] = {2, 0, 1, 1, 0, 0};
    const int pb[6] = {0, 2, 1, 0, 1, 0};
#pragma unroll
    for (int s = 0; s < kSteps; ++s) {
#pragma unroll
      for (int pass = 0; pass < 6; ++pass) {
        const unsigned a0 = s32(c.a[pa[pass]]), b0 = s32(c.b[pb[pass]]);
        mma(c.tmem + (uint32_t)(64 * s), smem_desc(a0 + s * 2048, 1024, 128), smem_desc(b0 + s * 2048, 1024, 128),
            id, pass > 0 ? 1u : 0u);
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s32(c.bar))
                 : "memory");
  }
  {
    unsigned it = 0, ok = 0;
    for (;;) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(s32(c.bar)), "r"(c.phase)
          : "memory");
      if (ok) break;
      if (++it >= kWaitLimit) {
        if (tid == 0) flag(kStatusTimeout);
        for (unsigned j = 0; j < kWaitLimit; ++j) {
          asm volatile(
              "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
              : "=r"(ok)
              : "r"(s32(c.bar)), "r"(c.phase)
              : "memory");
          if (ok) break;
        }
        break;
      }
    }
    c.phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int warp = tid >> 5, lane = tid & 31;
  if ((warp & 3) < 2) {
    const int row = (warp & 3) * 32 + lane;
    const int c0 = warp >= 4 ? 32 : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float sum[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) sum[j] = 0.0f;
      for (int s = 0; s < kSteps; ++s) {
        uint32_t v[16];
        const uint32_t addr =
            c.tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(64 * s + c0 + 16 * h);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(addr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) sum[j] += __uint_as_float(v[j]);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) out(row, c0 + 16 * h + j, sum[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

}  // namespace tc
}  // namespace lqt
