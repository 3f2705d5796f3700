// Device helpers of the tcgen05 (sm_103a) kernels: TF32 hi/lo split, the
// K-major no-swizzle shared-memory operand layout and its descriptor, the
// instruction descriptor of kind::tf32, MMA issue, bounded mbarrier polling
// and 32-lane TMEM loads.
#pragma once

#include <cstdint>

namespace lddmm {
namespace tc {

constexpr int kMTile = 128;   // M of every tcgen05 tile here (cta_group::1)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float offset of element (row r, k) in a K-major no-swizzle operand tile with
// Kp columns: core matrix (r/8, k/4) of 8 rows x 4 elements, rows 16 bytes apart
__device__ __forceinline__ int kmajor_off(int r, int k, int Kp) {
  return (((r >> 3) * (Kp >> 2) + (k >> 2)) << 5) + ((r & 7) << 2) + (k & 3);
}

// tcgen05 shared-memory descriptor: no swizzle, K-major; LBO = distance of
// K-adjacent core matrices, SBO = distance of 8-row groups (bytes).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// instruction descriptor: kind::f16 with A = B = BF16 (the two operands of one
// MMA must have the same type), D = F32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// element offset of (row r, k) in a K-major no-swizzle operand tile of 16-bit
// elements with Kp columns: core matrix (r/8, k/8) of 8 rows x 8 elements
__device__ __forceinline__ int kmajor_off16(int r, int k, int Kp) {
  return (((r >> 3) * (Kp >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// the same 32-lane x 16-column load, the wait left to the caller (several
// loads in flight, then tmem_wait)
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 columns summed over NACC accumulators `stride` columns apart (the 3xTF32
// products may be kept in separate accumulators; NACC = 1: one accumulator)
template <int NACC>
__device__ __forceinline__ void tmem_ld16_sum(uint32_t taddr, uint32_t stride, float* v) {
  uint32_t r[NACC][16];
#pragma unroll
  for (int a = 0; a < NACC; ++a) tmem_ld16_async(taddr + (uint32_t)a * stride, r[a]);
  tmem_wait();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    float x = __uint_as_float(r[0][j]);
#pragma unroll
    for (int a = 1; a < NACC; ++a) x += __uint_as_float(r[a][j]);
    v[j] = x;
  }
}

// K-loop of one 3xTF32 product tile over NACC accumulators `stride` columns
// apart: hi*hi into accumulator 0, hi*lo and lo*hi into 1 and 2 (NACC = 3) or
// both into 1 (NACC = 2).  Descriptors: K-major, no swizzle, 16-byte rows,
// LBO = 128 bytes, SBO = (K / 4) * 128 bytes; K a multiple of 8.
template <int NACC>
__device__ __forceinline__ void mma_3xtf32(uint32_t dcol, uint32_t stride, const float* ah, const float* al,
                                           const float* bh, const float* bl, int K, uint32_t idesc) {
  const uint32_t sbo = (uint32_t)(K >> 2) * 128;
  for (int s = 0; s < K / 8; ++s) {
    const uint32_t so = (uint32_t)s * 256;
    const uint64_t dah = smem_desc(smem_u32(ah) + so, 128, sbo);
    const uint64_t dal = smem_desc(smem_u32(al) + so, 128, sbo);
    const uint64_t dbh = smem_desc(smem_u32(bh) + so, 128, sbo);
    const uint64_t dbl = smem_desc(smem_u32(bl) + so, 128, sbo);
    const uint32_t first = s > 0 ? 1u : 0u;
    mma_tf32(dcol, dah, dbh, idesc, first);
    if (NACC == 3) {
      mma_tf32(dcol + stride, dah, dbl, idesc, first);
      mma_tf32(dcol + 2 * stride, dal, dbh, idesc, first);
    } else if (NACC == 2) {
      mma_tf32(dcol + stride, dah, dbl, idesc, first);
      mma_tf32(dcol + stride, dal, dbh, idesc, 1u);
    } else {
      mma_tf32(dcol, dah, dbl, idesc, 1u);
      mma_tf32(dcol, dal, dbh, idesc, 1u);
    }
  }
}

}  // namespace tc
}  // namespace lddmm
