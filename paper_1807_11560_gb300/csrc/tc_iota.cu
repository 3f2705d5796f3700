// Tensor-core (tcgen05, sm_103a) form of the image-grid iota stage C, the
// k1 -> x1 contraction of the band-limited-to-grid map (Eq. 46):
//
//   out_f[x1][i] = sum_h Re(E1f[h][x1] T2[f][h][i]) = sum_k A_f[i][k] B[x1][k]
//   A_f[i][2h] = Re T2[f][h][i],  A_f[i][2h+1] = Im T2[f][h][i]
//   B[x1][2h]  = Re E1f[h][x1],   B[x1][2h+1]  = -Im E1f[h][x1]
//
// a real GEMM D = A B^T with M = 128 grid pencils i per tile, N = N1 (x1,
// padded to a multiple of 16, at most 256) and K = K1 (padded to a multiple of
// 8).  FP32 accuracy from TF32 tensor cores by the 3xTF32 split x = hi + lo
// (hi = TF32 rounding of x): A B^T ~ Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T,
// accumulated in FP32 in tensor memory.
//
// One CTA (256 threads) walks (field, 128-pencil tile) work items:
//   1. all threads write the tile's T2 values (fetched into registers while
//      the previous item ran) into shared memory, hi and lo, in the K-major
//      no-swizzle canonical layout (8 x 16-byte core matrices);
//   2. one thread issues the MMAs into a TMEM accumulator (lane = pencil,
//      column = x1) and commits them to an mbarrier; meanwhile every thread
//      issues the global loads of its next item;
//   3. all threads wait (bounded) and read their TMEM lane quadrant with
//      tcgen05.ld: for each x1 a warp holds 32 consecutive pencils and stores
//      them as one 128-byte row segment straight from registers.
// B (the twiddles) is staged once per CTA.  At least 96 KB of shared memory
// keeps at most two CTAs on an SM, so the two 256-column TMEM allocations
// always fit.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_common.cuh"

namespace lddmm {
namespace {

using namespace tc;

constexpr int kThreadsTC = 256;
constexpr int kNT = 128;                 // grid pencils per work item
constexpr int kMT = 128;                 // M tile (TMEM lanes = pencils)
constexpr int kMaxKp = 48;               // K1 <= 48 (shared memory)
constexpr long long kWaitLimit = 1LL << 24;

__global__ void __launch_bounds__(kThreadsTC)
k_iota_C_tc(Plan<float> p, IotaDesc<float> d, const float2* __restrict__ T2, int Kp, int Np, double* flag) {
  extern __shared__ __align__(128) unsigned char smraw[];
  float* sm = reinterpret_cast<float*>(smraw);
  const int tileA = kMT * Kp, tileB = Np * Kp;
  float* Ahi = sm;                                           // data tile (M = 128 pencils)
  float* Alo = Ahi + tileA;
  float* Bhi = Alo + tileA;                                  // twiddles (N = Np rows of x1)
  float* Blo = Bhi + tileB;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + tileB);  // 16-byte aligned (sizes are)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int G1 = p.g.n1, H1 = p.b.h1, K = 2 * H1;
  const long long P = (long long)p.g.n2 * p.g.n3;
  const int ntn = (int)((P + kNT - 1) / kNT);
  const long long nitems = (long long)d.nf * ntn;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & (kNT - 1), h0 = tid >> 7;              // staging: pencil r, slots h0 + 2j

  // B (both halves of the split) and the zero K padding of A, once per CTA;
  // eight twiddle loads per thread in flight at a time
  for (int base = 0; base < Np * Kp; base += 8 * kThreadsTC) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * kThreadsTC + tid;
      const int x1 = idx / Kp, k = idx - x1 * Kp;
      v[u] = 0.f;
      if (idx < Np * Kp && x1 < G1 && k < K) {
        const float2 e = p.E1f[(k >> 1) * G1 + x1];
        v[u] = (k & 1) ? -e.y : e.x;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * kThreadsTC + tid;
      if (idx < Np * Kp) {
        const int x1 = idx / Kp, k = idx - x1 * Kp;
        const float hi = tf32_hi(v[u]);
        const int o = kmajor_off(x1, k, Kp);
        Bhi[o] = hi;
        Blo[o] = v[u] - hi;
      }
    }
  }
  for (int idx = tid; idx < kMT * (Kp - K); idx += kThreadsTC) {
    const int row = idx / (Kp - K), k = K + idx % (Kp - K);
    Ahi[kmajor_off(row, k, Kp)] = 0.f;
    Alo[kmajor_off(row, k, Kp)] = 0.f;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;

  const uint32_t idesc = idesc_tf32(kMT, Np);
  const uint32_t lbo = 128, sbo = (uint32_t)(Kp >> 2) * 128;
  // this thread's T2 values of an item: pencil r, slots h = h0, h0 + 2, ...
  float2 pre[kMaxKp / 4];
  auto fetch = [&](long long item) {
    const int f = (int)(item / ntn);
    const long long n = (item % ntn) * kNT + r;
    const float2* __restrict__ src = T2 + (long long)f * H1 * P + n;
#pragma unroll
    for (int j = 0; j < kMaxKp / 4; ++j) {
      const int h = h0 + 2 * j;
      pre[j] = (h < H1 && n < P) ? src[(long long)h * P] : make_float2(0.f, 0.f);
    }
  };
  uint32_t phase = 0;
  bool ok = true;
  long long item = blockIdx.x;
  if (item < nitems) fetch(item);
  for (; item < nitems && ok; item += gridDim.x) {
    const int f = (int)(item / ntn);
    const long long n0 = (item % ntn) * kNT;
    // 1. A tile, hi and lo, from the fetched registers
#pragma unroll
    for (int j = 0; j < kMaxKp / 4; ++j) {
      const int h = h0 + 2 * j;
      if (h < H1) {
        const float hr = tf32_hi(pre[j].x), hi_ = tf32_hi(pre[j].y);
        const int o = kmajor_off(r, 2 * h, Kp);
        *reinterpret_cast<float2*>(Ahi + o) = make_float2(hr, hi_);
        *reinterpret_cast<float2*>(Alo + o) = make_float2(pre[j].x - hr, pre[j].y - hi_);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 2. MMAs, one issuing thread; everyone fetches the next item meanwhile
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int s = 0; s < Kp / 8; ++s) {
        const uint32_t so = (uint32_t)s * 256;
        const uint64_t ah = smem_desc(smem_u32(Ahi) + so, lbo, sbo);
        const uint64_t al = smem_desc(smem_u32(Alo) + so, lbo, sbo);
        const uint64_t bh = smem_desc(smem_u32(Bhi) + so, lbo, sbo);
        const uint64_t bl = smem_desc(smem_u32(Blo) + so, lbo, sbo);
        mma_tf32(tbase, ah, bh, idesc, s > 0 ? 1u : 0u);
        mma_tf32(tbase, ah, bl, idesc, 1u);
        mma_tf32(tbase, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    if (item + gridDim.x < nitems) fetch(item + gridDim.x);
    // 3. wait for the MMAs (bounded), then store D from registers
    long long it = 0;
    while (!mbar_try_wait(smem_u32(mbar), phase)) {
      if (++it > kWaitLimit) {
        ok = false;
        break;
      }
    }
    phase ^= 1u;
    if (!__syncthreads_and(ok ? 1 : 0)) {
      ok = false;
      if (tid == 0) *(volatile double*)flag = 1.0;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warp w reads lane quadrant w % 4 (pencils n0 + 32 (w % 4) + lane) and
    // every other 16-column chunk of x1, starting at 16 (w / 4)
    const int q = warp & 3, half = warp >> 2;
    const long long n = n0 + 32 * q + (tid & 31);
    float* __restrict__ dst = d.dst[f] + n;
    for (int c = 16 * half; c < Np; c += 32) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
      if (n < P) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < G1) dst[(long long)(c + j) * P] = v[j];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase) : "memory");
}

// The BF16x3 split of the same GEMM: x = hi + mid + lo with hi = bf16(x),
// mid = bf16(x - hi), lo = bf16(x - hi - mid) (24 significant bits), and
//   A B^T ~ Ah Bh + Ah Bm + Am Bh + Ah Bl + Al Bh + Am Bm
// (the dropped products are below 2^-24 of the result), six kind::f16 MMAs
// with BF16 operands (K = 16) per 16 columns of K, FP32 accumulation in tensor
// memory.  Same work items, staging and epilogue as the 3xTF32 kernel above.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

__global__ void __launch_bounds__(kThreadsTC)
k_iota_C_bf3(Plan<float> p, IotaDesc<float> d, const float2* __restrict__ T2, int Kp, int Np, double* flag) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(smraw);
  const int tileA = kMT * Kp, tileB = Np * Kp;
  __nv_bfloat16* A[3] = {sm, sm + tileA, sm + 2 * tileA};             // hi, mid, lo
  __nv_bfloat16* B[3] = {sm + 3 * tileA, sm + 3 * tileA + tileB, sm + 3 * tileA + 2 * tileB};
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 3 * tileA + 3 * tileB);   // 16-byte aligned (sizes are)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int G1 = p.g.n1, H1 = p.b.h1, K = 2 * H1;
  const long long P = (long long)p.g.n2 * p.g.n3;
  const int ntn = (int)((P + kNT - 1) / kNT);
  const long long nitems = (long long)d.nf * ntn;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & (kNT - 1), h0 = tid >> 7;

  for (int idx = tid; idx < Np * Kp; idx += kThreadsTC) {   // twiddles, once per CTA
    const int x1 = idx / Kp, k = idx - x1 * Kp;
    float v = 0.f;
    if (x1 < G1 && k < K) {
      const float2 e = p.E1f[(k >> 1) * G1 + x1];
      v = (k & 1) ? -e.y : e.x;
    }
    __nv_bfloat16 hh, mm, ll;
    split3(v, hh, mm, ll);
    const int o = kmajor_off16(x1, k, Kp);
    B[0][o] = hh;
    B[1][o] = mm;
    B[2][o] = ll;
  }
  for (int idx = tid; idx < kMT * (Kp - K); idx += kThreadsTC) {   // zero K padding of A
    const int row = idx / (Kp - K), k = K + idx % (Kp - K);
    const int o = kmajor_off16(row, k, Kp);
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    A[0][o] = z;
    A[1][o] = z;
    A[2][o] = z;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;

  const uint32_t idesc = idesc_bf16(kMT, Np);
  const uint32_t lbo = 128, sbo = (uint32_t)(Kp >> 3) * 128;
  float2 pre[kMaxKp / 4];
  auto fetch = [&](long long item) {
    const int f = (int)(item / ntn);
    const long long n = (item % ntn) * kNT + r;
    const float2* __restrict__ src = T2 + (long long)f * H1 * P + n;
#pragma unroll
    for (int j = 0; j < kMaxKp / 4; ++j) {
      const int h = h0 + 2 * j;
      pre[j] = (h < H1 && n < P) ? src[(long long)h * P] : make_float2(0.f, 0.f);
    }
  };
  uint32_t phase = 0;
  bool ok = true;
  long long item = blockIdx.x;
  if (item < nitems) fetch(item);
  for (; item < nitems && ok; item += gridDim.x) {
    const int f = (int)(item / ntn);
    const long long n0 = (item % ntn) * kNT;
#pragma unroll
    for (int j = 0; j < kMaxKp / 4; ++j) {
      const int h = h0 + 2 * j;
      if (h < H1) {
        __nv_bfloat16 rh, rm, rl, ih, im, il;
        split3(pre[j].x, rh, rm, rl);
        split3(pre[j].y, ih, im, il);
        const int o = kmajor_off16(r, 2 * h, Kp);
        *reinterpret_cast<__nv_bfloat162*>(A[0] + o) = __halves2bfloat162(rh, ih);
        *reinterpret_cast<__nv_bfloat162*>(A[1] + o) = __halves2bfloat162(rm, im);
        *reinterpret_cast<__nv_bfloat162*>(A[2] + o) = __halves2bfloat162(rl, il);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // (a, b) plane pairs of the six products; the first one starts the sum
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
      for (int s = 0; s < Kp / 16; ++s) {
        const uint32_t so = (uint32_t)s * 256;
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const uint64_t da = smem_desc(smem_u32(A[pa[t]]) + so, lbo, sbo);
          const uint64_t db = smem_desc(smem_u32(B[pb[t]]) + so, lbo, sbo);
          mma_bf16(tbase, da, db, idesc, (s > 0 || t > 0) ? 1u : 0u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    if (item + gridDim.x < nitems) fetch(item + gridDim.x);
    long long it = 0;
    while (!mbar_try_wait(smem_u32(mbar), phase)) {
      if (++it > kWaitLimit) {
        ok = false;
        break;
      }
    }
    phase ^= 1u;
    if (!__syncthreads_and(ok ? 1 : 0)) {
      ok = false;
      if (tid == 0) *(volatile double*)flag = 1.0;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp & 3, half = warp >> 2;
    const long long n = n0 + 32 * q + (tid & 31);
    float* __restrict__ dst = d.dst[f] + n;
    for (int c = 16 * half; c < Np; c += 32) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
      if (n < P) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < G1) dst[(long long)(c + j) * P] = v[j];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase) : "memory");
}

}  // namespace

static int tc_np(int G1) { return ((G1 + 15) / 16) * 16; }

size_t iota_C_tc_smem(int K1, int G1) {
  const int Kp = ((K1 + 7) / 8) * 8;
  return (size_t)(2 * kMT * Kp + 2 * tc_np(G1) * Kp) * sizeof(float) + 16;
}

bool iota_C_tc_supported(const Plan<float>& p) {
  const int Kp = ((2 * p.b.h1 + 7) / 8) * 8;
  if (p.split == 1) {
    const int Kb = ((2 * p.b.h1 + 15) / 16) * 16;
    return tc_np(p.g.n1) <= 256 && Kb <= kMaxKp &&
           (size_t)(3 * kMT * Kb + 3 * tc_np(p.g.n1) * Kb) * 2 + 16 <= 200 * 1024;
  }
  return tc_np(p.g.n1) <= 256 && Kp <= kMaxKp && iota_C_tc_smem(2 * p.b.h1, p.g.n1) <= 200 * 1024;
}

static cudaError_t iota_C_bf3(const Plan<float>& p, const IotaDesc<float>& d, const float2* T2, double* flag,
                              cudaStream_t st) {
  const int Kp = ((2 * p.b.h1 + 15) / 16) * 16;
  const size_t need = (size_t)(3 * kMT * Kp + 3 * tc_np(p.g.n1) * Kp) * 2 + 16;
  // at least 96 KB per CTA: at most two CTAs (two 256-column TMEM allocations) per SM
  const size_t smem = std::max<size_t>(need, 96 * 1024 + 16);
  cudaError_t e = cudaFuncSetAttribute(k_iota_C_bf3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long long P = (long long)p.g.n2 * p.g.n3;
  const long long items = (long long)d.nf * ((P + kNT - 1) / kNT);
  const unsigned grid = (unsigned)std::min<long long>(items, 2LL * sms);
  k_iota_C_bf3<<<grid, kThreadsTC, smem, st>>>(p, d, T2, Kp, tc_np(p.g.n1), flag);
  return cudaGetLastError();
}

cudaError_t iota_C_tc(const Plan<float>& p, const IotaDesc<float>& d, const float2* T2, double* flag,
                      cudaStream_t st) {
  if (p.split == 1) return iota_C_bf3(p, d, T2, flag, st);
  const int Kp = ((2 * p.b.h1 + 7) / 8) * 8;
  // at least 96 KB per CTA: at most two CTAs (two 256-column TMEM allocations) per SM
  const size_t smem = std::max<size_t>(iota_C_tc_smem(2 * p.b.h1, p.g.n1), 96 * 1024 + 16);
  cudaError_t e = cudaFuncSetAttribute(k_iota_C_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long long P = (long long)p.g.n2 * p.g.n3;
  const long long items = (long long)d.nf * ((P + kNT - 1) / kNT);
  const unsigned grid = (unsigned)std::min<long long>(items, 2LL * sms);
  k_iota_C_tc<<<grid, kThreadsTC, smem, st>>>(p, d, T2, Kp, tc_np(p.g.n1), flag);
  return cudaGetLastError();
}

}  // namespace lddmm
