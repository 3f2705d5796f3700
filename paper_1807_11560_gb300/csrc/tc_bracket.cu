// Tensor-core (tcgen05, sm_103a) form of iota stages A and B on the padded
// product grid (the first phase of a bracket evaluation, Eqs. 46 and 48):
// for a band slab (field f, h) with its spectral multiplier applied,
//
//   A   S1[k2][x3]  = sum_k3 S0[k2][k3] E3[k3][x3]
//   B   T2[x2][x3]  = sum_k2 E2[k2][x2] S1[k2][x3]
//
// two complex GEMMs with inner dimensions K3 and K2.  In real form (re/im
// interleaved along every dimension) each is a TN GEMM D = A B^T on tcgen05
// with the 3xTF32 split of both operands:
//   A: D_A[(s, k2)][(x3, c)] = sum_(k3, c') S0[(s, k2)][(k3, c')] E3x[(x3, c)][(k3, c')]
//      M = S slabs x K2 rows (one 128-row tile), N = 2 G3, K = 2 K3;
//   B: D_B[(s, x3)][(x2, c)] = sum_(k2, c') S1[(s, x3)][(k2, c')] E2x[(x2, c)][(k2, c')]
//      M = S G3 rows in 128-row passes, N = 2 G2, K = 2 K2,
// where E3x, E2x are the real forms of the twiddles ([[re, -im], [im, re]]
// blocks), staged once per CTA.  D_A leaves TMEM (lane = (s, k2)) and is
// written into the K-major A operand of stage B (row = (s, x3)), each lane
// walking its x3 values in a lane-rotated order so the warp's shared-memory
// writes spread over the banks.  D_B leaves TMEM with lane = (s, x3), so for
// every x2 a warp stores 32 consecutive x3 of T2 (256 contiguous bytes).
// Global loads are batched (eight per thread in flight); the twiddle operands
// are expanded once per context and copied into each CTA; the common padded
// sizes are compile-time constants.  One CTA of 512 threads per SM (512 TMEM
// columns); every MMA wait is bounded.
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_common.cuh"

namespace lddmm {
namespace {

using namespace tc;

constexpr int kThr = 512;
constexpr int kWarps = kThr / 32;
constexpr long long kWait = 1LL << 24;

struct AbTc {
  int S;        // slabs per work item
  int KA, KB;   // K of stages A and B (2 K3, 2 K2)
  int NA, NB;   // N of stages A and B (2 G3, 2 G2, rounded up to 16)
  int passes;   // 128-row passes of stage B
  int rows;     // operand rows stored (max(S K2, S G3 up to 128), rounded up to 8)
  int tw;       // floats of the twiddle buffer (hi + lo of the larger stage)
  int tcols;    // TMEM columns allocated
  int colB;     // first TMEM column of stage B
};

__device__ __forceinline__ int sfq(int q, int K) { return (2 * q < K) ? q : q - K; }
__device__ __forceinline__ bool nyqq(int q, int K) { return (K % 2 == 0) && (2 * q == K); }

// real form of a complex twiddle: row (x, c) of the output, column (k, c')
__host__ __device__ __forceinline__ float twx(float2 e, int c, int cp) {
  return c == 0 ? (cp == 0 ? e.x : -e.y) : (cp == 0 ? e.y : e.x);
}

__host__ __device__ constexpr int r16d(int n) { return ((n + 15) / 16) * 16; }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(src) : "memory");
}

// the expanded twiddle operands [E3x hi | E3x lo | E2x hi | E2x lo], each in
// the K-major layout of its shared-memory tile, one element per thread
__global__ void k_ab_tc_twiddles(Plan<float> p, float* dst, int NA, int KA, int NB, int KB) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nA = (long long)NA * KA, nB = (long long)NB * KB;
  if (i >= nA + nB) return;
  const bool isA = i < nA;
  const int Kx = isA ? KA : KB;
  const int e = (int)(isA ? i : i - nA);
  const int n = e / Kx, k = e - n * Kx;
  const int G = isA ? p.g.n3 : p.g.n2;
  const float2* E = isA ? p.E3f : p.E2f;
  const float v = (n >> 1) < G ? twx(E[(k >> 1) * G + (n >> 1)], n & 1, k & 1) : 0.f;
  const float h = tf32_hi(v);
  float* base = isA ? dst : dst + 2 * nA;
  const int o = kmajor_off(n, k, Kx);
  base[o] = h;
  base[(isA ? nA : nB) + o] = v - h;
}

// sizes known at compile time for the common padded grids (0: read at run time),
// so the index arithmetic of the staging loops folds to constants
template <int K2c, int K3c, int G2c, int G3c>
__global__ void __launch_bounds__(kThr)
k_iota_ab_tc(Plan<float> p, IotaDesc<float> d, const float* __restrict__ Lhat, float2* __restrict__ T2, AbTc g,
             double* flag) {
  extern __shared__ __align__(128) unsigned char smraw[];
  float* sm = reinterpret_cast<float*>(smraw);
  const int G2 = G2c ? G2c : p.g.n2, G3 = G3c ? G3c : p.g.n3, K2 = K2c ? K2c : p.b.k2, K3 = K3c ? K3c : p.b.k3;
  const int H1 = p.b.h1;
  g.KA = 2 * K3;
  g.KB = 2 * K2;
  g.NA = r16d(2 * G3);
  g.NB = r16d(2 * G2);
  // Shared memory: the A operand's stored rows, hi then lo, then one twiddle
  // buffer holding E3x for stage A and then E2x for stage B (copied from the
  // operands expanded once per context).  An MMA reads 128 rows of A; the rows
  // past the stored ones fall inside this allocation (checked on the host) and
  // only feed accumulator rows that are never read.  The CTA stays under half
  // an SM's shared memory (and TMEM), so two work items share an SM.
  const int R = g.rows * max(g.KA, g.KB);
  float* Ahi = sm;                                  // A operand (stage A, then stage B)
  float* Alo = sm + R;
  float* Bhi = sm + 2 * R;                          // E3x, then E2x
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bhi + g.tw);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int nA2 = 2 * g.NA * g.KA, nB2 = 2 * g.NB * g.KB;   // floats of E3x, E2x (hi + lo)
  auto stage_twx = [&](const float* src, int n) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(Bhi);
    for (int i = threadIdx.x; i < n / 4; i += kThr) cp_async16(d4 + i, s4 + i);
  };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nslab = d.nf * H1;
  const int nitems = (nslab + g.S - 1) / g.S;
  // programmatic dependent launch: let the next kernel be scheduled; the
  // prologue below reads constants only, the wait precedes the band slabs
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  stage_twx(p.tc_ab, nA2);                          // E3x hi | lo
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(g.tcols)
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
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const uint32_t idA = idesc_tf32(kMTile, g.NA), idB = idesc_tf32(kMTile, g.NB);
  uint32_t phase = 0;
  bool ok = true;
  // one 3xTF32 product tile: D (+)= Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T
  auto issue = [&](uint32_t dcol, uint32_t stride, const float* ah, const float* al, const float* bh,
                   const float* bl, int K, uint32_t idesc) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    mma_3xtf32<1>(dcol, stride, ah, al, bh, bl, K, idesc);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
  };
  // bounded wait for the last commit; every thread polls, all agree
  auto wait = [&]() {
    long long it = 0;
    bool mine = true;
    while (!mbar_try_wait(smem_u32(mbar), phase)) {
      if (++it > kWait) {
        mine = false;
        break;
      }
    }
    phase ^= 1u;
    ok = __syncthreads_and(mine ? 1 : 0) != 0;
    if (!ok && tid == 0) *(volatile double*)flag = 1.0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return ok;
  };
  const int q = warp & 3, cg = warp >> 2;          // lane quadrant, column group (of 4)
  const uint32_t tlane = (uint32_t)(32 * q) << 16;

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int sl0 = item * g.S;
    if (item != (int)blockIdx.x) stage_twx(p.tc_ab, nA2);   // E3x again (E2x held the buffer)
    // 1. stage A operand: the multiplied band slabs, rows (s, k2), K = (k3, c).
    //    A warp takes 8 x 4 tiles (8 rows k2 x 4 columns k3): full 32-byte
    //    sectors from global memory and at most 2-way bank conflicts in the
    //    K-major layout; eight tiles' loads in flight per thread.
    {
      const int t2 = K2 / 8, t3 = K3 / 4, ntile = g.S * t2 * t3;
      const int r8 = lane >> 2, c4 = lane & 3;
      for (int base = warp; base < ntile; base += 8 * kWarps) {
        float2 a[8];
        float l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = base + u * kWarps;
          a[u] = make_float2(0.f, 0.f);
          l[u] = 1.f;
          if (t < ntile) {
            const int j = t / (t2 * t3), rem = t - j * (t2 * t3);
            const int k2 = (rem / t3) * 8 + r8, k3 = (rem % t3) * 4 + c4;
            const int sl = sl0 + j;
            if (sl < nslab) {
              const int f = sl / H1, h = sl - f * H1;
              const long long off = ((long long)h * K2 + k2) * K3 + k3;
              a[u] = d.src[f][off];
              if (d.applyL[f]) l[u] = Lhat[off];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = base + u * kWarps;
          if (t >= ntile) continue;
          const int j = t / (t2 * t3), rem = t - j * (t2 * t3);
          const int k2 = (rem / t3) * 8 + r8, k3 = (rem % t3) * 4 + c4;
          const int sl = sl0 + j;
          float2 v = make_float2(0.f, 0.f);
          if (sl < nslab && !nyqq(k2, K2) && !nyqq(k3, K3)) {
            const int f = sl / H1, h = sl - f * H1;
            v = a[u];
            v.x *= l[u];
            v.y *= l[u];
            const int dv = d.deriv[f];
            if (dv >= 0) {
              const float fr = dv == 0 ? (float)h : (dv == 1 ? (float)sfq(k2, K2) : (float)sfq(k3, K3));
              const float w = (float)6.283185307179586476925286766559 * fr;
              const float vx = -v.y * w;
              v.y = v.x * w;
              v.x = vx;
            }
          }
          const float hr = tf32_hi(v.x), hm = tf32_hi(v.y);
          const int o = kmajor_off(j * K2 + k2, 2 * k3, g.KA);
          *reinterpret_cast<float2*>(Ahi + o) = make_float2(hr, hm);
          *reinterpret_cast<float2*>(Alo + o) = make_float2(v.x - hr, v.y - hm);
        }
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");       // E3x has landed
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // stage A in columns [0, 2 NA); stage B in the same columns when one pass
    // reads stage A's result once, else after them (every pass re-reads it)
    if (tid == 0) issue(tbase, (uint32_t)g.NA, Ahi, Alo, Bhi, Bhi + g.NA * g.KA, g.KA, idA);
    if (!wait()) break;
    stage_twx(p.tc_ab + nA2, nB2);                 // E2x hi | lo, in flight during the re-layout
    // 2. D_A -> stage B operand, 128 rows (s, x3) per pass
    const int r = 32 * q + lane;                     // D_A row (s, k2)
    const int js = r / K2, k2 = r - js * K2;
    for (int ps = 0; ps < g.passes; ++ps) {
      if (ps > 0 && !wait()) break;                  // the previous pass has read the operand
      for (int c0 = 16 * cg; c0 < g.NA; c0 += 64) {
        float v[16];
        tmem_ld16_sum<1>(tbase + tlane + (uint32_t)c0, (uint32_t)g.NA, v);
        if (js < g.S) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int ii = (i + lane) & 7;
            const int x3 = (c0 >> 1) + ii;
            const int row = js * G3 + x3 - ps * kMTile;
            if (x3 < G3 && row >= 0 && row < kMTile) {
              float re = 0.f, im = 0.f;                 // v[2 ii], v[2 ii + 1] from registers
#pragma unroll
              for (int m = 0; m < 8; ++m)
                if (m == ii) {
                  re = v[2 * m];
                  im = v[2 * m + 1];
                }
              const float hr = tf32_hi(re), hm = tf32_hi(im);
              const int o = kmajor_off(row, 2 * k2, g.KB);
              *reinterpret_cast<float2*>(Ahi + o) = make_float2(hr, hm);
              *reinterpret_cast<float2*>(Alo + o) = make_float2(re - hr, im - hm);
            }
          }
        }
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");     // E2x has landed
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (tid == 0)
        issue(tbase + (uint32_t)(g.colB + ps * g.NB), (uint32_t)g.NB, Ahi, Alo, Bhi, Bhi + g.NB * g.KB, g.KB, idB);
    }
    if (!ok || !wait()) break;
    // 3. D_B -> T2[f][h][x2][x3]
    for (int ps = 0; ps < g.passes; ++ps) {
      const int row = ps * kMTile + 32 * q + lane;    // (s, x3)
      const int jj = row / G3, x3 = row - jj * G3;
      const int sl = sl0 + jj;
      const bool live = jj < g.S && sl < nslab;
      float2* __restrict__ dst = T2 + (long long)(live ? sl : 0) * G2 * G3 + x3;
      for (int c0 = 16 * cg; c0 < g.NB; c0 += 64) {
        float v[16];
        tmem_ld16_sum<1>(tbase + tlane + (uint32_t)(g.colB + ps * g.NB + c0), (uint32_t)g.NB, v);
        if (live) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int x2 = (c0 >> 1) + i;
            if (x2 < G2) dst[(long long)x2 * G3] = make_float2(v[2 * i], v[2 * i + 1]);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(g.tcols) : "memory");
}

int r16(int n) { return ((n + 15) / 16) * 16; }

int pow2t(int n) {
  int c = 32;
  while (c < n) c *= 2;
  return c;
}

bool ab_tc_geom(const Plan<float>& p, AbTc& g, size_t& smem) {
  const int K2 = p.b.k2, K3 = p.b.k3, G2 = p.g.n2, G3 = p.g.n3;
  if (K2 % 8 != 0 || K3 % 4 != 0 || K2 > kMTile) return false;
  g.KA = 2 * K3;
  g.KB = 2 * K2;
  g.NA = r16(2 * G3);
  g.NB = r16(2 * G2);
  if (g.NA > 256 || g.NB > 256) return false;
  // about 64 rows of band slabs per item: enough items for every SM, and a
  // short chain per item
  g.S = std::max(1, std::min(kMTile / K2, 64 / K2));
  g.passes = (g.S * G3 + kMTile - 1) / kMTile;
  // stage B reuses stage A's columns when a single pass reads stage A's
  // result once
  g.colB = g.passes == 1 ? 0 : g.NA;
  g.tcols = pow2t(std::max(g.NA, g.colB + g.passes * g.NB));
  if (g.tcols > 256) return false;                  // two items per SM
  const int Kmax = std::max(g.KA, g.KB);
  g.rows = (std::max(g.S * K2, std::min(g.S * G3, kMTile)) + 7) / 8 * 8;
  g.tw = 2 * std::max(g.NA * g.KA, g.NB * g.KB);
  size_t floats = (size_t)2 * g.rows * Kmax + g.tw;
  // the 128-row reads of the lo half stay inside the allocation
  floats = std::max(floats, (size_t)g.rows * Kmax + (size_t)kMTile * Kmax);
  smem = floats * sizeof(float) + 16;
  return smem <= 112 * 1024;
}

}  // namespace

bool iota_ab_tc_supported(const Plan<float>& p) {
  AbTc g;
  size_t smem = 0;
  return ab_tc_geom(p, g, smem);
}

size_t iota_ab_tc_twiddle_floats(const Plan<float>& p) {
  AbTc g;
  size_t smem = 0;
  if (!ab_tc_geom(p, g, smem)) return 0;
  return (size_t)2 * g.NA * g.KA + (size_t)2 * g.NB * g.KB;
}

cudaError_t iota_ab_tc_twiddles(const Plan<float>& p, float* dst, cudaStream_t st) {
  AbTc g;
  size_t smem = 0;
  if (!ab_tc_geom(p, g, smem)) return cudaErrorInvalidValue;
  const long long n = (long long)g.NA * g.KA + (long long)g.NB * g.KB;
  k_ab_tc_twiddles<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, dst, g.NA, g.KA, g.NB, g.KB);
  return cudaGetLastError();
}

template <int K2c, int K3c, int G2c, int G3c>
cudaError_t launch_ab_tc(const Plan<float>& p, const IotaDesc<float>& d, const float* Lhat, float2* T2,
                         const AbTc& g, size_t smem, double* flag, cudaStream_t st) {
  auto kern = k_iota_ab_tc<K2c, K3c, G2c, G3c>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int nitems = (d.nf * p.b.h1 + g.S - 1) / g.S;
  const unsigned grid = (unsigned)std::min(nitems, 2 * sms);
  // programmatic stream serialisation: the prologue (twiddle copy, TMEM
  // allocation) overlaps the tail of the previous kernel
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  cfg.attrs = at;
  cfg.numAttrs = chain_attrs(at);
  if ((e = cudaLaunchKernelEx(&cfg, kern, p, d, Lhat, T2, g, flag)) != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t iota_ab_tc(const Plan<float>& p, const IotaDesc<float>& d, const float* Lhat, float2* T2,
                       double* flag, cudaStream_t st) {
  AbTc g;
  size_t smem = 0;
  if (!ab_tc_geom(p, g, smem)) return cudaErrorInvalidValue;
  if (p.tc_ab == nullptr) return cudaErrorInvalidValue;
  const int K2 = p.b.k2, K3 = p.b.k3, G2 = p.g.n2, G3 = p.g.n3;
  if (K2 == 32 && K3 == 32 && G2 == 48 && G3 == 48)
    return launch_ab_tc<32, 32, 48, 48>(p, d, Lhat, T2, g, smem, flag, st);
  if (K2 == 24 && K3 == 24 && G2 == 36 && G3 == 36)
    return launch_ab_tc<24, 24, 36, 36>(p, d, Lhat, T2, g, smem, flag, st);
  return launch_ab_tc<0, 0, 0, 0>(p, d, Lhat, T2, g, smem, flag, st);
}

}  // namespace lddmm
