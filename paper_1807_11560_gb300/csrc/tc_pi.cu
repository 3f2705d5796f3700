// Tensor-core (tcgen05, sm_103a) form of pi stages A' and B' with the
// epilogue, on the padded product grid (the last phase of a bracket
// evaluation, Eqs. 46 and 48-49): for one band slab (component c, h) and each
// of the nper product fields o,
//
//   A'  Z_o[x2][k3]  = sum_x3 P_o[x2][x3] E3b[x3][k3]
//   B'  Y_o[k2][k3]  = sum_x2 E2b[x2][k2] Z_o[x2][k3]
//
// two complex GEMMs with inner dimensions G3 and G2, then the combination of
// the Y_o (K~, Heun/Krylov coefficients, X terms) into the band outputs.  In
// real form (re/im interleaved) each is a TN GEMM D = A B^T on tcgen05 with the
// 3xTF32 split of both operands (A B^T ~ Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T,
// FP32 accumulation in tensor memory):
//   A': D[x2][(k3, c)] = sum_(x3, c') P[x2][(x3, c')] E3x[(k3, c)][(x3, c')]
//       M = G2 rows, N = 2 K3, K = 2 G3.  A slab of P is G2 rows of 2 G3
//       contiguous floats, exactly the operand's K order, so it is staged with
//       16-byte loads;
//   B': D[k3][(k2, c)] = sum_(x2, c') Z[k3][(x2, c')] E2x[(k2, c)][(x2, c')]
//       M = K3 rows, N = 2 K2, K = 2 G2; its operand is D of A' read from
//       tensor memory (lane = x2) and written transposed into the K-major
//       layout, each lane walking its k3 values in a lane-rotated order so a
//       warp's shared-memory writes spread over the banks.
// E3x, E2x are the real forms of the pi twiddles ([[re, -im], [im, re]]
// blocks), expanded once per context into the shared-memory layout and copied
// into each CTA.  One CTA per (c, h, o); the nper CTAs of a slab form a thread
// block cluster, and the epilogue (which combines the nper fields) reads the
// Y_o of the peers through distributed shared memory, each CTA finishing a
// share of the slab's band slots.  One thread finishes every output of a slot,
// reading all of the slot's X terms before writing (outputs may alias them).
// Every MMA wait is bounded (a give-up sets the flag the host reads) and every
// CTA passes both cluster barriers whatever its waits returned.
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_common.cuh"

namespace lddmm {
namespace {

using namespace tc;

constexpr int kThrP = 256;
constexpr int kWarpsP = kThrP / 32;
constexpr long long kWaitP = 1LL << 24;
constexpr int kLdA = 8;    // 16-byte loads of the slab per thread, all in flight at once

struct PiTc {
  int KA, KB;        // K of stages A' (2 G3) and B' (2 G2)
  int NA, NB;        // N of stages A' (2 K3) and B' (2 K2)
  int rows;          // operand rows stored (max(G2, K3), rounded up to 8)
  int tw;            // floats of the twiddle buffer (hi + lo of the larger stage)
  int tcols;         // TMEM columns allocated
};

// real form of a complex twiddle: row (k, c) of the output, column (x, c')
__host__ __device__ __forceinline__ float twr(float2 e, int c, int cp) {
  return c == 0 ? (cp == 0 ? e.x : -e.y) : (cp == 0 ? e.y : e.x);
}

__device__ __forceinline__ bool nyqp(int q, int K) { return (K % 2 == 0) && (2 * q == K); }

__device__ __forceinline__ void cp_async16p(void* dst, const void* src) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(src) : "memory");
}

// 32-bit shared-memory address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 ld_peer(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// the expanded twiddle operands [E3x hi | E3x lo | E2x hi | E2x lo] in the
// K-major layouts of their shared-memory tiles, one element per thread
__global__ void k_pi_tc_twiddles(Plan<float> p, float* dst, int NA, int KA, int NB, int KB) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nA = (long long)NA * KA, nB = (long long)NB * KB;
  if (i >= nA + nB) return;
  const bool isA = i < nA;
  const int Kx = isA ? KA : KB;
  const int e = (int)(isA ? i : i - nA);
  const int n = e / Kx, k = e - n * Kx;        // n = (kout, c), k = (x, c')
  float v;
  if (isA) v = twr(p.E3b[(long long)(k >> 1) * p.b.k3 + (n >> 1)], n & 1, k & 1);
  else v = twr(p.E2b[(long long)(k >> 1) * p.b.k2 + (n >> 1)], n & 1, k & 1);
  const float h = tf32_hi(v);
  float* base = isA ? dst : dst + 2 * nA;
  const int o = kmajor_off(n, k, Kx);
  base[o] = h;
  base[(isA ? nA : nB) + o] = v - h;
}

// Sizes known at compile time for the common padded grid (0: read at run time).
template <int G2c, int G3c, int K2c, int K3c>
__global__ void __launch_bounds__(kThrP)
k_pi_ba_tc(Plan<float> p, PiEpi<float> e, const float* __restrict__ Lhat, const float2* __restrict__ P2,
           PiTc g, double* flag) {
  extern __shared__ __align__(128) unsigned char smraw[];
  float* sm = reinterpret_cast<float*>(smraw);
  const int G2 = G2c ? G2c : p.g.n2, G3 = G3c ? G3c : p.g.n3, K2 = K2c ? K2c : p.b.k2, K3 = K3c ? K3c : p.b.k3;
  const int KA = 2 * G3, KB = 2 * G2, NA = 2 * K3, NB = 2 * K2;
  const int Kmax = KA > KB ? KA : KB;
  // Shared memory: the A operand's stored rows (G2 for A', K3 for B'), hi then
  // lo, then one twiddle buffer holding E3x for stage A' and then E2x for stage
  // B'.  An MMA reads 128 rows of A; the rows past the stored ones fall inside
  // this allocation (checked on the host) and only feed accumulator rows that
  // are never read.  Keeping the CTA under half the SM's shared memory lets
  // two CTAs share an SM, so every cluster of a launch is resident at once.
  const int R = g.rows * Kmax;
  float* Ahi = sm;                                  // A operand (stage A', then stage B')
  float* Alo = sm + R;
  float* Bhi = sm + 2 * R;                          // E3x, then E2x
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bhi + g.tw);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  float2* Y = reinterpret_cast<float2*>(sm);        // [K2][K3] after stage B' (aliases the operand)

  const int K1 = p.b.k1, H1 = p.b.h1;
  const int ncomp = e.ncomp, nper = e.nper;
  const long long kvol = (long long)K1 * K2 * K3;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int o = blockIdx.x % nper;                  // = rank in the cluster
  const int item = blockIdx.x / nper;
  const int c = item / H1, h = item - c * H1;

  // programmatic dependent launch: the next kernel may be scheduled now; the
  // prologue reads constants only, the wait precedes the product field
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  auto stage_tw = [&](const float* src, int n) {   // n floats, a multiple of 4
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(Bhi);
    for (int i = tid; i < n / 4; i += kThrP) cp_async16p(d4 + i, s4 + i);
  };
  stage_tw(p.tc_pi, 2 * NA * KA);                   // E3x hi | lo
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
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // 1. stage A' operand: a warp moves tiles of 8 rows x 4 chunks of 16 bytes
  //    (one core matrix per chunk column: conflict-free stores); every load of
  //    a thread is issued before its first store
  const int nq = KA / 4, cgn = (nq + 3) / 4, ntile = (G2 / 8) * cgn;
  const int rr = lane >> 2, qq = lane & 3;
  const float* slab = reinterpret_cast<const float*>(P2 + (long long)((o * ncomp + c) * H1 + h) * G2 * G3);
  float4 ld[kLdA];
#pragma unroll
  for (int u = 0; u < kLdA; ++u) {
    const int t = warp + u * kWarpsP;
    const int Rg = t / cgn, Qg = t - Rg * cgn;
    const int row = 8 * Rg + rr, qi = 4 * Qg + qq;
    ld[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < ntile && qi < nq) ld[u] = *reinterpret_cast<const float4*>(slab + (long long)row * KA + 4 * qi);
  }
#pragma unroll
  for (int u = 0; u < kLdA; ++u) {
    const int t = warp + u * kWarpsP;
    const int Rg = t / cgn, Qg = t - Rg * cgn;
    const int row = 8 * Rg + rr, qi = 4 * Qg + qq;
    if (t >= ntile || qi >= nq) continue;
    const float4 v = ld[u];
    const float4 hv = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
    const int o4 = kmajor_off(row, 4 * qi, KA);
    *reinterpret_cast<float4*>(Ahi + o4) = hv;
    *reinterpret_cast<float4*>(Alo + o4) = make_float4(v.x - hv.x, v.y - hv.y, v.z - hv.z, v.w - hv.w);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");   // the twiddle operands have landed
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;

  const uint32_t idA = idesc_tf32(kMTile, NA), idB = idesc_tf32(kMTile, NB);
  uint32_t phase = 0;
  bool ok = true;
  // both stages accumulate in columns 0 .. N (stage B' after A' has been read)
  auto issue = [&](const float* ah, const float* al, const float* bh, const float* bl, int K, uint32_t stride,
                   uint32_t idesc) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    mma_3xtf32<1>(tbase, stride, ah, al, bh, bl, K, idesc);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
  };
  auto wait = [&]() {
    long long it = 0;
    bool mine = true;
    while (!mbar_try_wait(smem_u32(mbar), phase)) {
      if (++it > kWaitP) {
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
  const int q = warp & 3, cg = warp >> 2;           // lane quadrant, column group (of 2)
  const uint32_t tlane = (uint32_t)(32 * q) << 16;

  if (tid == 0) issue(Ahi, Alo, Bhi, Bhi + NA * KA, KA, (uint32_t)NA, idA);
  if (wait()) {
    stage_tw(p.tc_pi + 2 * NA * KA, 2 * NB * KB);   // E2x hi | lo, in flight during the re-layout
    // 2. D of A' (lane = x2) -> stage B' operand: row k3, K = (x2, c'), each
    //    lane walking its k3 values in a lane-rotated order
    const int x2 = 32 * q + lane;
    if (32 * q < G2) {
      for (int c0 = 16 * cg; c0 < NA; c0 += 32) {
        float v[16];
        tmem_ld16_sum<1>(tbase + tlane + (uint32_t)c0, (uint32_t)NA, v);
        if (x2 < G2) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int ii = (i + lane) & 7;
            const int k3 = (c0 >> 1) + ii;
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int m = 0; m < 8; ++m)
              if (m == ii) {
                re = v[2 * m];
                im = v[2 * m + 1];
              }
            const float hr = tf32_hi(re), hm = tf32_hi(im);
            const int ob = kmajor_off(k3, 2 * x2, KB);
            *reinterpret_cast<float2*>(Ahi + ob) = make_float2(hr, hm);
            *reinterpret_cast<float2*>(Alo + ob) = make_float2(re - hr, im - hm);
          }
        }
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) issue(Ahi, Alo, Bhi, Bhi + NB * KB, KB, (uint32_t)NB, idB);
    if (wait()) {
      // 3. D of B' (lane = k3) -> Y[k2][k3] (the operand area is free again)
      const int k3 = 32 * q + lane;
      if (32 * q < K3) {
        for (int c0 = 16 * cg; c0 < NB; c0 += 32) {
          float v[16];
          tmem_ld16_sum<1>(tbase + tlane + (uint32_t)c0, (uint32_t)NB, v);
          if (k3 < K3) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              Y[((c0 >> 1) + i) * K3 + k3] = make_float2(v[2 * i], v[2 * i + 1]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();                                   // every Y_o of the slab is complete
  // 4. epilogue: the slab's band slots shared among the cluster's CTAs
  if (ok) {
    for (int it = o * kThrP + tid; it < K2 * K3; it += kThrP * nper) {
      const int k2 = it / K3, k3 = it - k2 * K3;
      const bool nq_ = nyqp(k2, K2) || nyqp(k3, K3);
      const long long kin = ((long long)h * K2 + k2) * K3 + k3;
      const long long at = (long long)c * kvol + kin;
      float2 yo[kMaxPer];
#pragma unroll
      for (int r = 0; r < kMaxPer; ++r)
        yo[r] = r < nper ? ld_peer(peer_addr(Y + it, (uint32_t)r)) : make_float2(0.f, 0.f);
      float2 out[kMaxOut];
#pragma unroll
      for (int j = 0; j < kMaxOut; ++j) out[j] = make_float2(0.f, 0.f);
      if (!nq_) {
        const float kh = 1.f / Lhat[kin];
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
          if (j >= e.nout) break;
          float2 v = make_float2(0.f, 0.f);
          if (e.r[j] >= 0) {
            float2 Rj = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < kMaxPer; ++r) {
              if (r < nper && e.grp[r] == e.r[j]) {
                const float sc = e.coef[r] * (e.applyK[r] ? kh : 1.f);
                Rj.x += sc * yo[r].x;
                Rj.y += sc * yo[r].y;
              }
            }
            v.x = e.cR[j] * Rj.x;
            v.y = e.cR[j] * Rj.y;
          }
#pragma unroll
          for (int x = 0; x < kMaxX; ++x) {
            if (x < e.nx[j]) {
              const float2 xv = e.X[j][x][at];
              v.x += e.cX[j][x] * xv.x;
              v.y += e.cX[j][x] * xv.y;
            }
          }
          out[j] = v;
        }
      }
#pragma unroll
      for (int j = 0; j < kMaxOut; ++j) {
        if (j >= e.nout) break;
        e.dst[j][at] = out[j];
        if (h > 0) {
          const long long mir = (long long)c * kvol +
              (((long long)((K1 - h) % K1) * K2 + (K2 - k2) % K2) * K3 + (K3 - k3) % K3);
          e.dst[j][mir] = make_float2(out[j].x, -out[j].y);
        }
        if (h == 0 && K1 % 2 == 0)
          e.dst[j][(long long)c * kvol + (((long long)(K1 / 2) * K2 + k2) * K3 + k3)] = make_float2(0.f, 0.f);
      }
    }
  }
  cluster_sync();                                   // no CTA leaves while a peer reads its Y
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(g.tcols) : "memory");
}

int pow2_cols(int n) {
  int c = 32;
  while (c < n) c *= 2;
  return c;
}

// geometry; false if the plan is outside the kernel's envelope (the SIMT
// kernel runs instead)
bool pi_tc_geom(const Plan<float>& p, int nper, PiTc& g, size_t& smem) {
  const int K2 = p.b.k2, K3 = p.b.k3, G2 = p.g.n2, G3 = p.g.n3;
  if (G2 % 8 != 0 || G3 % 4 != 0 || K2 % 8 != 0 || K3 % 8 != 0) return false;
  if (G2 > kMTile || K3 > kMTile || nper < 1 || nper > kMaxPer) return false;
  g.KA = 2 * G3;
  g.KB = 2 * G2;
  g.NA = 2 * K3;
  g.NB = 2 * K2;
  if (g.NA > 256 || g.NB > 256 || g.NA % 16 != 0 || g.NB % 16 != 0) return false;
  if ((G2 / 8) * ((g.KA / 4 + 3) / 4) > kLdA * kWarpsP) return false;   // the slab's loads in registers
  g.tcols = pow2_cols(std::max(g.NA, g.NB));       // stage B' reuses the columns of stage A'
  if (g.tcols > 256) return false;                  // two CTAs per SM
  const int Kmax = std::max(g.KA, g.KB);
  g.rows = (std::max(G2, K3) + 7) / 8 * 8;
  g.tw = 2 * std::max(g.NA * g.KA, g.NB * g.KB);
  if ((size_t)K2 * K3 * 2 > (size_t)g.rows * Kmax) return false;   // Y fits the hi rows
  size_t floats = (size_t)2 * g.rows * Kmax + g.tw;
  // the 128-row reads of the lo half stay inside the allocation
  floats = std::max(floats, (size_t)g.rows * Kmax + (size_t)kMTile * Kmax);
  smem = floats * sizeof(float) + 16;
  return smem <= 112 * 1024;
}

template <int G2c, int G3c, int K2c, int K3c>
cudaError_t launch_pi_tc(const Plan<float>& p, const PiEpi<float>& e, const float* Lhat, const float2* P2,
                         const PiTc& g, size_t smem, double* flag, cudaStream_t st) {
  auto kern = k_pi_ba_tc<G2c, G3c, K2c, K3c>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(e.ncomp * p.b.h1 * e.nper));
  cfg.blockDim = dim3(kThrP);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[3];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)e.nper;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1 + chain_attrs(at + 1);
  if ((err = cudaLaunchKernelEx(&cfg, kern, p, e, Lhat, P2, g, flag)) != cudaSuccess) return err;
  return cudaGetLastError();
}

}  // namespace

bool pi_ba_tc_supported(const Plan<float>& p) {
  PiTc g;
  size_t smem = 0;
  return pi_tc_geom(p, 3, g, smem) && pi_tc_geom(p, 1, g, smem);
}

size_t pi_ba_tc_twiddle_floats(const Plan<float>& p) {
  PiTc g;
  size_t smem = 0;
  if (!pi_tc_geom(p, 1, g, smem)) return 0;
  return (size_t)2 * g.NA * g.KA + (size_t)2 * g.NB * g.KB;
}

cudaError_t pi_ba_tc_twiddles(const Plan<float>& p, float* dst, cudaStream_t st) {
  PiTc g;
  size_t smem = 0;
  if (!pi_tc_geom(p, 1, g, smem)) return cudaErrorInvalidValue;
  const long long n = (long long)g.NA * g.KA + (long long)g.NB * g.KB;
  k_pi_tc_twiddles<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, dst, g.NA, g.KA, g.NB, g.KB);
  return cudaGetLastError();
}

cudaError_t pi_ba_tc(const Plan<float>& p, const PiEpi<float>& e, const float* Lhat, const float2* P2,
                     double* flag, cudaStream_t st) {
  PiTc g;
  size_t smem = 0;
  if (p.tc_pi == nullptr || !pi_tc_geom(p, e.nper, g, smem)) return cudaErrorInvalidValue;
  if (p.g.n2 == 48 && p.g.n3 == 48 && p.b.k2 == 32 && p.b.k3 == 32)
    return launch_pi_tc<48, 48, 32, 32>(p, e, Lhat, P2, g, smem, flag, st);
  return launch_pi_tc<0, 0, 0, 0>(p, e, Lhat, P2, g, smem, flag, st);
}

}  // namespace lddmm
