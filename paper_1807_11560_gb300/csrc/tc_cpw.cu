// Tensor-core (tcgen05, sm_103a) form of the middle phase of a bracket
// evaluation on the padded product grid (Eqs. 46, 48-49): for a tile of TP
// pencils (x2, x3) and every x1,
//
//   C   g_f[x1][p]  = sum_h Re(E1f[h][x1] T2[f][h][p])     24 fields f
//       the bracket products of the mode (P / Q of Eqs. 4, 49) at every point
//   C'  P2[q][h][p] = sum_x1 E1b[x1][h] prod_q[x1][p]        3 or 9 fields q
//
// C and C' are real GEMMs on tcgen05 with the 3xTF32 split of both operands
// (FP32 accumulation in tensor memory):
//   C:  D[(f, pp)][x1]     = sum_(h, c') T2x[(f, pp)][(h, c')] E1fx[x1][(h, c')]
//       M = 24 TP rows in 128-row tiles, N = G1, K = 2 H1 (re/im interleaved;
//       E1fx holds Re E1f and -Im E1f, so the real part comes out directly);
//   C': D[(q, pp)][(h, c)] = sum_x1 prod[(q, pp)][x1] E1bx[(h, c)][x1]
//       M = NP TP rows, N = 2 H1, K = G1.
// Between them the 24 grid values of each point go from tensor memory (lane =
// (field, pencil)) through shared memory to the thread of the point, which
// forms the products (with the stage-point fields cached by the forward sweep,
// prefetched at the start) and writes them into the K-major operand of C'.
// The forward sweep's cache slot (tile-major [tile][24][G1][TP]) is written
// here too.  The twiddle operands are expanded once per context.  Shared
// memory stays under half an SM, so two tiles share an SM; the 128-row reads
// of the MMAs past the stored rows fall inside the allocation (checked on the
// host) and feed accumulator rows that are never read.  Every MMA wait is
// bounded; a give-up sets the flag the host reads.
#include <algorithm>
#include <cstdint>

#include "bracket.cuh"
#include "tc_common.cuh"

namespace lddmm {
namespace {

using namespace tc;

constexpr int kThrC = 256;
constexpr int kWarpsC = kThrC / 32;
constexpr int kTPc = 8;                 // pencils per tile
constexpr long long kWaitC = 1LL << 24;

struct CpwTc {
  int N1, K1;        // stage C: N = G1, K = 2 H1
  int N2, K2;        // stage C': N = 2 H1, K = G1
  int rows1, tiles1; // stage C rows (24 TP) and 128-row tiles
  int rows2s;        // stage C' rows stored (NP TP, rounded up to 8)
  int SF;            // row stride (floats) of one field's [G1][TP] block of the grid values
  int off_a2lo, off_a1hi, off_a1lo, off_b1, off_b2, off_bar;   // float offsets in shared memory
  int tcols;
};

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(src) : "memory");
}

// the twiddle operands [E1fx hi | lo | E1bx hi | lo], K-major, one element per thread
__global__ void k_cpw_tc_twiddles(Plan<float> p, float* dst, int N1, int K1, int N2, int K2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n1 = (long long)N1 * K1, n2 = (long long)N2 * K2;
  if (i >= n1 + n2) return;
  const int G1 = p.g.n1, H1 = p.b.h1;
  float v;
  int o, Kx;
  float* base;
  long long nn;
  if (i < n1) {                          // row x1, column (h, c'): Re E1f, -Im E1f
    const int x1 = (int)(i / K1), k = (int)(i % K1);
    const float2 e = p.E1f[(long long)(k >> 1) * G1 + x1];
    v = (k & 1) ? -e.y : e.x;
    o = kmajor_off(x1, k, K1);
    base = dst;
    nn = n1;
  } else {                               // row (h, c), column x1: Re E1b, Im E1b
    const long long j = i - n1;
    const int n = (int)(j / K2), x1 = (int)(j % K2);
    const float2 e = p.E1b[(long long)x1 * H1 + (n >> 1)];
    v = (n & 1) ? e.y : e.x;
    o = kmajor_off(n, x1, K2);
    base = dst + 2 * n1;
    nn = n2;
  }
  const float h = tf32_hi(v);
  base[o] = h;
  base[nn + o] = v - h;
}

template <int MODE>
__global__ void __launch_bounds__(kThrC)
k_cpw_tc(Plan<float> p, const float2* __restrict__ T2, float* __restrict__ slot, float* __restrict__ slot2,
         float2* __restrict__ P2, CpwTc g, double* flag) {
  constexpr int NP = (MODE == PW_GT) ? 9 : 3;
  constexpr int TP = kTPc;
  extern __shared__ __align__(128) unsigned char smraw[];
  float* sm = reinterpret_cast<float*>(smraw);
  float* A2hi = sm;
  float* A2lo = sm + g.off_a2lo;
  float* A1hi = sm + g.off_a1hi;
  float* A1lo = sm + g.off_a1lo;
  float* B1 = sm + g.off_b1;               // hi | lo
  float* B2 = sm + g.off_b2;               // hi | lo
  float* sG = A1hi;                        // [24][SF] grid values, after stage C (aliases its operand)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + g.off_bar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long P = (long long)p.g.n2 * p.g.n3;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long p0 = (long long)blockIdx.x * TP;

  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  {                                                 // twiddle operands (constants)
    const int n4 = (2 * g.N1 * g.K1 + 2 * g.N2 * g.K2) / 4;
    const float4* src = reinterpret_cast<const float4*>(p.tc_cpw);
    float4* d1 = reinterpret_cast<float4*>(B1);
    for (int i = tid; i < n4; i += kThrC) cp16(d1 + i, src + i);
  }
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

  // 1. stage C operand: T2[f][h][p0 .. p0 + TP) -> row (f, pp), K = (h, c');
  //    one float4 = two pencils of one (f, h); every load issued before the
  //    first store.  The cached stage-point fields of this thread's product
  //    points are fetched in the same batch.
  constexpr int kLd = 24 * 16 * (TP / 2) / kThrC;   // float4 per thread at H1 <= 16
  const int nld = 24 * H1 * (TP / 2);
  float4 ld[kLd];
#pragma unroll
  for (int u = 0; u < kLd; ++u) {
    const int i = tid + u * kThrC;
    ld[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < nld) {
      const int fh = i / (TP / 2), j = i - fh * (TP / 2);
      ld[u] = *reinterpret_cast<const float4*>(T2 + (long long)fh * P + p0 + 2 * j);
    }
  }
  const float* tsl = slot + (long long)blockIdx.x * 24 * G1 * TP;   // this tile's cache block
  float cv[2][12], cl[2][12];
  if (MODE != PW_F) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = tid + r * kThrC;                // point (x1, pp), pp fastest
      const bool okp = i < G1 * TP;
#pragma unroll
      for (int f = 0; f < 12; ++f) {
        cv[r][f] = okp ? tsl[f * G1 * TP + i] : 0.f;
        cl[r][f] = okp ? tsl[(12 + f) * G1 * TP + i] : 0.f;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kLd; ++u) {
    const int i = tid + u * kThrC;
    if (i >= nld) continue;
    const int fh = i / (TP / 2), j = i - fh * (TP / 2);
    const int f = fh / H1, h = fh - f * H1;
    const float4 v = ld[u];
    const int row = f * TP + 2 * j;
    const int oa = kmajor_off(row, 2 * h, g.K1), ob = kmajor_off(row + 1, 2 * h, g.K1);
    const float h0 = tf32_hi(v.x), h1 = tf32_hi(v.y), h2 = tf32_hi(v.z), h3 = tf32_hi(v.w);
    *reinterpret_cast<float2*>(A1hi + oa) = make_float2(h0, h1);
    *reinterpret_cast<float2*>(A1lo + oa) = make_float2(v.x - h0, v.y - h1);
    *reinterpret_cast<float2*>(A1hi + ob) = make_float2(h2, h3);
    *reinterpret_cast<float2*>(A1lo + ob) = make_float2(v.z - h2, v.w - h3);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;

  uint32_t phase = 0;
  bool ok = true;
  // one 3xTF32 product tile: D (+)= Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T
  auto issue = [&](uint32_t dcol, uint32_t stride, const float* ah, const float* al, const float* bh,
                   const float* bl, int K, uint32_t idesc) {
    mma_3xtf32<1>(dcol, stride, ah, al, bh, bl, K, idesc);
  };
  auto commit = [&]() {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
  };
  auto wait = [&]() {
    long long it = 0;
    bool mine = true;
    while (!mbar_try_wait(smem_u32(mbar), phase)) {
      if (++it > kWaitC) {
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
  const uint32_t rowsA1 = (uint32_t)(kMTile / 8) * (uint32_t)(g.K1 >> 2) * 32;   // floats per 128 rows

  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t id1 = idesc_tf32(kMTile, g.N1);
    for (int t = 0; t < g.tiles1; ++t)
      issue(tbase + (uint32_t)(t * g.N1), (uint32_t)(g.tiles1 * g.N1), A1hi + t * rowsA1, A1lo + t * rowsA1, B1,
            B1 + g.N1 * g.K1, g.K1, id1);
    commit();
  }
  if (wait()) {
    // 2. grid values: D of C (lane = (f, pp)) -> sG[f][x1][pp]
    const int nunits = g.tiles1 * (g.N1 / 16);
    for (int uidx = cg; uidx < nunits; uidx += 2) {
      const int t = uidx / (g.N1 / 16), c0 = 16 * (uidx - t * (g.N1 / 16));
      const int row = t * kMTile + 32 * q;
      if (row >= g.rows1) continue;                 // the whole warp skips: uniform
      float v[16];
      tmem_ld16_sum<1>(tbase + tlane + (uint32_t)(t * g.N1 + c0), (uint32_t)(g.tiles1 * g.N1), v);
      const int r = row + lane;
      if (r < g.rows1) {
        const int f = r / TP, pp = r - f * TP;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < G1) sG[f * g.SF + (c0 + j) * TP + pp] = v[j];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // 3. bracket products at the tile's points (x1, pp), into the C' operand:
    //    row (q, pp), K = x1
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = tid + r * kThrC;
      if (i >= G1 * TP) break;
      const int x1 = i / TP, pp = i - x1 * TP;
      float xv[12], xl[12];
#pragma unroll
      for (int f = 0; f < 12; ++f) {
        xv[f] = sG[f * g.SF + x1 * TP + pp];
        xl[f] = sG[(12 + f) * g.SF + x1 * TP + pp];
      }
      if (MODE == PW_F) {
        float* ts = slot + (long long)blockIdx.x * 24 * G1 * TP + i;
#pragma unroll
        for (int f = 0; f < 12; ++f) {
          ts[f * G1 * TP] = xv[f];
          ts[(12 + f) * G1 * TP] = xl[f];
        }
      }
      if (MODE == PW_T && slot2 != nullptr) {
        float* ts = slot2 + (long long)blockIdx.x * 24 * G1 * TP + i;
#pragma unroll
        for (int f = 0; f < 12; ++f) {
          ts[f * G1 * TP] = xv[f];
          ts[(12 + f) * G1 * TP] = xl[f];
        }
      }
      float o[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) o[k] = 0.f;
      if (MODE == PW_F) {
        dev::bracketP(xv, xl, o);                   // P(v, L v)
      } else if (MODE == PW_T) {
        dev::bracketP(xv, cl[r], o);                // P(dv, L v)
        dev::bracketP(cv[r], xl, o);                // P(v, L dv)
      } else {
        dev::bracketP(cv[r], xl, o);                // P(v, L U)
        dev::bracketP(xv, cl[r], o + 3);            // P(W, L v)
        dev::bracketQ(cv[r], xv, o + 6);            // Q(v, W)
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int oo = kmajor_off(k * TP + pp, x1, g.K2);
        const float hv = tf32_hi(o[k]);
        A2hi[oo] = hv;
        A2lo[oo] = o[k] - hv;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // C' reuses the columns of C (read out above)
      issue(tbase, (uint32_t)g.N2, A2hi, A2lo, B2, B2 + g.N2 * g.K2, g.K2, idesc_tf32(kMTile, g.N2));
      commit();
    }
    if (wait()) {
      // 4. D of C' (lane = (q, pp)) -> P2[q][h][p0 + pp]
      const int r = 32 * q + lane;
      if (32 * q < NP * TP) {
        for (int c0 = 16 * cg; c0 < g.N2; c0 += 32) {
          float v[16];
          tmem_ld16_sum<1>(tbase + tlane + (uint32_t)c0, (uint32_t)g.N2, v);
          if (r < NP * TP) {
            const int qf = r / TP, pp = r - qf * TP;
            float2* dst = P2 + (long long)qf * H1 * P + p0 + pp;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int h = (c0 >> 1) + j;
              if (h < H1) dst[(long long)h * P] = make_float2(v[2 * j], v[2 * j + 1]);
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(g.tcols) : "memory");
}

int pow2c(int n) {
  int c = 32;
  while (c < n) c *= 2;
  return c;
}

// geometry for NP product fields; false outside the kernel's envelope
bool cpw_tc_geom(const Plan<float>& p, int NP, CpwTc& g, size_t& smem) {
  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long P = (long long)p.g.n2 * p.g.n3;
  if (G1 % 16 != 0 || G1 > 256 || H1 % 4 != 0 || H1 > 16 || P % kTPc != 0) return false;
  if (G1 * kTPc > 2 * kThrC) return false;          // at most two product points per thread
  g.N1 = G1;
  g.K1 = 2 * H1;
  g.N2 = 2 * H1;
  g.K2 = G1;
  if (g.N2 % 16 != 0) return false;
  g.rows1 = 24 * kTPc;
  g.tiles1 = (g.rows1 + kMTile - 1) / kMTile;
  g.rows2s = (NP * kTPc + 7) / 8 * 8;
  if (NP * kTPc > kMTile) return false;
  g.SF = G1 * kTPc + ((G1 * kTPc) % 32 == 0 ? 8 : 0);
  g.tcols = pow2c(std::max(g.tiles1 * g.N1, g.N2));   // C' reuses C's columns
  if (g.tcols > 256) return false;                  // two tiles per SM
  // layout (floats): A2 hi, A2 lo, A1 hi, A1 lo, E1fx hi|lo, E1bx hi|lo, barrier
  const int a2 = g.rows2s * g.K2;
  const int a1 = g.tiles1 * kMTile * g.K1;           // a full tile of rows per 128-row tile
  const int a1s = ((g.rows1 + 7) / 8 * 8) * g.K1;    // rows stored
  g.off_a2lo = a2;
  g.off_a1hi = 2 * a2;
  g.off_a1lo = g.off_a1hi + a1s;
  g.off_b1 = g.off_a1lo + a1s;
  g.off_b2 = g.off_b1 + 2 * g.N1 * g.K1;
  g.off_bar = g.off_b2 + 2 * g.N2 * g.K2;
  if (24 * g.SF > 2 * a1s) return false;            // the grid values fit the stage-C operand area
  // every 128-row MMA read stays inside the allocation
  int end = g.off_bar + 4;
  end = std::max(end, 0 + kMTile * g.K2);
  end = std::max(end, g.off_a2lo + kMTile * g.K2);
  end = std::max(end, g.off_a1hi + a1);
  end = std::max(end, g.off_a1lo + a1);
  smem = (size_t)end * sizeof(float) + 16;
  return smem <= 112 * 1024;
}

}  // namespace

bool cpw_tc_supported(const Plan<float>& p) {
  CpwTc g;
  size_t smem = 0;
  return cpw_tc_geom(p, 3, g, smem) && cpw_tc_geom(p, 9, g, smem);
}

int cpw_tc_tile() { return kTPc; }

size_t cpw_tc_twiddle_floats(const Plan<float>& p) {
  CpwTc g;
  size_t smem = 0;
  if (!cpw_tc_geom(p, 3, g, smem)) return 0;
  return (size_t)2 * g.N1 * g.K1 + (size_t)2 * g.N2 * g.K2;
}

cudaError_t cpw_tc_twiddles(const Plan<float>& p, float* dst, cudaStream_t st) {
  CpwTc g;
  size_t smem = 0;
  if (!cpw_tc_geom(p, 3, g, smem)) return cudaErrorInvalidValue;
  const long long n = (long long)g.N1 * g.K1 + (long long)g.N2 * g.K2;
  k_cpw_tc_twiddles<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, dst, g.N1, g.K1, g.N2, g.K2);
  return cudaGetLastError();
}

cudaError_t cpw_tc(const Plan<float>& p, PwMode mode, const float2* T2, float* slot, float* slot2, float2* P2,
                   double* flag, cudaStream_t st) {
  CpwTc g;
  size_t smem = 0;
  const int NP = mode == PW_GT ? 9 : 3;
  if (p.tc_cpw == nullptr || !cpw_tc_geom(p, NP, g, smem)) return cudaErrorInvalidValue;
  const long long P = (long long)p.g.n2 * p.g.n3;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(P / kTPc));
  cfg.blockDim = dim3(kThrC);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  cfg.attrs = at;
  cfg.numAttrs = chain_attrs(at);
  cudaError_t e;
  switch (mode) {
    case PW_F:
      if ((e = cudaFuncSetAttribute(k_cpw_tc<PW_F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
        return e;
      e = cudaLaunchKernelEx(&cfg, k_cpw_tc<PW_F>, p, T2, slot, slot2, P2, g, flag);
      break;
    case PW_T:
      if ((e = cudaFuncSetAttribute(k_cpw_tc<PW_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
        return e;
      e = cudaLaunchKernelEx(&cfg, k_cpw_tc<PW_T>, p, T2, slot, slot2, P2, g, flag);
      break;
    default:
      if ((e = cudaFuncSetAttribute(k_cpw_tc<PW_GT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
        return e;
      e = cudaLaunchKernelEx(&cfg, k_cpw_tc<PW_GT>, p, T2, slot, slot2, P2, g, flag);
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace lddmm
