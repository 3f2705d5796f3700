// Truncated separable DFTs between band-limited coefficients and grid values
// (iota and pi of Section 3.1, Eq. 46) and the stand-alone kernels of one
// bracket evaluation of ad~* / ad~ (Eqs. 4, 48, 49) on the padded product
// grid, for sm_103a.
//
// iota runs three contractions:
//   A  k3 -> x3   T1[k2][x3]       = sum_k3 m_f(k) a_f(h,k2,k3) E3f[k3][x3]
//   B  k2 -> x2   T2[f][h][x2][x3] = sum_k2 E2f[k2][x2] T1[k2][x3]
//   C  k1 -> x1   out_f[x1][x2][x3] = sum_h Re(E1f[h][x1] T2[f][h][x2][x3])
// where h runs over the non-negative k1 slots only: the field is real, so the
// k1 < 0 half is the conjugate of the k1 > 0 half (E1f carries weight 2 for
// h > 0).  m_f is the field's spectral multiplier (L^ and/or 2 pi i k_j).
// pi runs the transposed contractions C' (x1 -> h), B' (x2 -> k2), A' (x3 -> k3),
// the last one fused with an epilogue that applies K^ = 1/L^, the Heun or
// Krylov linear combination, and writes the k1 < 0 half by conjugation.
//
// Kernels (CTAs of 256 threads; bodies in bracket.cuh):
//   k_iota_AB  CTA per (field, h): A and B through shared memory -> T2.
//   k_iota_C   CTA per (field, 256 pencils): C -> grid field (image-grid
//              transforms); each pencil's K1/2 coefficients read once.
//   k_cpw      CTA per tile of (x2,x3) pencils: C of the 24 fields of a
//              bracket evaluation, the bracket products, C' -> P2.
//   k_pi_C     CTA per (field, 256 pencils): C' of image-grid fields -> P2,
//              each pencil streamed once.
//   k_pi_BA    CTA per (component, h, k2 chunk): B', A', epilogue.
#include <utility>

#include "bracket.cuh"

namespace lddmm {
namespace {

using dev::kThreads;
using dev::kMaxSmem;


template <auto Kernel>
void allow_smem() {
  // one attribute call per kernel instantiation (thread-safe static init)
  static const bool done = [] {
    cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    return true;
  }();
  (void)done;
}

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the previous kernel of the stream still runs (its phase body waits in
// pdl_wait before reading what earlier kernels wrote).  Used for the chain of
// bracket-evaluation kernels, whose prologues (twiddle staging) then overlap
// the tail of the kernel before.  Recorded as programmatic edges when the
// stream is captured into a graph.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), unsigned grid, size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  cfg.attrs = at;
  cfg.numAttrs = chain_attrs(at);
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename T, bool TWS>
__global__ void __launch_bounds__(kThreads)
k_iota_AB(Plan<T> p, IotaDesc<T> d, const T* __restrict__ Lhat, cplx<T>* __restrict__ T2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  dev::pdl_trigger();
  const int f = blockIdx.x / p.b.h1, h = blockIdx.x % p.b.h1;
  const dev::FieldSpec<T> fs{d.src[f], d.deriv[f], d.applyL[f] != 0};
  dev::phase_iota_ab<T, TWS>(p, fs, f, h, Lhat, T2, smraw);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads)
k_cpw(Plan<T> p, const cplx<T>* __restrict__ T2, T* __restrict__ slot, T* __restrict__ slot2,
      cplx<T>* __restrict__ P2, int TP) {
  extern __shared__ __align__(16) unsigned char smraw[];
  dev::pdl_trigger();
  dev::phase_cpw<T, MODE>(p, T2, slot, slot2, P2, TP, blockIdx.x, smraw);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pi_BA(Plan<T> p, PiEpi<T> e, const T* __restrict__ Lhat, const cplx<T>* __restrict__ P2, dev::BAGeom g) {
  extern __shared__ __align__(16) unsigned char smraw[];
  dev::pdl_trigger();
  dev::phase_pi_ba<T>(p, e, Lhat, P2, g, blockIdx.x, smraw);
}

// ---- iota C: half-spectrum k1 -> x1, real output ----------------------------------
// CTA per (field, 256 consecutive (x2,x3) positions): every thread loads the
// H1 complex values of its position once into registers and walks all x1,
// the twiddle row E1f[.][x1] broadcast from shared memory.
constexpr int kMaxH1Reg = 32;
template <typename T, int HR>
__global__ void __launch_bounds__(kThreads)
k_iota_C(Plan<T> p, IotaDesc<T> d, const cplx<T>* __restrict__ T2) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sE = reinterpret_cast<C*>(smraw);                     // [G1][H1] = E1f transposed
  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long inner = (long long)p.g.n2 * p.g.n3;
  const long long nblk = (inner + kThreads - 1) / kThreads;
  const int f = (int)(blockIdx.x / nblk);
  const long long i = (blockIdx.x % nblk) * kThreads + threadIdx.x;
  for (int j = threadIdx.x; j < H1 * G1; j += kThreads) {   // written in shared-memory order
    const int x = j / H1, h = j - x * H1;
    sE[j] = p.E1f[h * G1 + x];
  }
  C a[HR];
  const bool live = i < inner;
  const C* __restrict__ src = T2 + (long long)f * H1 * inner + i;
#pragma unroll
  for (int h = 0; h < HR; ++h) a[h] = (live && h < H1) ? src[(long long)h * inner] : C{T(0), T(0)};
  __syncthreads();
  if (!live) return;
  T* __restrict__ dst = d.dst[f] + i;
  for (int x = 0; x < G1; ++x) {
    const C* e = sE + x * H1;
    T v0 = T(0), v1 = T(0);
#pragma unroll
    for (int h = 0; h < HR; h += 2) {
      if (h < H1) v0 = fma(a[h].x, e[h].x, fma(-a[h].y, e[h].y, v0));
      if (h + 1 < H1) v1 = fma(a[h + 1].x, e[h + 1].x, fma(-a[h + 1].y, e[h + 1].y, v1));
    }
    dst[(long long)x * inner] = v0 + v1;
  }
}

// ---- pi C': real grid x1 -> half-spectrum h ----------------------------------------
// CTA per (field, 256 consecutive positions): each thread streams its pencil
// over x1 once (coalesced) and keeps the H1 complex sums in registers.  The
// pencil is read kPiCBatch rows at a time, all loads of a batch issued before
// its sums, so each thread keeps that many HBM reads in flight; the sums keep
// their x1 order.
constexpr int kPiCBatch = 8;
template <typename T, int HR>
__global__ void __launch_bounds__(kThreads)
k_pi_C(Plan<T> p, PiSrc<T> s, cplx<T>* __restrict__ P2) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sE = reinterpret_cast<C*>(smraw);                     // [G1][H1] = E1b
  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long inner = (long long)p.g.n2 * p.g.n3;
  const long long nblk = (inner + kThreads - 1) / kThreads;
  const int f = (int)(blockIdx.x / nblk);
  const long long i = (blockIdx.x % nblk) * kThreads + threadIdx.x;
  for (int j = threadIdx.x; j < H1 * G1; j += kThreads) sE[j] = p.E1b[j];
  __syncthreads();
  if (i >= inner) return;
  C acc[HR];
#pragma unroll
  for (int h = 0; h < HR; ++h) acc[h] = C{T(0), T(0)};
  const T* __restrict__ src = s.src[f] + i;
  for (int x0 = 0; x0 < G1; x0 += kPiCBatch) {
    T v[kPiCBatch];
#pragma unroll
    for (int u = 0; u < kPiCBatch; ++u) v[u] = x0 + u < G1 ? src[(long long)(x0 + u) * inner] : T(0);
#pragma unroll
    for (int u = 0; u < kPiCBatch; ++u) {
      if (x0 + u >= G1) break;
      const C* e = sE + (x0 + u) * H1;
#pragma unroll
      for (int h = 0; h < HR; ++h)
        if (h < H1) {
          acc[h].x = fma(v[u], e[h].x, acc[h].x);
          acc[h].y = fma(v[u], e[h].y, acc[h].y);
        }
    }
  }
  C* dst = P2 + (long long)f * H1 * inner + i;
#pragma unroll
  for (int h = 0; h < HR; ++h)
    if (h < H1) dst[(long long)h * inner] = acc[h];
}

template <typename T>
void launch_iota_AB(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2, cudaStream_t st,
                    bool pdl = false) {
  const unsigned grid = (unsigned)(d.nf * p.b.h1);
  if (dev::ab_tws(p)) {
    allow_smem<k_iota_AB<T, true>>();
    if (pdl) launch_pdl(k_iota_AB<T, true>, grid, dev::ab_smem(p, true), st, p, d, Lhat, T2);
    else k_iota_AB<T, true><<<grid, kThreads, dev::ab_smem(p, true), st>>>(p, d, Lhat, T2);
  } else {
    allow_smem<k_iota_AB<T, false>>();
    if (pdl) launch_pdl(k_iota_AB<T, false>, grid, dev::ab_smem(p, false), st, p, d, Lhat, T2);
    else k_iota_AB<T, false><<<grid, kThreads, dev::ab_smem(p, false), st>>>(p, d, Lhat, T2);
  }
}

template <typename T>
void launch_pi_BA(const Plan<T>& p, const PiEpi<T>& e, const T* Lhat, const cplx<T>* P2, cudaStream_t st,
                  bool pdl = false) {
  const dev::BAGeom g = dev::ba_geom(p, e.ncomp, e.nper);
  const unsigned grid = (unsigned)(e.ncomp * p.b.h1 * g.nch);
  const size_t smem = dev::ba_smem(p, e.nper, g);
  allow_smem<k_pi_BA<T>>();
  if (pdl) launch_pdl(k_pi_BA<T>, grid, smem, st, p, e, Lhat, P2, g);
  else k_pi_BA<T><<<grid, kThreads, smem, st>>>(p, e, Lhat, P2, g);
}

}  // namespace

template <typename T>
size_t max_smem_needed(const Plan<T>& p, int nper_max, bool brackets) {
  // every B' column of a CTA needs its own accumulators, and the image-grid
  // C/C' kernels keep the K1/2 slots of a pencil in registers
  if ((long long)nper_max * p.g.n3 > (long long)dev::kAccB * kThreads) return ~size_t(0);
  if (p.b.h1 > kMaxH1Reg) return ~size_t(0);
  if ((size_t)p.b.h1 * p.g.n1 * sizeof(cplx<T>) > (size_t)kMaxSmem) return ~size_t(0);
  const size_t ab = dev::ab_smem(p, dev::ab_tws(p));
  if (brackets && p.g.n1 > 2 * kThreads) return ~size_t(0);
  const size_t cpw = brackets ? dev::cpw_smem(p, dev::cpw_tile(p), 9) : 0;
  size_t ba = 0;
  for (int nper = 1; nper <= nper_max; ++nper)
    ba = std::max(ba, dev::ba_smem(p, nper, dev::ba_geom(p, 36, nper)));
  return std::max(ab, std::max(cpw, ba));
}

size_t smem_limit() { return kMaxSmem; }

template <typename T>
void tile_config(const Plan<T>& p, int* tws, int* tp, int* kc) {
  *tws = dev::ab_tws(p) ? 2 : 1;
  *tp = dev::cpw_tile(p);
  *kc = dev::ba_geom(p, 3, 3).KC;
}

template <typename T>
bool tile_valid(const Plan<T>& p, int tws, int tp, int kc) {
  if (tws == 2 && dev::ab_smem(p, true) > (size_t)kMaxSmem) return false;
  if (tp > 0 && !dev::cpw_tile_ok(p, tp)) return false;
  if (kc > p.b.k2 || kc > dev::kMaxKC) return false;
  Plan<T> q = p;
  q.tws = tws;
  q.tp = tp;
  q.kc = kc;
  return max_smem_needed(q, 3, true) <= (size_t)kMaxSmem;
}

template <typename T>
void staged_twiddle_dims(const Plan<T>& p, int* G3e, int* G2e, int* G1q, int* H1q, int* G3s) {
  *G3e = dev::even_up(p.g.n3);
  *G2e = dev::even_up(p.g.n2);
  *G1q = dev::quad_up(p.g.n1);
  *H1q = dev::quad_up(p.b.h1);
  *G3s = dev::e3_stride<T>(p.g.n3);
}

template <typename T>
long long cache_slot_elems(const Plan<T>& p) {
  const long long P = (long long)p.g.n2 * p.g.n3;
  const int TP = dev::cpw_tile(p);
  return 24LL * p.g.n1 * TP * ((P + TP - 1) / TP);
}

// register slots of the image-grid C / C' kernels: the smallest of 8/16/32 >= K1/2
template <typename T, int HR>
void launch_C(const Plan<T>& p, const IotaDesc<T>& d, const cplx<T>* T2, unsigned grid, size_t smem,
              cudaStream_t st) {
  allow_smem<k_iota_C<T, HR>>();
  k_iota_C<T, HR><<<grid, kThreads, smem, st>>>(p, d, T2);
}
template <typename T, int HR>
void launch_Cb(const Plan<T>& p, const PiSrc<T>& s, cplx<T>* P2, unsigned grid, size_t smem, cudaStream_t st) {
  allow_smem<k_pi_C<T, HR>>();
  k_pi_C<T, HR><<<grid, kThreads, smem, st>>>(p, s, P2);
}

template <typename T>
bool try_tc(const Plan<T>&, const IotaDesc<T>&, const cplx<T>*, double*, cudaStream_t) {
  return false;
}
template <>
bool try_tc<float>(const Plan<float>& p, const IotaDesc<float>& d, const float2* T2, double* flag,
                   cudaStream_t st) {
  if (!flag || !iota_C_tc_supported(p)) return false;
  return iota_C_tc(p, d, T2, flag, st) == cudaSuccess;
}

template <typename T>
void iota_c_stage(const Plan<T>& p, const IotaDesc<T>& d, cplx<T>* T2, cudaStream_t st, double* tc_flag) {
  if (try_tc<T>(p, d, T2, tc_flag, st)) return;
  const long long nblk = ((long long)p.g.n2 * p.g.n3 + kThreads - 1) / kThreads;
  const size_t smem = (size_t)p.b.h1 * p.g.n1 * sizeof(cplx<T>);
  const unsigned grid = (unsigned)(d.nf * nblk);
  if (p.b.h1 <= 8) launch_C<T, 8>(p, d, T2, grid, smem, st);
  else if (p.b.h1 <= 16) launch_C<T, 16>(p, d, T2, grid, smem, st);
  else launch_C<T, 32>(p, d, T2, grid, smem, st);
}

template <typename T>
void iota_batch(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2, cudaStream_t st,
                double* tc_flag) {
  launch_iota_AB<T>(p, d, Lhat, T2, st);
  iota_c_stage<T>(p, d, T2, st, tc_flag);
}

template <typename T>
void pi_c_stage(const Plan<T>& p, const PiSrc<T>& s, cplx<T>* P2, cudaStream_t st) {
  const long long nblk = ((long long)p.g.n2 * p.g.n3 + kThreads - 1) / kThreads;
  const size_t smem = (size_t)p.b.h1 * p.g.n1 * sizeof(cplx<T>);
  const unsigned grid = (unsigned)(s.nf * nblk);
  if (p.b.h1 <= 8) launch_Cb<T, 8>(p, s, P2, grid, smem, st);
  else if (p.b.h1 <= 16) launch_Cb<T, 16>(p, s, P2, grid, smem, st);
  else launch_Cb<T, 32>(p, s, P2, grid, smem, st);
}

template <typename T>
void pi_batch(const Plan<T>& p, const PiSrc<T>& s, const PiEpi<T>& e, const T* Lhat, cplx<T>* P2,
              cudaStream_t st) {
  pi_c_stage<T>(p, s, P2, st);
  launch_pi_BA<T>(p, e, Lhat, P2, st);
}

template <typename T>
bool try_ab_tc(const Plan<T>&, const IotaDesc<T>&, const T*, cplx<T>*, double*, cudaStream_t) {
  return false;
}
template <>
bool try_ab_tc<float>(const Plan<float>& p, const IotaDesc<float>& d, const float* Lhat, float2* T2,
                      double* flag, cudaStream_t st) {
  if (!flag || !iota_ab_tc_supported(p)) return false;
  return iota_ab_tc(p, d, Lhat, T2, flag, st) == cudaSuccess;
}

template <typename T>
void bracket_iota(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2, cudaStream_t st,
                  double* tc_flag) {
  if (try_ab_tc<T>(p, d, Lhat, T2, tc_flag, st)) return;
  launch_iota_AB<T>(p, d, Lhat, T2, st, true);
}

template <typename T>
bool try_cpw_tc(const Plan<T>&, PwMode, const cplx<T>*, T*, T*, cplx<T>*, double*, cudaStream_t) {
  return false;
}
template <>
bool try_cpw_tc<float>(const Plan<float>& p, PwMode mode, const float2* T2, float* slot, float* slot2,
                       float2* P2, double* flag, cudaStream_t st) {
  if (!flag || p.tc_cpw == nullptr) return false;
  if (cpw_tc(p, mode, T2, slot, slot2, P2, flag, st) == cudaSuccess) return true;
  cudaGetLastError();   // a refused launch configuration: the SIMT kernel runs instead
  return false;
}

template <typename T>
void bracket_cpw(const Plan<T>& p, PwMode mode, const cplx<T>* T2, T* slot, T* slot2, cplx<T>* P2,
                 cudaStream_t st, double* tc_flag) {
  if (try_cpw_tc<T>(p, mode, T2, slot, slot2, P2, tc_flag, st)) return;
  const int TP = dev::cpw_tile(p);
  const int NP = (mode == PW_GT) ? 9 : 3;
  const size_t smem = dev::cpw_smem(p, TP, NP);
  const long long P = (long long)p.g.n2 * p.g.n3;
  const unsigned grid = (unsigned)((P + TP - 1) / TP);
  switch (mode) {
    case PW_F:
      allow_smem<k_cpw<T, PW_F>>();
      launch_pdl(k_cpw<T, PW_F>, grid, smem, st, p, T2, slot, slot2, P2, TP);
      break;
    case PW_T:
      allow_smem<k_cpw<T, PW_T>>();
      launch_pdl(k_cpw<T, PW_T>, grid, smem, st, p, T2, slot, slot2, P2, TP);
      break;
    case PW_GT:
      allow_smem<k_cpw<T, PW_GT>>();
      launch_pdl(k_cpw<T, PW_GT>, grid, smem, st, p, T2, slot, slot2, P2, TP);
      break;
  }
}

template <typename T>
bool try_pi_tc(const Plan<T>&, const PiEpi<T>&, const T*, const cplx<T>*, double*, cudaStream_t) {
  return false;
}
template <>
bool try_pi_tc<float>(const Plan<float>& p, const PiEpi<float>& e, const float* Lhat, const float2* P2,
                      double* flag, cudaStream_t st) {
  if (!flag || p.tc_pi == nullptr) return false;
  if (pi_ba_tc(p, e, Lhat, P2, flag, st) == cudaSuccess) return true;
  cudaGetLastError();   // a refused launch configuration: the SIMT kernel runs instead
  return false;
}

template <typename T>
void bracket_pi(const Plan<T>& p, const PiEpi<T>& e, const T* Lhat, const cplx<T>* P2, cudaStream_t st,
                double* tc_flag) {
  if (try_pi_tc<T>(p, e, Lhat, P2, tc_flag, st)) return;
  launch_pi_BA<T>(p, e, Lhat, P2, st, true);
}

#define LDDMM_DFT_INST(T)                                                                          \
  template size_t max_smem_needed<T>(const Plan<T>&, int, bool);                                   \
  template long long cache_slot_elems<T>(const Plan<T>&);                                           \
  template void staged_twiddle_dims<T>(const Plan<T>&, int*, int*, int*, int*, int*);               \
  template void tile_config<T>(const Plan<T>&, int*, int*, int*);                                   \
  template bool tile_valid<T>(const Plan<T>&, int, int, int);                                        \
  template void iota_batch<T>(const Plan<T>&, const IotaDesc<T>&, const T*, cplx<T>*, cudaStream_t,    \
                              double*);                                                            \
  template void iota_c_stage<T>(const Plan<T>&, const IotaDesc<T>&, cplx<T>*, cudaStream_t, double*); \
  template void pi_c_stage<T>(const Plan<T>&, const PiSrc<T>&, cplx<T>*, cudaStream_t);             \
  template void pi_batch<T>(const Plan<T>&, const PiSrc<T>&, const PiEpi<T>&, const T*, cplx<T>*,  \
                            cudaStream_t);                                                         \
  template void bracket_iota<T>(const Plan<T>&, const IotaDesc<T>&, const T*, cplx<T>*, cudaStream_t, double*); \
  template void bracket_cpw<T>(const Plan<T>&, PwMode, const cplx<T>*, T*, T*, cplx<T>*, cudaStream_t, double*); \
  template void bracket_pi<T>(const Plan<T>&, const PiEpi<T>&, const T*, const cplx<T>*, cudaStream_t, double*);
LDDMM_DFT_INST(float)
LDDMM_DFT_INST(double)

}  // namespace lddmm
