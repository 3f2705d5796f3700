// Truncated separable DFTs between band-limited coefficients and grid values
// (iota and pi of Section 3.1, Eq. 46), on sm_103a.
//
// iota of a batch of scalar fields runs three stages:
//   A  k3 -> x3   T1[f][h][k2][x3] = sum_k3 m_f(k) a_f(h,k2,k3) E3f[k3][x3]
//   B  k2 -> x2   T2[f][h][x2][x3] = sum_k2 E2f[k2][x2] T1[f][h][k2][x3]
//   C  k1 -> x1   out_f[x1][x2][x3] = sum_h Re(E1f[h][x1] T2[f][h][x2][x3])
// where h runs over the non-negative k1 slots only: the field is real, so the
// k1 < 0 half is the conjugate of the k1 > 0 half and E1f carries weight 2
// for h > 0.  m_f is the field's spectral multiplier (L^ and/or 2 pi i k_j).
// pi runs the transposed stages C' (x1 -> h), B' (x2 -> k2) and A' (x3 -> k3),
// the last one fused with an epilogue that applies K^ = 1/L^, the Heun or
// Krylov linear combination, and writes the k1 < 0 half by conjugation.
//
// Every stage is a batched small complex contraction (inner dimension K/2..G);
// each thread owns YT consecutive outputs along the transformed axis and
// streams the contracted operand from L1/L2 with coalesced loads.
#include "internal.h"

namespace lddmm {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kThreads = 256;

__device__ __forceinline__ int sfreq(int q, int K) { return (2 * q < K) ? q : q - K; }
__device__ __forceinline__ bool nyq(int q, int K) { return (K % 2 == 0) && (2 * q == K); }

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

template <typename C, typename T>
__device__ __forceinline__ void cmac(C& acc, const C& a, const C& e) {
  acc.x = fma(a.x, e.x, fma(-a.y, e.y, acc.x));
  acc.y = fma(a.x, e.y, fma(a.y, e.x, acc.y));
}

// ---- iota stage A: band slab (with multiplier) -> T1 -----------------------
template <typename T, int YT>
__global__ void __launch_bounds__(kThreads)
k_iota_A(Plan<T> p, IotaDesc<T> d, const T* __restrict__ Lhat, cplx<T>* __restrict__ T1) {
  using C = cplx<T>;
  const int G3 = p.g.n3, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  const int nt3 = (G3 + YT - 1) / YT;
  const long long total = (long long)d.nf * H1 * K2 * nt3;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int t3 = (int)(idx % nt3);
  long long r = idx / nt3;
  const int k2 = (int)(r % K2);
  r /= K2;
  const int h = (int)(r % H1);
  const int f = (int)(r / H1);
  const int x0 = t3 * YT;
  C acc[YT];
#pragma unroll
  for (int t = 0; t < YT; ++t) acc[t] = C{T(0), T(0)};
  if (!nyq(k2, K2)) {
    const long long row = ((long long)h * K2 + k2) * K3;
    const C* __restrict__ src = d.src[f] + row;
    const T* __restrict__ Lrow = Lhat + row;
    const int dv = d.deriv[f];
    const bool aL = d.applyL[f] != 0;
    const T frow = (dv == 0) ? T(h) : (dv == 1 ? T(sfreq(k2, K2)) : T(0));
    for (int k3 = 0; k3 < K3; ++k3) {
      if (nyq(k3, K3)) continue;
      C a = src[k3];
      if (aL) { const T l = Lrow[k3]; a.x *= l; a.y *= l; }
      if (dv >= 0) {
        const T w = T(kTwoPi) * ((dv == 2) ? T(sfreq(k3, K3)) : frow);
        const T ax = -a.y * w;
        a.y = a.x * w;
        a.x = ax;
      }
      const C* __restrict__ E = p.E3f + (long long)k3 * G3 + x0;
#pragma unroll
      for (int t = 0; t < YT; ++t)
        if (x0 + t < G3) cmac<C, T>(acc[t], a, E[t]);
    }
  }
  C* out = T1 + (((long long)f * H1 + h) * K2 + k2) * G3 + x0;
#pragma unroll
  for (int t = 0; t < YT; ++t)
    if (x0 + t < G3) out[t] = acc[t];
}

// ---- middle-axis complex contraction: out[b][y][i] = sum_k E[k][y] in[b][k][i]
template <typename T, int YT>
__global__ void __launch_bounds__(kThreads)
k_mid_cc(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out,
         const cplx<T>* __restrict__ E, int B, int nin, int nout, int inner) {
  using C = cplx<T>;
  const int nyt = (nout + YT - 1) / YT;
  const long long total = (long long)B * nyt * inner;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int i = (int)(idx % inner);
  long long r = idx / inner;
  const int ty = (int)(r % nyt);
  const int b = (int)(r / nyt);
  const int y0 = ty * YT;
  C acc[YT];
#pragma unroll
  for (int t = 0; t < YT; ++t) acc[t] = C{T(0), T(0)};
  const C* __restrict__ src = in + (long long)b * nin * inner + i;
  for (int k = 0; k < nin; ++k) {
    const C a = src[(long long)k * inner];
    const C* __restrict__ Ek = E + (long long)k * nout + y0;
#pragma unroll
    for (int t = 0; t < YT; ++t)
      if (y0 + t < nout) cmac<C, T>(acc[t], a, Ek[t]);
  }
  C* dst = out + ((long long)b * nout + y0) * inner + i;
#pragma unroll
  for (int t = 0; t < YT; ++t)
    if (y0 + t < nout) dst[(long long)t * inner] = acc[t];
}

// ---- iota stage C: half-spectrum k1 -> x1, real output ---------------------
template <typename T, int YT>
__global__ void __launch_bounds__(kThreads)
k_iota_C(Plan<T> p, IotaDesc<T> d, const cplx<T>* __restrict__ T2) {
  using C = cplx<T>;
  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long inner = (long long)p.g.n2 * p.g.n3;
  const int nyt = (G1 + YT - 1) / YT;
  const long long total = (long long)d.nf * nyt * inner;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long i = idx % inner;
  long long r = idx / inner;
  const int ty = (int)(r % nyt);
  const int f = (int)(r / nyt);
  const int y0 = ty * YT;
  T acc[YT];
#pragma unroll
  for (int t = 0; t < YT; ++t) acc[t] = T(0);
  const C* __restrict__ src = T2 + (long long)f * H1 * inner + i;
  for (int h = 0; h < H1; ++h) {
    const C a = src[(long long)h * inner];
    const C* __restrict__ Eh = p.E1f + (long long)h * G1 + y0;
#pragma unroll
    for (int t = 0; t < YT; ++t)
      if (y0 + t < G1) acc[t] = fma(a.x, Eh[t].x, fma(-a.y, Eh[t].y, acc[t]));
  }
  T* dst = d.dst[f] + (long long)y0 * inner + i;
#pragma unroll
  for (int t = 0; t < YT; ++t)
    if (y0 + t < G1) dst[(long long)t * inner] = acc[t];
}

// ---- pi stage C': real grid x1 -> half-spectrum h ---------------------------
template <typename T, int YT>
__global__ void __launch_bounds__(kThreads)
k_pi_C(Plan<T> p, PiSrc<T> s, cplx<T>* __restrict__ T2) {
  using C = cplx<T>;
  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long inner = (long long)p.g.n2 * p.g.n3;
  const int nyt = (H1 + YT - 1) / YT;
  const long long total = (long long)s.nf * nyt * inner;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long i = idx % inner;
  long long r = idx / inner;
  const int ty = (int)(r % nyt);
  const int f = (int)(r / nyt);
  const int y0 = ty * YT;
  C acc[YT];
#pragma unroll
  for (int t = 0; t < YT; ++t) acc[t] = C{T(0), T(0)};
  const T* __restrict__ src = s.src[f] + i;
  for (int x = 0; x < G1; ++x) {
    const T a = src[(long long)x * inner];
    const C* __restrict__ Ex = p.E1b + (long long)x * H1 + y0;
#pragma unroll
    for (int t = 0; t < YT; ++t)
      if (y0 + t < H1) {
        acc[t].x = fma(a, Ex[t].x, acc[t].x);
        acc[t].y = fma(a, Ex[t].y, acc[t].y);
      }
  }
  C* dst = T2 + ((long long)f * H1 + y0) * inner + i;
#pragma unroll
  for (int t = 0; t < YT; ++t)
    if (y0 + t < H1) dst[(long long)t * inner] = acc[t];
}

// ---- pi stage A' (x3 -> k3) fused with the epilogue -------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pi_A(Plan<T> p, PiEpi<T> e, const T* __restrict__ Lhat, const cplx<T>* __restrict__ T1) {
  using C = cplx<T>;
  const int G3 = p.g.n3, K1 = p.b.k1, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  const long long kvol = (long long)K1 * K2 * K3;
  const long long total = (long long)e.ncomp * H1 * K2 * K3;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int k3 = (int)(idx % K3);
  long long r = idx / K3;
  const int k2 = (int)(r % K2);
  r /= K2;
  const int h = (int)(r % H1);
  const int c = (int)(r / H1);
  const long long kin = ((long long)h * K2 + k2) * K3 + k3;   // slot within a component
  const bool nq = nyq(k2, K2) || nyq(k3, K3);

  C R[2] = {C{T(0), T(0)}, C{T(0), T(0)}};
  if (!nq) {
    const T kh = T(1) / Lhat[kin];
    for (int o = 0; o < e.nper; ++o) {
      const int f = o * e.ncomp + c;
      const C* __restrict__ row = T1 + (((long long)f * H1 + h) * K2 + k2) * G3;
      C y{T(0), T(0)};
      for (int x = 0; x < G3; ++x) cmac<C, T>(y, row[x], p.E3b[(long long)x * K3 + k3]);
      const T sc = e.coef[o] * (e.applyK[o] ? kh : T(1));
      R[e.grp[o]].x += sc * y.x;
      R[e.grp[o]].y += sc * y.y;
    }
  }
  // read every X term before any write: outputs may alias inputs
  C val[kMaxOut];
  const long long at = (long long)c * kvol + kin;
  for (int j = 0; j < e.nout; ++j) {
    C v{T(0), T(0)};
    if (!nq) {
      if (e.r[j] >= 0) { v.x = e.cR[j] * R[e.r[j]].x; v.y = e.cR[j] * R[e.r[j]].y; }
      for (int q = 0; q < e.nx[j]; ++q) {
        const C xv = e.X[j][q][at];
        v.x += e.cX[j][q] * xv.x;
        v.y += e.cX[j][q] * xv.y;
      }
    }
    val[j] = v;
  }
  const long long mir = (long long)c * kvol +
      (((long long)((K1 - h) % K1) * K2 + (K2 - k2) % K2) * K3 + (K3 - k3) % K3);
  const long long nyq1 = (long long)c * kvol + (((long long)(K1 / 2) * K2 + k2) * K3 + k3);
  for (int j = 0; j < e.nout; ++j) {
    e.dst[j][at] = val[j];
    if (h > 0) e.dst[j][mir] = C{val[j].x, -val[j].y};
    if (h == 0 && K1 % 2 == 0) e.dst[j][nyq1] = C{T(0), T(0)};
  }
}

}  // namespace

template <typename T>
void iota_batch(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T1,
                cplx<T>* T2, cudaStream_t st) {
  constexpr int YT = 4;
  const int H1 = p.b.h1;
  const long long nA = (long long)d.nf * H1 * p.b.k2 * ((p.g.n3 + YT - 1) / YT);
  k_iota_A<T, YT><<<blocks_for(nA), kThreads, 0, st>>>(p, d, Lhat, T1);
  const int B = d.nf * H1;
  const long long nB = (long long)B * ((p.g.n2 + YT - 1) / YT) * p.g.n3;
  k_mid_cc<T, YT><<<blocks_for(nB), kThreads, 0, st>>>(T1, T2, p.E2f, B, p.b.k2, p.g.n2, p.g.n3);
  const long long nC = (long long)d.nf * ((p.g.n1 + YT - 1) / YT) * p.g.n2 * p.g.n3;
  k_iota_C<T, YT><<<blocks_for(nC), kThreads, 0, st>>>(p, d, T2);
}

template <typename T>
void pi_batch(const Plan<T>& p, const PiSrc<T>& s, const PiEpi<T>& e, const T* Lhat,
              cplx<T>* T1, cplx<T>* T2, cudaStream_t st) {
  constexpr int YT = 4;
  const int H1 = p.b.h1;
  const long long nC = (long long)s.nf * ((H1 + YT - 1) / YT) * p.g.n2 * p.g.n3;
  k_pi_C<T, YT><<<blocks_for(nC), kThreads, 0, st>>>(p, s, T2);
  const int B = s.nf * H1;
  const long long nB = (long long)B * ((p.b.k2 + YT - 1) / YT) * p.g.n3;
  k_mid_cc<T, YT><<<blocks_for(nB), kThreads, 0, st>>>(T2, T1, p.E2b, B, p.g.n2, p.b.k2, p.g.n3);
  const long long nA = (long long)e.ncomp * H1 * p.b.k2 * p.b.k3;
  k_pi_A<T><<<blocks_for(nA), kThreads, 0, st>>>(p, e, Lhat, T1);
}

template void iota_batch<float>(const Plan<float>&, const IotaDesc<float>&, const float*,
                                cplx<float>*, cplx<float>*, cudaStream_t);
template void iota_batch<double>(const Plan<double>&, const IotaDesc<double>&, const double*,
                                 cplx<double>*, cplx<double>*, cudaStream_t);
template void pi_batch<float>(const Plan<float>&, const PiSrc<float>&, const PiEpi<float>&,
                              const float*, cplx<float>*, cplx<float>*, cudaStream_t);
template void pi_batch<double>(const Plan<double>&, const PiSrc<double>&, const PiEpi<double>&,
                               const double*, cplx<double>*, cplx<double>*, cudaStream_t);

}  // namespace lddmm
