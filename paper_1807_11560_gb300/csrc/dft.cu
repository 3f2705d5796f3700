// Truncated separable DFTs between band-limited coefficients and grid values
// (iota and pi of Section 3.1, Eq. 46) and the fused bracket evaluation of
// ad~* / ad~ (Eqs. 4, 48, 49) on the padded product grid, for sm_103a.
//
// iota runs three contractions:
//   A  k3 -> x3   T1[k2][x3]      = sum_k3 m_f(k) a_f(h,k2,k3) E3f[k3][x3]
//   B  k2 -> x2   T2[f][h][x2][x3] = sum_k2 E2f[k2][x2] T1[k2][x3]
//   C  k1 -> x1   out_f[x1][x2][x3] = sum_h Re(E1f[h][x1] T2[f][h][x2][x3])
// where h runs over the non-negative k1 slots only: the field is real, so the
// k1 < 0 half is the conjugate of the k1 > 0 half (E1f carries weight 2 for
// h > 0).  m_f is the field's spectral multiplier (L^ and/or 2 pi i k_j).
// pi runs the transposed contractions C' (x1 -> h), B' (x2 -> k2), A' (x3 -> k3),
// the last one fused with an epilogue that applies K^ = 1/L^, the Heun or
// Krylov linear combination, and writes the k1 < 0 half by conjugation.
//
// Kernels (one CTA of 256 threads each):
//   k_iota_AB  CTA per (field, h): A and B through shared memory -> T2.
//   k_iota_C   thread per output, C -> grid field (image-grid transforms).
//   k_cpw      CTA per tile of (x2,x3) pencils, all x1: C for the 24 fields of
//              a bracket evaluation, the bracket products, and C' of the 3 or
//              9 product fields -> P2; the grid fields stay in shared memory
//              (they are written out only when they become a stage-point cache).
//   k_pi_C     thread per output, C' of image-grid fields -> P2.
//   k_pi_BA    CTA per (component, h, k2 chunk): B' and A' through shared
//              memory, then the epilogue -> band vectors.
#include <algorithm>

#include "internal.h"

namespace lddmm {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kThreads = 256;
constexpr int kMaxSmem = 200 * 1024;

__device__ __forceinline__ int sfreq(int q, int K) { return (2 * q < K) ? q : q - K; }
__device__ __forceinline__ bool nyq(int q, int K) { return (K % 2 == 0) && (2 * q == K); }

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

template <typename C>
__device__ __forceinline__ void cmac(C& acc, const C& a, const C& e) {
  acc.x = fma(a.x, e.x, fma(-a.y, e.y, acc.x));
  acc.y = fma(a.x, e.y, fma(a.y, e.x, acc.y));
}

template <auto Kernel>
void allow_smem() {
  static bool done = false;   // one attribute call per kernel instantiation
  if (!done) {
    cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    done = true;
  }
}

// ---- iota A + B ---------------------------------------------------------------
// TWS: the two twiddle tables are staged in shared memory too (small plans).
template <typename T, bool TWS>
__global__ void __launch_bounds__(kThreads)
k_iota_AB(Plan<T> p, IotaDesc<T> d, const T* __restrict__ Lhat, cplx<T>* __restrict__ T2) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int G2 = p.g.n2, G3 = p.g.n3, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  C* S0 = reinterpret_cast<C*>(smraw);       // [K2][K3] multiplied band slab
  C* S1 = S0 + K2 * K3;                      // [K2][G3] after stage A
  const C* E3 = p.E3f;
  const C* E2 = p.E2f;
  const int f = blockIdx.x / H1, h = blockIdx.x % H1;
  const int tid = threadIdx.x;
  if (TWS) {
    C* e3 = S1 + K2 * G3;                    // [K3][G3]
    C* e2 = e3 + K3 * G3;                    // [K2][G2]
    for (int i = tid; i < K3 * G3; i += kThreads) e3[i] = p.E3f[i];
    for (int i = tid; i < K2 * G2; i += kThreads) e2[i] = p.E2f[i];
    E3 = e3;
    E2 = e2;
  }
  const C* __restrict__ src = d.src[f] + (long long)h * K2 * K3;
  const T* __restrict__ Lrow = Lhat + (long long)h * K2 * K3;
  const int dv = d.deriv[f];
  const bool aL = d.applyL[f] != 0;
  for (int i = tid; i < K2 * K3; i += kThreads) {
    const int k2 = i / K3, k3 = i % K3;
    C a{T(0), T(0)};
    if (!nyq(k2, K2) && !nyq(k3, K3)) {
      a = src[i];
      if (aL) { const T l = Lrow[i]; a.x *= l; a.y *= l; }
      if (dv >= 0) {
        const T fr = dv == 0 ? T(h) : (dv == 1 ? T(sfreq(k2, K2)) : T(sfreq(k3, K3)));
        const T w = T(kTwoPi) * fr;
        const T ax = -a.y * w;
        a.y = a.x * w;
        a.x = ax;
      }
    }
    S0[i] = a;
  }
  __syncthreads();
  for (int it = tid; it < K2 * G3; it += kThreads) {            // A: k3 -> x3
    const int k2 = it / G3, x3 = it % G3;
    C acc{T(0), T(0)};
    const C* s0 = S0 + k2 * K3;
    for (int k3 = 0; k3 < K3; ++k3) cmac(acc, s0[k3], E3[k3 * G3 + x3]);
    S1[it] = acc;
  }
  __syncthreads();
  C* __restrict__ out = T2 + (long long)(f * H1 + h) * G2 * G3;
  for (int it = tid; it < G2 * G3; it += kThreads) {            // B: k2 -> x2
    const int x2 = it / G3, x3 = it % G3;
    C acc{T(0), T(0)};
    for (int k2 = 0; k2 < K2; ++k2) cmac(acc, S1[k2 * G3 + x3], E2[k2 * G2 + x2]);
    out[it] = acc;
  }
}

// ---- iota C: half-spectrum k1 -> x1, real output ----------------------------------
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

// ---- pi C': real grid x1 -> half-spectrum h ----------------------------------------
template <typename T, int YT>
__global__ void __launch_bounds__(kThreads)
k_pi_C(Plan<T> p, PiSrc<T> s, cplx<T>* __restrict__ P2) {
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
  C* dst = P2 + ((long long)f * H1 + y0) * inner + i;
#pragma unroll
  for (int t = 0; t < YT; ++t)
    if (y0 + t < H1) dst[(long long)t * inner] = acc[t];
}

// ---- bracket products ----------------------------------------------------------------
// Field block layout: a[c] at c, Da[c][j] = d_j a_c at 3 + 3c + j.
// P(a, m)_i = sum_j Da[j][i] m_j + sum_j Dm[i][j] a_j + m_i div a   (ad* bracket, Eq. 4)
// Q(a, w)_i = sum_j Da[i][j] w_j - Dw[i][j] a_j                      (ad bracket, Eq. 49)
template <typename T>
__device__ __forceinline__ void bracketP(const T* a, const T* m, T* out) {
  const T* Da = a + 3;
  const T* Dm = m + 3;
  const T div = Da[0] + Da[4] + Da[8];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T s = m[i] * div;
#pragma unroll
    for (int j = 0; j < 3; ++j) s = fma(Da[3 * j + i], m[j], fma(Dm[3 * i + j], a[j], s));
    out[i] += s;
  }
}

template <typename T>
__device__ __forceinline__ void bracketQ(const T* a, const T* w, T* out) {
  const T* Da = a + 3;
  const T* Dw = w + 3;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) s = fma(Da[3 * i + j], w[j], fma(-Dw[3 * i + j], a[j], s));
    out[i] += s;
  }
}

// ---- fused C + bracket products + C' on the padded grid -------------------------------
// Tile of TP consecutive pencils p = x2*G3 + x3 and all G1 planes in shared
// memory.  X = the 24 fields of this evaluation (from T2), Cc = the 24 cached
// fields of the stage point (read from, or in PW_F written to, the slot).
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads)
k_cpw(Plan<T> p, const cplx<T>* __restrict__ T2, T* __restrict__ slot, cplx<T>* __restrict__ P2,
      int TP) {
  using C = cplx<T>;
  constexpr int NP = (MODE == PW_GT) ? 9 : 3;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long P = (long long)p.g.n2 * p.g.n3;
  C* sT2 = reinterpret_cast<C*>(smraw);                    // [24][H1][TP]
  C* sE1f = sT2 + 24 * H1 * TP;                            // [H1][G1]
  C* sE1b = sE1f + H1 * G1;                                // [G1][H1]
  T* sG = reinterpret_cast<T*>(sE1b + G1 * H1);            // [24][G1][TP]
  T* sP = sG + 24 * G1 * TP;                               // [NP][G1][TP]
  const int tid = threadIdx.x;
  const long long p0 = (long long)blockIdx.x * TP;

  for (int i = tid; i < 24 * H1 * TP; i += kThreads) {
    const int pp = i % TP, fh = i / TP;                     // fh = f * H1 + h
    sT2[i] = (p0 + pp < P) ? T2[(long long)fh * P + p0 + pp] : C{T(0), T(0)};
  }
  for (int i = tid; i < H1 * G1; i += kThreads) {
    sE1f[i] = p.E1f[i];
    sE1b[i] = p.E1b[i];
  }
  __syncthreads();
  // C: the 24 grid fields on G1 x TP points
  const long long fs = (long long)G1 * P;                  // field stride of a slot
  for (int i = tid; i < 24 * G1 * TP; i += kThreads) {
    const int pp = i % TP, x1 = (i / TP) % G1, f = i / (TP * G1);
    const C* s = sT2 + f * H1 * TP + pp;
    T v = T(0);
    for (int h = 0; h < H1; ++h) {
      const C e = sE1f[h * G1 + x1];
      const C a = s[h * TP];
      v = fma(a.x, e.x, fma(-a.y, e.y, v));
    }
    sG[i] = v;
    if (MODE == PW_F && p0 + pp < P) slot[f * fs + (long long)x1 * P + p0 + pp] = v;
  }
  __syncthreads();
  // bracket products
  for (int i = tid; i < G1 * TP; i += kThreads) {
    const int pp = i % TP, x1 = i / TP;
    T o[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] = T(0);
    if (p0 + pp < P) {
      T xv[12], xl[12];
#pragma unroll
      for (int f = 0; f < 12; ++f) {
        xv[f] = sG[f * G1 * TP + i];
        xl[f] = sG[(12 + f) * G1 * TP + i];
      }
      if (MODE == PW_F) {
        bracketP(xv, xl, o);                               // P(v, L v)
      } else {
        T cv[12], cl[12];
        const T* __restrict__ cs = slot + (long long)x1 * P + p0 + pp;
#pragma unroll
        for (int f = 0; f < 12; ++f) {
          cv[f] = cs[f * fs];
          cl[f] = cs[(12 + f) * fs];
        }
        if (MODE == PW_T) {
          bracketP(xv, cl, o);                             // P(dv, L v)
          bracketP(cv, xl, o);                             // P(v, L dv)
        } else {
          bracketP(cv, xl, o);                             // P(v, L U)
          bracketP(xv, cl, o + 3);                         // P(W, L v)
          bracketQ(cv, xv, o + 6);                         // Q(v, W)
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) sP[q * G1 * TP + i] = o[q];
  }
  __syncthreads();
  // C': x1 -> h for the NP product fields
  for (int i = tid; i < NP * H1 * TP; i += kThreads) {
    const int pp = i % TP, h = (i / TP) % H1, q = i / (TP * H1);
    if (p0 + pp >= P) continue;
    const T* sp = sP + q * G1 * TP + pp;
    C acc{T(0), T(0)};
    for (int x1 = 0; x1 < G1; ++x1) {
      const T v = sp[x1 * TP];
      const C e = sE1b[x1 * H1 + h];
      acc.x = fma(v, e.x, acc.x);
      acc.y = fma(v, e.y, acc.y);
    }
    P2[(long long)(q * H1 + h) * P + p0 + pp] = acc;
  }
}

// ---- pi B' + A' + epilogue ---------------------------------------------------------------
// CTA per (component c, h, k2 chunk of KC rows).  B' streams the P2 slab of
// every product field of c in chunks of XB rows of x2 through shared memory;
// each thread keeps up to kAccB complex accumulators of S1[o][kk][x3].
constexpr int kAccB = 4;
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pi_BA(Plan<T> p, PiEpi<T> e, const T* __restrict__ Lhat, const cplx<T>* __restrict__ P2,
        int KC, int nch, int XB) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int G2 = p.g.n2, G3 = p.g.n3, K1 = p.b.k1, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  const long long P = (long long)G2 * G3;
  const long long kvol = (long long)K1 * K2 * K3;
  const int nper = e.nper;
  C* slab = reinterpret_cast<C*>(smraw);                   // [nper][XB][G3]
  C* E2s = slab + nper * XB * G3;                          // [G2][KC]
  C* E3s = E2s + G2 * KC;                                  // [G3][K3]
  C* S1 = E3s + G3 * K3;                                   // [nper][KC][G3]
  const int chunk = blockIdx.x % nch;
  const int h = (blockIdx.x / nch) % H1;
  const int c = blockIdx.x / (nch * H1);
  const int kb = chunk * KC;
  const int kc = min(KC, K2 - kb);
  const int tid = threadIdx.x;

  for (int i = tid; i < G2 * KC; i += kThreads) {
    const int x2 = i / KC, kk = i % KC;
    E2s[i] = kk < kc ? p.E2b[(long long)x2 * K2 + kb + kk] : C{T(0), T(0)};
  }
  for (int i = tid; i < G3 * K3; i += kThreads) E3s[i] = p.E3b[i];
  C acc[kAccB];
#pragma unroll
  for (int r = 0; r < kAccB; ++r) acc[r] = C{T(0), T(0)};
  const int nitem = nper * kc * G3;
  for (int x2c = 0; x2c < G2; x2c += XB) {
    const int xb = min(XB, G2 - x2c);
    __syncthreads();
    for (int i = tid; i < nper * xb * G3; i += kThreads) {
      const int x3 = i % G3, xr = (i / G3) % xb, o = i / (G3 * xb);
      const int f = o * e.ncomp + c;
      slab[(o * XB + xr) * G3 + x3] = P2[(long long)(f * H1 + h) * P + (long long)(x2c + xr) * G3 + x3];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kAccB; ++r) {
      const int it = tid + r * kThreads;
      if (it < nitem) {
        const int x3 = it % G3, kk = (it / G3) % kc, o = it / (G3 * kc);
        const C* sl = slab + o * XB * G3 + x3;
        for (int xr = 0; xr < xb; ++xr) cmac(acc[r], sl[xr * G3], E2s[(x2c + xr) * KC + kk]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kAccB; ++r) {
    const int it = tid + r * kThreads;
    if (it < nitem) {
      const int x3 = it % G3, kk = (it / G3) % kc, o = it / (G3 * kc);
      S1[(o * KC + kk) * G3 + x3] = acc[r];
    }
  }
  __syncthreads();

  // A' + epilogue for band slots (c, h, kb + kk, k3)
  for (int it = tid; it < kc * K3; it += kThreads) {
    const int k3 = it % K3, kk = it / K3;
    const int k2 = kb + kk;
    const long long kin = ((long long)h * K2 + k2) * K3 + k3;
    const bool nq = nyq(k2, K2) || nyq(k3, K3);
    C R[2] = {C{T(0), T(0)}, C{T(0), T(0)}};
    if (!nq) {
      const T kh = T(1) / Lhat[kin];
      for (int o = 0; o < nper; ++o) {
        const C* row = S1 + (o * KC + kk) * G3;
        C y{T(0), T(0)};
        for (int x = 0; x < G3; ++x) cmac(y, row[x], E3s[x * K3 + k3]);
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
}

// ---- launch geometry -----------------------------------------------------------------------
template <typename T>
size_t ab_smem(const Plan<T>& p, bool tws) {
  size_t n = (size_t)p.b.k2 * p.b.k3 + (size_t)p.b.k2 * p.g.n3;
  if (tws) n += (size_t)p.b.k3 * p.g.n3 + (size_t)p.b.k2 * p.g.n2;
  return n * sizeof(cplx<T>);
}

template <typename T>
size_t cpw_smem(const Plan<T>& p, int TP, int NP) {
  const int G1 = p.g.n1, H1 = p.b.h1;
  return ((size_t)24 * H1 * TP + 2 * (size_t)H1 * G1) * sizeof(cplx<T>) +
         (size_t)(24 + NP) * G1 * TP * sizeof(T);
}

template <typename T>
int cpw_tile(const Plan<T>& p) {
  const long long P = (long long)p.g.n2 * p.g.n3;
  int TP = (int)std::max(1LL, std::min(8LL, P / 152));
  while (TP > 1 && cpw_smem(p, TP, 9) > (size_t)kMaxSmem) --TP;
  return TP;
}

struct BAGeom {
  int KC, nch, XB;
};
template <typename T>
BAGeom ba_geom(const Plan<T>& p, int ncomp, int nper) {
  const int G2 = p.g.n2, G3 = p.g.n3, K2 = p.b.k2, K3 = p.b.k3;
  const int groups = ncomp * p.b.h1;
  const int want = std::max(1, (304 + groups - 1) / groups);
  int KC = std::max(1, (K2 + want - 1) / want);
  KC = std::max(1, std::min(KC, (kAccB * kThreads) / std::max(1, nper * G3)));
  KC = std::min(KC, K2);
  const int nch = (K2 + KC - 1) / KC;
  const size_t c = sizeof(cplx<T>);
  const size_t fixed = ((size_t)G2 * KC + (size_t)G3 * K3 + (size_t)nper * KC * G3) * c;
  const size_t budget = fixed < (size_t)kMaxSmem ? (size_t)kMaxSmem - fixed : 0;
  const size_t rows = std::min<size_t>(budget, 96 * 1024) / ((size_t)nper * G3 * c);
  const int XB = (int)std::min<size_t>((size_t)G2, std::max<size_t>(1, rows));
  return BAGeom{KC, nch, XB};
}

template <typename T>
size_t ba_smem(const Plan<T>& p, int nper, const BAGeom& g) {
  return ((size_t)nper * g.XB * p.g.n3 + (size_t)p.g.n2 * g.KC + (size_t)p.g.n3 * p.b.k3 +
          (size_t)nper * g.KC * p.g.n3) * sizeof(cplx<T>);
}

template <typename T>
void launch_iota_AB(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2, cudaStream_t st) {
  if (ab_smem(p, true) <= 64 * 1024) {
    allow_smem<k_iota_AB<T, true>>();
    k_iota_AB<T, true><<<d.nf * p.b.h1, kThreads, ab_smem(p, true), st>>>(p, d, Lhat, T2);
  } else {
    allow_smem<k_iota_AB<T, false>>();
    k_iota_AB<T, false><<<d.nf * p.b.h1, kThreads, ab_smem(p, false), st>>>(p, d, Lhat, T2);
  }
}

template <typename T>
void launch_pi_BA(const Plan<T>& p, const PiEpi<T>& e, const T* Lhat, const cplx<T>* P2, cudaStream_t st) {
  const BAGeom g = ba_geom(p, e.ncomp, e.nper);
  allow_smem<k_pi_BA<T>>();
  k_pi_BA<T><<<e.ncomp * p.b.h1 * g.nch, kThreads, ba_smem(p, e.nper, g), st>>>(p, e, Lhat, P2, g.KC,
                                                                                g.nch, g.XB);
}

}  // namespace

template <typename T>
size_t max_smem_needed(const Plan<T>& p, int nper_max, bool brackets) {
  // every B' item of a CTA needs its own accumulator
  if ((long long)nper_max * p.g.n3 > (long long)kAccB * kThreads) return ~size_t(0);
  const size_t ab = ab_smem(p, false);
  const size_t cpw = brackets ? cpw_smem(p, cpw_tile(p), 9) : 0;
  size_t ba = 0;
  for (int nper = 1; nper <= nper_max; ++nper) ba = std::max(ba, ba_smem(p, nper, ba_geom(p, 36, nper)));
  return std::max(ab, std::max(cpw, ba));
}

size_t smem_limit() { return kMaxSmem; }

template <typename T>
void iota_batch(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2, cudaStream_t st) {
  constexpr int YT = 4;
  launch_iota_AB<T>(p, d, Lhat, T2, st);
  const long long nC = (long long)d.nf * ((p.g.n1 + YT - 1) / YT) * p.g.n2 * p.g.n3;
  k_iota_C<T, YT><<<blocks_for(nC), kThreads, 0, st>>>(p, d, T2);
}

template <typename T>
void pi_batch(const Plan<T>& p, const PiSrc<T>& s, const PiEpi<T>& e, const T* Lhat, cplx<T>* P2,
              cudaStream_t st) {
  constexpr int YT = 4;
  const long long nC = (long long)s.nf * ((p.b.h1 + YT - 1) / YT) * p.g.n2 * p.g.n3;
  k_pi_C<T, YT><<<blocks_for(nC), kThreads, 0, st>>>(p, s, P2);
  launch_pi_BA<T>(p, e, Lhat, P2, st);
}

template <typename T>
void bracket_iota(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2, cudaStream_t st) {
  launch_iota_AB<T>(p, d, Lhat, T2, st);
}

template <typename T>
void bracket_cpw(const Plan<T>& p, PwMode mode, const cplx<T>* T2, T* slot, cplx<T>* P2, cudaStream_t st) {
  const int TP = cpw_tile(p);
  const int NP = (mode == PW_GT) ? 9 : 3;
  const size_t smem = cpw_smem(p, TP, NP);
  const long long P = (long long)p.g.n2 * p.g.n3;
  const unsigned grid = (unsigned)((P + TP - 1) / TP);
  switch (mode) {
    case PW_F:
      allow_smem<k_cpw<T, PW_F>>();
      k_cpw<T, PW_F><<<grid, kThreads, smem, st>>>(p, T2, slot, P2, TP);
      break;
    case PW_T:
      allow_smem<k_cpw<T, PW_T>>();
      k_cpw<T, PW_T><<<grid, kThreads, smem, st>>>(p, T2, slot, P2, TP);
      break;
    case PW_GT:
      allow_smem<k_cpw<T, PW_GT>>();
      k_cpw<T, PW_GT><<<grid, kThreads, smem, st>>>(p, T2, slot, P2, TP);
      break;
  }
}

template <typename T>
void bracket_pi(const Plan<T>& p, const PiEpi<T>& e, const T* Lhat, const cplx<T>* P2, cudaStream_t st) {
  launch_pi_BA<T>(p, e, Lhat, P2, st);
}

#define LDDMM_DFT_INST(T)                                                                          \
  template size_t max_smem_needed<T>(const Plan<T>&, int, bool);                                              \
  template void iota_batch<T>(const Plan<T>&, const IotaDesc<T>&, const T*, cplx<T>*, cudaStream_t); \
  template void pi_batch<T>(const Plan<T>&, const PiSrc<T>&, const PiEpi<T>&, const T*, cplx<T>*,  \
                            cudaStream_t);                                                         \
  template void bracket_iota<T>(const Plan<T>&, const IotaDesc<T>&, const T*, cplx<T>*, cudaStream_t); \
  template void bracket_cpw<T>(const Plan<T>&, PwMode, const cplx<T>*, T*, cplx<T>*, cudaStream_t); \
  template void bracket_pi<T>(const Plan<T>&, const PiEpi<T>&, const T*, const cplx<T>*, cudaStream_t);
LDDMM_DFT_INST(float)
LDDMM_DFT_INST(double)

}  // namespace lddmm
