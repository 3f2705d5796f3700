// Device bodies of the three phases of one bracket evaluation on the padded
// product grid (ad~* and ad~ of Eqs. 4, 48, 49 with the truncated DFTs of
// Eq. 46), shared by the stand-alone kernels (dft.cu) and the persistent
// sweep kernel (sweep.cu).  Each body processes one "virtual block" vb with
// 256 threads and a caller-provided dynamic shared-memory buffer.
//
//   phase_iota_ab  vb = (field f, h): iota stages A (k3 -> x3) and B (k2 -> x2)
//                  of one band slab -> T2[f][h][x2][x3]
//   phase_cpw      vb = tile of TP pencils (x2, x3): iota stage C of the 24
//                  fields, the bracket products, pi stage C' of the 3 or 9
//                  product fields -> P2[q][h][x2][x3]
//   phase_pi_ba    vb = (component c, h, k2 chunk): pi stages B' and A' and the
//                  epilogue (K~, Heun/Krylov combination, conjugate half)
#pragma once

#include <algorithm>

#include "internal.h"

namespace lddmm {
namespace dev {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kThreads = 256;
constexpr int kMaxSmem = 200 * 1024;
constexpr int kAccB = 4;      // B' accumulators per thread in phase_pi_ba
constexpr int kRed = 8;       // threads sharing one A' sum in phase_pi_ba

__host__ __device__ __forceinline__ int sfreq(int q, int K) { return (2 * q < K) ? q : q - K; }
__host__ __device__ __forceinline__ bool nyq(int q, int K) { return (K % 2 == 0) && (2 * q == K); }

template <typename C>
__device__ __forceinline__ void cmac(C& acc, const C& a, const C& e) {
  acc.x = fma(a.x, e.x, fma(-a.y, e.y, acc.x));
  acc.y = fma(a.x, e.y, fma(a.y, e.x, acc.y));
}

// One scalar band field entering iota: a component slab with its multiplier.
template <typename T>
struct FieldSpec {
  const cplx<T>* src;   // [K1][K2][K3]
  int deriv;            // -1 or axis
  bool applyL;
};

// Field f of a 24-field bracket block: value/Jacobian of A (f < 12) or of
// L~ B (f >= 12); per half: value[3], then jac[c][j] = d_j (.)_c at 3 + 3c + j.
template <typename T>
__device__ __forceinline__ FieldSpec<T> field24(const cplx<T>* A, const cplx<T>* B, long long kvol, int f) {
  const bool L = f >= 12;
  const int g = L ? f - 12 : f;
  const cplx<T>* s = L ? B : A;
  if (g < 3) return FieldSpec<T>{s + g * kvol, -1, L};
  return FieldSpec<T>{s + ((g - 3) / 3) * kvol, (g - 3) % 3, L};
}

// ---------------------------------------------------------------------------
// bracket products on one grid point
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

// ---------------------------------------------------------------------------
// iota stages A + B of one slab.  TWS: twiddles staged in shared memory too.
template <typename T, bool TWS>
__device__ __forceinline__ void phase_iota_ab(const Plan<T>& p, const FieldSpec<T>& fs, int f, int h,
                                              const T* __restrict__ Lhat, cplx<T>* __restrict__ T2,
                                              unsigned char* smraw) {
  using C = cplx<T>;
  const int G2 = p.g.n2, G3 = p.g.n3, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  C* S0 = reinterpret_cast<C*>(smraw);       // [K2][K3] multiplied band slab
  C* S1 = S0 + K2 * K3;                      // [K2][G3] after stage A
  const C* E3 = p.E3f;
  const C* E2 = p.E2f;
  const int tid = threadIdx.x;
  if (TWS) {
    C* e3 = S1 + K2 * G3;                    // [K3][G3]
    C* e2 = e3 + K3 * G3;                    // [K2][G2]
    for (int i = tid; i < K3 * G3; i += kThreads) e3[i] = p.E3f[i];
    for (int i = tid; i < K2 * G2; i += kThreads) e2[i] = p.E2f[i];
    E3 = e3;
    E2 = e2;
  }
  const C* __restrict__ src = fs.src + (long long)h * K2 * K3;
  const T* __restrict__ Lrow = Lhat + (long long)h * K2 * K3;
  for (int i = tid; i < K2 * K3; i += kThreads) {
    const int k2 = i / K3, k3 = i % K3;
    C a{T(0), T(0)};
    if (!nyq(k2, K2) && !nyq(k3, K3)) {
      a = src[i];
      if (fs.applyL) { const T l = Lrow[i]; a.x *= l; a.y *= l; }
      if (fs.deriv >= 0) {
        const T fr = fs.deriv == 0 ? T(h) : (fs.deriv == 1 ? T(sfreq(k2, K2)) : T(sfreq(k3, K3)));
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

// ---------------------------------------------------------------------------
// C + bracket products + C' on one tile of TP pencils, all G1 planes.
template <typename T, int MODE>
__device__ __forceinline__ void phase_cpw(const Plan<T>& p, const cplx<T>* __restrict__ T2,
                                          T* __restrict__ slot, cplx<T>* __restrict__ P2, int TP, int vb,
                                          unsigned char* smraw) {
  using C = cplx<T>;
  constexpr int NP = (MODE == PW_GT) ? 9 : 3;
  const int G1 = p.g.n1, H1 = p.b.h1;
  const long long P = (long long)p.g.n2 * p.g.n3;
  C* sT2 = reinterpret_cast<C*>(smraw);                    // [24][H1][TP]
  C* sE1f = sT2 + 24 * H1 * TP;                            // [H1][G1]
  C* sE1b = sE1f + H1 * G1;                                // [G1][H1]
  T* sG = reinterpret_cast<T*>(sE1b + G1 * H1);            // [24][G1][TP]
  T* sP = sG + 24 * G1 * TP;                               // [NP][G1][TP]
  const int tid = threadIdx.x;
  const long long p0 = (long long)vb * TP;

  for (int i = tid; i < 24 * H1 * TP; i += kThreads) {
    const int pp = i % TP, fh = i / TP;                     // fh = f * H1 + h
    sT2[i] = (p0 + pp < P) ? T2[(long long)fh * P + p0 + pp] : C{T(0), T(0)};
  }
  for (int i = tid; i < H1 * G1; i += kThreads) {
    sE1f[i] = p.E1f[i];
    sE1b[i] = p.E1b[i];
  }
  __syncthreads();
  const long long fs = (long long)G1 * P;                  // field stride of a slot
  for (int i = tid; i < 24 * G1 * TP; i += kThreads) {     // C: 24 grid fields
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
  for (int i = tid; i < G1 * TP; i += kThreads) {          // bracket products
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
  for (int i = tid; i < NP * H1 * TP; i += kThreads) {     // C': x1 -> h
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

// ---------------------------------------------------------------------------
// pi B' + A' + epilogue for (component c, h, k2 chunk).  B' streams the P2
// slab of every product field of c in chunks of XB rows of x2 through shared
// memory, each thread keeping up to kAccB accumulators of S1[o][kk][x3]; A'
// splits every band-slot sum over kRed threads and reduces with shuffles.
struct BAGeom {
  int KC, nch, XB;
};

template <typename T>
__device__ __forceinline__ void phase_pi_ba(const Plan<T>& p, const PiEpi<T>& e, const T* __restrict__ Lhat,
                                            const cplx<T>* __restrict__ P2, const BAGeom& g, int vb,
                                            unsigned char* smraw) {
  using C = cplx<T>;
  const int G2 = p.g.n2, G3 = p.g.n3, K1 = p.b.k1, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  const int KC = g.KC, nch = g.nch, XB = g.XB;
  const long long P = (long long)G2 * G3;
  const long long kvol = (long long)K1 * K2 * K3;
  const int nper = e.nper, ncomp = e.ncomp, nout = e.nout;
  C* slab = reinterpret_cast<C*>(smraw);                   // [nper][XB][G3]
  C* E2s = slab + nper * XB * G3;                          // [G2][KC]
  C* E3s = E2s + G2 * KC;                                  // [G3][K3]
  C* S1 = E3s + G3 * K3;                                   // [nper][KC][G3]
  const int chunk = vb % nch;
  const int h = (vb / nch) % H1;
  const int c = vb / (nch * H1);
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
    if (x2c > 0) __syncthreads();
    for (int i = tid; i < nper * xb * G3; i += kThreads) {
      const int x3 = i % G3, xr = (i / G3) % xb, o = i / (G3 * xb);
      const int f = o * ncomp + c;
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

  // A' + epilogue: kRed consecutive lanes share one band slot (c, h, kb+kk, k3)
  const int nslot = kc * K3;
  for (int base = 0; base < nslot * kRed; base += kThreads) {
    const int lin = base + tid;
    const int it = lin / kRed, part = lin % kRed;
    const bool live = it < nslot;
    const int k3 = live ? it % K3 : 0, kk = live ? it / K3 : 0;
    const int k2 = kb + kk;
    const bool nq = !live || nyq(k2, K2) || nyq(k3, K3);
    C R[2] = {C{T(0), T(0)}, C{T(0), T(0)}};
    for (int o = 0; o < nper; ++o) {
      C y{T(0), T(0)};
      if (!nq) {
        const C* row = S1 + (o * KC + kk) * G3;
        for (int x = part; x < G3; x += kRed) cmac(y, row[x], E3s[x * K3 + k3]);
      }
#pragma unroll
      for (int off = kRed / 2; off > 0; off >>= 1) {
        y.x += __shfl_down_sync(0xffffffffu, y.x, off, kRed);
        y.y += __shfl_down_sync(0xffffffffu, y.y, off, kRed);
      }
      if (part == 0 && !nq) {
        const long long kin = ((long long)h * K2 + k2) * K3 + k3;
        const T sc = e.coef[o] * (e.applyK[o] ? T(1) / Lhat[kin] : T(1));
        R[e.grp[o]].x += sc * y.x;
        R[e.grp[o]].y += sc * y.y;
      }
    }
    if (part != 0 || !live) continue;
    const long long kin = ((long long)h * K2 + k2) * K3 + k3;
    const long long at = (long long)c * kvol + kin;
    // read every X term before any write: outputs may alias inputs
    C val[kMaxOut];
    for (int j = 0; j < nout; ++j) {
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
    for (int j = 0; j < nout; ++j) {
      e.dst[j][at] = val[j];
      if (h > 0) e.dst[j][mir] = C{val[j].x, -val[j].y};
      if (h == 0 && K1 % 2 == 0) e.dst[j][nyq1] = C{T(0), T(0)};
    }
  }
}

// ---------------------------------------------------------------------------
// launch geometry (host and device)
template <typename T>
__host__ __device__ inline size_t ab_smem(const Plan<T>& p, bool tws) {
  size_t n = (size_t)p.b.k2 * p.b.k3 + (size_t)p.b.k2 * p.g.n3;
  if (tws) n += (size_t)p.b.k3 * p.g.n3 + (size_t)p.b.k2 * p.g.n2;
  return n * sizeof(cplx<T>);
}

template <typename T>
__host__ __device__ inline bool ab_tws(const Plan<T>& p) {
  return ab_smem(p, true) <= 64 * 1024;
}

template <typename T>
__host__ __device__ inline size_t cpw_smem(const Plan<T>& p, int TP, int NP) {
  const int G1 = p.g.n1, H1 = p.b.h1;
  return ((size_t)24 * H1 * TP + 2 * (size_t)H1 * G1) * sizeof(cplx<T>) +
         (size_t)(24 + NP) * G1 * TP * sizeof(T);
}

template <typename T>
inline int cpw_tile(const Plan<T>& p) {
  const long long P = (long long)p.g.n2 * p.g.n3;
  int TP = (int)std::max(1LL, std::min(8LL, P / 152));
  while (TP > 1 && cpw_smem(p, TP, 9) > (size_t)kMaxSmem) --TP;
  return TP;
}

template <typename T>
inline BAGeom ba_geom(const Plan<T>& p, int ncomp, int nper) {
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
inline size_t ba_smem(const Plan<T>& p, int nper, const BAGeom& g) {
  return ((size_t)nper * g.XB * p.g.n3 + (size_t)p.g.n2 * g.KC + (size_t)p.g.n3 * p.b.k3 +
          (size_t)nper * g.KC * p.g.n3) * sizeof(cplx<T>);
}

}  // namespace dev
}  // namespace lddmm
