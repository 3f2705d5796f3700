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
constexpr int kAccB = 2;      // B' columns per thread in phase_pi_ba (nper * G3 <= 512)
constexpr int kRed = 8;       // threads sharing one A' sum in phase_pi_ba

__host__ __device__ __forceinline__ int sfreq(int q, int K) { return (2 * q < K) ? q : q - K; }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor runs; it stages its constant
// operands (twiddles, symbols) first and waits here before touching anything
// an earlier kernel wrote.  Without that launch attribute (and inside the
// persistent sweep) the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the next kernel of the stream be scheduled (it still waits in pdl_wait)
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
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

// velocity component whose band slab field f of a 24-field block reads
__host__ __device__ __forceinline__ int field24_comp(int f) {
  const int g = f >= 12 ? f - 12 : f;
  return g < 3 ? g : (g - 3) / 3;
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
// paired loads of two consecutive complex values (16-byte aligned for float)
template <typename C>
__device__ __forceinline__ void ld2(const C* p, C& a, C& b) {
  a = p[0];
  b = p[1];
}
template <>
__device__ __forceinline__ void ld2<float2>(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}

// asynchronous global -> shared copies (cp.async): a staging loop issues all of
// its requests before the first one returns, so a phase pays one L2 round trip
// for its inputs instead of one per loop iteration
template <typename V>
__device__ __forceinline__ void cp_async(V* dst, const V* src) {
  static_assert(sizeof(V) == 4 || sizeof(V) == 8 || sizeof(V) == 16, "cp.async size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(sizeof(V)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// n contiguous elements, copied by all threads of the CTA: 16-byte requests
// when both ends allow it, else one request per element
template <typename V>
__device__ __forceinline__ void cp_async_run(V* dst, const V* src, int n) {
  constexpr int per = 16 / (int)sizeof(V);
  if (per > 1 && n % per == 0 && ((reinterpret_cast<size_t>(dst) | reinterpret_cast<size_t>(src)) & 15) == 0) {
    float4* d = reinterpret_cast<float4*>(dst);
    const float4* q = reinterpret_cast<const float4*>(src);
    for (int i = threadIdx.x; i < n / per; i += kThreads) cp_async(d + i, q + i);
  } else {
    for (int i = threadIdx.x; i < n; i += kThreads) cp_async(dst + i, src + i);
  }
}

__host__ __device__ __forceinline__ int even_up(int n) { return n + (n & 1); }
__host__ __device__ __forceinline__ int quad_up(int n) { return (n + 3) & ~3; }

// ---------------------------------------------------------------------------
// iota stages A + B of one slab, in 2 x 2 complex register tiles.
// Shared memory: S0 [K2][K3], S1 [K2][G3e], with TWS the twiddles
// E3 [K3][G3e] and E2 [K2][G2e] (G*e = even-rounded, zero padded), then the
// multiplier row sL [K2][K3].
template <typename T, bool TWS>
__device__ __forceinline__ void phase_iota_ab(const Plan<T>& p, const FieldSpec<T>& fs, int f, int h,
                                              const T* __restrict__ Lhat, cplx<T>* __restrict__ T2,
                                              unsigned char* smraw) {
  using C = cplx<T>;
  const int G2 = p.g.n2, G3 = p.g.n3, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  const int G2e = even_up(G2), G3e = even_up(G3);
  C* S0 = reinterpret_cast<C*>(smraw);       // [K2][K3] multiplied band slab
  C* S1 = S0 + K2 * K3;                      // [K2][G3e] after stage A
  C* E3s = S1 + K2 * G3e;                    // [K3][G3e]
  C* E2s = E3s + K3 * G3e;                   // [K2][G2e]
  T* sL = reinterpret_cast<T*>(TWS ? E2s + K2 * G2e : E3s);   // [K2][K3]
  const int tid = threadIdx.x;
  const C zero{T(0), T(0)};
  if (TWS && p.E3fp != nullptr) {
    cp_async_run(E3s, p.E3fp, K3 * G3e);
    cp_async_run(E2s, p.E2fp, K2 * G2e);
  } else if (TWS) {
    for (int i = tid; i < K3 * G3e; i += kThreads) {
      const int r = i / G3e, x = i - r * G3e;
      if (x < G3) cp_async(E3s + i, p.E3f + r * G3 + x); else E3s[i] = zero;
    }
    for (int i = tid; i < K2 * G2e; i += kThreads) {
      const int r = i / G2e, x = i - r * G2e;
      if (x < G2) cp_async(E2s + i, p.E2f + r * G2 + x); else E2s[i] = zero;
    }
  }
  const C* __restrict__ src = fs.src + (long long)h * K2 * K3;
  const T* __restrict__ Lrow = Lhat + (long long)h * K2 * K3;
  pdl_wait();
  cp_async_run(S0, src, K2 * K3);
  if (fs.applyL) cp_async_run(sL, Lrow, K2 * K3);
  cp_async_wait_all();
  __syncthreads();
  for (int i = tid; i < K2 * K3; i += kThreads) {   // multiplier in place
    const int k2 = i / K3, k3 = i - k2 * K3;
    C a = zero;
    if (!nyq(k2, K2) && !nyq(k3, K3)) {
      a = S0[i];
      if (fs.applyL) { const T l = sL[i]; a.x *= l; a.y *= l; }
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
  // A: S1[k2][x3] = sum_k3 S0[k2][k3] E3[k3][x3]   (K2 is even)
  const int n3p = G3e / 2;
  for (int it = tid; it < (K2 / 2) * n3p; it += kThreads) {
    const int kp = it / n3p, xp = it - kp * n3p;
    const int k2 = 2 * kp, x3 = 2 * xp;
    C c00 = zero, c01 = zero, c10 = zero, c11 = zero;
    const C* s0 = S0 + k2 * K3;
#pragma unroll 4
    for (int k3 = 0; k3 < K3; ++k3) {
      const C a0 = s0[k3], a1 = s0[K3 + k3];
      C e0, e1;
      if (TWS) {
        ld2(E3s + k3 * G3e + x3, e0, e1);
      } else {
        e0 = p.E3f[k3 * G3 + x3];
        e1 = x3 + 1 < G3 ? p.E3f[k3 * G3 + x3 + 1] : zero;
      }
      cmac(c00, a0, e0); cmac(c01, a0, e1); cmac(c10, a1, e0); cmac(c11, a1, e1);
    }
    S1[k2 * G3e + x3] = c00;
    S1[k2 * G3e + x3 + 1] = c01;
    S1[(k2 + 1) * G3e + x3] = c10;
    S1[(k2 + 1) * G3e + x3 + 1] = c11;
  }
  __syncthreads();
  // B: out[x2][x3] = sum_k2 E2[k2][x2] S1[k2][x3]
  C* __restrict__ out = T2 + (long long)(f * H1 + h) * G2 * G3;
  const int n2p = G2e / 2;
  for (int it = tid; it < n2p * n3p; it += kThreads) {
    const int yp = it / n3p, xp = it - yp * n3p;
    const int x2 = 2 * yp, x3 = 2 * xp;
    C c00 = zero, c01 = zero, c10 = zero, c11 = zero;
#pragma unroll 4
    for (int k2 = 0; k2 < K2; ++k2) {
      C s0, s1, e0, e1;
      ld2(S1 + k2 * G3e + x3, s0, s1);
      if (TWS) {
        ld2(E2s + k2 * G2e + x2, e0, e1);
      } else {
        e0 = p.E2f[k2 * G2 + x2];
        e1 = x2 + 1 < G2 ? p.E2f[k2 * G2 + x2 + 1] : zero;
      }
      cmac(c00, s0, e0); cmac(c01, s1, e0); cmac(c10, s0, e1); cmac(c11, s1, e1);
    }
    out[(long long)x2 * G3 + x3] = c00;
    if (x3 + 1 < G3) out[(long long)x2 * G3 + x3 + 1] = c01;
    if (x2 + 1 < G2) {
      out[(long long)(x2 + 1) * G3 + x3] = c10;
      if (x3 + 1 < G3) out[(long long)(x2 + 1) * G3 + x3 + 1] = c11;
    }
  }
}

// ---------------------------------------------------------------------------
// C + bracket products + C' on one tile of TP pencils, all G1 planes.
// Twiddles staged zero-padded: E1f [H1][G1q] and E1b [G1][H1q] (q = rounded
// up to 4), so C works on 4 planes and C' on 4 band slots per thread.
template <typename T, int MODE>
__device__ __forceinline__ void phase_cpw(const Plan<T>& p, const cplx<T>* __restrict__ T2,
                                          T* __restrict__ slot, T* __restrict__ slot2,
                                          cplx<T>* __restrict__ P2, int TP, int vb, unsigned char* smraw) {
  using C = cplx<T>;
  constexpr int NP = (MODE == PW_GT) ? 9 : 3;
  const int G1 = p.g.n1, H1 = p.b.h1;
  const int G1q = quad_up(G1), H1q = quad_up(H1);
  const long long P = (long long)p.g.n2 * p.g.n3;
  C* sT2 = reinterpret_cast<C*>(smraw);                    // [24][H1][TP]
  C* sE1f = sT2 + 24 * H1 * TP;                            // [H1][G1q]
  C* sE1b = sE1f + H1 * G1q;                               // [G1][H1q]
  T* sG = reinterpret_cast<T*>(sE1b + G1 * H1q);           // [24][G1][TP]
  T* sP = sG + 24 * G1 * TP;                               // [NP][G1][TP]
  const int tid = threadIdx.x;
  const long long p0 = (long long)vb * TP;
  const C zero{T(0), T(0)};

  if (p.E1fp != nullptr) {                                 // constant operands first
    cp_async_run(sE1f, p.E1fp, H1 * G1q);
    cp_async_run(sE1b, p.E1bp, G1 * H1q);
  } else {
    for (int i = tid; i < H1 * G1q; i += kThreads) {
      const int h = i / G1q, x = i - h * G1q;
      if (x < G1) cp_async(sE1f + i, p.E1f + h * G1 + x); else sE1f[i] = zero;
    }
    for (int i = tid; i < G1 * H1q; i += kThreads) {
      const int x = i / H1q, h = i - x * H1q;
      if (h < H1) cp_async(sE1b + i, p.E1b + x * H1 + h); else sE1b[i] = zero;
    }
  }
  pdl_wait();
  for (int fh = tid / TP, pp = tid - (tid / TP) * TP; fh < 24 * H1;) {
    if (p0 + pp < P) cp_async(sT2 + fh * TP + pp, T2 + (long long)fh * P + p0 + pp);
    else sT2[fh * TP + pp] = zero;
    pp += kThreads % TP;
    fh += kThreads / TP;
    if (pp >= TP) { pp -= TP; ++fh; }
  }
  // the cached stage-point fields of this thread's (up to 2) product points,
  // fetched now so their latency overlaps the transform stage.  The slot is
  // tile-major, [tile][24][G1][TP] (the layout of sG), so these loads are
  // contiguous across the threads of a warp.
  T* __restrict__ tslot = slot + (long long)vb * 24 * G1 * TP;
  // tangent sweeps may also cache the fields they transform (full-Newton products)
  T* __restrict__ tslot2 = (MODE == PW_T && slot2 != nullptr) ? slot2 + (long long)vb * 24 * G1 * TP : nullptr;
  T cv[2][12], cl[2][12];
  if (MODE != PW_F) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = tid + r * kThreads;
      const int pp = i - (i / TP) * TP;
      const bool ok = i < G1 * TP && p0 + pp < P;
      const T* __restrict__ cs = tslot + i;
#pragma unroll
      for (int f = 0; f < 12; ++f) {
        cv[r][f] = ok ? cs[f * G1 * TP] : T(0);
        cl[r][f] = ok ? cs[(12 + f) * G1 * TP] : T(0);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int nq = G1q / 4;
  for (int it = tid; it < 24 * TP * nq; it += kThreads) {  // C: 24 grid fields, 4 planes each
    const int f = it / (TP * nq);                          // pencil fastest: the sT2 reads are
    const int rem = it - f * TP * nq;                      // consecutive and the twiddle reads
    const int xq = rem / TP, pp = rem - xq * TP;           // broadcast
    const int x0 = 4 * xq;
    const C* s = sT2 + f * H1 * TP + pp;
    T v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
#pragma unroll 4
    for (int h = 0; h < H1; ++h) {
      const C a = s[h * TP];
      C e0, e1, e2, e3;
      ld2(sE1f + h * G1q + x0, e0, e1);
      ld2(sE1f + h * G1q + x0 + 2, e2, e3);
      v0 = fma(a.x, e0.x, fma(-a.y, e0.y, v0));
      v1 = fma(a.x, e1.x, fma(-a.y, e1.y, v1));
      v2 = fma(a.x, e2.x, fma(-a.y, e2.y, v2));
      v3 = fma(a.x, e3.x, fma(-a.y, e3.y, v3));
    }
    const T vv[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int x1 = x0 + t;
      if (x1 < G1) {
        sG[(f * G1 + x1) * TP + pp] = vv[t];
        if (MODE == PW_F) tslot[(f * G1 + x1) * TP + pp] = vv[t];
        if (MODE == PW_T && tslot2 != nullptr) tslot2[(f * G1 + x1) * TP + pp] = vv[t];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 2; ++r) {                           // bracket products
    const int i = tid + r * kThreads;
    if (i >= G1 * TP) break;
    const int x1 = i / TP, pp = i - x1 * TP;
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
      } else if (MODE == PW_T) {
        bracketP(xv, cl[r], o);                            // P(dv, L v)
        bracketP(cv[r], xl, o);                            // P(v, L dv)
      } else {
        bracketP(cv[r], xl, o);                            // P(v, L U)
        bracketP(xv, cl[r], o + 3);                        // P(W, L v)
        bracketQ(cv[r], xv, o + 6);                        // Q(v, W)
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) sP[q * G1 * TP + i] = o[q];
  }
  __syncthreads();
  const int nh = H1q / 4;
  for (int it = tid; it < NP * TP * nh; it += kThreads) {  // C': x1 -> h, 4 slots each
    const int q = it / (TP * nh);
    const int rem = it - q * TP * nh;
    const int hq = rem / TP, pp = rem - hq * TP;
    const int h0 = 4 * hq;
    if (p0 + pp >= P) continue;
    const T* sp = sP + q * G1 * TP + pp;
    C a0 = zero, a1 = zero, a2 = zero, a3 = zero;
#pragma unroll 4
    for (int x1 = 0; x1 < G1; ++x1) {
      const T v = sp[x1 * TP];
      C e0, e1, e2, e3;
      ld2(sE1b + x1 * H1q + h0, e0, e1);
      ld2(sE1b + x1 * H1q + h0 + 2, e2, e3);
      a0.x = fma(v, e0.x, a0.x); a0.y = fma(v, e0.y, a0.y);
      a1.x = fma(v, e1.x, a1.x); a1.y = fma(v, e1.y, a1.y);
      a2.x = fma(v, e2.x, a2.x); a2.y = fma(v, e2.y, a2.y);
      a3.x = fma(v, e3.x, a3.x); a3.y = fma(v, e3.y, a3.y);
    }
    const C aa[4] = {a0, a1, a2, a3};
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (h0 + t < H1) P2[(long long)(q * H1 + h0 + t) * P + p0 + pp] = aa[t];
  }
}

// ---------------------------------------------------------------------------
// pi B' + A' + epilogue for (component c, h, k2 chunk of kc <= kMaxKC rows).
// B' streams the P2 slab of every product field of c in chunks of XB rows of
// x2 through shared memory; a (virtual) thread owns one (field, x3) column and
// accumulates the kc band rows of every R-th x2 row (R row groups use the
// threads a narrow slab would leave idle; their partial sums are added in
// fixed order).  A' splits every band-slot sum over kRed lanes and reduces
// with shuffles.  The epilogue's inputs (the X terms and L^ of every band
// slot) are prefetched with the slab.
constexpr int kMaxKC = 8;
constexpr int kMaxRows = 8;   // row groups R of B'
constexpr int kEpiX = kMaxOut * kMaxX;

// row stride of the transposed E3 twiddles in phase_pi_ba: an odd multiple of
// half a 128-byte bank line, so the kRed-lane groups of different band slots
// of a warp read different banks
template <typename T>
__host__ __device__ __forceinline__ int e3_stride(int G3) {
  constexpr int E = 128 / (int)sizeof(cplx<T>);
  return G3 + ((E / 2 - G3 % E) + E) % E;
}
struct BAGeom {
  int KC, nch, XB, R;
};

template <typename T>
__device__ __forceinline__ void phase_pi_ba(const Plan<T>& p, const PiEpi<T>& e, const T* __restrict__ Lhat,
                                            const cplx<T>* __restrict__ P2, const BAGeom& g, int vb,
                                            unsigned char* smraw) {
  using C = cplx<T>;
  const int G2 = p.g.n2, G3 = p.g.n3, K1 = p.b.k1, K2 = p.b.k2, K3 = p.b.k3, H1 = p.b.h1;
  const int KC = g.KC, nch = g.nch, XB = g.XB, R = g.R;
  const long long P = (long long)G2 * G3;
  const long long kvol = (long long)K1 * K2 * K3;
  const int nper = e.nper, ncomp = e.ncomp, nout = e.nout;
  const int ncol = nper * G3;
  C* slab = reinterpret_cast<C*>(smraw);                   // [nper][XB][G3]
  C* E2s = slab + nper * XB * G3;                          // [G2][KC]
  const int G3s = e3_stride<T>(G3);
  C* E3s = E2s + G2 * KC;                                  // [K3][G3s] (transposed E3b)
  C* S1 = E3s + G3s * K3;                                  // [R][nper][KC][G3] (part 0: the sums)
  const int NS = KC * K3;                                  // band slots of an item (at most)
  C* sX = S1 + R * nper * KC * G3;                         // [kEpiX][NS] epilogue terms
  T* sLh = reinterpret_cast<T*>(sX + NS * kEpiX);          // [NS] L^ of the band slots
  const int chunk = vb % nch;
  const int h = (vb / nch) % H1;
  const int c = vb / (nch * H1);
  const int kb = chunk * KC;
  const int kc = min(KC, K2 - kb);
  const int nslot = kc * K3;
  const int tid = threadIdx.x;
  const C zero{T(0), T(0)};

  for (int i = tid; i < G2 * KC; i += kThreads) {
    const int x2 = i / KC, kk = i - x2 * KC;
    if (kk < kc) cp_async(E2s + i, p.E2b + (long long)x2 * K2 + kb + kk); else E2s[i] = zero;
  }
  if (p.E3bt != nullptr) {
    cp_async_run(E3s, p.E3bt, K3 * G3s);
  } else {
    for (int i = tid; i < G3 * K3; i += kThreads) {
      const int x = i / K3, k = i - x * K3;
      cp_async(E3s + k * G3s + x, p.E3b + i);
    }
  }
  for (int it = tid; it < nslot; it += kThreads) {
    const int kk = it / K3, k3 = it - kk * K3;
    cp_async(sLh + it, Lhat + ((long long)h * K2 + kb + kk) * K3 + k3);
  }
  pdl_wait();
  for (int i = tid; i < nslot * kEpiX; i += kThreads) {
    const int jq = i / nslot, it = i - jq * nslot;
    const int j = jq / kMaxX, q = jq - j * kMaxX;
    if (j < nout && q < e.nx[j]) {
      const int kk = it / K3, k3 = it - kk * K3;
      const long long at = (long long)c * kvol + ((long long)h * K2 + kb + kk) * K3 + k3;
      cp_async(sX + jq * NS + it, e.X[j][q] + at);
    }
  }

  C acc[kAccB][kMaxKC];
#pragma unroll
  for (int r = 0; r < kAccB; ++r)
#pragma unroll
    for (int kk = 0; kk < kMaxKC; ++kk) acc[r][kk] = zero;
  for (int x2c = 0; x2c < G2; x2c += XB) {
    const int xb = min(XB, G2 - x2c);
    if (x2c > 0) __syncthreads();
    for (int o = 0; o < nper; ++o) {
      const C* __restrict__ src = P2 + (long long)((o * ncomp + c) * H1 + h) * P + (long long)x2c * G3;
      cp_async_run(slab + o * XB * G3, src, xb * G3);
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kAccB; ++r) {
      const int vt = tid + r * kThreads;
      const int part = vt / ncol, col = vt - part * ncol;
      if (part < R) {
        const int o = col / G3, x3 = col - o * G3;
        const C* sl = slab + o * XB * G3 + x3;
#pragma unroll 4
        for (int xr = ((part - x2c) % R + R) % R; xr < xb; xr += R) {
          const C a = sl[xr * G3];
          const C* er = E2s + (x2c + xr) * KC;
#pragma unroll
          for (int kk = 0; kk < kMaxKC; ++kk)
            if (kk < kc) cmac(acc[r][kk], a, er[kk]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kAccB; ++r) {
    const int vt = tid + r * kThreads;
    const int part = vt / ncol, col = vt - part * ncol;
    if (part < R) {
      const int o = col / G3, x3 = col - o * G3;
      C* Sp = S1 + part * nper * KC * G3;
#pragma unroll
      for (int kk = 0; kk < kMaxKC; ++kk)
        if (kk < kc) Sp[(o * KC + kk) * G3 + x3] = acc[r][kk];
    }
  }
  __syncthreads();
  if (R > 1) {                                             // add the row groups in fixed order
    const int n1 = nper * KC * G3;
    for (int i = tid; i < n1; i += kThreads) {
      C a = S1[i];
      for (int part = 1; part < R; ++part) {
        const C b = S1[part * n1 + i];
        a.x += b.x;
        a.y += b.y;
      }
      S1[i] = a;
    }
    __syncthreads();
  }

  // A': kRed consecutive lanes share one band-slot sum; the sums of every
  // product field go to shared memory (Y [nslot][nper], over the slab area)
  C* Y = slab;                                             // slab no longer read (synced above)
  for (int base = 0; base < nslot * kRed; base += kThreads) {
    const int lin = base + tid;
    const int it = lin / kRed, part = lin % kRed;
    const bool live = it < nslot;
    const int kk = live ? it / K3 : 0;
    const int k3 = live ? it - kk * K3 : 0;
    for (int o = 0; o < nper; ++o) {
      C y = zero;
      if (live) {
        const C* row = S1 + (o * KC + kk) * G3;
        const C* er = E3s + k3 * G3s;
        for (int x = part; x < G3; x += kRed) cmac(y, row[x], er[x]);
      }
#pragma unroll
      for (int off = kRed / 2; off > 0; off >>= 1) {
        y.x += __shfl_down_sync(0xffffffffu, y.x, off, kRed);
        y.y += __shfl_down_sync(0xffffffffu, y.y, off, kRed);
      }
      if (part == 0 && live) Y[it * nper + o] = y;
    }
  }
  __syncthreads();
  // epilogue: one (band slot, output) pair per thread; the X terms were read
  // into shared memory before any output was written (outputs may alias inputs)
  for (int w = tid; w < nslot * nout; w += kThreads) {
    const int it = w / nout, j = w - it * nout;
    const int kk = it / K3, k3 = it - kk * K3;
    const int k2 = kb + kk;
    const bool nq = nyq(k2, K2) || nyq(k3, K3);
    const long long kin = ((long long)h * K2 + k2) * K3 + k3;
    const long long at = (long long)c * kvol + kin;
    C v = zero;
    if (!nq) {
      if (e.r[j] >= 0) {
        const T kh = T(1) / sLh[it];
        C Rj = zero;
#pragma unroll
        for (int o = 0; o < kMaxPer; ++o) {
          if (o < nper && e.grp[o] == e.r[j]) {
            const C y = Y[it * nper + o];
            const T sc = e.coef[o] * (e.applyK[o] ? kh : T(1));
            Rj.x += sc * y.x;
            Rj.y += sc * y.y;
          }
        }
        v.x = e.cR[j] * Rj.x;
        v.y = e.cR[j] * Rj.y;
      }
      const C* xs = sX + j * kMaxX * NS + it;
#pragma unroll
      for (int q = 0; q < kMaxX; ++q) {
        if (q < e.nx[j]) {
          const C x = xs[q * NS];
          v.x += e.cX[j][q] * x.x;
          v.y += e.cX[j][q] * x.y;
        }
      }
    }
    e.dst[j][at] = v;
    if (h > 0) {
      const long long mir = (long long)c * kvol +
          (((long long)((K1 - h) % K1) * K2 + (K2 - k2) % K2) * K3 + (K3 - k3) % K3);
      e.dst[j][mir] = C{v.x, -v.y};
    }
    if (h == 0 && K1 % 2 == 0) e.dst[j][(long long)c * kvol + (((long long)(K1 / 2) * K2 + k2) * K3 + k3)] = zero;
  }
}

// ---------------------------------------------------------------------------
// launch geometry (host and device)
template <typename T>
__host__ __device__ inline size_t ab_smem(const Plan<T>& p, bool tws) {
  const size_t G2e = even_up(p.g.n2), G3e = even_up(p.g.n3);
  size_t n = (size_t)p.b.k2 * p.b.k3 + (size_t)p.b.k2 * G3e;
  if (tws) n += (size_t)p.b.k3 * G3e + (size_t)p.b.k2 * G2e;
  return n * sizeof(cplx<T>) + (size_t)p.b.k2 * p.b.k3 * sizeof(T);
}

// stage the twiddles only while the tile stays small enough for several CTAs
// per SM (large image-grid planes are latency-bound at one CTA per SM)
template <typename T>
__host__ __device__ inline bool ab_tws(const Plan<T>& p) {
  if (p.tws == 1) return false;
  if (p.tws == 2 && ab_smem(p, true) <= (size_t)kMaxSmem) return true;
  return ab_smem(p, true) <= (size_t)64 * 1024;
}

template <typename T>
__host__ __device__ inline size_t cpw_smem(const Plan<T>& p, int TP, int NP) {
  const int G1 = p.g.n1, H1 = p.b.h1;
  return ((size_t)24 * H1 * TP + (size_t)H1 * quad_up(G1) + (size_t)G1 * quad_up(H1)) * sizeof(cplx<T>) +
         (size_t)(24 + NP) * G1 * TP * sizeof(T);
}

template <typename T>
inline bool cpw_tile_ok(const Plan<T>& p, int TP) {
  return TP >= 1 && cpw_smem(p, TP, 9) <= (size_t)kMaxSmem && p.g.n1 * TP <= 2 * kThreads;
}

template <typename T>
inline int cpw_tile(const Plan<T>& p) {
  if (p.tp > 0 && cpw_tile_ok(p, p.tp)) return p.tp;
  const long long P = (long long)p.g.n2 * p.g.n3;
  int TP = (int)std::max(1LL, std::min(8LL, P / 152));
  // products: at most two points per thread, and the tile must fit shared memory
  while (TP > 1 && (cpw_smem(p, TP, 9) > (size_t)kMaxSmem || p.g.n1 * TP > 2 * kThreads)) --TP;
  return TP;
}


template <typename T>
inline size_t ba_smem(const Plan<T>& p, int nper, const BAGeom& g) {
  const size_t G2 = p.g.n2, G3 = p.g.n3, K3 = p.b.k3, KC = g.KC;
  const size_t G3s = (size_t)e3_stride<T>(p.g.n3);
  return ((size_t)nper * g.XB * G3 + G2 * KC + G3s * K3 + (size_t)g.R * nper * KC * G3 + KC * K3 * kEpiX) *
             sizeof(cplx<T>) +
         KC * K3 * sizeof(T);
}

template <typename T>
inline BAGeom ba_geom(const Plan<T>& p, int ncomp, int nper) {
  const int G2 = p.g.n2, G3 = p.g.n3, K2 = p.b.k2;
  const int groups = ncomp * p.b.h1;
  const int want = std::max(1, (304 + groups - 1) / groups);
  int KC = p.kc > 0 ? p.kc : std::max(1, (K2 + want - 1) / want);
  KC = std::min(std::min(KC, kMaxKC), K2);
  const int ncol = nper * G3;
  const int R = std::max(1, std::min(kMaxRows, kThreads / ncol));
  BAGeom g{KC, (K2 + KC - 1) / KC, 1, R};
  const size_t row = (size_t)nper * G3 * sizeof(cplx<T>);
  auto fixed = [&]() { return ba_smem(p, nper, g) - row; };    // all but the slab rows
  // the slab area later holds the A' sums of kc * K3 slots, so XB >= KC (G3 >= K3)
  while (g.KC > 1 && fixed() + row * g.KC > (size_t)kMaxSmem) {
    --g.KC;
    g.nch = (K2 + g.KC - 1) / g.KC;
  }
  // slab rows: as many as keep the CTA within 72 KB (three CTAs per SM); on
  // wide image-grid planes, whose fixed part alone nearly fills that, up to
  // 150 KB instead: every chunk of rows costs one L2 round trip and two block
  // barriers, which dominate when only a few rows fit
  size_t target = 72 * 1024;
  if (fixed() + (size_t)16 * row > target) target = 150 * 1024;
  const size_t rows = fixed() < target ? (target - fixed()) / row : 0;
  g.XB = std::max(g.KC, (int)std::min<size_t>((size_t)G2, rows));
  return g;
}

}  // namespace dev
}  // namespace lddmm
