// Grid-point kernels of the GB300 LDDMM library (sm_103a):
//   * semi-Lagrangian state and incremental-state transport on the image grid
//     (Eqs. 52 and 31),
//   * terminal adjoint fields lambda(1) grad m(1) (Eq. 55, Eq. 58 under GN),
//   * band-vector updates and deterministic FP64 reductions (Eq. 47, Eq. 50),
//   * the deformation-state form (Section 3.3): terminal sampling of I0 at the
//     inverse map, its force fields, and the padded-grid products of the
//     band-limited deformation sweep.
// One thread per grid point or band slot; the transport kernels are bound by
// HBM traffic (coalesced streams plus an L1/L2-served 8-corner gather).
#include "internal.h"

namespace lddmm {
namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ bool nyq(int q, int K) { return (K % 2 == 0) && (2 * q == K); }

// ---- periodic trilinear interpolation ------------------------------------------
// Cell of the point ix - dsp on an axis of n nodes: lower node c0, upper c1,
// weight w of the upper node.  The foot point is kept as integer index plus a
// small offset, never as an absolute coordinate.
template <typename T>
__device__ __forceinline__ void cell(int ix, T dsp, int n, int& c0, int& c1, T& w) {
  const T nd = -dsp;
  T fl = floor(nd);
  w = nd - fl;
  // a non-finite or absurd displacement keeps its NaN weight but a safe index
  if (!(fabs(fl) < T(1e6))) fl = T(0);
  int c = ix + (int)fl;
  if ((unsigned)c >= (unsigned)n) {          // rare: more than one period away
    c %= n;
    if (c < 0) c += n;
  }
  c0 = c;
  c1 = (c + 1 == n) ? 0 : c + 1;
}

__device__ __forceinline__ void corners(const int* c0, const int* c1, int n2, int n3, int* o) {
  const int a0 = c0[0] * n2, a1 = c1[0] * n2;
  o[0] = (a0 + c0[1]) * n3 + c0[2];
  o[1] = (a0 + c0[1]) * n3 + c1[2];
  o[2] = (a0 + c1[1]) * n3 + c0[2];
  o[3] = (a0 + c1[1]) * n3 + c1[2];
  o[4] = (a1 + c0[1]) * n3 + c0[2];
  o[5] = (a1 + c0[1]) * n3 + c1[2];
  o[6] = (a1 + c1[1]) * n3 + c0[2];
  o[7] = (a1 + c1[1]) * n3 + c1[2];
}

template <typename T>
__device__ __forceinline__ T trilin(const T* __restrict__ f, const int* o, const T* w) {
  const T u0 = f[o[0]] + w[2] * (f[o[1]] - f[o[0]]);
  const T u1 = f[o[2]] + w[2] * (f[o[3]] - f[o[2]]);
  const T u2 = f[o[4]] + w[2] * (f[o[5]] - f[o[4]]);
  const T u3 = f[o[6]] + w[2] * (f[o[7]] - f[o[6]]);
  const T v0 = u0 + w[1] * (u1 - u0);
  const T v1 = u2 + w[1] * (u3 - u2);
  return v0 + w[0] * (v1 - v0);
}

// grid index of a flat voxel index (volumes stay below 2^31)
__device__ __forceinline__ void unflat(unsigned idx, unsigned n2, unsigned n3, int* ix) {
  const unsigned r = idx / n3;
  ix[2] = (int)(idx - r * n3);
  const unsigned q = r / n2;
  ix[1] = (int)(r - q * n2);
  ix[0] = (int)q;
}

// This thread's voxel: with G3D the launch is a (32 x 8) block per 32 x3 by 8
// x2 of one x1 plane (no index division; a warp covers 32 consecutive x3),
// else one flat index per thread.  False for threads past the grid.
template <bool G3D>
__device__ __forceinline__ bool voxel(Dims g, unsigned& idx, int* ix) {
  if (G3D) {
    ix[2] = blockIdx.x * 32 + threadIdx.x;
    ix[1] = blockIdx.y * 8 + threadIdx.y;
    ix[0] = blockIdx.z;
    if (ix[2] >= g.n3 || ix[1] >= g.n2) return false;
    idx = ((unsigned)ix[0] * (unsigned)g.n2 + (unsigned)ix[1]) * (unsigned)g.n3 + (unsigned)ix[2];
    return true;
  }
  idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.vol()) return false;
  unflat(idx, g.n2, g.n3, ix);
  return true;
}

// central difference d_j m at grid index ix (periodic), in unit-domain units
template <typename T>
__device__ __forceinline__ T cdiff(const T* __restrict__ m, const int* ix, int j, Dims g) {
  const int n[3] = {g.n1, g.n2, g.n3};
  int p[3] = {ix[0], ix[1], ix[2]}, q[3] = {ix[0], ix[1], ix[2]};
  p[j] = (ix[j] + 1 == n[j]) ? 0 : ix[j] + 1;
  q[j] = (ix[j] == 0) ? n[j] - 1 : ix[j] - 1;
  const T mp = m[(p[0] * g.n2 + p[1]) * g.n3 + p[2]];
  const T mq = m[(q[0] * g.n2 + q[1]) * g.n3 + q[2]];
  return (mp - mq) * (T(0.5) * T(n[j]));
}

// (FP32 plane launches: 32 registers, so eight blocks per SM keep more of the
// 32 corner gathers of a voxel in flight)
template <typename T, bool G3D>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 4 && G3D) ? 8 : 0)
k_transport(const T* __restrict__ m, const T* __restrict__ vn, const T* __restrict__ vc,
            T* __restrict__ mn, T* __restrict__ off, Dims g, T dt) {
  const long long vol = g.vol();
  unsigned idx;
  int ix[3];
  if (!voxel<G3D>(g, idx, ix)) return;
  const int n[3] = {g.n1, g.n2, g.n3};
  T a[3], c0w[3];
  int c0[3], c1[3];
  int o[8];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    a[j] = vn[j * vol + idx];
    cell(ix[j], dt * T(n[j]) * a[j], n[j], c0[j], c1[j], c0w[j]);
  }
  corners(c0, c1, g.n2, g.n3, o);
  T dsp[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T u = trilin(vc + j * vol, o, c0w);
    dsp[j] = T(0.5) * dt * T(n[j]) * (a[j] + u);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) cell(ix[j], dsp[j], n[j], c0[j], c1[j], c0w[j]);
  corners(c0, c1, g.n2, g.n3, o);
  mn[idx] = trilin(m, o, c0w);
#pragma unroll
  for (int j = 0; j < 3; ++j) off[j * vol + idx] = dsp[j];
}

template <typename T, bool G3D>
__global__ void __launch_bounds__(kThreads)
k_grad_dot(const T* __restrict__ m, const T* __restrict__ dv, T* __restrict__ s, Dims g) {
  const long long vol = g.vol();
  unsigned idx;
  int ix[3];
  if (!voxel<G3D>(g, idx, ix)) return;
  T acc = T(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) acc = fma(cdiff(m, ix, j, g), dv[j * vol + idx], acc);
  s[idx] = acc;
}

template <typename T, bool G3D>
__global__ void __launch_bounds__(kThreads)
k_inc_step(const T* __restrict__ dm, const T* __restrict__ s, const T* __restrict__ mnext,
           const T* __restrict__ dvn, const T* __restrict__ off, T* __restrict__ dmn,
           T* __restrict__ sn, Dims g, T dt) {
  const long long vol = g.vol();
  unsigned idx;
  int ix[3];
  if (!voxel<G3D>(g, idx, ix)) return;
  const int n[3] = {g.n1, g.n2, g.n3};
  T snew = T(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) snew = fma(cdiff(mnext, ix, j, g), dvn[j * vol + idx], snew);
  int c0[3], c1[3];
  T w[3];
  int o[8];
#pragma unroll
  for (int j = 0; j < 3; ++j) cell(ix[j], off[j * vol + idx], n[j], c0[j], c1[j], w[j]);
  corners(c0, c1, g.n2, g.n3, o);
  const T dmi = dm ? trilin(dm, o, w) : T(0);
  const T si = trilin(s, o, w);
  dmn[idx] = dmi - T(0.5) * dt * (si + snew);
  sn[idx] = snew;
}

// weights of the 8 cell corners in the order of corners(); w = upper-node weights
template <typename T>
__device__ __forceinline__ void corner_weights(const T* w, T* c) {
  const T a0 = T(1) - w[0], a1 = T(1) - w[1], a2 = T(1) - w[2];
  c[0] = a0 * a1 * a2;
  c[1] = a0 * a1 * w[2];
  c[2] = a0 * w[1] * a2;
  c[3] = a0 * w[1] * w[2];
  c[4] = w[0] * a1 * a2;
  c[5] = w[0] * a1 * w[2];
  c[6] = w[0] * w[1] * a2;
  c[7] = w[0] * w[1] * w[2];
}

// derivatives of the trilinear interpolant (corner values f) with respect to
// the three index coordinates, inside the cell of upper-node weights w
template <typename T>
__device__ __forceinline__ void trilin_grad(const T* f, const T* w, T* g) {
  const T a0 = T(1) - w[0], a1 = T(1) - w[1], a2 = T(1) - w[2];
  g[0] = a1 * (a2 * (f[4] - f[0]) + w[2] * (f[5] - f[1])) + w[1] * (a2 * (f[6] - f[2]) + w[2] * (f[7] - f[3]));
  g[1] = a0 * (a2 * (f[2] - f[0]) + w[2] * (f[3] - f[1])) + w[0] * (a2 * (f[6] - f[4]) + w[2] * (f[7] - f[5]));
  g[2] = a0 * (a1 * (f[1] - f[0]) + w[1] * (f[3] - f[2])) + w[0] * (a1 * (f[5] - f[4]) + w[1] * (f[7] - f[6]));
}

// One step of the exact discrete adjoint of the state transport (the
// semi-Lagrangian form of Eq. 13, reversed): with xi = x - dt v_{n+1}(x),
// u = v_n(xi), X = x - dt/2 (v_{n+1}(x) + u) and m_{n+1}(x) = m_n(X),
//   lam_n      += scatter of lam_{n+1}(x) at X            (atomic)
//   G_n        += scatter of alpha(x) at xi                (atomic)
//   G_{n+1}(x) += alpha - dt N (sum_j alpha_j d v_n,j(xi)/d xi)
// where alpha = -dt/2 N lam_{n+1}(x) d m_n(X)/dX (index units, N per axis).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_adj_step(const T* __restrict__ lam, const T* __restrict__ m, const T* __restrict__ vc,
           const T* __restrict__ vn, const T* __restrict__ off, T* __restrict__ lam_out,
           T* __restrict__ gnext, T* __restrict__ gcur, Dims g, T dt) {
  const long long vol = g.vol();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vol) return;
  int ix[3];
  unflat(idx, g.n2, g.n3, ix);
  const int n[3] = {g.n1, g.n2, g.n3};
  const T l = lam[idx];
  int c0[3], c1[3], o[8];
  T w[3], cw[8], f[8], d[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) cell(ix[j], off[j * vol + idx], n[j], c0[j], c1[j], w[j]);
  corners(c0, c1, g.n2, g.n3, o);
  corner_weights(w, cw);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    f[c] = m[o[c]];
    atomicAdd(lam_out + o[c], cw[c] * l);
  }
  trilin_grad(f, w, d);
  T alpha[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) alpha[j] = T(-0.5) * dt * T(n[j]) * l * d[j];
#pragma unroll
  for (int j = 0; j < 3; ++j) cell(ix[j], dt * T(n[j]) * vn[j * vol + idx], n[j], c0[j], c1[j], w[j]);
  corners(c0, c1, g.n2, g.n3, o);
  corner_weights(w, cw);
  T beta[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T* __restrict__ vj = vc + j * vol;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      f[c] = vj[o[c]];
      atomicAdd(gcur + j * vol + o[c], cw[c] * alpha[j]);
    }
    trilin_grad(f, w, d);
#pragma unroll
    for (int i = 0; i < 3; ++i) beta[i] = fma(alpha[j], d[i], beta[i]);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) gnext[j * vol + idx] += alpha[j] - dt * T(n[j]) * beta[j];
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_terminal_newton(const T* __restrict__ m, const T* __restrict__ y, const T* __restrict__ dm, T c,
                  T* __restrict__ out, Dims g) {
  const long long vol = g.vol();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vol) return;
  int ix[3];
  unflat(idx, g.n2, g.n3, ix);
  const T d = dm[idx], r = m[idx] - y[idx];
#pragma unroll
  for (int j = 0; j < 3; ++j) out[j * vol + idx] = c * (d * cdiff(m, ix, j, g) + r * cdiff(dm, ix, j, g));
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_scaled_diff(const T* __restrict__ a, const T* __restrict__ b, T c, T* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = c * (a[i] - b[i]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_terminal(const T* __restrict__ m, const T* __restrict__ y, int diff, T coef, T* __restrict__ out,
           Dims g) {
  const long long vol = g.vol();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vol) return;
  int ix[3];
  unflat(idx, g.n2, g.n3, ix);
  const T r = coef * (diff ? (m[idx] - y[idx]) : y[idx]);
#pragma unroll
  for (int j = 0; j < 3; ++j) out[j * vol + idx] = r * cdiff(m, ix, j, g);
}

// ---- band vectors -----------------------------------------------------------------
template <typename T>
__global__ void k_hermitianize(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int ncomp,
                               Band b) {
  const long long kvol = b.vol();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncomp * kvol) return;
  const long long c = idx / kvol;
  const long long r = idx % kvol;
  const int k3 = (int)(r % b.k3);
  const int k2 = (int)((r / b.k3) % b.k2);
  const int k1 = (int)(r / ((long long)b.k2 * b.k3));
  cplx<T> v{T(0), T(0)};
  if (!(nyq(k1, b.k1) || nyq(k2, b.k2) || nyq(k3, b.k3))) {
    const long long m = c * kvol +
        (((long long)((b.k1 - k1) % b.k1) * b.k2 + (b.k2 - k2) % b.k2) * b.k3 + (b.k3 - k3) % b.k3);
    const cplx<T> a = in[idx], am = in[m];
    v.x = T(0.5) * (a.x + am.x);
    v.y = T(0.5) * (a.y - am.y);
  }
  out[idx] = v;
}

// ---- conjugate gradients with device-resident scalars (Eq. 45) ------------------
// s[] holds rho, ||b||, <d, Hd>, alpha, rho_new, beta, the stop flag, the
// iterations done, the iteration counter and the "x = d" flag; every update
// reads its coefficient here and does nothing once the stop flag is set, so the
// host needs no round trip per iteration.
__global__ void k_pcg_init(double* s) {
  s[PCG_B] = sqrt(s[PCG_R]);
  s[PCG_DONE] = 0.0;
  s[PCG_ITS] = 0.0;
  s[PCG_K] = 0.0;
  s[PCG_COPY] = 0.0;
}

// out = x + sign s[ci] y unless stopped
template <typename T>
__global__ void k_axpy_dev(cplx<T>* out, const cplx<T>* x, const cplx<T>* y, const double* s, int ci, double sign,
                           long long n) {
  if (s[PCG_DONE] != 0.0) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T b = (T)(sign * s[ci]);
  cplx<T> v = x[i];
  v.x = fma(b, y[i].x, v.x);
  v.y = fma(b, y[i].y, v.y);
  out[i] = v;
}

template <typename T>
__global__ void k_axpby(cplx<T>* out, T a, const cplx<T>* x, T bc, const cplx<T>* y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cplx<T> v = x[i];
  v.x *= a;
  v.y *= a;
  if (y) {
    v.x = fma(bc, y[i].x, v.x);
    v.y = fma(bc, y[i].y, v.y);
  }
  out[i] = v;
}

template <typename T>
__global__ void k_scale_L(cplx<T>* out, const cplx<T>* x, const T* __restrict__ L, long long kvol,
                          long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T l = L[i % kvol];
  out[i] = cplx<T>{l * x[i].x, l * x[i].y};
}

// ---- deterministic FP64 reductions ------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < kThreads / 32) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_sumsq_diff(const T* __restrict__ a, const T* __restrict__ b, long long n, double* partial) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)a[i] - (double)b[i];
    acc = fma(d, d, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_inner_V(const cplx<T>* __restrict__ a, const cplx<T>* __restrict__ b, const T* __restrict__ L,
          long long kvol, long long n, double* partial) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double l = (double)L[i % kvol];
    acc = fma(l, (double)a[i].x * (double)b[i].x + (double)a[i].y * (double)b[i].y, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_finalize(const double* partial, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) acc += partial[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}


// ---- deformation-state form (Section 3.3) ------------------------------------
// central-difference gradient of an image, [3][vol]
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_central_grad(const T* __restrict__ m, T* __restrict__ g3, Dims g) {
  const long long vol = g.vol();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vol) return;
  int ix[3];
  unflat(idx, g.n2, g.n3, ix);
#pragma unroll
  for (int j = 0; j < 3; ++j) g3[j * vol + idx] = cdiff(m, ix, j, g);
}

// m(1)(x) = I0(x + u(x)) and gs(x) = (grad I0)(x + u(x)), both by periodic
// trilinear interpolation; u is the grid displacement in unit-box units
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_def_sample(const T* __restrict__ I0, const T* __restrict__ gI0, const T* __restrict__ u,
             T* __restrict__ m1, T* __restrict__ gs, Dims g) {
  const long long vol = g.vol();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vol) return;
  int ix[3];
  unflat(idx, g.n2, g.n3, ix);
  const int n[3] = {g.n1, g.n2, g.n3};
  T w[3];
  int c0[3], c1[3], o[8];
#pragma unroll
  for (int j = 0; j < 3; ++j) cell(ix[j], -u[j * vol + idx] * T(n[j]), n[j], c0[j], c1[j], w[j]);
  corners(c0, c1, g.n2, g.n3, o);
  m1[idx] = trilin(I0, o, w);
#pragma unroll
  for (int j = 0; j < 3; ++j) gs[j * vol + idx] = trilin(gI0 + j * vol, o, w);
}

// terminal force of the deformation form on the image grid, f = [3][vol]:
//   du == nullptr:  f = c (m1 - I1) gs             (lambda(1) grad I0 o phi^-1, c = -2/sigma^2)
//   otherwise:      dm = gs . du,  f = c dm gs     (its Gauss-Newton increment); dm -> dm_out
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_def_force(const T* __restrict__ gs, const T* __restrict__ m1, const T* __restrict__ I1,
            const T* __restrict__ du, T* __restrict__ dm_out, T c, T* __restrict__ f, long long vol) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vol) return;
  const T g0 = gs[idx], g1 = gs[vol + idx], g2 = gs[2 * vol + idx];
  T a;
  if (du == nullptr) {
    a = c * (m1[idx] - I1[idx]);
  } else {
    const T dm = fma(g0, du[idx], fma(g1, du[vol + idx], g2 * du[2 * vol + idx]));
    if (dm_out) dm_out[idx] = dm;
    a = c * dm;
  }
  f[idx] = a * g0;
  f[vol + idx] = a * g1;
  f[2 * vol + idx] = a * g2;
}

// pointwise products of the deformation form on the padded grid; fields are
// [12][vol] blocks {Jacobian D[3 i + j] = d_j a_i, values}:
//   mode 0:  out_i = -(v_i + sum_j D_ij v_j)                      fl = {D u, v}
//   mode 1:  out_i = -(dv_i + sum_j dD_ij v_j + D_ij dv_j)         fl = {D du, dv}, fc = {D u, v}
//   mode 2:  out_i = r_i + sum_j D_ji r_j                           fl = {D u, r}
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_def_products(int mode, const T* __restrict__ fl, const T* __restrict__ fc, T* __restrict__ out,
               long long vol) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vol) return;
  const T* src = mode == 1 ? fc : fl;       // the block holding D u and v (or r)
  T D[9], v[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) D[q] = src[q * vol + idx];
#pragma unroll
  for (int j = 0; j < 3; ++j) v[j] = src[(9 + j) * vol + idx];
  if (mode == 2) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T acc = v[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) acc = fma(D[3 * j + i], v[j], acc);
      out[i * vol + idx] = acc;
    }
    return;
  }
  if (mode == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T a = T(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) a = fma(D[3 * i + j], v[j], a);
      out[i * vol + idx] = -(v[i] + a);
    }
    return;
  }
  T dD[9], dv[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) dD[q] = fl[q * vol + idx];
#pragma unroll
  for (int j = 0; j < 3; ++j) dv[j] = fl[(9 + j) * vol + idx];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T a = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) a = fma(dD[3 * i + j], v[j], fma(D[3 * i + j], dv[j], a));
    out[i * vol + idx] = -(dv[i] + a);
  }
}


// ---- PCG steps with the scalar logic folded into the reductions ---------------
// <d, q>_V from the block partials, then alpha, or the stop at non-positive
// curvature (a stop on the first iteration returns x = d, the steepest-descent
// direction)
__global__ void __launch_bounds__(kThreads) k_finalize_alpha(const double* partial, int n, double* s) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) acc += partial[i];
  acc = block_sum(acc);
  if (threadIdx.x != 0) return;
  const double k = s[PCG_K] + 1.0;
  s[PCG_K] = k;
  s[PCG_COPY] = 0.0;
  s[PCG_DQ] = acc;
  if (s[PCG_DONE] != 0.0) {
    s[PCG_A] = 0.0;
    return;
  }
  if (!(acc > 0.0)) {
    s[PCG_DONE] = 1.0;
    s[PCG_ITS] = k - 1.0;
    if (k == 1.0) s[PCG_COPY] = 1.0;
    s[PCG_A] = 0.0;
    return;
  }
  s[PCG_A] = s[PCG_R] / acc;
}

// x = d on a first-iteration curvature stop; else (unless stopped) x += alpha d,
// r -= alpha q; block partials of <r, r>_V
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pcg_xr(cplx<T>* __restrict__ x, cplx<T>* __restrict__ r, const cplx<T>* __restrict__ d,
         const cplx<T>* __restrict__ q, const T* __restrict__ L, long long kvol, long long n,
         const double* s, double* partial) {
  const bool copy = s[PCG_COPY] != 0.0;
  const bool done = s[PCG_DONE] != 0.0;
  const T a = (T)s[PCG_A];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (copy) x[i] = d[i];
    if (done) continue;
    cplx<T> xv = x[i], rv = r[i];
    const cplx<T> dv = d[i], qv = q[i];
    xv.x = fma(a, dv.x, xv.x);
    xv.y = fma(a, dv.y, xv.y);
    rv.x = fma(-a, qv.x, rv.x);
    rv.y = fma(-a, qv.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    const double l = (double)L[i % kvol];
    acc = fma(l, (double)rv.x * (double)rv.x + (double)rv.y * (double)rv.y, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// <r, r>_V from the block partials, then the stop on the relative residual
// ||r||_V <= tol ||b||_V, or beta = rho_new / rho
__global__ void __launch_bounds__(kThreads) k_finalize_beta(const double* partial, int n, double* s, double tol) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) acc += partial[i];
  acc = block_sum(acc);
  if (threadIdx.x != 0) return;
  s[PCG_RN] = acc;
  if (s[PCG_DONE] != 0.0) return;
  s[PCG_ITS] = s[PCG_K];
  if (sqrt(acc) <= tol * s[PCG_B]) {
    s[PCG_DONE] = 1.0;
    return;
  }
  s[PCG_BETA] = acc / s[PCG_R];
  s[PCG_R] = acc;
}

}  // namespace

// planes of at least 32 x3 points take the (32 x 8)-block launch of voxel<true>
inline bool plane_launch(Dims g) { return g.n3 >= 32; }
inline dim3 plane_grid(Dims g) { return dim3((unsigned)(g.n3 + 31) / 32, (unsigned)(g.n2 + 7) / 8, (unsigned)g.n1); }

template <typename T>
void transport_step(const T* m, const T* vnext, const T* vcur, T* mnext, T* off, Dims g, double dt,
                    cudaStream_t st) {
  if (plane_launch(g))
    k_transport<T, true><<<plane_grid(g), dim3(32, 8), 0, st>>>(m, vnext, vcur, mnext, off, g, (T)dt);
  else
    k_transport<T, false><<<blocks_for(g.vol()), kThreads, 0, st>>>(m, vnext, vcur, mnext, off, g, (T)dt);
}

template <typename T>
void grad_dot(const T* m, const T* dv, T* s, Dims g, cudaStream_t st) {
  if (plane_launch(g))
    k_grad_dot<T, true><<<plane_grid(g), dim3(32, 8), 0, st>>>(m, dv, s, g);
  else
    k_grad_dot<T, false><<<blocks_for(g.vol()), kThreads, 0, st>>>(m, dv, s, g);
}

template <typename T>
void inc_step(const T* dm, const T* s, const T* mnext, const T* dvnext, const T* off, T* dmnext,
              T* snext, Dims g, double dt, cudaStream_t st) {
  if (plane_launch(g))
    k_inc_step<T, true><<<plane_grid(g), dim3(32, 8), 0, st>>>(dm, s, mnext, dvnext, off, dmnext, snext, g,
                                                               (T)dt);
  else
    k_inc_step<T, false><<<blocks_for(g.vol()), kThreads, 0, st>>>(dm, s, mnext, dvnext, off, dmnext, snext,
                                                                   g, (T)dt);
}

template <typename T>
void adjoint_step(const T* lam, const T* m, const T* vcur, const T* vnext, const T* off, T* lam_out, T* gnext,
                  T* gcur, Dims g, double dt, cudaStream_t st) {
  k_adj_step<T><<<blocks_for(g.vol()), kThreads, 0, st>>>(lam, m, vcur, vnext, off, lam_out, gnext, gcur, g,
                                                         (T)dt);
}

template <typename T>
void terminal_newton(const T* m, const T* y, const T* dm, double c, T* out, Dims g, cudaStream_t st) {
  k_terminal_newton<T><<<blocks_for(g.vol()), kThreads, 0, st>>>(m, y, dm, (T)c, out, g);
}

template <typename T>
void scaled_diff(const T* a, const T* b, double c, T* out, long long n, cudaStream_t st) {
  k_scaled_diff<T><<<blocks_for(n), kThreads, 0, st>>>(a, b, (T)c, out, n);
}

template <typename T>
void terminal_field(const T* m, const T* y, int diff, double coef, T* out, Dims g, cudaStream_t st) {
  k_terminal<T><<<blocks_for(g.vol()), kThreads, 0, st>>>(m, y, diff, (T)coef, out, g);
}

template <typename T>
void hermitianize(const cplx<T>* in, cplx<T>* out, int ncomp, Band b, cudaStream_t st) {
  k_hermitianize<T><<<blocks_for(ncomp * b.vol()), kThreads, 0, st>>>(in, out, ncomp, b);
}

template <typename T>
void axpby(cplx<T>* out, double a, const cplx<T>* x, double bcoef, const cplx<T>* y, long long n,
           cudaStream_t st) {
  k_axpby<T><<<blocks_for(n), kThreads, 0, st>>>(out, (T)a, x, (T)bcoef, y, n);
}

void pcg_init(double* s, cudaStream_t st) { k_pcg_init<<<1, 1, 0, st>>>(s); }

template <typename T>
void scale_L(cplx<T>* out, const cplx<T>* x, const T* Lhat, int ncomp, long long kvol, cudaStream_t st) {
  k_scale_L<T><<<blocks_for(ncomp * kvol), kThreads, 0, st>>>(out, x, Lhat, kvol, ncomp * kvol);
}

template <typename T>
void sum_sq_diff(const T* a, const T* b, long long n, double* partial, double* out, cudaStream_t st) {
  k_sumsq_diff<T><<<kReduceBlocks, kThreads, 0, st>>>(a, b, n, partial);
  k_finalize<<<1, kThreads, 0, st>>>(partial, kReduceBlocks, out);
}

template <typename T>
void inner_V(const cplx<T>* a, const cplx<T>* b, const T* Lhat, int ncomp, long long kvol,
             double* partial, double* out, cudaStream_t st) {
  k_inner_V<T><<<kReduceBlocks, kThreads, 0, st>>>(a, b, Lhat, kvol, ncomp * kvol, partial);
  k_finalize<<<1, kThreads, 0, st>>>(partial, kReduceBlocks, out);
}

template <typename T>
void pcg_step(cplx<T>* x, cplx<T>* r, cplx<T>* d, const cplx<T>* q, const T* Lhat, long long kvol, int ncomp,
              double* partial, double* s, double tol, cudaStream_t st) {
  const long long n = ncomp * kvol;
  k_inner_V<T><<<kReduceBlocks, kThreads, 0, st>>>(d, q, Lhat, kvol, n, partial);
  k_finalize_alpha<<<1, kThreads, 0, st>>>(partial, kReduceBlocks, s);
  k_pcg_xr<T><<<kReduceBlocks, kThreads, 0, st>>>(x, r, d, q, Lhat, kvol, n, s, partial);
  k_finalize_beta<<<1, kThreads, 0, st>>>(partial, kReduceBlocks, s, tol);
  k_axpy_dev<T><<<blocks_for(n), kThreads, 0, st>>>(d, r, d, s, PCG_BETA, 1.0, n);
}

template <typename T>
void central_grad(const T* m, T* g3, Dims g, cudaStream_t st) {
  k_central_grad<T><<<blocks_for(g.vol()), kThreads, 0, st>>>(m, g3, g);
}

template <typename T>
void def_sample(const T* I0, const T* gI0, const T* u, T* m1, T* gs, Dims g, cudaStream_t st) {
  k_def_sample<T><<<blocks_for(g.vol()), kThreads, 0, st>>>(I0, gI0, u, m1, gs, g);
}

template <typename T>
void def_force(const T* gs, const T* m1, const T* I1, const T* du, T* dm_out, double c, T* f, long long vol,
               cudaStream_t st) {
  k_def_force<T><<<blocks_for(vol), kThreads, 0, st>>>(gs, m1, I1, du, dm_out, (T)c, f, vol);
}

template <typename T>
void def_products(int mode, const T* fields, const T* cached, T* out, long long vol, cudaStream_t st) {
  k_def_products<T><<<blocks_for(vol), kThreads, 0, st>>>(mode, fields, cached, out, vol);
}

#define LDDMM_INST(T)                                                                              \
  template void pcg_step<T>(cplx<T>*, cplx<T>*, cplx<T>*, const cplx<T>*, const T*, long long, int,  \
                            double*, double*, double, cudaStream_t);                                \
  template void central_grad<T>(const T*, T*, Dims, cudaStream_t);                                 \
  template void def_sample<T>(const T*, const T*, const T*, T*, T*, Dims, cudaStream_t);           \
  template void def_force<T>(const T*, const T*, const T*, const T*, T*, double, T*, long long,    \
                             cudaStream_t);                                                        \
  template void def_products<T>(int, const T*, const T*, T*, long long, cudaStream_t);            \
  template void transport_step<T>(const T*, const T*, const T*, T*, T*, Dims, double,            \
                                  cudaStream_t);                                                 \
  template void grad_dot<T>(const T*, const T*, T*, Dims, cudaStream_t);                         \
  template void inc_step<T>(const T*, const T*, const T*, const T*, const T*, T*, T*, Dims,      \
                            double, cudaStream_t);                                               \
  template void terminal_field<T>(const T*, const T*, int, double, T*, Dims, cudaStream_t);      \
  template void adjoint_step<T>(const T*, const T*, const T*, const T*, const T*, T*, T*, T*, Dims,  \
                                double, cudaStream_t);                                              \
  template void scaled_diff<T>(const T*, const T*, double, T*, long long, cudaStream_t);          \
  template void terminal_newton<T>(const T*, const T*, const T*, double, T*, Dims, cudaStream_t);  \
  template void hermitianize<T>(const cplx<T>*, cplx<T>*, int, Band, cudaStream_t);             \
  template void axpby<T>(cplx<T>*, double, const cplx<T>*, double, const cplx<T>*, long long,    \
                         cudaStream_t);                                                          \
  template void scale_L<T>(cplx<T>*, const cplx<T>*, const T*, int, long long, cudaStream_t);    \
  template void sum_sq_diff<T>(const T*, const T*, long long, double*, double*, cudaStream_t);   \
  template void inner_V<T>(const cplx<T>*, const cplx<T>*, const T*, int, long long, double*,    \
                           double*, cudaStream_t);
LDDMM_INST(float)
LDDMM_INST(double)

}  // namespace lddmm
