// Internal declarations of the GB300 LDDMM library: data layouts, transform
// plans, launch descriptors and kernel launchers.  Not part of the C interface.
//
// Internally every problem is three-dimensional with three velocity
// components: a 2D problem is the slab N_3 = 1, K_3 = 1 with a zero third
// component (the 3D formulas then reduce exactly to the 2D ones).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace lddmm {

// The kernels of a bracket evaluation launch with programmatic dependent
// launch (their prologues overlap the previous kernel); building with
// -DLDDMM_NO_PDL launches them plainly (same results, for comparison).
#ifdef LDDMM_NO_PDL
constexpr bool kUsePdl = false;
#else
constexpr bool kUsePdl = true;
#endif

// Launch attributes of the bracket-evaluation chain, written from at[0]:
// programmatic stream serialisation, unless built with LDDMM_NO_PDL.
// Returns the number of attributes written (at most 1).
inline unsigned chain_attrs(cudaLaunchAttribute* at) {
  if (!kUsePdl) return 0;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  return 1;
}

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

// Grid sizes of one transform plan: the image grid N or the padded product
// grid M = ceil(3K/2).
struct Dims {
  int n1, n2, n3;
  __host__ __device__ long long vol() const { return (long long)n1 * n2 * n3; }
};

// Band sizes K_j and h1 = number of non-negative k1 slots kept by the
// Hermitian half-spectrum transforms (K_1/2, or 1 for a degenerate axis).
struct Band {
  int k1, k2, k3, h1;
  __host__ __device__ long long vol() const { return (long long)k1 * k2 * k3; }
};

// Twiddle tables of one (grid, band) pair, device resident, precision T.
//   E3f[k3][x3] = exp(+2 pi i f(k3) x3 / G3)          (iota, axis 3)
//   E2f[k2][x2] = exp(+2 pi i f(k2) x2 / G2)          (iota, axis 2)
//   E1f[h][x1]  = w(h) exp(+2 pi i h x1 / G1), w = 1 (h = 0) or 2
//   E1b[x1][h]  = exp(-2 pi i h x1 / G1)              (pi, axis 1)
//   E2b[x2][k2] = exp(-2 pi i f(k2) x2 / G2)
//   E3b[x3][k3] = exp(-2 pi i f(k3) x3 / G3)
template <typename T>
struct Plan {
  Dims g;
  Band b;
  cplx<T>* E3f;
  cplx<T>* E2f;
  cplx<T>* E1f;
  cplx<T>* E1b;
  cplx<T>* E2b;
  cplx<T>* E3b;
  // tile overrides of the bracket kernels, set by the autotuner (0: the size
  // heuristics): tws 1 = twiddles from global memory, 2 = staged in shared
  // memory (iota A+B); tp = pencils per tile (C/products/C'); kc = band rows
  // per item (pi B'/A')
  int tws = 0, tp = 0, kc = 0;
  // split of the FP32 tensor-core image-grid transform: 0 3xTF32, 1 BF16x3
  int split = 0;
  // FP32 padded plans: the tcgen05 iota A+B twiddle operands, expanded once
  // into the kernel's shared-memory layout (nullptr: expanded in the kernel)
  const float* tc_ab = nullptr;
  // FP32 padded plans: the tcgen05 pi B'+A' twiddle operands (real form, hi/lo,
  // in the kernel's shared-memory layout); nullptr: the SIMT kernel runs
  const float* tc_pi = nullptr;
  // FP32 padded plans: the tcgen05 C / C' twiddle operands of the middle phase
  // (tc_cpw.cu); with them set, tp is the tensor-core tile (8 pencils)
  const float* tc_cpw = nullptr;
  // the twiddle tiles exactly as the phase bodies stage them in shared memory
  // (zero padded / transposed), so a phase copies them contiguously; nullptr:
  // the phases build the tiles from the tables above
  cplx<T>* E3fp = nullptr;   // [K3][G3e]  iota A (E3f, rows padded to even length)
  cplx<T>* E2fp = nullptr;   // [K2][G2e]  iota B (E2f, padded to even length)
  cplx<T>* E1fp = nullptr;   // [H1][G1q]  iota C (E1f, padded to a multiple of 4)
  cplx<T>* E1bp = nullptr;   // [G1][H1q]  pi C' (E1b, padded to a multiple of 4)
  cplx<T>* E3bt = nullptr;   // [K3][G3s]  pi A' (E3b transposed, bank-spread row stride)
};

// iota batch: field f is iota of (multiplier x one scalar band slab), where
// the multiplier is L^(k) if applyL and 2 pi i f_deriv(k) if deriv >= 0.
constexpr int kMaxIota = 36;
template <typename T>
struct IotaDesc {
  int nf;
  const cplx<T>* src[kMaxIota];   // scalar band slab [K1][K2][K3]
  T* dst[kMaxIota];               // grid field [G1][G2][G3]
  signed char deriv[kMaxIota];    // -1 or axis 0..2
  signed char applyL[kMaxIota];
};

// pi batch inputs: nf real grid fields.
constexpr int kMaxPi = 36;
template <typename T>
struct PiSrc {
  int nf;
  const T* src[kMaxPi];
};

// Epilogue of the last pi stage.  The pi fields are indexed f = o*ncomp + c
// (o < nper).  For band slot k of component c:
//   R_r(k) = sum_{o: grp[o]==r} coef[o] * (applyK[o] ? 1/L^(k) : 1) * pi_o(k)
//   dst_j(k) = cR[j] * R_{r[j]}(k) + sum_i cX[j][i] * X[j][i](k)
// coef includes the 1/(G1 G2 G3) normalisation.  X and dst are band vectors
// [ncomp][K1][K2][K3]; outputs are written Hermitian with zero Nyquist slots.
constexpr int kMaxPer = 3, kMaxOut = 4, kMaxX = 4;
template <typename T>
struct PiEpi {
  int ncomp, nper;
  int grp[kMaxPer];
  T coef[kMaxPer];
  int applyK[kMaxPer];
  int nout;
  cplx<T>* dst[kMaxOut];
  int r[kMaxOut];
  T cR[kMaxOut];
  int nx[kMaxOut];
  const cplx<T>* X[kMaxOut][kMaxX];
  T cX[kMaxOut][kMaxX];
};

// ---- transforms (dft.cu) --------------------------------------------------
// Scratch: T2 holds [F][h1][G2][G3] complex (iota intermediate, and the C'
// output of pi), P2 holds [9][h1][M2][M3] complex (C' of a bracket evaluation).
// tc_flag != nullptr selects the tcgen05 3xTF32 form of stage C (FP32 plans
// it supports); the kernel sets *tc_flag = 1 if its bounded MMA wait gives up.
template <typename T>
void iota_batch(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2,
                cudaStream_t st, double* tc_flag = nullptr);
// stage C of iota alone (T2 from bracket_iota): the tcgen05 form where
// tc_flag != nullptr and the plan supports it, else the SIMT kernel
template <typename T>
void iota_c_stage(const Plan<T>& p, const IotaDesc<T>& d, cplx<T>* T2, cudaStream_t st, double* tc_flag);
// stage C' of pi alone: the C' sums of s into P2 [nf][h1][G2][G3] (for bracket_pi)
template <typename T>
void pi_c_stage(const Plan<T>& p, const PiSrc<T>& s, cplx<T>* P2, cudaStream_t st);
// tcgen05 image-grid stage C (tc_iota.cu)
bool iota_C_tc_supported(const Plan<float>& p);
// tcgen05 iota stages A + B of a padded-grid bracket block (tc_bracket.cu)
bool iota_ab_tc_supported(const Plan<float>& p);
// floats of the expanded twiddle operands, and the expansion into dst (device)
size_t iota_ab_tc_twiddle_floats(const Plan<float>& p);
cudaError_t iota_ab_tc_twiddles(const Plan<float>& p, float* dst, cudaStream_t st);
cudaError_t iota_ab_tc(const Plan<float>& p, const IotaDesc<float>& d, const float* Lhat, float2* T2,
                       double* flag, cudaStream_t st);
cudaError_t iota_C_tc(const Plan<float>& p, const IotaDesc<float>& d, const float2* T2, double* flag,
                      cudaStream_t st);
// tcgen05 C + bracket products + C' of a padded-grid bracket block (tc_cpw.cu)
enum PwMode : int;
bool cpw_tc_supported(const Plan<float>& p);
int cpw_tc_tile();
size_t cpw_tc_twiddle_floats(const Plan<float>& p);
cudaError_t cpw_tc_twiddles(const Plan<float>& p, float* dst, cudaStream_t st);
cudaError_t cpw_tc(const Plan<float>& p, PwMode mode, const float2* T2, float* slot, float* slot2, float2* P2,
                   double* flag, cudaStream_t st);
// tcgen05 pi stages B' + A' with the epilogue on a padded-grid bracket block (tc_pi.cu)
bool pi_ba_tc_supported(const Plan<float>& p);
size_t pi_ba_tc_twiddle_floats(const Plan<float>& p);
cudaError_t pi_ba_tc_twiddles(const Plan<float>& p, float* dst, cudaStream_t st);
cudaError_t pi_ba_tc(const Plan<float>& p, const PiEpi<float>& e, const float* Lhat, const float2* P2,
                     double* flag, cudaStream_t st);
template <typename T>
void pi_batch(const Plan<T>& p, const PiSrc<T>& s, const PiEpi<T>& e, const T* Lhat,
              cplx<T>* P2, cudaStream_t st);
// number of kernel launches of one iota_batch / pi_batch call
constexpr int kIotaLaunches = 2, kPiLaunches = 2, kBracketLaunches = 3;

enum PwMode : int { PW_F = 0, PW_T = 1, PW_GT = 2 };
// One bracket evaluation on the padded plan p runs three kernels:
//   bracket_iota  iota stages A+B of the 24 fields of d (layout per field
//                 block: value[3], jac[3][3], Lvalue[3], Ljac[3][3], with
//                 jac[c][j] = d_j a_c) -> T2;
//   bracket_cpw   stage C, the bracket products and pi stage C' of the 3
//                 (PW_F: P(v, L v); PW_T: P(dv, L v) + P(v, L dv)) or 9
//                 (PW_GT: P(v, L U), P(W, L v), Q(v, W)) product fields -> P2;
//                 slot holds the 24 fields of the stage point, written in PW_F
//                 (d's own fields) and read in PW_T and PW_GT;
//   bracket_pi    pi stages B'+A' of P2 and the epilogue e.
template <typename T>
void bracket_iota(const Plan<T>& p, const IotaDesc<T>& d, const T* Lhat, cplx<T>* T2, cudaStream_t st,
                  double* tc_flag = nullptr);
template <typename T>
void bracket_cpw(const Plan<T>& p, PwMode mode, const cplx<T>* T2, T* slot, T* slot2, cplx<T>* P2,
                 cudaStream_t st, double* tc_flag = nullptr);
// tc_flag != nullptr selects the tcgen05 form (FP32 plans with p.tc_pi set)
template <typename T>
void bracket_pi(const Plan<T>& p, const PiEpi<T>& e, const T* Lhat, const cplx<T>* P2,
                cudaStream_t st, double* tc_flag = nullptr);
// One bracket evaluation of a persistent sweep: iota sources (value/Jacobian
// block from srcA, L~ block from srcB), stage-point slot and pi epilogue.
template <typename T>
struct EvalDesc {
  const cplx<T>* srcA;
  const cplx<T>* srcB;
  T* slot;
  T* slot2;      // tangent sweeps: where to cache the fields of A (nullptr: none)
  PiEpi<T> epi;
};
// Every evaluation of a band-limited sweep in one cooperative launch
// (sweep.cu); ev is a device array of nev descriptors of one mode.  bar:
// kSweepBarWords device unsigned ints of barrier state (the grid-barrier
// arrival counter and one completion counter per (component, h) band slab);
// flag: device double set to 1 if a wait gave up.  stall > 0 is the test hook
// of the time-out path: the first grid barrier then waits for one arrival more
// than the grid has and every wait gives up after `stall` polls.
constexpr int kSweepBarWords = 128;
template <typename T>
cudaError_t sweep_launch(const Plan<T>& p, PwMode mode, const EvalDesc<T>* ev, int nev, const T* Lhat,
                         cplx<T>* T2, cplx<T>* P2, unsigned* bar, double* flag, cudaStream_t st,
                         int stall = 0);

// largest dynamic shared memory the transform kernels need on plan p when pi
// batches hold up to nper_max fields per component and (brackets) bracket
// evaluations run on it; SIZE_MAX if the plan's G3 is too long for the pi
// kernel's accumulators.  smem_limit() is the configured maximum.
template <typename T>
size_t max_smem_needed(const Plan<T>& p, int nper_max, bool brackets);
size_t smem_limit();
// floats of one stage-point cache slot of a bracket evaluation: the 24 grid
// fields of every pencil tile of the C/products/C' phase, tile-major
// [tile][24][M1][TP] so that a tile's fields are one contiguous block
template <typename T>
long long cache_slot_elems(const Plan<T>& p);
// row lengths of the staged twiddle tiles: G3e, G2e, G1q, H1q, G3s
template <typename T>
void staged_twiddle_dims(const Plan<T>& p, int* G3e, int* G2e, int* G1q, int* H1q, int* G3s);
// tile shapes in effect for a padded-grid plan (overrides or size heuristics):
// twiddle staging of iota A+B (1 off, 2 on), pencils per tile of the
// C/products/C' phase, band rows per pi B'/A' item (for 3 product fields)
template <typename T>
void tile_config(const Plan<T>& p, int* tws, int* tp, int* kc);
// whether a tile override is usable on this plan
template <typename T>
bool tile_valid(const Plan<T>& p, int tws, int tp, int kc);

// ---- grid kernels (grid.cu) -----------------------------------------------
// Semi-Lagrangian state step (Eq. 52): m_next(x) = m(X_n(x)), foot point from
// v_next (at x) and v_cur (trilinear); also writes the displacement off[3].
template <typename T>
void transport_step(const T* m, const T* vnext, const T* vcur, T* mnext, T* off,
                    Dims g, double dt, cudaStream_t st);
// s = grad m . dv (central differences).
template <typename T>
void grad_dot(const T* m, const T* dv, T* s, Dims g, cudaStream_t st);
// Incremental state step (Eq. 31) along the stored characteristic; dm may be
// null (dm_0 = 0).
template <typename T>
void inc_step(const T* dm, const T* s, const T* mnext, const T* dvnext, const T* off,
              T* dmnext, T* snext, Dims g, double dt, cudaStream_t st);
// out_j = coef * r * d_j m, r = (m - y) if diff else y.
template <typename T>
void terminal_field(const T* m, const T* y, int diff, double coef, T* out, Dims g,
                    cudaStream_t st);
// ---- deformation-state form (Section 3.3) ----
// central-difference gradient of an image -> [3][vol]
template <typename T>
void central_grad(const T* m, T* g3, Dims g, cudaStream_t st);
// m1(x) = I0(x + u(x)), gs(x) = (grad I0)(x + u(x)) (trilinear, periodic); u [3][vol]
// in unit-box units
template <typename T>
void def_sample(const T* I0, const T* gI0, const T* u, T* m1, T* gs, Dims g, cudaStream_t st);
// f = c (m1 - I1) gs (du == nullptr), else dm = gs . du (-> dm_out if given) and
// f = c dm gs; f [3][vol]
template <typename T>
void def_force(const T* gs, const T* m1, const T* I1, const T* du, T* dm_out, double c, T* f, long long vol,
               cudaStream_t st);
// padded-grid products (blocks of 12 fields [12][vol]: Jacobian D[3 i + j] = d_j a_i,
// then 3 values):
//   0: out_i = -(v_i + D_ij v_j)                 fields {D u, v}
//   1: out_i = -(dv_i + dD_ij v_j + D_ij dv_j)    fields {D du, dv}, cached {D u, v}
//   2: out_i = r_i + D_ji r_j                     fields {D u, r}
template <typename T>
void def_products(int mode, const T* fields, const T* cached, T* out, long long vol, cudaStream_t st);
// one reversed step of the exact discrete adjoint of the state transport:
// lam_out (zeroed by the caller) and gcur gain atomic scatters, gnext gains the
// per-voxel terms (see grid.cu); off is the step's stored displacement.
template <typename T>
void adjoint_step(const T* lam, const T* m, const T* vcur, const T* vnext, const T* off, T* lam_out, T* gnext,
                  T* gcur, Dims g, double dt, cudaStream_t st);
// out_j = c (dm d_j m + (m - y) d_j dm): the terminal field of the full-Newton
// incremental adjoint (central differences)
template <typename T>
void terminal_newton(const T* m, const T* y, const T* dm, double c, T* out, Dims g, cudaStream_t st);
// out = c (a - b)
template <typename T>
void scaled_diff(const T* a, const T* b, double c, T* out, long long n, cudaStream_t st);

// ---- band vectors and reductions (grid.cu) --------------------------------
template <typename T>
void hermitianize(const cplx<T>* in, cplx<T>* out, int ncomp, Band b, cudaStream_t st);
// out = a x + b y (complex arrays of n entries; y may be null).
template <typename T>
void axpby(cplx<T>* out, double a, const cplx<T>* x, double bcoef, const cplx<T>* y,
           long long n, cudaStream_t st);
// out = L^ x per band slot (V representative -> l2 gradient).
template <typename T>
void scale_L(cplx<T>* out, const cplx<T>* x, const T* Lhat, int ncomp, long long kvol, cudaStream_t st);
// FP64 reductions written to a device double (deterministic two-pass tree).
template <typename T>
void sum_sq_diff(const T* a, const T* b, long long n, double* partial, double* out,
                 cudaStream_t st);
template <typename T>
void inner_V(const cplx<T>* a, const cplx<T>* b, const T* Lhat, int ncomp, long long kvol,
             double* partial, double* out, cudaStream_t st);
constexpr int kReduceBlocks = 304;   // 2 x 152 SMs
// device-resident conjugate-gradient scalars (grid.cu)
enum PcgSlot { PCG_R = 0, PCG_B, PCG_DQ, PCG_A, PCG_RN, PCG_BETA, PCG_DONE, PCG_ITS, PCG_K, PCG_COPY,
               PCG_SLOTS = 16 };
void pcg_init(double* s, cudaStream_t st);                 // ||b|| = sqrt(rho), counters reset
// one whole PCG step after q = H d in five launches: <d, q>_V partials; alpha
// (or the curvature stop) folded into their sum; x, r updates with the
// <r, r>_V partials; beta (or the residual stop) folded into their sum; d
template <typename T>
void pcg_step(cplx<T>* x, cplx<T>* r, cplx<T>* d, const cplx<T>* q, const T* Lhat, long long kvol, int ncomp,
              double* partial, double* s, double tol, cudaStream_t st);

}  // namespace lddmm
