// Host side of the GB300 LDDMM library: the per-problem context behind the
// C interface of include/lddmm.h (internal; not part of the interface).
//
// A context owns, per problem, every device buffer of the method:
//   * twiddle tables of the image-grid plan (N) and of the padded product
//     plan (M = ceil(3K/2)), and the symbol table L^(k);
//   * two trajectories ("lin", the Gauss-Newton linearisation point, and
//     "trial", used by energy evaluations and component calls), each with the
//     BL history v_n, the Heun predictors v*_{n+1}, the 24 padded-grid fields
//     (v, Dv, L v, D(L v)) of every Heun stage point, the grid velocities
//     iota(v_n), the state history m_n and the characteristic displacements;
//   * the tangent history dv_n and its grid velocities, two ping-pong pairs
//     for dm and s = grad m . dv, the transform scratch and BL temporaries;
//   * with the deformation state equation (Section 3.3, opts.state_eq = 1):
//     per trajectory the band-limited inverse-map displacement u_n and its
//     predictors, the padded-grid fields {D u, v} of lin's stage points, and
//     grad I0 on the image grid.
// The time loops run on the host and enqueue kernels on one stream; the
// Hessian-vector product can be captured once per linearisation point into a
// CUDA graph and replayed.
//
// The members are defined by responsibility: host_context.cu (allocation,
// plans, autotuner, probe), host_sweeps.cu (bracket evaluations and the time
// sweeps), host_deform.cu (the deformation-state form), host_objective.cu
// (energy, gradient, Hessian-vector products, graph capture), host_solver.cu
// (GN-Krylov), host_components.cu (the component calls); api.cu holds the C
// interface.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <initializer_list>
#include <utility>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lddmm.h"
#include "internal.h"

namespace lddmm {
namespace host {

constexpr double kPi = 3.141592653589793238462643383279;

struct Fail {
  int code;
};

enum ProbeClass { PR_TRANSPORT = 0, PR_INC, PR_IOTA_AB, PR_CPW, PR_PI_BA, PR_IOTA_FULL, PR_PI_FULL,
                  PR_SWEEP, PR_DEFORM, PR_COUNT };
const char* const kProbeNames[PR_COUNT] = {"transport", "inc_step", "iota_ab", "cpw", "pi_ba",
                                           "iota_full", "pi_full", "sweep", "deform"};

template <typename T>
struct State {
  cplx<T>* vh = nullptr;    // [Nt+1][3][Kvol]
  cplx<T>* vsh = nullptr;   // [Nt][3][Kvol]
  T* cache = nullptr;       // [2 Nt][cache_slot_elems]: 24 padded-grid fields per stage point
  T* vgrid = nullptr;       // [Nt+1][3][Nvol]  (recompute: [2][3][Nvol], step n in n & 1)
  T* mh = nullptr;          // [Nt+1][Nvol]     (recompute: [2][Nvol])
  T* off = nullptr;         // [Nt][3][Nvol]    (recompute: [3][Nvol], the current step)
  // deformation-state form (Section 3.3): band-limited inverse-map displacement
  cplx<T>* uh = nullptr;    // [Nt+1][3][Kvol]
  cplx<T>* ush = nullptr;   // [Nt][3][Kvol]    Heun predictors u*_n
};

template <typename T>
struct Impl {
  using C = cplx<T>;
  std::string* err = nullptr;
  int ndim = 3, duser = 3;
  Dims N{}, M{};
  Band K{};
  int Nt = 1, s = 2;
  double alpha = 0, sigma = 1, dt = 1;
  long long Nvol = 0, Mvol = 0, Kvol = 0;
  lddmm_opts opts{};
  int split = 0;             // FP32 tensor-core split of the image-grid transform: 0 3xTF32, 1 BF16x3
  cudaStream_t st = nullptr;
  Plan<T> full{}, pad{};
  T* Lhat = nullptr;
  T *I0 = nullptr, *I1 = nullptr;
  State<T> lin, trial;
  bool have_images = false, have_lin = false, have_dm1 = false;
  C *T2 = nullptr, *P2 = nullptr;
  C *k1 = nullptr, *aU = nullptr, *aW = nullptr, *Ut = nullptr, *Wt = nullptr, *U = nullptr,
    *W = nullptr, *dstar = nullptr, *vin = nullptr, *vout = nullptr, *gbuf = nullptr;
  C *px = nullptr, *pr = nullptr, *vsol = nullptr, *vtry = nullptr;
  C* dvh = nullptr;          // [Nt+1][3][Kvol]
  C* srcs = nullptr;         // [Nt+1][3][Kvol] band sources of the exact discrete adjoint
  C* dvsh = nullptr;         // [Nt][3][Kvol] tangent predictor stages dv*_n
  C *Uh = nullptr, *Wh = nullptr;     // [Nt+1][3][Kvol] gradient sweep (U, W) per time level
  C *Uth = nullptr, *Wth = nullptr;   // [Nt][3][Kvol] gradient sweep stage values (U~, W~)
  C *bU = nullptr, *bW = nullptr;     // full-Newton sweep scratch
  T* tcache = nullptr;       // [2 Nt][cache_slot_elems] tangent stage-point fields (full Newton)
  C* zero3 = nullptr;        // [3][Kvol] zeros
  T* dvgrid = nullptr;       // [Nt+1][3][Nvol]  (recompute: [2][3][Nvol])
  T *dm[2] = {nullptr, nullptr}, *sb[2] = {nullptr, nullptr};
  T* fterm = nullptr;        // [3][Nvol]
  double *partial = nullptr, *dres = nullptr;   // dres[7]: sweep barrier time-out flag
  double* dpcg = nullptr;    // [PCG_SLOTS] device conjugate-gradient scalars
  double* hres = nullptr;    // pinned host mirror of dres
  // persistent sweeps: evaluation descriptors recorded once at creation
  std::vector<EvalDesc<T>>* rec = nullptr;
  EvalDesc<T> *ev_shoot_lin = nullptr, *ev_shoot_trial = nullptr, *ev_tangent = nullptr,
              *ev_backward = nullptr, *ev_exact = nullptr, *ev_tangent_c = nullptr,
              *ev_backward_hist = nullptr, *ev_newton = nullptr;
  unsigned* bar = nullptr;
  double sweep_flops[3] = {0, 0, 0};   // algorithmic flops of one sweep per mode
  long long launches = 0;
  std::vector<void*> allocs;
  unsigned long long device_bytes = 0;
  // graph of one Hessian-vector product (input dvh[0], output vout)
  cudaGraphExec_t hv_exec = nullptr, hv_exec_newton = nullptr;
  long long hv_nodes = 0, hv_nodes_newton = 0;
  bool have_zhist = false;   // Uh/Wh/Uth/Wth hold the last gradient's backward sweep
  // deformation-state form (Section 3.3)
  T* gI0 = nullptr;           // [3][Nvol] central-difference gradient of I0
  T* defM = nullptr;          // [12][Mvol] padded-grid fields of the deformation products
  T* defcache = nullptr;      // [2 Nt][12][Mvol] {D u, v} at the stage points of lin's sweep
  T* prodM = nullptr;         // [3][Mvol] their products
  C *dk1 = nullptr, *rhob = nullptr, *dua = nullptr, *dub = nullptr, *dup = nullptr;   // [3][Kvol]
  cudaStream_t cap = nullptr;
  cudaEvent_t ev = nullptr;
  bool capturing = false;
  // kernel-class probe: CUDA events around every launch of one class, read
  // back after each stream synchronisation (also inside the captured graph,
  // as external event-record nodes)
  int probe = -1;
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  cudaEvent_t pstart = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pend_direct, graph_pairs;
  std::vector<cudaEvent_t> graph_events;
  bool graph_pending = false;
  double probe_ms = 0.0, probe_work = 0.0;
  long long probe_n = 0;
  std::vector<double> pend_work, graph_work;

  // ---------------------------------------------------------------- utils
  void cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
      *err = std::string(what) + ": " + cudaGetErrorString(e);
      throw Fail{LDDMM_ECUDA};
    }
  }
  void check_launch(const char* what) { cuda(cudaGetLastError(), what); }
  template <typename P_>
  void alloc(P_*& p, size_t count) {
    void* q = nullptr;
    const size_t bytes = count * sizeof(P_);
    cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e);
      throw Fail{LDDMM_ENOMEM};
    }
    allocs.push_back(q);
    device_bytes += bytes > 0 ? bytes : 16;
    p = static_cast<P_*>(q);
  }
  void release();

  static C tw(long long p, int G, int sign, double w = 1.0) {
    const long long r = ((p % G) + G) % G;
    const double a = 2.0 * kPi * (double)r / (double)G;
    return C{(T)(w * std::cos(a)), (T)(w * sign * std::sin(a))};
  }
  static int sfreq(int q, int Kq) { return (2 * q < Kq) ? q : q - Kq; }

  void make_plan(Plan<T>& p, Dims g);

  void make_state(State<T>& S);
  // ------------------------------------------------------------ autotuner
  // Times the candidate tile shapes of the three padded-grid bracket kernels
  // on this context's sizes (CUDA events on the context stream, best of three
  // after a warm-up launch) and keeps the fastest of each.  Tile shapes change
  // no result: every sum keeps its order whatever the tiling.
  void autotune();

  // image-grid history accessors (step n of a kept or a two-step rolling history)
  long long hstep(int n) const { return opts.recompute ? (n & 1) : n; }
  T* mstate(State<T>& S, int n) { return S.mh + hstep(n) * Nvol; }
  T* m1(State<T>& S) { return mstate(S, Nt); }
  T* vgr(State<T>& S, int n) { return S.vgrid + hstep(n) * 3 * Nvol; }
  T* offp(State<T>& S, int n) { return S.off + (opts.recompute ? 0 : (long long)n) * 3 * Nvol; }
  T* dvg(int n) { return dvgrid + hstep(n) * 3 * Nvol; }

  void create(int nd, const int* grid, const int* band, double a, int s_, double sg, int nt,
              const lddmm_opts& o);

  // descriptors of every persistent sweep, recorded by running the sweep
  // loops once without launching anything
  void record_sweeps();

  // a persistent sweep whose barrier wait gave up left dres[7] = 1
  void check_flag(double f) {
    if (f != 0.0) {
      *err = "a bounded device wait (sweep barrier or tensor-core MMA) timed out";
      throw Fail{LDDMM_ETIMEOUT};
    }
  }

  // ------------------------------------------------------------ staging
  // user BL vector (duser comps) -> hermitian 3-comp device vector
  void load_bl(const void* user, C* dst);
  void store_bl(const C* src, void* user);
  void sync(const char* what) {
    cuda(cudaStreamSynchronize(st), what);
    collect();
  }

  // ------------------------------------------------------------- probe
  cudaEvent_t probe_event() {
    cudaEvent_t e = nullptr;
    if (capturing) {
      cuda(cudaEventCreate(&e), "probe event");
      graph_events.push_back(e);
      return e;
    }
    if (evnext == evpool.size()) {
      cuda(cudaEventCreate(&e), "probe event");
      evpool.push_back(e);
    }
    return evpool[evnext++];
  }
  void probe_record(cudaEvent_t e) {
    cuda(cudaEventRecordWithFlags(e, st, capturing ? cudaEventRecordExternal : cudaEventRecordDefault),
         "probe record");
  }
  void pb(int cls) {
    if (cls != probe) return;
    pstart = probe_event();
    probe_record(pstart);
  }
  // work: algorithmic flops (transforms, brackets) or bytes (transport steps)
  void pe(int cls, double work) {
    if (cls != probe) return;
    cudaEvent_t e = probe_event();
    probe_record(e);
    (capturing ? graph_pairs : pend_direct).push_back({pstart, e});
    (capturing ? graph_work : pend_work).push_back(work);
  }
  void collect();

  // -------------------------------------------------------- descriptors
  IotaDesc<T> block24(const C* srcA, const C* srcB, T* dst) const {
    IotaDesc<T> d{};
    d.nf = 24;
    for (int c = 0; c < 3; ++c) {
      d.src[c] = srcA + c * Kvol;
      d.deriv[c] = -1;
      d.applyL[c] = 0;
      d.src[12 + c] = srcB + c * Kvol;
      d.deriv[12 + c] = -1;
      d.applyL[12 + c] = 1;
      for (int j = 0; j < 3; ++j) {
        d.src[3 + 3 * c + j] = srcA + c * Kvol;
        d.deriv[3 + 3 * c + j] = (signed char)j;
        d.applyL[3 + 3 * c + j] = 0;
        d.src[15 + 3 * c + j] = srcB + c * Kvol;
        d.deriv[15 + 3 * c + j] = (signed char)j;
        d.applyL[15 + 3 * c + j] = 1;
      }
    }
    for (int f = 0; f < 24; ++f) d.dst[f] = dst + f * Mvol;
    return d;
  }
  static PiEpi<T> epi(int ncomp, int nper) {
    PiEpi<T> e;
    std::memset(&e, 0, sizeof(e));
    e.ncomp = ncomp;
    e.nper = nper;
    return e;
  }
  static void add_out(PiEpi<T>& e, C* dst, int r, double cR,
                      std::initializer_list<std::pair<const C*, double>> xs) {
    const int j = e.nout++;
    e.dst[j] = dst;
    e.r[j] = r;
    e.cR[j] = (T)cR;
    e.nx[j] = 0;
    for (auto& x : xs) {
      e.X[j][e.nx[j]] = x.first;
      e.cX[j][e.nx[j]] = (T)x.second;
      ++e.nx[j];
    }
  }

  // one evaluation of a bracket expression at a Heun stage point
  // algorithmic flops of the three phases of one bracket evaluation
  double flops_iota_ab() const {
    const double H1 = K.h1, K2 = K.k2, K3 = K.k3, M2 = M.n2, M3 = M.n3;
    return 8.0 * 24 * H1 * (K2 * K3 * M3 + K2 * M2 * M3);
  }
  double flops_cpw(PwMode mode) const {
    const int NP = (mode == PW_GT) ? 9 : 3;
    const double bflops = mode == PW_F ? 44.0 : (mode == PW_T ? 88.0 : 124.0);
    return 4.0 * (24 + NP) * K.h1 * (double)Mvol + bflops * (double)Mvol;
  }
  double flops_pi_ba(int nper) const {
    const double H1 = K.h1, K2 = K.k2, K3 = K.k3, M2 = M.n2, M3 = M.n3;
    return 8.0 * 3 * nper * H1 * (K2 * M2 * M3 + K2 * K3 * M3);
  }

  void eval(PwMode mode, T* slot, const C* srcA, const C* srcB, const PiEpi<T>& e, T* slot2 = nullptr);

  // one band-limited sweep as a single persistent cooperative kernel
  void run_sweep(PwMode mode, const EvalDesc<T>* ev, int nev = 0);
  // persistent sweeps pay off while the phases are latency-bound (small padded
  // grids); beyond that one launch's worst-phase footprint costs occupancy
  static constexpr long long kPersistentMaxPadded = 32768;   // M1 M2 M3
  // tensor-core image-grid transforms pay off once the grid write dominates
  static constexpr long long kTensorMinVoxels = 1LL << 20;
  bool use_tc() const {
    return opts.tensor_cores == 2 || (opts.tensor_cores == 1 && Nvol >= kTensorMinVoxels);
  }
  // tensor-core iota A+B of the bracket evaluations: the per-evaluation
  // launches of padded grids above the persistent-sweep size
  bool use_tc_pad() const {
    return !persistent() &&
           (opts.tensor_cores == 2 || (opts.tensor_cores == 1 && Mvol > kPersistentMaxPadded));
  }
  bool deform() const { return opts.state_eq == 1; }
  void state_form_only(const char* what) {
    if (!deform()) return;
    *err = std::string(what) + " is defined for the image state form only (opts.state_eq = 0)";
    throw Fail{LDDMM_EINVAL};
  }
  bool persistent() const {
    if (rec != nullptr || opts.persistent == 0) return false;
    return opts.persistent == 2 || Mvol <= kPersistentMaxPadded;
  }

  // algorithmic flops of iota (or pi) of nf scalar fields on the image grid,
  // Hermitian half spectrum along axis 1
  double iota_flops(int nf) const {
    const double H1 = K.h1, K2 = K.k2, K3 = K.k3;
    return nf * (8.0 * H1 * (K2 * K3 * N.n3 + K2 * (double)N.n2 * N.n3) + 4.0 * H1 * (double)Nvol);
  }

  // iota of `count` BL vectors (3 comps each) onto the image grid
  void to_grid(const C* hist, int count, T* grid);

  // K~ pi (or pi alone) of a 3-component image-grid field -> band vector out
  void project_K(const T* f3, C* out, bool applyK = true);

  // K~ sum_x f(x) e^{-2 pi i k.x} of a 3-component grid field: the V-representer
  // of the cotangent of iota (the adjoint of iota is N pi)
  void project_adjoint(const T* f3, C* out);

  // ------------------------------------------------------------- sweeps
  T* slot(State<T>& S, int k) { return S.cache + (long long)k * cache_slot_elems<T>(pad); }
  C* vec(C* base, int n) { return base + (long long)n * 3 * Kvol; }

  // Heun shoot of BL EPDiff (Eq. 51); S.vh[0] must hold v0
  void shoot(State<T>& S);

  // one semi-Lagrangian state step m_n -> m_{n+1} (Eq. 52) from the kept or
  // regenerated velocity grids of steps n and n + 1
  void state_step(State<T>& S, int n);

  // grid velocities and semi-Lagrangian transport of I0 (Eq. 52)
  void transport(State<T>& S);

  void forward(State<T>& S);

  // ------------------------------------- deformation-state form (Section 3.3)
  // Jacobian (d_j a_i in block 3 i + j) of band vector a and values of b onto
  // the padded grid: iota fields base .. base + 11
  void jac_val(IotaDesc<T>& d, int base, const C* a, const C* b);
  // algorithmic flops of iota (or pi) of nf scalar fields on grid g
  double grid_flops(const Dims& g, int nf) const {
    const double H1 = K.h1, K2 = K.k2, K3 = K.k3;
    return nf * (8.0 * H1 * (K2 * K3 * g.n3 + K2 * (double)g.n2 * g.n3) + 4.0 * H1 * (double)g.vol());
  }
  // one padded-grid product of the deformation form (def_products mode): iota
  // of the fields {D a, b} into fl (defM when null), the product (mode 1 with
  // the cached stage-point block {D u, v}) and pi with epilogue e
  void def_eval(int mode, const C* a, const C* b, const PiEpi<T>& e, T* fl = nullptr,
                const T* cached = nullptr);
  PiEpi<T> def_epi(bool applyK) const {
    PiEpi<T> e = epi(3, 1);
    e.grp[0] = 0;
    e.coef[0] = (T)(1.0 / (double)Mvol);
    e.applyK[0] = applyK ? 1 : 0;
    return e;
  }

  // padded-grid block {D u, v} of stage point k (2 n, 2 n + 1) of lin's sweep
  T* def_slot(int k) { return defcache + (long long)k * 12 * Mvol; }

  // Heun sweep of d/dt u~ = -v~ - D~u~ * v~ jointly with the shoot (stage 2 at
  // the EPDiff predictor v*_n), u~(0) = 0.  For lin the padded-grid fields of
  // each stage point stay in defcache for the tangent sweeps.
  void deform_sweep(State<T>& S);

  // m(1) = I0(x + u(1)(x)) into m1(S) and (grad I0)(x + u(1)(x)) into the first
  // three fields of S.vgrid (u(1) on the grid goes to the next three)
  void deform_sample(State<T>& S);

  // exact tangent of lin's deformation sweep along the shoot tangent (dvh,
  // dvsh), reading {D u, v} of each stage point from defcache; returns the
  // buffer holding delta u~(1)
  C* deform_tangent();

  // U~(1) = K~ pi[r + (D u)^T r] on the padded grid, r = iota(r~), u = u~(1)
  void terminal_deform(const C* r, const C* u, C* out);

  // energy pieces into dres[0] (<v0,v0>_V) and dres[1] (sum (m1 - I1)^2)
  void energy_terms(State<T>& S);
  double read_energy();
  double dot_V(const C* a, const C* b);

  // backward reduced adjoint Jacobi sweep (Eqs. 53-54) from (U, W) = (U, 0);
  // leaves W(0) in W
  void backward(State<T>& S);

  // incremental EPDiff (Eq. 30) from dvh[0], exact tangent of the Heun shoot
  T* tslot(int k) { return tcache + (long long)k * cache_slot_elems<T>(pad); }

  // incremental BL EPDiff (Eq. 30) from dvh[0]; with cache, also stores the
  // padded-grid fields of dv_n and dv*_n (full-Newton products)
  void tangent(State<T>& S, bool cache = false);

  // transpose of the Heun shoot tangent with a band source at every time level
  // (the exact discrete adjoint's band sweep): W_Nt = s_Nt, W_n = T_n^T W_{n+1}
  // + s_n with T_n^T the W part of the backward Jacobi sweep (U = 0); leaves
  // W_0 in W
  void backward_sources(State<T>& S);

  // the gradient's backward sweep (Eqs. 53-54) with its time levels and stage
  // values kept: level n in (Uh[n], Wh[n]) (Uh[Nt] = U~(1) set by the caller),
  // stage of step n in (Uth[n], Wth[n]); W(0) = Wh[0]
  void backward_hist(State<T>& S);

  // full-Newton incremental adjoint sweep (Eqs. 56-57 without the Gauss-Newton
  // drop): the derivative of the gradient's Heun-transposed recursion along the
  // tangent trajectory.  Per step four evaluations of the ad~ / ad~^dagger
  // bracket: G^T at v on (dU, dW) (the Gauss-Newton terms) and the same bracket
  // with dv in place of v on the gradient sweep's (U, W) (the dropped terms:
  // ad~^dagger_dv U, ad~^dagger_W dv - ad~_dv W), at the predictor and at the
  // step's start.  Starts from (U, W) = (dU(1), 0); leaves dW(0) in W.
  void newton_backward(State<T>& S);

  // V-gradient of the discretised energy itself (Section 2.5's route in
  // discrete form, Eqs. 12-14): the state transport reversed step by step on
  // the image grid, each time level's velocity sensitivity projected to the
  // band, then carried back to v0 by backward_sources.  Needs the kept
  // histories (every reversed step reads m_n, v_n, v_{n+1} and the displacement
  // in reverse time order).
  double exact_gradient_dev(const C* v0dev, C* gdev);

  // forward sweep of lin at v0 with the histories the exact adjoint reads
  void exact_forward(const C* v0dev);

  // reverse-mode sweep of the discrete map v0 -> m(1) from the cotangent
  // lambda(1) = dL/dm(1) held in dm[0]: the transport reversed step by step,
  // each level's velocity sensitivity projected to the band, the Heun shoot
  // transposed; leaves the V-representer of dL/dv0 in W
  void exact_backward();

  // enqueue one GN Hessian-vector product: input dvh[0], output vout
  void enqueue_hessvec(bool newton = false);

  // ------------------------------------------------------- public calls
  void need_images() {
    if (!have_images) {
      *err = "images not set (call lddmm_set_images first)";
      throw Fail{LDDMM_ESTATE};
    }
  }

  void set_images(const void* a, const void* b);

  double energy_dev(const C* v0dev);

  double energy(const void* v0);

  // gradient at the device vector v0dev (hermitian, 3 comps); g -> gdev
  double gradient_dev(const C* v0dev, C* gdev);

  // the rest of the gradient once lin holds the forward sweep of the point and
  // dres[0..1] its energy terms
  double gradient_tail(C* gdev);

  double gradient(const void* v0, void* g);

  double exact_gradient(const void* v0, void* g);

  void invalidate_graph();

  void set_probe(int cls);

  // Hessian-vector product with input already in dvh[0]; result in vout
  void hessvec_dev(bool newton = false);

  void build_graph(bool newton = false);

  void hessvec(const void* dv, void* out);

  void hessvec_newton(const void* dv, void* out);

  void gn_solve(void* v0, int n_gn, int n_pcg, lddmm_report* rep);

  // component calls ---------------------------------------------------------
  void iota_call(const void* a, int ncomp, void* out);

  void pi_call(const void* f, int ncomp, void* out);

  void ad_dagger_call(const void* v, const void* u, void* out);

  void ad_call(const void* v, const void* w, void* out);

  void shoot_call(const void* v0, void* v1);

  void transport_call(const void* v0, void* m1out);

  // l2 gradient of a loss of m(1) with respect to v0 (adjoint Jacobi sweep)
  void transport_vjp(const void* v0, const void* gm1, void* out);

  // the same vector-Jacobian product through the exact discrete adjoint of the
  // discretised map (the transposes of the semi-Lagrangian steps and of the Heun
  // shoot): the derivative of the discrete m(1) itself
  void transport_vjp_exact(const void* v0, const void* gm1, void* out);

  void last_dm1(void* out);
};

}  // namespace host
}  // namespace lddmm
