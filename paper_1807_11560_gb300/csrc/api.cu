// Host side of the GB300 LDDMM library: the C interface of include/lddmm.h.
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
#include <algorithm>
#include <atomic>
#include <cmath>
#include <initializer_list>
#include <utility>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/lddmm.h"
#include "internal.h"

struct lddmm_ctx {
  int precision;
  int device;      // the CUDA device current at lddmm_create; every call runs on it
  void* impl;
  std::string err;
};

namespace lddmm {
namespace {

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
  void release() {
    if (hv_exec) cudaGraphExecDestroy(hv_exec);
    hv_exec = nullptr;
    if (hv_exec_newton) cudaGraphExecDestroy(hv_exec_newton);
    hv_exec_newton = nullptr;
    if (cap) cudaStreamDestroy(cap);
    cap = nullptr;
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    evpool.clear();
    for (cudaEvent_t e : graph_events) cudaEventDestroy(e);
    graph_events.clear();
    for (void* q : allocs) cudaFree(q);
    allocs.clear();
    if (hres) cudaFreeHost(hres);
    hres = nullptr;
  }

  static C tw(long long p, int G, int sign, double w = 1.0) {
    const long long r = ((p % G) + G) % G;
    const double a = 2.0 * kPi * (double)r / (double)G;
    return C{(T)(w * std::cos(a)), (T)(w * sign * std::sin(a))};
  }
  static int sfreq(int q, int Kq) { return (2 * q < Kq) ? q : q - Kq; }

  void make_plan(Plan<T>& p, Dims g) {
    p.g = g;
    p.b = K;
    const int H1 = K.h1;
    std::vector<C> e3f((size_t)K.k3 * g.n3), e2f((size_t)K.k2 * g.n2), e1f((size_t)H1 * g.n1),
        e1b((size_t)g.n1 * H1), e2b((size_t)g.n2 * K.k2), e3b((size_t)g.n3 * K.k3);
    for (int k = 0; k < K.k3; ++k)
      for (int x = 0; x < g.n3; ++x) {
        e3f[(size_t)k * g.n3 + x] = tw((long long)sfreq(k, K.k3) * x, g.n3, +1);
        e3b[(size_t)x * K.k3 + k] = tw((long long)sfreq(k, K.k3) * x, g.n3, -1);
      }
    for (int k = 0; k < K.k2; ++k)
      for (int x = 0; x < g.n2; ++x) {
        e2f[(size_t)k * g.n2 + x] = tw((long long)sfreq(k, K.k2) * x, g.n2, +1);
        e2b[(size_t)x * K.k2 + k] = tw((long long)sfreq(k, K.k2) * x, g.n2, -1);
      }
    for (int h = 0; h < H1; ++h)
      for (int x = 0; x < g.n1; ++x) {
        e1f[(size_t)h * g.n1 + x] = tw((long long)h * x, g.n1, +1, h == 0 ? 1.0 : 2.0);
        e1b[(size_t)x * H1 + h] = tw((long long)h * x, g.n1, -1);
      }
    auto up = [&](C*& dst, std::vector<C>& src) {
      alloc(dst, src.size());
      cuda(cudaMemcpy(dst, src.data(), src.size() * sizeof(C), cudaMemcpyHostToDevice), "twiddles");
    };
    up(p.E3f, e3f);
    up(p.E2f, e2f);
    up(p.E1f, e1f);
    up(p.E1b, e1b);
    up(p.E2b, e2b);
    up(p.E3b, e3b);
    // the same tables in the padded / transposed tile layouts of the phases
    int G3e = 0, G2e = 0, G1q = 0, H1q = 0, G3s = 0;
    staged_twiddle_dims<T>(p, &G3e, &G2e, &G1q, &H1q, &G3s);
    const C zero{T(0), T(0)};
    std::vector<C> e3fp((size_t)K.k3 * G3e, zero), e2fp((size_t)K.k2 * G2e, zero),
        e1fp((size_t)H1 * G1q, zero), e1bp((size_t)g.n1 * H1q, zero), e3bt((size_t)K.k3 * G3s, zero);
    for (int k = 0; k < K.k3; ++k)
      for (int x = 0; x < g.n3; ++x) {
        e3fp[(size_t)k * G3e + x] = e3f[(size_t)k * g.n3 + x];
        e3bt[(size_t)k * G3s + x] = e3b[(size_t)x * K.k3 + k];
      }
    for (int k = 0; k < K.k2; ++k)
      for (int x = 0; x < g.n2; ++x) e2fp[(size_t)k * G2e + x] = e2f[(size_t)k * g.n2 + x];
    for (int h = 0; h < H1; ++h)
      for (int x = 0; x < g.n1; ++x) {
        e1fp[(size_t)h * G1q + x] = e1f[(size_t)h * g.n1 + x];
        e1bp[(size_t)x * H1q + h] = e1b[(size_t)x * H1 + h];
      }
    up(p.E3fp, e3fp);
    up(p.E2fp, e2fp);
    up(p.E1fp, e1fp);
    up(p.E1bp, e1bp);
    up(p.E3bt, e3bt);
  }

  void make_state(State<T>& S) {
    alloc(S.vh, (size_t)(Nt + 1) * 3 * Kvol);
    alloc(S.vsh, (size_t)Nt * 3 * Kvol);
    alloc(S.cache, (size_t)2 * Nt * cache_slot_elems<T>(pad));
    const size_t steps = opts.recompute ? 2 : (size_t)Nt + 1;
    alloc(S.vgrid, steps * 3 * Nvol);
    alloc(S.mh, steps * Nvol);
    alloc(S.off, (opts.recompute ? 1 : (size_t)Nt) * 3 * Nvol);
    if (deform()) {
      alloc(S.uh, (size_t)(Nt + 1) * 3 * Kvol);
      alloc(S.ush, (size_t)Nt * 3 * Kvol);
    }
  }
  // ------------------------------------------------------------ autotuner
  // Times the candidate tile shapes of the three padded-grid bracket kernels
  // on this context's sizes (CUDA events on the context stream, best of three
  // after a warm-up launch) and keeps the fastest of each.  Tile shapes change
  // no result: every sum keeps its order whatever the tiling.
  void autotune() {
    const size_t bbytes = (size_t)3 * Kvol * sizeof(C);
    cuda(cudaMemsetAsync(px, 0, bbytes, st), "memset");
    cuda(cudaMemsetAsync(pr, 0, bbytes, st), "memset");
    static const int kTp[] = {1, 2, 4, 8, 16};
    static const int kKc[] = {1, 2, 3, 4, 6, 8};
    long long slot_max = 0;
    for (int tp : kTp) {
      if (!tile_valid<T>(pad, 0, tp, 0)) continue;
      Plan<T> q = pad;
      q.tp = tp;
      slot_max = std::max(slot_max, cache_slot_elems<T>(q));
    }
    T* slot = nullptr;
    cuda(cudaMalloc(&slot, (size_t)std::max(1LL, slot_max) * sizeof(T)), "autotune scratch");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
      cuda(cudaMemsetAsync(slot, 0, (size_t)std::max(1LL, slot_max) * sizeof(T), st), "memset");
      cuda(cudaEventCreate(&e0), "event");
      cuda(cudaEventCreate(&e1), "event");
      auto best_of = [&](auto&& launch) {
        launch();
        check_launch("autotune");
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
          cuda(cudaEventRecord(e0, st), "event");
          launch();
          cuda(cudaEventRecord(e1, st), "event");
          cuda(cudaEventSynchronize(e1), "autotune");
          float ms = 0.f;
          cuda(cudaEventElapsedTime(&ms, e0, e1), "event");
          best = std::min(best, ms);
        }
        return best;
      };
      const IotaDesc<T> d = block24(px, pr, slot);
      float best = 1e30f;
      int pick = 0;
      for (int tws : {1, 2}) {
        if (!tile_valid<T>(pad, tws, 0, 0)) continue;
        pad.tws = tws;
        const float t = best_of([&] { bracket_iota<T>(pad, d, Lhat, T2, st); });
        if (t < best) { best = t; pick = tws; }
      }
      pad.tws = pick;
      if (pad.tc_cpw == nullptr) {   // the tensor-core middle phase fixes its own tile
        best = 1e30f;
        pick = 0;
        for (int tp : kTp) {
          if (!tile_valid<T>(pad, pad.tws, tp, 0)) continue;
          pad.tp = tp;
          const float t = best_of([&] { bracket_cpw<T>(pad, PW_GT, T2, slot, nullptr, P2, st); });
          if (t < best) { best = t; pick = tp; }
        }
        pad.tp = pick;
      }
      PiEpi<T> e = epi(3, 3);
      for (int o = 0; o < 3; ++o) {
        e.grp[o] = 0;
        e.coef[o] = (T)1;
      }
      add_out(e, vout, 0, 1.0, {});
      best = 1e30f;
      pick = 0;
      for (int kc : kKc) {
        if (!tile_valid<T>(pad, pad.tws, pad.tp, kc)) continue;
        pad.kc = kc;
        const float t = best_of([&] { bracket_pi<T>(pad, e, Lhat, P2, st); });
        if (t < best) { best = t; pick = kc; }
      }
      pad.kc = pick;
    } catch (...) {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      cudaFree(slot);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(slot);
  }

  // image-grid history accessors (step n of a kept or a two-step rolling history)
  long long hstep(int n) const { return opts.recompute ? (n & 1) : n; }
  T* mstate(State<T>& S, int n) { return S.mh + hstep(n) * Nvol; }
  T* m1(State<T>& S) { return mstate(S, Nt); }
  T* vgr(State<T>& S, int n) { return S.vgrid + hstep(n) * 3 * Nvol; }
  T* offp(State<T>& S, int n) { return S.off + (opts.recompute ? 0 : (long long)n) * 3 * Nvol; }
  T* dvg(int n) { return dvgrid + hstep(n) * 3 * Nvol; }

  void create(int nd, const int* grid, const int* band, double a, int s_, double sg, int nt,
              const lddmm_opts& o) {
    ndim = nd;
    duser = nd;
    N = Dims{grid[0], grid[1], nd == 3 ? grid[2] : 1};
    K.k1 = band[0];
    K.k2 = band[1];
    K.k3 = nd == 3 ? band[2] : 1;
    K.h1 = K.k1 / 2;
    auto padn = [](int k) { return k == 1 ? 1 : (3 * k + 1) / 2; };
    M = Dims{padn(K.k1), padn(K.k2), padn(K.k3)};
    Nt = nt;
    s = s_;
    alpha = a;
    sigma = sg;
    dt = 1.0 / nt;
    Nvol = N.vol();
    Mvol = M.vol();
    Kvol = K.vol();
    opts = o;
    st = (cudaStream_t)o.stream;
    cuda(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "stream");
    cuda(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");

    make_plan(full, N);
    make_plan(pad, M);
    full.split = split;
    if (max_smem_needed<T>(full, 1, false) > smem_limit() || max_smem_needed<T>(pad, 3, true) > smem_limit()) {
      *err = "grid or band too large for the transform tiles (N_3 <= 1024, shared memory)";
      throw Fail{LDDMM_EINVAL};
    }
    std::vector<T> L((size_t)Kvol);
    for (int q1 = 0; q1 < K.k1; ++q1)
      for (int q2 = 0; q2 < K.k2; ++q2)
        for (int q3 = 0; q3 < K.k3; ++q3) {
          const double f1 = sfreq(q1, K.k1), f2 = sfreq(q2, K.k2), f3 = sfreq(q3, K.k3);
          L[((size_t)q1 * K.k2 + q2) * K.k3 + q3] =
              (T)std::pow(1.0 + 4.0 * kPi * kPi * alpha * (f1 * f1 + f2 * f2 + f3 * f3), (double)s);
        }
    alloc(Lhat, (size_t)Kvol);
    cuda(cudaMemcpy(Lhat, L.data(), L.size() * sizeof(T), cudaMemcpyHostToDevice), "Lhat");

    alloc(I0, (size_t)Nvol);
    alloc(I1, (size_t)Nvol);
    const long long H1 = K.h1;
    const long long t2 = std::max(33LL * H1 * N.n2 * N.n3, 24LL * H1 * M.n2 * M.n3);
    alloc(T2, (size_t)t2);
    alloc(P2, (size_t)9 * H1 * M.n2 * M.n3);
    for (C** b : {&k1, &aU, &aW, &Ut, &Wt, &U, &W, &dstar, &vin, &vout, &gbuf, &px, &pr,
                  &vsol, &vtry})
      alloc(*b, (size_t)3 * Kvol);
    alloc(dvh, (size_t)(Nt + 1) * 3 * Kvol);
    alloc(srcs, (size_t)(Nt + 1) * 3 * Kvol);
    alloc(dvsh, (size_t)Nt * 3 * Kvol);
    alloc(Uh, (size_t)(Nt + 1) * 3 * Kvol);
    alloc(Wh, (size_t)(Nt + 1) * 3 * Kvol);
    alloc(Uth, (size_t)Nt * 3 * Kvol);
    alloc(Wth, (size_t)Nt * 3 * Kvol);
    alloc(bU, (size_t)3 * Kvol);
    alloc(bW, (size_t)3 * Kvol);
    alloc(zero3, (size_t)3 * Kvol);
    cuda(cudaMemset(zero3, 0, (size_t)3 * Kvol * sizeof(C)), "memset");
    alloc(dvgrid, (opts.recompute ? 2 : (size_t)Nt + 1) * 3 * Nvol);
    for (int i = 0; i < 2; ++i) {
      alloc(dm[i], (size_t)Nvol);
      alloc(sb[i], (size_t)Nvol);
    }
    alloc(fterm, (size_t)3 * Nvol);
    if (deform()) {
      alloc(gI0, (size_t)3 * Nvol);
      alloc(defM, (size_t)12 * Mvol);
      alloc(defcache, (size_t)2 * Nt * 12 * Mvol);
      alloc(prodM, (size_t)3 * Mvol);
      for (C** b : {&dk1, &rhob, &dua, &dub, &dup}) alloc(*b, (size_t)3 * Kvol);
    }
    alloc(partial, (size_t)kReduceBlocks);
    alloc(dres, 8);
    alloc(dpcg, PCG_SLOTS);
    cuda(cudaMemset(dres, 0, 8 * sizeof(double)), "memset");
    cuda(cudaMallocHost(&hres, 8 * sizeof(double)), "cudaMallocHost");
    if constexpr (std::is_same<T, float>::value) {
      // the tcgen05 iota A+B twiddle operands, expanded once (on request)
      if (opts.tensor_cores != 0 && iota_ab_tc_supported(pad)) {
        float* tw = nullptr;
        alloc(tw, iota_ab_tc_twiddle_floats(pad));
        cuda(iota_ab_tc_twiddles(pad, tw, st), "tensor-core twiddles");
        pad.tc_ab = tw;
      }
      // and those of the tcgen05 pi B'+A' of the same launches
      if (opts.tensor_cores != 0 && pi_ba_tc_supported(pad)) {
        float* tw = nullptr;
        alloc(tw, pi_ba_tc_twiddle_floats(pad));
        cuda(pi_ba_tc_twiddles(pad, tw, st), "tensor-core pi twiddles");
        pad.tc_pi = tw;
      }
      // and of the tcgen05 C / products / C' (its tile fixes the cache layout)
      if (use_tc_pad() && cpw_tc_supported(pad) && tile_valid<T>(pad, 0, cpw_tc_tile(), 0)) {
        float* tw = nullptr;
        alloc(tw, cpw_tc_twiddle_floats(pad));
        cuda(cpw_tc_twiddles(pad, tw, st), "tensor-core cpw twiddles");
        pad.tc_cpw = tw;
        pad.tp = cpw_tc_tile();
      }
    }
    if (opts.autotune && !persistent()) autotune();
    make_state(lin);                       // the cache layout follows the tile shapes
    make_state(trial);
    alloc(tcache, (size_t)2 * Nt * cache_slot_elems<T>(pad));
    alloc(bar, kSweepBarWords);
    record_sweeps();
    cuda(cudaDeviceSynchronize(), "create");
  }

  // descriptors of every persistent sweep, recorded by running the sweep
  // loops once without launching anything
  void record_sweeps() {
    std::vector<EvalDesc<T>> v;
    rec = &v;
    auto upload = [&](EvalDesc<T>*& dst) {
      alloc(dst, v.size());
      cuda(cudaMemcpy(dst, v.data(), v.size() * sizeof(EvalDesc<T>), cudaMemcpyHostToDevice), "descriptors");
      v.clear();
    };
    shoot(lin);
    upload(ev_shoot_lin);
    shoot(trial);
    upload(ev_shoot_trial);
    tangent(lin);
    upload(ev_tangent);
    backward(lin);
    upload(ev_backward);
    backward_sources(lin);
    upload(ev_exact);
    tangent(lin, true);
    upload(ev_tangent_c);
    backward_hist(lin);
    upload(ev_backward_hist);
    newton_backward(lin);
    upload(ev_newton);
    rec = nullptr;
    sweep_flops[PW_F] = 2.0 * Nt * (flops_iota_ab() + flops_cpw(PW_F) + flops_pi_ba(1));
    sweep_flops[PW_T] = 2.0 * Nt * (flops_iota_ab() + flops_cpw(PW_T) + flops_pi_ba(1));
    sweep_flops[PW_GT] = 2.0 * Nt * (flops_iota_ab() + flops_cpw(PW_GT) + flops_pi_ba(3));
  }

  // a persistent sweep whose barrier wait gave up left dres[7] = 1
  void check_flag(double f) {
    if (f != 0.0) {
      *err = "a bounded device wait (sweep barrier or tensor-core MMA) timed out";
      throw Fail{LDDMM_ETIMEOUT};
    }
  }

  // ------------------------------------------------------------ staging
  // user BL vector (duser comps) -> hermitian 3-comp device vector
  void load_bl(const void* user, C* dst) {
    cuda(cudaMemcpyAsync(vin, user, (size_t)duser * Kvol * sizeof(C), cudaMemcpyDefault, st),
         "copy BL input");
    if (duser < 3)
      cuda(cudaMemsetAsync(vin + (size_t)duser * Kvol, 0, (size_t)(3 - duser) * Kvol * sizeof(C), st),
           "memset");
    hermitianize<T>(vin, dst, 3, K, st);
    ++launches;
    check_launch("hermitianize");
  }
  void store_bl(const C* src, void* user) {
    cuda(cudaMemcpyAsync(user, src, (size_t)duser * Kvol * sizeof(C), cudaMemcpyDefault, st),
         "copy BL output");
  }
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
  void collect() {
    float ms = 0.f;
    for (size_t i = 0; i < pend_direct.size(); ++i) {
      cuda(cudaEventElapsedTime(&ms, pend_direct[i].first, pend_direct[i].second), "probe elapsed");
      probe_ms += ms;
      probe_work += pend_work[i];
      ++probe_n;
    }
    pend_direct.clear();
    pend_work.clear();
    evnext = 0;
    if (graph_pending) {
      for (size_t i = 0; i < graph_pairs.size(); ++i) {
        cuda(cudaEventElapsedTime(&ms, graph_pairs[i].first, graph_pairs[i].second), "probe elapsed");
        probe_ms += ms;
        probe_work += graph_work[i];
        ++probe_n;
      }
      graph_pending = false;
    }
  }

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

  void eval(PwMode mode, T* slot, const C* srcA, const C* srcB, const PiEpi<T>& e, T* slot2 = nullptr) {
    if (rec) {
      rec->push_back(EvalDesc<T>{srcA, srcB, slot, slot2, e});
      return;
    }
    pb(PR_IOTA_AB);
    bracket_iota<T>(pad, block24(srcA, srcB, slot), Lhat, T2, st, use_tc_pad() ? dres + 7 : nullptr);
    pe(PR_IOTA_AB, flops_iota_ab());
    pb(PR_CPW);
    bracket_cpw<T>(pad, mode, T2, slot, slot2, P2, st, use_tc_pad() ? dres + 7 : nullptr);
    pe(PR_CPW, flops_cpw(mode));
    pb(PR_PI_BA);
    bracket_pi<T>(pad, e, Lhat, P2, st, use_tc_pad() ? dres + 7 : nullptr);
    pe(PR_PI_BA, flops_pi_ba(e.nper));
    launches += kBracketLaunches;
    check_launch("bracket evaluation");
  }

  // one band-limited sweep as a single persistent cooperative kernel
  void run_sweep(PwMode mode, const EvalDesc<T>* ev, int nev = 0) {
    if (nev == 0) nev = 2 * Nt;
    pb(PR_SWEEP);
    cuda(sweep_launch<T>(pad, mode, ev, nev, Lhat, T2, P2, bar, dres + 7, st, opts.debug_stall),
         "persistent sweep");
    pe(PR_SWEEP, sweep_flops[mode] * nev / (2.0 * Nt));
    ++launches;
  }
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
  void to_grid(const C* hist, int count, T* grid) {
    for (int v0 = 0; v0 < count; v0 += 11) {
      const int nv = std::min(11, count - v0);
      IotaDesc<T> d{};
      d.nf = 3 * nv;
      for (int v = 0; v < nv; ++v)
        for (int c = 0; c < 3; ++c) {
          const int f = 3 * v + c;
          d.src[f] = hist + ((long long)(v0 + v) * 3 + c) * Kvol;
          d.dst[f] = grid + ((long long)(v0 + v) * 3 + c) * Nvol;
          d.deriv[f] = -1;
          d.applyL[f] = 0;
        }
      pb(PR_IOTA_FULL);
      iota_batch<T>(full, d, Lhat, T2, st, use_tc() ? dres + 7 : nullptr);
      pe(PR_IOTA_FULL, iota_flops(d.nf));
      launches += kIotaLaunches;
    }
    check_launch("iota to image grid");
  }

  // K~ pi (or pi alone) of a 3-component image-grid field -> band vector out
  void project_K(const T* f3, C* out, bool applyK = true) {
    PiSrc<T> ps{};
    ps.nf = 3;
    for (int c = 0; c < 3; ++c) ps.src[c] = f3 + c * Nvol;
    PiEpi<T> e = epi(3, 1);
    e.grp[0] = 0;
    e.coef[0] = (T)(1.0 / (double)Nvol);
    e.applyK[0] = applyK ? 1 : 0;
    add_out(e, out, 0, 1.0, {});
    pb(PR_PI_FULL);
    pi_batch<T>(full, ps, e, Lhat, T2, st);
    pe(PR_PI_FULL, iota_flops(3));
    launches += kPiLaunches;
    check_launch("projection");
  }

  // K~ sum_x f(x) e^{-2 pi i k.x} of a 3-component grid field: the V-representer
  // of the cotangent of iota (the adjoint of iota is N pi)
  void project_adjoint(const T* f3, C* out) {
    PiSrc<T> ps{};
    ps.nf = 3;
    for (int c = 0; c < 3; ++c) ps.src[c] = f3 + c * Nvol;
    PiEpi<T> e = epi(3, 1);
    e.grp[0] = 0;
    e.coef[0] = (T)1;
    e.applyK[0] = 1;
    add_out(e, out, 0, 1.0, {});
    pb(PR_PI_FULL);
    pi_batch<T>(full, ps, e, Lhat, T2, st);
    pe(PR_PI_FULL, iota_flops(3));
    launches += kPiLaunches;
    check_launch("projection");
  }

  // ------------------------------------------------------------- sweeps
  T* slot(State<T>& S, int k) { return S.cache + (long long)k * cache_slot_elems<T>(pad); }
  C* vec(C* base, int n) { return base + (long long)n * 3 * Kvol; }

  // Heun shoot of BL EPDiff (Eq. 51); S.vh[0] must hold v0
  void shoot(State<T>& S) {
    if (persistent()) {
      run_sweep(PW_F, &S == &lin ? ev_shoot_lin : ev_shoot_trial);
      return;
    }
    const double m = 1.0 / (double)Mvol;
    for (int n = 0; n < Nt; ++n) {
      C* vn = vec(S.vh, n);
      C* vs = vec(S.vsh, n);
      C* vn1 = vec(S.vh, n + 1);
      PiEpi<T> e1 = epi(3, 1);
      e1.grp[0] = 0;
      e1.coef[0] = (T)(-m);
      e1.applyK[0] = 1;
      add_out(e1, k1, 0, 1.0, {});
      add_out(e1, vs, 0, dt, {{vn, 1.0}});
      eval(PW_F, slot(S, 2 * n), vn, vn, e1);
      PiEpi<T> e2 = epi(3, 1);
      e2.grp[0] = 0;
      e2.coef[0] = (T)(-m);
      e2.applyK[0] = 1;
      add_out(e2, vn1, 0, 0.5 * dt, {{vn, 1.0}, {k1, 0.5 * dt}});
      eval(PW_F, slot(S, 2 * n + 1), vs, vs, e2);
    }
  }

  // one semi-Lagrangian state step m_n -> m_{n+1} (Eq. 52) from the kept or
  // regenerated velocity grids of steps n and n + 1
  void state_step(State<T>& S, int n) {
    pb(PR_TRANSPORT);
    transport_step<T>(mstate(S, n), vgr(S, n + 1), vgr(S, n), mstate(S, n + 1), offp(S, n), N, dt, st);
    pe(PR_TRANSPORT, 8.0 * (double)Nvol);
    ++launches;
  }

  // grid velocities and semi-Lagrangian transport of I0 (Eq. 52)
  void transport(State<T>& S) {
    cuda(cudaMemcpyAsync(mstate(S, 0), I0, (size_t)Nvol * sizeof(T), cudaMemcpyDeviceToDevice, st),
         "copy I0");
    if (!opts.recompute) {
      to_grid(S.vh, Nt + 1, S.vgrid);
      for (int n = 0; n < Nt; ++n) state_step(S, n);
    } else {
      to_grid(S.vh, 1, vgr(S, 0));
      for (int n = 0; n < Nt; ++n) {
        to_grid(vec(S.vh, n + 1), 1, vgr(S, n + 1));
        state_step(S, n);
      }
    }
    check_launch("transport");
  }

  void forward(State<T>& S) {
    shoot(S);
    if (deform()) {
      deform_sweep(S);
      deform_sample(S);
      return;
    }
    transport(S);
  }

  // ------------------------------------- deformation-state form (Section 3.3)
  // Jacobian (d_j a_i in block 3 i + j) of band vector a and values of b onto
  // the padded grid: iota fields base .. base + 11
  void jac_val(IotaDesc<T>& d, int base, const C* a, const C* b) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int f = base + 3 * i + j;
        d.src[f] = a + (long long)i * Kvol;
        d.deriv[f] = (signed char)j;
        d.applyL[f] = 0;
      }
    for (int c = 0; c < 3; ++c) {
      const int f = base + 9 + c;
      d.src[f] = b + (long long)c * Kvol;
      d.deriv[f] = -1;
      d.applyL[f] = 0;
    }
  }
  // algorithmic flops of iota (or pi) of nf scalar fields on grid g
  double grid_flops(const Dims& g, int nf) const {
    const double H1 = K.h1, K2 = K.k2, K3 = K.k3;
    return nf * (8.0 * H1 * (K2 * K3 * g.n3 + K2 * (double)g.n2 * g.n3) + 4.0 * H1 * (double)g.vol());
  }
  // one padded-grid product of the deformation form (def_products mode): iota
  // of the fields {D a, b} into fl (defM when null), the product (mode 1 with
  // the cached stage-point block {D u, v}) and pi with epilogue e
  void def_eval(int mode, const C* a, const C* b, const PiEpi<T>& e, T* fl = nullptr,
                const T* cached = nullptr) {
    if (!fl) fl = defM;
    IotaDesc<T> d{};
    d.nf = 12;
    jac_val(d, 0, a, b);
    for (int f = 0; f < d.nf; ++f) d.dst[f] = fl + (long long)f * Mvol;
    PiSrc<T> ps{};
    ps.nf = 3;
    for (int c = 0; c < 3; ++c) ps.src[c] = prodM + (long long)c * Mvol;
    pb(PR_DEFORM);
    if (use_tc_pad()) {
      // with the per-evaluation tensor-core kernels: iota A+B and pi B'+A' as in
      // the bracket evaluations, stages C and C' through the tcgen05 / SIMT
      // transform kernels on the padded plan
      bracket_iota<T>(pad, d, Lhat, T2, st, dres + 7);
      iota_c_stage<T>(pad, d, T2, st, dres + 7);
      def_products<T>(mode, fl, cached, prodM, Mvol, st);
      pi_c_stage<T>(pad, ps, T2, st);
      bracket_pi<T>(pad, e, Lhat, T2, st, dres + 7);
    } else {
      iota_batch<T>(pad, d, Lhat, T2, st, nullptr);
      def_products<T>(mode, fl, cached, prodM, Mvol, st);
      pi_batch<T>(pad, ps, e, Lhat, T2, st);
    }
    pe(PR_DEFORM, grid_flops(M, d.nf + 3) + (mode == 1 ? 36.0 : 18.0) * (double)Mvol);
    launches += kIotaLaunches + 1 + kPiLaunches;
    check_launch("deformation product");
  }
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
  void deform_sweep(State<T>& S) {
    const bool keep = &S == &lin;
    cuda(cudaMemsetAsync(S.uh, 0, (size_t)3 * Kvol * sizeof(C), st), "memset u0");
    for (int n = 0; n < Nt; ++n) {
      C* un = vec(S.uh, n);
      C* us = vec(S.ush, n);
      PiEpi<T> e1 = def_epi(false);
      add_out(e1, dk1, 0, 1.0, {});
      add_out(e1, us, 0, dt, {{un, 1.0}});
      def_eval(0, un, vec(S.vh, n), e1, keep ? def_slot(2 * n) : nullptr);
      PiEpi<T> e2 = def_epi(false);
      add_out(e2, vec(S.uh, n + 1), 0, 0.5 * dt, {{un, 1.0}, {dk1, 0.5 * dt}});
      def_eval(0, us, vec(S.vsh, n), e2, keep ? def_slot(2 * n + 1) : nullptr);
    }
  }

  // m(1) = I0(x + u(1)(x)) into m1(S) and (grad I0)(x + u(1)(x)) into the first
  // three fields of S.vgrid (u(1) on the grid goes to the next three)
  void deform_sample(State<T>& S) {
    T* u1 = S.vgrid + 3 * Nvol;
    to_grid(vec(S.uh, Nt), 1, u1);
    def_sample<T>(I0, gI0, u1, m1(S), S.vgrid, N, st);
    ++launches;
    check_launch("deformation terminal sampling");
  }

  // exact tangent of lin's deformation sweep along the shoot tangent (dvh,
  // dvsh), reading {D u, v} of each stage point from defcache; returns the
  // buffer holding delta u~(1)
  C* deform_tangent() {
    C* cur = dua;
    C* nxt = dub;
    cuda(cudaMemsetAsync(cur, 0, (size_t)3 * Kvol * sizeof(C), st), "memset du0");
    for (int n = 0; n < Nt; ++n) {
      PiEpi<T> e1 = def_epi(false);
      add_out(e1, dk1, 0, 1.0, {});
      add_out(e1, dup, 0, dt, {{cur, 1.0}});
      def_eval(1, cur, vec(dvh, n), e1, nullptr, def_slot(2 * n));
      PiEpi<T> e2 = def_epi(false);
      add_out(e2, nxt, 0, 0.5 * dt, {{cur, 1.0}, {dk1, 0.5 * dt}});
      def_eval(1, dup, vec(dvsh, n), e2, nullptr, def_slot(2 * n + 1));
      std::swap(cur, nxt);
    }
    return cur;
  }

  // U~(1) = K~ pi[r + (D u)^T r] on the padded grid, r = iota(r~), u = u~(1)
  void terminal_deform(const C* r, const C* u, C* out) {
    PiEpi<T> e = def_epi(true);
    add_out(e, out, 0, 1.0, {});
    def_eval(2, u, r, e);
  }

  // energy pieces into dres[0] (<v0,v0>_V) and dres[1] (sum (m1 - I1)^2)
  void energy_terms(State<T>& S) {
    inner_V<T>(S.vh, S.vh, Lhat, 3, Kvol, partial, dres, st);
    sum_sq_diff<T>(m1(S), I1, Nvol, partial, dres + 1, st);
    launches += 4;
    check_launch("energy reductions");
  }
  double read_energy() {
    cuda(cudaMemcpyAsync(hres, dres, 8 * sizeof(double), cudaMemcpyDeviceToHost, st), "read E");
    sync("energy");
    check_flag(hres[7]);
    return 0.5 * hres[0] + hres[1] / (sigma * sigma * (double)Nvol);
  }
  double dot_V(const C* a, const C* b) {
    inner_V<T>(a, b, Lhat, 3, Kvol, partial, dres + 2, st);
    launches += 2;
    cuda(cudaMemcpyAsync(hres + 2, dres + 2, 6 * sizeof(double), cudaMemcpyDeviceToHost, st), "read dot");
    sync("inner product");
    check_flag(hres[7]);
    return hres[2];
  }

  // backward reduced adjoint Jacobi sweep (Eqs. 53-54) from (U, W) = (U, 0);
  // leaves W(0) in W
  void backward(State<T>& S) {
    const double m = 1.0 / (double)Mvol;
    if (!rec) cuda(cudaMemsetAsync(W, 0, (size_t)3 * Kvol * sizeof(C), st), "memset W");
    if (persistent()) {
      run_sweep(PW_GT, ev_backward);
      return;
    }
    for (int n = Nt - 1; n >= 0; --n) {
      PiEpi<T> e1 = epi(3, 3);
      e1.grp[0] = 0; e1.coef[0] = (T)m;  e1.applyK[0] = 1;   // ad^dag_v U
      e1.grp[1] = 1; e1.coef[1] = (T)m;  e1.applyK[1] = 1;   // ad^dag_W v
      e1.grp[2] = 1; e1.coef[2] = (T)-m; e1.applyK[2] = 0;   // -ad_v W
      add_out(e1, aU, 0, 1.0, {});
      add_out(e1, aW, 1, 1.0, {{U, 1.0}});
      add_out(e1, Ut, 0, dt, {{U, 1.0}});
      add_out(e1, Wt, 1, dt, {{W, 1.0}, {U, dt}});
      eval(PW_GT, slot(S, 2 * n + 1), W, U, e1);
      PiEpi<T> e2 = epi(3, 3);
      e2.grp[0] = 0; e2.coef[0] = (T)m;  e2.applyK[0] = 1;
      e2.grp[1] = 1; e2.coef[1] = (T)m;  e2.applyK[1] = 1;
      e2.grp[2] = 1; e2.coef[2] = (T)-m; e2.applyK[2] = 0;
      add_out(e2, U, 0, 0.5 * dt, {{U, 1.0}, {aU, 0.5 * dt}});
      add_out(e2, W, 1, 0.5 * dt, {{W, 1.0}, {aW, 0.5 * dt}, {Ut, 0.5 * dt}});
      eval(PW_GT, slot(S, 2 * n), Wt, Ut, e2);
    }
  }

  // incremental EPDiff (Eq. 30) from dvh[0], exact tangent of the Heun shoot
  T* tslot(int k) { return tcache + (long long)k * cache_slot_elems<T>(pad); }

  // incremental BL EPDiff (Eq. 30) from dvh[0]; with cache, also stores the
  // padded-grid fields of dv_n and dv*_n (full-Newton products)
  void tangent(State<T>& S, bool cache = false) {
    if (persistent()) {
      run_sweep(PW_T, cache ? ev_tangent_c : ev_tangent);
      return;
    }
    const double m = 1.0 / (double)Mvol;
    for (int n = 0; n < Nt; ++n) {
      C* dn = vec(dvh, n);
      C* dn1 = vec(dvh, n + 1);
      C* dstar = vec(dvsh, n);
      PiEpi<T> e1 = epi(3, 1);
      e1.grp[0] = 0;
      e1.coef[0] = (T)(-m);
      e1.applyK[0] = 1;
      add_out(e1, k1, 0, 1.0, {});
      add_out(e1, dstar, 0, dt, {{dn, 1.0}});
      eval(PW_T, slot(S, 2 * n), dn, dn, e1, cache ? tslot(2 * n) : nullptr);
      PiEpi<T> e2 = epi(3, 1);
      e2.grp[0] = 0;
      e2.coef[0] = (T)(-m);
      e2.applyK[0] = 1;
      add_out(e2, dn1, 0, 0.5 * dt, {{dn, 1.0}, {k1, 0.5 * dt}});
      eval(PW_T, slot(S, 2 * n + 1), dstar, dstar, e2, cache ? tslot(2 * n + 1) : nullptr);
    }
  }

  // transpose of the Heun shoot tangent with a band source at every time level
  // (the exact discrete adjoint's band sweep): W_Nt = s_Nt, W_n = T_n^T W_{n+1}
  // + s_n with T_n^T the W part of the backward Jacobi sweep (U = 0); leaves
  // W_0 in W
  void backward_sources(State<T>& S) {
    const double m = 1.0 / (double)Mvol;
    if (!rec)
      cuda(cudaMemcpyAsync(W, srcs + (long long)Nt * 3 * Kvol, (size_t)3 * Kvol * sizeof(C),
                           cudaMemcpyDeviceToDevice, st), "copy source");
    if (persistent()) {
      run_sweep(PW_GT, ev_exact);
      return;
    }
    for (int n = Nt - 1; n >= 0; --n) {
      PiEpi<T> e1 = epi(3, 3);
      e1.grp[0] = 0; e1.coef[0] = (T)0;  e1.applyK[0] = 1;   // (U = 0)
      e1.grp[1] = 1; e1.coef[1] = (T)m;  e1.applyK[1] = 1;   // ad^dag_W v
      e1.grp[2] = 1; e1.coef[2] = (T)-m; e1.applyK[2] = 0;   // -ad_v W
      add_out(e1, aW, 1, 1.0, {});
      add_out(e1, Wt, 1, dt, {{W, 1.0}});
      eval(PW_GT, slot(S, 2 * n + 1), W, zero3, e1);
      PiEpi<T> e2 = epi(3, 3);
      e2.grp[0] = 0; e2.coef[0] = (T)0;  e2.applyK[0] = 1;
      e2.grp[1] = 1; e2.coef[1] = (T)m;  e2.applyK[1] = 1;
      e2.grp[2] = 1; e2.coef[2] = (T)-m; e2.applyK[2] = 0;
      add_out(e2, W, 1, 0.5 * dt, {{W, 1.0}, {aW, 0.5 * dt}, {srcs + (long long)n * 3 * Kvol, 1.0}});
      eval(PW_GT, slot(S, 2 * n), Wt, zero3, e2);
    }
  }

  // the gradient's backward sweep (Eqs. 53-54) with its time levels and stage
  // values kept: level n in (Uh[n], Wh[n]) (Uh[Nt] = U~(1) set by the caller),
  // stage of step n in (Uth[n], Wth[n]); W(0) = Wh[0]
  void backward_hist(State<T>& S) {
    const double m = 1.0 / (double)Mvol;
    if (!rec) cuda(cudaMemsetAsync(vec(Wh, Nt), 0, (size_t)3 * Kvol * sizeof(C), st), "memset W");
    if (persistent()) {
      run_sweep(PW_GT, ev_backward_hist);
      return;
    }
    for (int n = Nt - 1; n >= 0; --n) {
      C *U1 = vec(Uh, n + 1), *W1 = vec(Wh, n + 1), *Ut_ = vec(Uth, n), *Wt_ = vec(Wth, n);
      PiEpi<T> e1 = epi(3, 3);
      e1.grp[0] = 0; e1.coef[0] = (T)m;  e1.applyK[0] = 1;   // ad^dag_v U
      e1.grp[1] = 1; e1.coef[1] = (T)m;  e1.applyK[1] = 1;   // ad^dag_W v
      e1.grp[2] = 1; e1.coef[2] = (T)-m; e1.applyK[2] = 0;   // -ad_v W
      add_out(e1, aU, 0, 1.0, {});
      add_out(e1, aW, 1, 1.0, {{U1, 1.0}});
      add_out(e1, Ut_, 0, dt, {{U1, 1.0}});
      add_out(e1, Wt_, 1, dt, {{W1, 1.0}, {U1, dt}});
      eval(PW_GT, slot(S, 2 * n + 1), W1, U1, e1);
      PiEpi<T> e2 = epi(3, 3);
      e2.grp[0] = 0; e2.coef[0] = (T)m;  e2.applyK[0] = 1;
      e2.grp[1] = 1; e2.coef[1] = (T)m;  e2.applyK[1] = 1;
      e2.grp[2] = 1; e2.coef[2] = (T)-m; e2.applyK[2] = 0;
      add_out(e2, vec(Uh, n), 0, 0.5 * dt, {{U1, 1.0}, {aU, 0.5 * dt}});
      add_out(e2, vec(Wh, n), 1, 0.5 * dt, {{W1, 1.0}, {aW, 0.5 * dt}, {Ut_, 0.5 * dt}});
      eval(PW_GT, slot(S, 2 * n), Wt_, Ut_, e2);
    }
  }

  // full-Newton incremental adjoint sweep (Eqs. 56-57 without the Gauss-Newton
  // drop): the derivative of the gradient's Heun-transposed recursion along the
  // tangent trajectory.  Per step four evaluations of the ad~ / ad~^dagger
  // bracket: G^T at v on (dU, dW) (the Gauss-Newton terms) and the same bracket
  // with dv in place of v on the gradient sweep's (U, W) (the dropped terms:
  // ad~^dagger_dv U, ad~^dagger_W dv - ad~_dv W), at the predictor and at the
  // step's start.  Starts from (U, W) = (dU(1), 0); leaves dW(0) in W.
  void newton_backward(State<T>& S) {
    const double m = 1.0 / (double)Mvol;
    if (!rec) cuda(cudaMemsetAsync(W, 0, (size_t)3 * Kvol * sizeof(C), st), "memset W");
    if (persistent()) {
      run_sweep(PW_GT, ev_newton, 4 * Nt);
      return;
    }
    auto groups = [&](PiEpi<T>& e) {
      e.grp[0] = 0; e.coef[0] = (T)m;  e.applyK[0] = 1;   // ad^dag_v U
      e.grp[1] = 1; e.coef[1] = (T)m;  e.applyK[1] = 1;   // ad^dag_W v
      e.grp[2] = 1; e.coef[2] = (T)-m; e.applyK[2] = 0;   // -ad_v W
    };
    for (int n = Nt - 1; n >= 0; --n) {
      // predictor stage: a = G^T_{v*}(dz) + G'_{dv*}(z_{n+1})
      PiEpi<T> e1 = epi(3, 3);
      groups(e1);
      add_out(e1, aU, 0, 1.0, {});
      add_out(e1, aW, 1, 1.0, {{U, 1.0}});
      eval(PW_GT, slot(S, 2 * n + 1), W, U, e1);
      PiEpi<T> e2 = epi(3, 3);
      groups(e2);
      add_out(e2, aU, 0, 1.0, {{aU, 1.0}});
      add_out(e2, aW, 1, 1.0, {{aW, 1.0}});
      add_out(e2, Ut, 0, dt, {{U, 1.0}, {aU, dt}});
      add_out(e2, Wt, 1, dt, {{W, 1.0}, {aW, dt}});
      eval(PW_GT, tslot(2 * n + 1), vec(Wh, n + 1), vec(Uh, n + 1), e2);
      // step start: b = G^T_{v_n}(dz~) + G'_{dv_n}(z~); dz_n = dz + dt/2 (a + b)
      PiEpi<T> e3 = epi(3, 3);
      groups(e3);
      add_out(e3, bU, 0, 1.0, {});
      add_out(e3, bW, 1, 1.0, {{Ut, 1.0}});
      eval(PW_GT, slot(S, 2 * n), Wt, Ut, e3);
      PiEpi<T> e4 = epi(3, 3);
      groups(e4);
      add_out(e4, U, 0, 0.5 * dt, {{U, 1.0}, {aU, 0.5 * dt}, {bU, 0.5 * dt}});
      add_out(e4, W, 1, 0.5 * dt, {{W, 1.0}, {aW, 0.5 * dt}, {bW, 0.5 * dt}});
      eval(PW_GT, tslot(2 * n), vec(Wth, n), vec(Uth, n), e4);
    }
  }

  // V-gradient of the discretised energy itself (Section 2.5's route in
  // discrete form, Eqs. 12-14): the state transport reversed step by step on
  // the image grid, each time level's velocity sensitivity projected to the
  // band, then carried back to v0 by backward_sources.  Needs the kept
  // histories (every reversed step reads m_n, v_n, v_{n+1} and the displacement
  // in reverse time order).
  double exact_gradient_dev(const C* v0dev, C* gdev) {
    need_images();
    exact_forward(v0dev);
    energy_terms(lin);
    // dE/dm(1) of the data term sigma^-2 h^d sum (m(1) - I1)^2
    scaled_diff<T>(m1(lin), I1, 2.0 / (sigma * sigma * (double)Nvol), dm[0], Nvol, st);
    ++launches;
    exact_backward();
    axpby<T>(gdev, 1.0, lin.vh, 1.0, W, 3 * Kvol, st);
    ++launches;
    check_launch("exact gradient");
    const double E = read_energy();
    have_lin = true;
    have_dm1 = false;
    have_zhist = false;
    return E;
  }

  // forward sweep of lin at v0 with the histories the exact adjoint reads
  void exact_forward(const C* v0dev) {
    if (opts.recompute) {
      *err = "the exact discrete adjoint reads the histories in reverse: create the context with recompute = 0";
      throw Fail{LDDMM_EINVAL};
    }
    cuda(cudaMemcpyAsync(lin.vh, v0dev, (size_t)3 * Kvol * sizeof(C), cudaMemcpyDeviceToDevice, st),
         "copy v0");
    forward(lin);
  }

  // reverse-mode sweep of the discrete map v0 -> m(1) from the cotangent
  // lambda(1) = dL/dm(1) held in dm[0]: the transport reversed step by step,
  // each level's velocity sensitivity projected to the band, the Heun shoot
  // transposed; leaves the V-representer of dL/dv0 in W
  void exact_backward() {
    T* lam_next = dm[0];
    T* lam_cur = dm[1];
    T* Gn = dvgrid;                       // G[n+1]
    T* Gc = dvgrid + 3 * Nvol;            // G[n]
    const size_t gbytes = (size_t)3 * Nvol * sizeof(T);
    cuda(cudaMemsetAsync(Gn, 0, gbytes, st), "memset");
    cuda(cudaMemsetAsync(Gc, 0, gbytes, st), "memset");
    for (int n = Nt - 1; n >= 0; --n) {
      cuda(cudaMemsetAsync(lam_cur, 0, (size_t)Nvol * sizeof(T), st), "memset");
      adjoint_step<T>(lam_next, mstate(lin, n), vgr(lin, n), vgr(lin, n + 1), offp(lin, n), lam_cur, Gn, Gc,
                      N, dt, st);
      ++launches;
      project_adjoint(Gn, srcs + (long long)(n + 1) * 3 * Kvol);   // G[n+1] is complete
      std::swap(Gn, Gc);
      cuda(cudaMemsetAsync(Gc, 0, gbytes, st), "memset");
      std::swap(lam_next, lam_cur);
    }
    project_adjoint(Gn, srcs);
    backward_sources(lin);
    check_launch("exact adjoint sweep");
  }

  // enqueue one GN Hessian-vector product: input dvh[0], output vout
  void enqueue_hessvec(bool newton = false) {
    State<T>& S = lin;
    if (deform()) {                           // Section 3.3 under Gauss-Newton
      tangent(S);
      const C* du1 = deform_tangent();
      to_grid(du1, 1, dvgrid);
      def_force<T>(S.vgrid, m1(S), I1, dvgrid, dm[Nt & 1], -2.0 / (sigma * sigma), fterm, Nvol, st);
      ++launches;
      project_K(fterm, rhob, false);
      terminal_deform(rhob, vec(S.uh, Nt), U);
      backward(S);
      axpby<T>(vout, 1.0, dvh, 1.0, W, 3 * Kvol, st);
      ++launches;
      check_launch("hessvec");
      return;
    }
    tangent(S, newton);
    if (!opts.recompute) {
      to_grid(dvh, Nt + 1, dvgrid);
    } else {                                  // regenerate step 0 of the state history
      cuda(cudaMemcpyAsync(mstate(S, 0), I0, (size_t)Nvol * sizeof(T), cudaMemcpyDeviceToDevice, st),
           "copy I0");
      to_grid(S.vh, 1, vgr(S, 0));
      to_grid(dvh, 1, dvg(0));
    }
    grad_dot<T>(mstate(S, 0), dvg(0), sb[0], N, st);
    ++launches;
    for (int n = 0; n < Nt; ++n) {
      if (opts.recompute) {                   // step n + 1 of the state and velocity histories
        to_grid(vec(S.vh, n + 1), 1, vgr(S, n + 1));
        to_grid(vec(dvh, n + 1), 1, dvg(n + 1));
        state_step(S, n);
      }
      pb(PR_INC);
      inc_step<T>(n == 0 ? nullptr : dm[n & 1], sb[n & 1], mstate(S, n + 1), dvg(n + 1), offp(S, n),
                  dm[(n + 1) & 1], sb[(n + 1) & 1], N, dt, st);
      pe(PR_INC, 12.0 * (double)Nvol);
    }
    launches += Nt;
    if (newton)
      terminal_newton<T>(m1(S), I1, dm[Nt & 1], -2.0 / (sigma * sigma), fterm, N, st);
    else
      terminal_field<T>(m1(S), dm[Nt & 1], 0, -2.0 / (sigma * sigma), fterm, N, st);
    ++launches;
    project_K(fterm, U);
    if (newton)
      newton_backward(S);
    else
      backward(S);
    axpby<T>(vout, 1.0, dvh, 1.0, W, 3 * Kvol, st);
    ++launches;
    check_launch("hessvec");
  }

  // ------------------------------------------------------- public calls
  void need_images() {
    if (!have_images) {
      *err = "images not set (call lddmm_set_images first)";
      throw Fail{LDDMM_ESTATE};
    }
  }

  void set_images(const void* a, const void* b) {
    cuda(cudaMemcpyAsync(I0, a, (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy I0");
    cuda(cudaMemcpyAsync(I1, b, (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy I1");
    if (deform()) {
      central_grad<T>(I0, gI0, N, st);
      ++launches;
      check_launch("gradient of I0");
    }
    sync("set_images");
    have_images = true;
    have_lin = false;
    have_dm1 = false;
  }

  double energy_dev(const C* v0dev) {
    cuda(cudaMemcpyAsync(trial.vh, v0dev, (size_t)3 * Kvol * sizeof(C), cudaMemcpyDeviceToDevice, st),
         "copy v0");
    forward(trial);
    energy_terms(trial);
    return read_energy();
  }

  double energy(const void* v0) {
    need_images();
    load_bl(v0, vtry);
    return energy_dev(vtry);
  }

  // gradient at the device vector v0dev (hermitian, 3 comps); g -> gdev
  double gradient_dev(const C* v0dev, C* gdev) {
    need_images();
    cuda(cudaMemcpyAsync(lin.vh, v0dev, (size_t)3 * Kvol * sizeof(C), cudaMemcpyDeviceToDevice, st),
         "copy v0");
    forward(lin);
    energy_terms(lin);
    return gradient_tail(gdev);
  }

  // the rest of the gradient once lin holds the forward sweep of the point and
  // dres[0..1] its energy terms
  double gradient_tail(C* gdev) {
    if (deform()) {                           // U~(1) of Section 3.3
      def_force<T>(lin.vgrid, m1(lin), I1, nullptr, nullptr, -2.0 / (sigma * sigma), fterm, Nvol, st);
      ++launches;
      project_K(fterm, rhob, false);
      terminal_deform(rhob, vec(lin.uh, Nt), vec(Uh, Nt));
    } else {
      terminal_field<T>(m1(lin), I1, 1, -2.0 / (sigma * sigma), fterm, N, st);
      ++launches;
      project_K(fterm, vec(Uh, Nt));
    }
    backward_hist(lin);
    axpby<T>(gdev, 1.0, lin.vh, 1.0, Wh, 3 * Kvol, st);
    ++launches;
    have_zhist = true;
    check_launch("gradient");
    const double E = read_energy();
    have_lin = true;
    have_dm1 = false;
    if (!std::isfinite(E)) {
      *err = "energy is not finite";
      throw Fail{LDDMM_ENONFINITE};
    }
    return E;
  }

  double gradient(const void* v0, void* g) {
    load_bl(v0, vsol);
    const double E = gradient_dev(vsol, gbuf);
    store_bl(gbuf, g);
    sync("gradient output");
    return E;
  }

  double exact_gradient(const void* v0, void* g) {
    state_form_only("lddmm_exact_gradient");
    load_bl(v0, vsol);
    const double E = exact_gradient_dev(vsol, gbuf);
    store_bl(gbuf, g);
    sync("exact gradient output");
    return E;
  }

  void invalidate_graph() {
    if (hv_exec_newton) {
      cudaGraphExecDestroy(hv_exec_newton);
      hv_exec_newton = nullptr;
    }
    if (hv_exec) {
      cudaGraphExecDestroy(hv_exec);
      hv_exec = nullptr;
    }
    for (cudaEvent_t e : graph_events) cudaEventDestroy(e);
    graph_events.clear();
    graph_pairs.clear();
    graph_work.clear();
    graph_pending = false;
  }

  void set_probe(int cls) {
    sync("probe");
    if (cls != probe) invalidate_graph();
    probe = cls;
    probe_ms = 0.0;
    probe_work = 0.0;
    probe_n = 0;
  }

  // Hessian-vector product with input already in dvh[0]; result in vout
  void hessvec_dev(bool newton = false) {
    if (!have_lin) {
      *err = "no linearisation point (call lddmm_gradient first)";
      throw Fail{LDDMM_ESTATE};
    }
    if (newton && !have_zhist) {
      *err = "the full-Newton product needs the backward sweep of lddmm_gradient at this point";
      throw Fail{LDDMM_ESTATE};
    }
    cudaGraphExec_t& exec = newton ? hv_exec_newton : hv_exec;
    if (opts.use_graphs && !exec) {
      try {
        build_graph(newton);
      } catch (const Fail&) {
        // capture refused (e.g. a launch kind the graph cannot hold): run the
        // product with direct launches from now on
        cudaGetLastError();
        opts.use_graphs = 0;
        err->clear();
      }
    }
    if (opts.use_graphs) {
      cuda(cudaEventRecord(ev, st), "event record");
      cuda(cudaStreamWaitEvent(cap, ev, 0), "wait");
      cuda(cudaGraphLaunch(exec, cap), "graph launch");
      cuda(cudaEventRecord(ev, cap), "event record");
      cuda(cudaStreamWaitEvent(st, ev, 0), "wait");
      if (!graph_pairs.empty()) {
        // probing inside the graph: the next replay re-records the same
        // events, so read this replay's pairs now
        graph_pending = true;
        sync("probe graph replay");
      }
      launches += newton ? hv_nodes_newton : hv_nodes;
    } else {
      enqueue_hessvec(newton);
    }
    have_dm1 = true;
  }

  void build_graph(bool newton = false) {
    cudaStream_t user = st;
    st = cap;
    const long long before = launches;
    cudaGraph_t g = nullptr;
    cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    capturing = true;
    try {
      enqueue_hessvec(newton);
    } catch (...) {
      capturing = false;
      cudaStreamEndCapture(cap, &g);
      if (g) cudaGraphDestroy(g);
      st = user;
      throw;
    }
    capturing = false;
    st = user;
    cuda(cudaStreamEndCapture(cap, &g), "end capture");
    (newton ? hv_nodes_newton : hv_nodes) = launches - before;
    launches = before;
    cudaError_t e = cudaGraphInstantiate(newton ? &hv_exec_newton : &hv_exec, g, 0);
    cudaGraphDestroy(g);
    cuda(e, "graph instantiate");
  }

  void hessvec(const void* dv, void* out) {
    if (!have_lin) {
      *err = "no linearisation point (call lddmm_gradient first)";
      throw Fail{LDDMM_ESTATE};
    }
    load_bl(dv, dvh);
    hessvec_dev();
    store_bl(vout, out);
    cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
    sync("hessvec");
    check_flag(hres[7]);
  }

  void hessvec_newton(const void* dv, void* out) {
    state_form_only("lddmm_hessvec_newton");
    if (!have_lin) {
      *err = "no linearisation point (call lddmm_gradient first)";
      throw Fail{LDDMM_ESTATE};
    }
    load_bl(dv, dvh);
    hessvec_dev(true);
    store_bl(vout, out);
    cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
    sync("hessvec");
    check_flag(hres[7]);
  }

  void gn_solve(void* v0, int n_gn, int n_pcg, lddmm_report* rep) {
    need_images();
    load_bl(v0, vsol);
    lddmm_report r{};
    if (rep) {
      r.E_hist = rep->E_hist;
      r.eps_hist = rep->eps_hist;
      r.pcg_hist = rep->pcg_hist;
    }
    const double c = opts.armijo_c;
    const size_t bytes = (size_t)3 * Kvol * sizeof(C);
    // after PCG the linearisation is no longer needed in this iteration, so the
    // line search's trial sweeps run in lin: the accepted trial's forward sweep
    // and energy terms are then those of the next iterate, whose gradient
    // continues from them
    bool lin_at_vsol = false;
    double E_last = 0.0;
    for (int it = 0; it < n_gn; ++it) {
      const double E = lin_at_vsol ? gradient_tail(gbuf) : gradient_dev(vsol, gbuf);
      E_last = E;
      const double gn = std::sqrt(dot_V(gbuf, gbuf));
      if (it == 0) {
        r.E_initial = E;
        r.gnorm_initial = gn;
      }
      r.gnorm_final = gn;
      if (r.E_hist) r.E_hist[it] = E;
      // CG in the V inner product on H p = -g (Eq. 45).  The direction is kept
      // in the product's input slot dvh[0] (no sweep writes it) and q is read
      // from the product's output, so no vector is copied per iteration.
      const long long n3 = 3 * Kvol;
      cuda(cudaMemsetAsync(px, 0, bytes, st), "memset");
      axpby<T>(pr, -1.0, gbuf, 0.0, nullptr, n3, st);
      cuda(cudaMemcpyAsync(dvh, pr, bytes, cudaMemcpyDeviceToDevice, st), "copy");
      ++launches;
      // the scalars stay on the device; the host looks at the stop flag every
      // fourth iteration (iterations after a stop only repeat the product)
      inner_V<T>(pr, pr, Lhat, 3, Kvol, partial, dpcg + PCG_R, st);
      pcg_init(dpcg, st);
      launches += 3;
      for (int k = 1; k <= n_pcg; ++k) {
        hessvec_dev(opts.newton != 0);
        pcg_step<T>(px, pr, dvh, vout, Lhat, Kvol, 3, partial, dpcg, opts.pcg_tol, st);
        launches += 5;
        if (k % 4 == 0 && k < n_pcg) {
          cuda(cudaMemcpyAsync(hres, dpcg + PCG_DONE, sizeof(double), cudaMemcpyDeviceToHost, st), "read");
          sync("pcg");
          if (hres[0] != 0.0) break;
        }
      }
      cuda(cudaMemcpyAsync(hres, dpcg + PCG_ITS, sizeof(double), cudaMemcpyDeviceToHost, st), "read");
      sync("pcg");
      const int its = (int)hres[0];
      r.pcg_iters += its;
      if (r.pcg_hist) r.pcg_hist[it] = its;
      // Armijo backtracking along p (Eq. 44 with the step sign read as +)
      const double slope = dot_V(gbuf, px);
      double eps = 1.0;
      bool ok = false;
      have_lin = have_zhist = have_dm1 = false;
      lin_at_vsol = false;
      for (int h = 0; h <= opts.max_halvings; ++h) {
        axpby<T>(vtry, 1.0, vsol, eps, px, 3 * Kvol, st);
        ++launches;
        cuda(cudaMemcpyAsync(lin.vh, vtry, bytes, cudaMemcpyDeviceToDevice, st), "copy trial");
        forward(lin);
        energy_terms(lin);
        const double Et = read_energy();
        if (Et <= E + c * eps * slope) {
          ok = true;
          E_last = Et;
          break;
        }
        eps *= 0.5;
      }
      if (!ok) {
        r.ls_failed = 1;
        r.gn_iters = it;
        break;
      }
      if (r.eps_hist) r.eps_hist[it] = eps;
      cuda(cudaMemcpyAsync(vsol, vtry, bytes, cudaMemcpyDeviceToDevice, st), "copy");
      lin_at_vsol = true;
      r.gn_iters = it + 1;
    }
    // the energy of the returned iterate is already known unless no iteration ran
    r.E_final = n_gn > 0 ? E_last : energy_dev(vsol);
    store_bl(vsol, v0);
    sync("gn_solve");
    if (rep) *rep = r;
  }

  // component calls ---------------------------------------------------------
  void iota_call(const void* a, int ncomp, void* out) {
    for (int c0 = 0; c0 < ncomp; c0 += 3) {
      const int nc = std::min(3, ncomp - c0);
      cuda(cudaMemcpyAsync(vin, (const C*)a + (long long)c0 * Kvol, (size_t)nc * Kvol * sizeof(C),
                           cudaMemcpyDefault, st), "copy");
      hermitianize<T>(vin, px, nc, K, st);
      ++launches;
      IotaDesc<T> d{};
      d.nf = nc;
      for (int c = 0; c < nc; ++c) {
        d.src[c] = px + c * Kvol;
        d.dst[c] = fterm + c * Nvol;
        d.deriv[c] = -1;
        d.applyL[c] = 0;
      }
      iota_batch<T>(full, d, Lhat, T2, st, use_tc() ? dres + 7 : nullptr);
      launches += kIotaLaunches;
      check_launch("iota");
      cuda(cudaMemcpyAsync((T*)out + (long long)c0 * Nvol, fterm, (size_t)nc * Nvol * sizeof(T),
                           cudaMemcpyDefault, st), "copy");
    }
    cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
    sync("iota");
    check_flag(hres[7]);
  }

  void pi_call(const void* f, int ncomp, void* out) {
    for (int c0 = 0; c0 < ncomp; c0 += 3) {
      const int nc = std::min(3, ncomp - c0);
      cuda(cudaMemcpyAsync(fterm, (const T*)f + (long long)c0 * Nvol, (size_t)nc * Nvol * sizeof(T),
                           cudaMemcpyDefault, st), "copy");
      PiSrc<T> ps{};
      ps.nf = nc;
      for (int c = 0; c < nc; ++c) ps.src[c] = fterm + c * Nvol;
      PiEpi<T> e = epi(nc, 1);
      e.grp[0] = 0;
      e.coef[0] = (T)(1.0 / (double)Nvol);
      e.applyK[0] = 0;
      add_out(e, vout, 0, 1.0, {});
      pi_batch<T>(full, ps, e, Lhat, T2, st);
      launches += kPiLaunches;
      check_launch("pi");
      cuda(cudaMemcpyAsync((C*)out + (long long)c0 * Kvol, vout, (size_t)nc * Kvol * sizeof(C),
                           cudaMemcpyDefault, st), "copy");
    }
    sync("pi");
  }

  void ad_dagger_call(const void* v, const void* u, void* out) {
    load_bl(v, px);
    load_bl(u, pr);
    PiEpi<T> e = epi(3, 1);
    e.grp[0] = 0;
    e.coef[0] = (T)(1.0 / (double)Mvol);
    e.applyK[0] = 1;
    add_out(e, vout, 0, 1.0, {});
    eval(PW_F, slot(trial, 0), px, pr, e);   // P(v, L u): v-fields from px, L-fields from pr
    store_bl(vout, out);
    sync("ad_dagger");
  }

  void ad_call(const void* v, const void* w, void* out) {
    load_bl(v, px);
    load_bl(w, pr);
    T* vslot = slot(trial, 0);
    eval(PW_F, vslot, px, px, epi(3, 1));          // caches the fields of v; no output
    PiEpi<T> e = epi(3, 3);                          // keep only Q(v, w) = Dv w - Dw v
    e.grp[0] = 0; e.coef[0] = (T)0;
    e.grp[1] = 0; e.coef[1] = (T)0;
    e.grp[2] = 0; e.coef[2] = (T)(1.0 / (double)Mvol);
    add_out(e, vout, 0, 1.0, {});
    eval(PW_GT, vslot, pr, pr, e);
    store_bl(vout, out);
    sync("ad");
  }

  void shoot_call(const void* v0, void* v1) {
    load_bl(v0, trial.vh);
    shoot(trial);
    store_bl(vec(trial.vh, Nt), v1);
    cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
    sync("shoot");
    check_flag(hres[7]);
  }

  void transport_call(const void* v0, void* m1out) {
    need_images();
    load_bl(v0, trial.vh);
    forward(trial);
    cuda(cudaMemcpyAsync(m1out, m1(trial), (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy m1");
    cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
    sync("transport");
    check_flag(hres[7]);
  }

  // l2 gradient of a loss of m(1) with respect to v0 (adjoint Jacobi sweep)
  void transport_vjp(const void* v0, const void* gm1, void* out) {
    state_form_only("lddmm_transport_vjp");
    need_images();
    load_bl(v0, vsol);
    cuda(cudaMemcpyAsync(lin.vh, vsol, (size_t)3 * Kvol * sizeof(C), cudaMemcpyDeviceToDevice, st),
         "copy v0");
    forward(lin);
    cuda(cudaMemcpyAsync(dm[0], gm1, (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy grad m1");
    // lambda(1) = -N dL/dm(1): the L2_h adjoint of the grid values
    terminal_field<T>(m1(lin), dm[0], 0, -(double)Nvol, fterm, N, st);
    ++launches;
    project_K(fterm, U);
    backward(lin);
    scale_L<T>(gbuf, W, Lhat, 3, Kvol, st);
    ++launches;
    check_launch("transport vjp");
    store_bl(gbuf, out);
    cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
    sync("transport vjp");
    check_flag(hres[7]);
    have_lin = true;
    have_zhist = false;
    have_dm1 = false;
  }

  // the same vector-Jacobian product through the exact discrete adjoint of the
  // discretised map (the transposes of the semi-Lagrangian steps and of the Heun
  // shoot): the derivative of the discrete m(1) itself
  void transport_vjp_exact(const void* v0, const void* gm1, void* out) {
    state_form_only("lddmm_transport_vjp_exact");
    need_images();
    load_bl(v0, vsol);
    exact_forward(vsol);
    cuda(cudaMemcpyAsync(dm[0], gm1, (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy grad m1");
    exact_backward();
    scale_L<T>(gbuf, W, Lhat, 3, Kvol, st);
    ++launches;
    check_launch("exact transport vjp");
    store_bl(gbuf, out);
    cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
    sync("exact transport vjp");
    check_flag(hres[7]);
    have_lin = true;
    have_zhist = false;
    have_dm1 = false;
  }

  void last_dm1(void* out) {
    if (!have_dm1) {
      *err = "no Hessian-vector product computed at this linearisation point";
      throw Fail{LDDMM_ESTATE};
    }
    cuda(cudaMemcpyAsync(out, dm[Nt & 1], (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy dm1");
    sync("dm1");
  }
};

template <typename F>
int guarded(lddmm_ctx* ctx, F&& f) {
  if (!ctx) return LDDMM_EINVAL;
  try {
    f();
    return LDDMM_OK;
  } catch (const Fail& e) {
    return e.code;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return LDDMM_ENOMEM;
  } catch (...) {
    ctx->err = "unexpected exception";
    return LDDMM_ECUDA;
  }
}

// Makes the context's device current for the duration of one call (host
// threads start on device 0, and a caller may have switched devices since the
// context was created) and restores the caller's device afterwards.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename Fn>
int dispatch(lddmm_ctx* ctx, Fn&& fn) {
  if (!ctx) return LDDMM_EINVAL;
  DeviceScope scope(ctx->device);
  if (!scope.ok) {
    ctx->err = "cannot make the context's device current";
    return LDDMM_ECUDA;
  }
  if (ctx->precision == LDDMM_FP64)
    return guarded(ctx, [&] { fn(*static_cast<Impl<double>*>(ctx->impl)); });
  return guarded(ctx, [&] { fn(*static_cast<Impl<float>*>(ctx->impl)); });
}

bool bad_ptr(lddmm_ctx* ctx, const void* p, const char* name) {
  if (p) return false;
  ctx->err = std::string("null pointer: ") + name;
  return true;
}

}  // namespace
}  // namespace lddmm

using lddmm::Impl;
using lddmm::bad_ptr;

extern "C" {

void lddmm_default_opts(lddmm_opts* o) {
  if (!o) return;
  o->precision = LDDMM_FP32;
  o->stream = nullptr;
  o->pcg_tol = 1e-12;
  o->armijo_c = 1e-4;
  o->max_halvings = 10;
  o->use_graphs = 1;
  o->persistent = 1;
  o->tensor_cores = 1;
  o->recompute = 0;
  o->autotune = 1;
  o->newton = 0;
  o->state_eq = 0;
  o->debug_stall = 0;
}

int lddmm_create(lddmm_ctx** out, int ndim, const int* grid, const int* K, double alpha, int s,
                 double sigma, int Nt, const lddmm_opts* opts) {
  if (!out) return LDDMM_EINVAL;
  *out = nullptr;
  if ((ndim != 2 && ndim != 3) || !grid || !K || !(alpha > 0) || s < 1 || !(sigma > 0) || Nt < 1)
    return LDDMM_EINVAL;
  for (int j = 0; j < ndim; ++j) {
    if (grid[j] < 2 || K[j] < 2 || (K[j] & 1) || K[j] > grid[j] || grid[j] > (1 << 16) || K[j] > 512 || (j == 0 && K[j] > 64))
      return LDDMM_EINVAL;
  }
  long long nvox = 1;
  for (int j = 0; j < ndim; ++j) nvox *= grid[j];
  if (nvox >= (1LL << 31)) return LDDMM_EINVAL;
  lddmm_opts o;
  lddmm_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision < LDDMM_FP64 || o.precision > LDDMM_BF16X3) return LDDMM_EINVAL;
  // the split modes are FP32 contexts whose contractions take the tensor cores
  // wherever a tcgen05 kernel covers their sizes
  int split = 0;
  if (o.precision == LDDMM_3XTF32 || o.precision == LDDMM_BF16X3) {
    split = o.precision == LDDMM_BF16X3 ? 1 : 0;
    o.precision = LDDMM_FP32;
    o.tensor_cores = 2;
  }
  if (o.state_eq != 0 && o.state_eq != 1) return LDDMM_EINVAL;
  if (o.state_eq == 1 && o.newton != 0) return LDDMM_EINVAL;
  if (o.debug_stall < 0) return LDDMM_EINVAL;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return LDDMM_ECUDA;
  }
  lddmm_ctx* ctx = new (std::nothrow) lddmm_ctx();
  if (!ctx) return LDDMM_ENOMEM;
  ctx->precision = o.precision;
  ctx->device = device;
  ctx->impl = nullptr;
  int rc;
  if (o.precision == LDDMM_FP64) {
    auto* im = new (std::nothrow) Impl<double>();
    if (!im) { delete ctx; return LDDMM_ENOMEM; }
    im->err = &ctx->err;
    ctx->impl = im;
    rc = lddmm::guarded(ctx, [&] { im->create(ndim, grid, K, alpha, s, sigma, Nt, o); });
  } else {
    auto* im = new (std::nothrow) Impl<float>();
    if (!im) { delete ctx; return LDDMM_ENOMEM; }
    im->err = &ctx->err;
    im->split = split;
    ctx->impl = im;
    rc = lddmm::guarded(ctx, [&] { im->create(ndim, grid, K, alpha, s, sigma, Nt, o); });
  }
  if (rc != LDDMM_OK) {
    lddmm_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return LDDMM_OK;
}

int lddmm_set_images(lddmm_ctx* ctx, const void* I0, const void* I1) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, I0, "I0") || bad_ptr(ctx, I1, "I1")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.set_images(I0, I1); });
}

int lddmm_energy(lddmm_ctx* ctx, const void* v0, double* E) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0") || bad_ptr(ctx, E, "E_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { *E = im.energy(v0); });
}

int lddmm_gradient(lddmm_ctx* ctx, const void* v0, void* g, double* E) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0") || bad_ptr(ctx, g, "g_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) {
    const double e = im.gradient(v0, g);
    if (E) *E = e;
  });
}

int lddmm_hessvec_newton(lddmm_ctx* ctx, const void* dv, void* out) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, dv, "dv") || bad_ptr(ctx, out, "Hdv_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.hessvec_newton(dv, out); });
}

int lddmm_exact_gradient(lddmm_ctx* ctx, const void* v0, void* g, double* E) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0") || bad_ptr(ctx, g, "g_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) {
    const double e = im.exact_gradient(v0, g);
    if (E) *E = e;
  });
}

int lddmm_hessvec(lddmm_ctx* ctx, const void* dv, void* out) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, dv, "dv") || bad_ptr(ctx, out, "Hdv_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.hessvec(dv, out); });
}

int lddmm_gn_solve(lddmm_ctx* ctx, void* v0, int n_gn, int n_pcg, lddmm_report* rep) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0_inout")) return LDDMM_EINVAL;
  if (n_gn < 0 || n_pcg < 1) {
    ctx->err = "n_gn must be >= 0 and n_pcg >= 1";
    return LDDMM_EINVAL;
  }
  return lddmm::dispatch(ctx, [&](auto& im) { im.gn_solve(v0, n_gn, n_pcg, rep); });
}

int lddmm_batch_gn_solve(lddmm_ctx* const* ctxs, int n, void* const* v0s, int n_gn, int n_pcg,
                         lddmm_report* reps, int nthreads) {
  if (!ctxs || !v0s || n < 1 || n_gn < 0 || n_pcg < 1 || nthreads < 0) return LDDMM_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !ctxs[i]->impl) return LDDMM_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) {
        ctxs[i]->err = "a context appears twice in the batch";
        return LDDMM_EINVAL;
      }
    if (bad_ptr(ctxs[i], v0s[i], "v0_inout")) return LDDMM_EINVAL;
    // independent cooperative grids are not guaranteed to be co-resident, so
    // contexts whose sweeps would run as persistent kernels cannot share the GPU
    const bool pers = ctxs[i]->precision == LDDMM_FP64
                          ? static_cast<Impl<double>*>(ctxs[i]->impl)->persistent()
                          : static_cast<Impl<float>*>(ctxs[i]->impl)->persistent();
    if (pers) {
      ctxs[i]->err = "batched contexts need opts.persistent = 0 (or padded grids above 32^3)";
      return LDDMM_EINVAL;
    }
  }
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nw = std::min(n, nthreads > 0 ? nthreads : (int)hw);
  std::vector<int> status(n, LDDMM_OK);
  std::atomic<int> next{0};
  auto work = [&] {
    for (int i = next++; i < n; i = next++)
      status[i] = lddmm_gn_solve(ctxs[i], v0s[i], n_gn, n_pcg, reps ? reps + i : nullptr);
  };
  std::vector<std::thread> pool;
  try {
    for (int w = 1; w < nw; ++w) pool.emplace_back(work);
  } catch (...) {
    // fewer threads than asked: the calling thread still drains the queue
  }
  work();
  for (auto& t : pool) t.join();
  for (int i = 0; i < n; ++i)
    if (status[i] != LDDMM_OK) return status[i];
  return LDDMM_OK;
}

int lddmm_iota(lddmm_ctx* ctx, const void* a, int ncomp, void* f) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, a, "a") || bad_ptr(ctx, f, "f_out") || ncomp < 1) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.iota_call(a, ncomp, f); });
}

int lddmm_pi(lddmm_ctx* ctx, const void* f, int ncomp, void* a) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, f, "f") || bad_ptr(ctx, a, "a_out") || ncomp < 1) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.pi_call(f, ncomp, a); });
}

int lddmm_ad_dagger(lddmm_ctx* ctx, const void* v, const void* u, void* out) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v, "v") || bad_ptr(ctx, u, "u") || bad_ptr(ctx, out, "out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.ad_dagger_call(v, u, out); });
}

int lddmm_ad(lddmm_ctx* ctx, const void* v, const void* w, void* out) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v, "v") || bad_ptr(ctx, w, "w") || bad_ptr(ctx, out, "out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.ad_call(v, w, out); });
}

int lddmm_shoot(lddmm_ctx* ctx, const void* v0, void* v1) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0") || bad_ptr(ctx, v1, "v1_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.shoot_call(v0, v1); });
}

int lddmm_transport(lddmm_ctx* ctx, const void* v0, void* m1) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0") || bad_ptr(ctx, m1, "m1_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.transport_call(v0, m1); });
}

int lddmm_transport_vjp(lddmm_ctx* ctx, const void* v0, const void* grad_m1, void* grad_v0) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0") || bad_ptr(ctx, grad_m1, "grad_m1") || bad_ptr(ctx, grad_v0, "grad_v0_out"))
    return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.transport_vjp(v0, grad_m1, grad_v0); });
}

int lddmm_transport_vjp_exact(lddmm_ctx* ctx, const void* v0, const void* grad_m1, void* grad_v0) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, v0, "v0") || bad_ptr(ctx, grad_m1, "grad_m1") || bad_ptr(ctx, grad_v0, "grad_v0_out"))
    return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.transport_vjp_exact(v0, grad_m1, grad_v0); });
}

int lddmm_last_dm1(lddmm_ctx* ctx, void* out) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, out, "dm1_out")) return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) { im.last_dm1(out); });
}

int lddmm_probe(lddmm_ctx* ctx, const char* kernel_class) {
  if (!ctx) return LDDMM_EINVAL;
  int cls = -1;
  if (kernel_class && kernel_class[0]) {
    for (int i = 0; i < lddmm::PR_COUNT; ++i)
      if (std::strcmp(kernel_class, lddmm::kProbeNames[i]) == 0) cls = i;
    if (cls < 0) {
      ctx->err = std::string("unknown kernel class: ") + kernel_class;
      return LDDMM_EINVAL;
    }
  }
  return lddmm::dispatch(ctx, [&](auto& im) { im.set_probe(cls); });
}

int lddmm_probe_read(lddmm_ctx* ctx, double* total_ms, long long* launches, double* work) {
  if (!ctx) return LDDMM_EINVAL;
  if (bad_ptr(ctx, total_ms, "total_ms") || bad_ptr(ctx, launches, "launches") || bad_ptr(ctx, work, "work"))
    return LDDMM_EINVAL;
  return lddmm::dispatch(ctx, [&](auto& im) {
    im.sync("probe read");
    *total_ms = im.probe_ms;
    *launches = im.probe_n;
    *work = im.probe_work;
    im.probe_ms = 0.0;
    im.probe_work = 0.0;
    im.probe_n = 0;
  });
}

long long lddmm_kernel_count(const lddmm_ctx* ctx) {
  if (!ctx || !ctx->impl) return 0;
  if (ctx->precision == LDDMM_FP64) return static_cast<const Impl<double>*>(ctx->impl)->launches;
  return static_cast<const Impl<float>*>(ctx->impl)->launches;
}

int lddmm_tile_config(const lddmm_ctx* ctx, int* tws, int* tp, int* kc) {
  if (!ctx || !ctx->impl || !tws || !tp || !kc) return LDDMM_EINVAL;
  if (ctx->precision == LDDMM_FP64)
    lddmm::tile_config<double>(static_cast<const Impl<double>*>(ctx->impl)->pad, tws, tp, kc);
  else
    lddmm::tile_config<float>(static_cast<const Impl<float>*>(ctx->impl)->pad, tws, tp, kc);
  return LDDMM_OK;
}

unsigned long long lddmm_device_bytes(const lddmm_ctx* ctx) {
  if (!ctx || !ctx->impl) return 0;
  if (ctx->precision == LDDMM_FP64) return static_cast<const Impl<double>*>(ctx->impl)->device_bytes;
  return static_cast<const Impl<float>*>(ctx->impl)->device_bytes;
}

const char* lddmm_last_error(const lddmm_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

void lddmm_destroy(lddmm_ctx* ctx) {
  if (!ctx) return;
  lddmm::DeviceScope scope(ctx->device);
  if (ctx->impl) {
    if (ctx->precision == LDDMM_FP64) {
      auto* im = static_cast<Impl<double>*>(ctx->impl);
      im->release();
      delete im;
    } else {
      auto* im = static_cast<Impl<float>*>(ctx->impl);
      im->release();
      delete im;
    }
  }
  delete ctx;
}

}  // extern "C"
