// Host side, context resources: the per-problem allocations and plans
// (create / release), the twiddle tables, the tile autotuner, the
// recorded persistent-sweep descriptors, host<->device marshalling of band
// vectors and the kernel-class probe.
#include "impl.h"

namespace lddmm {
namespace host {

template <typename T>
void Impl<T>::release() {
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

template <typename T>
void Impl<T>::make_plan(Plan<T>& p, Dims g) {
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

template <typename T>
void Impl<T>::make_state(State<T>& S) {
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

template <typename T>
void Impl<T>::autotune() {
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

template <typename T>
void Impl<T>::create(int nd, const int* grid, const int* band, double a, int s_, double sg, int nt,
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

template <typename T>
void Impl<T>::record_sweeps() {
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

template <typename T>
void Impl<T>::load_bl(const void* user, C* dst) {
  cuda(cudaMemcpyAsync(vin, user, (size_t)duser * Kvol * sizeof(C), cudaMemcpyDefault, st),
       "copy BL input");
  if (duser < 3)
    cuda(cudaMemsetAsync(vin + (size_t)duser * Kvol, 0, (size_t)(3 - duser) * Kvol * sizeof(C), st),
         "memset");
  hermitianize<T>(vin, dst, 3, K, st);
  ++launches;
  check_launch("hermitianize");
}

template <typename T>
void Impl<T>::store_bl(const C* src, void* user) {
  cuda(cudaMemcpyAsync(user, src, (size_t)duser * Kvol * sizeof(C), cudaMemcpyDefault, st),
       "copy BL output");
}

template <typename T>
void Impl<T>::collect() {
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

template <typename T>
void Impl<T>::invalidate_graph() {
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

template <typename T>
void Impl<T>::set_probe(int cls) {
  sync("probe");
  if (cls != probe) invalidate_graph();
  probe = cls;
  probe_ms = 0.0;
  probe_work = 0.0;
  probe_n = 0;
}

// the members defined here, for both precisions
template void Impl<float>::release();
template void Impl<float>::make_plan(Plan<float>& p, Dims g);
template void Impl<float>::make_state(State<float>& S);
template void Impl<float>::autotune();
template void Impl<float>::create(int nd, const int* grid, const int* band, double a, int s_, double sg, int nt, const lddmm_opts& o);
template void Impl<float>::record_sweeps();
template void Impl<float>::load_bl(const void* user, C* dst);
template void Impl<float>::store_bl(const C* src, void* user);
template void Impl<float>::collect();
template void Impl<float>::invalidate_graph();
template void Impl<float>::set_probe(int cls);
template void Impl<double>::release();
template void Impl<double>::make_plan(Plan<double>& p, Dims g);
template void Impl<double>::make_state(State<double>& S);
template void Impl<double>::autotune();
template void Impl<double>::create(int nd, const int* grid, const int* band, double a, int s_, double sg, int nt, const lddmm_opts& o);
template void Impl<double>::record_sweeps();
template void Impl<double>::load_bl(const void* user, C* dst);
template void Impl<double>::store_bl(const C* src, void* user);
template void Impl<double>::collect();
template void Impl<double>::invalidate_graph();
template void Impl<double>::set_probe(int cls);

}  // namespace host
}  // namespace lddmm
