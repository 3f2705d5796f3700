// Host side, the objective: energy (Eq. 44), gradient (Eq. 50 / 55),
// the Gauss-Newton and full-Newton Hessian-vector products (Eqs. 56-58),
// the exact discrete-adjoint gradient, and the CUDA-graph capture and replay
// of the product.
#include "impl.h"

namespace lddmm {
namespace host {

template <typename T>
void Impl<T>::energy_terms(State<T>& S) {
  inner_V<T>(S.vh, S.vh, Lhat, 3, Kvol, partial, dres, st);
  sum_sq_diff<T>(m1(S), I1, Nvol, partial, dres + 1, st);
  launches += 4;
  check_launch("energy reductions");
}

template <typename T>
double Impl<T>::read_energy() {
  cuda(cudaMemcpyAsync(hres, dres, 8 * sizeof(double), cudaMemcpyDeviceToHost, st), "read E");
  sync("energy");
  check_flag(hres[7]);
  return 0.5 * hres[0] + hres[1] / (sigma * sigma * (double)Nvol);
}

template <typename T>
double Impl<T>::dot_V(const C* a, const C* b) {
  inner_V<T>(a, b, Lhat, 3, Kvol, partial, dres + 2, st);
  launches += 2;
  cuda(cudaMemcpyAsync(hres + 2, dres + 2, 6 * sizeof(double), cudaMemcpyDeviceToHost, st), "read dot");
  sync("inner product");
  check_flag(hres[7]);
  return hres[2];
}

template <typename T>
double Impl<T>::exact_gradient_dev(const C* v0dev, C* gdev) {
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

template <typename T>
void Impl<T>::enqueue_hessvec(bool newton) {
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

template <typename T>
void Impl<T>::set_images(const void* a, const void* b) {
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

template <typename T>
double Impl<T>::energy_dev(const C* v0dev) {
  cuda(cudaMemcpyAsync(trial.vh, v0dev, (size_t)3 * Kvol * sizeof(C), cudaMemcpyDeviceToDevice, st),
       "copy v0");
  forward(trial);
  energy_terms(trial);
  return read_energy();
}

template <typename T>
double Impl<T>::energy(const void* v0) {
  need_images();
  load_bl(v0, vtry);
  return energy_dev(vtry);
}

template <typename T>
double Impl<T>::gradient_dev(const C* v0dev, C* gdev) {
  need_images();
  cuda(cudaMemcpyAsync(lin.vh, v0dev, (size_t)3 * Kvol * sizeof(C), cudaMemcpyDeviceToDevice, st),
       "copy v0");
  forward(lin);
  energy_terms(lin);
  return gradient_tail(gdev);
}

template <typename T>
double Impl<T>::gradient_tail(C* gdev) {
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

template <typename T>
double Impl<T>::gradient(const void* v0, void* g) {
  load_bl(v0, vsol);
  const double E = gradient_dev(vsol, gbuf);
  store_bl(gbuf, g);
  sync("gradient output");
  return E;
}

template <typename T>
double Impl<T>::exact_gradient(const void* v0, void* g) {
  state_form_only("lddmm_exact_gradient");
  load_bl(v0, vsol);
  const double E = exact_gradient_dev(vsol, gbuf);
  store_bl(gbuf, g);
  sync("exact gradient output");
  return E;
}

template <typename T>
void Impl<T>::hessvec_dev(bool newton) {
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

template <typename T>
void Impl<T>::build_graph(bool newton) {
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

template <typename T>
void Impl<T>::hessvec(const void* dv, void* out) {
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

template <typename T>
void Impl<T>::hessvec_newton(const void* dv, void* out) {
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

// the members defined here, for both precisions
template void Impl<float>::energy_terms(State<float>& S);
template double Impl<float>::read_energy();
template double Impl<float>::dot_V(const C* a, const C* b);
template double Impl<float>::exact_gradient_dev(const C* v0dev, C* gdev);
template void Impl<float>::enqueue_hessvec(bool newton);
template void Impl<float>::set_images(const void* a, const void* b);
template double Impl<float>::energy_dev(const C* v0dev);
template double Impl<float>::energy(const void* v0);
template double Impl<float>::gradient_dev(const C* v0dev, C* gdev);
template double Impl<float>::gradient_tail(C* gdev);
template double Impl<float>::gradient(const void* v0, void* g);
template double Impl<float>::exact_gradient(const void* v0, void* g);
template void Impl<float>::hessvec_dev(bool newton);
template void Impl<float>::build_graph(bool newton);
template void Impl<float>::hessvec(const void* dv, void* out);
template void Impl<float>::hessvec_newton(const void* dv, void* out);
template void Impl<double>::energy_terms(State<double>& S);
template double Impl<double>::read_energy();
template double Impl<double>::dot_V(const C* a, const C* b);
template double Impl<double>::exact_gradient_dev(const C* v0dev, C* gdev);
template void Impl<double>::enqueue_hessvec(bool newton);
template void Impl<double>::set_images(const void* a, const void* b);
template double Impl<double>::energy_dev(const C* v0dev);
template double Impl<double>::energy(const void* v0);
template double Impl<double>::gradient_dev(const C* v0dev, C* gdev);
template double Impl<double>::gradient_tail(C* gdev);
template double Impl<double>::gradient(const void* v0, void* g);
template double Impl<double>::exact_gradient(const void* v0, void* g);
template void Impl<double>::hessvec_dev(bool newton);
template void Impl<double>::build_graph(bool newton);
template void Impl<double>::hessvec(const void* dv, void* out);
template void Impl<double>::hessvec_newton(const void* dv, void* out);

}  // namespace host
}  // namespace lddmm
