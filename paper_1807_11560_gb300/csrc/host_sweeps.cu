// Host side, time sweeps: one bracket evaluation (three kernels or a
// persistent sweep), the Heun shoot (Eq. 51), the state transport (Eq. 52),
// the tangent (Eq. 30) and the backward adjoint Jacobi sweeps (Eqs. 53-54),
// the full-Newton sweep (Eqs. 56-57) and the exact discrete adjoint.
#include "impl.h"

namespace lddmm {
namespace host {

template <typename T>
void Impl<T>::eval(PwMode mode, T* slot, const C* srcA, const C* srcB, const PiEpi<T>& e, T* slot2) {
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

template <typename T>
void Impl<T>::run_sweep(PwMode mode, const EvalDesc<T>* ev, int nev) {
  if (nev == 0) nev = 2 * Nt;
  pb(PR_SWEEP);
  cuda(sweep_launch<T>(pad, mode, ev, nev, Lhat, T2, P2, bar, dres + 7, st, opts.debug_stall),
       "persistent sweep");
  pe(PR_SWEEP, sweep_flops[mode] * nev / (2.0 * Nt));
  ++launches;
}

template <typename T>
void Impl<T>::to_grid(const C* hist, int count, T* grid) {
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

template <typename T>
void Impl<T>::project_K(const T* f3, C* out, bool applyK) {
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

template <typename T>
void Impl<T>::project_adjoint(const T* f3, C* out) {
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

template <typename T>
void Impl<T>::shoot(State<T>& S) {
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

template <typename T>
void Impl<T>::state_step(State<T>& S, int n) {
  pb(PR_TRANSPORT);
  transport_step<T>(mstate(S, n), vgr(S, n + 1), vgr(S, n), mstate(S, n + 1), offp(S, n), N, dt, st);
  pe(PR_TRANSPORT, 8.0 * (double)Nvol);
  ++launches;
}

template <typename T>
void Impl<T>::transport(State<T>& S) {
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

template <typename T>
void Impl<T>::forward(State<T>& S) {
  shoot(S);
  if (deform()) {
    deform_sweep(S);
    deform_sample(S);
    return;
  }
  transport(S);
}

template <typename T>
void Impl<T>::backward(State<T>& S) {
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

template <typename T>
void Impl<T>::tangent(State<T>& S, bool cache) {
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

template <typename T>
void Impl<T>::backward_sources(State<T>& S) {
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

template <typename T>
void Impl<T>::backward_hist(State<T>& S) {
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

template <typename T>
void Impl<T>::newton_backward(State<T>& S) {
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

template <typename T>
void Impl<T>::exact_forward(const C* v0dev) {
  if (opts.recompute) {
    *err = "the exact discrete adjoint reads the histories in reverse: create the context with recompute = 0";
    throw Fail{LDDMM_EINVAL};
  }
  cuda(cudaMemcpyAsync(lin.vh, v0dev, (size_t)3 * Kvol * sizeof(C), cudaMemcpyDeviceToDevice, st),
       "copy v0");
  forward(lin);
}

template <typename T>
void Impl<T>::exact_backward() {
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

// the members defined here, for both precisions
template void Impl<float>::eval(PwMode mode, float* slot, const C* srcA, const C* srcB, const PiEpi<float>& e, float* slot2);
template void Impl<float>::run_sweep(PwMode mode, const EvalDesc<float>* ev, int nev);
template void Impl<float>::to_grid(const C* hist, int count, float* grid);
template void Impl<float>::project_K(const float* f3, C* out, bool applyK);
template void Impl<float>::project_adjoint(const float* f3, C* out);
template void Impl<float>::shoot(State<float>& S);
template void Impl<float>::state_step(State<float>& S, int n);
template void Impl<float>::transport(State<float>& S);
template void Impl<float>::forward(State<float>& S);
template void Impl<float>::backward(State<float>& S);
template void Impl<float>::tangent(State<float>& S, bool cache);
template void Impl<float>::backward_sources(State<float>& S);
template void Impl<float>::backward_hist(State<float>& S);
template void Impl<float>::newton_backward(State<float>& S);
template void Impl<float>::exact_forward(const C* v0dev);
template void Impl<float>::exact_backward();
template void Impl<double>::eval(PwMode mode, double* slot, const C* srcA, const C* srcB, const PiEpi<double>& e, double* slot2);
template void Impl<double>::run_sweep(PwMode mode, const EvalDesc<double>* ev, int nev);
template void Impl<double>::to_grid(const C* hist, int count, double* grid);
template void Impl<double>::project_K(const double* f3, C* out, bool applyK);
template void Impl<double>::project_adjoint(const double* f3, C* out);
template void Impl<double>::shoot(State<double>& S);
template void Impl<double>::state_step(State<double>& S, int n);
template void Impl<double>::transport(State<double>& S);
template void Impl<double>::forward(State<double>& S);
template void Impl<double>::backward(State<double>& S);
template void Impl<double>::tangent(State<double>& S, bool cache);
template void Impl<double>::backward_sources(State<double>& S);
template void Impl<double>::backward_hist(State<double>& S);
template void Impl<double>::newton_backward(State<double>& S);
template void Impl<double>::exact_forward(const C* v0dev);
template void Impl<double>::exact_backward();

}  // namespace host
}  // namespace lddmm
