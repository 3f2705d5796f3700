// Host side, the deformation-state form (Section 3.3): the band-limited
// inverse-map sweep, its tangent, the terminal sampling and U~(1).
#include "impl.h"

namespace lddmm {
namespace host {

template <typename T>
void Impl<T>::jac_val(IotaDesc<T>& d, int base, const C* a, const C* b) {
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

template <typename T>
void Impl<T>::def_eval(int mode, const C* a, const C* b, const PiEpi<T>& e, T* fl,
                const T* cached) {
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

template <typename T>
void Impl<T>::deform_sweep(State<T>& S) {
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

template <typename T>
void Impl<T>::deform_sample(State<T>& S) {
  T* u1 = S.vgrid + 3 * Nvol;
  to_grid(vec(S.uh, Nt), 1, u1);
  def_sample<T>(I0, gI0, u1, m1(S), S.vgrid, N, st);
  ++launches;
  check_launch("deformation terminal sampling");
}

template <typename T>
auto Impl<T>::deform_tangent() -> C* {
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

template <typename T>
void Impl<T>::terminal_deform(const C* r, const C* u, C* out) {
  PiEpi<T> e = def_epi(true);
  add_out(e, out, 0, 1.0, {});
  def_eval(2, u, r, e);
}

// the members defined here, for both precisions
template void Impl<float>::jac_val(IotaDesc<float>& d, int base, const C* a, const C* b);
template void Impl<float>::def_eval(int mode, const C* a, const C* b, const PiEpi<float>& e, float* fl, const float* cached);
template void Impl<float>::deform_sweep(State<float>& S);
template void Impl<float>::deform_sample(State<float>& S);
template auto Impl<float>::deform_tangent() -> C*;
template void Impl<float>::terminal_deform(const C* r, const C* u, C* out);
template void Impl<double>::jac_val(IotaDesc<double>& d, int base, const C* a, const C* b);
template void Impl<double>::def_eval(int mode, const C* a, const C* b, const PiEpi<double>& e, double* fl, const double* cached);
template void Impl<double>::deform_sweep(State<double>& S);
template void Impl<double>::deform_sample(State<double>& S);
template auto Impl<double>::deform_tangent() -> C*;
template void Impl<double>::terminal_deform(const C* r, const C* u, C* out);

}  // namespace host
}  // namespace lddmm
