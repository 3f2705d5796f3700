// Host side, the component calls of the C interface: iota, pi, the
// brackets, the shoot, the transport and its vector-Jacobian products.
#include "impl.h"

namespace lddmm {
namespace host {

template <typename T>
void Impl<T>::iota_call(const void* a, int ncomp, void* out) {
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

template <typename T>
void Impl<T>::pi_call(const void* f, int ncomp, void* out) {
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

template <typename T>
void Impl<T>::ad_dagger_call(const void* v, const void* u, void* out) {
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

template <typename T>
void Impl<T>::ad_call(const void* v, const void* w, void* out) {
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

template <typename T>
void Impl<T>::shoot_call(const void* v0, void* v1) {
  load_bl(v0, trial.vh);
  shoot(trial);
  store_bl(vec(trial.vh, Nt), v1);
  cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
  sync("shoot");
  check_flag(hres[7]);
}

template <typename T>
void Impl<T>::transport_call(const void* v0, void* m1out) {
  need_images();
  load_bl(v0, trial.vh);
  forward(trial);
  cuda(cudaMemcpyAsync(m1out, m1(trial), (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy m1");
  cuda(cudaMemcpyAsync(hres + 7, dres + 7, sizeof(double), cudaMemcpyDeviceToHost, st), "read flag");
  sync("transport");
  check_flag(hres[7]);
}

template <typename T>
void Impl<T>::transport_vjp(const void* v0, const void* gm1, void* out) {
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

template <typename T>
void Impl<T>::transport_vjp_exact(const void* v0, const void* gm1, void* out) {
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

template <typename T>
void Impl<T>::last_dm1(void* out) {
  if (!have_dm1) {
    *err = "no Hessian-vector product computed at this linearisation point";
    throw Fail{LDDMM_ESTATE};
  }
  cuda(cudaMemcpyAsync(out, dm[Nt & 1], (size_t)Nvol * sizeof(T), cudaMemcpyDefault, st), "copy dm1");
  sync("dm1");
}

// the members defined here, for both precisions
template void Impl<float>::iota_call(const void* a, int ncomp, void* out);
template void Impl<float>::pi_call(const void* f, int ncomp, void* out);
template void Impl<float>::ad_dagger_call(const void* v, const void* u, void* out);
template void Impl<float>::ad_call(const void* v, const void* w, void* out);
template void Impl<float>::shoot_call(const void* v0, void* v1);
template void Impl<float>::transport_call(const void* v0, void* m1out);
template void Impl<float>::transport_vjp(const void* v0, const void* gm1, void* out);
template void Impl<float>::transport_vjp_exact(const void* v0, const void* gm1, void* out);
template void Impl<float>::last_dm1(void* out);
template void Impl<double>::iota_call(const void* a, int ncomp, void* out);
template void Impl<double>::pi_call(const void* f, int ncomp, void* out);
template void Impl<double>::ad_dagger_call(const void* v, const void* u, void* out);
template void Impl<double>::ad_call(const void* v, const void* w, void* out);
template void Impl<double>::shoot_call(const void* v0, void* v1);
template void Impl<double>::transport_call(const void* v0, void* m1out);
template void Impl<double>::transport_vjp(const void* v0, const void* gm1, void* out);
template void Impl<double>::transport_vjp_exact(const void* v0, const void* gm1, void* out);
template void Impl<double>::last_dm1(void* out);

}  // namespace host
}  // namespace lddmm
