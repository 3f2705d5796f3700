// Host side, the inexact Gauss-Newton-Krylov solve (Eqs. 44-45): PCG with
// the scalars on the device, and the Armijo line search.
#include "impl.h"

namespace lddmm {
namespace host {

template <typename T>
void Impl<T>::gn_solve(void* v0, int n_gn, int n_pcg, lddmm_report* rep) {
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

// the members defined here, for both precisions
template void Impl<float>::gn_solve(void* v0, int n_gn, int n_pcg, lddmm_report* rep);
template void Impl<double>::gn_solve(void* v0, int n_gn, int n_pcg, lddmm_report* rep);

}  // namespace host
}  // namespace lddmm
