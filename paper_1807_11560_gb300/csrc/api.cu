// Host side of the GB300 LDDMM library: the C interface of include/lddmm.h
// (argument checks, the device of a context, status codes, batching).  The
// per-problem context it drives is lddmm::host::Impl (impl.h).
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "impl.h"

struct lddmm_ctx {
  int precision;
  int device;      // the CUDA device current at lddmm_create; every call runs on it
  void* impl;
  std::string err;
};

namespace lddmm {
namespace {

using namespace host;


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

using lddmm::host::Impl;
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
    for (int i = 0; i < lddmm::host::PR_COUNT; ++i)
      if (std::strcmp(kernel_class, lddmm::host::kProbeNames[i]) == 0) cls = i;
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
