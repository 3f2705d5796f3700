// Persistent kernel for one whole band-limited time sweep (the Heun shoot of
// Eq. 51, its tangent of Eq. 30, or the backward adjoint Jacobi sweep of
// Eqs. 53-54): every bracket evaluation of the sweep runs in one cooperative
// launch, its three phases (bracket.cuh) separated by grid-wide barriers.
// At small grids the phases last a few microseconds each, so removing the
// kernel boundaries between them is what bounds the sweep time.
//
// Between the pi phase of one evaluation and the iota phase of the next there
// is no grid barrier: the iota item of (field f, h) reads only the band slab
// (component of f, h), so it waits for the completion counter of that slab
// (bumped by each pi item of the slab) instead of for the whole grid.  The
// other two phase boundaries are all-to-all (transposes) and keep barriers.
//
// Waits are bounded: a CTA that spins longer than the limit records the
// failure in a flag the host reads (LDDMM_ETIMEOUT) and every CTA leaves at
// its next barrier or wait.  The launch is cooperative, so all CTAs are
// resident, and no CTA waits on an item that comes after its own wait.
#include "bracket.cuh"

namespace lddmm {
namespace {

using dev::kThreads;
using dev::kMaxSmem;

constexpr long long kSpinLimit = 1LL << 24;   // polls of an L2 line: well over a second

template <typename T>
struct SweepArgs {
  Plan<T> p;                  // padded product-grid plan
  const T* Lhat;
  cplx<T>* T2;
  cplx<T>* P2;
  const EvalDesc<T>* ev;      // device array of nev evaluations
  int nev;
  int TP;                     // pencil tile of the C/products/C' phase
  dev::BAGeom ba;             // geometry of the pi B'/A' phase
  unsigned* bar;              // [0] arrival counter, [1 + c H1 + h] slab completion counters
  double* flag;               // set to 1 when a barrier wait gives up
  long long spin_limit;       // polls before a wait gives up
  unsigned stall;             // test hook: arrivals the first barrier waits for beyond the grid
};

__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier on a monotonic arrival counter (zeroed before the launch):
// the k-th barrier of the launch completes when the counter reaches
// k * gridDim.x.  One atomic per CTA, then acquire loads until the target.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned& target, double* flag,
                                             long long limit, unsigned extra = 0) {
  __syncthreads();
  target += gridDim.x + extra;
  int ok = 1;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    long long it = 0;
    while (load_acquire(count) < target) {
      if (++it > limit) {
        *(volatile double*)flag = 1.0;
        break;
      }
    }
    if (*(volatile double*)flag != 0.0) ok = 0;
  }
  return __syncthreads_and(ok) != 0;
}

// publish the completion of one pi item: its writes, then the counter
__device__ __forceinline__ void signal_slab(unsigned* cnt) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt, 1u);
  }
}

// wait until a slab completion counter reaches target (acquire), bounded
__device__ __forceinline__ bool wait_slab(const unsigned* cnt, unsigned target, double* flag, long long limit) {
  int ok = 1;
  if (threadIdx.x == 0) {
    long long it = 0;
    while (load_acquire(cnt) < target) {
      if (++it > limit) {
        *(volatile double*)flag = 1.0;
        break;
      }
    }
    if (*(volatile double*)flag != 0.0) ok = 0;
  }
  return __syncthreads_and(ok) != 0;
}

template <typename T, int MODE, bool TWS>
__global__ void __launch_bounds__(kThreads)
k_sweep(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // evaluation descriptors in shared memory (the epilogue indexes their
  // pointer and coefficient tables many times); the next one is fetched with
  // cp.async while the current evaluation runs
  __shared__ __align__(16) EvalDesc<T> sev[2];
  static_assert(sizeof(EvalDesc<T>) % sizeof(unsigned long long) == 0, "descriptor size");
  constexpr int kDescWords = (int)(sizeof(EvalDesc<T>) / sizeof(unsigned long long));
  const Plan<T>& p = a.p;
  const int H1 = p.b.h1;
  const long long P = (long long)p.g.n2 * p.g.n3;
  const long long kvol = p.b.vol();
  const int n_ab = 24 * H1;
  const int n_cpw = (int)((P + a.TP - 1) / a.TP);
  const int n_ba = 3 * H1 * a.ba.nch;
  unsigned target = 0;
  for (int ev = 0; ev < a.nev; ++ev) {
    if (ev == 0) {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(a.ev);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sev[0]);
      for (int i = threadIdx.x; i < kDescWords; i += kThreads) dst[i] = src[i];
    }
    dev::cp_async_wait_all();                      // descriptor ev has landed
    __syncthreads();
    if (ev + 1 < a.nev) {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(a.ev + ev + 1);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sev[(ev + 1) & 1]);
      for (int i = threadIdx.x; i < kDescWords; i += kThreads) dev::cp_async(dst + i, src + i);
    }
    const EvalDesc<T>* E = &sev[ev & 1];
    const cplx<T>* A = E->srcA;
    const cplx<T>* B = E->srcB;
    T* slot = E->slot;
    for (int vb = blockIdx.x; vb < n_ab; vb += gridDim.x) {
      const int f = vb / H1, h = vb % H1;
      const dev::FieldSpec<T> fs = dev::field24<T>(A, B, kvol, f);
      if (ev > 0 &&
          !wait_slab(a.bar + 1 + dev::field24_comp(f) * H1 + h, (unsigned)(a.ba.nch * ev), a.flag, a.spin_limit))
        return;
      dev::phase_iota_ab<T, TWS>(p, fs, f, h, a.Lhat, a.T2, smraw);
      __syncthreads();
    }
    // (the test hook makes the very first barrier wait for arrivals that never come)
    if (!grid_barrier(a.bar, target, a.flag, a.spin_limit, ev == 0 ? a.stall : 0u)) return;
    for (int vb = blockIdx.x; vb < n_cpw; vb += gridDim.x) {
      dev::phase_cpw<T, MODE>(p, a.T2, slot, E->slot2, a.P2, a.TP, vb, smraw);
      __syncthreads();
    }
    if (!grid_barrier(a.bar, target, a.flag, a.spin_limit)) return;
    for (int vb = blockIdx.x; vb < n_ba; vb += gridDim.x) {
      dev::phase_pi_ba<T>(p, E->epi, a.Lhat, a.P2, a.ba, vb, smraw);
      const int h = (vb / a.ba.nch) % H1, c = vb / (a.ba.nch * H1);
      signal_slab(a.bar + 1 + c * H1 + h);
    }
    __syncthreads();
  }
}

template <typename T, int MODE, bool TWS>
cudaError_t launch(const SweepArgs<T>& a, size_t smem, cudaStream_t st, int max_ctas) {
  auto kern = k_sweep<T, MODE, TWS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev_id = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem)) != cudaSuccess)
    return e;
  if ((e = cudaGetDevice(&dev_id)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(per_sm * sms, max_ctas));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T, int MODE>
cudaError_t dispatch_tws(const SweepArgs<T>& a, size_t smem, bool tws, cudaStream_t st, int max_ctas) {
  return tws ? launch<T, MODE, true>(a, smem, st, max_ctas) : launch<T, MODE, false>(a, smem, st, max_ctas);
}

}  // namespace

template <typename T>
cudaError_t sweep_launch(const Plan<T>& p, PwMode mode, const EvalDesc<T>* ev, int nev, const T* Lhat,
                         cplx<T>* T2, cplx<T>* P2, unsigned* bar, double* flag, cudaStream_t st, int stall) {
  SweepArgs<T> a;
  a.spin_limit = stall > 0 ? (long long)stall : kSpinLimit;
  a.stall = stall > 0 ? 1u : 0u;
  a.p = p;
  a.Lhat = Lhat;
  a.T2 = T2;
  a.P2 = P2;
  a.ev = ev;
  a.nev = nev;
  a.TP = dev::cpw_tile(p);
  const int nper = (mode == PW_GT) ? 3 : 1;
  a.ba = dev::ba_geom(p, 3, nper);
  a.bar = bar;
  a.flag = flag;
  const bool tws = dev::ab_tws(p);
  const int NP = (mode == PW_GT) ? 9 : 3;
  const size_t smem = std::max(dev::ab_smem(p, tws),
                               std::max(dev::cpw_smem(p, a.TP, NP), dev::ba_smem(p, nper, a.ba)));
  const long long P = (long long)p.g.n2 * p.g.n3;
  const int max_ctas = (int)std::max<long long>(
      24LL * p.b.h1, std::max<long long>((P + a.TP - 1) / a.TP, 3LL * p.b.h1 * a.ba.nch));
  if (1 + 3 * p.b.h1 > kSweepBarWords) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(bar, 0, kSweepBarWords * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  switch (mode) {
    case PW_F: return dispatch_tws<T, PW_F>(a, smem, tws, st, max_ctas);
    case PW_T: return dispatch_tws<T, PW_T>(a, smem, tws, st, max_ctas);
    default: return dispatch_tws<T, PW_GT>(a, smem, tws, st, max_ctas);
  }
}

template cudaError_t sweep_launch<float>(const Plan<float>&, PwMode, const EvalDesc<float>*, int,
                                         const float*, cplx<float>*, cplx<float>*, unsigned*, double*,
                                         cudaStream_t, int);
template cudaError_t sweep_launch<double>(const Plan<double>&, PwMode, const EvalDesc<double>*, int,
                                          const double*, cplx<double>*, cplx<double>*, unsigned*, double*,
                                          cudaStream_t, int);

}  // namespace lddmm
