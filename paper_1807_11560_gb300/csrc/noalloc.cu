// Allocation-free variant of the band-limited -> grid transform (iota).
//
// Some callers cannot let a library call cudaMalloc: a host framework whose
// caching allocator already holds nearly all device memory, a latency-bound
// loop that cannot absorb the device-wide synchronisation cudaFree implies,
// or a plugin host that forbids libraries from allocating at all.  For them
// lddmm_iota_noalloc runs the same transform kernels as lddmm_iota,
// but every intermediate lives in the fixed device array below instead of in
// buffers of a context.  The caller passes device inputs and outputs only.
#include <mutex>

#include "../../include/lddmm.h"
#include "internal.h"

namespace lddmm {
namespace {

// Fixed scratch: every GPU that loads this library holds it until exit.
constexpr size_t kNoAllocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host code must not use g_noalloc_scratch as an address: its host name is a
// stand-in symbol.  The device address is looked up once per device.
struct DeviceScratch {
  std::once_flag once;
  cudaError_t err = cudaSuccess;
  unsigned char* ptr = nullptr;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_scratch_of[kMaxDevices];

__device__ __forceinline__ int sfreq_dev(int q, int K) { return (2 * q < K) ? q : q - K; }

__device__ __forceinline__ float2 twiddle(long long p, int G, double w) {
  const long long r = ((p % G) + G) % G;
  double s, c;
  sincospi(2.0 * (double)r / (double)G, &s, &c);
  return make_float2((float)(w * c), (float)(w * s));
}

// The three iota twiddle tables of Plan (E3f, E2f, E1f), one entry per thread.
__global__ void k_iota_twiddles(float2* E3f, float2* E2f, float2* E1f, Band b, Dims g) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n3 = (long long)b.k3 * g.n3, n2 = (long long)b.k2 * g.n2,
                  n1 = (long long)b.h1 * g.n1;
  if (i < n3) {
    const int k = (int)(i / g.n3), x = (int)(i % g.n3);
    E3f[i] = twiddle((long long)sfreq_dev(k, b.k3) * x, g.n3, 1.0);
    return;
  }
  i -= n3;
  if (i < n2) {
    const int k = (int)(i / g.n2), x = (int)(i % g.n2);
    E2f[i] = twiddle((long long)sfreq_dev(k, b.k2) * x, g.n2, 1.0);
    return;
  }
  i -= n2;
  if (i < n1) {
    const int h = (int)(i / g.n1), x = (int)(i % g.n1);
    E1f[i] = twiddle((long long)h * x, g.n1, h == 0 ? 1.0 : 2.0);
  }
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// device memory of device dev (or managed memory, which every device reaches)
bool is_device_pointer(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace
}  // namespace lddmm

extern "C" int lddmm_iota_noalloc(int ndim, const int* grid, const int* K, const void* a, int ncomp,
                                  void* f_out, void* stream) {
  using namespace lddmm;
  if ((ndim != 2 && ndim != 3) || !grid || !K || !a || !f_out || ncomp < 1 || ncomp > kMaxIota)
    return LDDMM_EINVAL;
  for (int j = 0; j < ndim; ++j)
    if (grid[j] < 2 || K[j] < 2 || (K[j] & 1) || K[j] > grid[j] || grid[j] > (1 << 16))
      return LDDMM_EINVAL;
  const Dims N{grid[0], grid[1], ndim == 3 ? grid[2] : 1};
  Band b;
  b.k1 = K[0];
  b.k2 = K[1];
  b.k3 = ndim == 3 ? K[2] : 1;
  b.h1 = b.k1 / 2;
  const size_t c8 = sizeof(float2);
  const size_t s3 = align256((size_t)b.k3 * N.n3 * c8), s2 = align256((size_t)b.k2 * N.n2 * c8),
               s1 = align256((size_t)b.h1 * N.n1 * c8), sh = align256((size_t)ncomp * b.vol() * c8),
               st2 = align256((size_t)ncomp * b.h1 * N.n2 * N.n3 * c8);
  if (s3 + s2 + s1 + sh + st2 > kNoAllocBytes) return LDDMM_ENOMEM;

  // an error left pending by earlier work of the caller is not this call's:
  // report it without launching anything (and leave it for the caller)
  if (cudaPeekAtLastError() != cudaSuccess) return LDDMM_ECUDA;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LDDMM_ECUDA;
  }
  DeviceScratch& ds = g_scratch_of[dev];
  std::call_once(ds.once, [&] {
    ds.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&ds.ptr), g_noalloc_scratch);
  });
  if (ds.err != cudaSuccess || !ds.ptr) return LDDMM_ECUDA;
  if (!is_device_pointer(a, dev) || !is_device_pointer(f_out, dev)) return LDDMM_EINVAL;

  unsigned char* base = ds.ptr;
  Plan<float> p{};
  p.g = N;
  p.b = b;
  p.E3f = reinterpret_cast<float2*>(base);
  p.E2f = reinterpret_cast<float2*>(base + s3);
  p.E1f = reinterpret_cast<float2*>(base + s3 + s2);
  float2* herm = reinterpret_cast<float2*>(base + s3 + s2 + s1);
  float2* T2 = reinterpret_cast<float2*>(base + s3 + s2 + s1 + sh);
  if (max_smem_needed<float>(p, 1, false) > smem_limit()) return LDDMM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  const long long ntw = (long long)b.k3 * N.n3 + (long long)b.k2 * N.n2 + (long long)b.h1 * N.n1;
  k_iota_twiddles<<<(unsigned)((ntw + 255) / 256), 256, 0, st>>>(p.E3f, p.E2f, p.E1f, b, N);
  hermitianize<float>(static_cast<const float2*>(a), herm, ncomp, b, st);
  if (cudaGetLastError() != cudaSuccess) return LDDMM_ECUDA;   // nothing further is enqueued
  IotaDesc<float> d{};
  d.nf = ncomp;
  for (int c = 0; c < ncomp; ++c) {
    d.src[c] = herm + (long long)c * b.vol();
    d.dst[c] = static_cast<float*>(f_out) + (long long)c * N.vol();
    d.deriv[c] = -1;
    d.applyL[c] = 0;
  }
  // applyL is off for every field, so the symbol table is never read
  iota_batch<float>(p, d, reinterpret_cast<const float*>(herm), T2, st);
  return cudaGetLastError() == cudaSuccess ? LDDMM_OK : LDDMM_ECUDA;
}
