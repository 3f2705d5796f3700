/*
 * lddmm.h -- C interface of the GB300 library for band-limited Jacobi
 * PDE-EPDiff LDDMM subject to the state equation, solved by inexact
 * Gauss-Newton-Krylov (Hernandez, arXiv:1807.11560, Sections 2.5, 2.7, 3.1, 3.2).
 *
 * Problem (Section 3.2, Eqs. 50-52): minimise over the band-limited initial
 * velocity v0
 *     E(v0) = 1/2 <L~ v0, v0>_{l2} + sigma^-2 || m(1) - I1 ||^2_{L2}
 * subject to BL EPDiff  d_t v + ad~^dagger_v v = 0 (Eq. 51) and the state
 * equation d_t m + grad m . iota(v) = 0 on the image grid (Eq. 52), m(0) = I0,
 * with L = (Id - alpha Lap)^s (Eq. 1).
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every call
 * ---------------------------------------------------------------------------
 * Domain      the periodic unit box [0,1)^d, d = 2 or 3; grid N_1 x .. x N_d,
 *             spacing h_j = 1/N_j; <f,g>_{L2} = h^d sum_x f g.
 * Images      real, C order [N_1][N_2]([N_3]), axis 0 slowest.
 * BL fields   complex interleaved (re, im), layout [d][K_1][K_2]([K_3]),
 *             band index q_j in FFT order with signed frequency
 *             f = q (q < K/2) or q - K.  The Nyquist slot q_j = K_j/2 is held
 *             at zero; a field is the Hermitian array of a real vector field.
 *             Inputs are symmetrised on entry ((a(k) + conj a(-k))/2, Nyquist
 *             slots dropped), which is what the real field iota(a) depends on
 *             (Eq. 46).  Outputs are Hermitian with zero Nyquist slots.
 * iota/pi     iota(a)(x) = sum_k a(k) exp(2 pi i k.x) (Eq. 46);
 *             pi(f)(k) = N^-d sum_x f(x) exp(-2 pi i k.x) on the band.
 * L~, K~      symbols (1 + 4 pi^2 alpha |k|^2)^s and its inverse.
 * <.,.>_V     Re sum_k Lhat(k) conj(a(k)) b(k)  (Eq. 47).
 * Precision   LDDMM_FP32: float images and complex64 BL fields, FP32
 *             arithmetic with FP64 reductions; LDDMM_FP64: double and
 *             complex128 throughout.  Every pointer argument has the element
 *             type of the context's precision.
 * Pointers    any pointer argument may be a device pointer or a host pointer
 *             (pageable or pinned); host data are staged through the
 *             context's device buffers with cudaMemcpyAsync on the context
 *             stream.  The caller owns every pointer it passes; the library
 *             never keeps one after the call returns.
 * Ordering    work is issued on the context stream (opts.stream, default the
 *             legacy default stream); every call returns after that stream
 *             has finished the call's work, so outputs are ready on return.
 * Errors      every call returns an lddmm_status; nothing aborts or throws
 *             across this interface.  On failure lddmm_last_error() holds a
 *             one-line message.  A CUDA error leaves the context unusable
 *             except for lddmm_destroy.
 * Threads     a context is used by one host thread at a time.
 * Discretisation (the paper states continuous equations only):
 *             Nt uniform Heun steps for the BL sweeps; semi-Lagrangian
 *             RK2-characteristic transport with trilinear periodic
 *             interpolation on the image grid; central differences for
 *             grad m; products of BL fields formed on a padded grid of
 *             ceil(3K/2) points per axis (exact truncated convolution).
 */
#ifndef LDDMM_H
#define LDDMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lddmm_ctx lddmm_ctx;

typedef enum {
  LDDMM_OK = 0,
  LDDMM_EINVAL = 1,      /* bad argument (sizes, null pointer, unknown option) */
  LDDMM_ENOMEM = 2,      /* device allocation failed */
  LDDMM_ECUDA = 3,       /* a CUDA call failed; see lddmm_last_error */
  LDDMM_ESTATE = 4,      /* call out of order (e.g. hessvec before gradient) */
  LDDMM_ENONFINITE = 5,  /* energy or gradient became NaN/Inf */
  LDDMM_ETIMEOUT = 6,    /* a bounded device wait (persistent-sweep barrier) gave up */
  LDDMM_ENOTCONV = 7     /* reserved for callers; gn_solve reports line-search
                            failure in lddmm_report.ls_failed instead */
} lddmm_status;

/* Arithmetic of a context.  LDDMM_FP64: double throughout.  LDDMM_FP32:
 * float data and arithmetic with FP64 reductions; the tensor cores take the
 * contractions as opts.tensor_cores says (3xTF32 split).  The two split modes
 * are FP32 contexts (float / complex64 arrays) whose contractions run on the
 * tcgen05 tensor cores wherever a kernel covers their sizes (opts.tensor_cores
 * is then 2): LDDMM_3XTF32 splits every operand x = hi + lo into two TF32
 * values and sums three TF32 products; LDDMM_BF16X3 splits the operands of the
 * image-grid band-to-grid stage into three BF16 values (hi + mid + lo) and sums
 * six BF16 products (the other tensor-core kernels keep 3xTF32).  Every mode
 * agrees with FP64 to FP32 rounding (~1e-7 relative per transform).  FP32 with
 * opts.tensor_cores = 0 is the plain FP32 SIMT form. */
typedef enum { LDDMM_FP64 = 0, LDDMM_FP32 = 1, LDDMM_3XTF32 = 2, LDDMM_BF16X3 = 3 } lddmm_precision;

typedef struct {
  int precision;        /* lddmm_precision; default LDDMM_FP32 */
  void* stream;         /* cudaStream_t; NULL = legacy default stream */
  double pcg_tol;       /* PCG stops when ||r||_V <= pcg_tol ||b||_V; default 1e-12 */
  double armijo_c;      /* Armijo constant; default 1e-4 */
  int max_halvings;     /* line-search halvings of eps = 1; default 10 */
  int use_graphs;       /* replay the Hessian-vector product from a CUDA graph; default 1 */
  int persistent;       /* band-limited time sweeps as one persistent cooperative kernel
                           (grid barriers with bounded waits): 0 never (three kernels per
                           bracket evaluation), 1 when the padded product grid has at
                           most 32^3 points (default), 2 always */
  int tensor_cores;     /* FP32 contexts, tcgen05 tensor cores with the 3xTF32 split:
                           iota stage C on the image grid, and the three kernels of a
                           bracket evaluation launched per evaluation (iota A+B;
                           C, the bracket products and C'; pi B'+A' with the
                           epilogue), each where its tile geometry fits the sizes
                           (the SIMT kernel otherwise).  0 never; 1 (default) for
                           image grids of at least 2^20 voxels and padded grids
                           above 32^3 points; 2 whenever supported */
  int recompute;        /* image-grid histories of the time sweeps (velocity grids v_n,
                           characteristic displacements, states m_n, incremental
                           velocity grids): 0 keep all Nt + 1 steps (default); 1 keep
                           two steps and regenerate the rest in forward time order where
                           a sweep reads them (every reader runs forward in time, so no
                           reverse-order checkpoints are needed).  Results are identical;
                           the image-grid footprint drops from about 17 Nt + 20 to about 37
                           floats per voxel (plus the transform scratch), and each
                           Hessian-vector product re-runs the state transport (Nt steps
                           and 2 (Nt + 1) vector iotas more). */
  int autotune;         /* 1 (default): at creation, time the candidate tile shapes of the
                           three padded-grid bracket kernels (twiddle staging, pencils per
                           tile, band rows per item) on this context's sizes and keep the
                           fastest; 0: size heuristics.  Contexts whose sweeps run as
                           persistent kernels keep the heuristics.  No result depends on
                           the tile shapes. */
  int newton;           /* Hessian used by lddmm_gn_solve's PCG: 0 Gauss-Newton (default),
                           1 full Newton (lddmm_hessvec_newton); PCG stops at the first
                           direction of non-positive curvature either way. */
  int state_eq;         /* constraint of the registration problem: 0 the image state
                           equation of Section 3.2 (default: m(t) transported on the
                           image grid); 1 the deformation state equation of Section 3.3
                           (the inverse map x + u(t)(x) carried as a band-limited
                           displacement u~(t), m(1) = I0(x + u(1)(x))).  With 1,
                           lddmm_energy, lddmm_gradient, lddmm_hessvec, lddmm_gn_solve,
                           lddmm_batch_gn_solve and lddmm_transport follow Section 3.3;
                           lddmm_exact_gradient, lddmm_hessvec_newton, lddmm_transport_vjp
                           and newton = 1 are state-form only (LDDMM_EINVAL). */
  int debug_stall;      /* test hook of the time-out path, 0 (default) off.  n > 0: the
                           first grid barrier of every persistent sweep waits for one
                           arrival more than the grid has (it never comes) and every
                           bounded wait gives up after n polls, so the sweep returns
                           early and the call reports LDDMM_ETIMEOUT (the context is
                           unusable afterwards: destroy it).  No GPU fault or hang is
                           involved: every wait stays bounded. */
} lddmm_opts;

/* Report of lddmm_gn_solve.  The per-iteration arrays are optional
 * caller-owned host arrays of length n_gn (NULL to skip). */
typedef struct {
  int gn_iters;          /* Gauss-Newton iterations completed */
  int pcg_iters;         /* total PCG iterations (Hessian-vector products) */
  int ls_failed;         /* 1 if the last line search accepted no step */
  double E_initial;      /* E at the starting v0 */
  double E_final;        /* E at the returned v0 */
  double gnorm_initial;  /* ||g||_V at the starting v0 */
  double gnorm_final;    /* ||g||_V at the last gradient evaluation */
  double* E_hist;        /* optional: E before each GN iteration */
  double* eps_hist;      /* optional: accepted step length of each iteration */
  int* pcg_hist;         /* optional: PCG iterations of each iteration */
} lddmm_report;

/* Defaults for lddmm_opts (precision FP32, legacy stream, tol 1e-12,
 * c = 1e-4, 10 halvings, graphs on, persistent sweeps on small grids,
 * tensor-core image-grid transforms on large grids, kept histories,
 * autotuned tiles). */
void lddmm_default_opts(lddmm_opts* opts);

/* Create a registration context (Section 3.2).
 *   ndim    2 or 3.
 *   grid    ndim image sizes N_j >= 2, N_1 N_2 N_3 < 2^31 (int array, host).
 *   K       ndim band sizes: even, 2 <= K_j <= N_j, K_1 <= 64 (int array, host).
 *   alpha   > 0, s >= 1: L = (Id - alpha Lap)^s (Eq. 1).
 *   sigma   > 0: data weight 1/sigma^2 (Eq. 50).
 *   Nt      >= 1 time steps on [0,1].
 *   opts    NULL for defaults.
 * Allocates every device buffer the context needs (histories for Nt steps,
 * padded-grid caches, transform scratch).  Returns LDDMM_ENOMEM if the
 * device lacks memory, LDDMM_EINVAL for bad sizes (including N_3 > 1024 and
 * grids whose transform tiles exceed shared memory: N_3 above about 700 at
 * K = 32 in FP32, half that in FP64).  *out is NULL on failure. */
int lddmm_create(lddmm_ctx** out, int ndim, const int* grid, const int* K,
                 double alpha, int s, double sigma, int Nt, const lddmm_opts* opts);

/* Copy the source I0 and target I1 images (Section 2.1) into the context.
 * Invalidates any linearisation point. */
int lddmm_set_images(lddmm_ctx* ctx, const void* I0, const void* I1);

/* E(v0) of Eq. 50 (shoot, transport, FP64 reductions).  Does not disturb the
 * linearisation point left by lddmm_gradient. */
int lddmm_energy(lddmm_ctx* ctx, const void* v0, double* E_out);

/* V-gradient g = v0 + W(0) (Eqs. 53-55): forward shoot and transport, the
 * terminal U(1) = K~ pi(lambda(1) grad m(1)), lambda(1) = -2/sigma^2 (m(1)-I1),
 * and the backward reduced adjoint Jacobi sweep.  Writes g (BL field) and,
 * if E_out is not NULL, E(v0).  Sets the linearisation point for hessvec. */
int lddmm_gradient(lddmm_ctx* ctx, const void* v0, void* g_out, double* E_out);

/* Full-Newton Hessian-vector product at the last lddmm_gradient point (Eqs.
 * 56-58 without the Gauss-Newton drop): the derivative of the paper-form
 * gradient along dv.  Adds to the Gauss-Newton product the terms carried by
 * the adjoint variables - ad~^dagger_dv U, ad~^dagger_W dv - ad~_dv W in the
 * backward sweep (with the gradient sweep's (U, W) at every Heun stage and the
 * tangent's dv) and lambda(1) grad dm(1) in the terminal value.  Not symmetric
 * and not positive definite in general.  Same arguments as lddmm_hessvec;
 * LDDMM_ESTATE unless the last call that set the linearisation point was
 * lddmm_gradient (or lddmm_gn_solve). */
int lddmm_hessvec_newton(lddmm_ctx* ctx, const void* dv, void* Hdv_out);

/* V-gradient of the discretised energy itself: the route of Section 2.5
 * (Eqs. 12-14) in discrete form, as a cross-check of the paper-form Jacobi
 * gradient.  The semi-Lagrangian state transport is reversed step by step on
 * the image grid (lambda scattered through the interpolation weights; the
 * characteristic's dependence on v_n and v_{n+1} through the interpolants'
 * exact derivatives), each time level's velocity sensitivity is projected to
 * the band (K~ times the adjoint of iota), and the transpose of the Heun shoot
 * carries the sources back to v0.  Same arguments and outputs as
 * lddmm_gradient (g_out in the V representation, *E_out the energy; the
 * linearisation point for lddmm_hessvec is set too).  Atomic scatters make the
 * FP rounding order vary from run to run.  Needs opts.recompute = 0
 * (LDDMM_EINVAL otherwise). */
int lddmm_exact_gradient(lddmm_ctx* ctx, const void* v0, void* g_out, double* E_out);

/* Gauss-Newton Hessian-vector product in V at the last gradient point
 * (Eqs. 30-31 and 56-58 with every adjoint-weighted term dropped, Section 2.7):
 * incremental BL EPDiff from dv, incremental state transport on the grid,
 * dU(1) = K~ pi(-2/sigma^2 dm(1) grad m(1)), backward adjoint Jacobi sweep;
 * Hdv = dv + dW(0).  LDDMM_ESTATE if no gradient was computed since the
 * last set_images. */
int lddmm_hessvec(lddmm_ctx* ctx, const void* dv, void* Hdv_out);

/* Inexact Gauss-Newton-Krylov (Eqs. 44-45): for each of n_gn iterations,
 * gradient, n_pcg iterations of CG in the V inner product on H p = -g
 * (early stop on ||r||_V <= pcg_tol ||b||_V or non-positive curvature),
 * Armijo backtracking v0 <- v0 + eps p.  v0_inout is read and overwritten.
 * rep may be NULL.  Stops early, with rep->ls_failed = 1, when a line search
 * accepts no step.  The trial sweeps of the line search reuse the state of
 * the linearisation (the accepted one becomes the next iteration's forward
 * sweep), so on return there is no linearisation point: call lddmm_gradient
 * before lddmm_hessvec. */
int lddmm_gn_solve(lddmm_ctx* ctx, void* v0_inout, int n_gn, int n_pcg, lddmm_report* rep);

/* Batched population: lddmm_gn_solve on n independent contexts at once (one
 * registration per context: its own grid, band, images and v0s[i]), driven
 * from min(n, nthreads) host threads (0: one per hardware thread).  Each
 * context runs its calls in order on its own opts.stream, so contexts created
 * with distinct non-NULL streams overlap on the GPU; contexts sharing a stream
 * (or the legacy NULL stream) serialise but stay correct.  Contexts whose
 * sweeps would run as persistent cooperative kernels are refused
 * (LDDMM_EINVAL): independent cooperative grids are not guaranteed to be
 * co-resident.  reps: NULL or n reports.  Returns LDDMM_OK or the first
 * failing context's status (its lddmm_last_error says why); every context is
 * run to the end whatever the others return. */
int lddmm_batch_gn_solve(lddmm_ctx* const* ctxs, int n, void* const* v0s, int n_gn, int n_pcg,
                         lddmm_report* reps, int nthreads);

/* ---------------------------------------------------------------------------
 * Component calls: single steps of the hot path, exposed for testing and for
 * callers composing their own solvers.  Same conventions as above.
 * ------------------------------------------------------------------------- */

/* iota (Eq. 46): ncomp band-limited scalar fields [ncomp][K..] -> grid
 * values [ncomp][N..] on the image grid. */
int lddmm_iota(lddmm_ctx* ctx, const void* a, int ncomp, void* f_out);

/* Allocation-free iota for callers that cannot let a library allocate
 * device memory: a host framework whose caching allocator already holds
 * nearly all device memory, a latency-bound loop that cannot absorb the
 * device-wide synchronisation cudaFree implies, or a plugin host that forbids
 * libraries from allocating.  The paper has no counterpart; this is the same
 * transform as lddmm_iota on an FP32 context, without a context.
 *   ndim, grid, K  as in lddmm_create (host int arrays).
 *   a              device pointer, complex64 [ncomp][K..], symmetrised on entry.
 *   ncomp          1..36 scalar fields.
 *   f_out          device pointer, float32 [ncomp][N..].
 *   a and f_out must be memory of the current device (or managed memory);
 *   the call cannot see their extents, so the caller guarantees the sizes.
 *   stream         cudaStream_t (NULL = legacy default stream).
 * The call is asynchronous: it returns once its kernels are enqueued.
 * It calls no cudaMalloc or cudaFree.  Its scratch is one fixed 32 MiB
 * static device array that every GPU loading this library holds until the
 * process exits.  A problem needs, each rounded up to 256 bytes, the twiddle
 * tables (K3 N3 + K2 N2 + K1/2 N1 complex64 values), the symmetrised input
 * (ncomp K1 K2 K3) and one intermediate (ncomp K1/2 N2 N3); if that exceeds
 * 32 MiB the call returns LDDMM_ENOMEM and does nothing (3 fields on
 * 160x192x160 with band 32^3 need about 13 MiB).  LDDMM_EINVAL for bad sizes
 * (as in lddmm_create) or for a or f_out not being memory of the current
 * device.  LDDMM_ECUDA without launching anything if a CUDA error of earlier
 * work is pending on entry (it is left for the caller to read). 
 * The first call on each device performs a one-time set-up (it looks up the
 * device address of the scratch array); make that first call before any
 * stream capture.  All calls share the one array and it keeps the last
 * call's contents; every call rewrites everything it reads, so nothing has
 * to start at zero.  Calls that overlap on the GPU (on different streams, or
 * from several host threads on one device) race on the array: serialise
 * them. */
int lddmm_iota_noalloc(int ndim, const int* grid, const int* K, const void* a, int ncomp,
                       void* f_out, void* stream);

/* pi: ncomp grid fields [ncomp][N..] -> band coefficients [ncomp][K..]. */
int lddmm_pi(lddmm_ctx* ctx, const void* f, int ncomp, void* a_out);

/* ad~^dagger_v u = K~ pi[(Dv)^T L~u + D(L~u) v + L~u div v] (Eq. 48), products
 * on the padded grid. */
int lddmm_ad_dagger(lddmm_ctx* ctx, const void* v, const void* u, void* out);

/* ad~_v w = pi[Dv w - Dw v] (Eq. 49). */
int lddmm_ad(lddmm_ctx* ctx, const void* v, const void* w, void* out);

/* Heun shoot of BL EPDiff (Eq. 51) from v0; writes v(1).  Uses its own
 * buffers: the linearisation point is kept. */
int lddmm_shoot(lddmm_ctx* ctx, const void* v0, void* v1_out);

/* Shoot and transport I0 (Eqs. 51-52); writes m(1) on the image grid.  Keeps
 * the linearisation point. */
int lddmm_transport(lddmm_ctx* ctx, const void* v0, void* m1_out);

/* Vector-Jacobian product of the map v0 -> m(1) (shoot and transport,
 * Eqs. 51-52) for any scalar loss of m(1).  grad_m1 [N..] is dLoss/dm(1)
 * with respect to the grid values; grad_v0_out [d][K..] receives the l2
 * gradient L~ W(0) with respect to the band coefficients, W the backward
 * reduced adjoint Jacobi sweep (Eqs. 53-54) started from
 * U(1) = K~ pi(lambda(1) grad m(1)) with lambda(1) = -N1 N2 N3 grad_m1 (the
 * L2_h adjoint of the grid values; for the data term of Eq. 50 this is
 * -(2/sigma^2)(m(1) - I1), so L~^-1 of the result is the data part of
 * lddmm_gradient).  Runs the forward shoot and transport at v0 first and
 * leaves it as the linearisation point. */
int lddmm_transport_vjp(lddmm_ctx* ctx, const void* v0, const void* grad_m1, void* grad_v0_out);

/* The same vector-Jacobian product through the exact discrete adjoint of the
 * discretised map v0 -> m(1) (the route of Section 2.5, Eqs. 12-14, in discrete
 * form, as in lddmm_exact_gradient): lambda(1) = grad_m1 is carried back through
 * the transposes of the semi-Lagrangian steps, each time level's velocity
 * sensitivity is projected to the band and the Heun shoot is transposed.  The
 * result is the derivative of the discrete m(1) itself (central differences of
 * the forward map converge to it), where lddmm_transport_vjp follows the
 * paper's reduced adjoint Jacobi sweep.  Same arguments and output convention
 * as lddmm_transport_vjp; needs opts.recompute = 0 and the image state form
 * (LDDMM_EINVAL otherwise).  Atomic scatters make the rounding order vary from
 * run to run.  Leaves v0 as the linearisation point. */
int lddmm_transport_vjp_exact(lddmm_ctx* ctx, const void* v0, const void* grad_m1, void* grad_v0_out);

/* dm(1) of the last lddmm_hessvec call (incremental state, Eq. 31). */
int lddmm_last_dm1(lddmm_ctx* ctx, void* dm1_out);

/* Timing probe.  Brackets every launch of one kernel class with CUDA events
 * on the stream it runs on (also inside the captured Hessian-vector graph)
 * and accumulates the elapsed device time and the algorithmic work of each
 * timed launch.  kernel_class is one of
 *   "transport"  semi-Lagrangian state step (Eq. 52); work = 8 N bytes
 *                (read m_n, write m_{n+1});
 *   "inc_step"   incremental state step (Eq. 31); work = 12 N bytes
 *                (read m_n and dm_n, write dm_{n+1});
 *   "iota_ab", "cpw", "pi_ba"  the three kernels of a bracket evaluation on
 *                the padded product grid (Eqs. 48-49); work = flops of their
 *                contractions and bracket products;
 *   "iota_full", "pi_full"  transforms on the image grid; work = flops;
 *   "sweep"      one persistent band-limited sweep kernel; work = flops;
 * NULL or "" switches the probe off.  Changing the class rebuilds the graph
 * on the next product.  Not part of the method; the paper has no
 * counterpart. */
int lddmm_probe(lddmm_ctx* ctx, const char* kernel_class);

/* Accumulated probe time (ms), number of timed launches and algorithmic work
 * (bytes or flops, see lddmm_probe) since the last read or lddmm_probe call;
 * resets all three. */
int lddmm_probe_read(lddmm_ctx* ctx, double* total_ms, long long* launches, double* work);

/* Number of CUDA kernels this context has launched since creation (graph
 * replays count each kernel node). */
long long lddmm_kernel_count(const lddmm_ctx* ctx);

/* Tile shapes the context's padded-grid bracket kernels use (after the
 * autotuner, or the size heuristics): tws 1/2 = iota A+B twiddles from global
 * / shared memory, tp = pencils per C/products/C' tile, kc = band rows per
 * pi B'/A' item.  LDDMM_EINVAL on NULL arguments. */
int lddmm_tile_config(const lddmm_ctx* ctx, int* tws, int* tp, int* kc);

/* Bytes of device memory the context holds (all of it is allocated by
 * lddmm_create; no later call allocates).  0 for NULL. */
unsigned long long lddmm_device_bytes(const lddmm_ctx* ctx);

/* One-line description of the last error on this context (never NULL). */
const char* lddmm_last_error(const lddmm_ctx* ctx);

/* Free every device buffer of the context.  NULL is allowed. */
void lddmm_destroy(lddmm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LDDMM_H */
