"""Python binding of liblddmm.so (C interface in include/lddmm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be torch tensors (CUDA or CPU, contiguous) or numpy
arrays (host); their element type must match the context's precision
(float32/complex64 for ``"fp32"``, float64/complex128 for ``"fp64"``).
There is no CPU fallback: if the shared library is missing, every call raises.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblddmm.so")
_lib = None

LDDMM_FP64, LDDMM_FP32, LDDMM_3XTF32, LDDMM_BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": LDDMM_FP64, "fp32": LDDMM_FP32, "3xtf32": LDDMM_3XTF32, "bf16x3": LDDMM_BF16X3}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ENONFINITE",
          6: "ETIMEOUT", 7: "ENOTCONV"}


class LddmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lddmm error {STATUS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("pcg_tol", ctypes.c_double), ("armijo_c", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("persistent", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("recompute", ctypes.c_int), ("autotune", ctypes.c_int), ("newton", ctypes.c_int),
                ("state_eq", ctypes.c_int), ("debug_stall", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("gn_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int), ("ls_failed", ctypes.c_int),
                ("E_initial", ctypes.c_double), ("E_final", ctypes.c_double),
                ("gnorm_initial", ctypes.c_double), ("gnorm_final", ctypes.c_double),
                ("E_hist", ctypes.POINTER(ctypes.c_double)),
                ("eps_hist", ctypes.POINTER(ctypes.c_double)),
                ("pcg_hist", ctypes.POINTER(ctypes.c_int))]


def _report(n_gn):
    """A Report with caller-owned history arrays (kept alive by the second item)."""
    r = Report()
    E = (ctypes.c_double * max(1, n_gn))()
    eps = (ctypes.c_double * max(1, n_gn))()
    its = (ctypes.c_int * max(1, n_gn))()
    r.E_hist = ctypes.cast(E, ctypes.POINTER(ctypes.c_double))
    r.eps_hist = ctypes.cast(eps, ctypes.POINTER(ctypes.c_double))
    r.pcg_hist = ctypes.cast(its, ctypes.POINTER(ctypes.c_int))
    return r, (E, eps, its)


def _report_dict(r, keep):
    E, eps, its = keep
    n = r.gn_iters
    extra = 1 if r.ls_failed else 0
    return {"gn_iters": n, "pcg_iters": r.pcg_iters, "ls_failed": bool(r.ls_failed),
            "E_initial": r.E_initial, "E_final": r.E_final, "gnorm_initial": r.gnorm_initial,
            "gnorm_final": r.gnorm_final, "E": list(E[:n + extra][:max(n, 1)]),
            "eps": list(eps[:n]), "pcg": list(its[:n + extra])}


def batch_gn_solve(contexts, v0s, n_gn, n_pcg, threads=0):
    """lddmm_batch_gn_solve: GN-Krylov on independent registrations at once (each
    Context on its own stream); v0s are updated in place.  Returns the reports."""
    n = len(contexts)
    if n != len(v0s) or n == 0:
        raise ValueError("one v0 per context")
    hs = (ctypes.c_void_p * n)(*[c._h for c in contexts])
    ps = (ctypes.c_void_p * n)(*[c._arg(v, "cplx", c.nband) for c, v in zip(contexts, v0s)])
    reps = (Report * n)()
    keeps = []
    for i in range(n):
        r, keep = _report(n_gn)
        reps[i] = r
        keeps.append(keep)
    code = lib().lddmm_batch_gn_solve(hs, n, ps, int(n_gn), int(n_pcg), reps, int(threads))
    if code != 0:
        bad = [c for c in contexts if lib().lddmm_last_error(c._h)]
        msg = "; ".join(lib().lddmm_last_error(c._h).decode() for c in bad) or "batch failed"
        raise LddmmError(code, msg)
    return [_report_dict(reps[i], keeps[i]) for i in range(n)]


def lib():
    """Load liblddmm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1807_11560_gb300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "lddmm_default_opts": (None, [ctypes.POINTER(Opts)]),
        "lddmm_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I), ctypes.POINTER(I), D, I, D, I,
                             ctypes.POINTER(Opts)]),
        "lddmm_set_images": (I, [P, P, P]),
        "lddmm_energy": (I, [P, P, ctypes.POINTER(D)]),
        "lddmm_gradient": (I, [P, P, P, ctypes.POINTER(D)]),
        "lddmm_hessvec": (I, [P, P, P]),
        "lddmm_exact_gradient": (I, [P, P, P, ctypes.POINTER(D)]),
        "lddmm_hessvec_newton": (I, [P, P, P]),
        "lddmm_gn_solve": (I, [P, P, I, I, ctypes.POINTER(Report)]),
        "lddmm_batch_gn_solve": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P), I, I,
                                     ctypes.POINTER(Report), I]),
        "lddmm_iota": (I, [P, P, I, P]),
        "lddmm_pi": (I, [P, P, I, P]),
        "lddmm_ad_dagger": (I, [P, P, P, P]),
        "lddmm_ad": (I, [P, P, P, P]),
        "lddmm_shoot": (I, [P, P, P]),
        "lddmm_transport": (I, [P, P, P]),
        "lddmm_last_dm1": (I, [P, P]),
        "lddmm_transport_vjp": (I, [P, P, P, P]),
        "lddmm_transport_vjp_exact": (I, [P, P, P, P]),
        "lddmm_kernel_count": (ctypes.c_longlong, [P]),
        "lddmm_device_bytes": (ctypes.c_ulonglong, [P]),
        "lddmm_tile_config": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "lddmm_probe": (I, [P, ctypes.c_char_p]),
        "lddmm_probe_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(D)]),
        "lddmm_iota_noalloc": (I, [I, ctypes.POINTER(I), ctypes.POINTER(I), P, I, P, P]),
        "lddmm_last_error": (ctypes.c_char_p, [P]),
        "lddmm_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(x):
    """Device or host address of a contiguous torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _dtype_name(x):
    return str(x.dtype).replace("torch.", "")


def iota_noalloc(grid, K, a, ncomp, out, stream=None):
    """lddmm_iota_noalloc: iota of ncomp band-limited scalar fields without any
    device allocation (FP32; a and out must be CUDA tensors).  Asynchronous on
    ``stream``; returns the status code (0 = OK)."""
    grid, K = tuple(int(g) for g in grid), tuple(int(k) for k in K)
    if len(grid) != len(K):
        raise ValueError("grid and K need one size per axis each")
    if _dtype_name(a) != "complex64" or _dtype_name(out) != "float32":
        raise TypeError("iota_noalloc takes complex64 input and float32 output")
    # the C entry point cannot see extents: an undersized array would be read or
    # written out of bounds on the device, so the sizes are checked here
    if int(np.prod(a.shape)) != int(ncomp) * int(np.prod(K)):
        raise ValueError(f"a must hold ncomp * prod(K) = {int(ncomp) * int(np.prod(K))} values")
    if int(np.prod(out.shape)) != int(ncomp) * int(np.prod(grid)):
        raise ValueError(f"out must hold ncomp * prod(grid) = {int(ncomp) * int(np.prod(grid))} values")
    import torch
    if not (isinstance(a, torch.Tensor) and isinstance(out, torch.Tensor) and a.is_cuda and out.is_cuda):
        raise TypeError("iota_noalloc takes CUDA tensors")
    cur = torch.cuda.current_device()
    if a.device.index != cur or out.device.index != cur:
        raise ValueError("a and out must be on the current CUDA device")
    arr = ctypes.c_int * len(grid)
    return lib().lddmm_iota_noalloc(len(grid), arr(*grid), arr(*K), _ptr(a), int(ncomp), _ptr(out), stream)


class Context:
    """One registration problem on the GPU (wraps an ``lddmm_ctx``).

    grid, K: per-axis image and band sizes (2 or 3 axes); alpha, s: L =
    (Id - alpha Lap)^s; sigma: data weight 1/sigma^2; Nt: time steps.
    state: "image" (the image state equation, Section 3.2) or "deformation"
    (the band-limited deformation state equation, Section 3.3).
    precision: "fp64", "fp32" (tensor cores as ``tensor_cores`` says),
    "3xtf32" or "bf16x3" (FP32 arrays; contractions on the tensor cores with
    that operand split wherever a kernel covers their sizes).
    """

    def __init__(self, grid, K, alpha, s, sigma, Nt, precision="fp32", stream=None,
                 use_graphs=True, pcg_tol=1e-12, armijo_c=1e-4, max_halvings=10, persistent="auto",
                 tensor_cores="auto", recompute=False, autotune=True, newton=False, state="image",
                 debug_stall=0):
        L = lib()
        self.grid, self.K = tuple(int(g) for g in grid), tuple(int(k) for k in K)
        self.ndim = len(self.grid)
        self.precision = precision
        self.real = "float64" if precision == "fp64" else "float32"
        self.complex = "complex128" if precision == "fp64" else "complex64"
        o = Opts()
        L.lddmm_default_opts(ctypes.byref(o))
        if precision not in PRECISIONS:
            raise ValueError(f"precision is one of {sorted(PRECISIONS)}")
        o.precision = PRECISIONS[precision]
        o.stream = stream
        o.use_graphs = 1 if use_graphs else 0
        o.persistent = {True: 2, False: 0, "auto": 1}[persistent]
        o.tensor_cores = {True: 2, False: 0, "auto": 1}[tensor_cores]
        o.recompute = 1 if recompute else 0
        o.autotune = 1 if autotune else 0
        o.newton = 1 if newton else 0
        o.state_eq = {"image": 0, "deformation": 1}[state]
        o.debug_stall = int(debug_stall)
        o.pcg_tol, o.armijo_c, o.max_halvings = pcg_tol, armijo_c, max_halvings
        arr = ctypes.c_int * self.ndim
        h = ctypes.c_void_p()
        rc = L.lddmm_create(ctypes.byref(h), self.ndim, arr(*self.grid), arr(*self.K), float(alpha),
                            int(s), float(sigma), int(Nt), ctypes.byref(o))
        if rc != 0:
            raise LddmmError(rc, "lddmm_create failed")
        self._h = h

    # -- plumbing --------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise LddmmError(rc, lib().lddmm_last_error(self._h).decode())

    def _arg(self, x, kind, n):
        name = _dtype_name(x)
        want = self.real if kind == "real" else self.complex
        if name != want:
            raise TypeError(f"expected {want} array, got {name}")
        if int(np.prod(x.shape)) != n:
            raise ValueError(f"expected {n} elements, got shape {tuple(x.shape)}")
        return _ptr(x)

    @property
    def nvox(self):
        return int(np.prod(self.grid))

    @property
    def nband(self):
        return self.ndim * int(np.prod(self.K))

    def close(self):
        if getattr(self, "_h", None):
            lib().lddmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls -----------------------------------------------------------
    def set_images(self, I0, I1):
        self._check(lib().lddmm_set_images(self._h, self._arg(I0, "real", self.nvox),
                                           self._arg(I1, "real", self.nvox)))

    def energy(self, v0):
        E = ctypes.c_double()
        self._check(lib().lddmm_energy(self._h, self._arg(v0, "cplx", self.nband), ctypes.byref(E)))
        return E.value

    def gradient(self, v0, g_out):
        E = ctypes.c_double()
        self._check(lib().lddmm_gradient(self._h, self._arg(v0, "cplx", self.nband),
                                         self._arg(g_out, "cplx", self.nband), ctypes.byref(E)))
        return E.value

    def hessvec_newton(self, dv, out):
        """Full-Newton Hessian-vector product at the last gradient point."""
        self._check(lib().lddmm_hessvec_newton(self._h, self._arg(dv, "cplx", self.nband),
                                               self._arg(out, "cplx", self.nband)))

    def exact_gradient(self, v0, g_out):
        """V-gradient of the discretised energy (exact discrete adjoint); returns E."""
        E = ctypes.c_double()
        self._check(lib().lddmm_exact_gradient(self._h, self._arg(v0, "cplx", self.nband),
                                               self._arg(g_out, "cplx", self.nband), ctypes.byref(E)))
        return E.value

    def hessvec(self, dv, out):
        self._check(lib().lddmm_hessvec(self._h, self._arg(dv, "cplx", self.nband),
                                        self._arg(out, "cplx", self.nband)))

    def gn_solve(self, v0_inout, n_gn, n_pcg):
        r, keep = _report(n_gn)
        self._check(lib().lddmm_gn_solve(self._h, self._arg(v0_inout, "cplx", self.nband), int(n_gn),
                                         int(n_pcg), ctypes.byref(r)))
        return _report_dict(r, keep)

    def iota(self, a, ncomp, out):
        kv, nv = int(np.prod(self.K)), self.nvox
        self._check(lib().lddmm_iota(self._h, self._arg(a, "cplx", ncomp * kv), int(ncomp),
                                     self._arg(out, "real", ncomp * nv)))

    def pi(self, f, ncomp, out):
        kv, nv = int(np.prod(self.K)), self.nvox
        self._check(lib().lddmm_pi(self._h, self._arg(f, "real", ncomp * nv), int(ncomp),
                                   self._arg(out, "cplx", ncomp * kv)))

    def ad_dagger(self, v, u, out):
        self._check(lib().lddmm_ad_dagger(self._h, self._arg(v, "cplx", self.nband),
                                          self._arg(u, "cplx", self.nband),
                                          self._arg(out, "cplx", self.nband)))

    def ad(self, v, w, out):
        self._check(lib().lddmm_ad(self._h, self._arg(v, "cplx", self.nband),
                                   self._arg(w, "cplx", self.nband), self._arg(out, "cplx", self.nband)))

    def shoot(self, v0, out):
        self._check(lib().lddmm_shoot(self._h, self._arg(v0, "cplx", self.nband),
                                      self._arg(out, "cplx", self.nband)))

    def transport(self, v0, m1_out):
        self._check(lib().lddmm_transport(self._h, self._arg(v0, "cplx", self.nband),
                                          self._arg(m1_out, "real", self.nvox)))

    def transport_vjp(self, v0, grad_m1, out, exact=False):
        """l2 gradient of a loss of m(1) in v0 from dL/dm(1): the paper's adjoint
        Jacobi sweep, or (exact=True) the exact discrete adjoint of the map."""
        fn = lib().lddmm_transport_vjp_exact if exact else lib().lddmm_transport_vjp
        self._check(fn(self._h, self._arg(v0, "cplx", self.nband), self._arg(grad_m1, "real", self.nvox),
                       self._arg(out, "cplx", self.nband)))

    def last_dm1(self, out):
        self._check(lib().lddmm_last_dm1(self._h, self._arg(out, "real", self.nvox)))

    def probe(self, kernel_class):
        """Time every launch of one kernel class with CUDA events (None: off)."""
        self._check(lib().lddmm_probe(self._h, (kernel_class or "").encode()))

    def probe_read(self):
        """(total device ms, timed launches, algorithmic work) since the last read."""
        ms, n, w = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        self._check(lib().lddmm_probe_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
        return ms.value, n.value, w.value

    @property
    def kernel_count(self):
        return int(lib().lddmm_kernel_count(self._h))

    @property
    def tiles(self):
        """(twiddle staging 1/2, pencils per tile, band rows per item) in effect."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().lddmm_tile_config(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    @property
    def device_bytes(self):
        """Device memory held by the context (all allocated at creation)."""
        return int(lib().lddmm_device_bytes(self._h))
