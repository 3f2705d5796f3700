"""Shared helpers of the GPU parity tests (not a test module)."""

import numpy as np

from oracle import bl, objective
from paper_1807_11560_gb300 import Context, inputs

ALPHA, S, SIGMA = 0.0025, 2, 0.03


def torch_dev(x, precision):
    import torch
    if np.iscomplexobj(x):
        dt = torch.complex128 if precision == "fp64" else torch.complex64
    else:
        dt = torch.float64 if precision == "fp64" else torch.float32
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dt).contiguous()


def host(x):
    return x.detach().cpu().numpy().astype(np.complex128 if x.is_complex() else np.float64)


def quantise(x, precision):
    """The values the GPU actually receives (so input rounding is not counted as error)."""
    if precision == "fp64":
        return np.asarray(x)
    return np.asarray(x).astype(np.complex64 if np.iscomplexobj(x) else np.float32).astype(
        np.complex128 if np.iscomplexobj(x) else np.float64)


def rel_inf(a, b):
    """Element-wise relative error: max |a - b| over the largest |b|."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_V(a, b, Ks):
    """The larger of the relative error in the V norm (Eq. 47) and the
    element-wise relative error, so an error confined to a few band slots
    cannot hide inside the norm."""
    L = bl.lhat(tuple(Ks), ALPHA, S)
    norm = float(np.sqrt(np.sum(L * np.abs(a - b) ** 2) / np.sum(L * np.abs(b) ** 2)))
    return max(norm, rel_inf(a, b))


def rel_2(a, b):
    """The larger of the relative l2 error and the element-wise relative error,
    so an error confined to a few voxels (a boundary wrap, one plane of a tile)
    cannot hide inside the norm."""
    norm = float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))
    return max(norm, rel_inf(a, b))


def problem(kind, Ns, Ks, seed, Nt, precision, max_disp=2.0, v_disp=2.0, **ctx_kw):
    """(Context with images set, oracle Problem on the same quantised images, v0, p)."""
    I0, I1 = inputs.make_pair(kind, Ns, seed, max_disp=max_disp)
    I0, I1 = quantise(I0, precision), quantise(I1, precision)
    d = len(Ns)
    v0 = quantise(inputs.random_bl(Ks, d, seed + 1, v_disp, Ns), precision)
    p = quantise(inputs.random_bl(Ks, d, seed + 2, 1.0, Ns), precision)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision=precision, **ctx_kw)
    ctx.set_images(torch_dev(I0, precision), torch_dev(I1, precision))
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    return ctx, P, v0, p


# ---- central differences of the FP64 oracle's energy, one direction per task.
# Runs in worker processes (spawn context): each worker builds the problem once.
_FD_PROBLEM = {}


def _fd_problem(name):
    from oracle import objective
    from paper_1807_11560_gb300 import inputs
    if name not in _FD_PROBLEM:
        kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[name]
        I0, I1 = inputs.make_pair(kind, Ns, seed)
        I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
        v0 = quantise(inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns), "fp32")
        _FD_PROBLEM[name] = (objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt), v0, Ns, Ks)
    return _FD_PROBLEM[name]


def fd_data_term(task):
    """(seed, directional derivative of the data term along the seeded direction,
    the direction) by central differences of the oracle forward."""
    from paper_1807_11560_gb300 import inputs
    name, seed, eps = task
    P, v0, Ns, Ks = _fd_problem(name)
    p = inputs.random_bl(Ks, 3, seed, 1.0, Ns)
    Ep = P.data_term(P.forward(v0 + eps * p)[3][-1])
    Em = P.data_term(P.forward(v0 - eps * p)[3][-1])
    return seed, (Ep - Em) / (2 * eps), p


def spawn_pool(n):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n)


def oracle_grad_hessvec(task):
    """(E, g, H p) of the FP64 oracle for one workload entry (kind, grid, band,
    Nt, seed) with the seeded v0 and p of the batch tests (runs in a worker)."""
    from oracle import objective
    from paper_1807_11560_gb300 import inputs
    kind, Ns, Ks, Nt, seed = task
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, 3, seed + 2, 1.0, Ns), "fp32")
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    lin = P.gradient(v0)
    return lin.E, lin.g, P.hessvec(lin, p)
