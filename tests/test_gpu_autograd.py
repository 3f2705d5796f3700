"""torch.autograd through the shoot-and-transport map (lddmm_transport_vjp): the
backward is the library's adjoint Jacobi sweep.  Checked against the FP64 oracle's
adjoint-Jacobi gradient of the same loss, against the library's own gradient for
the data term, and against central finite differences of the oracle forward."""

import numpy as np
import pytest

from oracle import bl, objective, sweeps
from paper_1807_11560_gb300 import Context, inputs
from paper_1807_11560_gb300.autograd import shoot_transport

from helpers import (ALPHA, S, SIGMA, _fd_problem, fd_data_term, host, quantise, rel_2, spawn_pool,
                     torch_dev)

pytestmark = pytest.mark.gpu


def _oracle_l2_grad(P, v0, w):
    """l2 gradient of sum(w * m(1)) in v0: L~ W(0) from U(1) = K~ pi(-N w grad m(1))."""
    lin = P.gradient(v0)
    U1 = P.terminal_U(lin.ms[-1], -float(np.prod(P.Ns)) * w)
    W0 = sweeps.adjoint_jacobi_backward(lin.vs, lin.vstar, U1, ALPHA, S)
    return P.L * W0, lin


def _oracle_exact_l2_grad(P, v0, w):
    """l2 gradient of sum(w * m(1)) in v0 through the exact discrete adjoint of
    the oracle's forward map (transport reversed step by step, Heun shoot
    transposed): L~ W_0 with lambda(1) = w."""
    vs, vstar, vgrid, ms, feet = P.forward(v0)
    G = sweeps.transport_adjoint(ms, vgrid, w, P.dt)
    nd = float(np.prod(P.Ns))
    sources = [nd * bl.pi(Gn, P.Ks) / P.L for Gn in G]
    return P.L * sweeps.transpose_shoot(vs, vstar, sources, ALPHA, S), ms[-1]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exact_autograd_matches_oracle_discrete_adjoint(precision):
    import torch
    Ns, Ks, Nt = (20, 18, 16), (8, 6, 6), 4
    I0, I1 = inputs.make_pair("ellipsoids", Ns, 36, max_disp=2.0)
    I0, I1 = quantise(I0, precision), quantise(I1, precision)
    v0 = quantise(inputs.random_bl(Ks, 3, 37, 2.0, Ns), precision)
    w = quantise(np.random.default_rng(38).normal(size=Ns), precision)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision=precision)
    ctx.set_images(torch_dev(I0, precision), torch_dev(I1, precision))
    v = torch_dev(v0, precision).requires_grad_(True)
    m1 = shoot_transport(ctx, v, adjoint="exact")
    (m1 * torch_dev(w, precision)).sum().backward()
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    g_ref, m1_ref = _oracle_exact_l2_grad(P, v0, w)
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert rel_2(host(m1.detach()), m1_ref) < tol
    assert rel_2(host(v.grad), g_ref) < tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autograd_matches_oracle_adjoint_gradient(precision):
    import torch
    Ns, Ks, Nt = (20, 18, 16), (8, 6, 6), 4
    I0, I1 = inputs.make_pair("ellipsoids", Ns, 31, max_disp=2.0)
    I0, I1 = quantise(I0, precision), quantise(I1, precision)
    v0 = quantise(inputs.random_bl(Ks, 3, 32, 2.0, Ns), precision)
    w = quantise(np.random.default_rng(33).normal(size=Ns), precision)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision=precision)
    ctx.set_images(torch_dev(I0, precision), torch_dev(I1, precision))
    v = torch_dev(v0, precision).requires_grad_(True)
    m1 = shoot_transport(ctx, v)
    (m1 * torch_dev(w, precision)).sum().backward()
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    g_ref, lin = _oracle_l2_grad(P, v0, w)
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert rel_2(host(m1.detach()), lin.ms[-1]) < tol
    assert rel_2(host(v.grad), g_ref) < tol


def test_autograd_of_the_data_term_is_the_library_gradient():
    import torch
    Ns, Ks, Nt = (20, 18, 16), (8, 6, 6), 4
    I0, I1 = inputs.make_pair("ellipsoids", Ns, 34, max_disp=2.0)
    v0 = inputs.random_bl(Ks, 3, 35, 2.0, Ns)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp64")
    ctx.set_images(torch_dev(I0, "fp64"), torch_dev(I1, "fp64"))
    v = torch_dev(v0, "fp64").requires_grad_(True)
    m1 = shoot_transport(ctx, v)
    I1d = torch_dev(I1, "fp64")
    loss = ((m1 - I1d) ** 2).mean() / SIGMA ** 2            # h^d sum = mean on the unit box
    loss.backward()
    g = torch.empty_like(v)
    ctx.gradient(torch_dev(v0, "fp64"), g)
    L = bl.lhat(Ks, ALPHA, S)
    data_part = host(g) - v0                                  # V-gradient minus the regulariser
    np.testing.assert_allclose(host(v.grad) / L, data_part, atol=1e-10 * np.abs(data_part).max())


def test_differentiation_check_96cubed():
    """The 96^3 brain configuration, band 24^3, Nt = 16: GPU FP32 autograd against the
    FP64 oracle's adjoint gradient (1e-5) and against central differences of the FP64
    oracle forward along 20 seeded directions (step 1e-3), with the image-grid
    histories kept and regenerated (recompute mode); the device footprint of both
    modes is printed.  The FD comparison measures the discretisation gap of the
    paper-form gradient (it is not the exact derivative of the discrete energy away
    from v0 = 0): the gradient must track the differences across directions."""
    import os
    import torch
    name = "3d_96_brain"
    kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[name]
    seeds = list(range(2000, 2020))
    pool = spawn_pool(min(len(seeds), os.cpu_count() or 1))   # before any oracle work here
    try:
        fd_async = pool.map_async(fd_data_term, [(name, s_, 1e-3) for s_ in seeds])
        P, v0, _, _ = _fd_problem(name)
        I0, I1 = P.I0.astype(np.float32), P.I1.astype(np.float32)
        grads, footprint = {}, {}
        for recompute in (False, True):
            free0 = torch.cuda.mem_get_info()[0]
            ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", recompute=recompute)
            footprint[recompute] = (ctx.device_bytes, free0 - torch.cuda.mem_get_info()[0])
            ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
            v = torch_dev(v0, "fp32").requires_grad_(True)
            m1 = shoot_transport(ctx, v)
            I1d = torch_dev(I1, "fp32")
            (((m1 - I1d) ** 2).mean() / SIGMA ** 2).backward()
            grads[recompute] = host(v.grad)
            ctx.close()
        lin = P.gradient(v0)
        g_ref = P.L * (lin.g - v0)                           # l2 form of the data part
        out = fd_async.get(timeout=3600)
    finally:
        pool.terminate()
        pool.join()
    g = grads[False]
    assert rel_2(g, g_ref) < 1e-5
    assert rel_2(grads[True], g) < 1e-6
    fd = np.array([r[1] for r in out])
    gp = np.array([bl.inner_l2(g, r[2]) for r in out])
    rms = float(np.sqrt(np.mean(fd ** 2)))
    gaps = np.abs(fd - gp) / rms
    corr = float(np.corrcoef(fd, gp)[0, 1])
    mib = {k: (a / 2**20, b / 2**20) for k, (a, b) in footprint.items()}
    print(f"96^3 Nt=16: context MiB (held, measured) kept {mib[False]}, recompute {mib[True]}; "
          f"FD gap / rms(fd): median {np.median(gaps):.3f} max {gaps.max():.3f}; corr {corr:.4f}")
    assert footprint[True][0] < footprint[False][0]
    assert corr > 0.95
    assert gaps.max() < 0.5


def test_exact_autograd_differentiation_check_96cubed():
    """The 96^3 brain configuration (band 24^3, Nt = 16) through the exact
    discrete adjoint backward, in FP64 on the GPU: against central differences of
    the FP64 oracle forward along 20 seeded directions with step 1e-6 (the
    oracle's forward is the same discrete map, so the differences converge to
    this gradient; at this step the foot points' cell crossings inside the
    stencil are negligible).  Each directional derivative within 1e-4 of the
    differences, relative to their rms."""
    import os
    import torch
    name = "3d_96_brain"
    kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[name]
    seeds = list(range(2000, 2020))
    pool = spawn_pool(min(len(seeds), os.cpu_count() or 1))   # before any oracle work here
    try:
        fd_async = pool.map_async(fd_data_term, [(name, s_, 1e-6) for s_ in seeds])
        P, v0, _, _ = _fd_problem(name)
        ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp64")
        ctx.set_images(torch_dev(P.I0, "fp64"), torch_dev(P.I1, "fp64"))
        v = torch_dev(v0, "fp64").requires_grad_(True)
        m1 = shoot_transport(ctx, v, adjoint="exact")
        I1d = torch_dev(P.I1, "fp64")
        (((m1 - I1d) ** 2).mean() / SIGMA ** 2).backward()
        g = host(v.grad)
        ctx.close()
        out = fd_async.get(timeout=3600)
    finally:
        pool.terminate()
        pool.join()
    fd = np.array([r[1] for r in out])
    gp = np.array([bl.inner_l2(g, r[2]) for r in out])
    rms = float(np.sqrt(np.mean(fd ** 2)))
    gaps = np.abs(fd - gp) / rms
    print(f"96^3 Nt=16 exact adjoint (FP64): FD gap / rms(fd) median {np.median(gaps):.2e} max {gaps.max():.2e}")
    assert gaps.max() < 1e-4
