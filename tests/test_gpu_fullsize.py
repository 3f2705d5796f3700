"""GPU parity at the benchmark sizes, in the configuration bench.py times (FP32,
CUDA-graph replay of the Hessian-vector product), against the FP64 oracle on the
same seeded phantoms.  Spec tolerances: 1e-5 relative (V norm) on the
gradient and the Hessian-vector product, 1e-6 on E."""

import numpy as np
import pytest

from oracle import objective
from paper_1807_11560_gb300 import Context, inputs

from helpers import ALPHA, S, SIGMA, host, quantise, rel_2, rel_V, torch_dev

pytestmark = pytest.mark.gpu


def _run(name, v_disp):
    import torch
    kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[name]
    d = len(Ns)
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, d, seed + 1, v_disp, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, d, seed + 2, 1.0, Ns), "fp32")
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32")
    ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
    g = torch.empty((d,) + Ks, device="cuda", dtype=torch.complex64)
    E = ctx.gradient(torch_dev(v0, "fp32"), g)
    Hp = torch.empty_like(g)
    ctx.hessvec(torch_dev(p, "fp32"), Hp)
    ctx.hessvec(torch_dev(p, "fp32"), Hp)            # replayed graph
    m1 = torch.empty(Ns, device="cuda", dtype=torch.float32)
    ctx.transport(torch_dev(v0, "fp32"), m1)
    out = (E, host(g), host(Hp), host(m1))
    ctx.close()
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    lin = P.gradient(v0)
    return out, (lin.E, lin.g, P.hessvec(lin, p), lin.ms[-1]), Ks


def test_bench_workload_64cubed():
    (E, g, Hp, m1), (Er, gr, Hr, mr), Ks = _run("3d_64_ellipsoids", 2.0)
    assert abs(E - Er) / Er < 1e-6
    assert rel_V(g, gr, Ks) < 1e-5
    assert rel_V(Hp, Hr, Ks) < 1e-5
    assert rel_2(m1, mr) < 1e-5


def test_brain_workload_160x192x160():
    (E, g, Hp, m1), (Er, gr, Hr, mr), Ks = _run("3d_160x192x160_brain", 3.0)
    assert abs(E - Er) / Er < 1e-6
    assert rel_V(g, gr, Ks) < 1e-5
    assert rel_V(Hp, Hr, Ks) < 1e-5
    assert rel_2(m1, mr) < 1e-5


def test_differentiation_workload_96cubed_nt16():
    (E, g, Hp, m1), (Er, gr, Hr, mr), Ks = _run("3d_96_brain", 2.0)
    assert abs(E - Er) / Er < 1e-6
    assert rel_V(g, gr, Ks) < 1e-5
    assert rel_V(Hp, Hr, Ks) < 1e-5
    assert rel_2(m1, mr) < 1e-5


@pytest.mark.parametrize("Ks", [(64, 48, 56), (48, 48, 48)])
def test_large_bands(Ks):
    """Bands of the band-size sweep beyond the configs (K up to 64, anisotropic):
    gradient and Hessian-vector product against the FP64 oracle at the 1e-5 target
    (Nt = 2 keeps the oracle's padded-grid products affordable)."""
    import torch
    Ns, Nt, seed = (64, 64, 64), 2, 1811
    I0, I1 = inputs.make_pair("brain", Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, 3, seed + 2, 1.0, Ns), "fp32")
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32")
    ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
    g = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
    E = ctx.gradient(torch_dev(v0, "fp32"), g)
    Hp = torch.empty_like(g)
    ctx.hessvec(torch_dev(p, "fp32"), Hp)
    g, Hp = host(g), host(Hp)
    ctx.close()
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    lin = P.gradient(v0)
    assert abs(E - lin.E) / lin.E < 1e-6
    assert rel_V(g, lin.g, Ks) < 1e-5
    assert rel_V(Hp, P.hessvec(lin, p), Ks) < 1e-5
