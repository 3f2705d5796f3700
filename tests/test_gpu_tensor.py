"""The tcgen05 (3xTF32) form of the image-grid band-to-grid transform against the
FP64 oracle, and end to end inside the gradient and Hessian-vector product."""

import numpy as np
import pytest

from oracle import bl
from paper_1807_11560_gb300 import Context, inputs

from helpers import ALPHA, S, SIGMA, host, problem, quantise, rel_2, rel_V, torch_dev

pytestmark = pytest.mark.gpu

# (grid, band): K1 padding (10 -> 16), one and two 128-row M tiles, ragged N tiles
SHAPES = [((64, 64, 64), (16, 16, 16)), ((100, 36, 20), (10, 8, 6)), ((200, 24, 26), (24, 8, 8)),
          ((160, 192, 160), (32, 32, 32)), ((48, 40), (16, 12))]


@pytest.mark.parametrize("Ns,Ks", SHAPES)
def test_tensor_core_iota_matches_oracle(Ns, Ks):
    import torch
    d = len(Ns)
    a = quantise(inputs.random_bl(Ks, d, 3, 2.0, Ns), "fp32")
    ref = bl.iota(a, Ns)
    outs = []
    for tc in (True, False):
        ctx = Context(Ns, Ks, ALPHA, S, SIGMA, 2, precision="fp32", tensor_cores=tc)
        out = torch.empty((d,) + Ns, device="cuda", dtype=torch.float32)
        ctx.iota(torch_dev(a, "fp32"), d, out)
        outs.append(host(out))
        ctx.close()
    err_tc, err_simt = rel_2(outs[0], ref), rel_2(outs[1], ref)
    assert err_tc < 4e-6, (err_tc, err_simt)


def test_tensor_core_gradient_and_hessvec():
    kind, Ns, Ks, seed, Nt = "ellipsoids", (40, 36, 34), (12, 10, 8), 41, 4
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, "fp32", tensor_cores=True)
    import torch
    lin = P.gradient(v0)
    g = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
    E = ctx.gradient(torch_dev(v0, "fp32"), g)
    Hp = torch.empty_like(g)
    ctx.hessvec(torch_dev(p, "fp32"), Hp)
    assert abs(E - lin.E) / lin.E < 1e-6
    assert rel_V(host(g), lin.g, Ks) < 1e-5
    assert rel_V(host(Hp), P.hessvec(lin, p), Ks) < 1e-5


@pytest.mark.parametrize("Ns,Ks", [((64, 64, 64), (32, 32, 32)), ((56, 48, 40), (24, 16, 24))])
def test_tensor_core_bracket_iota_ab(Ns, Ks):
    """tensor_cores=True also runs iota stages A+B of the padded-grid bracket
    evaluations on tcgen05 (per-evaluation launches: persistent sweeps off):
    gradient and Hessian-vector product against the FP64 oracle at 1e-5."""
    import torch
    Nt, seed = 2, 1812
    I0, I1 = inputs.make_pair("brain", Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, 3, seed + 2, 1.0, Ns), "fp32")
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", tensor_cores=True, persistent=False)
    ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
    g = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
    E = ctx.gradient(torch_dev(v0, "fp32"), g)
    Hp = torch.empty_like(g)
    ctx.hessvec(torch_dev(p, "fp32"), Hp)
    g, Hp = host(g), host(Hp)
    ctx.close()
    from oracle import objective
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    lin = P.gradient(v0)
    assert abs(E - lin.E) / lin.E < 1e-6
    assert rel_V(g, lin.g, Ks) < 1e-5
    assert rel_V(Hp, P.hessvec(lin, p), Ks) < 1e-5


# the two operand splits of the tensor-core transforms against the FP64 oracle
# and against each other: the image-grid band-to-grid stage (2^21 voxels, and a
# ragged 100 x 36 x 20 grid) and the whole gradient / Gauss-Newton product
@pytest.mark.parametrize("Ns,Ks", [((128, 128, 128), (16, 16, 16)), ((100, 36, 20), (10, 8, 6)),
                                   ((160, 192, 160), (32, 32, 32))])
def test_bf16x3_and_3xtf32_iota_match_oracle(Ns, Ks):
    import torch
    d = len(Ns)
    a = quantise(inputs.random_bl(Ks, d, 3, 2.0, Ns), "fp32")
    ref = bl.iota(a, Ns)
    errs = {}
    for prec in ("3xtf32", "bf16x3", "fp32"):
        with Context(Ns, Ks, ALPHA, S, SIGMA, 2, precision=prec,
                     tensor_cores=False if prec == "fp32" else "auto") as ctx:
            out = torch.empty((d,) + Ns, device="cuda", dtype=torch.float32)
            ctx.iota(torch_dev(a, "fp32"), d, out)
            errs[prec] = rel_2(host(out), ref)
    print(f"{Ns} iota rel. err: " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["3xtf32"] < 4e-6 and errs["bf16x3"] < 4e-6


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3"])
def test_split_modes_gradient_and_hessvec(prec):
    kind, Ns, Ks, seed, Nt = "ellipsoids", (64, 56, 48), (16, 16, 16), 43, 3
    import torch
    I0, I1 = inputs.make_pair(kind, Ns, seed, max_disp=2.0)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, 3, seed + 2, 1.0, Ns), "fp32")
    from oracle import objective
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    lin = P.gradient(v0)
    with Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision=prec) as ctx:
        ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
        g = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
        E = ctx.gradient(torch_dev(v0, "fp32"), g)
        Hp = torch.empty_like(g)
        ctx.hessvec(torch_dev(p, "fp32"), Hp)
        g, Hp = host(g), host(Hp)
    assert abs(E - lin.E) / lin.E < 1e-6
    assert rel_V(g, lin.g, Ks) < 1e-5
    assert rel_V(Hp, P.hessvec(lin, p), Ks) < 1e-5
