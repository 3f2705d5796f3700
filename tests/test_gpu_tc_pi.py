"""The tcgen05 (3xTF32) forms of the bracket evaluation's middle phase (C,
products, C') and of pi stages B'+A' with the bracket epilogue (per-evaluation
launches on the padded grid) against the FP64 oracle:
ad~^dagger and ad~ alone (Eqs. 48-49), the Heun shoot (its epilogues update
band vectors in place), and the gradient and Gauss-Newton product at shapes
with one and two 128-row passes of the first stage, ragged K and ragged tiles.
The SIMT kernel runs where the tensor-core tiles do not apply (padded sizes
not multiples of 4); those shapes are checked too."""

import numpy as np
import pytest

from oracle import bl, objective, sweeps
from paper_1807_11560_gb300 import Context, inputs

from helpers import ALPHA, S, SIGMA, host, quantise, rel_V, torch_dev

pytestmark = pytest.mark.gpu

# padded grids (24, 24, 24) / (36, 24, 36) / (48, 48, 48) / (12, 60, 24) /
# (48, 36, 48) / (12, 12, 9): the tensor-core pi where M2 is a multiple of 8, the
# tensor-core middle phase where M1 is a multiple of 16 and K1/2 of 4 (48^3 and
# 48 x 36 x 48), the SIMT kernels elsewhere
SHAPES = [((32, 32, 32), (16, 16, 16)), ((56, 48, 40), (24, 16, 24)), ((64, 64, 64), (32, 32, 32)),
          ((20, 44, 30), (8, 40, 16)), ((24, 20, 14), (8, 8, 6)), ((56, 40, 52), (32, 24, 32))]


def _ctx(Ns, Ks, Nt=2):
    return Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", tensor_cores=True, persistent=False)


@pytest.mark.parametrize("Ns,Ks", SHAPES)
def test_tc_pi_brackets_match_oracle(Ns, Ks):
    import torch
    v = quantise(inputs.random_bl(Ks, 3, 7, 3.0, Ns), "fp32")
    u = quantise(inputs.random_bl(Ks, 3, 8, 3.0, Ns), "fp32")
    with _ctx(Ns, Ks) as ctx:
        out = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
        ctx.ad_dagger(torch_dev(v, "fp32"), torch_dev(u, "fp32"), out)
        assert rel_V(host(out), bl.ad_dagger(v, u, ALPHA, S), Ks) < 2e-5
        ctx.ad(torch_dev(v, "fp32"), torch_dev(u, "fp32"), out)
        assert rel_V(host(out), bl.ad(v, u), Ks) < 2e-5


@pytest.mark.parametrize("Ns,Ks", SHAPES[:3])
def test_tc_pi_shoot_matches_oracle(Ns, Ks):
    import torch
    Nt = 4
    v0 = quantise(inputs.random_bl(Ks, 3, 9, 2.0, Ns), "fp32")
    with _ctx(Ns, Ks, Nt) as ctx:
        out = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
        ctx.shoot(torch_dev(v0, "fp32"), out)
        vs, _ = sweeps.shoot(v0, Nt, ALPHA, S)
        assert rel_V(host(out), vs[-1], Ks) < 1e-5


@pytest.mark.parametrize("Ns,Ks", [SHAPES[1], SHAPES[3], SHAPES[5]])
def test_tc_pi_gradient_and_hessvec(Ns, Ks):
    import torch
    Nt, seed = 3, 1813
    I0, I1 = inputs.make_pair("brain", Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, 3, seed + 2, 1.0, Ns), "fp32")
    with _ctx(Ns, Ks, Nt) as ctx:
        ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
        g = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
        E = ctx.gradient(torch_dev(v0, "fp32"), g)
        Hp = torch.empty_like(g)
        ctx.hessvec(torch_dev(p, "fp32"), Hp)
        g, Hp = host(g), host(Hp)
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    lin = P.gradient(v0)
    assert abs(E - lin.E) / lin.E < 1e-6
    assert rel_V(g, lin.g, Ks) < 1e-5
    assert rel_V(Hp, P.hessvec(lin, p), Ks) < 1e-5
