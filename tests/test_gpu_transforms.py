"""GPU parity of the band-limited maps and brackets (Section 3.1) against the oracle."""

import numpy as np
import pytest

from oracle import bl
from paper_1807_11560_gb300 import Context, inputs

from helpers import ALPHA, S, SIGMA, host, quantise, rel_2, torch_dev

pytestmark = pytest.mark.gpu

SHAPES = [((20, 18, 14), (8, 6, 4)), ((24, 20), (8, 8)), ((33, 17), (10, 6)),
          ((64, 64, 64), (16, 16, 16))]
TOL = {"fp64": 1e-11, "fp32": 2e-6}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("Ns,Ks", SHAPES)
def test_iota_pi_match_oracle(Ns, Ks, precision):
    import torch
    d = len(Ns)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, 2, precision=precision)
    a = quantise(inputs.random_bl(Ks, d, 3, 2.0, Ns), precision)
    out = torch.empty((d,) + Ns, device="cuda", dtype=torch.float64 if precision == "fp64" else torch.float32)
    ctx.iota(torch_dev(a, precision), d, out)
    ref = bl.iota(a, Ns)
    assert rel_2(host(out), ref) < TOL[precision]
    rng = np.random.default_rng(5)
    f = quantise(rng.normal(size=(d,) + Ns), precision)
    outk = torch.empty((d,) + Ks, device="cuda", dtype=torch.complex128 if precision == "fp64" else torch.complex64)
    ctx.pi(torch_dev(f, precision), d, outk)
    refk = bl.pi(f, Ks)
    assert rel_2(host(outk), refk) < TOL[precision]
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_iota_uses_the_hermitian_part_of_any_input(precision):
    import torch
    Ns, Ks = (16, 12, 10), (8, 6, 4)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, 2, precision=precision)
    rng = np.random.default_rng(1)
    a = quantise(rng.normal(size=(3,) + Ks) + 1j * rng.normal(size=(3,) + Ks), precision)
    out = torch.empty((3,) + Ns, device="cuda", dtype=torch.float64 if precision == "fp64" else torch.float32)
    ctx.iota(torch_dev(a, precision), 3, out)
    assert rel_2(host(out), bl.iota(a, Ns)) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("Ns,Ks", [((20, 18, 14), (8, 6, 4)), ((24, 20), (8, 8)), ((64, 64, 64), (16, 16, 16))])
def test_brackets_match_oracle(Ns, Ks, precision):
    import torch
    d = len(Ns)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, 2, precision=precision)
    v = quantise(inputs.random_bl(Ks, d, 7, 3.0, Ns), precision)
    u = quantise(inputs.random_bl(Ks, d, 8, 3.0, Ns), precision)
    ct = torch.complex128 if precision == "fp64" else torch.complex64
    out = torch.empty((d,) + Ks, device="cuda", dtype=ct)
    ctx.ad_dagger(torch_dev(v, precision), torch_dev(u, precision), out)
    assert rel_2(host(out), bl.ad_dagger(v, u, ALPHA, S)) < 10 * TOL[precision]
    ctx.ad(torch_dev(v, precision), torch_dev(u, precision), out)
    assert rel_2(host(out), bl.ad(v, u)) < 10 * TOL[precision]


def test_host_and_device_pointers_agree():
    import torch
    Ns, Ks = (20, 18, 14), (8, 6, 4)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, 2, precision="fp32")
    a = inputs.random_bl(Ks, 3, 3, 2.0, Ns).astype(np.complex64)
    out_h = np.empty((3,) + Ns, dtype=np.float32)
    ctx.iota(a, 3, out_h)
    out_d = torch.empty((3,) + Ns, device="cuda", dtype=torch.float32)
    ctx.iota(torch.as_tensor(a).cuda(), 3, out_d)
    np.testing.assert_array_equal(out_h, out_d.cpu().numpy())
