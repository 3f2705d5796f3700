"""Full-Newton Hessian-vector product on the GPU (lddmm_hessvec_newton) against
the FP64 oracle's hessvec_newton, on both sweep paths; equal to the Gauss-Newton
product when the residual vanishes; GN-Krylov with the Newton Hessian; state
errors."""

import numpy as np
import pytest

from oracle import objective
from paper_1807_11560_gb300 import Context, LddmmError, inputs

from helpers import ALPHA, S, SIGMA, host, problem, quantise, rel_V, torch_dev

pytestmark = pytest.mark.gpu

CASES = [("blobs", (20, 18), (8, 6), 5, 3),
         ("ellipsoids", (24, 20, 18), (8, 6, 6), 6, 4),
         ("ellipsoids", (40, 36, 34), (12, 10, 8), 7, 5)]
TOL = {"fp64": 1e-9, "fp32": 1e-5}


def _cplx(precision, shape):
    import torch
    return torch.empty(shape, device="cuda", dtype=torch.complex128 if precision == "fp64" else torch.complex64)


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_newton_hessvec_matches_oracle(case, precision, persistent):
    kind, Ns, Ks, seed, Nt = case
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, precision, persistent=persistent)
    d = len(Ns)
    g = _cplx(precision, (d,) + Ks)
    ctx.gradient(torch_dev(v0, precision), g)
    Hn = _cplx(precision, (d,) + Ks)
    ctx.hessvec_newton(torch_dev(p, precision), Hn)
    Hg = _cplx(precision, (d,) + Ks)
    ctx.hessvec(torch_dev(p, precision), Hg)
    ctx.hessvec_newton(torch_dev(p, precision), Hn)     # after a GN product: graphs kept apart
    lin = P.gradient(v0)
    ref = P.hessvec_newton(lin, p)
    assert rel_V(host(Hn), ref, Ks) < TOL[precision]
    assert rel_V(host(Hg), P.hessvec(lin, p), Ks) < TOL[precision]
    ctx.close()


def test_newton_equals_gauss_newton_at_zero_residual():
    import torch
    kind, Ns, Ks, seed, Nt = CASES[1]
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, "fp64")
    m1 = torch.empty(Ns, device="cuda", dtype=torch.float64)
    ctx.transport(torch_dev(v0, "fp64"), m1)
    I0 = inputs.make_pair(kind, Ns, seed, max_disp=2.0)[0]
    ctx.set_images(torch_dev(I0, "fp64"), m1)            # target = m(1)[v0]: lambda(1) = 0
    g = _cplx("fp64", (3,) + Ks)
    ctx.gradient(torch_dev(v0, "fp64"), g)
    Hn, Hg = _cplx("fp64", (3,) + Ks), _cplx("fp64", (3,) + Ks)
    ctx.hessvec_newton(torch_dev(p, "fp64"), Hn)
    ctx.hessvec(torch_dev(p, "fp64"), Hg)
    assert rel_V(host(Hn), host(Hg), Ks) < 1e-13
    ctx.close()


def test_gn_krylov_with_the_newton_hessian_decreases_the_energy():
    kind, Ns, Ks, seed, Nt = CASES[1]
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, "fp32", newton=True)
    v = np.zeros((3,) + Ks, np.complex64)
    rep = ctx.gn_solve(v, 3, 5)
    assert rep["gn_iters"] >= 1 and rep["E_final"] < rep["E_initial"]
    assert all(b <= a for a, b in zip(rep["E"], rep["E"][1:]))
    ctx.close()


def test_newton_needs_the_gradient_sweep():
    kind, Ns, Ks, seed, Nt = CASES[1]
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, "fp32")
    g = _cplx("fp32", (3,) + Ks)
    ctx.exact_gradient(torch_dev(v0, "fp32"), g)        # sets the point, not the (U, W) history
    with pytest.raises(LddmmError) as ei:
        ctx.hessvec_newton(torch_dev(p, "fp32"), _cplx("fp32", (3,) + Ks))
    assert ei.value.code == 4
    ctx.gradient(torch_dev(v0, "fp32"), g)
    ctx.hessvec_newton(torch_dev(p, "fp32"), _cplx("fp32", (3,) + Ks))
    ctx.close()
