"""Degenerate and extreme sizes against the FP64 oracle: the smallest band (two
slots per axis, so only the constant mode survives the Nyquist rule), a band as
large as the grid, the largest K1 (64) with thin other axes, odd grid sizes, a
2D band of 2 x 2, and a single time step.  Energy, gradient (Eq. 50) and GN
Hessian-vector product (Eqs. 56-58) on both sweep paths (persistent and
per-evaluation launches), FP64 and FP32."""

import pytest

from helpers import host, problem, rel_V, torch_dev

pytestmark = pytest.mark.gpu

CASES = [((9, 7, 5), (2, 2, 2), 3), ((12, 10, 8), (12, 10, 8), 2), ((64, 16, 12), (64, 4, 2), 2),
         ((10, 8), (2, 2), 3), ((20, 18, 14), (8, 6, 4), 1)]
TOL = {"fp64": 1e-9, "fp32": 1e-5}


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("Ns,Ks,Nt", CASES)
def test_edge_sizes_match_oracle(Ns, Ks, Nt, precision, persistent):
    import torch
    kind = "blobs" if len(Ns) == 2 else "ellipsoids"
    ctx, P, v0, p = problem(kind, Ns, Ks, 5, Nt, precision, v_disp=1.0, persistent=persistent)
    ct = torch.complex128 if precision == "fp64" else torch.complex64
    d = len(Ns)
    with ctx:
        g = torch.empty((d,) + Ks, device="cuda", dtype=ct)
        E = ctx.gradient(torch_dev(v0, precision), g)
        Hp = torch.empty_like(g)
        ctx.hessvec(torch_dev(p, precision), Hp)
        g, Hp = host(g), host(Hp)
    lin = P.gradient(v0)
    tol = TOL[precision]
    assert abs(E - lin.E) / lin.E < (1e-12 if precision == "fp64" else 1e-6)
    assert rel_V(g, lin.g, Ks) < tol
    assert rel_V(Hp, P.hessvec(lin, p), Ks) < tol
