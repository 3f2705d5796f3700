"""Pins of the oracle's exact discrete-adjoint gradient (the PDE-LDDMM route of
Section 2.5 in discrete form: state transport reversed step by step, Eqs. 12-14,
then the transpose of the Heun shoot).  Each piece is pinned by what the
mathematics fixes: transposes by inner-product identities, derivatives by
central differences, and the whole gradient by central differences of the
discretised energy (exact up to O(eps^2): this gradient is the derivative of the
discrete energy, unlike the paper-form Jacobi gradient)."""

import numpy as np
import pytest

from oracle import bl, objective, sweeps
from paper_1807_11560_gb300 import inputs

ALPHA, S, SIGMA = 0.0025, 2, 0.03
RNG = np.random.default_rng(2024)


@pytest.mark.parametrize("Ns", [(9, 7), (6, 5, 4)])
def test_interp_adjoint_is_the_transpose(Ns):
    d = len(Ns)
    f = RNG.normal(size=Ns)
    g = RNG.normal(size=Ns)
    xi = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in Ns], indexing="ij"))
    xi = xi + RNG.uniform(-3.0, 3.0, size=xi.shape)
    lhs = float(np.sum(sweeps.interp(f, xi) * g))
    rhs = float(np.sum(f * sweeps.interp_adjoint(g, xi, Ns)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("Ns", [(9, 7), (6, 5, 4)])
def test_interp_gradient_matches_central_differences(Ns):
    d = len(Ns)
    f = RNG.normal(size=Ns)
    xi = RNG.uniform(0.1, 0.9, size=(d, 5)) + RNG.integers(0, 4, size=(d, 5))
    gr = sweeps.interp_gradient(f, xi)
    eps = 1e-6
    for a in range(d):
        e = np.zeros_like(xi)
        e[a] = eps
        fd = (sweeps.interp(f, xi + e) - sweeps.interp(f, xi - e)) / (2 * eps)
        np.testing.assert_allclose(gr[a], fd, rtol=1e-7, atol=1e-8)


def test_transpose_shoot_is_the_transpose_of_the_tangent_shoot():
    """sum_n <dv_n, s_n>_V = <p, W_0>_V for the Heun tangent dv of the shoot."""
    Ks, Nt = (6, 6, 4), 4
    v0 = inputs.random_bl(Ks, 3, 31, 1.5, (12, 12, 10))
    vs, vstar = sweeps.shoot(v0, Nt, ALPHA, S)
    p = inputs.random_bl(Ks, 3, 32, 1.0, (12, 12, 10))
    dvs = sweeps.tangent_shoot(vs, vstar, p, ALPHA, S)
    src = [inputs.random_bl(Ks, 3, 40 + n, 1.0, (12, 12, 10)) for n in range(Nt + 1)]
    W0 = sweeps.transpose_shoot(vs, vstar, src, ALPHA, S)
    lhs = sum(bl.inner_V(dvs[n], src[n], ALPHA, S) for n in range(Nt + 1))
    rhs = bl.inner_V(p, W0, ALPHA, S)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


@pytest.mark.parametrize("Ns", [(12, 10), (8, 7, 6)])
def test_transport_adjoint_matches_central_differences(Ns):
    d, Nt, dt = len(Ns), 3, 1.0 / 3
    I0 = inputs.make_pair("blobs" if d == 2 else "ellipsoids", Ns, 3, max_disp=1.0)[0]
    vg = [0.02 * RNG.normal(size=(d,) + Ns) for _ in range(Nt + 1)]
    dvg = [0.02 * RNG.normal(size=(d,) + Ns) for _ in range(Nt + 1)]
    lam = RNG.normal(size=Ns)
    ms, _ = sweeps.transport(I0, vg, dt)
    G = sweeps.transport_adjoint(ms, vg, lam, dt)
    eps = 1e-6

    def L(e):
        return float(np.sum(lam * sweeps.transport(I0, [a + e * b for a, b in zip(vg, dvg)], dt)[0][-1]))

    fd = (L(eps) - L(-eps)) / (2 * eps)
    ad = sum(float(np.sum(g * b)) for g, b in zip(G, dvg))
    assert abs(fd - ad) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("kind,Ns,Ks", [("blobs", (20, 18), (8, 6)), ("ellipsoids", (14, 12, 10), (6, 6, 4))])
def test_exact_gradient_matches_central_differences_of_the_energy(kind, Ns, Ks):
    I0, I1 = inputs.make_pair(kind, Ns, 5, max_disp=2.0)
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, 3)
    d = len(Ns)
    v0 = inputs.random_bl(Ks, d, 6, 1.5, Ns)
    E, g = P.exact_gradient(v0)
    assert abs(E - P.energy(v0)) <= 1e-13 * E
    for seed in (7, 8, 9):
        p = inputs.random_bl(Ks, d, seed, 1.0, Ns)
        eps = 1e-5
        fd = (P.energy(v0 + eps * p) - P.energy(v0 - eps * p)) / (2 * eps)
        assert abs(fd - P.inner_V(g, p)) <= 1e-7 * abs(fd), seed
