"""Pins of the oracle's energy, gradient, GN Hessian-vector product and GN-Krylov solve."""

import numpy as np
import pytest

from oracle import bl, objective, sweeps
from paper_1807_11560_gb300 import inputs

ALPHA, S, SIGMA = 0.0025, 2, 0.03


def _direct_pi(f, Ks):
    """Grid -> band as an explicit sum (no FFT), for closed-form checks."""
    Ns = f.shape[1:]
    X = np.meshgrid(*[np.arange(n) / n for n in Ns], indexing="ij")
    out = np.zeros((f.shape[0],) + tuple(Ks), dtype=np.complex128)
    for q in np.ndindex(*Ks):
        if any(K % 2 == 0 and qq == K // 2 for qq, K in zip(q, Ks)):
            continue
        fr = [qq if qq < K / 2 else qq - K for qq, K in zip(q, Ks)]
        ph = np.exp(-2j * np.pi * sum(a * b for a, b in zip(fr, X)))
        for c in range(f.shape[0]):
            out[(c,) + q] = np.sum(f[c] * ph) / np.prod(Ns)
    return out


def _lhat_direct(Ks):
    out = np.empty(Ks)
    for q in np.ndindex(*Ks):
        fr = [qq if qq < K / 2 else qq - K for qq, K in zip(q, Ks)]
        out[q] = (1 + 4 * np.pi ** 2 * ALPHA * sum(x * x for x in fr)) ** S
    return out


def _grad_direct(m):
    """(m[i+1] - m[i-1]) / (2h), element by element."""
    Ns = m.shape
    out = np.zeros((len(Ns),) + Ns)
    for i in np.ndindex(*Ns):
        for j in range(len(Ns)):
            ip = list(i); im = list(i)
            ip[j] = (ip[j] + 1) % Ns[j]; im[j] = (im[j] - 1) % Ns[j]
            out[(j,) + i] = (m[tuple(ip)] - m[tuple(im)]) * Ns[j] / 2.0
    return out


@pytest.fixture(scope="module")
def small2d():
    Ns, Ks = (20, 16), (8, 6)
    I0, I1 = inputs.make_pair("blobs", Ns, 5, max_disp=1.5)
    return objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, 6)


def test_energy_at_zero_and_regulariser(small2d):
    P = small2d
    z = np.zeros((2,) + P.Ks, dtype=np.complex128)
    want = np.mean((P.I0 - P.I1) ** 2) / SIGMA ** 2          # h^d sum = mean on the unit box
    assert abs(P.energy(z) - want) <= 1e-14 * want
    # regulariser alone: sigma -> infinity
    v0 = inputs.random_bl(P.Ks, 2, 3, 1.0, P.Ns)
    Q = objective.Problem(P.I0, P.I1, P.Ks, ALPHA, S, 1e100, 6)
    L = _lhat_direct(P.Ks)
    assert np.isclose(Q.energy(v0), 0.5 * np.sum(L * np.abs(v0) ** 2), rtol=1e-13)


def test_gradient_at_zero_closed_form(small2d):
    """v0 = 0: v_t = 0, m(1) = I0, U constant, W(0) = U(1), so
    g = -(2/sigma^2) K~ pi((I0 - I1) grad_h I0) (Eq. 55 with the text after Eq. 14)."""
    P = small2d
    z = np.zeros((2,) + P.Ks, dtype=np.complex128)
    g = P.gradient(z).g
    want = -(2 / SIGMA ** 2) * _direct_pi((P.I0 - P.I1)[None] * _grad_direct(P.I0), P.Ks) / _lhat_direct(P.Ks)
    np.testing.assert_allclose(g, want, atol=1e-12 * np.abs(want).max())


def test_gradient_matches_central_differences_at_zero(small2d):
    """At v0 = 0 the one-sided kinks of multilinear interpolation average to the central
    difference, so the FD of E approaches <g, p>_V at first order in eps."""
    P = small2d
    z = np.zeros((2,) + P.Ks, dtype=np.complex128)
    g = P.gradient(z).g
    for seed in (11, 12):
        p = inputs.random_bl(P.Ks, 2, seed, 1.0, P.Ns)
        ref = P.inner_V(g, p)
        gaps = []
        for eps in (1e-3, 1e-4, 1e-5):
            fd = (P.energy(eps * p) - P.energy(-eps * p)) / (2 * eps)
            gaps.append(abs(fd - ref) / abs(ref))
        assert gaps[2] < 1e-5, gaps
        assert 5 < gaps[0] / gaps[1] < 20 and 5 < gaps[1] / gaps[2] < 20, gaps


def test_hessvec_at_zero_closed_form(small2d):
    """v0 = 0: dv_t = p, dm(1) = -grad I0 . iota(p), so
    H p = p + (2/sigma^2) K~ pi(grad I0 (grad I0 . iota(p)))."""
    P = small2d
    z = np.zeros((2,) + P.Ks, dtype=np.complex128)
    lin = P.gradient(z)
    p = inputs.random_bl(P.Ks, 2, 7, 1.0, P.Ns)
    gI = _grad_direct(P.I0)
    want = p + (2 / SIGMA ** 2) * _direct_pi(gI * np.sum(gI * bl.iota(p, P.Ns), axis=0)[None], P.Ks) \
        / _lhat_direct(P.Ks)
    np.testing.assert_allclose(P.hessvec(lin, p), want, atol=1e-12 * np.abs(want).max())


@pytest.fixture(scope="module")
def lin3d():
    Ns, Ks = (16, 12, 12), (6, 6, 4)
    I0, I1 = inputs.make_pair("ellipsoids", Ns, 9, max_disp=1.5)
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, 4)
    v0 = inputs.random_bl(Ks, 3, 31, 2.0, Ns)
    return P, P.gradient(v0)


def test_J_form_hessian_is_symmetric_positive_definite(lin3d):
    P, lin = lin3d
    xs = [inputs.random_bl(P.Ks, 3, s_, 1.0, P.Ns) for s_ in (40, 41, 42)]
    Hx = [P.hessvec_J(lin, x) for x in xs]
    for i in range(3):
        for j in range(i + 1, 3):
            a, b = P.inner_V(Hx[i], xs[j]), P.inner_V(xs[i], Hx[j])
            assert abs(a - b) <= 1e-12 * np.sqrt(P.inner_V(Hx[i], Hx[i]) * P.inner_V(xs[j], xs[j]))
        assert P.inner_V(Hx[i], xs[i]) >= P.inner_V(xs[i], xs[i]) * (1 - 1e-12)


def test_paper_form_hessian_close_to_J_form_and_linear(lin3d):
    """The GN product transports dm on the full grid (Eq. 31) and the J form uses the BL
    Jacobi field; they discretise the same operator, and both are linear in p."""
    P, lin = lin3d
    x = inputs.random_bl(P.Ks, 3, 50, 1.0, P.Ns)
    y = inputs.random_bl(P.Ks, 3, 51, 1.0, P.Ns)
    hx, hy = P.hessvec(lin, x), P.hessvec(lin, y)
    hj = P.hessvec_J(lin, x)
    gap = np.sqrt(P.inner_V(hx - hj, hx - hj) / P.inner_V(hj, hj))
    # about 0.06 on this coarse grid; a sign error in the ad term of the Jacobi
    # equation J' = dv + ad_v J raises it above 0.25
    assert gap < 0.1, gap
    h = P.hessvec(lin, 2.0 * x - 3.0 * y)
    np.testing.assert_allclose(h, 2.0 * hx - 3.0 * hy, atol=1e-12 * np.abs(h).max())
    assert P.inner_V(hx, x) > P.inner_V(x, x)


def test_pcg_solves_the_linear_system(lin3d):
    """CG in the V inner product converges on the exactly symmetric J-form operator.
    (The paper-form product is symmetric only up to the discretisation gap, so CG on
    it stalls near that level; the solver uses few iterations per GN step.)"""
    Ns, Ks = (12, 12), (4, 4)          # 18 real unknowns: CG ends within ~18 steps
    I0, I1 = inputs.make_pair("blobs", Ns, 4, max_disp=1.0)
    Q = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, 3)
    lq = Q.gradient(inputs.random_bl(Ks, 2, 5, 1.0, Ns))
    b = -lq.g
    x, its = Q.pcg(lq, b, 40, tol=1e-11, op=Q.hessvec_J)
    r = Q.hessvec_J(lq, x) - b
    assert its <= 30
    assert np.sqrt(Q.inner_V(r, r) / Q.inner_V(b, b)) < 1e-8
    P, lin = lin3d
    b = -lin.g
    # a single iteration is the exact line minimiser along b
    x1, _ = P.pcg(lin, b, 1)
    hb = P.hessvec(lin, b)
    np.testing.assert_allclose(x1, b * P.inner_V(b, b) / P.inner_V(b, hb), atol=1e-14 * np.abs(x1).max())


def test_gn_solve_decreases_energy_and_mismatch():
    Ns, Ks = (24, 24), (8, 8)
    I0, I1 = inputs.make_pair("blobs", Ns, 3, max_disp=2.0)
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, 5)
    z = np.zeros((2,) + Ks, dtype=np.complex128)
    v, rep = P.gn_solve(z, 4, 5)
    E = rep["E"] + [rep["E_final"]]
    assert all(E[i + 1] < E[i] for i in range(len(E) - 1)), E
    assert not rep["ls_failed"]
    m1 = P.forward(v)[3][-1]
    assert P.mse_rel(m1) < 0.5 * P.mse_rel(I0)
