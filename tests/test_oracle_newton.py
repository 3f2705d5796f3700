"""Pins of the oracle's full-Newton Hessian-vector product (Eqs. 56-58 without the
Gauss-Newton drop), taken as the derivative of the paper-form gradient
g = v0 + W(0)[v; U~(1)].  Its two new pieces are pinned separately by central
differences of the functions they differentiate, both smooth (polynomial in
their arguments), so the differences are exact to O(eps^2):
  * the band sweep: d/dv0 of W(0)[shoot(v0); U1 fixed] = newton_backward with
    dU1 = 0 (the ad~^dagger_dv U, ad~^dagger_w dv, -ad~_dv w terms and the stage
    bookkeeping);
  * the terminal value: d/dm1 of K~ pi(lambda(1) grad m(1)).
"""

import numpy as np
import pytest

from oracle import bl, objective, sweeps
from paper_1807_11560_gb300 import inputs

ALPHA, S, SIGMA = 0.0025, 2, 0.03


def test_newton_backward_is_the_derivative_of_the_backward_sweep():
    Ks, Ns, Nt = (6, 6, 4), (12, 12, 10), 4
    v0 = inputs.random_bl(Ks, 3, 51, 1.5, Ns)
    p = inputs.random_bl(Ks, 3, 52, 1.0, Ns)
    U1 = inputs.random_bl(Ks, 3, 53, 1.0, Ns)

    def W0(v):
        vs, vstar = sweeps.shoot(v, Nt, ALPHA, S)
        return sweeps.adjoint_jacobi_backward(vs, vstar, U1, ALPHA, S)

    eps = 1e-5
    fd = (W0(v0 + eps * p) - W0(v0 - eps * p)) / (2 * eps)
    vs, vstar = sweeps.shoot(v0, Nt, ALPHA, S)
    dvs, dstar = sweeps.tangent_shoot_stages(vs, vstar, p, ALPHA, S)
    _, zs, zt = sweeps.adjoint_jacobi_backward_stages(vs, vstar, U1, ALPHA, S)
    dW = sweeps.newton_backward(vs, vstar, dvs, dstar, zs, zt, np.zeros_like(U1), ALPHA, S)
    rel = np.sqrt(bl.inner_V(dW - fd, dW - fd, ALPHA, S) / bl.inner_V(fd, fd, ALPHA, S))
    assert rel < 1e-8


def test_stage_histories_reproduce_the_plain_sweeps():
    Ks, Ns, Nt = (6, 4, 4), (10, 8, 8), 3
    v0 = inputs.random_bl(Ks, 3, 54, 1.5, Ns)
    p = inputs.random_bl(Ks, 3, 55, 1.0, Ns)
    U1 = inputs.random_bl(Ks, 3, 56, 1.0, Ns)
    vs, vstar = sweeps.shoot(v0, Nt, ALPHA, S)
    dvs, dstar = sweeps.tangent_shoot_stages(vs, vstar, p, ALPHA, S)
    for a, b in zip(dvs, sweeps.tangent_shoot(vs, vstar, p, ALPHA, S)):
        np.testing.assert_array_equal(a, b)
    W0, zs, zt = sweeps.adjoint_jacobi_backward_stages(vs, vstar, U1, ALPHA, S)
    np.testing.assert_array_equal(W0, sweeps.adjoint_jacobi_backward(vs, vstar, U1, ALPHA, S))
    np.testing.assert_array_equal(zs[Nt][0], U1)
    np.testing.assert_array_equal(zs[0][1], W0)


def test_newton_terminal_is_the_derivative_of_the_terminal_value():
    Ns, Ks = (16, 14, 12), (8, 6, 6)
    I0, I1 = inputs.make_pair("ellipsoids", Ns, 57, max_disp=2.0)
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, 2)
    rng = np.random.default_rng(58)
    m1 = I0 + 0.05 * rng.normal(size=Ns)
    dm = rng.normal(size=Ns)

    def U(m):
        return P.terminal_U(m, -(2.0 / SIGMA ** 2) * (m - I1))

    eps = 1e-3                                   # U is quadratic in m: the difference is exact
    fd = (U(m1 + eps * dm) - U(m1 - eps * dm)) / (2 * eps)
    dU = P.terminal_U_newton(m1, dm)
    np.testing.assert_allclose(dU, fd, rtol=1e-9, atol=1e-9 * np.abs(fd).max())


def test_newton_product_is_gauss_newton_plus_the_dropped_terms_and_linear():
    Ns, Ks, Nt = (16, 14, 12), (6, 6, 4), 3
    I0, I1 = inputs.make_pair("ellipsoids", Ns, 59, max_disp=2.0)
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    v0 = inputs.random_bl(Ks, 3, 60, 1.5, Ns)
    lin = P.gradient(v0)
    x = inputs.random_bl(Ks, 3, 61, 1.0, Ns)
    y = inputs.random_bl(Ks, 3, 62, 1.0, Ns)
    Hx, Hy = P.hessvec_newton(lin, x), P.hessvec_newton(lin, y)
    Hxy = P.hessvec_newton(lin, 2.0 * x - 3.0 * y)
    np.testing.assert_allclose(Hxy, 2.0 * Hx - 3.0 * Hy, rtol=1e-10, atol=1e-10 * np.abs(Hxy).max())
    # the dropped terms matter away from v0 = 0 but the Gauss-Newton part dominates
    Gx = P.hessvec(lin, x)
    gap = np.sqrt(P.inner_V(Hx - Gx, Hx - Gx) / P.inner_V(Gx, Gx))
    assert 1e-6 < gap < 1.0


def test_newton_equals_gauss_newton_when_the_residual_vanishes():
    """With I1 = m(1)[v0] the residual lambda(1) is zero, so U and W vanish along
    the gradient sweep and every dropped term is zero: H_Newton = H_GN exactly."""
    Ns, Ks, Nt = (14, 12, 10), (6, 4, 4), 3
    I0 = inputs.make_pair("ellipsoids", Ns, 63, max_disp=2.0)[0]
    P0 = objective.Problem(I0, I0, Ks, ALPHA, S, SIGMA, Nt)
    v0 = inputs.random_bl(Ks, 3, 64, 1.5, Ns)
    m1 = P0.forward(v0)[3][-1]
    P = objective.Problem(I0, m1, Ks, ALPHA, S, SIGMA, Nt)
    lin = P.gradient(v0)
    x = inputs.random_bl(Ks, 3, 65, 1.0, Ns)
    np.testing.assert_allclose(P.hessvec_newton(lin, x), P.hessvec(lin, x), rtol=1e-12, atol=1e-14)
