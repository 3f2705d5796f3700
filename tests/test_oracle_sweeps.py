"""Pins of the oracle's time sweeps (Section 3.2) against invariants, orders and special cases."""

import numpy as np
import pytest

from oracle import bl, sweeps
from paper_1807_11560_gb300 import inputs

ALPHA, S = 0.0025, 2


def test_shoot_zero_and_constant_fields():
    Ks, Ns = (8, 8, 8), (16, 16, 16)
    z = np.zeros((3,) + Ks, dtype=np.complex128)
    vs, vstar = sweeps.shoot(z, 5, ALPHA, S)
    assert all(np.abs(v).max() == 0.0 for v in vs + vstar)
    c = z.copy()
    c[:, 0, 0, 0] = [0.1, -0.2, 0.05]          # constant velocity (k = 0 mode)
    vs, vstar = sweeps.shoot(c, 5, ALPHA, S)
    for v in vs:
        np.testing.assert_allclose(v, c, atol=1e-17)


def test_shoot_mode_beyond_band_is_steady():
    """v = a cos(2 pi k x1) e1 with 2k >= K/2: ad^dagger_v v = 0 on the band, so v is steady."""
    Ks = (8, 8)
    a = np.zeros((2,) + Ks, dtype=np.complex128)
    a[0, 2, 0] = a[0, 6, 0] = 0.15
    vs, _ = sweeps.shoot(a, 7, ALPHA, S)
    np.testing.assert_allclose(vs[-1], a, atol=1e-16)


def test_energy_drift_has_heun_order():
    """Semi-discrete BL EPDiff conserves <L v, v> exactly (<ad^dag_v v, v>_V = <v, ad_v v>_V = 0).
    Heun's stability function gives |R(iy)|^2 = 1 + y^4/4: the drift is third order, so
    doubling Nt divides it by 8."""
    Ks, Ns = (8, 8), (16, 16)
    v0 = inputs.random_bl(Ks, 2, 1, 4.0, Ns)
    drifts = []
    for Nt in (20, 40, 80):
        vs, _ = sweeps.shoot(v0, Nt, ALPHA, S)
        e0 = bl.inner_V(vs[0], vs[0], ALPHA, S)
        drifts.append(abs(bl.inner_V(vs[-1], vs[-1], ALPHA, S) - e0) / e0)
    assert drifts[-1] < 1e-5
    for r in (drifts[0] / drifts[1], drifts[1] / drifts[2]):
        assert 7.0 < r < 9.0, drifts
    # and the field really moved, so conservation is not trivial
    vs, _ = sweeps.shoot(v0, 20, ALPHA, S)
    assert np.abs(vs[-1] - vs[0]).max() > 0.2 * np.abs(vs[0]).max()


def test_tangent_shoot_is_derivative_of_shoot():
    Ks, Ns = (6, 6, 4), (12, 12, 8)
    v0 = inputs.random_bl(Ks, 3, 2, 3.0, Ns)
    p = inputs.random_bl(Ks, 3, 3, 1.0, Ns)
    vs, vstar = sweeps.shoot(v0, 6, ALPHA, S)
    dvs = sweeps.tangent_shoot(vs, vstar, p, ALPHA, S)
    errs = []
    for eps in (1e-2, 1e-3):
        fp = sweeps.shoot(v0 + eps * p, 6, ALPHA, S)[0][-1]
        fm = sweeps.shoot(v0 - eps * p, 6, ALPHA, S)[0][-1]
        errs.append(np.abs((fp - fm) / (2 * eps) - dvs[-1]).max() / np.abs(dvs[-1]).max())
    assert errs[1] < 1e-6
    assert 80 < errs[0] / errs[1] < 120          # central difference: O(eps^2)


def test_adjoint_sweep_is_exact_transpose_of_jacobi_tangent():
    """<W(0)[U1], p>_V = <U1, J(1)[p]>_V for the Heun tangent of (J, dv)."""
    Ks, Ns = (8, 6, 6), (16, 12, 12)
    v0 = inputs.random_bl(Ks, 3, 4, 3.0, Ns)
    vs, vstar = sweeps.shoot(v0, 5, ALPHA, S)
    for seed in (10, 11, 12):
        p = inputs.random_bl(Ks, 3, seed, 1.0, Ns)
        U1 = inputs.random_bl(Ks, 3, seed + 100, 1.0, Ns)
        J1 = sweeps.jacobi_tangent(vs, vstar, p, ALPHA, S)
        W0 = sweeps.adjoint_jacobi_backward(vs, vstar, U1, ALPHA, S)
        a = bl.inner_V(W0, p, ALPHA, S)
        b = bl.inner_V(U1, J1, ALPHA, S)
        assert abs(a - b) <= 1e-12 * (abs(a) + 1e-30) + 1e-14 * np.sqrt(
            bl.inner_V(W0, W0, ALPHA, S) * bl.inner_V(p, p, ALPHA, S)), (a, b)


def test_adjoint_sweep_at_zero_velocity():
    """v = 0: U stays U1 and W(0) = U1 (sum of Nt steps of dt U1)."""
    Ks = (6, 6)
    z = np.zeros((2,) + Ks, dtype=np.complex128)
    vs, vstar = sweeps.shoot(z, 7, ALPHA, S)
    U1 = inputs.random_bl(Ks, 2, 3, 1.0, (12, 12))
    np.testing.assert_allclose(sweeps.adjoint_jacobi_backward(vs, vstar, U1, ALPHA, S), U1, atol=1e-15)


def test_interp_is_textbook_linear_interpolation_in_1d_slices():
    rng = np.random.default_rng(0)
    f = rng.normal(size=(13, 1))
    x = rng.uniform(-20, 20, size=50)
    xi = np.stack([x, np.zeros_like(x)])
    xp = np.arange(-26, 27)
    ref = np.interp(x, xp, f[xp % 13, 0])
    np.testing.assert_allclose(sweeps.interp(f, xi), ref, atol=1e-14)
    # multilinear reproduces linear functions exactly (away from the wrap)
    g = np.fromfunction(lambda i, j, k: 0.3 * i - 0.7 * j + 0.2 * k + 1, (9, 8, 7))
    pts = np.stack([rng.uniform(0, 7.9, 40), rng.uniform(0, 6.9, 40), rng.uniform(0, 5.9, 40)])
    np.testing.assert_allclose(sweeps.interp(g, pts), 0.3 * pts[0] - 0.7 * pts[1] + 0.2 * pts[2] + 1,
                               atol=1e-13)


def test_central_grad_exact_on_discrete_sinusoid():
    N = 16
    x = np.arange(N) / N
    m = np.sin(2 * np.pi * 3 * x)[:, None] * np.ones((1, 5))
    g = sweeps.central_grad(m)
    want = np.sin(2 * np.pi * 3 / N) * N * np.cos(2 * np.pi * 3 * x)   # (sin(x+h)-sin(x-h))/(2h)
    np.testing.assert_allclose(g[0][:, 0], want, atol=1e-12)
    assert np.abs(g[1]).max() < 1e-12


def test_transport_identity_and_integer_shift():
    Ks, Ns = (8, 8, 8), (16, 12, 16)
    rng = np.random.default_rng(1)
    I0 = rng.uniform(size=Ns)
    zero = [np.zeros((3,) + Ns)] * 5
    ms, _ = sweeps.transport(I0, zero, 0.25)
    np.testing.assert_array_equal(ms[-1], I0)
    # constant velocity: dt * v * N_j integer voxels per step => exact shift
    Nt = 4
    dt = 1.0 / Nt
    c = np.zeros((3,) + Ks, dtype=np.complex128)
    c[:, 0, 0, 0] = [1.0 / (dt * Ns[0]), -2.0 / (dt * Ns[1]), 0.0]
    vs, _ = sweeps.shoot(c, Nt, ALPHA, S)
    vg = [bl.iota(v, Ns) for v in vs]
    ms, _ = sweeps.transport(I0, vg, dt)
    np.testing.assert_allclose(ms[-1], np.roll(I0, (Nt * 1, Nt * -2, 0), axis=(0, 1, 2)), atol=1e-13)


def test_incremental_transport_at_zero_velocity():
    """v = 0, dv = const in time: dm(1) = -grad I0 . dv exactly (trapezoid of a constant)."""
    Ns = (12, 10)
    rng = np.random.default_rng(2)
    I0 = rng.uniform(size=Ns)
    dv = rng.normal(size=(2,) + Ns)
    zero = [np.zeros((2,) + Ns)] * 6
    ms, feet = sweeps.transport(I0, zero, 0.2)
    dm = sweeps.incremental_transport(ms, feet, [dv] * 6, 0.2)
    np.testing.assert_allclose(dm, -np.sum(sweeps.central_grad(I0) * dv, axis=0), atol=1e-13)


def test_incremental_transport_converges_to_derivative_of_transport():
    """dm(1) (Eq. 31) against a central difference of the transported m(1) (Eq. 52):
    both discretise the same derivative; the gap shrinks as the grid is refined."""
    Ks = (8, 8)
    gaps = []
    for N in (16, 32, 64):
        Ns = (N, N)
        x = np.arange(N) / N
        I0 = (np.sin(2 * np.pi * x)[:, None] * np.cos(2 * np.pi * x)[None, :]
              + 0.5 * np.cos(4 * np.pi * x)[None, :])
        v0 = inputs.random_bl(Ks, 2, 21, 2.0 * N / 16, Ns)
        p = inputs.random_bl(Ks, 2, 11, 1.0 * N / 16, Ns)
        vs, vstar = sweeps.shoot(v0, 10, ALPHA, S)
        vg = [bl.iota(v, Ns) for v in vs]
        ms, feet = sweeps.transport(I0, vg, 0.1)
        dvs = sweeps.tangent_shoot(vs, vstar, p, ALPHA, S)
        dm = sweeps.incremental_transport(ms, feet, [bl.iota(d, Ns) for d in dvs], 0.1)
        eps = 1e-5
        mp = sweeps.transport(I0, [bl.iota(v, Ns) for v in sweeps.shoot(v0 + eps * p, 10, ALPHA, S)[0]], 0.1)[0][-1]
        mm = sweeps.transport(I0, [bl.iota(v, Ns) for v in sweeps.shoot(v0 - eps * p, 10, ALPHA, S)[0]], 0.1)[0][-1]
        fd = (mp - mm) / (2 * eps)
        gaps.append(np.sqrt(np.mean((dm - fd) ** 2) / np.mean(fd ** 2)))
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 0.06, gaps


# ---- the characteristic of the state transport at time- and space-varying
# velocity.  Fields built from the periodic triangle wave tri (slope 1 on
# [-1/4, 1/4], slope -1 on [1/4, 3/4], kinks on grid nodes when 4 | N) are
# reproduced exactly by multilinear interpolation, and near the origin they are
# linear: v(t, x) = V(t) x with V(t) = A + t B, [A, B] != 0.  There the exact
# flow is linear, every interpolation the scheme makes is exact, and what is
# left is the time discretisation of the characteristic alone.

def _tri(x):
    y = np.mod(x + 0.25, 1.0) - 0.25
    return np.where(y <= 0.25, y, 0.5 - y)


_A = np.array([[0.15, 0.45], [-0.35, -0.05]])
_B = np.array([[0.30, -0.20], [0.40, 0.10]])
_C = np.array([1.0, -0.7])          # I0 = C . tri(x)


def _affine_case(N, Nt):
    """(signed node coordinates (2, N, N), I0, velocity grids at t_n)."""
    s = np.arange(N) / N
    s = np.where(s < 0.5, s, s - 1.0)
    X = np.stack(np.meshgrid(s, s, indexing="ij"))
    T = _tri(X)
    I0 = _C[0] * T[0] + _C[1] * T[1]
    vg = [np.einsum("jk,k...->j...", _A + (n / Nt) * _B, T) for n in range(Nt + 1)]
    return X, I0, vg


def _flow_back(nsub=4000):
    """Psi with Y(0) = Psi Y(1) for Y' = (A + t B) Y: classical RK4 on the 2x2
    fundamental matrix from t = 1 down to t = 0."""
    P = np.eye(2)
    h = -1.0 / nsub
    V = lambda t: _A + t * _B
    t = 1.0
    for _ in range(nsub):
        k1 = V(t) @ P
        k2 = V(t + 0.5 * h) @ (P + 0.5 * h * k1)
        k3 = V(t + 0.5 * h) @ (P + 0.5 * h * k2)
        k4 = V(t + h) @ (P + h * k3)
        P = P + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += h
    return P


def test_transport_characteristic_is_second_order_at_time_varying_velocity():
    """m(1) against I0 at the exact inverse flow (a time-dependent linear flow
    whose matrices do not commute): the error at the nodes near the origin falls
    by 4 per halving of dt.  Evaluating v_n at the point reached with v_{n+1}
    (the midpoint of the RK2 characteristic) is what makes the step second
    order; evaluating both at x would fall by 2."""
    N = 512
    Psi = _flow_back()
    errs = []
    for Nt in (10, 20, 40):
        X, I0, vg = _affine_case(N, Nt)
        ms, _ = sweeps.transport(I0, vg, 1.0 / Nt)
        inner = (np.abs(X[0]) <= 1.0 / 32) & (np.abs(X[1]) <= 1.0 / 32)
        want = np.einsum("k,kj,j...->...", _C, Psi, X)
        errs.append(np.abs(ms[-1] - want)[inner].max())
    assert errs[-1] < 1e-5, errs
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 3.6 < r < 4.4, errs


def test_transport_foot_points_are_the_trapezoid_with_midpoint_velocity():
    """Under the same exact interpolation each step's foot map is the matrix
    I - dt/2 (V_{n+1} + V_n (I - dt V_{n+1})): v_{n+1} at the node, v_n at the
    node moved back by dt v_{n+1} (the RK2 characteristic of the state equation).
    m_Nt(x) = C . (X_0 X_1 ... X_{Nt-1}) x at the inner nodes to rounding; with
    the roles of v_n and v_{n+1} exchanged the product differs by dt^3 [A, B]
    per step."""
    N, Nt = 256, 10
    dt = 1.0 / Nt
    X, I0, vg = _affine_case(N, Nt)
    ms, feet = sweeps.transport(I0, vg, dt)
    V = [_A + (n / Nt) * _B for n in range(Nt + 1)]
    P = np.eye(2)
    for n in range(Nt):
        P = P @ (np.eye(2) - 0.5 * dt * (V[n + 1] + V[n] @ (np.eye(2) - dt * V[n + 1])))
    inner = (np.abs(X[0]) <= 1.0 / 32) & (np.abs(X[1]) <= 1.0 / 32)
    want = np.einsum("k,kj,j...->...", _C, P, X)
    np.testing.assert_allclose(ms[-1][inner], want[inner], rtol=0, atol=1e-13)
    # one step's foot points in index units, at every inner node
    Xn = np.eye(2) - 0.5 * dt * (V[1] + V[0] @ (np.eye(2) - dt * V[1]))
    want_feet = np.einsum("jk,k...->j...", Xn, X) * N
    got = feet[0] - np.round(feet[0] / N) * N          # signed index coordinates
    np.testing.assert_allclose(got[:, inner], want_feet[:, inner], rtol=0, atol=1e-10)
