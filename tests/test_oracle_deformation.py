"""Pins of the oracle's deformation-state form (Section 3.3) against brute-force
sums, closed forms, convergence orders, derivatives and the special case v0 = 0,
where the deformation and state forms coincide exactly."""

import itertools

import numpy as np

from oracle import bl, sweeps
from oracle.deformation import (DeformationProblem, deform_rhs, deform_shoot, deform_tangent,
                                product_Dv, product_DTr, sample_terminal)
from oracle.objective import Problem
from paper_1807_11560_gb300 import inputs

ALPHA, S, SIGMA = 0.0025, 2, 0.03


def _rand_bl(rng, Ks, d, scale=1.0):
    a = rng.standard_normal((d,) + Ks) + 1j * rng.standard_normal((d,) + Ks)
    return bl.hermitian_part(a) * scale


def _brute_products(u, v):
    """Truncated convolutions by the double sum over band frequencies p + q = k:
    (Du * v)_i(k) = sum_j sum_{p+q=k} (2 pi i p_j) u_i(p) v_j(q) and
    (Du^T * v)_i(k) = sum_j sum_{p+q=k} (2 pi i p_i) u_j(p) v_j(q)."""
    Ks = u.shape[1:]
    d = u.shape[0]
    f = [bl.freqs(K).astype(int) for K in Ks]
    mask = bl.nyquist_mask(Ks)
    A = np.zeros_like(u)
    B = np.zeros_like(u)
    slots = [k for k in itertools.product(*[range(K) for K in Ks]) if mask[k] != 0]
    for k in slots:
        kf = [f[a][k[a]] for a in range(d)]
        for p in slots:
            pf = [f[a][p[a]] for a in range(d)]
            qf = [kf[a] - pf[a] for a in range(d)]
            if not all(-(Ks[a] // 2) < qf[a] < (Ks[a] + 1) // 2 for a in range(d)):
                continue
            q = tuple(qf[a] % Ks[a] for a in range(d))
            for i in range(d):
                for j in range(d):
                    A[i][k] += 2j * np.pi * pf[j] * u[i][p] * v[j][q]
                    B[i][k] += 2j * np.pi * pf[i] * u[j][p] * v[j][q]
    return A, B


def test_products_match_brute_force_truncated_convolution():
    rng = np.random.default_rng(10)
    for Ks in ((6, 4), (4, 4, 2)):
        d = len(Ks)
        u, v = _rand_bl(rng, Ks, d), _rand_bl(rng, Ks, d)
        A, B = _brute_products(u, v)
        assert np.abs(product_Dv(u, v) - A).max() < 1e-13 * np.abs(A).max()
        assert np.abs(product_DTr(u, v) - B).max() < 1e-13 * np.abs(B).max()


def test_products_do_not_depend_on_the_padded_grid():
    rng = np.random.default_rng(11)
    Ks = (8, 6, 4)
    u, v = _rand_bl(rng, Ks, 3), _rand_bl(rng, Ks, 3)
    for fn in (product_Dv, product_DTr):
        a = fn(u, v)
        b = fn(u, v, Ms=tuple(2 * k for k in Ks))
        assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


def test_terminal_product_is_the_transpose_of_the_deformation_product():
    """<r + Du^T * r, J>_l2 = <r, J + Du * J>_l2: the U~(1) map is the adjoint of
    J -> (Id + D~u) J, the linearised inverse map along a Jacobi field."""
    rng = np.random.default_rng(12)
    Ks = (8, 6, 6)
    u, r, J = (_rand_bl(rng, Ks, 3) for _ in range(3))
    lhs = bl.inner_l2(r + product_DTr(u, r), J)
    rhs = bl.inner_l2(r, J + product_Dv(u, J))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_constant_velocity_translates_the_image_exactly():
    """v = c (the k = 0 mode) is steady under EPDiff; then u(t) = -t c and, for a
    shift of whole voxels, m(1)(x) = I0(x - c) is a roll of I0."""
    rng = np.random.default_rng(13)
    Ns, Ks = (16, 12), (8, 6)
    I0 = rng.standard_normal(Ns)
    P = DeformationProblem(I0, I0, Ks, ALPHA, S, SIGMA, 5)
    v0 = np.zeros((2,) + Ks, dtype=np.complex128)
    v0[0][0, 0], v0[1][0, 0] = 2.0 / 16, -3.0 / 12
    vs, vstar, us, ustar, u1, m1, gs = P.forward_deformation(v0)
    np.testing.assert_allclose(us[-1], -v0, atol=1e-15)
    np.testing.assert_array_equal(m1, np.roll(I0, (2, -3), axis=(0, 1)))
    g = sweeps.central_grad(I0)
    np.testing.assert_allclose(gs, np.roll(g, (2, -3), axis=(1, 2)), atol=1e-12)


def _flow_field(rng, Ks, amp):
    """A smooth band-limited field: modes |k|^2 <= 5, damped by exp(-0.6 |k|^2)."""
    w = _rand_bl(rng, Ks, len(Ks), amp)
    k2 = sum(f * f for f in np.meshgrid(*[bl.freqs(K) for K in Ks], indexing="ij"))
    return w * np.exp(-0.6 * k2) * (k2 <= 5)


def _inverse_map(w, Ns, T, nsub=40):
    """x -> phi_T^-1(x) - x for the stationary field w, by classical RK4 on the
    backward characteristic X' = -w(X) with w summed as its exact Fourier series
    at the off-grid points (independent of iota, pi and the padded products)."""
    Ks = w.shape[1:]
    d = len(Ks)
    F = np.meshgrid(*[bl.freqs(K) for K in Ks], indexing="ij")
    modes = list(zip(*np.nonzero(bl.nyquist_mask(Ks) * (np.abs(w).sum(axis=0) > 0))))

    def vel(X):
        out = np.zeros_like(X)
        for i in range(d):
            acc = np.zeros(X.shape[1:], dtype=np.complex128)
            for k in modes:
                acc += w[i][k] * np.exp(2j * np.pi * sum(F[a][k] * X[a] for a in range(d)))
            out[i] = acc.real
        return out

    X0 = np.stack(np.meshgrid(*[np.arange(n) / n for n in Ns], indexing="ij"))
    X = X0.copy()
    h = -T / nsub
    for _ in range(nsub):
        k1 = vel(X)
        k2 = vel(X + 0.5 * h * k1)
        k3 = vel(X + 0.5 * h * k2)
        k4 = vel(X + h * k3)
        X = X + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return X - X0


def test_deformation_sweep_is_the_inverse_flow_map_to_second_order():
    """For a prescribed velocity history the sweep integrates the inverse map of
    the flow.  Stationary w: phi_1^-1 is the backward flow of w over time 1;
    v(t) = (1 + t) w: the backward flow of w over time 3/2 (the Heun stage
    velocity is v at t_{n+1}).  Errors fall by 4 per halving of dt."""
    rng = np.random.default_rng(14)
    Ks, Ns = (16, 16), (32, 32)
    w = _flow_field(rng, Ks, 0.004)
    for a, T in ((lambda t: 1.0, 1.0), (lambda t: 1.0 + t, 1.5)):
        ref = _inverse_map(w, Ns, T)
        errs = []
        for Nt in (10, 20, 40):
            vs = [a(n / Nt) * w for n in range(Nt + 1)]
            vstar = [a((n + 1) / Nt) * w for n in range(Nt)]
            us, _ = deform_shoot(vs, vstar)
            errs.append(np.abs(bl.iota(us[-1], Ns) - ref).max() / np.abs(ref).max())
        assert errs[-1] < 1e-5, errs
        for r in (errs[0] / errs[1], errs[1] / errs[2]):
            assert 3.6 < r < 4.4, errs


def test_deformation_sweep_is_the_joint_heun_step():
    """The sweep equals a generic Heun integrator run on the stacked state (v, u)
    with right side (-ad~^dagger_v v, F(u, v))."""
    Ks, Ns, Nt = (6, 6, 4), (12, 12, 8), 4
    v0 = inputs.random_bl(Ks, 3, 15, 3.0, Ns)

    def rhs(y):
        v, u = y
        return np.stack([sweeps.epdiff_rhs(v, ALPHA, S), deform_rhs(u, v)])

    y = np.stack([v0.astype(np.complex128), np.zeros_like(v0, dtype=np.complex128)])
    dt = 1.0 / Nt
    for _ in range(Nt):
        k1 = rhs(y)
        k2 = rhs(y + dt * k1)
        y = y + 0.5 * dt * (k1 + k2)
    vs, vstar = sweeps.shoot(v0, Nt, ALPHA, S)
    us, _ = deform_shoot(vs, vstar)
    assert np.abs(us[-1] - y[1]).max() < 1e-13 * np.abs(y[1]).max()
    assert np.abs(y[1]).max() > 1e-3


def test_deformation_tangent_is_the_derivative_of_the_sweep():
    Ks, Ns, Nt = (10, 8), (32, 28), 5
    v0 = inputs.random_bl(Ks, 2, 16, 1.0, Ns)
    p = inputs.random_bl(Ks, 2, 17, 1.0, Ns)
    vs, vstar = sweeps.shoot(v0, Nt, ALPHA, S)
    us, ustar = deform_shoot(vs, vstar)
    dvs, dstar = sweeps.tangent_shoot_stages(vs, vstar, p, ALPHA, S)
    du = deform_tangent(us, ustar, vs, vstar, dvs, dstar)
    errs = []
    for eps in (1e-3, 1e-4):
        up = deform_shoot(*sweeps.shoot(v0 + eps * p, Nt, ALPHA, S))[0][-1]
        um = deform_shoot(*sweeps.shoot(v0 - eps * p, Nt, ALPHA, S))[0][-1]
        errs.append(np.abs((up - um) / (2 * eps) - du).max() / np.abs(du).max())
    assert errs[-1] < 1e-3
    assert 80.0 < errs[0] / errs[1] < 120.0, errs          # central differences: eps^2


def test_zero_velocity_reduces_to_the_state_form():
    """At v0 = 0 both forms leave I0 in place (u = 0, m(1) = I0, grad I0 at the grid
    points): energy, gradient and GN product agree to rounding."""
    Ns, Ks, Nt = (32, 28), (10, 8), 5
    I0, I1 = inputs.make_pair("blobs", Ns, 21)
    D = DeformationProblem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    St = Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    z = np.zeros((2,) + Ks, dtype=np.complex128)
    p = inputs.random_bl(Ks, 2, 18, 1.0, Ns)
    assert D.energy(z) == St.energy(z)
    lD, lS = D.gradient(z), St.gradient(z)
    assert np.abs(lD.g - lS.g).max() <= 1e-13 * np.abs(lS.g).max()
    HD, HS = D.hessvec(lD, p), St.hessvec(lS, p)
    assert np.abs(HD - HS).max() <= 1e-13 * np.abs(HS).max()


def test_sample_terminal_at_zero_displacement():
    rng = np.random.default_rng(19)
    I0 = rng.standard_normal((10, 8, 6))
    m1, gs = sample_terminal(I0, np.zeros((3, 10, 8, 6)))
    np.testing.assert_array_equal(m1, I0)
    np.testing.assert_allclose(gs, sweeps.central_grad(I0), atol=1e-13)


def test_gn_hessian_is_positive_and_gn_solve_descends():
    """Paper form: the GN product is positive on random directions and nearly
    symmetric (the gap is the discretisation/truncation gap of the Jacobi form),
    and GN-Krylov on it lowers the energy monotonically."""
    Ns, Ks, Nt = (32, 28), (10, 8), 5
    I0, I1 = inputs.make_pair("blobs", Ns, 21)
    D = DeformationProblem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    v0 = inputs.random_bl(Ks, 2, 5, 1.0, Ns)
    lin = D.gradient(v0)
    p = inputs.random_bl(Ks, 2, 20, 1.0, Ns)
    q = inputs.random_bl(Ks, 2, 21, 1.0, Ns)
    Hp, Hq = D.hessvec(lin, p), D.hessvec(lin, q)
    assert D.inner_V(Hp, p) > D.inner_V(p, p)
    assert abs(D.inner_V(Hp, q) - D.inner_V(p, Hq)) < 0.05 * np.sqrt(D.inner_V(Hp, p) * D.inner_V(Hq, q))
    z = np.zeros((2,) + Ks, dtype=np.complex128)
    v, rep = D.gn_solve(z, 3, 4)
    assert not rep["ls_failed"]
    E = rep["E"] + [rep["E_final"]]
    assert all(b < a for a, b in zip(E, E[1:])), E
    assert rep["E_final"] < 0.5 * rep["E"][0]


def test_terminal_U_is_the_V_representer_of_the_linearised_inverse_map():
    """<U~(1), J>_V = <f, iota(J + D~u * J)>_{L2_h} for the U~(1) built from a grid
    field f (the right side evaluated on the image grid, without pi)."""
    rng = np.random.default_rng(22)
    Ns, Ks = (16, 12, 10), (8, 6, 6)
    P = DeformationProblem(np.zeros(Ns), np.zeros(Ns), Ks, ALPHA, S, SIGMA, 4)
    u, J = _rand_bl(rng, Ks, 3), _rand_bl(rng, Ks, 3)
    f = rng.standard_normal((3,) + Ns)
    U1 = P.terminal_U_deformation(u, f)
    rhs = float(np.sum(f * bl.iota(J + product_Dv(u, J), Ns))) / float(np.prod(Ns))
    assert abs(P.inner_V(U1, J) - rhs) < 1e-12 * abs(rhs)


def test_gn_product_is_the_composition_of_its_pinned_pieces():
    """<H p - p, q>_V = -(2/sigma^2) h^d sum_x (g . du(1)[p]) (g . iota(J + D~u(1) * J)[q])
    with g = (grad I0)(phi_1^-1), du(1) from the deformation tangent and J = J(1)[q]
    from the Jacobi tangent whose transpose the backward sweep is."""
    Ns, Ks, Nt = (32, 28), (10, 8), 5
    I0, I1 = inputs.make_pair("blobs", Ns, 21)
    D = DeformationProblem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    v0 = inputs.random_bl(Ks, 2, 5, 1.0, Ns)
    lin = D.gradient(v0)
    p = inputs.random_bl(Ks, 2, 23, 1.0, Ns)
    q = inputs.random_bl(Ks, 2, 24, 1.0, Ns)
    lhs = D.inner_V(D.hessvec(lin, p) - p, q)
    du1 = bl.iota(D.incremental_u1(lin, p), Ns)
    J1 = sweeps.jacobi_tangent(lin.vs, lin.vstar, q, ALPHA, S)
    a = np.sum(lin.gs * du1, axis=0)
    b = np.sum(lin.gs * bl.iota(J1 + product_Dv(lin.us[-1], J1), Ns), axis=0)
    rhs = -(2.0 / SIGMA ** 2) * float(np.sum(a * b)) / float(np.prod(Ns))
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)
