"""BL Jacobi PDE-EPDiff LDDMM subject to the deformation state equation
(Section 3.3 of Hernandez, arXiv:1807.11560).

TEST INFRASTRUCTURE ONLY (see the package docstring).  FP64 throughout.

Section 3.3 replaces the image state m(t) on the full grid by a deformation
state phi~(t) carried in the band-limited space.  It prints the equations and
the terminal conditions but leaves these points open; the readings used here:

* phi~(t) is the inverse map phi_t^-1, stored by its band-limited displacement
  u~(t): phi_t^-1(x) = x + iota(u~(t))(x), u~(0) = 0.  The identity part is not
  band-limited, but its Jacobian is the identity, so the deformation state
  equation d/dt phi~ + D~phi~ * v~ = 0 becomes
      d/dt u~ = F(u~, v~) := -v~ - D~u~ * v~,
  component i of D~u~ * v~ being pi[sum_j (d_j u_i) v_j], the product taken
  on the padded grid (the truncated convolution, as for ad~).
* Time stepping: the deformation equation is integrated jointly with BL
  EPDiff by the same Heun step, so its second stage uses the EPDiff predictor
  v*_n:   k1 = F(u_n, v_n),  u*_n = u_n + dt k1,  k2 = F(u*_n, v*_n),
          u_{n+1} = u_n + dt/2 (k1 + k2).
* The warped image is m(1)(x) = I0(x + iota(u~(1))(x)): iota on the image
  grid, then multilinear periodic interpolation of I0 (the same interpolation
  as the state transport).  The energy is Eq. 50 with this m(1).
* grad I0 at the off-grid points x + u(1)(x) is the multilinear interpolation of
  the central-difference grid gradient (as for grad m in the state form).
* The terminal multiplier the paper names rho~(1) without a formula is read as
  rho~(1) = pi[lambda(1) (grad I0)(phi_1^-1(x))], lambda(1) = -(2/sigma^2)(m(1) - I1):
  with it, U~(1) = K~(D~phi~(1)^T * rho~(1)) reproduces Eq. 55 in the continuum,
  because grad m(1) = (D phi_1^-1)^T (grad I0) o phi_1^-1.  The transpose, which
  the printed formula omits, follows from delta phi_1^-1 = -D phi_1^-1 J(1) for a
  Jacobi field J.  So
      U~(1) = K~ pi[ r + (D u(1))^T r ],   r = iota(rho~(1)) on the padded grid,
  component i of (Du)^T r being sum_j (d_i u_j) r_j.
* Gradient: the backward reduced adjoint Jacobi sweep of the state form
  (Eqs. 53-54), unchanged, started from this U~(1); g = v0 + W(0).
* Gauss-Newton Hessian-vector product: the incremental EPDiff (Eq. 30 form),
  the exact tangent of the deformation sweep (the linearised Heun step of
      d/dt delta u~ = -delta v~ - D~delta u~ * v~ - D~u~ * delta v~),
  delta m(1) = (grad I0)(phi_1^-1) . iota(delta u~(1)), delta lambda(1) =
  -(2/sigma^2) delta m(1), delta rho~(1) = pi[delta lambda(1) (grad I0)(phi_1^-1)],
  and, dropping every term multiplied by an adjoint variable (the
  D~delta phi~(1)^T * rho~(1) term of the printed delta U~(1) and the second
  derivative of I0 against lambda(1)),
      delta U~(1) = K~ pi[ dr + (D u(1))^T dr ],  dr = iota(delta rho~(1));
  then the backward sweep of the gradient from delta U~(1): H p = p + delta W(0).
"""

import numpy as np

from . import bl, sweeps
from .objective import Problem

__all__ = [
    "product_Dv", "product_DTr", "deform_rhs", "deform_rhs_tangent", "deform_shoot",
    "deform_tangent", "sample_terminal", "DeformationProblem", "DeformationLinearisation",
]


def _jac_on(a, Ms):
    """Grid values on Ms of the Jacobian of a BL vector field: jac[i][j] = d_j a_i."""
    d = a.shape[0]
    jac = [[None] * d for _ in range(d)]
    for j in range(d):
        dj = bl.iota(bl.deriv(a, j), Ms)
        for i in range(d):
            jac[i][j] = dj[i]
    return jac


def product_Dv(u, v, Ms=None):
    """D~u * v~: component i is pi[sum_j (d_j u_i) v_j] on the padded grid."""
    Ks = u.shape[1:]
    d = u.shape[0]
    Ms = bl.pad_grid(Ks) if Ms is None else tuple(Ms)
    Du = _jac_on(u, Ms)
    vv = bl.iota(v, Ms)
    P = np.empty((d,) + tuple(Ms))
    for i in range(d):
        P[i] = sum(Du[i][j] * vv[j] for j in range(d))
    return bl.pi(P, Ks)


def product_DTr(u, r, Ms=None):
    """(D~u)^T * r~: component i is pi[sum_j (d_i u_j) r_j] on the padded grid."""
    Ks = u.shape[1:]
    d = u.shape[0]
    Ms = bl.pad_grid(Ks) if Ms is None else tuple(Ms)
    Du = _jac_on(u, Ms)
    rr = bl.iota(r, Ms)
    P = np.empty((d,) + tuple(Ms))
    for i in range(d):
        P[i] = sum(Du[j][i] * rr[j] for j in range(d))
    return bl.pi(P, Ks)


def deform_rhs(u, v):
    """F(u, v) = -v - D~u * v (the deformation state equation of Section 3.3)."""
    return -v - product_Dv(u, v)


def deform_rhs_tangent(u, v, du, dv):
    """Linearisation of ``deform_rhs`` at (u, v) along (du, dv)."""
    return -dv - product_Dv(du, v) - product_Dv(u, dv)


def deform_shoot(vs, vstar):
    """Heun sweep of the deformation state from u(0) = 0, jointly with the
    shoot whose states ``vs`` and predictors ``vstar`` are given.

    Returns (us, ustar): us[n] = u~ at t = n dt (n = 0..Nt), ustar[n] = the
    predictor of step n -> n+1.
    """
    Nt = len(vstar)
    dt = 1.0 / Nt
    us = [np.zeros_like(np.asarray(vs[0], dtype=np.complex128))]
    ustar = []
    for n in range(Nt):
        u = us[-1]
        k1 = deform_rhs(u, vs[n])
        up = u + dt * k1
        k2 = deform_rhs(up, vstar[n])
        ustar.append(up)
        us.append(u + 0.5 * dt * (k1 + k2))
    return us, ustar


def deform_tangent(us, ustar, vs, vstar, dvs, dstar):
    """Exact tangent of ``deform_shoot`` along the shoot tangent (dvs, dstar)
    (the stages of ``sweeps.tangent_shoot_stages``); delta u(0) = 0.  Returns
    delta u~(1)."""
    Nt = len(vstar)
    dt = 1.0 / Nt
    du = np.zeros_like(np.asarray(us[0], dtype=np.complex128))
    for n in range(Nt):
        k1 = deform_rhs_tangent(us[n], vs[n], du, dvs[n])
        dup = du + dt * k1
        k2 = deform_rhs_tangent(ustar[n], vstar[n], dup, dstar[n])
        du = du + 0.5 * dt * (k1 + k2)
    return du


def sample_terminal(I0, u1):
    """m(1) = I0(x + u(1)(x)) and (grad I0)(x + u(1)(x)) by multilinear periodic
    interpolation; ``u1`` is the grid displacement (d, N..) in unit-box units."""
    Ns = I0.shape
    d = len(Ns)
    xi = np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in Ns], indexing="ij"))
    xi = xi + u1 * np.array(Ns, dtype=np.float64).reshape((d,) + (1,) * d)
    m1 = sweeps.interp(I0, xi)
    gI0 = sweeps.central_grad(I0)
    gs = np.stack([sweeps.interp(gI0[j], xi) for j in range(d)])
    return m1, gs


class DeformationLinearisation:
    """What one gradient evaluation of the deformation form leaves behind."""

    def __init__(self, v0, vs, vstar, us, ustar, u1, m1, gs, E, g):
        self.v0, self.vs, self.vstar = v0, vs, vstar
        self.us, self.ustar, self.u1 = us, ustar, u1
        self.m1, self.gs = m1, gs
        self.E, self.g = E, g


class DeformationProblem(Problem):
    """The registration problem of Section 3.3: same energy (Eq. 50), the image
    at t = 1 obtained from the band-limited deformation state."""

    def forward_deformation(self, v0):
        vs, vstar = sweeps.shoot(np.asarray(v0, dtype=np.complex128), self.Nt, self.alpha, self.s)
        us, ustar = deform_shoot(vs, vstar)
        u1 = self.grid_velocity(us[-1])
        m1, gs = sample_terminal(self.I0, u1)
        return vs, vstar, us, ustar, u1, m1, gs

    def energy(self, v0):
        v0 = np.asarray(v0, dtype=np.complex128)
        m1 = self.forward_deformation(v0)[5]
        return 0.5 * self.inner_V(v0, v0) + self.data_term(m1)

    def terminal_U_deformation(self, u1_band, f):
        """K~ pi[r + (Du(1))^T r] with r = iota(pi f): the U~(1) of Section 3.3
        for the grid field f = lambda(1) (grad I0)(phi_1^-1) (or its GN increment)."""
        rho = bl.pi(f, self.Ks)
        return (rho + product_DTr(u1_band, rho)) / self.L

    def gradient(self, v0):
        v0 = np.asarray(v0, dtype=np.complex128)
        vs, vstar, us, ustar, u1, m1, gs = self.forward_deformation(v0)
        E = 0.5 * self.inner_V(v0, v0) + self.data_term(m1)
        lam1 = -(2.0 / self.sigma ** 2) * (m1 - self.I1)
        U1 = self.terminal_U_deformation(us[-1], lam1[None] * gs)
        W0 = sweeps.adjoint_jacobi_backward(vs, vstar, U1, self.alpha, self.s)
        return DeformationLinearisation(v0, vs, vstar, us, ustar, u1, m1, gs, E, v0 + W0)

    def incremental_u1(self, lin, p):
        """delta u~(1) along the Hessian-vector direction p."""
        dvs, dstar = sweeps.tangent_shoot_stages(lin.vs, lin.vstar, np.asarray(p, dtype=np.complex128),
                                                 self.alpha, self.s)
        return deform_tangent(lin.us, lin.ustar, lin.vs, lin.vstar, dvs, dstar)

    def hessvec(self, lin, p):
        p = np.asarray(p, dtype=np.complex128)
        du1 = self.grid_velocity(self.incremental_u1(lin, p))
        dm1 = np.sum(lin.gs * du1, axis=0)
        dlam1 = -(2.0 / self.sigma ** 2) * dm1
        dU1 = self.terminal_U_deformation(lin.us[-1], dlam1[None] * lin.gs)
        dW0 = sweeps.adjoint_jacobi_backward(lin.vs, lin.vstar, dU1, self.alpha, self.s)
        return p + dW0

    def transport(self, v0):
        """m(1) of the deformation form (the image the registration produces)."""
        return self.forward_deformation(v0)[5]
