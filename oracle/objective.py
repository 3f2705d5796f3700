"""Energy, gradient, GN Hessian-vector product and GN-Krylov solve (arXiv:1807.11560).

TEST INFRASTRUCTURE ONLY (see the package docstring).  FP64 throughout.

Readings of the paper used here:

* Energy (Eq. 50): E = 1/2 <L~ v0, v0>_{l2} + sigma^-2 ||m(1) - I1||^2_{L2},
  with the 1/sigma^2 weight as printed (not 1/(2 sigma^2)).
* Terminal adjoint (text after Eq. 14): lambda(1) = -(2/sigma^2)(m(1) - I1);
  U~(1) = K~ pi(lambda(1) grad m(1)) (Eq. 55).  K~ and pi commute on the band,
  so Eq. 55 and Eq. 58's orders agree.
* V-gradient: g = v0 + W(0) where W is the backward adjoint Jacobi sweep
  (Eqs. 53-54) started from U~(1).  The regulariser contributes v0 because
  the gradient is taken in V ("CG ... computed on V", Section 2.7).
* Gauss-Newton (Section 2.7 drops terms to keep H positive definite): every
  term multiplied by an adjoint variable is dropped -- -lambda(1) grad dm(1)
  in Eq. 58 and ad~^dagger_{dv} U, -ad~_{dv} w, ad~^dagger_w dv in Eqs. 56-57.
  What is left of Eqs. 56-57 is the operator of Eqs. 53-54, started from
  dU~(1) = K~ pi(dlambda(1) grad m(1)), dlambda(1) = -(2/sigma^2) dm(1)
  (text after Eq. 17), with dm from the incremental state sweep (Eq. 31)
  driven by the incremental EPDiff (Eq. 30) from dv(0) = p.
  H p = p + dW(0).
* Update (Eqs. 44-45): the printed v - eps dv with H dv = -grad E would step
  uphill; the reading is v <- v + eps p with H p = -g.  eps by Armijo
  backtracking (eps0 = 1, halve, c = 1e-4, at most 10 halvings).
* PCG (Eq. 45, "CG on V"): conjugate gradients in the V inner product, fixed
  iteration count, early stop on ||r||_V <= tol ||b||_V or on non-positive
  curvature <d, H d>_V <= 0.
"""

import numpy as np

from . import bl, sweeps

__all__ = ["Problem", "Linearisation"]


class Linearisation:
    """Everything one gradient evaluation leaves behind for Hessian products."""

    def __init__(self, v0, vs, vstar, vgrid, ms, feet, E, g):
        self.v0, self.vs, self.vstar = v0, vs, vstar
        self.vgrid, self.ms, self.feet = vgrid, ms, feet
        self.E, self.g = E, g


class Problem:
    """One registration problem: I0, I1 on the grid, band K, alpha, s, sigma, Nt."""

    def __init__(self, I0, I1, Ks, alpha, s, sigma, Nt):
        self.I0 = np.asarray(I0, dtype=np.float64)
        self.I1 = np.asarray(I1, dtype=np.float64)
        self.Ns = self.I0.shape
        self.d = len(self.Ns)
        self.Ks = tuple(int(k) for k in Ks)
        self.alpha, self.s, self.sigma, self.Nt = float(alpha), int(s), float(sigma), int(Nt)
        self.dt = 1.0 / self.Nt
        self.L = bl.lhat(self.Ks, self.alpha, self.s)
        self.hd = 1.0 / float(np.prod(self.Ns))

    # ---- helpers ---------------------------------------------------------
    def inner_V(self, a, b):
        return bl.inner_V(a, b, self.alpha, self.s)

    def grid_velocity(self, a):
        return bl.iota(a, self.Ns)

    def data_term(self, m1):
        r = m1 - self.I1
        return float(np.sum(r * r)) * self.hd / self.sigma ** 2

    # ---- forward ---------------------------------------------------------
    def forward(self, v0):
        """Shoot (Eq. 51) and transport (Eq. 52); returns (vs, vstar, vgrid, ms, feet)."""
        vs, vstar = sweeps.shoot(v0, self.Nt, self.alpha, self.s)
        vgrid = [self.grid_velocity(v) for v in vs]
        ms, feet = sweeps.transport(self.I0, vgrid, self.dt)
        return vs, vstar, vgrid, ms, feet

    def energy(self, v0):
        """E(v0) of Eq. 50."""
        vs, vstar, vgrid, ms, feet = self.forward(v0)
        return 0.5 * self.inner_V(v0, v0) + self.data_term(ms[-1])

    def terminal_U(self, m1, lam1):
        """K~ pi(lambda(1) grad m(1)) (Eq. 55 / Eq. 58 under GN)."""
        f = lam1[None] * sweeps.central_grad(m1)
        return bl.pi(f, self.Ks) / self.L

    # ---- gradient --------------------------------------------------------
    def gradient(self, v0):
        """V-gradient g = v0 + W(0) (Eqs. 53-55) and E; returns a Linearisation."""
        v0 = np.asarray(v0, dtype=np.complex128)
        vs, vstar, vgrid, ms, feet = self.forward(v0)
        m1 = ms[-1]
        E = 0.5 * self.inner_V(v0, v0) + self.data_term(m1)
        lam1 = -(2.0 / self.sigma ** 2) * (m1 - self.I1)
        U1 = self.terminal_U(m1, lam1)
        W0 = sweeps.adjoint_jacobi_backward(vs, vstar, U1, self.alpha, self.s)
        return Linearisation(v0, vs, vstar, vgrid, ms, feet, E, v0 + W0)

    def exact_gradient(self, v0):
        """V-gradient of the discretised energy itself (the PDE-LDDMM route of
        Section 2.5 in discrete form: the state transport reversed step by step,
        Eqs. 12-14, then every time level's velocity sensitivity carried back to
        v0 through the transpose of the Heun shoot).  Returns (E, g).

        lambda(1) = dL/dm(1) = 2 sigma^-2 h^d (m(1) - I1) on the grid; the grid
        sensitivities G_n = dL/dv_n(grid) come from ``transport_adjoint``; their
        band V-representers are s_n = K~ sum_x G_n(x) e^{-2 pi i k.x} (the adjoint
        of iota is N^d pi); g = v0 + W_0 with W from ``transpose_shoot``."""
        v0 = np.asarray(v0, dtype=np.complex128)
        vs, vstar, vgrid, ms, feet = self.forward(v0)
        E = 0.5 * self.inner_V(v0, v0) + self.data_term(ms[-1])
        lam1 = 2.0 * self.hd / self.sigma ** 2 * (ms[-1] - self.I1)
        G = sweeps.transport_adjoint(ms, vgrid, lam1, self.dt)
        nd = float(np.prod(self.Ns))
        sources = [nd * bl.pi(Gn, self.Ks) / self.L for Gn in G]
        W0 = sweeps.transpose_shoot(vs, vstar, sources, self.alpha, self.s)
        return E, v0 + W0

    # ---- Gauss-Newton Hessian-vector product -----------------------------
    def incremental_m1(self, lin, p):
        """dm(1) from Eq. 30 (BL tangent shoot from p) and Eq. 31 (grid transport)."""
        dvs = sweeps.tangent_shoot(lin.vs, lin.vstar, p, self.alpha, self.s)
        dvgrid = [self.grid_velocity(d) for d in dvs]
        return sweeps.incremental_transport(lin.ms, lin.feet, dvgrid, self.dt)

    def hessvec(self, lin, p):
        """GN Hessian-vector product in V: H p = p + dW(0) (Eqs. 30-31, 56-58 under GN)."""
        p = np.asarray(p, dtype=np.complex128)
        dm1 = self.incremental_m1(lin, p)
        dlam1 = -(2.0 / self.sigma ** 2) * dm1
        dU1 = self.terminal_U(lin.ms[-1], dlam1)
        dW0 = sweeps.adjoint_jacobi_backward(lin.vs, lin.vstar, dU1, self.alpha, self.s)
        return p + dW0

    def terminal_U_newton(self, m1, dm1):
        """Derivative of U~(1) = K~ pi(lambda(1) grad m(1)) along dm(1):
        K~ pi(dlambda(1) grad m(1) + lambda(1) grad dm(1)), lambda(1) = -(2/sigma^2)
        (m(1) - I1), dlambda(1) = -(2/sigma^2) dm(1) (Eq. 58 without the
        Gauss-Newton drop; the sign of the second term follows from differentiating
        the gradient's own terminal value)."""
        c = -2.0 / self.sigma ** 2
        f = c * (dm1[None] * sweeps.central_grad(m1) + (m1 - self.I1)[None] * sweeps.central_grad(dm1))
        return bl.pi(f, self.Ks) / self.L

    def hessvec_newton(self, lin, p):
        """Full-Newton Hessian-vector product in V (Eqs. 56-58 without the
        Gauss-Newton drop): the derivative of the paper-form gradient
        g = v0 + W(0)[v; U~(1)] along p, with dm(1) from the incremental state
        sweep (Eq. 31) as in the Gauss-Newton product.  H p = p + dW(0)."""
        p = np.asarray(p, dtype=np.complex128)
        dvs, dstar = sweeps.tangent_shoot_stages(lin.vs, lin.vstar, p, self.alpha, self.s)
        dvgrid = [self.grid_velocity(d) for d in dvs]
        dm1 = sweeps.incremental_transport(lin.ms, lin.feet, dvgrid, self.dt)
        dU1 = self.terminal_U_newton(lin.ms[-1], dm1)
        m1 = lin.ms[-1]
        U1 = self.terminal_U(m1, -(2.0 / self.sigma ** 2) * (m1 - self.I1))
        _, zs, zt = sweeps.adjoint_jacobi_backward_stages(lin.vs, lin.vstar, U1, self.alpha, self.s)
        dW0 = sweeps.newton_backward(lin.vs, lin.vstar, dvs, dstar, zs, zt, dU1, self.alpha, self.s)
        return p + dW0

    def hessvec_J(self, lin, p):
        """Diagnostic J-form GN product: dm(1) replaced by -grad m(1) . iota(J(1)).

        J(1) is the BL Jacobi-field tangent whose exact transpose the backward
        sweep applies, so this H is symmetric positive definite to rounding.
        """
        p = np.asarray(p, dtype=np.complex128)
        J1 = sweeps.jacobi_tangent(lin.vs, lin.vstar, p, self.alpha, self.s)
        gm = sweeps.central_grad(lin.ms[-1])
        dm1 = -np.sum(gm * self.grid_velocity(J1), axis=0)
        dlam1 = -(2.0 / self.sigma ** 2) * dm1
        dU1 = self.terminal_U(lin.ms[-1], dlam1)
        dW0 = sweeps.adjoint_jacobi_backward(lin.vs, lin.vstar, dU1, self.alpha, self.s)
        return p + dW0

    # ---- Krylov and Gauss-Newton ----------------------------------------
    def pcg(self, lin, b, n_iter, tol=1e-12, op=None):
        """CG in the V inner product on H x = b (Eq. 45); returns (x, iterations).

        ``op`` replaces the GN product (the tests pass the exactly symmetric
        J form to check CG itself).
        """
        op = self.hessvec if op is None else op
        x = np.zeros_like(b)
        r = b.copy()
        d = r.copy()
        rho = self.inner_V(r, r)
        bnorm = np.sqrt(rho)
        it = 0
        for it in range(1, n_iter + 1):
            q = op(lin, d)
            dq = self.inner_V(d, q)
            if dq <= 0.0:
                if it == 1:
                    x = d.copy()
                it -= 1
                break
            a = rho / dq
            x = x + a * d
            r = r - a * q
            rho_new = self.inner_V(r, r)
            if np.sqrt(rho_new) <= tol * bnorm:
                break
            d = r + (rho_new / rho) * d
            rho = rho_new
        return x, it

    def mse_rel(self, m1):
        """100 ||m(1) - I1||^2 / ||I0 - I1||^2 (the MSE_rel of Table 1, in %)."""
        return 100.0 * float(np.sum((m1 - self.I1) ** 2) / np.sum((self.I0 - self.I1) ** 2))

    def gn_solve(self, v0, n_gn, n_pcg, armijo_c=1e-4, max_halvings=10, pcg_tol=1e-12):
        """Inexact Gauss-Newton-Krylov with Armijo backtracking (Eqs. 44-45).

        Returns (v0, report) where report holds per-iteration E, eps, PCG
        iteration counts and a flag telling whether the line search failed.
        """
        v = np.array(v0, dtype=np.complex128)
        rep = {"E": [], "eps": [], "pcg_iters": [], "gnorm": [], "ls_failed": False,
               "v_hist": [], "trials": []}
        for _ in range(n_gn):
            lin = self.gradient(v)
            rep["E"].append(lin.E)
            rep["gnorm"].append(np.sqrt(self.inner_V(lin.g, lin.g)))
            p, its = self.pcg(lin, -lin.g, n_pcg, pcg_tol)
            rep["pcg_iters"].append(its)
            slope = self.inner_V(lin.g, p)
            eps = 1.0
            accepted = False
            trials = []                  # (eps, trial energy, Armijo bound) of each trial
            for _h in range(max_halvings + 1):
                Et = self.energy(v + eps * p)
                trials.append((eps, Et, lin.E + armijo_c * eps * slope))
                if Et <= lin.E + armijo_c * eps * slope:
                    accepted = True
                    break
                eps *= 0.5
            rep["trials"].append(trials)
            if not accepted:
                rep["ls_failed"] = True
                break
            rep["eps"].append(eps)
            v = v + eps * p
            rep["v_hist"].append(v.copy())
        rep["E_final"] = self.energy(v)
        return v, rep
