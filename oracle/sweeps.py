"""Time sweeps of BL Jacobi PDE-EPDiff LDDMM (Section 3.2 of arXiv:1807.11560).

TEST INFRASTRUCTURE ONLY (see the package docstring).  FP64 throughout.

The paper states continuous equations only.  The discretisation read here:

* Nt uniform steps, dt = 1/Nt.
* BL sweeps use Heun's method (explicit trapezoid).  The forward shoot of
  BL EPDiff (Eq. 51) stores v_n (n = 0..Nt) and the predictors v*_{n+1}.
* The incremental EPDiff (Eq. 30 in BL form) is the exact linearisation of
  that Heun step, started from the Hessian-vector direction p (Eq. 30 prints
  delta v(0) = 0, which would make the data part of the product vanish; the
  reading is delta v(0) = p).
* The backward reduced adjoint Jacobi sweep (Eqs. 53-54; Eqs. 56-57 under
  Gauss-Newton) is the exact discrete transpose, in the V inner product, of
  the Heun tangent of the Jacobi pair (J, delta v):
      J' = delta v + ad~_v J,      delta v' = -ad~^dagger_{delta v} v - ad~^dagger_v delta v.
  The transpose of the right side is
      G^T(U, W) = (ad~^dagger_v U,  U + ad~^dagger_W v - ad~_v W),
  which is Eq. 54 with its delta v term read as ad~ (Eq. 8 and Eq. 40 print
  ad; the dagger in Eq. 54 is read as a typo).
* The state equation (Eq. 52) and the incremental state equation (Eq. 31)
  run on the full image grid by semi-Lagrangian steps: backward characteristic
  foot point by the trapezoid (RK2) rule
      X_n(x) = x - dt/2 [v_{n+1}(x) + v_n(x - dt v_{n+1}(x))],
  multilinear (bilinear in 2D, trilinear in 3D) periodic interpolation, the
  grid velocity being iota(v~_n) on the image grid.  The incremental source
  term -grad m . delta v is integrated by the trapezoid rule along the same
  characteristic; grad is the second-order central difference.
"""

import itertools

import numpy as np

from . import bl

__all__ = [
    "epdiff_rhs", "epdiff_rhs_tangent", "shoot", "tangent_shoot",
    "jacobi_tangent", "adjoint_jacobi_backward", "adjoint_jacobi_backward_stages",
    "tangent_shoot_stages", "newton_backward", "interp", "central_grad",
    "foot_points", "transport", "incremental_transport",
]


# --------------------------------------------------------------------------
# BL sweeps
# --------------------------------------------------------------------------

def epdiff_rhs(v, alpha, s):
    """Right side of BL EPDiff, -ad~^dagger_v v (Eq. 48 / Eq. 51)."""
    return -bl.ad_dagger(v, v, alpha, s)


def epdiff_rhs_tangent(v, dv, alpha, s):
    """Linearisation of ``epdiff_rhs`` at v in direction dv (Eq. 30, BL form)."""
    return -bl.ad_dagger(dv, v, alpha, s) - bl.ad_dagger(v, dv, alpha, s)


def shoot(v0, Nt, alpha, s):
    """Heun integration of BL EPDiff (Eq. 51) from v0 over [0,1].

    Returns (vs, vstar): vs[n] = v~ at t = n dt for n = 0..Nt, and vstar[n]
    = the Heun predictor of step n -> n+1 (the second stage point).
    """
    dt = 1.0 / Nt
    vs = [np.array(v0, dtype=np.complex128)]
    vstar = []
    for n in range(Nt):
        v = vs[-1]
        k1 = epdiff_rhs(v, alpha, s)
        vp = v + dt * k1
        k2 = epdiff_rhs(vp, alpha, s)
        vstar.append(vp)
        vs.append(v + 0.5 * dt * (k1 + k2))
    return vs, vstar


def tangent_shoot(vs, vstar, p, alpha, s):
    """Incremental BL EPDiff (Eq. 30): exact tangent of the Heun shoot, dv(0) = p.

    Returns the list dvs[n], n = 0..Nt.
    """
    Nt = len(vstar)
    dt = 1.0 / Nt
    out = [np.array(p, dtype=np.complex128)]
    for n in range(Nt):
        d = out[-1]
        k1 = epdiff_rhs_tangent(vs[n], d, alpha, s)
        dp = d + dt * k1
        k2 = epdiff_rhs_tangent(vstar[n], dp, alpha, s)
        out.append(d + 0.5 * dt * (k1 + k2))
    return out


def tangent_shoot_stages(vs, vstar, p, alpha, s):
    """``tangent_shoot`` with its stage values: (dvs[n] for n = 0..Nt, dstar[n] =
    the tangent of the predictor v*_n)."""
    Nt = len(vstar)
    dt = 1.0 / Nt
    dvs, dstar = [np.array(p, dtype=np.complex128)], []
    for n in range(Nt):
        d = dvs[-1]
        k1 = epdiff_rhs_tangent(vs[n], d, alpha, s)
        dp = d + dt * k1
        k2 = epdiff_rhs_tangent(vstar[n], dp, alpha, s)
        dstar.append(dp)
        dvs.append(d + 0.5 * dt * (k1 + k2))
    return dvs, dstar


def _G(v, J, dv, alpha, s):
    """Right side of the Jacobi-field tangent: (dv + ad~_v J, linearised EPDiff)."""
    return dv + bl.ad(v, J), epdiff_rhs_tangent(v, dv, alpha, s)


def _GT(v, U, W, alpha, s):
    """V-transpose of ``_G``: (ad~^dagger_v U, U + ad~^dagger_W v - ad~_v W) (Eqs. 53-54)."""
    return (bl.ad_dagger(v, U, alpha, s),
            U + bl.ad_dagger(W, v, alpha, s) - bl.ad(v, W))


def jacobi_tangent(vs, vstar, p, alpha, s):
    """Heun tangent of the Jacobi pair (J, dv), J(0) = 0, dv(0) = p.

    Returns J(1).  This is the linear map whose V-transpose
    ``adjoint_jacobi_backward`` applies; the oracle uses it for the
    transpose identity and the exactly symmetric J-form Hessian.
    """
    Nt = len(vstar)
    dt = 1.0 / Nt
    J = np.zeros_like(p, dtype=np.complex128)
    d = np.array(p, dtype=np.complex128)
    for n in range(Nt):
        a1, b1 = _G(vs[n], J, d, alpha, s)
        Jp, dp = J + dt * a1, d + dt * b1
        a2, b2 = _G(vstar[n], Jp, dp, alpha, s)
        J = J + 0.5 * dt * (a1 + a2)
        d = d + 0.5 * dt * (b1 + b2)
    return J


def adjoint_jacobi_backward(vs, vstar, U1, alpha, s):
    """Backward reduced adjoint Jacobi sweep (Eqs. 53-54; Eqs. 56-57 under GN).

    Starts from (U, W)(1) = (U1, 0) and applies, for n = Nt-1 .. 0, the
    V-transpose of the Heun tangent step of (J, dv):
        a  = G^T_{v*_n}(z_{n+1});   z~ = z_{n+1} + dt a
        b  = G^T_{v_n}(z~);         z_n = z_{n+1} + dt/2 (a + b)
    Returns W(0), the data part of the V-gradient.
    """
    Nt = len(vstar)
    dt = 1.0 / Nt
    U = np.array(U1, dtype=np.complex128)
    W = np.zeros_like(U)
    for n in range(Nt - 1, -1, -1):
        aU, aW = _GT(vstar[n], U, W, alpha, s)
        Ut, Wt = U + dt * aU, W + dt * aW
        bU, bW = _GT(vs[n], Ut, Wt, alpha, s)
        U = U + 0.5 * dt * (aU + bU)
        W = W + 0.5 * dt * (aW + bW)
    return W


def adjoint_jacobi_backward_stages(vs, vstar, U1, alpha, s):
    """``adjoint_jacobi_backward`` with its stage values: (W(0), zs, zt) where
    zs[n] = (U, W) at time level n (n = 0..Nt) and zt[n] = the stage value
    (U~, W~) of step n -> n-1 ... i.e. z~ = z_{n+1} + dt a of step n."""
    Nt = len(vstar)
    dt = 1.0 / Nt
    U = np.array(U1, dtype=np.complex128)
    W = np.zeros_like(U)
    zs = [None] * (Nt + 1)
    zt = [None] * Nt
    zs[Nt] = (U, W)
    for n in range(Nt - 1, -1, -1):
        aU, aW = _GT(vstar[n], U, W, alpha, s)
        Ut, Wt = U + dt * aU, W + dt * aW
        zt[n] = (Ut, Wt)
        bU, bW = _GT(vs[n], Ut, Wt, alpha, s)
        U = U + 0.5 * dt * (aU + bU)
        W = W + 0.5 * dt * (aW + bW)
        zs[n] = (U, W)
    return W, zs, zt


def _Gp(dv, U, W, alpha, s):
    """Derivative of ``_GT`` with respect to its velocity along dv (the terms the
    Gauss-Newton form drops from Eqs. 56-57): (ad~^dagger_dv U,
    ad~^dagger_W dv - ad~_dv W)."""
    return (bl.ad_dagger(dv, U, alpha, s),
            bl.ad_dagger(W, dv, alpha, s) - bl.ad(dv, W))


def newton_backward(vs, vstar, dvs, dstar, zs, zt, dU1, alpha, s):
    """Full-Newton incremental adjoint sweep (Eqs. 56-57 without the Gauss-Newton
    drop): the derivative of the Heun-transposed recursion of
    ``adjoint_jacobi_backward`` along the velocity trajectory's tangent (dvs,
    dstar), started from (dU1, 0); the gradient sweep's stage values (zs, zt)
    carry the dropped terms.  Returns dW(0)."""
    Nt = len(vstar)
    dt = 1.0 / Nt
    dU = np.array(dU1, dtype=np.complex128)
    dW = np.zeros_like(dU)
    for n in range(Nt - 1, -1, -1):
        U, W = zs[n + 1]
        aU, aW = _GT(vstar[n], dU, dW, alpha, s)
        gU, gW = _Gp(dstar[n], U, W, alpha, s)
        aU, aW = aU + gU, aW + gW
        dUt, dWt = dU + dt * aU, dW + dt * aW
        Ut, Wt = zt[n]
        bU, bW = _GT(vs[n], dUt, dWt, alpha, s)
        hU, hW = _Gp(dvs[n], Ut, Wt, alpha, s)
        dU = dU + 0.5 * dt * (aU + bU + hU)
        dW = dW + 0.5 * dt * (aW + bW + hW)
    return dW


# --------------------------------------------------------------------------
# full-grid transport
# --------------------------------------------------------------------------

def interp(f, xi):
    """Multilinear periodic interpolation of grid function f at index coords xi.

    ``f``: array of shape N (d axes).  ``xi``: (d, ...) index coordinates
    (position / h).  Sum over the 2^d cell corners with weights
    prod_j (w_j or 1 - w_j), w_j = xi_j - floor(xi_j).
    """
    Ns = f.shape
    d = len(Ns)
    i0 = [np.floor(xi[j]) for j in range(d)]
    w = [xi[j] - i0[j] for j in range(d)]
    i0 = [i0[j].astype(np.int64) for j in range(d)]
    out = np.zeros(xi.shape[1:])
    for corner in itertools.product((0, 1), repeat=d):
        idx = tuple((i0[j] + corner[j]) % Ns[j] for j in range(d))
        wt = np.ones(xi.shape[1:])
        for j in range(d):
            wt = wt * (w[j] if corner[j] else 1.0 - w[j])
        out = out + wt * f[idx]
    return out


def central_grad(m):
    """Second-order central-difference gradient on the periodic unit grid."""
    Ns = m.shape
    return np.stack([(np.roll(m, -1, axis=j) - np.roll(m, 1, axis=j)) * (Ns[j] / 2.0)
                     for j in range(len(Ns))])


def _index_grid(Ns):
    return np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in Ns],
                                indexing="ij"))


def foot_points(v_next, v_cur, dt):
    """Index coordinates of X_n(x) = x - dt/2 [v_{n+1}(x) + v_n(x - dt v_{n+1}(x))].

    ``v_next``, ``v_cur``: (d, N..) grid velocities at t_{n+1} and t_n.
    """
    Ns = v_next.shape[1:]
    d = len(Ns)
    I = _index_grid(Ns)
    scale = np.array(Ns, dtype=np.float64).reshape((d,) + (1,) * d)
    xi1 = I - dt * v_next * scale
    u = np.stack([interp(v_cur[j], xi1) for j in range(d)])
    return I - 0.5 * dt * (v_next + u) * scale


def interp_adjoint(g, xi, Ns):
    """Transpose of ``interp`` in its grid argument: scatter g(x) with the same
    corner weights onto the grid (the discrete counterpart of the backward
    lambda transport of Eq. 13)."""
    d = len(Ns)
    i0 = [np.floor(xi[j]) for j in range(d)]
    w = [xi[j] - i0[j] for j in range(d)]
    i0 = [i0[j].astype(np.int64) for j in range(d)]
    out = np.zeros(Ns)
    for corner in itertools.product((0, 1), repeat=d):
        idx = tuple(((i0[j] + corner[j]) % Ns[j]).ravel() for j in range(d))
        wt = np.ones(xi.shape[1:])
        for j in range(d):
            wt = wt * (w[j] if corner[j] else 1.0 - w[j])
        np.add.at(out, idx, (wt * g).ravel())
    return out


def interp_gradient(f, xi):
    """Derivatives of the multilinear interpolant of f at index coords xi with
    respect to each coordinate (exact inside a cell; the lower cell's value at
    a node).  Returns (d, ...)."""
    Ns = f.shape
    d = len(Ns)
    i0 = [np.floor(xi[j]) for j in range(d)]
    w = [xi[j] - i0[j] for j in range(d)]
    i0 = [i0[j].astype(np.int64) for j in range(d)]
    out = np.zeros((d,) + xi.shape[1:])
    for corner in itertools.product((0, 1), repeat=d):
        idx = tuple((i0[j] + corner[j]) % Ns[j] for j in range(d))
        fc = f[idx]
        for a in range(d):
            wt = np.ones(xi.shape[1:])
            for j in range(d):
                if j == a:
                    wt = wt * (1.0 if corner[j] else -1.0)
                else:
                    wt = wt * (w[j] if corner[j] else 1.0 - w[j])
            out[a] = out[a] + wt * fc
    return out


def transport_adjoint(ms, vgrid, lam1, dt):
    """Exact reverse-mode derivative of ``transport`` (the discrete adjoint of
    the state equation, Eqs. 12-13).

    ``lam1``: dL/dm_Nt on the grid.  Returns G[n] = dL/dvgrid[n], n = 0..Nt,
    each (d, N..), through every dependence of the semi-Lagrangian step
        xi(x) = x - dt v_{n+1}(x),  u(x) = v_n(xi(x)),
        X(x)  = x - dt/2 [v_{n+1}(x) + u(x)],  m_{n+1}(x) = m_n(X(x))
    (index units: velocities scaled by N_j)."""
    Nt = len(vgrid) - 1
    Ns = ms[0].shape
    d = len(Ns)
    I = _index_grid(Ns)
    scale = np.array(Ns, dtype=np.float64).reshape((d,) + (1,) * d)
    G = [np.zeros((d,) + Ns) for _ in range(Nt + 1)]
    lam = np.array(lam1, dtype=np.float64)
    for n in range(Nt - 1, -1, -1):
        vn, vc = vgrid[n + 1], vgrid[n]
        xi1 = I - dt * vn * scale
        u = np.stack([interp(vc[j], xi1) for j in range(d)])
        X = I - 0.5 * dt * (vn + u) * scale
        mu = lam[None] * interp_gradient(ms[n], X)          # dL/dX
        alpha = -0.5 * dt * scale * mu                       # dL/du and the direct dL/dv_{n+1}
        G[n + 1] += alpha
        beta = np.zeros((d,) + Ns)                           # dL/dxi
        for j in range(d):
            G[n][j] += interp_adjoint(alpha[j], xi1, Ns)
            beta += alpha[j][None] * interp_gradient(vc[j], xi1)
        G[n + 1] += -dt * scale * beta
        lam = interp_adjoint(lam, X, Ns)
    return G


def transpose_shoot(vs, vstar, sources, alpha, s):
    """V-transpose of the Heun shoot tangent with a source at every time level:
    W_Nt = s_Nt;  W_n = T_n^T W_{n+1} + s_n, where T_n^T applies
        a = F'(v*_n)^T W,  W~ = W + dt a,  b = F'(v_n)^T W~,  W + dt/2 (a + b)
    and F'(v)^T W = ad~^dagger_W v - ad~_v W is the W part of ``_GT``.
    Returns W_0."""
    Nt = len(vstar)
    dt = 1.0 / Nt
    W = np.array(sources[Nt], dtype=np.complex128)
    for n in range(Nt - 1, -1, -1):
        _, aW = _GT(vstar[n], np.zeros_like(W), W, alpha, s)
        Wt = W + dt * aW
        _, bW = _GT(vs[n], np.zeros_like(W), Wt, alpha, s)
        W = W + 0.5 * dt * (aW + bW) + sources[n]
    return W


def transport(I0, vgrid, dt):
    """Semi-Lagrangian state transport (Eq. 52): m_{n+1}(x) = m_n(X_n(x)).

    ``vgrid``: list of Nt+1 grid velocities.  Returns the list m_0..m_Nt and
    the foot points xi_0..xi_{Nt-1}.
    """
    ms = [np.array(I0, dtype=np.float64)]
    feet = []
    for n in range(len(vgrid) - 1):
        xi = foot_points(vgrid[n + 1], vgrid[n], dt)
        feet.append(xi)
        ms.append(interp(ms[-1], xi))
    return ms, feet


def incremental_transport(ms, feet, dvgrid, dt):
    """Incremental state equation (Eq. 31) along the same characteristics.

    dm_0 = 0;  with s_n = grad m_n . delta v_n on the grid,
    dm_{n+1}(x) = dm_n(X_n(x)) - dt/2 [ s_n(X_n(x)) + s_{n+1}(x) ].
    Returns dm_Nt.
    """
    s_cur = np.sum(central_grad(ms[0]) * dvgrid[0], axis=0)
    dm = np.zeros_like(ms[0])
    for n in range(len(feet)):
        s_next = np.sum(central_grad(ms[n + 1]) * dvgrid[n + 1], axis=0)
        dm = interp(dm, feet[n]) - 0.5 * dt * (interp(s_cur, feet[n]) + s_next)
        s_cur = s_next
    return dm
