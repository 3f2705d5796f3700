"""Band-limited vector-field algebra, Section 3.1 of Hernandez, arXiv:1807.11560.

TEST INFRASTRUCTURE ONLY (see the package docstring).  FP64 throughout.

Conventions (the readings the whole library shares):

* Domain: the periodic unit box [0,1)^d, grid N = (N_1..N_d), spacing h_j = 1/N_j,
  node x_i = i*h.  The discrete L2 product is <f,g>_{L2} = h^d * sum_x f g.
* A band-limited (BL) field is an array ``a`` of shape (d, K_1, .., K_d),
  complex, index q_j stored in FFT order; its signed frequency is
  f_j(q) = q if q < K_j/2 else q - K_j.  The slot q_j = K_j/2 (frequency
  -K_j/2, the Nyquist slot) is held at zero, so the band is symmetric and a
  Hermitian array maps to a real field.  (Eq. 46 prints the sum from 0 to K,
  which cannot produce a real field; this symmetric band is the reading.)
* iota (Eq. 46): iota(a)(x) = sum_k a(k) exp(2 pi i k.x), evaluated on a grid.
  pi: pi(f)(k) = N^-d sum_x f(x) exp(-2 pi i k.x), kept on the band.  Then
  pi(iota(a)) = a and pi is the adjoint of iota between (l2, L2_h).
* L~ has the symbol Lhat(k) = (1 + 4 pi^2 alpha |k|^2)^s of L = (Id - alpha Lap)^s
  (Eq. 1); K~ has 1/Lhat.  Spectral derivative: D_j a = 2 pi i f_j a.
* <a,b>_{l2} = Re sum conj(a) b;  <a,b>_V = <L~ a, b>_{l2} (Eq. 47).
* Truncated convolution (the star of Section 3.1): the product of two BL fields
  is formed on a padded grid M_j >= ceil(3 K_j / 2) and projected back onto the
  band; on such a grid no product frequency aliases into the band, so the
  result is the exact truncated convolution and does not depend on M.
"""

import numpy as np

__all__ = [
    "freqs", "nyquist_mask", "lhat", "embed_index", "iota", "pi", "deriv",
    "hermitian_part", "ad_star", "ad", "ad_dagger", "inner_l2", "inner_V",
    "pad_grid",
]


def freqs(K):
    """Signed frequency of each band slot of one axis, FFT order (Section 3.1)."""
    q = np.arange(K)
    return np.where(q < K / 2.0, q, q - K).astype(np.float64)


def nyquist_mask(Ks):
    """1 on the band, 0 on every Nyquist slot (q_j = K_j/2 for even K_j)."""
    m = np.ones(tuple(Ks))
    for j, K in enumerate(Ks):
        if K % 2 == 0 and K > 1:
            idx = [slice(None)] * len(Ks)
            idx[j] = K // 2
            m[tuple(idx)] = 0.0
    return m


def _freq_grids(Ks):
    return np.meshgrid(*[freqs(K) for K in Ks], indexing="ij")


def lhat(Ks, alpha, s):
    """Symbol of L~ on the band: (1 + 4 pi^2 alpha |k|^2)^s (Eq. 1, Eq. 47)."""
    k2 = sum(f * f for f in _freq_grids(Ks))
    return (1.0 + 4.0 * np.pi ** 2 * alpha * k2) ** s


def embed_index(K, N):
    """Position of each band slot of one axis inside a length-N spectrum."""
    return (freqs(K).astype(np.int64)) % N


def iota(a, Ns):
    """BL -> grid (Eq. 46), exact Fourier sum on the grid Ns via inverse FFT.

    ``a``: (c, K_1..K_d) complex (any number c of scalar fields).
    Returns (c, N_1..N_d) real: the real part of the sum, which is the sum
    itself for a Hermitian ``a``.  Nyquist slots are treated as zero.
    """
    a = np.asarray(a, dtype=np.complex128)
    Ks = a.shape[1:]
    Ns = tuple(int(n) for n in Ns)
    am = a * nyquist_mask(Ks)
    out = np.empty((a.shape[0],) + Ns)
    ix = np.ix_(*[embed_index(K, N) for K, N in zip(Ks, Ns)])
    scale = float(np.prod(Ns))
    for c in range(a.shape[0]):
        S = np.zeros(Ns, dtype=np.complex128)
        S[ix] = am[c]
        out[c] = (np.fft.ifftn(S) * scale).real
    return out


def pi(f, Ks):
    """Grid -> BL projection, N^-d sum_x f(x) exp(-2 pi i k.x) on the band.

    ``f``: (c, N_1..N_d) real.  Returns (c, K_1..K_d) complex, Nyquist zeroed.
    """
    f = np.asarray(f, dtype=np.float64)
    Ns = f.shape[1:]
    Ks = tuple(int(k) for k in Ks)
    ix = np.ix_(*[embed_index(K, N) for K, N in zip(Ks, Ns)])
    mask = nyquist_mask(Ks)
    scale = 1.0 / float(np.prod(Ns))
    out = np.empty((f.shape[0],) + Ks, dtype=np.complex128)
    for c in range(f.shape[0]):
        out[c] = np.fft.fftn(f[c])[ix] * scale * mask
    return out


def deriv(a, j):
    """Spectral derivative along axis j of every scalar field in ``a``."""
    Ks = a.shape[1:]
    fj = _freq_grids(Ks)[j]
    return a * (2j * np.pi * fj)


def hermitian_part(a):
    """(a(k) + conj(a(-k)))/2 with Nyquist slots zeroed: the field iota keeps."""
    Ks = a.shape[1:]
    flip = a
    for ax, K in enumerate(Ks, start=1):
        idx = (-np.arange(K)) % K
        flip = np.take(flip, idx, axis=ax)
    return 0.5 * (a + np.conj(flip)) * nyquist_mask(Ks)


def pad_grid(Ks):
    """Padded product grid M_j = ceil(3 K_j / 2) (1 for a degenerate axis)."""
    return tuple(1 if K == 1 else int(np.ceil(1.5 * K)) for K in Ks)


def _fields_on(a, Ms):
    """Grid values of a BL vector field and of its Jacobian on grid Ms.

    Returns (val[i], jac[i][j]) with jac[i][j] = d_j a_i.
    """
    d = a.shape[0]
    val = iota(a, Ms)
    jac = [[None] * d for _ in range(d)]
    for j in range(d):
        dj = iota(deriv(a, j), Ms)
        for i in range(d):
            jac[i][j] = dj[i]
    return val, jac


def ad_star(v, m, Ms=None):
    """Coadjoint action on the band: pi[(Dv)^T m + D(m) v + m div v] (Eq. 4, Eq. 48).

    Component i of the bracketed field is
        sum_j (d_i v_j) m_j + sum_j (d_j m_i) v_j + m_i sum_j d_j v_j,
    every product formed on the padded grid ``Ms`` (the truncated convolution).
    """
    Ks = v.shape[1:]
    d = v.shape[0]
    Ms = pad_grid(Ks) if Ms is None else tuple(Ms)
    vv, dv = _fields_on(v, Ms)
    mm, dm = _fields_on(m, Ms)
    div = sum(dv[j][j] for j in range(d))
    P = np.empty((d,) + tuple(Ms))
    for i in range(d):
        acc = mm[i] * div
        for j in range(d):
            acc = acc + dv[j][i] * mm[j] + dm[i][j] * vv[j]
        P[i] = acc
    return pi(P, Ks)


def ad(v, w, Ms=None):
    """Adjoint action on the band: pi[Dv.w - Dw.v] (Eq. 49).

    Component i is sum_j (d_j v_i) w_j - (d_j w_i) v_j.
    """
    Ks = v.shape[1:]
    d = v.shape[0]
    Ms = pad_grid(Ks) if Ms is None else tuple(Ms)
    vv, dv = _fields_on(v, Ms)
    ww, dw = _fields_on(w, Ms)
    Q = np.empty((d,) + tuple(Ms))
    for i in range(d):
        acc = np.zeros(tuple(Ms))
        for j in range(d):
            acc = acc + dv[i][j] * ww[j] - dw[i][j] * vv[j]
        Q[i] = acc
    return pi(Q, Ks)


def ad_dagger(v, u, alpha, s, Ms=None):
    """ad~^dagger_v u = K~ ad~*_v (L~ u): the V-adjoint of ad~_v (Eq. 4, Eq. 48)."""
    L = lhat(v.shape[1:], alpha, s)
    return ad_star(v, L * u, Ms) / L


def inner_l2(a, b):
    """<a,b>_{l2} = Re sum conj(a) b over all components and band slots."""
    return float(np.real(np.vdot(a, b)))


def inner_V(a, b, alpha, s):
    """<a,b>_V = <L~ a, b>_{l2} (Eq. 47)."""
    L = lhat(a.shape[1:], alpha, s)
    return float(np.real(np.vdot(L * a, b)))
