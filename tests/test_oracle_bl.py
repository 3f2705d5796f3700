"""Pins of the oracle's band-limited algebra (Section 3.1) against brute force and closed forms."""

import itertools

import numpy as np
import pytest

from oracle import bl
from paper_1807_11560_gb300 import inputs

ALPHA, S = 0.0025, 2


def _band_modes(Ks):
    """(index tuple, frequency tuple) of every non-Nyquist band slot."""
    out = []
    for q in itertools.product(*[range(K) for K in Ks]):
        f = tuple(qq if qq < K / 2 else qq - K for qq, K in zip(q, Ks))
        if any(K % 2 == 0 and qq == K // 2 for qq, K in zip(q, Ks)):
            continue
        out.append((q, f))
    return out


def _direct_iota(a, Ns):
    """Eq. 46 as a direct sum over the band, no FFT."""
    Ks = a.shape[1:]
    X = np.meshgrid(*[np.arange(n) / n for n in Ns], indexing="ij")
    out = np.zeros((a.shape[0],) + tuple(Ns), dtype=np.complex128)
    for q, f in _band_modes(Ks):
        ph = np.exp(2j * np.pi * sum(fj * xj for fj, xj in zip(f, X)))
        for c in range(a.shape[0]):
            out[c] += a[(c,) + q] * ph
    return out


def _direct_pi(f, Ks):
    Ns = f.shape[1:]
    X = np.meshgrid(*[np.arange(n) / n for n in Ns], indexing="ij")
    out = np.zeros((f.shape[0],) + tuple(Ks), dtype=np.complex128)
    for q, fr in _band_modes(Ks):
        ph = np.exp(-2j * np.pi * sum(fj * xj for fj, xj in zip(fr, X)))
        for c in range(f.shape[0]):
            out[(c,) + q] = np.sum(f[c] * ph) / np.prod(Ns)
    return out


CASES = [((8, 8), (4, 4)), ((7, 6), (4, 6)), ((6, 5, 8), (4, 2, 4)), ((8, 8, 8), (4, 4, 4))]


@pytest.mark.parametrize("Ns,Ks", CASES)
def test_iota_pi_match_direct_sums(Ns, Ks):
    d = len(Ns)
    a = inputs.random_bl(Ks, d, 3, 1.0, Ns) * 50
    ref = _direct_iota(a, Ns)
    assert np.abs(ref.imag).max() < 1e-13 * np.abs(ref).max()       # Hermitian in => real out
    np.testing.assert_allclose(bl.iota(a, Ns), ref.real, atol=1e-13 * np.abs(ref).max())
    rng = np.random.default_rng(4)
    f = rng.normal(size=(2,) + tuple(Ns))
    np.testing.assert_allclose(bl.pi(f, Ks), _direct_pi(f, Ks), atol=1e-14)


@pytest.mark.parametrize("Ns,Ks", CASES + [((64, 48), (16, 16))])
def test_pi_iota_identity_and_adjoint(Ns, Ks):
    d = len(Ns)
    a = inputs.random_bl(Ks, d, 5, 1.0, Ns)
    np.testing.assert_allclose(bl.pi(bl.iota(a, Ns), Ks), a, atol=1e-15 * 1 + 1e-13 * np.abs(a).max())
    rng = np.random.default_rng(6)
    f = rng.normal(size=(d,) + tuple(Ns))
    lhs = np.sum(bl.iota(a, Ns) * f) / np.prod(Ns)       # <iota a, f>_{L2_h}
    rhs = bl.inner_l2(a, bl.pi(f, Ks))                    # <a, pi f>_{l2}
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.abs(a).max())


def test_nyquist_slot_ignored_and_lhat():
    Ks, Ns = (4, 4), (8, 8)
    a = inputs.random_bl(Ks, 2, 1, 1.0, Ns)
    b = a.copy()
    b[:, 2, :] = 7.0 + 3j
    np.testing.assert_array_equal(bl.iota(a, Ns), bl.iota(b, Ns))
    L = bl.lhat((6, 4), 0.01, 3)
    assert L[0, 0] == 1.0
    assert np.isclose(L[1, 3], (1 + 4 * np.pi ** 2 * 0.01 * (1 + 1)) ** 3)
    assert np.isclose(L[5, 2], (1 + 4 * np.pi ** 2 * 0.01 * (1 + 4)) ** 3)


def _brute_ad_star(v, m):
    """Truncated convolution written as a frequency-domain double sum:
    P^(k) = sum_{k1+k2=k} [ sum_j (2 pi i k1_i) v_j(k1) m_j(k2) + sum_j (2 pi i k2_j) m_i(k2) v_j(k1)
                            + m_i(k2) sum_j (2 pi i k1_j) v_j(k1) ]."""
    d = v.shape[0]
    Ks = v.shape[1:]
    modes = _band_modes(Ks)
    lut = {f: q for q, f in modes}
    out = np.zeros_like(v)
    for q1, f1 in modes:
        for q2, f2 in modes:
            fk = tuple(a + b for a, b in zip(f1, f2))
            if fk not in lut:
                continue
            qk = lut[fk]
            div = sum(2j * np.pi * f1[j] * v[(j,) + q1] for j in range(d))
            for i in range(d):
                t = m[(i,) + q2] * div
                for j in range(d):
                    t += 2j * np.pi * f1[i] * v[(j,) + q1] * m[(j,) + q2]
                    t += 2j * np.pi * f2[j] * m[(i,) + q2] * v[(j,) + q1]
                out[(i,) + qk] += t
    return out


@pytest.mark.parametrize("Ks", [(6, 6), (4, 4, 4)])
def test_ad_star_equals_bruteforce_convolution(Ks):
    d = len(Ks)
    Ns = tuple(2 * k for k in Ks)
    v = inputs.random_bl(Ks, d, 8, 1.0, Ns)
    m = inputs.random_bl(Ks, d, 9, 1.0, Ns)
    ref = _brute_ad_star(v, m)
    got = bl.ad_star(v, m)
    np.testing.assert_allclose(got, ref, atol=1e-13 * np.abs(ref).max())


def test_truncated_convolution_independent_of_padding():
    Ks = (8, 6, 4)
    Ns = (16, 16, 16)
    v = inputs.random_bl(Ks, 3, 10, 1.0, Ns)
    m = inputs.random_bl(Ks, 3, 11, 1.0, Ns)
    r0 = bl.ad_star(v, m)                       # M = ceil(3K/2)
    for Ms in [(16, 12, 8), (13, 11, 7), Ns]:
        np.testing.assert_allclose(bl.ad_star(v, m, Ms), r0, atol=1e-13 * np.abs(r0).max())
        np.testing.assert_allclose(bl.ad(v, m, Ms), bl.ad(v, m), atol=1e-13 * np.abs(r0).max())


def test_ad_identities():
    Ks, Ns = (8, 8, 8), (12, 12, 12)
    v, u, w = (inputs.random_bl(Ks, 3, s_, 1.0, Ns) for s_ in (20, 21, 22))
    scale = np.abs(bl.ad(v, w)).max()
    assert np.abs(bl.ad(v, v)).max() <= 1e-14 * scale                    # ad_v v = 0
    np.testing.assert_allclose(bl.ad(v, w), -bl.ad(w, v), atol=1e-14 * scale)
    lhs = bl.inner_V(bl.ad_dagger(v, u, ALPHA, S), w, ALPHA, S)          # <ad^dag_v u, w>_V
    rhs = bl.inner_V(u, bl.ad(v, w), ALPHA, S)                           # <u, ad_v w>_V
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = bl.inner_l2(bl.ad_star(v, u), w)                               # <ad*_v m, w>_l2
    rhs = bl.inner_l2(u, bl.ad(v, w))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    L = bl.lhat(Ks, ALPHA, S)
    np.testing.assert_allclose((1.0 / L) * L, 1.0)


def _cos_mode(Ks, comp, axis, k, amp):
    """BL field amp*cos(2 pi k x_axis) e_comp."""
    d = len(Ks)
    a = np.zeros((d,) + Ks, dtype=np.complex128)
    idx = [0] * d
    idx[axis] = k
    a[(comp,) + tuple(idx)] += amp / 2
    idx[axis] = (-k) % Ks[axis]
    a[(comp,) + tuple(idx)] += amp / 2
    return a


def _sin_mode(Ks, comp, axis, k, amp):
    d = len(Ks)
    a = np.zeros((d,) + Ks, dtype=np.complex128)
    idx = [0] * d
    idx[axis] = k
    a[(comp,) + tuple(idx)] += amp / (2j)
    idx[axis] = (-k) % Ks[axis]
    a[(comp,) + tuple(idx)] -= amp / (2j)
    return a


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_ad_dagger_single_mode_closed_forms(k):
    """Hand-derived from Eq. 4: for v = a cos(2 pi k x1) e1 (compression wave)
    the bracket of Eq. 48 is -3 pi k a^2 Lhat(k) sin(4 pi k x1) e1; for the shear
    v = a cos(2 pi k x2) e1 it is -pi k a^2 Lhat(k) sin(4 pi k x2) e2.  ad^dagger
    divides by Lhat(2k) when 2k is inside the band and is zero otherwise."""
    Ks = (12, 12)
    a = 0.3
    Lk = (1 + 4 * np.pi ** 2 * ALPHA * k * k) ** S
    L2k = (1 + 4 * np.pi ** 2 * ALPHA * 4 * k * k) ** S
    inband = 2 * k < Ks[0] / 2
    v = _cos_mode(Ks, 0, 0, k, a)
    got = bl.ad_dagger(v, v, ALPHA, S)
    want = _sin_mode(Ks, 0, 0, 2 * k, -3 * np.pi * k * a * a * Lk / L2k) if inband else 0 * v
    np.testing.assert_allclose(got, want, atol=1e-13)
    v = _cos_mode(Ks, 0, 1, k, a)
    got = bl.ad_dagger(v, v, ALPHA, S)
    want = _sin_mode(Ks, 1, 1, 2 * k, -np.pi * k * a * a * Lk / L2k) if inband else 0 * v
    np.testing.assert_allclose(got, want, atol=1e-13)


def test_ad_single_mode_closed_form():
    """v = a cos(2 pi k x1) e1, w = c cos(2 pi l x1) e2: by Eq. 49,
    ad_v w = pi l a c [sin(2 pi (l+k) x1) + sin(2 pi (l-k) x1)] e2, truncated to the band."""
    Ks = (12, 12)
    a, c, k, l = 0.7, -0.4, 1, 3
    v = _cos_mode(Ks, 0, 0, k, a)
    w = _cos_mode(Ks, 1, 0, l, c)
    want = _sin_mode(Ks, 1, 0, l + k, np.pi * l * a * c) + _sin_mode(Ks, 1, 0, l - k, np.pi * l * a * c)
    np.testing.assert_allclose(bl.ad(v, w), want, atol=1e-13)
    # l + k outside the band: only the difference frequency survives
    l = 5
    w = _cos_mode(Ks, 1, 0, l, c)
    want = _sin_mode(Ks, 1, 0, l - k, np.pi * l * a * c)
    np.testing.assert_allclose(bl.ad(v, w), want, atol=1e-13)


def test_hermitian_part_is_what_iota_keeps():
    Ks, Ns = (6, 4, 4), (8, 8, 8)
    rng = np.random.default_rng(3)
    a = rng.normal(size=(3,) + Ks) + 1j * rng.normal(size=(3,) + Ks)
    np.testing.assert_allclose(bl.iota(a, Ns), bl.iota(bl.hermitian_part(a), Ns), atol=1e-12)
    h = bl.hermitian_part(a)
    np.testing.assert_allclose(bl.pi(bl.iota(h, Ns), Ks), h, atol=1e-13)
