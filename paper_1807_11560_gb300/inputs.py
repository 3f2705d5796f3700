"""Seeded synthetic inputs: phantoms, targets, band-limited fields.

This module holds no arithmetic of the registration method.  It only draws
random numbers (numpy PCG64 ``default_rng``) and evaluates closed-form
phantom functions, so the oracle and the GPU library can both be fed from it.

The paper's data (NIREP brain volumes, Section 4) are not available; the
phantoms below stand in for them with the shapes of the benchmark workloads:

* ``blobs_2d``: sum of 8 Gaussian blobs (centres uniform, widths U[3,8] px,
  amplitudes U[0,1]), clipped to [0,1].
* ``ellipsoids_3d``: 20 Gaussian ellipsoids (semi-axes U[3,10] voxels, random
  rotation, amplitudes U[0,1]) plus N(0, 0.02^2) noise smoothed by a unit
  Gaussian.
  On grids smaller than 64 per axis the blob widths and semi-axes shrink by
  min(N)/64 so that small test images are not saturated.
* ``brain_3d``: nested ellipsoidal shells at intensities 0.8/0.5/0.2 whose outer
  boundary is folded by 1 + 0.06 sin(7 theta) sin(9 phi), Gaussian-smoothed
  (sigma = 1 voxel) -- a cortex-like test volume.

A target is the same closed-form phantom evaluated at warped coordinates
x - u(x), u a smooth random displacement made of a few sinusoidal modes with
a maximum of ``max_disp`` voxels.

All arrays are float64 C-order with axis 0 the slowest.  Band-limited fields
are complex128 arrays (d, K_1..K_d) in FFT order with the Nyquist slots zero
and Hermitian symmetry, as the library's C interface expects.
"""

import numpy as np

__all__ = [
    "blobs_2d", "ellipsoids_3d", "brain_3d", "random_bl", "smooth_displacement",
    "make_pair", "WORKLOADS",
]


def _coords(Ns):
    return np.meshgrid(*[np.arange(n, dtype=np.float64) for n in Ns], indexing="ij")


def smooth_displacement(Ns, rng, max_disp, n_modes=6):
    """Random smooth periodic displacement (in voxels), max |u_j| = max_disp."""
    d = len(Ns)
    X = _coords(Ns)
    u = []
    for _ in range(d):
        comp = np.zeros(Ns)
        for _m in range(n_modes):
            kvec = rng.integers(0, 3, size=d)
            if not kvec.any():
                kvec[rng.integers(0, d)] = 1
            ph = rng.uniform(0, 2 * np.pi)
            amp = rng.normal()
            arg = sum(2 * np.pi * kvec[j] * X[j] / Ns[j] for j in range(d)) + ph
            comp += amp * np.sin(arg)
        m = np.abs(comp).max()
        u.append(comp * (max_disp / m if m > 0 else 0.0))
    return np.stack(u)


def _gauss_smooth(img, sigma):
    """Separable periodic Gaussian smoothing (sigma in voxels)."""
    out = img
    r = int(np.ceil(3 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma) ** 2)
    w /= w.sum()
    for ax in range(img.ndim):
        if img.shape[ax] == 1:
            continue
        acc = np.zeros_like(out)
        for o, wt in zip(t.astype(int), w):
            acc += wt * np.roll(out, o, axis=ax)
        out = acc
    return out


def _blob_params(rng, Ns, n):
    c = np.stack([rng.uniform(0, N, size=n) for N in Ns], axis=1)
    wid = rng.uniform(3, 8, size=n) * min(1.0, min(Ns) / 64.0)
    amp = rng.uniform(0, 1, size=n)
    return c, wid, amp


def _eval_blobs(X, Ns, params):
    c, wid, amp = params
    img = np.zeros(X[0].shape)
    for b in range(len(amp)):
        r2 = 0.0
        for j, N in enumerate(Ns):
            dx = (X[j] - c[b, j] + N / 2) % N - N / 2  # periodic distance
            r2 = r2 + dx * dx
        img += amp[b] * np.exp(-r2 / (2 * wid[b] ** 2))
    return np.clip(img, 0.0, 1.0)


def blobs_2d(Ns, seed, warp=None):
    rng = np.random.default_rng(seed)
    params = _blob_params(rng, Ns, 8)
    X = _coords(Ns)
    if warp is not None:
        X = [X[j] - warp[j] for j in range(len(Ns))]
    return _eval_blobs(X, Ns, params)


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def ellipsoids_3d(Ns, seed, warp=None, noise_seed=None):
    rng = np.random.default_rng(seed)
    n = 20
    c = np.stack([rng.uniform(0, N, size=n) for N in Ns], axis=1)
    axes = rng.uniform(3, 10, size=(n, 3)) * min(1.0, min(Ns) / 64.0)
    rots = [_rotation(rng) for _ in range(n)]
    amp = rng.uniform(0, 1, size=n)
    X = _coords(Ns)
    if warp is not None:
        X = [X[j] - warp[j] for j in range(3)]
    img = np.zeros(Ns)
    for b in range(n):
        dx = [(X[j] - c[b, j] + Ns[j] / 2) % Ns[j] - Ns[j] / 2 for j in range(3)]
        r2 = 0.0
        for a in range(3):
            y = rots[b][0, a] * dx[0] + rots[b][1, a] * dx[1] + rots[b][2, a] * dx[2]
            r2 = r2 + (y / axes[b, a]) ** 2
        img += amp[b] * np.exp(-0.5 * r2 * 4.0)
    nrng = np.random.default_rng(seed + 7919 if noise_seed is None else noise_seed)
    img += _gauss_smooth(nrng.normal(0.0, 0.02, size=Ns), 1.0)
    return img


def brain_3d(Ns, seed, warp=None):
    rng = np.random.default_rng(seed)
    ph_t, ph_p = rng.uniform(0, 2 * np.pi, size=2)
    X = _coords(Ns)
    if warp is not None:
        X = [X[j] - warp[j] for j in range(3)]
    semi = (0.40, 0.47, 0.36)
    y = [(X[j] - Ns[j] / 2.0) / (semi[j] * Ns[j]) for j in range(3)]
    r = np.sqrt(y[0] ** 2 + y[1] ** 2 + y[2] ** 2)
    theta = np.arccos(np.clip(y[2] / np.maximum(r, 1e-12), -1, 1))
    phi = np.arctan2(y[1], y[0])
    rho = 1.0 + 0.06 * np.sin(7 * theta + ph_t) * np.sin(9 * phi + ph_p)
    img = np.where(r < 0.55 * rho, 0.8, np.where(r < 0.8 * rho, 0.5, np.where(r < rho, 0.2, 0.0)))
    return _gauss_smooth(img, 1.0)


def random_bl(Ks, d, seed, max_disp_vox, Ns, decay=2.0):
    """Random Hermitian band-limited vector field, FFT order, Nyquist slots zero.

    Coefficients ~ (N(0,1) + i N(0,1)) / (1 + |k|^2)^decay, symmetrised, then
    scaled so that the sum of coefficient moduli of each component -- an upper
    bound of the field's maximum -- equals max_disp_vox / N_j.
    """
    rng = np.random.default_rng(seed)
    Ks = tuple(int(k) for k in Ks)
    f = [np.where(np.arange(K) < K / 2.0, np.arange(K), np.arange(K) - K) for K in Ks]
    F = np.meshgrid(*f, indexing="ij")
    k2 = sum(x.astype(np.float64) ** 2 for x in F)
    a = (rng.normal(size=(d,) + Ks) + 1j * rng.normal(size=(d,) + Ks)) / (1.0 + k2) ** decay
    # Hermitian symmetrisation and Nyquist zeroing
    flip = a
    for ax, K in enumerate(Ks, start=1):
        flip = np.take(flip, (-np.arange(K)) % K, axis=ax)
    a = 0.5 * (a + np.conj(flip))
    for j, K in enumerate(Ks):
        if K % 2 == 0 and K > 1:
            idx = [slice(None)] * (d + 1)
            idx[j + 1] = K // 2
            a[tuple(idx)] = 0.0
    for c in range(d):
        tot = np.abs(a[c]).sum()
        if tot > 0:
            a[c] *= (max_disp_vox / Ns[c]) / tot
    return a


# name -> (kind, grid, band, Nt, seed); kinds select the phantom generator
WORKLOADS = {
    "2d_64_blobs": ("blobs", (64, 64), (16, 16), 10, 1807),
    "3d_64_ellipsoids": ("ellipsoids", (64, 64, 64), (16, 16, 16), 10, 1808),
    "3d_160x192x160_brain": ("brain", (160, 192, 160), (32, 32, 32), 10, 1809),
    "3d_96_brain": ("brain", (96, 96, 96), (24, 24, 24), 16, 1810),
}


def population(n=32, seed=3000):
    """The batched population-to-atlas workload: n brain-phantom pairs, pair i with
    a grid drawn uniformly from {96^3, 128^3, 160x192x160} and a band from
    {24^3, 32^3} (both draws from `seed`), pair seed seed + 1 + i, Nt = 10.
    Entries have the WORKLOADS layout (kind, grid, band, Nt, seed)."""
    rng = np.random.default_rng(seed)
    grids = [(96, 96, 96), (128, 128, 128), (160, 192, 160)]
    bands = [(24, 24, 24), (32, 32, 32)]
    out = []
    for i in range(n):
        g = grids[int(rng.integers(len(grids)))]
        k = bands[int(rng.integers(len(bands)))]
        out.append(("brain", g, k, 10, seed + 1 + i))
    return out


def make_pair(kind, Ns, seed, max_disp=3.0):
    """(I0, I1): a phantom and its analytically warped copy."""
    Ns = tuple(int(n) for n in Ns)
    rng = np.random.default_rng(seed + 104729)
    u = smooth_displacement(Ns, rng, max_disp)
    if kind == "blobs":
        return blobs_2d(Ns, seed), blobs_2d(Ns, seed, warp=u)
    if kind == "ellipsoids":
        return (ellipsoids_3d(Ns, seed),
                ellipsoids_3d(Ns, seed, warp=u, noise_seed=seed + 15485863))
    if kind == "brain":
        return brain_3d(Ns, seed), brain_3d(Ns, seed, warp=u)
    raise ValueError(kind)
