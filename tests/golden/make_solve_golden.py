#!/usr/bin/env python3
"""Writes the stored expected values of the 3D Gauss-Newton-Krylov solve parity
tests (tests/test_gpu_solve3d.py) by running the FP64 oracle's solve.

Calls only the oracle (oracle/) and the seeded input generators; nothing here
comes from the CUDA path.  The images are the generator's phantoms rounded to
float32 (the values the FP32 library receives), the solve starts at v0 = 0 and
follows Eqs. 44-45 (Armijo c = 1e-4, at most 10 halvings, PCG tolerance 1e-12).

    python tests/golden/make_solve_golden.py [3d_64_ellipsoids|3d_160x192x160_brain ...]
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import objective  # noqa: E402
from paper_1807_11560_gb300 import inputs  # noqa: E402

ALPHA, S, SIGMA = 0.0025, 2, 0.03
# case -> (workload, GN iterations, PCG iterations per GN iteration)
CASES = {"3d_64_ellipsoids": ("3d_64_ellipsoids", 10, 20),
         "3d_64_ellipsoids_pcg3": ("3d_64_ellipsoids", 10, 3),
         "3d_160x192x160_brain": ("3d_160x192x160_brain", 2, 3)}


def path(name):
    return os.path.join(HERE, f"solve_{name}.npz")


def make(name):
    wl, n_gn, n_pcg = CASES[name]
    kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[wl]
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    I0 = I0.astype(np.float32).astype(np.float64)
    I1 = I1.astype(np.float32).astype(np.float64)
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    t0 = time.time()
    v, rep = P.gn_solve(np.zeros((3,) + tuple(Ks), np.complex128), n_gn, n_pcg)
    # per GN iteration: the iterate after it, and the Armijo margin of every trial
    # (bound - trial energy, relative to E; accepted when >= 0)
    margins = [[(b - Et) / E for (_, Et, b), E in zip(tr, [rep["E"][i]] * len(tr))]
               for i, tr in enumerate(rep["trials"])]
    width = max(len(m) for m in margins)
    marg = np.full((len(margins), width), np.nan)
    for i, m in enumerate(margins):
        marg[i, :len(m)] = m
    np.savez_compressed(path(name), v=v, v_hist=np.array(rep["v_hist"]), E=np.array(rep["E"]),
                        eps=np.array(rep["eps"]), pcg_iters=np.array(rep["pcg_iters"]),
                        gnorm=np.array(rep["gnorm"]), E_final=rep["E_final"], ls_failed=rep["ls_failed"],
                        armijo_margin=marg, n_gn=n_gn, n_pcg=n_pcg)
    print(f"{name}: {n_gn} GN x {n_pcg} PCG in {time.time() - t0:.0f} s, E {rep['E'][0]:.6g} -> "
          f"{rep['E_final']:.6g}, eps {rep['eps']}", flush=True)
    print("Armijo margins (relative to E) per iteration:", flush=True)
    for i, m in enumerate(margins):
        print(f"  {i}: " + ", ".join(f"{x:+.2e}" for x in m), flush=True)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        make(name)
