"""Parity of the whole 3D Gauss-Newton-Krylov solve (Eqs. 44-45) with the FP64
oracle's solve at the benchmark configurations.

The oracle's solves take minutes on one host core, so their results are stored
values written by tests/golden/make_solve_golden.py (oracle only): the iterate
after every Gauss-Newton iteration, the energies, the accepted Armijo steps and
the margin of every Armijo test.

A long solve is sensitive to rounding: with 20 PCG iterations per GN step the
conjugate-gradient iterates on the paper-form Gauss-Newton operator (not
exactly symmetric, Section 2.7 and the gap of the reduced gradient) amplify
rounding differences, so two correct implementations that differ only in
summation order drift apart over the GN iterations.  The tests therefore check
  * FP32, 3 PCG iterations per GN step (the 64^3 config over 10 GN iterations,
    the 160x192x160 config over 2): the same PCG counts and accepted steps, the
    energy history within 1e-4 and m(1) within 1e-4 (norm and element-wise);
  * FP64, the benchmark's 20 PCG iterations: the same accepted steps over the
    first three GN iterations, their energies within 1e-4 and m(1) after them
    within 1e-4 of the oracle's (measured: FP64 library and FP64 oracle, whose
    products agree to 1e-12, differ by 2e-6 in E after 3 iterations, 1e-4
    after 5 and 3e-3 after 10);
  * FP32, 20 PCG iterations over the whole 10-iteration solve: monotone
    descent to a final energy and image mismatch within 5% of the oracle's
    (the trajectories differ from the first PCG solve on; how far is printed).
"""

import os

import numpy as np
import pytest

from helpers import ALPHA, S, SIGMA, host, quantise, rel_2, rel_V, torch_dev
from oracle import objective
from paper_1807_11560_gb300 import Context, inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = {"3d_64_ellipsoids": "3d_64_ellipsoids", "3d_64_ellipsoids_pcg3": "3d_64_ellipsoids",
         "3d_160x192x160_brain": "3d_160x192x160_brain"}


def _setup(case, precision):
    ref = np.load(os.path.join(GOLDEN, f"solve_{case}.npz"))
    kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[CASES[case]]
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision=precision)
    ctx.set_images(torch_dev(I0, precision), torch_dev(I1, precision))
    P = objective.Problem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    return ref, ctx, P, Ns, Ks


def _solve(ctx, Ns, Ks, precision, n_gn, n_pcg):
    import torch
    ct = torch.complex64 if precision == "fp32" else torch.complex128
    rt = torch.float32 if precision == "fp32" else torch.float64
    v = torch.zeros((3,) + tuple(Ks), dtype=ct, device="cuda")
    rep = ctx.gn_solve(v, n_gn, n_pcg)
    m1 = torch.empty(tuple(Ns), dtype=rt, device="cuda")
    ctx.transport(v, m1)
    return rep, host(v), host(m1)


def _check_prefix(name, ref, rep, v, m1, P, Ks, n):
    assert not rep["ls_failed"]
    assert rep["gn_iters"] == n
    assert rep["pcg"][:n] == [int(k) for k in ref["pcg_iters"][:n]]
    assert rep["eps"] == [float(e) for e in ref["eps"][:n]]
    np.testing.assert_allclose(rep["E"][:n], ref["E"][:n], rtol=1e-4)
    v_ref = ref["v_hist"][n - 1]
    m1_ref = P.forward(v_ref)[3][-1]
    E_ref = 0.5 * P.inner_V(v_ref, v_ref) + P.data_term(m1_ref)
    e_m1, e_v = rel_2(m1, m1_ref), rel_V(v, v_ref, Ks)
    print(f"{name}: {n} GN iterations; m(1) rel. err {e_m1:.2e}, v0 rel. err {e_v:.2e}, "
          f"E {rep['E'][0]:.7g} -> {rep['E_final']:.7g} (oracle {E_ref:.7g})")
    assert abs(rep["E_final"] - E_ref) / E_ref < 1e-4
    assert e_m1 < 1e-4


@pytest.mark.parametrize("case", ["3d_64_ellipsoids_pcg3", "3d_160x192x160_brain"])
def test_fp32_gn_solve_matches_stored_oracle_solve(case):
    ref, ctx, P, Ns, Ks = _setup(case, "fp32")
    n, n_pcg = int(ref["n_gn"]), int(ref["n_pcg"])
    with ctx:
        rep, v, m1 = _solve(ctx, Ns, Ks, "fp32", n, n_pcg)
    _check_prefix(f"{case} fp32", ref, rep, v, m1, P, Ks, n)


def test_fp64_gn_solve_at_20_pcg_matches_stored_oracle_solve():
    case = "3d_64_ellipsoids"
    ref, ctx, P, Ns, Ks = _setup(case, "fp64")
    n = 3
    with ctx:
        rep, v, m1 = _solve(ctx, Ns, Ks, "fp64", n, int(ref["n_pcg"]))
    _check_prefix(f"{case} fp64", ref, rep, v, m1, P, Ks, n)


def test_fp32_gn_solve_at_20_pcg_reaches_the_oracle_solution_quality():
    case = "3d_64_ellipsoids"
    ref, ctx, P, Ns, Ks = _setup(case, "fp32")
    n, n_pcg = int(ref["n_gn"]), int(ref["n_pcg"])
    with ctx:
        rep, v, m1 = _solve(ctx, Ns, Ks, "fp32", n, n_pcg)
    v_ref = ref["v_hist"][-1]
    m1_ref = P.forward(v_ref)[3][-1]
    E = np.array(rep["E"] + [rep["E_final"]])
    E_ref = float(ref["E_final"])
    mse, mse_ref = P.mse_rel(m1), P.mse_rel(m1_ref)
    print(f"{case} fp32 10 x 20: E {E[0]:.7g} -> {E[-1]:.7g} (oracle {E_ref:.7g}), MSE_rel {mse:.4f}% "
          f"(oracle {mse_ref:.4f}%), steps {rep['eps']} (oracle {list(ref['eps'])}), "
          f"v0 rel. diff {rel_V(v, v_ref, Ks):.2e}, m(1) rel. diff {rel_2(m1, m1_ref):.2e}")
    assert rep["gn_iters"] == n and not rep["ls_failed"]
    assert np.all(np.diff(E) < 0)
    assert abs(E[-1] - E_ref) / E_ref < 0.05
    assert abs(mse - mse_ref) / mse_ref < 0.05
