"""GPU parity of the sweeps, energy, gradient, GN Hessian-vector product and GN solve
against the FP64 oracle (Sections 2.7 and 3.2)."""

import numpy as np
import pytest

from oracle import sweeps
from paper_1807_11560_gb300 import LddmmError

from helpers import host, problem, quantise, rel_2, rel_V, torch_dev

pytestmark = pytest.mark.gpu

# (kind, grid, band, seed, Nt): several tiles and ragged edges, 2D and 3D
CASES = [("blobs", (40, 36), (12, 10), 11, 5),
         ("ellipsoids", (24, 20, 18), (8, 6, 6), 12, 4),
         ("ellipsoids", (20, 20, 20), (8, 8, 8), 13, 10)]
# relative tolerances: fp64 is rounding only; fp32 is the 1e-5 gradient/Hessvec target
TOL = {"fp64": {"E": 1e-11, "g": 1e-9, "m": 1e-10},
       "fp32": {"E": 1e-6, "g": 1e-5, "m": 1e-5}}


def _cplx(precision, shape):
    import torch
    return torch.empty(shape, device="cuda", dtype=torch.complex128 if precision == "fp64" else torch.complex64)


def _real(precision, shape):
    import torch
    return torch.empty(shape, device="cuda", dtype=torch.float64 if precision == "fp64" else torch.float32)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_shoot_transport_energy(case, precision):
    kind, Ns, Ks, seed, Nt = case
    ctx, P, v0, _ = problem(kind, Ns, Ks, seed, Nt, precision)
    d = len(Ns)
    vs, vstar, vgrid, ms, feet = P.forward(v0)
    v1 = _cplx(precision, (d,) + Ks)
    ctx.shoot(torch_dev(v0, precision), v1)
    assert rel_V(host(v1), vs[-1], Ks) < TOL[precision]["g"]
    m1 = _real(precision, Ns)
    ctx.transport(torch_dev(v0, precision), m1)
    assert rel_2(host(m1), ms[-1]) < TOL[precision]["m"]
    E = ctx.energy(torch_dev(v0, precision))
    Eref = P.energy(v0)
    assert abs(E - Eref) / Eref < TOL[precision]["E"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_gradient_and_hessvec(case, precision):
    kind, Ns, Ks, seed, Nt = case
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, precision)
    d = len(Ns)
    lin = P.gradient(v0)
    g = _cplx(precision, (d,) + Ks)
    E = ctx.gradient(torch_dev(v0, precision), g)
    assert abs(E - lin.E) / lin.E < TOL[precision]["E"]
    assert rel_V(host(g), lin.g, Ks) < TOL[precision]["g"]
    Hp_ref = P.hessvec(lin, p)
    Hp = _cplx(precision, (d,) + Ks)
    ctx.hessvec(torch_dev(p, precision), Hp)
    assert rel_V(host(Hp), Hp_ref, Ks) < TOL[precision]["g"]
    dm1 = _real(precision, Ns)
    ctx.last_dm1(dm1)
    assert rel_2(host(dm1), P.incremental_m1(lin, p)) < TOL[precision]["m"]
    # a second product at the same point (graph replay) and linearity
    Hp2 = _cplx(precision, (d,) + Ks)
    ctx.hessvec(torch_dev(2.0 * p, precision), Hp2)
    assert rel_V(host(Hp2), 2.0 * Hp_ref, Ks) < TOL[precision]["g"]


def test_graph_replay_equals_direct_launches():
    import torch
    kind, Ns, Ks, seed, Nt = CASES[1]
    outs = []
    for graphs in (True, False):
        ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, "fp32", use_graphs=graphs)
        g = _cplx("fp32", (3,) + Ks)
        ctx.gradient(torch_dev(v0, "fp32"), g)
        Hp = _cplx("fp32", (3,) + Ks)
        ctx.hessvec(torch_dev(p, "fp32"), Hp)
        ctx.hessvec(torch_dev(p, "fp32"), Hp)
        outs.append(host(Hp))
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_sweeps_equal_per_evaluation_launches(precision):
    """One cooperative kernel per sweep runs the same phase code as three
    launches per bracket evaluation: the results must be bit-identical."""
    kind, Ns, Ks, seed, Nt = CASES[2]
    outs = []
    for persistent in (True, False):
        ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, precision, persistent=persistent)
        g = _cplx(precision, (3,) + Ks)
        E = ctx.gradient(torch_dev(v0, precision), g)
        Hp = _cplx(precision, (3,) + Ks)
        ctx.hessvec(torch_dev(p, precision), Hp)
        outs.append((E, host(g), host(Hp)))
    assert outs[0][0] == outs[1][0]
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_recompute_mode_equals_kept_histories(precision):
    """Regenerating the image-grid histories in forward order (recompute mode) runs
    the same kernels on the same inputs: energy, gradient, Hessian-vector product,
    m(1) and the line-search energy must be bit-identical, with a smaller footprint."""
    kind, Ns, Ks, seed, Nt = CASES[2]
    outs, held = [], []
    for recompute in (False, True):
        ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, precision, recompute=recompute)
        held.append(ctx.device_bytes)
        g = _cplx(precision, (3,) + Ks)
        E = ctx.gradient(torch_dev(v0, precision), g)
        Hp = _cplx(precision, (3,) + Ks)
        ctx.hessvec(torch_dev(p, precision), Hp)
        ctx.hessvec(torch_dev(p, precision), Hp)        # second call: graph replay
        E2 = ctx.energy(torch_dev(v0 + 0.5 * p, precision))
        Hp2 = _cplx(precision, (3,) + Ks)
        ctx.hessvec(torch_dev(p, precision), Hp2)        # linearisation point kept across energy()
        outs.append((E, host(g), host(Hp), E2, host(Hp2)))
        ctx.close()
    assert outs[0][0] == outs[1][0] and outs[0][3] == outs[1][3]
    for k in (1, 2, 4):
        np.testing.assert_array_equal(outs[0][k], outs[1][k])
    np.testing.assert_array_equal(outs[0][2], outs[0][4])
    assert held[1] < held[0]


def test_autotuned_tiles_change_no_result():
    """The autotuner only picks tile shapes (twiddle staging, pencils per tile, band
    rows per item); every sum keeps its order, so results are bit-identical."""
    kind, Ns, Ks, seed, Nt = "ellipsoids", (40, 36, 34), (12, 10, 8), 41, 3
    outs = []
    for autotune in (False, True):
        ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, "fp32", persistent=False, autotune=autotune)
        g = _cplx("fp32", (3,) + Ks)
        E = ctx.gradient(torch_dev(v0, "fp32"), g)
        Hp = _cplx("fp32", (3,) + Ks)
        ctx.hessvec(torch_dev(p, "fp32"), Hp)
        outs.append((E, host(g), host(Hp), ctx.tiles))
        ctx.close()
    print("tiles heuristic", outs[0][3], "autotuned", outs[1][3])
    assert outs[0][0] == outs[1][0]
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])


def test_host_pointers_and_state_errors():
    kind, Ns, Ks, seed, Nt = CASES[0]
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, "fp32")
    with pytest.raises(LddmmError) as ei:
        ctx.hessvec(p.astype(np.complex64), np.empty((2,) + Ks, np.complex64))
    assert ei.value.code == 4                         # ESTATE: no linearisation point yet
    g_h = np.empty((2,) + Ks, np.complex64)
    E_h = ctx.gradient(v0.astype(np.complex64), g_h)
    g_d = _cplx("fp32", (2,) + Ks)
    E_d = ctx.gradient(torch_dev(v0, "fp32"), g_d)
    assert E_h == E_d
    np.testing.assert_array_equal(g_h, g_d.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gn_solve_matches_oracle(precision):
    Ns, Ks, Nt = (32, 28), (10, 8), 5
    ctx, P, _, _ = problem("blobs", Ns, Ks, 21, Nt, precision, max_disp=2.0)
    z = np.zeros((2,) + Ks, dtype=np.complex128)
    v_ref, rep_ref = P.gn_solve(z, 3, 4)
    v = torch_dev(z, precision)
    rep = ctx.gn_solve(v, 3, 4)
    assert rep["gn_iters"] == len(rep_ref["eps"]) and rep["ls_failed"] == rep_ref["ls_failed"]
    assert rep["eps"] == rep_ref["eps"]
    tol = 1e-9 if precision == "fp64" else 1e-4
    np.testing.assert_allclose(rep["E"], rep_ref["E"], rtol=tol)
    m1 = _real(precision, Ns)
    ctx.transport(v, m1)
    m1_ref = P.forward(v_ref)[3][-1]
    assert rel_2(host(m1), m1_ref) < tol
    assert abs(rep["E_final"] - rep_ref["E_final"]) / rep_ref["E_final"] < tol
