"""GPU parity of the deformation-state form (Section 3.3: the inverse map carried
as a band-limited displacement, m(1) = I0(x + u(1)(x))) against the FP64 oracle:
energy, warped image, gradient, GN Hessian-vector product and GN solve, at small
sizes spanning several tiles and at the benchmark sizes."""

import numpy as np
import pytest

from oracle import bl
from oracle.deformation import DeformationProblem
from paper_1807_11560_gb300 import Context, LddmmError, batch_gn_solve, inputs

from helpers import ALPHA, S, SIGMA, host, problem, quantise, rel_2, rel_V, torch_dev

pytestmark = pytest.mark.gpu

CASES = [("blobs", (40, 36), (12, 10), 11, 5),
         ("ellipsoids", (24, 20, 18), (8, 6, 6), 12, 4),
         ("ellipsoids", (20, 20, 20), (8, 8, 8), 13, 10)]
TOL = {"fp64": {"E": 1e-11, "g": 1e-9, "m": 1e-10},
       "fp32": {"E": 1e-6, "g": 1e-5, "m": 1e-5}}


def _cplx(precision, shape):
    import torch
    return torch.empty(shape, device="cuda", dtype=torch.complex128 if precision == "fp64" else torch.complex64)


def _real(precision, shape):
    import torch
    return torch.empty(shape, device="cuda", dtype=torch.float64 if precision == "fp64" else torch.float32)


def dproblem(kind, Ns, Ks, seed, Nt, precision, **kw):
    ctx, P, v0, p = problem(kind, Ns, Ks, seed, Nt, precision, state="deformation", **kw)
    D = DeformationProblem(P.I0, P.I1, Ks, ALPHA, S, SIGMA, Nt)
    return ctx, D, v0, p


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_energy_and_warped_image(case, precision):
    kind, Ns, Ks, seed, Nt = case
    ctx, D, v0, _ = dproblem(kind, Ns, Ks, seed, Nt, precision)
    m1 = _real(precision, Ns)
    ctx.transport(torch_dev(v0, precision), m1)
    assert rel_2(host(m1), D.transport(v0)) < TOL[precision]["m"]
    E, Eref = ctx.energy(torch_dev(v0, precision)), D.energy(v0)
    assert abs(E - Eref) / Eref < TOL[precision]["E"]
    ctx.close()


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_gradient_and_hessvec(case, precision, persistent):
    kind, Ns, Ks, seed, Nt = case
    ctx, D, v0, p = dproblem(kind, Ns, Ks, seed, Nt, precision, persistent="auto" if persistent else False)
    d = len(Ns)
    lin = D.gradient(v0)
    g = _cplx(precision, (d,) + Ks)
    E = ctx.gradient(torch_dev(v0, precision), g)
    assert abs(E - lin.E) / lin.E < TOL[precision]["E"]
    assert rel_V(host(g), lin.g, Ks) < TOL[precision]["g"]
    Hp_ref = D.hessvec(lin, p)
    Hp = _cplx(precision, (d,) + Ks)
    ctx.hessvec(torch_dev(p, precision), Hp)
    assert rel_V(host(Hp), Hp_ref, Ks) < TOL[precision]["g"]
    dm1 = _real(precision, Ns)
    ctx.last_dm1(dm1)
    dm1_ref = np.sum(lin.gs * bl.iota(D.incremental_u1(lin, p), Ns), axis=0)
    assert rel_2(host(dm1), dm1_ref) < TOL[precision]["m"]
    Hp2 = _cplx(precision, (d,) + Ks)                   # graph replay, linearity
    ctx.hessvec(torch_dev(-3.0 * p, precision), Hp2)
    assert rel_V(host(Hp2), -3.0 * Hp_ref, Ks) < TOL[precision]["g"]
    ctx.close()


def test_zero_velocity_matches_the_state_form():
    """At v0 = 0 both forms leave I0 in place: their GPU energies, gradients and
    GN products agree to rounding (FP64)."""
    kind, Ns, Ks, seed, Nt = CASES[1]
    d = len(Ns)
    res = []
    for state in ("image", "deformation"):
        ctx, _, _, p = problem(kind, Ns, Ks, seed, Nt, "fp64", state=state)
        z = torch_dev(np.zeros((d,) + Ks, np.complex128), "fp64")
        g, Hp = _cplx("fp64", (d,) + Ks), _cplx("fp64", (d,) + Ks)
        E = ctx.gradient(z, g)
        ctx.hessvec(torch_dev(p, "fp64"), Hp)
        res.append((E, host(g), host(Hp)))
        ctx.close()
    (E0, g0, H0), (E1, g1, H1) = res
    assert abs(E0 - E1) <= 1e-13 * E0
    assert rel_V(g1, g0, Ks) < 1e-12
    assert rel_V(H1, H0, Ks) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gn_solve_matches_oracle(precision):
    Ns, Ks, Nt = (32, 28), (10, 8), 5
    ctx, D, _, _ = dproblem("blobs", Ns, Ks, 21, Nt, precision)
    z = np.zeros((2,) + Ks, dtype=np.complex128)
    v_ref, rep_ref = D.gn_solve(z, 3, 4)
    v = torch_dev(z, precision)
    rep = ctx.gn_solve(v, 3, 4)
    assert rep["gn_iters"] == len(rep_ref["eps"]) and rep["ls_failed"] == rep_ref["ls_failed"]
    assert rep["eps"] == rep_ref["eps"]
    tol = 1e-9 if precision == "fp64" else 1e-4
    np.testing.assert_allclose(rep["E"], rep_ref["E"], rtol=tol)
    assert abs(rep["E_final"] - rep_ref["E_final"]) / rep_ref["E_final"] < tol
    m1 = _real(precision, Ns)
    ctx.transport(v, m1)
    assert rel_2(host(m1), D.transport(v_ref)) < tol
    ctx.close()


def test_state_form_only_calls_are_refused():
    kind, Ns, Ks, seed, Nt = CASES[0]
    ctx, _, v0, p = dproblem(kind, Ns, Ks, seed, Nt, "fp32")
    d = len(Ns)
    g = _cplx("fp32", (d,) + Ks)
    for call in (lambda: ctx.exact_gradient(torch_dev(v0, "fp32"), g),
                 lambda: ctx.transport_vjp(torch_dev(v0, "fp32"), _real("fp32", Ns), g)):
        with pytest.raises(LddmmError) as ei:
            call()
        assert ei.value.code == 1
    ctx.gradient(torch_dev(v0, "fp32"), g)
    with pytest.raises(LddmmError) as ei:
        ctx.hessvec_newton(torch_dev(p, "fp32"), g)
    assert ei.value.code == 1
    ctx.close()
    with pytest.raises(LddmmError):
        Context(Ns, Ks, ALPHA, S, SIGMA, Nt, state="deformation", newton=True)


@pytest.mark.parametrize("name, v_disp", [("3d_64_ellipsoids", 2.0), ("3d_160x192x160_brain", 3.0)])
def test_benchmark_sizes(name, v_disp):
    """The bench configuration (FP32, graph replay) at full size against the oracle."""
    import torch
    kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[name]
    d = len(Ns)
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, d, seed + 1, v_disp, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, d, seed + 2, 1.0, Ns), "fp32")
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", state="deformation")
    ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
    g = torch.empty((d,) + Ks, device="cuda", dtype=torch.complex64)
    E = ctx.gradient(torch_dev(v0, "fp32"), g)
    Hp = torch.empty_like(g)
    ctx.hessvec(torch_dev(p, "fp32"), Hp)
    ctx.hessvec(torch_dev(p, "fp32"), Hp)
    m1 = torch.empty(Ns, device="cuda", dtype=torch.float32)
    ctx.transport(torch_dev(v0, "fp32"), m1)
    got = (E, host(g), host(Hp), host(m1))
    ctx.close()
    D = DeformationProblem(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    lin = D.gradient(v0)
    assert abs(got[0] - lin.E) / lin.E < 1e-6
    assert rel_V(got[1], lin.g, Ks) < 1e-5
    assert rel_V(got[2], D.hessvec(lin, p), Ks) < 1e-5
    assert rel_2(got[3], lin.m1) < 1e-5


def test_batch_of_deformation_contexts_equals_sequential_solves():
    """lddmm_batch_gn_solve on deformation-form contexts of uneven sizes, each on
    its own stream, reproduces the sequential solves bit for bit."""
    import torch
    members = [((28, 24, 20), (10, 8, 8), 81), ((24, 20, 18), (8, 6, 6), 82), ((32, 28), (10, 8), 83)]
    Nt, n_gn, n_pcg = 4, 2, 3

    def make(Ns, Ks, seed, stream=None):
        I0, I1 = inputs.make_pair("ellipsoids" if len(Ns) == 3 else "blobs", Ns, seed, max_disp=2.0)
        ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", persistent=False, state="deformation",
                      stream=stream.cuda_stream if stream is not None else None)
        I0d, I1d = torch_dev(quantise(I0, "fp32"), "fp32"), torch_dev(quantise(I1, "fp32"), "fp32")
        torch.cuda.synchronize()
        ctx.set_images(I0d, I1d)
        return ctx, np.zeros((len(Ns),) + Ks, np.complex64)

    seq = []
    for Ns, Ks, seed in members:
        ctx, v0 = make(Ns, Ks, seed)
        rep = ctx.gn_solve(v0, n_gn, n_pcg)
        seq.append((v0.copy(), rep))
        ctx.close()
    streams = [torch.cuda.Stream() for _ in members]
    made = [make(Ns, Ks, seed, st) for (Ns, Ks, seed), st in zip(members, streams)]
    ctxs, v0s = [c for c, _ in made], [v for _, v in made]
    reps = batch_gn_solve(ctxs, v0s, n_gn, n_pcg, threads=3)
    for (v_seq, r_seq), v_b, r_b in zip(seq, v0s, reps):
        np.testing.assert_array_equal(v_b, v_seq)
        assert r_b["E"] == r_seq["E"] and r_b["pcg"] == r_seq["pcg"]
        assert r_b["E_final"] < r_b["E_initial"]
    for c in ctxs:
        c.close()
