"""Batched population (lddmm_batch_gn_solve): independent registrations of
different grid and band sizes, each context on its own CUDA stream, solved at
once from host threads.  Every context runs the same kernels as alone, so the
batch must reproduce sequential solves bit for bit; the tensor-core form
(tcgen05 3xTF32 transforms and bracket kernels) and plain FP32 SIMT must both
agree with the FP64 oracle at the 1e-5 target on one member of each grid size
of the 32-pair population."""

import numpy as np
import pytest

from paper_1807_11560_gb300 import Context, LddmmError, batch_gn_solve, inputs

from helpers import ALPHA, S, SIGMA, host, oracle_grad_hessvec, quantise, rel_V, spawn_pool, torch_dev

pytestmark = pytest.mark.gpu

# (grid, band, seed): uneven sizes, all above the persistent-sweep limit or run with it off
SMALL = [((28, 24, 20), (10, 8, 8), 71), ((32, 32, 32), (12, 12, 12), 72),
         ((24, 20, 18), (8, 6, 6), 73), ((36, 30, 24), (12, 10, 8), 74)]


def _ctx(Ns, Ks, seed, Nt, stream=None, **kw):
    import torch
    I0, I1 = inputs.make_pair("ellipsoids", Ns, seed, max_disp=2.0)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32",
                  stream=stream.cuda_stream if stream is not None else None, **kw)
    I0d, I1d = torch_dev(quantise(I0, "fp32"), "fp32"), torch_dev(quantise(I1, "fp32"), "fp32")
    torch.cuda.synchronize()                     # the copies ran on torch's stream
    ctx.set_images(I0d, I1d)
    v0 = np.zeros((3,) + Ks, np.complex64)
    return ctx, v0


def test_batch_equals_sequential_solves():
    import torch
    Nt, n_gn, n_pcg = 4, 2, 3
    seq = []
    for Ns, Ks, seed in SMALL:
        ctx, v0 = _ctx(Ns, Ks, seed, Nt, persistent=False)
        rep = ctx.gn_solve(v0, n_gn, n_pcg)
        seq.append((v0.copy(), rep))
        ctx.close()
    streams = [torch.cuda.Stream() for _ in SMALL]
    made = [_ctx(Ns, Ks, seed, Nt, stream=st, persistent=False) for (Ns, Ks, seed), st in zip(SMALL, streams)]
    ctxs, v0s = [c for c, _ in made], [v for _, v in made]
    reps = batch_gn_solve(ctxs, v0s, n_gn, n_pcg, threads=4)
    for (v_seq, r_seq), v_b, r_b in zip(seq, v0s, reps):
        np.testing.assert_array_equal(v_b, v_seq)
        assert r_b["E"] == r_seq["E"] and r_b["pcg"] == r_seq["pcg"]
        assert r_b["E_final"] < r_b["E_initial"]
    for c in ctxs:
        c.close()


def test_batch_refuses_persistent_contexts():
    import torch
    st = torch.cuda.Stream()
    ctx, v0 = _ctx((20, 20, 20), (8, 8, 8), 75, 2, stream=st, persistent=True)
    with pytest.raises(LddmmError) as ei:
        batch_gn_solve([ctx], [v0], 1, 1)
    assert ei.value.code == 1
    ctx.close()


def test_population_split_precision_and_plain_fp32_match_oracle():
    """One pair of each grid size of the 32-pair population (96^3 to
    160x192x160, bands 24^3 and 32^3): gradient and Hessian-vector product with
    the tcgen05 3xTF32 kernels and with plain FP32 SIMT, each against the FP64
    oracle (1e-5 relative, norm and element-wise; E 1e-6), and against each
    other.  The oracle runs in worker processes beside the GPU work."""
    import os
    import torch
    pop = inputs.population()
    picked = []
    for entry in pop:                           # one pair of each grid size, largest first
        if entry[1] not in [e[1] for e in picked]:
            picked.append(entry)
    pool = spawn_pool(min(len(picked), os.cpu_count() or 1))
    try:
        ref_async = pool.map_async(oracle_grad_hessvec, picked)
        got = [_population_member(*entry) for entry in picked]
        refs = ref_async.get(timeout=3600)
    finally:
        pool.terminate()
        pool.join()
    for (kind, Ns, Ks, Nt, seed), outs, (Er, gr, Hr) in zip(picked, got, refs):
        for E, g, H in outs:
            assert abs(E - Er) / Er < 1e-6, (Ns, Ks)
            assert rel_V(g, gr, Ks) < 1e-5, (Ns, Ks)
            assert rel_V(H, Hr, Ks) < 1e-5, (Ns, Ks)
        (Et, gt, Ht), (Es, gs, Hs) = outs
        assert rel_V(gt, gs, Ks) < 1e-5, (Ns, Ks)
        assert rel_V(Ht, Hs, Ks) < 1e-5, (Ns, Ks)


def _population_member(kind, Ns, Ks, Nt, seed):
    """(E, g, H p) with the tensor cores, then without."""
    import torch
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    I0, I1 = quantise(I0, "fp32"), quantise(I1, "fp32")
    v0 = quantise(inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns), "fp32")
    p = quantise(inputs.random_bl(Ks, 3, seed + 2, 1.0, Ns), "fp32")
    outs = []
    for tc in (True, False):
        ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", tensor_cores=tc)
        ctx.set_images(torch_dev(I0, "fp32"), torch_dev(I1, "fp32"))
        g = torch.empty((3,) + Ks, device="cuda", dtype=torch.complex64)
        E = ctx.gradient(torch_dev(v0, "fp32"), g)
        Hp = torch.empty_like(g)
        ctx.hessvec(torch_dev(p, "fp32"), Hp)
        outs.append((E, host(g), host(Hp)))
        ctx.close()
    return outs
