"""The time-out path of the bounded device waits (LDDMM_ETIMEOUT).

The persistent sweep kernel waits on grid barriers and slab counters; every
wait gives up after a bounded number of polls, sets a flag the host reads and
lets every CTA leave.  The debug_stall option makes the first barrier wait for
an arrival that never comes, with a short poll limit, so the wait runs out on
purpose: no fault, no hang.  The call must report ETIMEOUT and the GPU must
stay usable for the next context.
"""

import numpy as np
import pytest

from helpers import ALPHA, S, SIGMA, rel_V
from oracle import sweeps
from paper_1807_11560_gb300 import Context, LddmmError, inputs

pytestmark = pytest.mark.gpu


def test_stalled_sweep_barrier_reports_timeout_and_the_gpu_stays_usable():
    import torch
    Ns, Ks, Nt = (32, 32, 32), (8, 8, 8), 3
    v0 = inputs.random_bl(Ks, 3, 5, 2.0, Ns)
    a = torch.as_tensor(v0, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(a)
    with Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", persistent=True, debug_stall=2000) as ctx:
        with pytest.raises(LddmmError) as ei:
            ctx.shoot(a, out)
        assert ei.value.code == 6                     # LDDMM_ETIMEOUT
    torch.cuda.synchronize()                          # the context of the process is intact
    with Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", persistent=True) as ctx:
        ctx.shoot(a, out)
        vs, _ = sweeps.shoot(v0.astype(np.complex64).astype(np.complex128), Nt, ALPHA, S)
        assert rel_V(out.cpu().numpy().astype(np.complex128), vs[-1], Ks) < 1e-5
