"""Guided against plain cloning: one batch of independent runs and its timing.

run_batch runs `seeds` independent populations of one method in one batch (plain
cloning, or GUIDED cloning under a window potential, Sec. 2.2 eqs. modpdef and upsdef)
and returns their steady-state psi estimates with the device time and hops; the
guided-against-plain comparison of bench.py and the GPU tests build on it.
"""
import numpy as np

from . import POP_GUIDED, PopulationBatch


def run_batch(L, N, s, dt, M, nc, seeds, seed0, mode, phi=None, burn=0):
    """psi_hat of `seeds` independent runs in one batch, device time and hops.  With
    burn > 0 the estimate is the steady-state one, (sum of the psi terms of intervals
    burn+1 .. burn+M) / (M dt), which drops the start-up term of eq. psihat (it depends
    on the dynamics and is of order 1/t_obs); the time counts all intervals."""
    import torch
    wm = POP_GUIDED if mode != "plain" else 0
    pops = [dict(L=L, N=N, n_clones=nc, seed=seed0 + r, weight_mode=wm) for r in range(seeds)]
    b = PopulationBatch(pops)
    if mode == "guided":
        for p in range(seeds):
            b.set_potential(p, phi)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    acc0 = np.zeros(seeds)
    if burn > 0:
        b.run(dt, [s] * seeds, burn)
        psi0, _, t0 = b.estimate_psi()
        acc0 = psi0 * t0
    b.run(dt, [s] * seeds, M)
    psi, _, t1 = b.estimate_psi()
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    ev = int(b.events().sum())
    b.close()
    return (psi * t1 - acc0) / (M * dt), sec, ev
