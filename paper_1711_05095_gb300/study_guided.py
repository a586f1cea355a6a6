"""Guided against plain cloning with a learned window potential (one GB300).

    python -m paper_1711_05095_gb300.study_guided [--L 128] [--lam 15] [--t-obs 200] [--quick]

1. Training data: plain cloning populations (L, N = L/2, s = lam / L^2); after `burn`
   intervals the population is recorded, and after `lag` more intervals every final
   clone is paired with its ancestor (pop_lineage): final clones sample p_end,
   ancestors sample p_ave (Sec. 2.2, eqs. Opave and Opend).  One population is held
   out for the classifier's test loss (disjoint lineages).
2. The window network is trained on the GPU (pop_mlp_step, Adam) as the classifier
   ancestral = 1 / end = 0 and compiled to the 512-entry potential table.
3. psi_hat over `seeds` independent seeds, each method in one batch: GUIDED with the
   learned potential at several N_c, GUIDED with the zero potential, and plain
   cloning at the same N_c and at a reference N_c.  Device time per batch; SE =
   std / sqrt(seeds); seconds to SE(psi) <= 1e-3 = (seconds per run) x (std / 1e-3)^2.
   Each estimate drops the first `burn-runs` intervals (steady-state psi), so methods
   with different dynamics are compared without their different start-up terms.

Prints one JSON object.
"""
import argparse
import json
import time

import numpy as np

from . import POP_GUIDED, PopulationBatch
from . import potential as pot


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


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--lam", type=float, default=15.0)
    ap.add_argument("--dt", type=float, default=0.05)
    ap.add_argument("--t-obs", type=float, default=200.0)
    ap.add_argument("--burn-runs", type=int, default=2000, help="intervals dropped from each estimate")
    ap.add_argument("--seeds", type=int, default=32)
    ap.add_argument("--data-pops", type=int, default=4)
    ap.add_argument("--data-nc", type=int, default=1 << 16)
    ap.add_argument("--burn", type=int, default=20000)
    ap.add_argument("--lag", type=int, default=20000)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--guided-nc", default="4096,16384")
    ap.add_argument("--plain-nc", default="16384,1048576")
    ap.add_argument("--quick", action="store_true", help="small sizes for a smoke run")
    a = ap.parse_args(argv)
    if a.quick:
        a.L, a.lam, a.dt, a.t_obs, a.seeds = 32, 15.0, 0.1, 50.0, 8
        a.data_pops, a.data_nc, a.burn, a.lag, a.train_steps = 3, 4096, 400, 400, 300
        a.burn_runs = 200
        a.guided_nc, a.plain_nc = "1024", "1024,16384"
    L, N = a.L, a.L // 2
    s = a.lam / L ** 2
    M = int(round(a.t_obs / a.dt))
    out = dict(workload="L=%d N=%d lambda=%g s=%.6g dt=%g t_obs=%g (M=%d) after %d intervals dropped, "
                        "%d seeds per method" % (L, N, a.lam, s, a.dt, a.t_obs, M, a.burn_runs, a.seeds))

    t0 = time.perf_counter()
    pops = [dict(L=L, N=N, n_clones=a.data_nc, seed=900000 + i) for i in range(a.data_pops)]
    end, anc = pot.ancestral_samples(pops, [s] * a.data_pops, a.dt, a.burn, a.lag)
    t_data = time.perf_counter() - t0
    cut = a.data_nc * (a.data_pops - 1)
    t0 = time.perf_counter()
    tr, losses = pot.train(end[:cut], anc[:cut], L, steps=a.train_steps, batch_size=a.batch, lr=a.lr,
                           log_every=max(1, a.train_steps // 8))
    held = pot.classifier_loss(tr, end[cut:], anc[cut:], L)
    phi = tr.potential()
    t_train = time.perf_counter() - t0
    out["training"] = dict(
        data="%d plain populations x %d clones, burn %d and lag %d intervals (%g and %g time units)"
             % (a.data_pops, a.data_nc, a.burn, a.lag, a.burn * a.dt, a.lag * a.dt),
        configurations=int(2 * len(end)), distinct_ancestors=int(len(np.unique(anc, axis=0))),
        steps=a.train_steps, batch=a.batch, lr=a.lr, losses=[[int(i), float(l)] for i, l in losses],
        heldout_loss=float(held), chance_loss=float(np.log(2.0)),
        phi_range=[float(phi.min()), float(phi.max())], seconds_data=t_data, seconds_train=t_train)

    rows = []
    gnc = [int(x) for x in a.guided_nc.split(",") if x]
    pnc = [int(x) for x in a.plain_nc.split(",") if x]
    plan = [("guided", n) for n in gnc] + [("zero", gnc[-1])] + [("plain", n) for n in pnc]
    for mode, nc in plan:
        psi, sec, ev = run_batch(L, N, s, a.dt, M, nc, a.seeds, 700000 + 1000 * len(rows), mode, phi,
                                 burn=a.burn_runs)
        sd = float(np.std(psi, ddof=1))
        per_run = sec / a.seeds
        rows.append(dict(method=mode, n_clones=nc, psi_mean=float(np.mean(psi)), psi_std=sd,
                         se=sd / np.sqrt(a.seeds), seconds_batch=sec, seconds_per_run=per_run,
                         seconds_to_se_1e3=per_run * max(1.0, (sd / 1e-3) ** 2),
                         clone_events_per_s=ev / sec))
    ref = rows[-1]
    for r in rows:
        r["z_vs_reference"] = (r["psi_mean"] - ref["psi_mean"]) / float(np.hypot(r["se"], ref["se"]))
    out["runs"] = rows
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
