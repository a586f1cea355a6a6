#!/usr/bin/env python3
"""Benchmark of the SSEP cloning estimator on GB300: clone-events per second.

Workload (the large-population batch): 32 populations of the SSEP on a ring of L = 128
sites with N = 64 particles, biases lambda = s L^2 in {5, 10, 15, 20} x 8 seeds,
N_c = 2^20 clones each (2^25 clones), cloning interval dt = 0.05, t_obs = 2000
(M = 40000 intervals per run).  One step is one block of `--block` (default 1000)
consecutive intervals of one continuing run: dynamical + cloning stages through
pop_run (captured CUDA graphs); a run that has reached M intervals is replaced by a
fresh one between steps (its initial state is not part of a step).  clone-events =
BKL hops executed by all clones (arXiv:1711.05095 measures the serial and parallel
cost of exactly this loop, Sec. 6).

Beside the headline the line carries: the dominant kernel's roofline from the launches
of the timed configuration, the end-to-end figure from host configurations, the other
batch shapes (s-sweep, uneven batch, the separate cloning stage against HBM), a
guided-against-plain comparison at L = 128, and the CPU oracle's throughput.

Prints one JSON line.  --impl reference times the CPU oracle on a bounded sample of
the same workload instead.  --config5 runs the learned-potential study at its full
size (a separate, longer measurement that prints its own JSON).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "clone-events/s"
UNIT = "events/s"

# Algorithmic 32-bit operations per BKL step (one waiting time, and for a hop one
# bond choice and the two-site flip), counted from the step's definition, not from
# compiled code:
#   Philox4x32-10 shared by two steps: (10 rounds x (2 widening products = 4 ops,
#     2 three-input XORs = 4 ops) + 9 x 2 key additions) / 2              = 49
#   -ln(u): 2w+1 (2), leading one (1), 24-bit head (2), mantissa bits (2),
#     table index (2), two table reads (2), r (1), cubic (3), add (1),
#     exponent to float (2), two fma (2)                                      = 20
#   time: 1/r lookup, multiply, add, compare                                   = 4
#   active bonds and rate: rotate (4), xor (1), popc (1), r == 0 test (1)      = 7
#   bond choice: multiply-high (1), k-th set bit of 64 bits (6 levels x 4)    = 25
#   hop: b+1 mod L (3), two bit masks (3), xor (1)                              = 7
#   loop bookkeeping (step and hop counters, exit test)                         = 3
OPS_HOP = 49 + 20 + 4 + 7 + 25 + 7 + 3          # a step that hops: 115
OPS_STOP = OPS_HOP - 25 - 7 - 1                 # the step that ends the interval: 82
# The same step on a two-word (65..128-site) lattice, in 32-bit operations:
#   active bonds and rate: rotate-by-one of four words with the wrap at L (10), xor of
#     four words (4), popc of four words and their sum (7), r == 0 test (1)    = 22
#   bond choice: multiply-high (1), k-th set bit of 128 bits (7 levels x 4)   = 29
#   hop: b+1 mod L (3), the two bits' word masks (6), xor of four words (4)     = 13
OPS_HOP_W2 = 49 + 20 + 4 + 22 + 29 + 13 + 3     # 140
OPS_STOP_W2 = OPS_HOP_W2 - 29 - 13 - 1          # 97


def step_ops(W):
    """(operations of a step that hops, of the step that ends the interval) for a
    batch of W-word lattices."""
    return (OPS_HOP, OPS_STOP) if W == 1 else (OPS_HOP_W2, OPS_STOP_W2)
# Cloning stage, per old clone ([eq], Sec. 2.3): weight = table[|dK - k_ref|] (3),
# its prefix sum (2), the inverse j_lo of the prefix by 128-bit products and compares
# (16), and for the new clone the ancestor lookup and its lattice and K (3)
OPS_GATHER = 3 + 2 + 16 + 3                     # 24
ISSUE_OPS_PER_SM_CLK = 128                      # 4 schedulers x 32 lanes

# Counters of one launch of the dominant kernel on this workload, from an ncu capture
# of a smaller batch of the same shape scaled to a full launch: DRAM bytes (read +
# write), issue slots busy, ALU pipe and active lanes per instruction; valid only for
# the kernel sources they were taken on (hash of the two device headers).
KERNEL_TRAFFIC = {"bytes_per_tile": 27086, "issue_slots_busy": 0.6520, "alu_pipe": 0.5550,
                  "lanes_per_instruction": 28.42, "sources": "0373849f1c8587ee",
                  "captured": "one 2048-tile launch of k_gather<2, 128, FUSE> (bench.py --profile-case fused): "
                              "51.36 MB read + 4.11 MB written"}


def kernel_sources_digest():
    import hashlib
    h = hashlib.sha256()
    for f in ("pop_common.cuh", "pop_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1711_05095_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--block", type=int, default=1000, help="intervals per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-guided", action="store_true", help="skip the guided-against-plain comparison")
    ap.add_argument("--no-others", action="store_true", help="skip the other batch shapes")
    ap.add_argument("--kernel-intervals", type=int, default=100)
    ap.add_argument("--config5", action="store_true",
                    help="the learned-potential study at full size instead of the bench line")
    ap.add_argument("--selection-study", action="store_true",
                    help="the cloning-interval and selection study (Sec. 4.3) instead of the bench line")
    ap.add_argument("--profile-case", choices=["fused", "guided"], default=None,
                    help="a small run of one kernel shape, for a profiler capture, instead of the bench line")
    ap.add_argument("--profile-dt", type=float, default=None,
                    help="interval length of the 'fused' profiling case (default: the workload's 0.05)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_populations(pops, rank):
    """Weak scaling: every rank runs the whole batch as an independent replica with
    its own seeds (populations never span ranks, so no data-path collective)."""
    return [dict(q, seed=q["seed"] + 100000 * rank) for q in pops]


def reduce_over_ranks(dist, device, seconds, units):
    """(max seconds over ranks, sum of units over ranks): value = units / seconds."""
    if dist is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    e = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def seconds_to_se(sigma, seconds_per_run, target):
    """Seconds of device time to bring the standard error of psi_hat to `target`: the
    variance of psi_hat over independent runs times the cost of one run, divided by
    target^2 (R = (sigma / target)^2 runs of this length, or one run R times as long:
    the variance of psi_hat falls as 1/t_obs once t_obs is many correlation times)."""
    return sigma * sigma * seconds_per_run / (target * target)


# ---------------------------------------------------------------------------
# CPU oracle (bench's cpu_baseline leg and the reference arm only)
# ---------------------------------------------------------------------------
def cpu_oracle_intervals(w, pop_idx, n_intervals):
    """The oracle as it stands, single-threaded: the listed populations are initialised
    (not timed) and then run n_intervals intervals (dynamical + cloning stage), timed.
    Returns (events, seconds)."""
    import oracle
    oracle.lib()
    events, sec = 0, 0.0
    for p in pop_idx:
        q = w["pops"][p]
        o = oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"])
        t0 = time.perf_counter()
        for _ in range(n_intervals):
            o.evolve(w["dt"])
            o.resample(w["s"][p])
        sec += time.perf_counter() - t0
        events += o.events
    return events, sec


def _oracle_one(args):
    w, p, n = args
    return cpu_oracle_intervals(w, [p], n)


def cpu_oracle_parallel(w, pop_idx, n_intervals):
    """The same oracle on as many host cores, one spawned process per population
    (nothing is forked from a process that has used the GPU); the rate is the events of
    all processes over the longest process's interval time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(pop_idx)) as pool:
        res = pool.map(_oracle_one, [(w, p, n_intervals) for p in pop_idx])
    events = sum(r[0] for r in res)
    sec = max(r[1] for r in res)
    return {"value": events / sec, "unit": UNIT, "cores": len(pop_idx), "kind": "oracle",
            "sample": "populations 0..%d of the large-population batch (N_c=2^20 each), %d intervals "
                      "each after an untimed initial state, one process per population; %.1f s"
                      % (len(pop_idx) - 1, n_intervals, sec)}


def workload_name(w, block):
    return ("large_population L=128 N=64 lambda in {5,10,15,20} x 8 seeds N_c=2^20 each dt=%g t_obs=%g "
            "(M=%d); one step = %d consecutive intervals of one continuing run"
            % (w["dt"], w["t_obs"], w["M"], block))


def reference_arm(args, w, rank):
    """The oracle on a bounded sample of the same workload: per step, one interval of
    one population (N_c = 2^20, L = 128), the population initialised before the steps."""
    if rank != 0:
        return
    import oracle
    oracle.lib()
    p = 0
    q = w["pops"][p]
    o = oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"])
    steps = []
    for i in range(args.warmup + args.steps):
        ev0 = o.events
        t0 = time.perf_counter()
        o.evolve(w["dt"])
        o.resample(w["s"][p])
        sec = time.perf_counter() - t0
        if i >= args.warmup:
            steps.append((o.events - ev0, sec))
    ev = sum(e for e, _ in steps)
    sec = sum(s for _, s in steps)
    value = ev / sec
    sample = ("population 0 of the 32 (L=128, N_c=2^20), one interval per step (dynamical + cloning "
              "stage), consecutive intervals of one run; initial state not timed")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / len(steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_name(w, args.block), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# guided against plain cloning at L = 128
# ---------------------------------------------------------------------------
def guided_vs_plain(dev, L, lam, dt, M, burn, seeds, nc_list, nc_plain_ref, data_pops, data_nc,
                    data_burn, data_lag, train_steps, batch, lr, target, seed0=700000):
    """Train the window potential from plain populations, then psi_hat over `seeds`
    independent runs of each method (steady state: `burn` intervals dropped).  Each
    row: mean, spread, device seconds per run, variance x cost, seconds to SE(psi) <=
    target, and z against plain cloning at the same N_c and against the reference."""
    from paper_1711_05095_gb300 import potential as pot
    from paper_1711_05095_gb300.study_guided import run_batch
    N = L // 2
    s = lam / L ** 2
    t0 = time.perf_counter()
    pops = [dict(L=L, N=N, n_clones=data_nc, seed=900000 + i) for i in range(data_pops)]
    end, anc = pot.ancestral_samples(pops, [s] * data_pops, dt, data_burn, data_lag, device=dev)
    t_data = time.perf_counter() - t0
    cut = data_nc * (data_pops - 1)
    t0 = time.perf_counter()
    tr, losses = pot.train(end[:cut], anc[:cut], L, steps=train_steps, batch_size=batch, lr=lr, device=dev)
    held = pot.classifier_loss(tr, end[cut:], anc[cut:], L, device=dev)
    phi = tr.potential()
    tr.close()
    t_train = time.perf_counter() - t0
    rows = {}
    plan = [("plain", n) for n in nc_list] + [("guided", n) for n in nc_list]
    if nc_plain_ref is not None and nc_plain_ref not in nc_list:
        plan.append(("plain", nc_plain_ref))
    for k, (mode, nc) in enumerate(plan):
        psi, sec, ev = run_batch(L, N, s, dt, M, nc, seeds, seed0 + 1000 * k, mode, phi, burn=burn)
        sd = float(np.std(psi, ddof=1))
        per_run = sec / seeds
        rows["%s_%d" % (mode, nc)] = dict(
            method=mode, n_clones=nc, psi_mean=float(np.mean(psi)), psi_std=sd, se=sd / math.sqrt(seeds),
            seconds_per_run=per_run, variance_x_cost=sd * sd * per_run,
            seconds_to_se=seconds_to_se(sd, per_run, target), clone_events_per_s=ev / sec)
    for nc in nc_list:
        g, p = rows["guided_%d" % nc], rows["plain_%d" % nc]
        g["z_vs_plain_same_nc"] = (g["psi_mean"] - p["psi_mean"]) / math.hypot(g["se"], p["se"])
        g["seconds_to_se_ratio_vs_plain_same_nc"] = g["seconds_to_se"] / p["seconds_to_se"]
    if nc_plain_ref is not None:
        ref = rows["plain_%d" % nc_plain_ref]
        for r in rows.values():
            if r is not ref:
                r["z_vs_plain_reference"] = (r["psi_mean"] - ref["psi_mean"]) / math.hypot(r["se"], ref["se"])
    best_g = min((r for r in rows.values() if r["method"] == "guided"), key=lambda r: r["seconds_to_se"])
    best_p = min((r for r in rows.values() if r["method"] == "plain"), key=lambda r: r["seconds_to_se"])
    return {
        "workload": "L=%d N=%d lambda=%g dt=%g t_obs=%g after %d intervals dropped, %d seeds per method"
                    % (L, N, lam, dt, M * dt, burn, seeds),
        "target_se": target, "rows": rows,
        "best_guided_over_best_plain_seconds_to_se": best_g["seconds_to_se"] / best_p["seconds_to_se"],
        "training": {"data": "%d plain populations x %d clones, burn %d and lag %d intervals"
                             % (data_pops, data_nc, data_burn, data_lag),
                     "configurations": int(2 * len(end)), "steps": train_steps, "batch": batch,
                     "heldout_loss": float(held), "chance_loss": float(np.log(2.0)),
                     "phi_range": [float(phi.min()), float(phi.max())],
                     "seconds_data": t_data, "seconds_train": t_train},
    }


def config5(args):
    """The learned-potential workload at full size: the window potential trained on
    2^22 end / ancestral configurations of L = 128, lambda = 15 populations; guided
    cloning at N_c in {2^12, 2^14, 2^16} against plain cloning at N_c = 2^20, 32 seeds
    each, dt = 0.05, t_obs = 2000 (plain at 2^12 .. 2^16 too, for z at equal N_c)."""
    import torch
    from paper_1711_05095_gb300 import build as pbuild
    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    out = guided_vs_plain(dev, L=128, lam=15.0, dt=0.05, M=40000, burn=2000, seeds=32,
                          nc_list=[2 ** 12, 2 ** 14, 2 ** 16], nc_plain_ref=2 ** 20,
                          data_pops=9, data_nc=2 ** 18, data_burn=20000, data_lag=2000,
                          train_steps=4000, batch=16384, lr=2e-3, target=1e-3)
    out["kind"] = "config5 learned guiding potential, full size"
    print(json.dumps(out), flush=True)


def selection_study(args):
    """The cloning interval and the selection method (Sec. 4.3, Fig. Tau; Sec. 4.4): at
    lambda = 28 on rings of L = 20 and 50 (N = L/2), t_obs = 10^4, N_c = 2^16, for
    dt in {0.1, 0.3, 1, 3, 10}, [eq] against [iid] selection, each with plain and
    MODIFIED weights, 16 seeds each: the mean and spread of k_hat (eq. khat) and
    psi_hat (eq. psihat), the [eq]/[iid] variance ratio of k_hat, and the device time.
    The paper's own runs at this state point extrapolate to k_inf = 0.3433-0.3437 (L = 20)
    and 0.3620-0.3666 (L = 50) (its Table of fits in t_obs, N_c = 10^5)."""
    import torch
    import paper_1711_05095_gb300 as pg
    from paper_1711_05095_gb300 import build as pbuild
    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    lam, t_obs, nc, seeds = 28.0, 1.0e4, 1 << 16, 16
    rows = []
    for L in (20, 50):
        s = lam / L ** 2
        for dt in (0.1, 0.3, 1.0, 3.0, 10.0):
            M = int(round(t_obs / dt))
            for sel_name, sel in (("eq", pg.POP_EQ), ("iid", pg.POP_IID)):
                pops = [dict(L=L, N=L // 2, n_clones=nc, seed=800000 + 100000 * L + 1000 * int(10 * dt) + r + 50 * m,
                             weight_mode=wm, selection=sel)
                        for m, wm in enumerate((pg.POP_PLAIN, pg.POP_MODIFIED)) for r in range(seeds)]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b = pg.PopulationBatch(pops, device=dev, stream=stream)
                b.run(dt, [s] * len(pops), M)
                psi, kh, _ = b.estimate_psi()
                e1.record(stream)
                e1.synchronize()
                sec = e0.elapsed_time(e1) / 1e3
                b.close()
                for m, wname in enumerate(("plain", "modified")):
                    k = kh[m * seeds:(m + 1) * seeds]
                    ps = psi[m * seeds:(m + 1) * seeds]
                    rows.append(dict(L=L, dt=dt, selection=sel_name, weights=wname, intervals=M,
                                     k_mean=float(np.mean(k)), k_std=float(np.std(k, ddof=1)),
                                     psi_mean=float(np.mean(ps)), psi_std=float(np.std(ps, ddof=1)),
                                     batch_seconds=sec))
    ratios = []
    for L in (20, 50):
        for dt in (0.1, 0.3, 1.0, 3.0, 10.0):
            for wname in ("plain", "modified"):
                eq = [r for r in rows if (r["L"], r["dt"], r["selection"], r["weights"]) == (L, dt, "eq", wname)][0]
                iid = [r for r in rows if (r["L"], r["dt"], r["selection"], r["weights"]) == (L, dt, "iid", wname)][0]
                ratios.append(dict(L=L, dt=dt, weights=wname, var_ratio_eq_over_iid=(eq["k_std"] / iid["k_std"]) ** 2))
    out = {"kind": "cloning interval and selection study", "lambda": lam, "t_obs": t_obs, "n_clones": nc,
           "seeds": seeds, "rows": rows, "variance_ratios": ratios,
           "paper_k_inf": {"20": [0.3433, 0.3437], "50": [0.3620, 0.3666]}}
    print(json.dumps(out), flush=True)


def profile_case(args):
    """A small run of one kernel shape for a profiler: 'fused', the L = 128 batch shape
    with 4 populations of 2^20 clones (lambda = 15, 20 intervals of --profile-dt through
    pop_run, then 4 through pop_kernel_times); 'guided', 32 GUIDED populations of 2^14 clones at L = 128
    (the guided batch of the bench line) under a seeded window potential (10 intervals)."""
    import torch
    import paper_1711_05095_gb300 as pg
    from paper_1711_05095_gb300 import build as pbuild
    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.profile_case == "fused":
        w = workloads.large_population(lams=(15.0,), n_seeds=4)
        dt = args.profile_dt if args.profile_dt is not None else w["dt"]
        b = pg.PopulationBatch(w["pops"], device=dev)
        b.run(dt, w["s"], 20)
        hops = int(b.events().sum()) / (20 * sum(q["n_clones"] for q in w["pops"]))
        kt = b.kernel_times(dt, w["s"], 4)
        print(json.dumps({"case": "fused", "dt": dt, "hops_per_clone_interval": hops, "chains": b.run_chains(),
                          "kernel_us": kt}))
    else:
        pops = [dict(L=128, N=64, n_clones=1 << 14, seed=300 + i, weight_mode=pg.POP_GUIDED) for i in range(32)]
        b = pg.PopulationBatch(pops, device=dev)
        phi = np.random.default_rng(3).normal(0, 0.05, 512).astype(np.float32)
        for p in range(len(pops)):
            b.set_potential(p, phi)
        s = [15.0 / 128 ** 2] * len(pops)
        b.run(0.05, s, 10)
        print(json.dumps({"case": "guided", "events": int(b.events().sum())}))
    b.close()


# ---------------------------------------------------------------------------
def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.config5:
        return config5(args)
    if args.selection_study:
        return selection_study(args)
    if args.profile_case:
        return profile_case(args)
    w = workloads.large_population()
    if args.impl == "reference":
        return reference_arm(args, w, rank)

    import torch
    import paper_1711_05095_gb300 as pg
    from paper_1711_05095_gb300 import build as pbuild
    pbuild.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    pops = rank_populations(w["pops"], rank)
    s, dt, M, block = w["s"], w["dt"], w["M"], int(args.block)
    P = len(pops)
    clones = sum(q["n_clones"] for q in pops)
    nbytes = pg.workspace_bytes(pops)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 2**20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # one continuing run; a run that has reached M intervals is replaced between steps
    state = {"b": None, "done": 0, "tuned": None}
    runs_closed = {"events": 0, "launches": 0}

    def fresh_run():
        if state["b"] is not None:
            runs_closed["events"] += int(state["b"].events().sum())
            runs_closed["launches"] += sum(state["b"].launch_count().values())
            state["b"].close()
        b = pg.PopulationBatch(pops, device=dev, stream=stream, workspace=ws)
        state["tuned"] = b.autotune(dt, s, trials=3)
        state["b"], state["done"] = b, 0

    def totals():
        b = state["b"]
        return (runs_closed["events"] + int(b.events().sum()),
                runs_closed["launches"] + sum(b.launch_count().values()))

    fresh_run()
    for _ in range(args.warmup):
        if state["done"] + block > M:
            fresh_run()
        state["b"].run(dt, s, block)
        state["done"] += block
    barrier()
    ev_start, launches_start = totals()
    sampler = ClockSampler(local)
    sampler.start()
    t_wall0 = time.perf_counter()
    ms = []
    torch.cuda.nvtx.range_push("timed_steps")  # selects the timed kernels in a profiler
    for _ in range(args.steps):
        if state["done"] + block > M:
            fresh_run()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        state["b"].run(dt, s, block)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        state["done"] += block
    torch.cuda.nvtx.range_pop()
    barrier()
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    ev_end, launches_end = totals()
    ev_total = ev_end - ev_start
    t_dev, ev_all = reduce_over_ranks(dist, dev, sum(ms) / 1e3, ev_total)
    value = ev_all / t_dev
    b = state["b"]
    psi_run, _, t_run = b.estimate_psi()
    chains = b.run_chains()

    # dominant kernel: the launches pop_run makes for this batch in the tuned
    # configuration, each between CUDA events recorded by the library on the stream it
    # launches on (pop_kernel_times; after the first fused interval, from one captured
    # graph as pop_run replays it), continuing the same run.  With several chains the
    # fused launches run side by side: the time is that during which at least one of
    # them runs, per interval, and the operations those of the whole interval
    R = args.kernel_intervals
    torch.cuda.nvtx.range_push("fused_kernel_timing")
    kt = b.kernel_times(dt, s, R + 1)
    torch.cuda.nvtx.range_pop()
    t_k_us, n_k, hops_k = kt["gather_evolve"]
    t_k = t_k_us / 1e6
    ops_hop, ops_stop = step_ops(pg.lattice_words(pops))
    ops_per_launch = ops_hop * hops_k / R + (ops_stop + OPS_GATHER) * clones
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_gops = n_sm * ISSUE_OPS_PER_SM_CLK * sm_max * 1e6 / 1e9
    achieved = ops_per_launch / t_k / 1e9
    ops_run = ops_hop * ev_total + (ops_stop + OPS_GATHER) * clones * block * args.steps
    # the same with the one-word step count, for comparison with earlier figures
    ops_run_w1 = OPS_HOP * ev_total + (OPS_STOP + OPS_GATHER) * clones * block * args.steps
    achieved_run = ops_run / (sum(ms) / 1e3) / 1e9
    per_interval_us = {k: v[0] for k, v in kt.items() if v[1]}
    counters_valid = KERNEL_TRAFFIC is not None and kernel_sources_digest() == KERNEL_TRAFFIC["sources"]

    # end to end through the C ABI from host memory: a fresh run from pinned host
    # configurations (pop_set_state: lattices and K), one block of intervals, the
    # estimates read back (pop_estimate_psi); wall clock, pop_init included
    W = pg.lattice_words(pops)
    host = workloads.random_subsets(pops[0]["L"], pops[0]["N"], pops[0]["n_clones"], seed=77)
    lat_pin = torch.empty(host.shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    lat_pin[...] = host
    k_pin = torch.zeros(pops[0]["n_clones"], dtype=torch.int32, pin_memory=True).numpy()
    h2d = sum(q["n_clones"] * (8 * W + 4) for q in pops)
    d2h = P * (64 + 8)      # per-population state record and K sum read by pop_estimate_psi
    b.close()
    state["b"] = None

    def e2e_step():
        bb = pg.PopulationBatch(pops, device=dev, stream=stream, workspace=ws)
        for p in range(P):
            bb.set_state(p, lat_pin, k_pin)
        bb.run(dt, s, block)
        bb.estimate_psi()
        ev = int(bb.events().sum())
        bb.close()
        return ev

    e2e_step()
    barrier()
    e2e_ev, e2e_t = 0, 0.0
    n_e2e = max(1, min(args.steps, 2))
    for _ in range(n_e2e):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_ev += e2e_step()
        e2e_t += time.perf_counter() - t0
    e2e_t_all, e2e_ev_all = reduce_over_ranks(dist, dev, e2e_t, e2e_ev)
    e2e_value = e2e_ev_all / e2e_t_all
    del ws

    others = {}
    if not args.no_others:
        # the other batch shapes: whole runs (device time, pop_init to the estimates)
        for name, wl in (("s_sweep", workloads.s_sweep()), ("uneven_batch", workloads.uneven_batch())):
            o0 = torch.cuda.Event(enable_timing=True)
            o1 = torch.cuda.Event(enable_timing=True)
            flush.zero_()
            o0.record(stream)
            bo = pg.PopulationBatch(wl["pops"], device=dev, stream=stream)
            tuned_o = bo.autotune(wl["dt"], wl["s"], trials=3)
            bo.run(wl["dt"], wl["s"], wl["M"])
            bo.estimate_psi()
            o1.record(stream)
            o1.synchronize()
            sec_o = o0.elapsed_time(o1) / 1e3
            ev_o = int(bo.events().sum())
            cl = sum(q["n_clones"] for q in wl["pops"])
            ch = bo.run_chains()
            others[name] = {"value": ev_o / sec_o, "unit": UNIT, "populations": len(wl["pops"]),
                            "clones": cl, "intervals": wl["M"], "seconds": sec_o,
                            "chains": len(ch) - 1 if ch else 0, "tuned": tuned_o}
            bo.close()
        others["s_sweep"]["workload"] = ("64 populations L=50 N=25 lambda in [-20,40] N_c=16384 dt=0.1 t_obs=1000, "
                                         "whole run")
        others["uneven_batch"]["workload"] = ("256 populations, L in {32,64,100,128}, N_c in [2^10, 2^18], "
                                              "lambda in [-10, 30], dt=0.1, t_obs=500, whole run")
        # the separate cloning stage (k_gather) on the 2^25-clone batch, far above L2:
        # algorithmic bytes per clone = old lattice 8W + K 4 + dK 4 read, new lattice
        # 8W + K 4 + ancestor 4 written
        bg = pg.PopulationBatch(pops, device=dev, stream=stream)
        bg.run(dt, s, 16)
        torch.cuda.nvtx.range_push("gather_timing")
        kt_g = bg.kernel_times(dt, s, 8, per_step=True)
        torch.cuda.nvtx.range_pop()
        bg.close()
        bytes_g = clones * (2 * (8 * W + 8))
        t_g = kt_g["gather"][0] / 1e6
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        t_scan = kt_g["other"][0] / 1e6   # k_tile_scan, launched before each gather
        others["gather_roofline"] = {
            "bound": "hbm", "kernel": "k_gather (separate cloning stage, two-word lattices)",
            "achieved": bytes_g / t_g / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": bytes_g / t_g / 1e9 / hbm, "bytes_per_launch": bytes_g,
            "launch_us": kt_g["gather"][0], "weights_us": kt_g["weights"][0],
            "tile_scan_us": kt_g["other"][0],
            "frac_with_tile_scan": bytes_g / (t_g + t_scan) / 1e9 / hbm,
            "workload": "large_population, 2^25 clones, %d B per clone" % (2 * (8 * W + 8)),
            "peak_kind": "measured copy bandwidth (%s)" % peak_kind}

    # guided against plain cloning at L = 128, lambda = 15 (a bounded version of the
    # learned-potential workload; --config5 runs it at full size)
    guided = None
    if not args.no_guided:
        guided = guided_vs_plain(dev, L=128, lam=15.0, dt=0.05, M=4000, burn=1000, seeds=32,
                                 nc_list=[2 ** 14], nc_plain_ref=None, data_pops=4, data_nc=2 ** 16,
                                 data_burn=2000, data_lag=400, train_steps=600, batch=8192, lr=2e-3,
                                 target=1e-4)
        guided["bounded"] = ("t_obs 200 (config: 2000), one N_c (2^14) per method, 2^19 training "
                             "configurations (config: 2^22); full size: bench.py --config5")

    n_chains = len(chains) - 1 if chains else 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_name(w, block),
                   "populations": P, "clones": clones, "intervals_per_step": block,
                   "l2": "inputs larger than L2 (2 GB of clone state) and a 512 MB write between steps",
                   "parallelism": "replicas%d" % world, "chains": n_chains, "tuned": state["tuned"]},
        "gpu_launches": int(launches_end - launches_start),
        "roofline": {"bound": "alu", "kernel": "k_gather<fused> (cloning stage + next dynamical stage)",
                     "achieved": achieved, "peak": peak_gops, "unit": "Gop/s", "frac": achieved / peak_gops,
                     "traffic": (KERNEL_TRAFFIC["bytes_per_tile"] * sum((q["n_clones"] + 1023) // 1024 for q in pops)
                                 if counters_valid else None),
                     "traffic_from": KERNEL_TRAFFIC["captured"] + ", scaled by tiles (writes mostly stay in L2 "
                                     "at that size)" if counters_valid else None,
                     "ncu": ({k: KERNEL_TRAFFIC[k] for k in ("issue_slots_busy", "alu_pipe", "lanes_per_instruction")}
                             if counters_valid else None),
                     "peak_kind": "issue rate %d SM x 128 lanes x %.0f MHz (%s max clock)"
                                  % (n_sm, sm_max, peak_kind),
                     "launch_us": t_k_us, "launches_timed": n_k, "intervals_timed": R,
                     "launches_per_interval": n_k / R, "ops_per_launch": ops_per_launch,
                     "per_interval_us": per_interval_us,
                     "launches_from": "pop_kernel_times: the launch sequence of pop_run for this batch "
                                      "(%d chain%s), continuing the timed run" % (n_chains, "s" if n_chains > 1 else ""),
                     "dominant_ms_per_step": t_k_us * block / 1e3,
                     "achieved_in_run": achieved_run, "frac_in_run": achieved_run / peak_gops,
                     "ops_per_hop_step": ops_hop, "ops_per_end_step": ops_stop, "ops_per_clone_cloning": OPS_GATHER,
                     "frac_in_run_one_word_count": ops_run_w1 / (sum(ms) / 1e3) / 1e9 / peak_gops},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "step": "pop_init + pop_set_state of every population from pinned host memory + %d intervals "
                        "+ pop_estimate_psi (wall clock; the 32 populations start from the same host "
                        "configurations)" % block},
        "guided_vs_plain_L128": guided,
        "clocks": clocks,
        "wall_s_timed": wall,
        "clone_intervals_per_s": clones * block * args.steps * world / t_dev,
        "psi_check": {"lambda=5": float(psi_run[0]), "lambda=20": float(psi_run[-1]), "t_obs": t_run},
        "other_workloads": others,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        idx = [0, 8, 16, 24]
        ev_c, sec_c = cpu_oracle_intervals(w, idx, 2)
        line["cpu_baseline"] = {"value": ev_c / sec_c, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "populations %s (L=128, N_c=2^20 each), the first 2 intervals after "
                                          "an untimed initial state; %.1f s" % (idx, sec_c)}
        ncores = os.cpu_count() or 1
        idx_all = list(range(min(32, ncores)))
        line["cpu_baseline_all_cores"] = cpu_oracle_parallel(w, idx_all, 2)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
