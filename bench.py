#!/usr/bin/env python3
"""Benchmark of the SSEP cloning estimator on GB300: clone-events per second.

Workload (the batched s-sweep): 64 populations of the SSEP on a ring of L = 50 sites
with N = 25 particles, biases lambda = s L^2 evenly spaced in [-20, 40], N_c = 16384
clones each (2^20 clones), cloning interval dt = 0.1, t_obs = 1000 (M = 10000
intervals).  One step is one whole run: pop_init (initial configurations), pop_autotune
(launch configuration), M intervals of dynamical + cloning stages (pop_run,
captured CUDA graphs), and pop_estimate_psi.  clone-events = BKL hops executed by all clones (arXiv:1711.05095
measures the serial and parallel cost of exactly this loop, Sec. 6).

Prints one JSON line.  --impl reference times the CPU oracle on a bounded sample of
the same workload instead.
"""
import argparse
import json
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
# Cloning stage, per old clone ([eq], Sec. 2.3): weight = table[|dK - k_ref|] (3),
# its prefix sum (2), the inverse j_lo of the prefix by 128-bit products and compares
# (16), and for the new clone the ancestor lookup and its lattice and K (3)
OPS_GATHER = 3 + 2 + 16 + 3                     # 24
N_SM = 152
ISSUE_OPS_PER_SM_CLK = 128                      # 4 schedulers x 32 lanes

# Counters of one whole-batch launch of the dominant kernel on this workload, from ncu
# captures: DRAM bytes (read + write), and issue slots busy, ALU pipe and
# active lanes per instruction; valid only for the kernel sources they were taken on
# (hash of the two device headers).
KERNEL_TRAFFIC = {"bytes": 17178624, "issue_slots_busy": 0.6165, "alu_pipe": 0.5161,
                  "lanes_per_instruction": 24.11, "sources": "9eaf7124658b13ee"}


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
    ap.add_argument("--intervals", type=int, default=None,
                    help="override M (profiling runs only; the bench line then names it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-guided", action="store_true", help="skip the guided-cloning SE measurement")
    ap.add_argument("--no-others", action="store_true", help="skip the other batch shapes")
    ap.add_argument("--kernel-intervals", type=int, default=200)
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


def dist_setup(args):
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


def seconds_to_se(sigma, batch_seconds, batch_runs, target=1e-3):
    """Device seconds to bring the standard error of psi_hat over independent runs to
    `target`: R = ceil((sigma / target)^2) runs at the measured time per run."""
    import math
    runs = max(2, int(math.ceil((sigma / target) ** 2)))
    return runs, batch_seconds * runs / batch_runs


def cpu_oracle_sample(w, pop_idx, M):
    """The oracle as it stands, single-threaded, on the listed populations for M
    intervals.  Returns (events, seconds)."""
    import oracle
    oracle.lib()
    events, t0 = 0, time.perf_counter()
    for p in pop_idx:
        q = w["pops"][p]
        r = oracle.run(q["L"], q["N"], q["n_clones"], q["seed"], w["s"][p], w["dt"], M)
        events += r["events"]
    return events, time.perf_counter() - t0


def _oracle_one(args):
    w, p, M = args
    return cpu_oracle_sample(w, [p], M)[0]


def cpu_oracle_parallel(w, pop_idx, M):
    """The oracle as it stands, one process per population on as many host cores
    (spawned processes: nothing is forked from a process that has used the GPU).
    Returns the cpu_baseline-style record over the wall time of the whole pool."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(pop_idx)) as pool:
        pool.map(_oracle_one, [(w, pop_idx[0], 1)] * len(pop_idx))   # start-up and oracle build
        t0 = time.perf_counter()
        events = sum(pool.map(_oracle_one, [(w, p, M) for p in pop_idx]))
        sec = time.perf_counter() - t0
    return {"value": events / sec, "unit": UNIT, "cores": len(pop_idx), "kind": "oracle",
            "sample": "populations 0..%d (N_c=16384 each), first %d of the 10000 intervals, one "
                      "process per population; %.1f s" % (len(pop_idx) - 1, M, sec)}


def reference_arm(args, w, world, rank):
    if rank != 0:
        return
    pops = [0, 32]
    M = 40
    steps = []
    for i in range(args.warmup + args.steps):
        ev, sec = cpu_oracle_sample(w, pops, M)
        if i >= args.warmup:
            steps.append((ev, sec))
    ev = sum(e for e, _ in steps)
    sec = sum(s for _, s in steps)
    value = ev / sec
    sample = "populations %s of the 64 (N_c=16384 each), first %d of 10000 intervals, per step" % (pops, M)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / len(steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "s_sweep L=50 N=25 64 biases N_c=16384 dt=0.1 t_obs=1000",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    w = workloads.s_sweep()
    if args.intervals is not None:
        w["M"] = int(args.intervals)
        w["t_obs"] = w["M"] * w["dt"]
    if args.impl == "reference":
        return reference_arm(args, w, world, rank)

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
    s, dt, M = w["s"], w["dt"], w["M"]
    P = len(pops)
    nbytes = pg.workspace_bytes(pops)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 2**20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def one_step():
        b = pg.PopulationBatch(pops, device=dev, stream=stream, workspace=ws)
        b.autotune(dt, s, trials=3)
        b.run(dt, s, M)
        psi, kh, t = b.estimate_psi()
        ev = int(b.events().sum())
        launches.append(sum(b.launch_count().values()))
        b.close()
        return ev, psi

    launches = []

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        one_step()
    launches.clear()
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    t_wall0 = time.perf_counter()
    ev_total, ms = 0, []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, psi = one_step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        ev_total += ev
    barrier()
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    t_dev, ev_all = reduce_over_ranks(dist, dev, sum(ms) / 1e3, ev_total)
    value = ev_all / t_dev

    # end to end through the C ABI with host buffers: initial configurations from
    # pinned host memory (pop_set_state), the run, estimates back to the host
    host_lat = []
    for q in pops:
        arr = workloads.random_subsets(q["L"], q["N"], q["n_clones"], seed=q["seed"])
        pinned = torch.empty(arr.shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        pinned[...] = arr
        kz = torch.zeros(q["n_clones"], dtype=torch.int32, pin_memory=True).numpy()
        host_lat.append((pinned, kz))
    W = pg.lattice_words(pops)
    h2d = sum(q["n_clones"] * (8 * W + 4) for q in pops)
    d2h = P * (40 + 8)      # per-population state record and K sum read by pop_estimate_psi

    def e2e_step():
        b = pg.PopulationBatch(pops, device=dev, stream=stream, workspace=ws)
        for p in range(P):
            b.set_state(p, host_lat[p][0], host_lat[p][1])
        b.run(dt, s, M)
        psi, kh, t = b.estimate_psi()
        ev = int(b.events().sum())
        b.close()
        return ev

    e2e_step()
    barrier()
    e2e_ev, e2e_t = 0, 0.0
    for _ in range(max(1, min(args.steps, 2))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_ev += e2e_step()
        e2e_t += time.perf_counter() - t0
    e2e_t_all, e2e_ev_all = reduce_over_ranks(dist, dev, e2e_t, e2e_ev)
    e2e_value = e2e_ev_all / e2e_t_all

    # dominant kernel: the cloning stage fused with the next dynamical stage
    # (k_gather<FUSE>), every launch between CUDA events recorded by the library on
    # the stream it launches on (pop_kernel_times), after 64 warm-up intervals
    R = args.kernel_intervals
    b = pg.PopulationBatch(pops, device=dev, stream=stream, workspace=ws)
    b.run(dt, s, 64)
    # an NVTX range, so that a profiler can select these whole-batch launches
    torch.cuda.nvtx.range_push("fused_kernel_timing")
    kt = b.kernel_times(dt, s, R + 1)
    torch.cuda.nvtx.range_pop()
    b.close()
    t_k_us, n_k, hops_k = kt["gather_evolve"]
    t_k = t_k_us / 1e6
    clone_intervals = sum(q["n_clones"] for q in pops)

    # the other batch shapes of the method, bounded runs (device time of `intervals`
    # intervals through pop_run after 32 warm-up intervals): two-word lattices at
    # N_c = 2^20 per population, and 256 uneven populations
    others = {}
    if not args.no_others:
        for name, wl, n_iv in (("large_population", workloads.large_population(), 200),
                               ("uneven_batch", workloads.uneven_batch(), 200)):
            b = pg.PopulationBatch(wl["pops"], device=dev, stream=stream)
            b.run(wl["dt"], wl["s"], 32)
            ev0 = int(b.events().sum())
            o0 = torch.cuda.Event(enable_timing=True)
            o1 = torch.cuda.Event(enable_timing=True)
            o0.record(stream)
            b.run(wl["dt"], wl["s"], n_iv)
            o1.record(stream)
            o1.synchronize()
            sec_o = o0.elapsed_time(o1) / 1e3
            ev_o = int(b.events().sum()) - ev0
            clones = sum(q["n_clones"] for q in wl["pops"])
            others[name] = {"value": ev_o / sec_o, "unit": UNIT, "populations": len(wl["pops"]),
                            "clones": clones, "intervals_timed": n_iv, "ms_per_interval": 1e3 * sec_o / n_iv,
                            "workload": wl["pops"][0]["L"] if name == "large_population" else "mixed L"}
            if name == "large_population":
                # the separate cloning stage (k_gather) on a working set far above L2:
                # algorithmic bytes per clone = old lattice 8W + K 4 + dK 4 read, new
                # lattice 8W + K 4 + ancestor 4 written
                torch.cuda.nvtx.range_push("gather_timing")
                kt_g = b.kernel_times(wl["dt"], wl["s"], 8, per_step=True)
                torch.cuda.nvtx.range_pop()
                W_g = pg.lattice_words(wl["pops"])
                bytes_g = clones * (2 * (8 * W_g + 8))
                t_g = kt_g["gather"][0] / 1e6
                peaks_g, kind_g = measured_peaks()
                hbm = float(peaks_g.get("hbm_gbs", 6800.0))
                t_scan = kt_g["other"][0] / 1e6   # k_tile_scan, launched before each gather
                others["gather_roofline"] = {
                    "bound": "hbm", "kernel": "k_gather (separate cloning stage, two-word lattices)",
                    "achieved": bytes_g / t_g / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": bytes_g / t_g / 1e9 / hbm, "bytes_per_launch": bytes_g,
                    "launch_us": kt_g["gather"][0], "weights_us": kt_g["weights"][0],
                    "tile_scan_us": kt_g["other"][0],
                    "frac_with_tile_scan": bytes_g / (t_g + t_scan) / 1e9 / hbm,
                    "workload": "large_population, 2^25 clones, %d B per clone" % (2 * (8 * W_g + 8)),
                    "peak_kind": "measured copy bandwidth (%s)" % kind_g}
            b.close()
        others["large_population"]["workload"] = ("L=128 N=64 lambda in {5,10,15,20} x 8 seeds, "
                                                  "N_c=2^20 each, dt=0.05")
        others["uneven_batch"]["workload"] = ("256 populations, L in {32,64,100,128}, N_c in [2^10, 2^18], "
                                              "lambda in [-10, 30], dt=0.1")

    # seconds to SE(psi_hat) <= 1e-3 at lambda = 20 (s = 0.008): 64 independent seeds
    # of the same population, one batch, full t_obs
    se_w = workloads.seed_replicas(w["pops"][0], 20.0 / 50**2, 64, seed=500000 + 1000 * rank)
    se_pops = se_w["pops"]
    ws_se = torch.empty(pg.workspace_bytes(se_pops), dtype=torch.uint8, device=dev)
    flush.zero_()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    b = pg.PopulationBatch(se_pops, device=dev, stream=stream, workspace=ws_se)
    b.run(dt, se_w["s"], M)
    psi_se, _, _ = b.estimate_psi()
    s1.record(stream)
    s1.synchronize()
    b.close()
    se_batch_s = s0.elapsed_time(s1) / 1e3
    sigma = float(np.std(psi_se, ddof=1))
    se_runs, se_seconds = seconds_to_se(sigma, se_batch_s, len(se_pops))
    del ws_se

    # the same target with GUIDED cloning under a learned window potential: the
    # potential is trained on the GPU from end / ancestral configurations of plain
    # runs of this population (4 x 8192 clones, 1000 + 1000 intervals), then 64 seeds
    # at N_c = 4096 run the full t_obs (training time counted separately)
    guided = None
    if not args.no_guided:
        from paper_1711_05095_gb300 import potential as pot
        q0 = w["pops"][0]
        g_s = 20.0 / q0["L"] ** 2
        t_g0 = time.perf_counter()
        dpops = [dict(q0, n_clones=8192, seed=600000 + 1000 * rank + i) for i in range(4)]
        end, anc = pot.ancestral_samples(dpops, [g_s] * 4, dt, 1000, 1000, device=dev)
        cut = 8192 * 3
        tr, _ = pot.train(end[:cut], anc[:cut], q0["L"], steps=600, batch_size=8192, lr=2e-3, device=dev)
        held = pot.classifier_loss(tr, end[cut:], anc[cut:], q0["L"], device=dev)
        phi = tr.potential()
        tr.close()
        t_train = time.perf_counter() - t_g0
        gpops = [dict(q, n_clones=4096, weight_mode=pg.POP_GUIDED) for q in se_pops]
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        g0.record(stream)
        b = pg.PopulationBatch(gpops, device=dev, stream=stream)
        for p_ in range(len(gpops)):
            b.set_potential(p_, phi)
        b.run(dt, se_w["s"], M)
        psi_g, _, _ = b.estimate_psi()
        g1.record(stream)
        g1.synchronize()
        ev_g = int(b.events().sum())
        b.close()
        g_batch = g0.elapsed_time(g1) / 1e3
        sig_g = float(np.std(psi_g, ddof=1))
        g_runs, g_seconds = seconds_to_se(sig_g, g_batch, len(gpops))
        se_comb = float(np.hypot(sig_g, sigma) / np.sqrt(len(gpops)))
        guided = {"value": g_seconds, "unit": "s", "target_se": 1e-3,
                  "workload": "L=50 N=25 lambda=20 N_c=4096 dt=0.1 t_obs=%g, GUIDED with a learned "
                              "window potential" % w["t_obs"],
                  "sigma_per_run": sig_g, "runs_needed": g_runs, "batch_runs": len(gpops),
                  "batch_seconds": g_batch, "clone_events_per_s": ev_g / g_batch,
                  "mean_psi": float(np.mean(psi_g)),
                  "z_vs_plain": (float(np.mean(psi_g)) - float(np.mean(psi_se))) / se_comb,
                  "classifier_heldout_loss": float(held), "classifier_chance_loss": float(np.log(2.0)),
                  "training_seconds": t_train}
    ops_per_launch = (OPS_HOP * hops_k + (OPS_STOP + OPS_GATHER) * clone_intervals * n_k) / n_k
    counters_valid = kernel_sources_digest() == KERNEL_TRAFFIC["sources"]
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_gops = N_SM * ISSUE_OPS_PER_SM_CLK * sm_max * 1e6 / 1e9
    achieved = ops_per_launch / t_k / 1e9
    # the same operation count over this rank's timed steps, whose time also holds the
    # other kernels of each interval and, with pop_run's two chains, their overlap
    ops_run = OPS_HOP * ev_total + (OPS_STOP + OPS_GATHER) * clone_intervals * M * args.steps
    achieved_run = ops_run / (sum(ms) / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "s_sweep L=50 N=25 64 biases lambda in [-20,40] N_c=16384 each "
                               "dt=0.1 t_obs=%g (M=%d)" % (w["t_obs"], M),
                   "populations": P, "clones": clone_intervals, "intervals": M,
                   "l2": "flushed (512 MB write) between timed steps",
                   "parallelism": "replicas%d" % world},
        "gpu_launches": int(sum(launches)),
        "roofline": {"bound": "alu", "kernel": "k_gather<fused> (cloning stage + next dynamical stage)",
                     "achieved": achieved, "peak": peak_gops,
                     "unit": "Gop/s", "frac": achieved / peak_gops,
                     "traffic": KERNEL_TRAFFIC["bytes"] if counters_valid else None,
                     "ncu": ({k: KERNEL_TRAFFIC[k] for k in ("issue_slots_busy", "alu_pipe", "lanes_per_instruction")}
                             if counters_valid else None),
                     "peak_kind": "issue rate 152 SM x 128 lanes x %.0f MHz (%s max clock)"
                                  % (sm_max, peak_kind),
                     "launch_us": t_k_us, "launches_timed": n_k,
                     "other_kernels_us": {k: v[0] for k, v in kt.items() if k != "gather_evolve" and v[1]},
                     "ops_per_launch": ops_per_launch,
                     "launches_from": "pop_kernel_times: whole-batch launches, one chain",
                     "achieved_in_run": achieved_run, "frac_in_run": achieved_run / peak_gops},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "seconds_to_se": {"value": se_seconds, "unit": "s", "target_se": 1e-3,
                          "workload": "L=50 N=25 lambda=20 N_c=16384 dt=0.1 t_obs=%g" % w["t_obs"],
                          "sigma_per_run": sigma, "runs_needed": se_runs,
                          "batch_runs": len(se_pops), "batch_seconds": se_batch_s,
                          "mean_psi": float(np.mean(psi_se)), "method": "plain cloning"},
        "seconds_to_se_guided": guided,
        "clocks": clocks,
        "wall_s_timed": wall,
        # the same steps counted in clone-intervals (one clone through one interval)
        "clone_intervals_per_s": clone_intervals * M * args.steps * world / t_dev,
        "psi_check": {"lambda=-20": float(psi[0]), "lambda=40": float(psi[-1])},
        "other_workloads": others,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        idx = list(range(0, 64, 8))
        ev_c, sec_c = cpu_oracle_sample(w, idx, 40)
        line["cpu_baseline"] = {"value": ev_c / sec_c, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "populations %s (N_c=16384 each), first 40 of the "
                                          "10000 intervals; %.1f s" % (idx, sec_c)}
        # the same oracle on every host core: one process per population (the
        # populations are independent, as the paper's OpenMP design splits clones)
        ncores = os.cpu_count() or 1
        idx_all = list(range(min(64, ncores)))
        line["cpu_baseline_all_cores"] = cpu_oracle_parallel(w, idx_all, 40)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
