"""Seeded synthetic workloads for the SSEP cloning estimator.

This module only describes inputs (ring sizes, particle numbers, clone numbers,
biases, seeds, interval lengths); it holds none of the method's arithmetic, and
both the CUDA path and the oracle take their inputs from it.  The SSEP needs no
dataset: every run starts from uniform random configurations drawn by the
method itself from the seed.

Each workload is a dict: pops (list of dicts L, N, n_clones, seed), s (list of
biases, one per population), dt, t_obs, M (= t_obs / dt intervals).
"""
import numpy as np


def _w(pops, s, dt, t_obs):
    M = int(round(t_obs / dt))
    return dict(pops=pops, s=[float(v) for v in s], dt=float(dt), t_obs=float(t_obs), M=M)


def ring_plain(L=20, N=10, s=0.05, n_clones=1000, dt=0.1, t_obs=200.0, seed=0):
    """Single population: L=20, N=10, s=0.05 (lambda = s L^2 = 20), N_c = 1000,
    dt = 0.1, t_obs = 200 (M = 2000)."""
    return _w([dict(L=L, N=N, n_clones=n_clones, seed=seed)], [s], dt, t_obs)


def s_sweep(L=50, n_lambda=64, lam_lo=-20.0, lam_hi=40.0, n_clones=16384, dt=0.1, t_obs=1000.0,
            seed=1000):
    """Batched s-sweep: L=50, N=25, 64 biases with lambda = s L^2 evenly spaced in
    [-20, 40], N_c = 16384 each (2^20 clones in all), dt = 0.1, t_obs = 1000."""
    lam = np.linspace(lam_lo, lam_hi, n_lambda)
    pops = [dict(L=L, N=L // 2, n_clones=n_clones, seed=seed + i) for i in range(n_lambda)]
    return _w(pops, lam / L**2, dt, t_obs)


def large_population(lams=(5.0, 10.0, 15.0, 20.0), n_seeds=8, L=128, n_clones=2**20, dt=0.05,
                     t_obs=2000.0, seed=2000):
    """L=128, N=64, lambda in {5,10,15,20}, N_c = 2^20, dt = 0.05, t_obs = 2000,
    8 seeds per lambda (32 populations)."""
    pops, s = [], []
    for i, lam in enumerate(lams):
        for r in range(n_seeds):
            pops.append(dict(L=L, N=L // 2, n_clones=n_clones, seed=seed + 100 * i + r))
            s.append(lam / L**2)
    return _w(pops, s, dt, t_obs)


def uneven_batch(n_pops=256, dt=0.1, t_obs=500.0, seed=12345):
    """256 populations: L uniform in {32, 64, 100, 128}, N = L/2,
    N_c = floor(2^U[10, 18]), lambda ~ U[-10, 30], s = lambda / L^2 (draws from a
    Philox generator seeded 12345)."""
    g = np.random.Generator(np.random.Philox(seed))
    Ls = g.choice([32, 64, 100, 128], size=n_pops)
    ncs = np.floor(2.0 ** g.uniform(10, 18, size=n_pops)).astype(np.int64)
    lam = g.uniform(-10, 30, size=n_pops)
    pops = [dict(L=int(L), N=int(L) // 2, n_clones=int(n), seed=seed + i)
            for i, (L, n) in enumerate(zip(Ls, ncs))]
    return _w(pops, lam / Ls.astype(np.float64) ** 2, dt, t_obs)


def seed_replicas(pop, s, n_runs, seed, dt=0.1, t_obs=1000.0):
    """n_runs independent copies (own seeds) of one population at bias s: the
    replicas whose spread gives the standard error of psi_hat."""
    pops = [dict(pop, seed=seed + r) for r in range(n_runs)]
    return _w(pops, [s] * n_runs, dt, t_obs)


def random_subsets(L, N, n_clones, seed):
    """Host-side uniform N-subsets packed as uint64 words (n_clones, ceil(L/64)):
    initial configurations supplied from host memory (pop_set_state).  Each row is an
    independent uniform shuffle of N ones and L - N zeros; site i is bit (i mod 64) of
    word (i div 64)."""
    g = np.random.default_rng(seed)
    W = (L + 63) // 64
    rows = np.zeros((n_clones, 64 * W), dtype=np.uint8)
    rows[:, :N] = 1
    rows[:, :L] = g.permuted(rows[:, :L], axis=1)
    packed = np.packbits(rows, axis=1, bitorder="little")          # 8 W bytes per row
    return np.ascontiguousarray(packed).view("<u8").reshape(n_clones, W).astype(np.uint64)
