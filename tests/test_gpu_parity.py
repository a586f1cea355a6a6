"""GPU path (through the C ABI) against the CPU oracle on identical Philox streams.

Bit-exact: lattices, cumulative activities K, interval activities dK and [eq]
ancestors, every interval.  psi_hat within 1e-12 relative (the psi terms use CUDA's
FP64 exp/expm1/log1p against glibc's; every other quantity is an integer).
Cases span several 1024-slot tiles with ragged tails, both lattice widths
(L <= 64 and 64 < L <= 128), both signs of s, s = 0, empty and full rings, one
clone, and a batch of uneven populations.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

PSI_RTOL = 1e-12


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05095_gb300 import build
    build.build()
    import paper_1711_05095_gb300 as pg
    return pg


def oracle_pops(pops):
    return [oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"],
                              modified=q.get("weight_mode", 0) == 1, iid=q.get("selection", 0) == 1)
            for q in pops]


def assert_state_equal(gpu, orc, W, what):
    words = oracle.sites_to_words(orc.sites, W)
    assert np.array_equal(gpu["lattice"], words), what + ": lattice"
    assert np.array_equal(gpu["K"], orc.K), what + ": K"


def run_parity(pg, pops, s, dt, M):
    batch = pg.PopulationBatch(pops)
    orcs = oracle_pops(pops)
    W = batch.W
    for p, o in enumerate(orcs):
        assert_state_equal(batch.copy_state(p), o, W, "init pop %d" % p)
    for beta in range(1, M + 1):
        batch.evolve(dt, s)
        for p, o in enumerate(orcs):
            o.evolve(dt, s[p])
            g = batch.copy_state(p)
            assert_state_equal(g, o, W, "evolve beta=%d pop %d" % (beta, p))
            assert np.array_equal(g["dK"], o.dK), "dK beta=%d pop %d" % (beta, p)
        batch.resample()
        for p, o in enumerate(orcs):
            o.resample(s[p])
            g = batch.copy_state(p)
            assert np.array_equal(g["anc"], o.anc), "anc beta=%d pop %d" % (beta, p)
            assert_state_equal(g, o, W, "resample beta=%d pop %d" % (beta, p))
    psi, kh, t_obs = batch.estimate_psi()
    ev = batch.events()
    for p, o in enumerate(orcs):
        ps, ks = o.estimates()
        np.testing.assert_allclose(psi[p], ps, rtol=PSI_RTOL, atol=0.0)
        np.testing.assert_allclose(kh[p], ks, rtol=1e-15, atol=0.0)
        assert int(ev[p]) == o.events
    return batch, orcs


@pytest.mark.parametrize("L,N,nc,s", [
    (20, 10, 1000, 0.05),      # one tile, ragged
    (20, 10, 2500, -0.3),      # three tiles, negative bias
    (50, 25, 3072, 0.3),       # exact tiles
    (64, 31, 1500, 0.8),       # widest one-word ring
    (65, 30, 1100, 0.2),       # narrowest two-word ring
    (100, 50, 2049, -0.05),
    (128, 64, 4100, 0.01),     # widest ring
    (3, 1, 777, 0.4),          # smallest ring
    (37, 5, 1, 0.5),           # one clone
    (20, 10, 1234, 0.0),       # no bias: identity ancestry
    (12, 0, 300, 0.3),         # empty ring: no hops
    (12, 12, 300, -0.3),       # full ring: no hops
    (40, 20, 3000, 2.5),       # strong bias: many deletions
])
def test_parity_single(pg, L, N, nc, s):
    pops = [dict(L=L, N=N, n_clones=nc, seed=1234 + L)]
    batch, orcs = run_parity(pg, pops, [s], 0.1 if L < 100 else 0.05, 6)
    if s == 0.0:
        g = batch.copy_state(0)
        assert np.array_equal(g["anc"], np.arange(nc))
        assert batch.estimate_psi()[0][0] == 0.0


def test_parity_uneven_batch(pg):
    rng = np.random.default_rng(5)
    pops, s = [], []
    for i, L in enumerate([32, 64, 100, 128, 20, 77]):
        pops.append(dict(L=L, N=L // 2 - i, n_clones=int(rng.integers(900, 3000)), seed=99 + i))
        s.append(float(rng.uniform(-10, 30)) / L**2)
    run_parity(pg, pops, s, 0.1, 5)


def test_parity_long_dt(pg):
    # many hops per interval (dt = 2 at L = 50: ~50 hops per clone)
    run_parity(pg, [dict(L=50, N=25, n_clones=1500, seed=3)], [0.02], 2.0, 3)


RUN_CASES = {
    # two-word lattices: fused run, two captured graphs of 32 intervals plus direct ones
    "w2_plain": ([dict(L=50, N=25, n_clones=2000, seed=7), dict(L=100, N=40, n_clones=1300, seed=8)],
                 [0.01, -0.004], [70]),
    # one-word lattices, MODIFIED next to plain, a ragged multi-tile population
    "w1_mixed_weights": ([dict(L=20, N=10, n_clones=2500, seed=11, weight_mode=1),
                          dict(L=64, N=31, n_clones=1100, seed=12)], [0.3, -0.2], [37]),
    # two-word MODIFIED, strong bias (many deletions), runs split across calls
    "w2_modified_split": ([dict(L=100, N=50, n_clones=1500, seed=13, weight_mode=1),
                           dict(L=33, N=16, n_clones=700, seed=14)], [0.05, 2.5], [1, 33, 2]),
    # an [iid] population: every interval through the separate kernels
    "iid_unfused": ([dict(L=30, N=15, n_clones=1200, seed=15, selection=1),
                     dict(L=50, N=25, n_clones=900, seed=16, weight_mode=1)], [0.1, -0.05], [35]),
    # a single interval: the fused run's first and last stages only
    "one_interval": ([dict(L=40, N=20, n_clones=3000, seed=17)], [0.2], [1]),
    # runs of 1, 2, 3 and 40 intervals; a population of 64 full tiles beside one of a
    # single ragged tile; s < 0
    "many_splits": ([dict(L=50, N=25, n_clones=64 * 1024, seed=18), dict(L=20, N=10, n_clones=700, seed=19)],
                    [0.01, -0.3], [1, 2, 3, 40]),
    # one population of 65 tiles and a ragged last tile
    "tiles_65": ([dict(L=30, N=15, n_clones=65 * 1024 + 5, seed=20)], [0.05], [35]),
    # five populations of 1, 4, 2, 3 and 2 tiles: pop_run runs three chains of 5, 2 and
    # 5 tiles; a graph replay, then direct launches of the chains
    "halves_of_five": ([dict(L=30, N=15, n_clones=1000, seed=30), dict(L=50, N=25, n_clones=4000, seed=31),
                        dict(L=70, N=30, n_clones=1900, seed=32, weight_mode=1),
                        dict(L=128, N=64, n_clones=3072, seed=33), dict(L=9, N=4, n_clones=1500, seed=34)],
                       [0.2, -0.01, 0.1, 0.004, -0.5], [33, 5]),
    # strong bias: a wide activity range and tiles whose old clones leave no copies
    "strong_bias": ([dict(L=64, N=32, n_clones=5000, seed=21), dict(L=128, N=64, n_clones=3000, seed=22)],
                    [2.0, 0.5], [34]),
    # rings that fill the lattice words (L = 64 W: the fused kernel rotates the words
    # without a closing bit), one and two words
    "w1_full_ring": ([dict(L=64, N=20, n_clones=3000, seed=23), dict(L=64, N=40, n_clones=2100, seed=24)],
                     [0.02, -0.05], [36]),
    "w2_full_ring": ([dict(L=128, N=64, n_clones=3000, seed=25), dict(L=128, N=50, n_clones=2100, seed=26)],
                     [0.01, -0.02], [35]),
}


def test_run_chains(pg):
    # the split rule: population starts nearest k/K of the tiles, every chain at least
    # half its share; up to 8 chains within two waves of the fused kernel, else 2
    five = pg.PopulationBatch(RUN_CASES["halves_of_five"][0])
    assert five.run_chains() == [0, 5, 7, 12]
    w = workloads.s_sweep()
    sweep = pg.PopulationBatch(w["pops"])                 # 64 x 16 tiles
    assert sweep.run_chains() == [128 * c for c in range(9)]
    sweep.close()
    big = pg.PopulationBatch([dict(L=50, N=25, n_clones=4096 * 1024, seed=40 + i) for i in range(3)])
    assert big.run_chains() == [0, 4096, 12288]            # 3 x 4096 tiles: two chains
    big.close()
    # batches that do not fuse run one sequence
    assert pg.PopulationBatch([dict(L=30, N=15, n_clones=1200, seed=15, selection=1),
                               dict(L=30, N=15, n_clones=1200, seed=16)]).run_chains() == []
    assert pg.PopulationBatch([dict(L=200, N=100, n_clones=1200, seed=17),
                               dict(L=30, N=15, n_clones=1200, seed=18)]).run_chains() == []


@pytest.mark.parametrize("case", sorted(RUN_CASES))
def test_run_equals_steps(pg, case):
    pops, s, splits = RUN_CASES[case]
    a = pg.PopulationBatch(pops)
    b = pg.PopulationBatch(pops)
    for n in splits:
        a.run(0.1, s, n)
    for _ in range(sum(splits)):
        b.evolve(0.1, s)
        b.resample()
    P = len(pops)
    for p in range(P):
        ga, gb = a.copy_state(p), b.copy_state(p)
        for key in ("lattice", "K", "anc", "dK"):
            assert np.array_equal(ga[key], gb[key]), key
    pa, ka, ta = a.estimate_psi()
    pb, kb, tb = b.estimate_psi()
    # same device arithmetic; only t_obs differs in rounding (n*dt against a sum of dt)
    np.testing.assert_allclose(pa * ta, pb * tb, rtol=1e-15)
    np.testing.assert_allclose(pa, pb, rtol=1e-14)
    np.testing.assert_allclose(ka, kb, rtol=1e-14)
    np.testing.assert_allclose(ta, tb, rtol=1e-13)
    np.testing.assert_array_equal(a.events(), b.events())


def test_full_size_s_sweep_sampled(pg):
    # the 64-population s-sweep at full size (2^20 clones) in the bench's launch
    # configuration (pop_run); three sampled populations checked bit for bit
    w = workloads.s_sweep()
    M = 4
    batch = pg.PopulationBatch(w["pops"])
    batch.run(w["dt"], w["s"], M)
    psi, _, _ = batch.estimate_psi()
    for p in (0, 31, 63):
        q = w["pops"][p]
        o = oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"])
        for _ in range(M):
            o.evolve(w["dt"])
            o.resample(w["s"][p])
        g = batch.copy_state(p)
        assert np.array_equal(g["anc"], o.anc)
        assert_state_equal(g, o, batch.W, "s-sweep pop %d" % p)
        np.testing.assert_allclose(psi[p], o.estimates()[0], rtol=PSI_RTOL)
    # properties at every population: N conserved, ancestors monotone and in range
    for p in range(0, 64, 9):
        g = batch.copy_state(p)
        counts = sum(np.vectorize(lambda v: bin(int(v)).count("1"))(g["lattice"][:, q])
                     for q in range(batch.W))
        assert np.all(counts == w["pops"][p]["N"])
        assert np.all(np.diff(g["anc"]) >= 0)
        assert g["anc"].min() >= 0 and g["anc"].max() < w["pops"][p]["n_clones"]


def test_full_size_large_population_run(pg):
    # the bench's population shape (L = 128, N_c = 2^20) through pop_run: the fused
    # kernel for rings that fill the words, with the per-tile activity counts, over
    # three intervals, against the oracle
    q = dict(L=128, N=64, n_clones=2**20, seed=2001)
    s = 15.0 / 128**2
    batch = pg.PopulationBatch([q])
    assert batch.get_tuning()["hist_mode"] == -1
    batch.run(0.05, [s], 3)
    o = oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"])
    for _ in range(3):
        o.evolve(0.05)
        o.resample(s)
    g = batch.copy_state(0)
    assert np.array_equal(g["anc"], o.anc)
    assert_state_equal(g, o, batch.W, "large population run")
    np.testing.assert_allclose(batch.estimate_psi()[0][0], o.estimates()[0], rtol=PSI_RTOL)


def test_full_size_large_population_one_interval(pg):
    # one population at the largest size (L = 128, N_c = 2^20), one interval
    q = dict(L=128, N=64, n_clones=2**20, seed=2000)
    s = 15.0 / 128**2
    batch = pg.PopulationBatch([q])
    batch.evolve(0.05, [s])
    batch.resample()
    o = oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"])
    o.evolve(0.05)
    o.resample(s)
    g = batch.copy_state(0)
    assert np.array_equal(g["anc"], o.anc)
    assert np.array_equal(g["dK"], o.dK)
    assert_state_equal(g, o, batch.W, "large population")
    np.testing.assert_allclose(batch.estimate_psi()[0][0], o.estimates()[0], rtol=PSI_RTOL)


def test_set_state_from_host(pg):
    q = dict(L=70, N=33, n_clones=1500, seed=42)
    words = workloads.random_subsets(q["L"], q["N"], q["n_clones"], seed=9)
    K0 = np.arange(q["n_clones"], dtype=np.int32)
    batch = pg.PopulationBatch([q])
    batch.set_state(0, words, K0)
    g = batch.copy_state(0)
    assert np.array_equal(g["lattice"], words) and np.array_equal(g["K"], K0)
    sites = np.zeros((q["n_clones"], q["L"]), dtype=np.uint8)
    for i in range(q["L"]):
        sites[:, i] = (words[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1)
    out, K, dK = oracle.evolve_sites(q["L"], sites, 0.1, beta=1, seed=q["seed"], K=K0)
    batch.evolve(0.1, [0.1])
    g = batch.copy_state(0)
    assert np.array_equal(g["lattice"], oracle.sites_to_words(out, batch.W))
    assert np.array_equal(g["K"], K) and np.array_equal(g["dK"], dK)
    with pytest.raises(pg.PopError):
        bad = words.copy()
        bad[0, 0] ^= np.uint64(1)   # wrong particle number
        pg.PopulationBatch([q]).set_state(0, bad)


def test_call_order_and_bias_errors(pg):
    batch = pg.PopulationBatch([dict(L=20, N=10, n_clones=100, seed=1)])
    with pytest.raises(pg.PopError) as e:
        batch.resample()
    assert e.value.status == pg.POP_ERR_STATE
    with pytest.raises(pg.PopError) as e:
        batch.estimate_psi()
    assert e.value.status == pg.POP_ERR_STATE
    batch.evolve(0.1, [0.2])
    with pytest.raises(pg.PopError) as e:
        batch.evolve(0.1, [0.2])
    assert e.value.status == pg.POP_ERR_STATE
    batch.resample()
    with pytest.raises(pg.PopError) as e:
        batch.evolve(0.1, [0.3])
    assert e.value.status == pg.POP_ERR_STATE
    with pytest.raises(pg.PopError) as e:
        batch.evolve(-0.1, [0.2])
    assert e.value.status == pg.POP_ERR_ARG


@pytest.mark.parametrize("L,N,nc,s,dt", [
    (129, 64, 1100, 0.01, 0.05),     # narrowest ring of the one-clone-per-warp evolve
    (200, 37, 2100, -0.02, 0.05),
    (256, 128, 1025, 0.003, 0.05),   # exactly two lanes of sites
    (1000, 500, 700, 0.001, 0.01),
    (4096, 2048, 300, 0.0001, 0.005),  # widest ring: all 32 lanes, closing bond in lane 31
    (3000, 1, 500, 0.5, 0.2),        # one particle on a long ring
])
def test_parity_wide_rings(pg, L, N, nc, s, dt):
    run_parity(pg, [dict(L=L, N=N, n_clones=nc, seed=77 + L)], [s], dt, 3)


def test_parity_mixed_batch_wide(pg):
    # one ring above 128 sites puts every population of the batch on the wide path
    pops = [dict(L=50, N=25, n_clones=1500, seed=1), dict(L=300, N=150, n_clones=1100, seed=2),
            dict(L=7, N=3, n_clones=900, seed=3)]
    run_parity(pg, pops, [0.02, 0.004, -0.3], 0.05, 3)


MOD, IID = 1, 1


@pytest.mark.parametrize("L,N,nc,s,mode,sel", [
    (20, 10, 1500, 0.3, MOD, 0),
    (50, 25, 2100, -0.2, MOD, 0),
    (100, 40, 1100, 0.05, MOD, 0),       # two-word lattices
    (300, 150, 600, 0.01, MOD, 0),       # one clone per warp
    (37, 5, 1, 0.5, MOD, 0),             # one clone
    (20, 10, 1500, 0.3, 0, IID),
    (64, 31, 1300, -0.1, MOD, IID),
    (200, 100, 800, 0.02, 0, IID),       # one clone per warp
    (12, 0, 300, 0.3, MOD, 0),           # empty ring: A = 0, equal weights
])
def test_parity_modified_and_iid(pg, L, N, nc, s, mode, sel):
    pops = [dict(L=L, N=N, n_clones=nc, seed=555 + L, weight_mode=mode, selection=sel)]
    run_parity(pg, pops, [s], 0.1 if L < 100 else 0.05, 5)


def test_parity_mixed_modes_batch(pg):
    pops = [dict(L=30, N=15, n_clones=1200, seed=1),
            dict(L=40, N=20, n_clones=2100, seed=2, weight_mode=MOD),
            dict(L=50, N=25, n_clones=900, seed=3, selection=IID),
            dict(L=60, N=20, n_clones=1500, seed=4, weight_mode=MOD, selection=IID)]
    run_parity(pg, pops, [0.1, -0.05, 0.02, 0.3], 0.1, 4)


def test_parity_iid_beyond_the_staged_tile_prefixes(pg):
    # [iid] selection searches the tile prefixes first: from shared memory for up to
    # 2048 tiles, from global memory beyond (here 2101 tiles with a ragged last one)
    # next to a population of 3 tiles
    pops = [dict(L=20, N=10, n_clones=2100 * 1024 + 5, seed=91, selection=IID),
            dict(L=30, N=12, n_clones=2500, seed=92, selection=IID)]
    run_parity(pg, pops, [0.05, -0.1], 0.1, 2)


@pytest.mark.parametrize("L,dt", [(20, 10.0), (50, 1.0), (50, 10.0)])
def test_selection_study_state_point_matches_oracle(pg, L, dt):
    # the cloning-interval and selection study's configuration (lambda = 28, [eq] and
    # [iid], plain and MODIFIED weights in one batch, long intervals with wide activity
    # spreads), truncated to a few intervals: bit for bit against the oracle
    s = 28.0 / L ** 2
    pops = [dict(L=L, N=L // 2, n_clones=2100, seed=70 + 10 * m + e, weight_mode=m, selection=e)
            for m in (0, MOD) for e in (0, IID)]
    run_parity(pg, pops, [s] * 4, dt, 3)


@pytest.mark.parametrize("L,N,nc,W_case", [(50, 25, 2500, 1), (100, 50, 1300, 2), (300, 90, 700, 0)])
def test_density_mode_matches_oracle(pg, L, N, nc, W_case):
    q = dict(L=L, N=N, n_clones=nc, seed=31 + L)
    s = 20.0 / L**2
    batch = pg.PopulationBatch([q])
    o = oracle.Population(L, N, nc, q["seed"])
    for _ in range(4):
        batch.evolve(0.1, [s]); batch.resample()
        o.evolve(0.1); o.resample(s)
    for n in (0, 1, 3):
        got = batch.density_mode(n)[0]
        np.testing.assert_allclose(got, oracle.density_mode(o.sites, n), rtol=1e-12)


def test_full_size_uneven_batch_sampled(pg):
    # 256 populations of uneven L (32..128), N_c (2^10..2^18) and s, one batch, in
    # the captured-graph launch (pop_run); three small populations checked bit for
    # bit, invariants everywhere
    w = workloads.uneven_batch()
    M = 3
    batch = pg.PopulationBatch(w["pops"])
    batch.run(w["dt"], w["s"], M)
    psi, _, _ = batch.estimate_psi()
    ncs = np.array([q["n_clones"] for q in w["pops"]])
    for p in np.argsort(ncs)[:3]:
        q = w["pops"][p]
        o = oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"])
        for _ in range(M):
            o.evolve(w["dt"])
            o.resample(w["s"][p])
        g = batch.copy_state(int(p))
        assert np.array_equal(g["anc"], o.anc)
        assert_state_equal(g, o, batch.W, "uneven pop %d" % p)
        np.testing.assert_allclose(psi[p], o.estimates()[0], rtol=PSI_RTOL)
    for p in range(0, 256, 17):
        g = batch.copy_state(p)
        assert np.all(np.diff(g["anc"]) >= 0)
        assert g["anc"].max() < w["pops"][p]["n_clones"]
        assert np.all(np.isfinite(psi))


@pytest.mark.parametrize("case", ["one_word", "two_words_modified"])
def test_cloning_stage_beyond_4096_tiles(pg, case):
    # batches of more than 4096 tiles take the 256-thread cloning stage, and
    # populations of more than 64 tiles take their tile prefixes from k_tile_scan
    # (here over several 1024-tile chunks): every population checked bit for bit
    # against the oracle each interval, and in the large ones every new clone is its
    # ancestor's evolved clone with [eq] ancestors non-decreasing
    if case == "one_word":
        pops = [dict(L=20, N=10, n_clones=1500, seed=41), dict(L=30, N=15, n_clones=2100 * 1024, seed=42),
                dict(L=64, N=31, n_clones=777, seed=43, selection=1), dict(L=50, N=25, n_clones=2048 * 1024, seed=44),
                dict(L=40, N=20, n_clones=3000, seed=45, weight_mode=1)]
        s = [0.05, 0.01, -0.2, 0.02, 0.3]
    else:
        pops = [dict(L=100, N=50, n_clones=1100, seed=46, weight_mode=1),
                dict(L=128, N=64, n_clones=4096 * 1024, seed=47),
                dict(L=65, N=30, n_clones=2500, seed=48, weight_mode=1)]
        s = [0.1, 0.003, -0.1]
    batch = pg.PopulationBatch(pops)
    assert batch.slots // 1024 > 4096
    big = [p for p, q in enumerate(pops) if q["n_clones"] > 64 * 1024]
    orcs = oracle_pops(pops)
    for beta in range(1, 3):
        batch.evolve(0.1, s)
        evolved = {p: batch.copy_state(p) for p in big}
        batch.resample()
        for p, o in enumerate(orcs):
            o.evolve(0.1, s[p])
            o.resample(s[p])
            g = batch.copy_state(p)
            assert np.array_equal(g["anc"], o.anc), "anc beta=%d pop %d" % (beta, p)
            assert_state_equal(g, o, batch.W, "beta=%d pop %d" % (beta, p))
        for p in big:
            g, e = batch.copy_state(p), evolved[p]
            anc = g["anc"]
            assert np.all(np.diff(anc) >= 0)
            assert np.array_equal(g["lattice"], e["lattice"][anc]), "lattice beta=%d pop %d" % (beta, p)
            assert np.array_equal(g["K"], e["K"][anc]), "K beta=%d pop %d" % (beta, p)
    psi, _, _ = batch.estimate_psi()
    for p, o in enumerate(orcs):
        np.testing.assert_allclose(psi[p], o.estimates()[0], rtol=PSI_RTOL, atol=0.0)


def test_autotune_changes_no_result(pg):
    pops = [dict(L=50, N=25, n_clones=5000, seed=9), dict(L=128, N=64, n_clones=3000, seed=10)]
    s = [0.01, -0.002]
    a = pg.PopulationBatch(pops)
    tuned = a.autotune(0.1, s, trials=3)
    assert tuned["evolve_grid"] > 0 and tuned["tuned_us_per_interval"] > 0
    assert tuned["tuned_us_per_interval"] <= tuned["default_us_per_interval"]
    b = pg.PopulationBatch(pops)
    a.run(0.1, s, 40)
    b.run(0.1, s, 40)
    for p in range(2):
        ga, gb = a.copy_state(p), b.copy_state(p)
        for key in ("lattice", "K", "anc", "dK"):
            assert np.array_equal(ga[key], gb[key]), key
    np.testing.assert_array_equal(a.estimate_psi()[0], b.estimate_psi()[0])
    np.testing.assert_array_equal(a.events(), b.events())
    with pytest.raises(pg.PopError):
        a.autotune(0.1, s)   # only before the first interval


@pytest.mark.parametrize("cfg", [
    dict(fuse_threads=128, fuse_clones=1, chains=1), dict(fuse_threads=128, fuse_clones=2, chains=1),
    dict(fuse_threads=256, fuse_clones=1, chains=1), dict(fuse_threads=128, fuse_clones=1, chains=2),
    dict(fuse_threads=128, fuse_clones=2, chains=4), dict(fuse_threads=256, fuse_clones=1, chains=8),
    dict(evolve_grid=7, chains=3), dict(gather_threads=256), dict(gather_threads=128),
    dict(hist_mode=0), dict(hist_mode=1, chains=4), dict(hist_mode=0, fuse_clones=2, chains=2)])
def test_every_tuned_parameter_changes_no_result(pg, cfg):
    # every value of every tuned parameter gives the same lattices, activities,
    # ancestors and psi as the configuration pop_init chose (a fused batch of five
    # populations, mixed L and tile counts, both signs of s)
    pops = [dict(L=50, N=25, n_clones=5000, seed=31), dict(L=128, N=64, n_clones=3000, seed=32),
            dict(L=100, N=40, n_clones=1100, seed=33), dict(L=70, N=35, n_clones=2500, seed=34),
            dict(L=128, N=60, n_clones=4100, seed=35)]
    s = [0.01, -0.002, 0.004, 0.0, 0.02]
    a = pg.PopulationBatch(pops)
    a.set_tuning(**cfg)
    got = a.get_tuning()
    for k, v in cfg.items():
        assert got[k] == v or (k == "chains" and 1 <= got[k] <= v), (k, got[k], v)
    b = pg.PopulationBatch(pops)
    a.run(0.1, s, 37)
    b.run(0.1, s, 37)
    for p in range(len(pops)):
        ga, gb = a.copy_state(p), b.copy_state(p)
        for key in ("lattice", "K", "anc", "dK"):
            assert np.array_equal(ga[key], gb[key]), (p, key)
    np.testing.assert_array_equal(a.estimate_psi()[0], b.estimate_psi()[0])
    np.testing.assert_array_equal(a.events(), b.events())


def test_gather_tuning_of_a_batch_that_does_not_fuse_changes_no_result(pg):
    # an [iid] population keeps the separate cloning stage, whose block size the tuner
    # times on trials that write the population (kept aside and put back)
    pops = [dict(L=50, N=25, n_clones=6000, seed=41, selection=pg.POP_IID),
            dict(L=128, N=64, n_clones=5000, seed=42)]
    s = [0.01, 0.003]
    a = pg.PopulationBatch(pops)
    tuned = a.autotune(0.1, s, trials=2)
    assert tuned["gather_threads"] in (0, 128, 256)
    b = pg.PopulationBatch(pops)
    a.run(0.1, s, 20)
    b.run(0.1, s, 20)
    for p in range(2):
        ga, gb = a.copy_state(p), b.copy_state(p)
        for key in ("lattice", "K", "anc", "dK"):
            assert np.array_equal(ga[key], gb[key]), (p, key)
    np.testing.assert_array_equal(a.estimate_psi()[0], b.estimate_psi()[0])


def test_set_tuning_rejects_out_of_range(pg):
    a = pg.PopulationBatch([dict(L=50, N=25, n_clones=2000, seed=1)])
    for bad in (dict(fuse_threads=64), dict(fuse_clones=3), dict(fuse_threads=256, fuse_clones=2),
                dict(chains=0), dict(chains=9), dict(gather_threads=512), dict(evolve_grid=0),
                dict(hist_mode=2), dict(hist_mode=-2)):
        with pytest.raises(pg.PopError):
            a.set_tuning(**bad)


def test_kernel_times_equals_run_and_counts(pg):
    # pop_kernel_times launches what pop_run launches (results identical); the
    # launch counters follow the fused sequence: one dynamical stage, then
    # (n - 1) x [weights, fused stage] per chain, then weights and the cloning stage.
    # With populations of more than 64 tiles (below) the fused stages count activities
    # per tile and, after the first fused interval, the tile scan takes k_weights' place
    # (a launch of the "weights" kind that also scans)
    pops = [dict(L=50, N=25, n_clones=3000, seed=21), dict(L=90, N=45, n_clones=2000, seed=22)]
    s = [0.02, -0.003]
    n = 40
    a = pg.PopulationBatch(pops)
    b = pg.PopulationBatch(pops)
    a.run(0.1, s, n)
    kt = b.kernel_times(0.1, s, n)
    for p in range(len(pops)):
        ga, gb = a.copy_state(p), b.copy_state(p)
        for key in ("lattice", "K", "anc", "dK"):
            assert np.array_equal(ga[key], gb[key]), key
    np.testing.assert_array_equal(a.events(), b.events())
    # two chains (below): each fused interval is two launches of each kind, and the
    # reported time is the time during which either runs, per interval
    assert kt["evolve"][1] == 1 and kt["gather_evolve"][1] == 2 * (n - 1)
    assert kt["weights"][1] == 2 * (n - 1) + 1 and kt["gather"][1] == 1
    assert kt["evolve"][2] + kt["gather_evolve"][2] == int(b.events().sum())
    for name in ("evolve", "weights", "gather", "gather_evolve"):
        assert kt[name][0] > 0.0
    # pop_run splits this batch (3 + 2 tiles, each at least a quarter) into two chains,
    # each with its own [weights, fused stage] per interval, and kernel_times launches
    # the same chains
    assert a.run_chains() == [0, 3, 5] and b.run_chains() == [0, 3, 5]
    for batch, chains in ((a, 2), (b, 2)):
        c = batch.launch_count()
        assert c["evolve"] == 1 and c["gather_evolve"] == chains * (n - 1)
        assert c["weights"] == chains * (n - 1) + 1
        # the initial state, and the tile scan before the one separate cloning stage
        # (the fused stages of these 2- and 3-tile populations sum their tile sums)
        assert c["gather"] == 1 and c["other"] == 2
    # one population, or a split that would leave less than a quarter: one chain
    for pops1 in ([dict(L=50, N=25, n_clones=3000, seed=24)],
                  [dict(L=50, N=25, n_clones=9000, seed=25), dict(L=40, N=20, n_clones=2000, seed=26)]):
        d = pg.PopulationBatch(pops1)
        assert d.run_chains() == [0, d.slots // 1024]
        d.run(0.1, [0.02] * len(pops1), n)
        c = d.launch_count()
        assert c["gather_evolve"] == n - 1 and c["weights"] == n, pops1
    # [iid] batches keep the three separate kernels (and the [iid] selection) per interval
    c = pg.PopulationBatch([dict(L=30, N=15, n_clones=1500, seed=23, selection=1)])
    c.run(0.1, [0.1], 35)
    cnt = c.launch_count()
    assert cnt["evolve"] == 35 and cnt["weights"] == 35 and cnt["gather"] == 70
    assert cnt["gather_evolve"] == 0 and cnt["other"] == 1 + 35
    # populations of more than 64 tiles: the fused stage after k_weights takes the tile
    # scan too (once per chain, in the first fused interval); without the tile
    # histograms, in every interval
    big = [dict(L=50, N=25, n_clones=65 * 1024, seed=60 + i) for i in range(2)]
    d = pg.PopulationBatch(big)
    d.run(0.1, [0.02, 0.03], n)
    cnt = d.launch_count()
    chains = len(d.run_chains()) - 1
    assert cnt["gather_evolve"] == chains * (n - 1) and cnt["other"] == 1 + chains
    assert cnt["weights"] == chains * (n - 1) + 1
    d = pg.PopulationBatch(big)
    d.set_tuning(hist_mode=0)
    d.run(0.1, [0.02, 0.03], n)
    cnt = d.launch_count()
    assert cnt["gather_evolve"] == chains * (n - 1) and cnt["other"] == 1 + chains * (n - 1) + 1


@pytest.mark.parametrize("dt", [0.1, 1.5])
def test_tile_histograms_change_no_result(pg, dt):
    # the fused stage's per-tile activity counts (hist_mode 1) against k_weights'
    # pass over every clone (hist_mode 0): the same lattices, activities, ancestors and
    # psi bit for bit, over two chains and populations of one and many tiles.  At
    # dt = 1.5 the L = 128 populations hop about 100 times an interval, beyond the 64
    # counted activities, so their tile sums come from the slower pass over the clones
    # while the L = 20 population's still come from the counts
    pops = [dict(L=20, N=10, n_clones=5000, seed=71), dict(L=128, N=64, n_clones=70 * 1024, seed=72),
            dict(L=128, N=40, n_clones=3000, seed=73), dict(L=100, N=50, n_clones=66 * 1024, seed=74)]
    s = [0.05, 0.002, -0.01, 0.0]
    runs = []
    for mode in (1, 0):
        b = pg.PopulationBatch(pops)
        b.set_tuning(hist_mode=mode, chains=2)
        b.run(dt, s, 7)
        b.run(dt, s, 5)   # a second call: the counts of the first were all consumed
        runs.append(b)
    a, b = runs
    assert a.run_chains() == b.run_chains() and len(a.run_chains()) == 3
    for p in range(len(pops)):
        ga, gb = a.copy_state(p), b.copy_state(p)
        for key in ("lattice", "K", "anc", "dK"):
            assert np.array_equal(ga[key], gb[key]), (p, key)
    np.testing.assert_array_equal(a.estimate_psi()[0], b.estimate_psi()[0])
    np.testing.assert_array_equal(a.events(), b.events())
    if dt > 1.0:
        assert int(b.copy_state(1)["dK"].max()) >= 64


def test_activity_spread_beyond_the_weight_table_is_reported(pg):
    # one particle on 128 sites, dt = 2.5e5: about 5e5 hops per clone with a spread of
    # ~5000 across 4000 clones, beyond the 4096-entry weight table: the cloning stage
    # reports POP_ERR_RANGE instead of indexing past the table
    b = pg.PopulationBatch([dict(L=128, N=1, n_clones=4000, seed=3)])
    b.evolve(2.5e5, [0.001])
    b.resample()
    with pytest.raises(pg.PopError) as e:
        b.events()
    assert e.value.status == pg.POP_ERR_RANGE
    b.close()
    # the device stays usable
    ok = pg.PopulationBatch([dict(L=20, N=10, n_clones=100, seed=4)])
    ok.run(0.1, [0.1], 3)
    assert np.isfinite(ok.estimate_psi()[0][0])


def test_an_interval_that_cannot_end_stops_at_the_step_limit(pg):
    # dt = 1e7 in FP32: once t is near 1e7 a waiting time of ~0.5 no longer changes t,
    # so only the per-interval step limit (2^24 steps) ends the clone's loop; the
    # kernel reports POP_ERR_RANGE and returns instead of spinning
    b = pg.PopulationBatch([dict(L=128, N=1, n_clones=1, seed=5)])
    b.evolve(1e7, [0.0])
    with pytest.raises(pg.PopError) as e:
        b.events()
    assert e.value.status == pg.POP_ERR_RANGE
    b.close()
    # the same through pop_run: the fused cloning + dynamical stage of the second
    # interval stops at the limit too
    b = pg.PopulationBatch([dict(L=128, N=1, n_clones=1, seed=6)])
    b.run(1e7, [0.0], 2)
    with pytest.raises(pg.PopError) as e:
        b.events()
    assert e.value.status == pg.POP_ERR_RANGE
    b.close()
