"""GUIDED dynamics on the GPU against the oracle (reading R15: modified dynamics of
Sec. 2.2 with a local potential), on identical Philox streams.

Bit-exact lattices, K, dK and ancestors every interval; psi within 1e-12 relative.
Cases: one- and two-word lattices, the smallest allowed ring (18: windows wrap),
ring lengths either side of 64, both signs of s, a zero potential, and run() against
the per-step calls.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

PSI_RTOL = 1e-12
GUIDED = 2


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05095_gb300 import build
    build.build()
    import paper_1711_05095_gb300 as pg
    return pg


def potential(seed, scale):
    return np.random.default_rng(seed).normal(0.0, scale, 512).astype(np.float32)


def guided_parity(pg, pops, s, dt, M, phis):
    pops = [dict(q, weight_mode=GUIDED) for q in pops]
    batch = pg.PopulationBatch(pops)
    for p, phi in enumerate(phis):
        batch.set_potential(p, phi)
    orcs = [oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"], phi=phi) for q, phi in zip(pops, phis)]
    W = batch.W
    for beta in range(1, M + 1):
        batch.evolve(dt, s)
        for p, o in enumerate(orcs):
            o.evolve(dt, s[p])
            g = batch.copy_state(p)
            words = oracle.sites_to_words(o.sites, W)
            assert np.array_equal(g["lattice"], words), "evolve beta=%d pop %d: lattice" % (beta, p)
            assert np.array_equal(g["K"], o.K), "evolve beta=%d pop %d: K" % (beta, p)
            assert np.array_equal(g["dK"], o.dK), "evolve beta=%d pop %d: dK" % (beta, p)
        batch.resample()
        for p, o in enumerate(orcs):
            o.resample(s[p])
            g = batch.copy_state(p)
            assert np.array_equal(g["anc"], o.anc), "resample beta=%d pop %d: anc" % (beta, p)
            assert np.array_equal(g["lattice"], oracle.sites_to_words(o.sites, W))
    psi, _, _ = batch.estimate_psi()
    ev = batch.events()
    for p, o in enumerate(orcs):
        np.testing.assert_allclose(psi[p], o.estimates()[0], rtol=PSI_RTOL, atol=0.0)
        assert int(ev[p]) == o.events
    return batch, orcs


@pytest.mark.parametrize("L,N,nc,s,scale", [
    (18, 9, 1500, 0.1, 0.3),      # smallest ring: the 18-site windows wrap
    (20, 10, 2100, 0.05, 0.4),
    (50, 25, 1100, -0.02, 0.3),
    (64, 32, 1200, 0.01, 0.2),    # widest one-word ring
    (65, 30, 1000, 0.02, 0.2),    # narrowest two-word ring
    (128, 64, 1300, 15.0 / 128**2, 0.25),
    (40, 20, 900, 0.2, 0.0),      # zero potential: rates e^-s
])
def test_guided_parity_single(pg, L, N, nc, s, scale):
    guided_parity(pg, [dict(L=L, N=N, n_clones=nc, seed=4000 + L)], [s], 0.1 if L < 100 else 0.05, 4,
                  [potential(L, scale)])


def test_guided_parity_batch(pg):
    pops = [dict(L=30, N=15, n_clones=1500, seed=1), dict(L=100, N=50, n_clones=1025, seed=2),
            dict(L=77, N=20, n_clones=700, seed=3)]
    guided_parity(pg, pops, [0.05, -0.01, 0.1], 0.1, 4, [potential(1, 0.3), potential(2, 0.2), potential(3, 0.5)])


def test_guided_parity_batch_one_word(pg):
    # one-word lattices (L <= 64): the kernel keeps exponent rows for 64 bonds
    pops = [dict(L=18, N=7, n_clones=1300, seed=11), dict(L=64, N=32, n_clones=2049, seed=12),
            dict(L=41, N=20, n_clones=600, seed=13)]
    guided_parity(pg, pops, [0.2, 0.004, -0.05], 0.1, 4, [potential(7, 0.4), potential(8, 0.1), potential(9, 0.3)])


def test_guided_run_equals_steps(pg):
    pops = [dict(L=50, N=25, n_clones=2000, seed=7, weight_mode=GUIDED),
            dict(L=100, N=40, n_clones=1300, seed=8, weight_mode=GUIDED)]
    s = [0.01, -0.004]
    a, b = pg.PopulationBatch(pops), pg.PopulationBatch(pops)
    for batch in (a, b):
        batch.set_potential(0, potential(5, 0.3))
        batch.set_potential(1, potential(6, 0.2))
    a.run(0.1, s, 37)
    for _ in range(37):
        b.evolve(0.1, s)
        b.resample()
    for p in range(2):
        ga, gb = a.copy_state(p), b.copy_state(p)
        for key in ("lattice", "K", "anc", "dK"):
            assert np.array_equal(ga[key], gb[key]), key
    np.testing.assert_allclose(a.estimate_psi()[0] * a.estimate_psi()[2],
                               b.estimate_psi()[0] * b.estimate_psi()[2], rtol=1e-15)
    c = a.launch_count()
    assert c["gather_evolve"] == 0 and c["evolve"] == 37


def test_guided_argument_errors(pg):
    with pytest.raises(pg.PopError):   # a ring below 18 sites
        pg.PopulationBatch([dict(L=12, N=6, n_clones=10, seed=1, weight_mode=GUIDED)])
    with pytest.raises(pg.PopError):   # GUIDED mixed with another mode
        pg.PopulationBatch([dict(L=20, N=10, n_clones=10, seed=1, weight_mode=GUIDED),
                            dict(L=20, N=10, n_clones=10, seed=2)])
    plain = pg.PopulationBatch([dict(L=20, N=10, n_clones=10, seed=1)])
    with pytest.raises(pg.PopError):   # the potential of a population that is not GUIDED
        plain.set_potential(0, np.zeros(512, np.float32))
    g = pg.PopulationBatch([dict(L=20, N=10, n_clones=10, seed=1, weight_mode=GUIDED)])
    bad = np.zeros(512, np.float32)
    bad[7] = 65.0
    with pytest.raises(pg.PopError):
        g.set_potential(0, bad)


def test_potential_changed_between_intervals(pg):
    # the clones carry their rate sums from one interval to the next; a new potential
    # invalidates them (they are formed again from the new bond tables): bit for bit
    # against the oracle with the potential switched after two intervals, also in run()
    L, N, nc, s, dt = 60, 30, 2300, 0.03, 0.1
    phi1, phi2 = potential(11, 0.3), potential(12, 0.4)
    q = dict(L=L, N=N, n_clones=nc, seed=77, weight_mode=GUIDED)
    batch = pg.PopulationBatch([q])
    batch.set_potential(0, phi1)
    o = oracle.Population(L, N, nc, q["seed"], phi=phi1)
    batch.run(dt, [s], 2)
    for _ in range(2):
        o.evolve(dt, s)
        o.resample(s)
    batch.set_potential(0, phi2)
    o.phi_q = oracle.phi_fixed(phi2)
    batch.run(dt, [s], 3)
    for _ in range(3):
        o.evolve(dt, s)
        o.resample(s)
    g = batch.copy_state(0)
    assert np.array_equal(g["lattice"], oracle.sites_to_words(o.sites, batch.W))
    assert np.array_equal(g["K"], o.K) and np.array_equal(g["anc"], o.anc)
    np.testing.assert_allclose(batch.estimate_psi()[0][0], o.estimates()[0], rtol=PSI_RTOL, atol=0.0)
