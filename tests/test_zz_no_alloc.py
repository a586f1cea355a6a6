"""pop_select_noalloc: the allocation-free selection entry point.

It exists for callers that cannot call cudaMalloc (a process whose device memory
is all reserved by another allocator, allocation-free latency-critical loops,
runtimes without a device allocator).  Its ancestors and psi term must equal those
of the batch path's pop_resample for the same interval activities, on two calls in
a row (the static scratch array keeps the previous call's contents, so the second
call checks that everything that must start at zero is cleared).  This file is
collected last so a run that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05095_gb300 import build
    build.build()
    import paper_1711_05095_gb300 as pg
    return pg


@pytest.mark.parametrize("L,N,nc,s", [(50, 25, 5000, 0.3), (100, 40, 3100, -0.05)])
def test_select_noalloc_matches_resample(pg, L, N, nc, s):
    import torch
    q = dict(L=L, N=N, n_clones=nc, seed=4242 + L)
    batch = pg.PopulationBatch([q])
    acc_prev = 0.0
    for interval in (1, 2):
        batch.evolve(0.1, [s])
        dK = batch.copy_state(0)["dK"]
        d_dK = torch.from_numpy(dK).to("cuda")
        d_anc = torch.full((nc,), -1, dtype=torch.int32, device="cuda")
        term = pg.select_noalloc(d_dK, s, q["seed"], interval, d_anc)
        batch.resample()
        ref = batch.copy_state(0)
        assert np.array_equal(d_anc.cpu().numpy(), ref["anc"]), "interval %d" % interval
        psi, _, t_obs = batch.estimate_psi()
        acc = float(psi[0]) * t_obs
        np.testing.assert_allclose(term, acc - acc_prev, rtol=1e-12, atol=1e-15)
        acc_prev = acc


def test_select_noalloc_rejects_oversize(pg):
    import torch
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    lib = pg.library()
    import ctypes
    rc = lib.pop_select_noalloc(ctypes.c_void_p(d.data_ptr()), pg.POP_NOALLOC_MAX_CLONES + 1, 0.1, 1, 1,
                                ctypes.c_void_p(d.data_ptr()), None, None)
    assert rc == pg.POP_ERR_ARG


def test_select_noalloc_at_the_clone_limit_matches_oracle(pg):
    # N_c = POP_NOALLOC_MAX_CLONES (1024 tiles, every block sums all 1024 tile sums):
    # ancestors bit for bit and the psi term to 1e-12 against the oracle's weights
    # (Sec. 4.1 eq. alpha-Ups with the exact fixed-point key) and eq. psihat term, on
    # two calls in a row with the same bias (the second reuses the uploaded tables)
    # and a third with another bias.
    import torch
    import oracle
    nc = pg.POP_NOALLOC_MAX_CLONES
    g = np.random.default_rng(20)
    seed = 99
    for interval, s in ((3, 0.01), (4, 0.01), (5, -0.004)):
        dK = g.poisson(3.2, nc).astype(np.int32)
        d_dK = torch.from_numpy(dK).to("cuda")
        d_anc = torch.full((nc,), -1, dtype=torch.int32, device="cuda")
        term = pg.select_noalloc(d_dK, s, seed, interval, d_anc)
        w, rc = oracle.weights(s, dK)
        assert rc == 0
        want = oracle.ancestors(w, interval, seed)
        assert np.array_equal(d_anc.cpu().numpy(), want), "interval %d" % interval
        want_term = oracle.psi_term(s, dK)
        assert abs(term - want_term) <= 1e-12 * abs(want_term), (term, want_term)


def test_select_noalloc_unbiased_is_the_identity(pg):
    # s = 0: every weight is 2^F, so [eq] selection keeps every clone (new j from old j)
    # and the psi term is exactly 0
    import torch
    nc = 70000
    dK = np.random.default_rng(5).poisson(2.0, nc).astype(np.int32)
    d_anc = torch.full((nc,), -1, dtype=torch.int32, device="cuda")
    term = pg.select_noalloc(torch.from_numpy(dK).to("cuda"), 0.0, 7, 1, d_anc)
    assert np.array_equal(d_anc.cpu().numpy(), np.arange(nc, dtype=np.int32))
    assert term == 0.0


def test_select_noalloc_reports_a_spread_beyond_the_table(pg):
    # an activity POP_KCAP or more away from the reference is a range error, never a clamp
    import torch
    dK = np.zeros(3000, dtype=np.int32)
    dK[17] = pg.POP_KCAP + 5
    d_anc = torch.zeros(3000, dtype=torch.int32, device="cuda")
    with pytest.raises(pg.PopError) as e:
        pg.select_noalloc(torch.from_numpy(dK).to("cuda"), 0.2, 1, 1, d_anc)
    assert e.value.status == pg.POP_ERR_RANGE
    # the array is usable again afterwards: a valid call still matches the oracle
    import oracle
    dK[17] = 3
    term = pg.select_noalloc(torch.from_numpy(dK).to("cuda"), 0.2, 1, 2, d_anc)
    w, _ = oracle.weights(0.2, dK)
    assert np.array_equal(d_anc.cpu().numpy(), oracle.ancestors(w, 2, 1))
    assert abs(term - oracle.psi_term(0.2, dK)) <= 1e-12 * abs(oracle.psi_term(0.2, dK))
