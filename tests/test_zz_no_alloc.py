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
