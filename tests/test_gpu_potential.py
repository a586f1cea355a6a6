"""The learned potential on the GPU (C ABI pop_mlp_*, pop_lineage) against the oracle
(oracle/mlp.py): loss, gradient and compiled table of the window network with BF16
operands and FP32 accumulation, one Adam step, and the ancestry composition."""
import numpy as np
import pytest

import oracle
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05095_gb300 import build
    build.build()
    import paper_1711_05095_gb300 as pg
    from paper_1711_05095_gb300 import potential
    return torch, pg, potential


def batch(n, L, seed):
    g = np.random.default_rng(seed)
    W = (L + 63) // 64
    words = np.zeros((n, W), dtype=np.uint64)
    for r in range(n):
        for i in g.choice(L, size=L // 2, replace=False):
            words[r, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return words, g.integers(0, 2, n).astype(np.uint8)


@pytest.mark.parametrize("L,n", [(20, 300), (70, 200), (128, 150), (50, 4096)])
def test_loss_and_gradient_match_oracle(env, L, n):
    # every element of the gradient against the FP64 oracle with BF16 operands, within
    # the element-wise tolerance oracle/mlp.py derives for an FP32 / BF16 evaluation:
    # twice the first-order running error bound of FP32 sums (n u / (1 - n u) times the
    # magnitudes summed, the tensor-core products as K/16 accumulation steps), FP32
    # GELU / exp to a few ulp, and one BF16 ulp wherever an operand lies within its
    # error of a rounding tie (tests/test_oracle_mlp.py pins that bound against an
    # independent FP32 evaluation and against planted mistakes)
    torch, pg, potential = env
    theta = potential.init_params(7) + np.random.default_rng(L).normal(0, 0.05, potential.N_PARAMS).astype(np.float32)
    words, labels = batch(n, L, L)
    tr = potential.Trainer(theta=theta)
    loss, g = tr.grad(torch.from_numpy(words.view(np.int64)).cuda(), torch.from_numpy(labels).cuda(), L)
    want_loss, want_g = mlp.loss_and_grad(theta, words, labels, L, bf=True)
    tol_loss, tol = mlp.grad_tolerance(theta, words, labels, L)
    assert abs(loss - want_loss) <= tol_loss, (loss, want_loss, tol_loss)
    k = 0
    for name, shape in mlp.SIZES:
        m = int(np.prod(shape))
        np.testing.assert_array_less(np.abs(g[k:k + m] - want_g[k:k + m]), tol[k:k + m] + 1e-30,
                                     err_msg=name)
        k += m


def test_compiled_table_matches_oracle(env):
    # the 512 potential values against the oracle's forward pass, element-wise within
    # twice the running error bound of the FP32 / BF16 evaluation
    torch, pg, potential = env
    theta = potential.init_params(3) + np.random.default_rng(1).normal(0, 0.1, potential.N_PARAMS).astype(np.float32)
    tr = potential.Trainer(theta=theta)
    phi = tr.potential()
    want, _ = mlp.forward(theta, bf=True)
    np.testing.assert_array_less(np.abs(phi - want), mlp.phi_tolerance(theta) + 1e-30)


def test_adam_step_matches_oracle(env):
    torch, pg, potential = env
    theta = potential.init_params(5)
    words, labels = batch(256, 30, 2)
    X, y = torch.from_numpy(words.view(np.int64)).cuda(), torch.from_numpy(labels).cuda()
    tr = potential.Trainer(theta=theta)
    _, g = tr.grad(X, y, 30)
    tr.step(X, y, 30, 1e-2)
    want, _, _ = mlp.adam(theta, g.astype(np.float64), np.zeros_like(theta), np.zeros_like(theta), 1, 1e-2)
    np.testing.assert_allclose(tr.params(), want, rtol=1e-5, atol=1e-7)


def test_lineage_composes_ancestors(env):
    torch, pg, potential = env
    pops = [dict(L=20, N=10, n_clones=1500, seed=3), dict(L=40, N=20, n_clones=900, seed=4)]
    s = [0.3, -0.1]
    batch_ = pg.PopulationBatch(pops)
    orcs = [oracle.Population(q["L"], q["N"], q["n_clones"], q["seed"]) for q in pops]
    lin = torch.zeros(batch_.slots, dtype=torch.int32, device="cuda")
    for p, q in enumerate(pops):
        off = batch_.first_slot(p)
        lin[off:off + q["n_clones"]] = torch.arange(q["n_clones"], dtype=torch.int32, device="cuda")
    other = torch.zeros_like(lin)
    comp = [np.arange(q["n_clones"]) for q in pops]
    for _ in range(6):
        batch_.evolve(0.1, s)
        batch_.resample()
        batch_.lineage(lin, other)
        lin, other = other, lin
        for p, o in enumerate(orcs):
            o.evolve(0.1)
            o.resample(s[p])
            comp[p] = comp[p][o.anc]
    h = lin.cpu().numpy()
    for p, q in enumerate(pops):
        off = batch_.first_slot(p)
        np.testing.assert_array_equal(h[off:off + q["n_clones"]], comp[p])


def test_learned_potential_separates_and_guides_without_bias(env):
    # What the trained network gains: on the ancestral / end configurations of
    # lambda = 15 populations (L = 32) it tells p_ave from p_end better than chance
    # on populations it never saw.  Guided cloning with it stays unbiased: over 32
    # seeds its steady-state psi agrees with plain cloning's within 3 standard errors.
    torch, pg, potential = env
    from paper_1711_05095_gb300.study_guided import run_batch
    L, N, lam, dt = 32, 16, 15.0, 0.1
    s = lam / L ** 2
    pops = [dict(L=L, N=N, n_clones=8192, seed=100 + i) for i in range(8)]
    end, anc = potential.ancestral_samples(pops, [s] * 8, dt, burn=600, lag=600)
    cut = 8192 * 7
    tr, _ = potential.train(end[:cut], anc[:cut], L, steps=600, batch_size=4096, lr=3e-3)
    held = potential.classifier_loss(tr, end[cut:], anc[cut:], L)
    assert held < np.log(2.0) - 0.005, held
    phi = tr.potential()
    assert np.ptp(phi) > 0.05
    g, _, _ = run_batch(L, N, s, dt, 1000, 1024, 32, 7000, "guided", phi, burn=300)
    p, _, _ = run_batch(L, N, s, dt, 1000, 16384, 32, 8000, "plain", burn=300)
    se = np.hypot(g.std(ddof=1), p.std(ddof=1)) / np.sqrt(32)
    assert abs(g.mean() - p.mean()) < 3 * se, (g.mean(), p.mean(), se)
