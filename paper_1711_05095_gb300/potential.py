"""Learned guiding potential for GUIDED cloning (C ABI ``pop_mlp_*``, ``pop_lineage``).

The potential U(C) = sum_i phi(sites i-4..i+4) steers the GUIDED dynamics (rates
e^-s e^{(U(C') - U(C))/2}; Sec. 2.2, eqs. modpdef and upsdef).  The optimal (Doob)
control of the SSEP has U = 2 ln v, v the top eigenvector of the symmetric tilted
generator; since the end-of-interval population is distributed as p_end ~ v and the
ancestral (time-averaged) one as p_ave ~ v^2 (Sec. 2.2, eqs. Opave and Opend), a
classifier of ancestral against end configurations has the logit ln v + const.  The
window network phi is trained as that classifier on the GPU and compiled to the
512-entry table ``PopulationBatch.set_potential`` takes.

Typical use::

    end, anc = ancestral_samples(pops, s, dt, burn, lag)        # plain cloning runs
    tr, losses = train(end, anc, L, steps=2000)                 # Adam on the GPU
    phi = tr.potential()                                        # 512 floats
    guided = PopulationBatch([dict(q, weight_mode=POP_GUIDED) ...]); guided.set_potential(p, phi)
"""
import ctypes
import math

import numpy as np

from . import POP_ERR_ARG, PopError, PopulationBatch, _check, library

HIDDEN = 128
N_PARAMS = HIDDEN * 9 + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1 + 1
_f32p = ctypes.POINTER(ctypes.c_float)


def init_params(seed):
    """Initial parameters: weights uniform in +-1/sqrt(fan in) (seeded), biases zero.
    Order W1[128][9], b1, W2[128][128], b2, W3, b3, c."""
    g = np.random.default_rng(seed)
    parts = [g.uniform(-1, 1, HIDDEN * 9) / 3.0, np.zeros(HIDDEN),
             g.uniform(-1, 1, HIDDEN * HIDDEN) / math.sqrt(HIDDEN), np.zeros(HIDDEN),
             g.uniform(-1, 1, HIDDEN) / math.sqrt(HIDDEN), np.zeros(1), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


class Trainer:
    """The window network and its Adam state on one GPU."""

    def __init__(self, theta=None, seed=0, device="cuda", stream=None):
        import torch
        self._lib = library()
        theta = init_params(seed) if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        if theta.size != N_PARAMS:
            raise PopError(POP_ERR_ARG, "parameter count")
        self.device = torch.device(device)
        nbytes = int(self._lib.pop_mlp_workspace_bytes())
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._h = ctypes.c_void_p()
        _check(self._lib.pop_mlp_init(ctypes.byref(self._h), theta.ctypes.data_as(_f32p),
                                      ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                      ctypes.c_void_p(self.stream.cuda_stream)), "pop_mlp_init")

    @staticmethod
    def _batch(lattice, labels):
        import torch
        if lattice.dtype != torch.int64 or labels.dtype != torch.uint8 or lattice.dim() != 2:
            raise PopError(POP_ERR_ARG, "batch tensors")
        if lattice.shape[0] != labels.shape[0] or not lattice.is_contiguous() or not labels.is_contiguous():
            raise PopError(POP_ERR_ARG, "batch shapes")
        return (ctypes.c_void_p(lattice.data_ptr()), int(lattice.shape[1]),
                ctypes.c_void_p(labels.data_ptr()), int(lattice.shape[0]))

    def grad(self, lattice, labels, L):
        """(mean loss, gradient) of a batch: lattice int64 (n, W) words, labels uint8."""
        lp, W, yp, n = self._batch(lattice, labels)
        loss = ctypes.c_double(0.0)
        g = np.zeros(N_PARAMS, dtype=np.float32)
        _check(self._lib.pop_mlp_grad(self._h, lp, W, int(L), yp, n, ctypes.byref(loss), g.ctypes.data_as(_f32p)),
               "pop_mlp_grad")
        return loss.value, g

    def step(self, lattice, labels, L, lr, want_loss=False):
        lp, W, yp, n = self._batch(lattice, labels)
        loss = ctypes.c_double(0.0)
        _check(self._lib.pop_mlp_step(self._h, lp, W, int(L), yp, n, float(lr),
                                      ctypes.byref(loss) if want_loss else None), "pop_mlp_step")
        return loss.value if want_loss else None

    def params(self):
        out = np.zeros(N_PARAMS, dtype=np.float32)
        _check(self._lib.pop_mlp_params(self._h, out.ctypes.data_as(_f32p)), "pop_mlp_params")
        return out

    def potential(self):
        """phi at the 512 window patterns (bit k of the index = site i-4+k)."""
        out = np.zeros(512, dtype=np.float32)
        _check(self._lib.pop_mlp_potential(self._h, out.ctypes.data_as(_f32p)), "pop_mlp_potential")
        return out

    def close(self):
        if self._h:
            self._lib.pop_mlp_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ancestral_samples(pops, s, dt, burn, lag, device="cuda"):
    """End-of-interval and ancestral configurations of cloning runs.

    Runs the populations (plain or MODIFIED) for ``burn`` intervals, records the
    population, runs ``lag`` more intervals while composing the ancestry of every
    clone on the GPU (pop_lineage), and returns (end, anc): int64 arrays (n, W) of the
    final configurations (distributed as p_end) and of each final clone's ancestor
    ``lag`` intervals earlier (as p_ave when both runs are long against the
    relaxation time)."""
    import torch
    batch = PopulationBatch(pops, device=device)
    batch.run(dt, s, burn)
    start = [batch.copy_state(p)["lattice"] for p in range(len(pops))]
    n_slots = batch.slots
    lin = torch.zeros(n_slots, dtype=torch.int32, device=batch.device)
    for p, q in enumerate(pops):
        off = batch.first_slot(p)
        lin[off:off + q["n_clones"]] = torch.arange(q["n_clones"], dtype=torch.int32, device=batch.device)
    other = torch.zeros_like(lin)
    for _ in range(int(lag)):
        batch.evolve(dt, s)
        batch.resample()
        batch.lineage(lin, other)
        lin, other = other, lin
    lin_h = lin.cpu().numpy()
    end, anc = [], []
    for p, q in enumerate(pops):
        off = batch.first_slot(p)
        end.append(batch.copy_state(p)["lattice"])
        anc.append(start[p][lin_h[off:off + q["n_clones"]]])
    batch.close()
    return np.concatenate(end).view(np.int64), np.concatenate(anc).view(np.int64)


def train(end, anc, L, steps=1000, batch_size=4096, lr=3e-3, seed=0, device="cuda", log_every=0):
    """Train the classifier (ancestral = 1, end = 0) with Adam on minibatches drawn
    from the shuffled samples; returns (trainer, losses)."""
    import torch
    dev = torch.device(device)
    X = torch.from_numpy(np.ascontiguousarray(np.concatenate([end, anc]))).to(dev)
    y = torch.cat([torch.zeros(len(end), dtype=torch.uint8), torch.ones(len(anc), dtype=torch.uint8)]).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    tr = Trainer(seed=seed, device=dev)
    losses = []
    n = X.shape[0]
    perm = torch.randperm(n, generator=gen, device=dev)
    at = 0
    for it in range(int(steps)):
        if at + batch_size > n:
            perm = torch.randperm(n, generator=gen, device=dev)
            at = 0
        idx = perm[at:at + batch_size]
        at += batch_size
        want = log_every > 0 and (it % log_every == 0 or it == steps - 1)
        loss = tr.step(X.index_select(0, idx).contiguous(), y.index_select(0, idx).contiguous(), L, lr, want)
        if want:
            losses.append((it, loss))
    return tr, losses


def classifier_loss(trainer, end, anc, L, device="cuda"):
    """Mean cross-entropy of the trained classifier on held-out samples (ln 2 = chance)."""
    import torch
    dev = torch.device(device)
    X = torch.from_numpy(np.ascontiguousarray(np.concatenate([end, anc]))).to(dev)
    y = torch.cat([torch.zeros(len(end), dtype=torch.uint8), torch.ones(len(anc), dtype=torch.uint8)]).to(dev)
    return trainer.grad(X, y, L)[0]
