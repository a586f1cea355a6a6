"""CPU oracle for the SSEP cloning estimator (arXiv:1711.05095).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path.

Two parts:
  * ``cloning_oracle.c`` (wrapped here with ctypes): the cloning algorithm of
    Sec. 2.3 / Sec. 4 step by step, plain and serial, one byte per site.
  * ``ed.py``: exact diagonalisation of the tilted SSEP generator (Sec. 2.1,
    eqs. P-Theta, biastraj, psi-z), the exact psi(s) for small rings.

Pins that tie the oracle to something other than itself live in
``tests/test_oracle_*.py``.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)

KCAP = 4096


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_philox.argtypes = [_u32p, ctypes.c_uint64, _u32p]
        L.orc_philox.restype = None
        L.orc_neg_ln_u.argtypes = [ctypes.c_uint32]
        L.orc_neg_ln_u.restype = ctypes.c_float
        L.orc_init.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _u8p, _i32p]
        L.orc_init.restype = ctypes.c_int
        L.orc_evolve.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32,
                                 ctypes.c_uint64, _u8p, _i32p, _i32p]
        L.orc_evolve.restype = ctypes.c_int
        L.orc_weight_scale.argtypes = [ctypes.c_int64]
        L.orc_weight_scale.restype = ctypes.c_int32
        L.orc_k_ref.argtypes = [ctypes.c_double, ctypes.c_int64, _i32p]
        L.orc_k_ref.restype = ctypes.c_int32
        L.orc_weights.argtypes = [ctypes.c_double, ctypes.c_int64, _i32p, _u64p]
        L.orc_weights.restype = ctypes.c_int
        L.orc_psi_term.argtypes = [ctypes.c_double, ctypes.c_int64, _i32p]
        L.orc_psi_term.restype = ctypes.c_double
        L.orc_resample_word.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
        L.orc_resample_word.restype = ctypes.c_uint32
        L.orc_ancestors.argtypes = [ctypes.c_int64, _u64p, ctypes.c_uint32, ctypes.c_uint64, _i32p]
        L.orc_ancestors.restype = ctypes.c_int
        L.orc_gather.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _u8p, _i32p, _u8p, _i32p]
        L.orc_gather.restype = None
        L.orc_run.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_double, ctypes.c_double, ctypes.c_int64, _f64p, _f64p,
                              _u64p, _u8p, _i32p]
        L.orc_run.restype = ctypes.c_int
        L.orc_run_ex.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                 ctypes.c_int32, _f64p, _f64p, _u64p, _u8p, _i32p]
        L.orc_run_ex.restype = ctypes.c_int
        _f32p = ctypes.POINTER(ctypes.c_float)
        L.orc_evolve_modified.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_uint32, ctypes.c_uint64, _u8p, _i32p, _i32p, _f32p]
        L.orc_evolve_modified.restype = ctypes.c_int
        L.orc_weight_exp.argtypes = [ctypes.c_float, ctypes.c_int]
        L.orc_weight_exp.restype = ctypes.c_uint64
        L.orc_weights_modified.argtypes = [ctypes.c_double, ctypes.c_int64, _f32p, _u64p]
        L.orc_weights_modified.restype = ctypes.c_int
        L.orc_psi_term_modified.argtypes = [ctypes.c_double, ctypes.c_int64, _f32p]
        L.orc_psi_term_modified.restype = ctypes.c_double
        L.orc_ancestors_iid.argtypes = [ctypes.c_int64, _u64p, ctypes.c_uint32, ctypes.c_uint64, _i32p]
        L.orc_ancestors_iid.restype = ctypes.c_int
        L.orc_density_mode.argtypes = [ctypes.c_int32, ctypes.c_int64, _u8p, ctypes.c_int32]
        L.orc_density_mode.restype = ctypes.c_double
        L.orc_phi_fixed.argtypes = [_f32p, _i32p]
        L.orc_phi_fixed.restype = ctypes.c_int
        L.orc_potential.argtypes = [ctypes.c_int32, _u8p, _i32p]
        L.orc_potential.restype = ctypes.c_int64
        L.orc_guided_q.argtypes = [ctypes.c_int32]
        L.orc_guided_q.restype = ctypes.c_uint64
        L.orc_s_q.argtypes = [ctypes.c_double]
        L.orc_s_q.restype = ctypes.c_int32
        L.orc_guided_k.argtypes = [ctypes.c_int32, _u8p, ctypes.c_int, _i32p, ctypes.c_int32]
        L.orc_guided_k.restype = ctypes.c_int32
        L.orc_evolve_guided.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_uint32, ctypes.c_uint64, _i32p, _u8p, _i32p, _i32p, _f32p]
        L.orc_evolve_guided.restype = ctypes.c_int
        L.orc_evolve_guided_table.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_uint32, ctypes.c_uint64, _f64p, _u8p, _i32p, _i32p, _f32p]
        L.orc_evolve_guided_table.restype = ctypes.c_int
        L.orc_weights_guided.argtypes = [ctypes.c_int64, _f32p, _u64p]
        L.orc_weights_guided.restype = ctypes.c_int
        L.orc_psi_term_guided.argtypes = [ctypes.c_int64, _f32p]
        L.orc_psi_term_guided.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def philox(ctr, seed):
    """Philox4x32-10 of a 4-word counter under a 64-bit key; returns 4 uint32."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c, _u32p), ctypes.c_uint64(int(seed)), _p(out, _u32p))
    return out


def neg_ln_u(w):
    """The specified FP32 -ln((2w+1)/2^33)."""
    return np.float32(lib().orc_neg_ln_u(ctypes.c_uint32(int(w))))


class Population:
    """One population of clones, one byte per site (clone-major).  modified: the
    MODIFIED dynamics and weights (reading R13); iid: [iid] selection (R14);
    phi: 512 potential values, GUIDED dynamics and weights (R15); U_table: a
    potential over all 2^L configurations instead (GUIDED, test pins only)."""

    def __init__(self, L, N, n_clones, seed, modified=False, iid=False, phi=None, U_table=None):
        self.L, self.N, self.n_clones, self.seed = int(L), int(N), int(n_clones), int(seed)
        self.modified, self.iid = bool(modified), bool(iid)
        self.guided = phi is not None or U_table is not None
        self.phi_q = None if phi is None else phi_fixed(phi)
        self.U_table = None if U_table is None else np.ascontiguousarray(np.asarray(U_table, dtype=np.float64))
        self.s = None
        self.A = np.zeros(int(n_clones), dtype=np.float32)
        self.sites = np.zeros((self.n_clones, self.L), dtype=np.uint8)
        self.K = np.zeros(self.n_clones, dtype=np.int32)
        self.dK = np.zeros(self.n_clones, dtype=np.int32)
        self.anc = np.arange(self.n_clones, dtype=np.int32)
        self.beta = 0
        self.psi_acc = 0.0
        self.t_obs = 0.0
        self.events = 0
        rc = lib().orc_init(self.L, self.N, self.n_clones, self.seed,
                            _p(self.sites, _u8p), _p(self.K, _i32p))
        if rc != 0:
            raise ValueError("orc_init rejected its arguments (rc=%d)" % rc)

    def evolve(self, dt, s=None):
        """Dynamical stage of the next interval (MODIFIED mode needs s)."""
        self.beta += 1
        if self.guided:
            self.s = float(s)
            if self.U_table is not None:
                rc = lib().orc_evolve_guided_table(self.L, self.n_clones, float(dt), self.s, self.beta,
                                                   self.seed, _p(self.U_table, _f64p), _p(self.sites, _u8p),
                                                   _p(self.K, _i32p), _p(self.dK, _i32p), _p(self.A, _f32p))
            else:
                rc = lib().orc_evolve_guided(self.L, self.n_clones, float(dt), self.s, self.beta, self.seed,
                                             _p(self.phi_q, _i32p), _p(self.sites, _u8p), _p(self.K, _i32p),
                                             _p(self.dK, _i32p), _p(self.A, _f32p))
        elif self.modified:
            self.s = float(s)
            rc = lib().orc_evolve_modified(self.L, self.n_clones, float(dt), self.s, self.beta, self.seed,
                                           _p(self.sites, _u8p), _p(self.K, _i32p), _p(self.dK, _i32p),
                                           _p(self.A, _f32p))
        else:
            rc = lib().orc_evolve(self.L, self.n_clones, float(dt), self.beta, self.seed,
                                  _p(self.sites, _u8p), _p(self.K, _i32p), _p(self.dK, _i32p))
        if rc != 0:
            raise ValueError("orc_evolve rc=%d" % rc)
        self.t_obs += float(dt)
        self.events += int(self.dK.sum())

    def weights(self, s):
        w = np.zeros(self.n_clones, dtype=np.uint64)
        if self.guided:
            rc = lib().orc_weights_guided(self.n_clones, _p(self.A, _f32p), _p(w, _u64p))
        elif self.modified:
            rc = lib().orc_weights_modified(float(s), self.n_clones, _p(self.A, _f32p), _p(w, _u64p))
        else:
            rc = lib().orc_weights(float(s), self.n_clones, _p(self.dK, _i32p), _p(w, _u64p))
        return w, rc

    def psi_term(self, s):
        if self.guided:
            return lib().orc_psi_term_guided(self.n_clones, _p(self.A, _f32p))
        if self.modified:
            return lib().orc_psi_term_modified(float(s), self.n_clones, _p(self.A, _f32p))
        return lib().orc_psi_term(float(s), self.n_clones, _p(self.dK, _i32p))

    def resample(self, s):
        """Cloning stage of the interval just evolved; returns (term, rc)."""
        term = self.psi_term(s)
        self.psi_acc += term
        w, rc = self.weights(s)
        anc = np.zeros(self.n_clones, dtype=np.int32)
        sel = lib().orc_ancestors_iid if self.iid else lib().orc_ancestors
        rc2 = sel(self.n_clones, _p(w, _u64p), self.beta, self.seed, _p(anc, _i32p))
        if rc2 != 0:
            raise ValueError("orc_ancestors rc=%d" % rc2)
        new_sites = np.zeros_like(self.sites)
        new_K = np.zeros_like(self.K)
        lib().orc_gather(self.L, self.n_clones, _p(anc, _i32p), _p(self.sites, _u8p),
                         _p(self.K, _i32p), _p(new_sites, _u8p), _p(new_K, _i32p))
        self.sites, self.K, self.anc = new_sites, new_K, anc
        return term, rc

    def estimates(self):
        psi = self.psi_acc / self.t_obs
        k_hat = float(self.K.astype(np.float64).sum()) / (self.n_clones * self.L * self.t_obs)
        return psi, k_hat


def weights(s, dK):
    dK = np.ascontiguousarray(np.asarray(dK, dtype=np.int32))
    w = np.zeros(dK.size, dtype=np.uint64)
    rc = lib().orc_weights(float(s), dK.size, _p(dK, _i32p), _p(w, _u64p))
    return w, rc


def weight_scale(n_clones):
    return int(lib().orc_weight_scale(int(n_clones)))


def psi_term(s, dK):
    dK = np.ascontiguousarray(np.asarray(dK, dtype=np.int32))
    return float(lib().orc_psi_term(float(s), dK.size, _p(dK, _i32p)))


def resample_word(beta, seed):
    return int(lib().orc_resample_word(int(beta), int(seed)))


def ancestors(w, beta, seed):
    w = np.ascontiguousarray(np.asarray(w, dtype=np.uint64))
    anc = np.zeros(w.size, dtype=np.int32)
    rc = lib().orc_ancestors(w.size, _p(w, _u64p), int(beta), int(seed), _p(anc, _i32p))
    if rc != 0:
        raise ValueError("orc_ancestors rc=%d" % rc)
    return anc


def evolve_sites(L, sites, dt, beta, seed, K=None):
    """Evolve given configurations (clone j is stream slot j); returns (sites, K, dK)."""
    sites = np.ascontiguousarray(np.array(sites, dtype=np.uint8))
    n = sites.shape[0]
    K = np.zeros(n, dtype=np.int32) if K is None else np.ascontiguousarray(np.array(K, dtype=np.int32))
    dK = np.zeros(n, dtype=np.int32)
    rc = lib().orc_evolve(int(L), n, float(dt), int(beta), int(seed), _p(sites, _u8p), _p(K, _i32p), _p(dK, _i32p))
    if rc != 0:
        raise ValueError("orc_evolve rc=%d" % rc)
    return sites, K, dK


def init_sites(L, N, n_clones, seed):
    sites = np.zeros((int(n_clones), int(L)), dtype=np.uint8)
    K = np.zeros(int(n_clones), dtype=np.int32)
    rc = lib().orc_init(int(L), int(N), int(n_clones), int(seed), _p(sites, _u8p), _p(K, _i32p))
    if rc != 0:
        raise ValueError("orc_init rc=%d" % rc)
    return sites


def density_mode(sites, n):
    """Population mean of |delta rho_n|^2 (eq. fourdens), FP32 per clone, FP64 mean."""
    sites = np.ascontiguousarray(np.asarray(sites, dtype=np.uint8))
    return float(lib().orc_density_mode(sites.shape[1], sites.shape[0], _p(sites, _u8p), int(n)))


def weight_exp(x, F):
    """floor(2^F exp(x)) for x <= 0 by the specified FP32 exponential (R13)."""
    return int(lib().orc_weight_exp(ctypes.c_float(float(x)), int(F)))


def ancestors_iid(w, beta, seed):
    w = np.ascontiguousarray(np.asarray(w, dtype=np.uint64))
    anc = np.zeros(w.size, dtype=np.int32)
    rc = lib().orc_ancestors_iid(w.size, _p(w, _u64p), int(beta), int(seed), _p(anc, _i32p))
    if rc != 0:
        raise ValueError("orc_ancestors_iid rc=%d" % rc)
    return anc


def evolve_sites_modified(L, sites, dt, s, beta, seed):
    """MODIFIED dynamics of given configurations; returns (sites, dK, A)."""
    sites = np.ascontiguousarray(np.array(sites, dtype=np.uint8))
    n = sites.shape[0]
    K = np.zeros(n, dtype=np.int32)
    dK = np.zeros(n, dtype=np.int32)
    A = np.zeros(n, dtype=np.float32)
    rc = lib().orc_evolve_modified(int(L), n, float(dt), float(s), int(beta), int(seed), _p(sites, _u8p),
                                   _p(K, _i32p), _p(dK, _i32p), _p(A, _f32p))
    if rc != 0:
        raise ValueError("orc_evolve_modified rc=%d" % rc)
    return sites, dK, A


def psi_term_modified(s, A):
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float32))
    return float(lib().orc_psi_term_modified(float(s), A.size, _p(A, _f32p)))


def run(L, N, n_clones, seed, s, dt, M, want_state=False, modified=False, iid=False):
    """Full run; returns dict(psi, k_hat, events[, sites, K])."""
    psi = ctypes.c_double(0.0)
    kh = ctypes.c_double(0.0)
    ev = ctypes.c_uint64(0)
    sites = K = None
    sp = kp = None
    if want_state:
        sites = np.zeros((int(n_clones), int(L)), dtype=np.uint8)
        K = np.zeros(int(n_clones), dtype=np.int32)
        sp, kp = _p(sites, _u8p), _p(K, _i32p)
    rc = lib().orc_run_ex(int(L), int(N), int(n_clones), int(seed), float(s), float(dt), int(M),
                          int(bool(modified)), int(bool(iid)),
                          ctypes.byref(psi), ctypes.byref(kh), ctypes.byref(ev), sp, kp)
    out = dict(psi=psi.value, k_hat=kh.value, events=int(ev.value), rc=rc)
    if want_state:
        out.update(sites=sites, K=K)
    return out


def phi_fixed(phi):
    """The 512 potential values as the fixed point of reading R15 (int32, phi 2^16)."""
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float32).reshape(512))
    out = np.zeros(512, dtype=np.int32)
    if lib().orc_phi_fixed(_p(phi, _f32p), _p(out, _i32p)) != 0:
        raise ValueError("potential values must satisfy |phi| <= 64")
    return out


def potential(sites, phi):
    """U(C) of each configuration (rows of sites) in units of 2^-16 (exact integers)."""
    sites = np.ascontiguousarray(np.atleast_2d(np.asarray(sites, dtype=np.uint8)))
    q = phi_fixed(phi)
    return np.array([lib().orc_potential(sites.shape[1], _p(np.ascontiguousarray(r), _u8p), _p(q, _i32p))
                     for r in sites], dtype=np.int64)


def guided_q(k):
    """Q(k) = floor(TA[a] TB[c] / 2^44), the rate 2^40 exp(k 2^-17) of reading R15."""
    return int(lib().orc_guided_q(int(k)))


def s_q(s):
    """s in units of 2^-17 (nearest integer), as the guided rates use it (R15)."""
    return int(lib().orc_s_q(float(s)))


def guided_k(sites_row, b, phi, s):
    """Rate exponent k_b (units of 2^-17) of reading R15 for one configuration and bond b."""
    row = np.ascontiguousarray(np.asarray(sites_row, dtype=np.uint8))
    q = phi_fixed(phi)
    return int(lib().orc_guided_k(row.size, _p(row, _u8p), int(b), _p(q, _i32p), s_q(s)))


def evolve_sites_guided(L, sites, dt, s, beta, seed, phi=None, U_table=None, K=None):
    """GUIDED dynamics of given configurations; returns (sites, K, dK, X)."""
    sites = np.ascontiguousarray(np.array(sites, dtype=np.uint8))
    n = sites.shape[0]
    K = np.zeros(n, dtype=np.int32) if K is None else np.ascontiguousarray(np.array(K, dtype=np.int32))
    dK = np.zeros(n, dtype=np.int32)
    X = np.zeros(n, dtype=np.float32)
    if U_table is not None:
        U = np.ascontiguousarray(np.asarray(U_table, dtype=np.float64))
        rc = lib().orc_evolve_guided_table(int(L), n, float(dt), float(s), int(beta), int(seed), _p(U, _f64p),
                                           _p(sites, _u8p), _p(K, _i32p), _p(dK, _i32p), _p(X, _f32p))
    else:
        q = phi_fixed(phi)
        rc = lib().orc_evolve_guided(int(L), n, float(dt), float(s), int(beta), int(seed), _p(q, _i32p),
                                     _p(sites, _u8p), _p(K, _i32p), _p(dK, _i32p), _p(X, _f32p))
    if rc != 0:
        raise ValueError("orc_evolve_guided rc=%d" % rc)
    return sites, K, dK, X


def psi_term_guided(X):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
    return float(lib().orc_psi_term_guided(X.size, _p(X, _f32p)))


def sites_to_words(sites, W=None):
    """Pack one-byte sites (n_clones, L) into uint64 words (n_clones, W): site i is
    bit (i mod 64) of word (i div 64)."""
    sites = np.asarray(sites, dtype=np.uint8)
    n, L = sites.shape
    if W is None:
        W = (L + 63) // 64
    words = np.zeros((n, W), dtype=np.uint64)
    for i in range(L):
        words[:, i // 64] |= sites[:, i].astype(np.uint64) << np.uint64(i % 64)
    return words
