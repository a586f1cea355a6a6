"""GB300 (sm_103a) population-dynamics estimator of psi(s) for the SSEP activity.

Thin Python binding of the C ABI in ``include/pop.h`` (arXiv:1711.05095, Sec. 2.3
cloning algorithm; Sec. 4 BKL dynamics and [eq] selection).  This module only
marshals arguments: every step of the path runs in the CUDA library
``_build/libpopgb300.so``.  PyTorch supplies device memory (the workspace) and the
CUDA stream.  There is no CPU fallback: if the library is not built, or no CUDA
device is present, the calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpopgb300.so")

POP_OK = 0
POP_ERR_ARG = -1
POP_ERR_CUDA = -2
POP_ERR_RANGE = -3
POP_ERR_STATE = -5
POP_PLAIN = 0
POP_MODIFIED = 1
POP_GUIDED = 2
POP_EQ = 0
POP_IID = 1
POP_KCAP = 4096
POP_MAX_L = 4096

# every symbol include/pop.h declares
EXPORTS = ("pop_workspace_bytes", "pop_init", "pop_set_state", "pop_evolve", "pop_resample",
           "pop_run", "pop_estimate_psi", "pop_copy_state", "pop_events", "pop_lattice_words",
           "pop_select_noalloc", "pop_density_mode", "pop_autotune", "pop_kernel_times",
           "pop_set_potential", "pop_lineage", "pop_slots", "pop_first_slot",
           "pop_mlp_workspace_bytes", "pop_mlp_init", "pop_mlp_grad", "pop_mlp_step",
           "pop_mlp_params", "pop_mlp_potential", "pop_mlp_free",
           "pop_launch_count", "pop_run_chains", "pop_get_tuning", "pop_set_tuning",
           "pop_strerror", "pop_free")
KERNEL_KINDS = ("evolve", "weights", "gather", "gather_evolve", "other")
POP_NOALLOC_MAX_CLONES = 1 << 20


class PopParams(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("N", ctypes.c_int32), ("n_clones", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("weight_mode", ctypes.c_int32),
                ("selection", ctypes.c_int32)]


class PopTuning(ctypes.Structure):
    _fields_ = [("evolve_grid", ctypes.c_int32), ("fuse_threads", ctypes.c_int32),
                ("fuse_clones", ctypes.c_int32), ("chains", ctypes.c_int32),
                ("gather_threads", ctypes.c_int32), ("hist_mode", ctypes.c_int32),
                ("default_us_per_interval", ctypes.c_float), ("tuned_us_per_interval", ctypes.c_float)]


TUNING_KEYS = ("evolve_grid", "fuse_threads", "fuse_clones", "chains", "gather_threads", "hist_mode")


class PopError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, strerror(status), status))


_lib = None
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def library():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library %s is missing: build it with "
                           "paper_1711_05095_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    pp = ctypes.POINTER(PopParams)
    L.pop_workspace_bytes.argtypes = [pp, ctypes.c_int32]
    L.pop_workspace_bytes.restype = ctypes.c_size_t
    L.pop_lattice_words.argtypes = [pp, ctypes.c_int32]
    L.pop_lattice_words.restype = ctypes.c_int32
    L.pop_init.argtypes = [ctypes.POINTER(ctypes.c_void_p), pp, ctypes.c_int32, ctypes.c_void_p,
                           ctypes.c_size_t, ctypes.c_void_p]
    L.pop_init.restype = ctypes.c_int
    L.pop_set_state.argtypes = [ctypes.c_void_p, ctypes.c_int32, _u64p, _i32p]
    L.pop_set_state.restype = ctypes.c_int
    L.pop_evolve.argtypes = [ctypes.c_void_p, ctypes.c_double, _f64p]
    L.pop_evolve.restype = ctypes.c_int
    L.pop_resample.argtypes = [ctypes.c_void_p]
    L.pop_resample.restype = ctypes.c_int
    L.pop_run.argtypes = [ctypes.c_void_p, ctypes.c_double, _f64p, ctypes.c_int64]
    L.pop_run.restype = ctypes.c_int
    L.pop_estimate_psi.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
    L.pop_estimate_psi.restype = ctypes.c_int
    L.pop_copy_state.argtypes = [ctypes.c_void_p, ctypes.c_int32, _u64p, _i32p, _i32p, _i32p]
    L.pop_copy_state.restype = ctypes.c_int
    L.pop_autotune.argtypes = [ctypes.c_void_p, ctypes.c_double, _f64p, ctypes.c_int32, _i32p]
    L.pop_autotune.restype = ctypes.c_int
    L.pop_density_mode.argtypes = [ctypes.c_void_p, ctypes.c_int32, _f64p]
    L.pop_density_mode.restype = ctypes.c_int
    L.pop_set_potential.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
    L.pop_set_potential.restype = ctypes.c_int
    L.pop_lineage.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.pop_lineage.restype = ctypes.c_int
    L.pop_slots.argtypes = [ctypes.c_void_p]
    L.pop_slots.restype = ctypes.c_int64
    L.pop_first_slot.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    L.pop_first_slot.restype = ctypes.c_int64
    _f32p = ctypes.POINTER(ctypes.c_float)
    L.pop_mlp_workspace_bytes.argtypes = []
    L.pop_mlp_workspace_bytes.restype = ctypes.c_size_t
    L.pop_mlp_init.argtypes = [ctypes.POINTER(ctypes.c_void_p), _f32p, ctypes.c_void_p, ctypes.c_size_t,
                               ctypes.c_void_p]
    L.pop_mlp_init.restype = ctypes.c_int
    L.pop_mlp_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                               ctypes.c_int64, _f64p, _f32p]
    L.pop_mlp_grad.restype = ctypes.c_int
    L.pop_mlp_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                               ctypes.c_int64, ctypes.c_float, _f64p]
    L.pop_mlp_step.restype = ctypes.c_int
    L.pop_mlp_params.argtypes = [ctypes.c_void_p, _f32p]
    L.pop_mlp_params.restype = ctypes.c_int
    L.pop_mlp_potential.argtypes = [ctypes.c_void_p, _f32p]
    L.pop_mlp_potential.restype = ctypes.c_int
    L.pop_mlp_free.argtypes = [ctypes.c_void_p]
    L.pop_mlp_free.restype = None
    L.pop_events.argtypes = [ctypes.c_void_p, _u64p]
    L.pop_events.restype = ctypes.c_int
    L.pop_kernel_times.argtypes = [ctypes.c_void_p, ctypes.c_double, _f64p, ctypes.c_int64, ctypes.c_int32, _f64p,
                                   ctypes.POINTER(ctypes.c_int64), _u64p]
    L.pop_kernel_times.restype = ctypes.c_int
    L.pop_launch_count.argtypes = [ctypes.c_void_p, _u64p]
    L.pop_launch_count.restype = ctypes.c_int
    L.pop_run_chains.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    L.pop_run_chains.restype = ctypes.c_int32
    L.pop_get_tuning.argtypes = [ctypes.c_void_p, ctypes.POINTER(PopTuning)]
    L.pop_get_tuning.restype = ctypes.c_int
    L.pop_set_tuning.argtypes = [ctypes.c_void_p, ctypes.POINTER(PopTuning)]
    L.pop_set_tuning.restype = ctypes.c_int
    L.pop_select_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_void_p, _f64p, ctypes.c_void_p]
    L.pop_select_noalloc.restype = ctypes.c_int
    L.pop_strerror.argtypes = [ctypes.c_int]
    L.pop_strerror.restype = ctypes.c_char_p
    L.pop_free.argtypes = [ctypes.c_void_p]
    L.pop_free.restype = None
    _lib = L
    return L


def strerror(status):
    try:
        return library().pop_strerror(int(status)).decode()
    except RuntimeError:
        return "status %d" % status


def _check(rc, where):
    if rc != POP_OK:
        raise PopError(rc, where)


def make_params(pops):
    """pops: sequence of dicts with L, N, n_clones, seed (weight_mode, selection optional)."""
    arr = (PopParams * len(pops))()
    for i, q in enumerate(pops):
        arr[i] = PopParams(int(q["L"]), int(q["N"]), int(q["n_clones"]), int(q["seed"]),
                           int(q.get("weight_mode", POP_PLAIN)), int(q.get("selection", POP_EQ)))
    return arr


def workspace_bytes(pops):
    arr = make_params(pops)
    return int(library().pop_workspace_bytes(arr, len(pops)))


def lattice_words(pops):
    arr = make_params(pops)
    return int(library().pop_lattice_words(arr, len(pops)))


class PopulationBatch:
    """A batch of independent clone populations on one GPU (C ABI ``pop_*``).

    ``pops`` is a list of dicts (L, N, n_clones, seed).  The workspace is a torch
    uint8 tensor on ``device``; work is queued on ``stream`` (default: the current
    torch stream of that device).
    """

    def __init__(self, pops, device="cuda", stream=None, workspace=None):
        import torch
        self.pops = [dict(q) for q in pops]
        self.n_pops = len(pops)
        self._lib = library()
        self._params = make_params(self.pops)
        nbytes = int(self._lib.pop_workspace_bytes(self._params, self.n_pops))
        if nbytes == 0:
            raise PopError(POP_ERR_ARG, "pop_workspace_bytes")
        self.W = int(self._lib.pop_lattice_words(self._params, self.n_pops))
        self.device = torch.device(device)
        if workspace is not None:
            if workspace.numel() * workspace.element_size() < nbytes or workspace.device.type != "cuda":
                raise PopError(POP_ERR_ARG, "workspace")
            self.workspace = workspace
        else:
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._h = ctypes.c_void_p()
        rc = self._lib.pop_init(ctypes.byref(self._h), self._params, self.n_pops,
                                ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                ctypes.c_void_p(self.stream.cuda_stream))
        _check(rc, "pop_init")

    def _s(self, s):
        s = np.ascontiguousarray(np.broadcast_to(np.asarray(s, dtype=np.float64), (self.n_pops,)))
        return s, s.ctypes.data_as(_f64p)

    def set_state(self, p, lattice, K=None):
        lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.uint64).reshape(-1))
        kp = None
        if K is not None:
            K = np.ascontiguousarray(np.asarray(K, dtype=np.int32))
            kp = K.ctypes.data_as(_i32p)
        _check(self._lib.pop_set_state(self._h, int(p), lat.ctypes.data_as(_u64p), kp), "pop_set_state")

    def evolve(self, dt, s):
        s, sp = self._s(s)
        _check(self._lib.pop_evolve(self._h, float(dt), sp), "pop_evolve")

    def resample(self):
        _check(self._lib.pop_resample(self._h), "pop_resample")

    def run(self, dt, s, n_intervals):
        s, sp = self._s(s)
        _check(self._lib.pop_run(self._h, float(dt), sp, int(n_intervals)), "pop_run")

    def estimate_psi(self):
        psi = np.zeros(self.n_pops)
        kh = np.zeros(self.n_pops)
        t = ctypes.c_double(0.0)
        _check(self._lib.pop_estimate_psi(self._h, psi.ctypes.data_as(_f64p), kh.ctypes.data_as(_f64p),
                                          ctypes.byref(t)), "pop_estimate_psi")
        return psi, kh, t.value

    def copy_state(self, p):
        n = int(self.pops[p]["n_clones"])
        lat = np.zeros((n, self.W), dtype=np.uint64)
        K = np.zeros(n, dtype=np.int32)
        anc = np.zeros(n, dtype=np.int32)
        dK = np.zeros(n, dtype=np.int32)
        _check(self._lib.pop_copy_state(self._h, int(p), lat.ctypes.data_as(_u64p), K.ctypes.data_as(_i32p),
                                        anc.ctypes.data_as(_i32p), dK.ctypes.data_as(_i32p)),
               "pop_copy_state")
        return dict(lattice=lat, K=K, anc=anc, dK=dK)

    def autotune(self, dt, s, trials=5):
        """Choose the launch configuration by timing on this batch (before the first
        interval); returns it as get_tuning() does."""
        s, sp = self._s(s)
        g = ctypes.c_int32(0)
        _check(self._lib.pop_autotune(self._h, float(dt), sp, int(trials), ctypes.byref(g)), "pop_autotune")
        return self.get_tuning()

    def get_tuning(self):
        """The launch configuration (pop_tuning) as a dict."""
        t = PopTuning()
        _check(self._lib.pop_get_tuning(self._h, ctypes.byref(t)), "pop_get_tuning")
        return {name: getattr(t, name) for name, _ in PopTuning._fields_}

    def set_tuning(self, **cfg):
        """Change entries of the launch configuration (results do not depend on it)."""
        cur = self.get_tuning()
        cur.update(cfg)
        t = PopTuning(*(int(cur[k]) for k in TUNING_KEYS), 0.0, 0.0)
        _check(self._lib.pop_set_tuning(self._h, ctypes.byref(t)), "pop_set_tuning")

    def run_chains(self):
        """First tile of each chain of run() and the tile count (K + 1 entries; [] when
        the batch does not fuse)."""
        t = np.zeros(9, dtype=np.int32)
        k = int(self._lib.pop_run_chains(self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        if k < 0:
            raise PopError(POP_ERR_ARG, "pop_run_chains")
        return [int(x) for x in t[:k + 1]] if k > 0 else []

    @property
    def slots(self):
        """Slots of the batch (populations padded to 1024-slot tiles)."""
        return int(self._lib.pop_slots(self._h))

    def first_slot(self, p):
        return int(self._lib.pop_first_slot(self._h, int(p)))

    def lineage(self, d_in, d_out):
        """d_out[off + j] = d_in[off + anc_j] across the last cloning stage (torch int32
        tensors of ``slots`` entries on the batch's device)."""
        for t in (d_in, d_out):
            if t.dtype != __import__("torch").int32 or t.numel() < self.slots or not t.is_cuda:
                raise PopError(POP_ERR_ARG, "lineage buffers")
        _check(self._lib.pop_lineage(self._h, ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr())),
               "pop_lineage")

    def set_potential(self, p, phi):
        """GUIDED population p: the 512-entry window potential (|phi| <= 64)."""
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float32).reshape(512))
        _check(self._lib.pop_set_potential(self._h, int(p), phi.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "pop_set_potential")

    def kernel_times(self, dt, s, n, per_step=False):
        """Advance n intervals as run() does (or as evolve() + resample() with
        per_step), timing every launch with CUDA events.
        Returns {kind: (mean microseconds, launches, hops)}."""
        s, sp = self._s(s)
        k = len(KERNEL_KINDS)
        us = np.zeros(k)
        cnt = np.zeros(k, dtype=np.int64)
        hops = np.zeros(k, dtype=np.uint64)
        _check(self._lib.pop_kernel_times(self._h, float(dt), sp, int(n), int(bool(per_step)), us.ctypes.data_as(_f64p),
                                          cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          hops.ctypes.data_as(_u64p)), "pop_kernel_times")
        return {name: (float(us[i]), int(cnt[i]), int(hops[i])) for i, name in enumerate(KERNEL_KINDS)}

    def launch_count(self):
        """Kernels launched by this batch so far, {kind: count}."""
        cnt = np.zeros(len(KERNEL_KINDS), dtype=np.uint64)
        _check(self._lib.pop_launch_count(self._h, cnt.ctypes.data_as(_u64p)), "pop_launch_count")
        return {name: int(cnt[i]) for i, name in enumerate(KERNEL_KINDS)}

    def density_mode(self, n=1):
        """Population mean of |delta rho_n|^2 (eq. fourdens) per population."""
        out = np.zeros(self.n_pops)
        _check(self._lib.pop_density_mode(self._h, int(n), out.ctypes.data_as(_f64p)), "pop_density_mode")
        return out

    def events(self):
        ev = np.zeros(self.n_pops, dtype=np.uint64)
        _check(self._lib.pop_events(self._h, ev.ctypes.data_as(_u64p)), "pop_events")
        return ev

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pop_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def select_noalloc(d_dK, s, seed, interval, d_anc, stream=None):
    """pop_select_noalloc on torch device tensors (int32 activities in, int32
    ancestors out, same length).  Returns the psi term of the interval.  For
    callers that cannot allocate device memory; nothing is allocated here."""
    import torch
    n = int(d_dK.numel())
    if (d_anc.numel() != n or d_dK.dtype != torch.int32 or d_anc.dtype != torch.int32
            or not d_dK.is_cuda or d_anc.device != d_dK.device):
        raise PopError(POP_ERR_ARG, "pop_select_noalloc")
    # the library uses the scratch array of the current device: make it the tensors' one
    with torch.cuda.device(d_dK.device):
        st = stream if stream is not None else torch.cuda.current_stream(d_dK.device)
        term = ctypes.c_double(0.0)
        rc = library().pop_select_noalloc(ctypes.c_void_p(d_dK.data_ptr()), n, float(s), int(seed),
                                          int(interval), ctypes.c_void_p(d_anc.data_ptr()),
                                          ctypes.byref(term), ctypes.c_void_p(st.cuda_stream))
    _check(rc, "pop_select_noalloc")
    return term.value
