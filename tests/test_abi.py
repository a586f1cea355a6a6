"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/pop.h declares, and argument validation happens
before any device work."""
import ctypes
import os
import re

import pytest

import paper_1711_05095_gb300 as pg
from paper_1711_05095_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pg.library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pop.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pop_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(pg.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def P(**kw):
    d = dict(L=20, N=10, n_clones=1000, seed=1)
    d.update(kw)
    return d


def test_workspace_bytes(lib):
    a = pg.workspace_bytes([P()])
    b = pg.workspace_bytes([P(n_clones=5000)])
    assert a > 0 and a % 256 == 0 and b > a
    assert pg.lattice_words([P(L=64)]) == 1
    assert pg.lattice_words([P(L=65), P(L=20)]) == 2
    assert pg.lattice_words([P(L=4096, N=5)]) == 64
    assert pg.workspace_bytes([P(weight_mode=1, selection=1)]) > 0
    for bad in (P(L=2), P(L=4097), P(N=-1), P(N=21), P(n_clones=0), P(weight_mode=7), P(selection=9)):
        assert pg.workspace_bytes([bad]) == 0, bad
    # GUIDED: 18 <= L <= 128, and the whole batch GUIDED
    G = pg.POP_GUIDED
    assert pg.workspace_bytes([P(L=18, N=9, weight_mode=G), P(L=128, N=64, weight_mode=G)]) > 0
    assert pg.workspace_bytes([P(L=17, N=8, weight_mode=G)]) == 0
    assert pg.workspace_bytes([P(L=129, N=64, weight_mode=G)]) == 0
    assert pg.workspace_bytes([P(weight_mode=G), P()]) == 0
    assert pg.workspace_bytes([P(), P(weight_mode=G)]) == 0
    # a GUIDED population adds its bond tables: dU (int32) and the rate Q (uint64) of
    # each of the 2^17 segments of an active bond; and every slot (1024 per tile) its
    # carried rate sums, 8 W per slot and interval parity
    per_pop = (1 << 17) * (4 + 8)
    carry = 2 * 1024 * 8 * 8
    assert pg.workspace_bytes([P(weight_mode=G)]) == pg.workspace_bytes([P()]) + per_pop + carry
    assert (pg.workspace_bytes([P(weight_mode=G), P(weight_mode=G, seed=2)])
            == pg.workspace_bytes([P(), P(seed=2)]) + 2 * per_pop + 2 * carry)


def test_init_rejects_bad_arguments_without_device(lib):
    h = ctypes.c_void_p()
    good = pg.make_params([P()])
    n = lib.pop_workspace_bytes(good, 1)
    # too small a workspace, misaligned workspace, null workspace, invalid params
    assert lib.pop_init(ctypes.byref(h), good, 1, ctypes.c_void_p(1 << 20), n - 256, None) == pg.POP_ERR_ARG
    assert lib.pop_init(ctypes.byref(h), good, 1, ctypes.c_void_p((1 << 20) + 8), n, None) == pg.POP_ERR_ARG
    assert lib.pop_init(ctypes.byref(h), good, 1, None, n, None) == pg.POP_ERR_ARG
    bad = pg.make_params([P(N=99)])
    assert lib.pop_init(ctypes.byref(h), bad, 1, ctypes.c_void_p(1 << 20), n, None) == pg.POP_ERR_ARG
    assert h.value is None
    assert lib.pop_evolve(None, 0.1, None) == pg.POP_ERR_ARG
    assert lib.pop_resample(None) == pg.POP_ERR_ARG
    assert lib.pop_set_potential(None, 0, None) == pg.POP_ERR_ARG
    lib.pop_free(None)


def test_every_handle_call_rejects_a_null_handle(lib):
    # host-side checks made before any device work, so they run without a GPU
    E = pg.POP_ERR_ARG
    assert lib.pop_set_state(None, 0, None, None) == E
    assert lib.pop_run(None, 0.1, None, 1) == E
    assert lib.pop_estimate_psi(None, None, None, None) == E
    assert lib.pop_copy_state(None, 0, None, None, None, None) == E
    assert lib.pop_events(None, None) == E
    assert lib.pop_launch_count(None, None) == E
    assert lib.pop_kernel_times(None, 0.1, None, 1, 0, None, None, None) == E
    assert lib.pop_autotune(None, 0.1, None, 1, None) == E
    assert lib.pop_lineage(None, None, None) == E
    assert lib.pop_density_mode(None, 1, None) == E
    assert lib.pop_get_tuning(None, None) == E
    assert lib.pop_set_tuning(None, None) == E
    assert lib.pop_run_chains(None, None) == -1
    assert lib.pop_slots(None) == -1
    assert lib.pop_first_slot(None, 0) == -1


def test_strerror(lib):
    for code in (0, -1, -2, -3, -5):
        assert lib.pop_strerror(code)
    assert pg.strerror(-3).startswith("interval activity")
