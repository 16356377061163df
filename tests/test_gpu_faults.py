"""Recovery from failed device allocations, injected on the host.

`nb_ctx_inject_alloc_failures(ctx, n)` makes the next n allocations of the
context fail as an out-of-memory would.  No GPU fault is involved: the
library's allocation wrapper reports NB_ERR_OOM before touching the device.
Every call that allocates must fail cleanly, leave the previous state
usable, and release nothing twice; after the faults, results still match
the oracle and the context's memory accounting returns to its start.
"""
import numpy as np
import pytest

import oracle
from oracle import pme as opme
from paper_1506_00716_gb300 import nb
from paper_1506_00716_gb300 import waterbox as wb
from _support import rel_rms

pytestmark = pytest.mark.gpu

OOM = 3


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_00716_gb300 import build as nbbuild

    nbbuild.build()
    c = nb.nb_ctx_create(0, None, 0)
    yield c
    nb.nb_ctx_destroy(c)


def _fails(fn, *args):
    with pytest.raises(nb.NbError) as ei:
        fn(*args)
    assert ei.value.status == OOM, ei.value


def _forces(h, s, flags=0):
    f = np.zeros((s.n, 3), dtype=np.float32)
    nb.nb_forces(h, None, f, None, None, flags)
    return f


def test_short_range_path_recovers(ctx):
    s = wb.small_box(seed=1)
    p = wb.params_rf()
    ref = oracle.forces(s, p)
    used0, _ = nb.nb_ctx_memory(ctx)
    tuning = nb.nb_ctx_get_tuning(ctx)

    nb.nb_ctx_inject_alloc_failures(ctx, 1)
    _fails(nb.nb_sys_create, ctx, p, s.n, s.box)
    assert nb.nb_ctx_memory(ctx)[0] == used0
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    # the list capacity is sized with the item split in force at the plan's
    # creation (about one item per (cluster, shift) run at 4096 entries)
    nb.nb_ctx_set_tuning(ctx, 4096, tuning["force_min_blocks"])
    try:
        # exclusions: a failed upload keeps the previous ones
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_ctx_inject_alloc_failures(ctx, 1)
        _fails(nb.nb_set_exclusions, h, s.excl_index, s.excl_atoms)
        # the plan (first grid put)
        nb.nb_ctx_inject_alloc_failures(ctx, 1)
        _fails(nb.nb_grid_put, h, np.ascontiguousarray(s.xq()), np.ascontiguousarray(s.type))
        nb.nb_grid_put(h, np.ascontiguousarray(s.xq()), np.ascontiguousarray(s.type))
        nb.nb_pairlist_build(h)
        assert rel_rms(_forces(h, s), ref) <= 1e-5

        # list growth: a finer item split (four entries per item) than the
        # buffers were sized for overflows the item buffer; the growth
        # allocation fails, the old list stays, and the next build grows it
        nb.nb_ctx_set_tuning(ctx, 4, tuning["force_min_blocks"])
        nb.nb_grid_put(h, np.ascontiguousarray(s.xq()), np.ascontiguousarray(s.type))
        nb.nb_ctx_inject_alloc_failures(ctx, 1)
        _fails(nb.nb_pairlist_build, h)
        with pytest.raises(nb.NbError) as ei:
            _forces(h, s)
        assert ei.value.status == 8  # NB_ERR_STATE: no list after the failed build
        nb.nb_pairlist_build(h)
        assert rel_rms(_forces(h, s), ref) <= 1e-5

        # the inner list of dynamic pruning: on failure the outer one serves
        nb.nb_ctx_inject_alloc_failures(ctx, 1)
        _fails(nb.nb_pairlist_prune, h, 1.05)
        assert rel_rms(_forces(h, s), ref) <= 1e-5
        nb.nb_pairlist_prune(h, 1.05)
        assert rel_rms(_forces(h, s), ref) <= 1e-5
    finally:
        nb.nb_ctx_inject_alloc_failures(ctx, 0)
        nb.nb_ctx_set_tuning(ctx, tuning["max_entries"], tuning["force_min_blocks"])
        nb.nb_sys_destroy(h)
    assert nb.nb_ctx_memory(ctx)[0] == used0


def test_long_range_init_failure_keeps_the_old_mesh(ctx):
    s = wb.small_box(seed=1)
    p = wb.params_ewald()
    used0, _ = nb.nb_ctx_memory(ctx)
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    try:
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_grid_put(h, np.ascontiguousarray(s.xq()), np.ascontiguousarray(s.type))
        nb.nb_pairlist_build(h)
        nb.nb_ctx_inject_alloc_failures(ctx, 1)
        _fails(nb.nb_pme_init, h, (24, 24, 24), 4)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pme_forces(h, None, None, None, None, 0)
        assert ei.value.status == 8  # no mesh yet
        nb.nb_pme_init(h, (24, 24, 24), 4)
        nb.nb_ctx_inject_alloc_failures(ctx, 1)
        _fails(nb.nb_pme_init, h, (32, 32, 32), 6)
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(3)
        nb.nb_pme_forces(h, None, f, e, None, nb.NB_F_ENERGY)
    finally:
        nb.nb_ctx_inject_alloc_failures(ctx, 0)
        nb.nb_sys_destroy(h)
    assert nb.nb_ctx_memory(ctx)[0] == used0
    # the 24^3 mesh of the first init is still the one in use
    rec = opme.pme(s, p, grid=(24, 24, 24), order=4)
    ex = opme.ewald_exclusions(s, p)
    assert rel_rms(f, rec["forces"] + ex["forces"]) <= 1e-5
    assert abs(e[0] - rec["energy"]) <= 1e-6 * abs(rec["energy"])


def test_injection_argument_validation(ctx):
    with pytest.raises(nb.NbError) as ei:
        nb.nb_ctx_inject_alloc_failures(ctx, -1)
    assert ei.value.status == 1
