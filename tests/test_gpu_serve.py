"""The continuous-batching server (nb_server_*).

A served request must give the same result alone and in a mix of other
requests that share its wave, match the oracle, respect the HBM budget, and
report timeouts without blocking.
"""
import numpy as np
import pytest

import oracle
from paper_1506_00716_gb300 import nb
from paper_1506_00716_gb300 import waterbox as wb
from _support import rel_rms

pytestmark = pytest.mark.gpu

FLAGS = nb.NB_F_ENERGY | nb.NB_F_VIRIAL


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_00716_gb300 import build as nbbuild

    nbbuild.build()
    torch.cuda.set_device(0)
    c = nb.nb_ctx_create(0, None, 0)
    yield c
    nb.nb_ctx_destroy(c)


def _submit(srv, s, flags=FLAGS):
    return nb.nb_server_submit(srv, s.n, s.box, s.xq(), s.type, s.excl_index, s.excl_atoms, flags)


def _wait(srv, s, t, timeout=-1):
    f = np.zeros((s.n, 3), dtype=np.float32)
    e = np.zeros(2)
    v = np.zeros(9)
    st = nb.nb_server_wait(srv, t, timeout, f, e, v)
    return f, e, v, st


@pytest.mark.parametrize("jcluster", [8, 4], ids=["8x8", "8x4"])
def test_same_result_alone_and_in_the_mix(ctx, jcluster):
    """Both cluster geometries (the server takes the context's tuning when it
    is created)."""
    p = wb.params_ewald()
    old = nb.nb_ctx_get_tuning(ctx)
    nb.nb_ctx_set_tuning(ctx, old["max_entries"], old["force_min_blocks"], old["search_mode"], old["energy_mode"],
                         jcluster)
    try:
        srv = nb.nb_server_create(ctx, p, 0, 64)
    finally:
        nb.nb_ctx_set_tuning(ctx, old["max_entries"], old["force_min_blocks"], old["search_mode"],
                             old["energy_mode"], old["jcluster"])
    try:
        target = wb.water_box(1500, None, seed=71)
        f0, e0, v0, st0 = _wait(srv, target, _submit(srv, target))
        assert st0["wave_size"] == 1
        # keep both streams busy, then queue a mix that contains the target
        big = [wb.water_box(60000, None, seed=72 + k) for k in range(2)]
        mix = [wb.water_box(m, None, seed=80 + k) for k, m in enumerate([900, 4000, 2500, 12000])]
        tb = [_submit(srv, b) for b in big]
        tm = [_submit(srv, m) for m in mix[:2]] + [_submit(srv, target)] + [_submit(srv, m) for m in mix[2:]]
        results = [_wait(srv, m, t) for m, t in zip(mix[:2] + [target] + mix[2:], tm)]
        for b, t in zip(big, tb):
            _wait(srv, b, t)
        f1, e1, v1, st1 = results[2]
        assert st1["wave_size"] >= 2, st1
        assert rel_rms(f1, f0) < 1e-6
        assert np.allclose(e1, e0, rtol=1e-10, atol=1e-12)
        assert np.abs(v1 - v0).max() <= 1e-7 * np.linalg.norm(v0)
        ref = oracle.energy_virial(target, p)
        assert rel_rms(f1, oracle.forces(target, p)) < 1e-5
        assert abs(e1[0] - ref["e_lj"]) <= 1e-6 * abs(ref["e_lj"])
        assert abs(e1[1] - ref["e_coul"]) <= 1e-6 * abs(ref["e_coul"])
        assert st1["n_pairs"] == ref["npairs"]
        # every other member of the mix is right too
        for m, (f, e, v, st) in zip(mix, results[:2] + results[3:]):
            assert rel_rms(f, oracle.forces(m, p)) < 1e-5
    finally:
        nb.nb_server_destroy(srv)


def test_budget_admission(ctx):
    p = wb.params_rf()
    boxes = [wb.water_box(m, None, seed=90 + k) for k, m in enumerate([3000, 3000, 3000])]
    one = nb.nb_sys_footprint(p, boxes[0].n, boxes[0].box)
    srv = nb.nb_server_create(ctx, p, int(1.5 * one) + (1 << 20), 64)
    try:
        ts = [_submit(srv, b) for b in boxes]
        for b, t in zip(boxes, ts):
            f, e, v, st = _wait(srv, b, t)
            assert st["wave_size"] == 1  # the budget holds one request at a time
            assert rel_rms(f, oracle.forces(b, p)) < 1e-5
        huge = wb.water_box(20000, None, seed=95)
        t = _submit(srv, huge)
        with pytest.raises(nb.NbError) as ei:
            _wait(srv, huge, t)
        assert ei.value.status == 4  # NB_ERR_BUDGET
    finally:
        nb.nb_server_destroy(srv)


def test_wait_times_out_without_blocking(ctx):
    p = wb.params_ewald()
    srv = nb.nb_server_create(ctx, p, 0, 64)
    try:
        big = wb.water_box(100000, None, seed=97)
        t = _submit(srv, big)
        with pytest.raises(nb.NbError) as ei:
            _wait(srv, big, t, timeout=0)
        assert ei.value.status == 7  # NB_ERR_TIMEOUT; the ticket stays valid
        f, e, v, st = _wait(srv, big, t)
        assert np.isfinite(f).all() and st["latency_s"] > 0
    finally:
        nb.nb_server_destroy(srv)
