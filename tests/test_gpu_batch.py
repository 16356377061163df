"""Batched evaluation (nb_batch_*) against per-system evaluation, and the oracle.

Several water boxes of different sizes run through one batch: one launch per
stage covers all of them and the force stage is one persistent kernel over
the flattened worklist of every system's cluster pairs.  With a non-default
stream the sequence is captured once in a CUDA graph and replayed.  Each
system's result must match its own plain evaluation and the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1506_00716_gb300 import nb
from paper_1506_00716_gb300 import waterbox as wb
from _support import gpu_eval, rel_rms

pytestmark = pytest.mark.gpu

FLAGS = nb.NB_F_ENERGY | nb.NB_F_VIRIAL


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_00716_gb300 import build as nbbuild

    nbbuild.build()
    torch.cuda.set_device(0)
    return torch


def _systems():
    # uneven sizes, every box edge >= 2 rlist (>= 400 molecules at 33.4 / nm^3)
    return [wb.water_box(m, None, seed=40 + k) for k, m in enumerate([400, 1000, 650, 2400, 520])]


def _run_batch(ctx, systems, params, submits=2):
    handles = []
    for s in systems:
        h = nb.nb_sys_create(ctx, params, s.n, s.box)
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_sys_set_coords(h, s.xq(), s.type)
        handles.append(h)
    b = nb.nb_batch_create(ctx, handles)
    out = []
    try:
        for _ in range(submits):
            t = nb.nb_batch_submit(b, FLAGS)
            assert nb.nb_batch_poll(b, t, 10_000_000)
            res = []
            for h, s in zip(handles, systems):
                f = np.zeros((s.n, 3), dtype=np.float32)
                e = np.zeros(2)
                v = np.zeros(9)
                nb.nb_sys_results(h, f, e, v)
                res.append((f, e, v))
            out.append(res)
    finally:
        nb.nb_batch_destroy(b)
        for h in handles:
            nb.nb_sys_destroy(h)
    return out


@pytest.mark.parametrize("use_stream,jcluster", [(True, 8), (False, 8), (True, 4)],
                         ids=["graph", "direct", "graph+8x4"])
@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_batch_matches_plain_and_oracle(torch_cuda, use_stream, jcluster, coul):
    torch = torch_cuda
    stream = torch.cuda.Stream() if use_stream else None
    ctx = nb.nb_ctx_create(0, stream, 0)
    nb.nb_ctx_set_tuning(ctx, 32, 3, 0, 0, jcluster)
    try:
        systems = _systems()
        p = wb.Params(coul=coul)
        runs = _run_batch(ctx, systems, p)
        for k, s in enumerate(systems):
            f0, e0, v0, _ = gpu_eval(ctx, s, p)
            for res in runs:  # every replay
                f, e, v = res[k]
                assert rel_rms(f, f0) < 1e-6
                assert np.allclose(e, e0, rtol=1e-10, atol=1e-12)
                assert np.abs(v - v0).max() <= 1e-7 * np.linalg.norm(v0)
            ref = oracle.energy_virial(s, p)
            f, e, v = runs[-1][k]
            assert rel_rms(f, oracle.forces(s, p)) < 1e-5
            assert abs(e[0] - ref["e_lj"]) <= 1e-6 * abs(ref["e_lj"])
            assert abs(e[1] - ref["e_coul"]) <= 1e-6 * abs(ref["e_coul"])
    finally:
        nb.nb_ctx_destroy(ctx)


def test_batch_poll_times_out_while_the_stream_is_busy(torch_cuda):
    torch = torch_cuda
    stream = torch.cuda.Stream()
    ctx = nb.nb_ctx_create(0, stream, 0)
    systems = _systems()[:2]
    handles = []
    try:
        for s in systems:
            h = nb.nb_sys_create(ctx, wb.params_rf(), s.n, s.box)
            nb.nb_sys_set_coords(h, s.xq(), s.type)
            handles.append(h)
        b = nb.nb_batch_create(ctx, handles)
        try:
            t = nb.nb_batch_submit(b, 0)  # capture + first replay
            assert nb.nb_batch_poll(b, t, 10_000_000)
            a = torch.randn(4096, 4096, device="cuda")
            with torch.cuda.stream(stream):
                for _ in range(40):  # keep the stream busy for a while (finite work)
                    a = a @ a
                    a = a / a.norm()
            t = nb.nb_batch_submit(b, 0)
            with pytest.raises(nb.NbError) as ei:
                nb.nb_batch_poll(b, t, 0)
            assert ei.value.status == 7  # NB_ERR_TIMEOUT, nothing waited on the device
            assert nb.nb_batch_poll(b, t, 60_000_000)
        finally:
            nb.nb_batch_destroy(b)
    finally:
        for h in handles:
            nb.nb_sys_destroy(h)
        nb.nb_ctx_destroy(ctx)


@pytest.mark.parametrize("search_mode,energy_mode", [(1, 0), (2, 0), (2, 1)],
                         ids=["warp_search", "thread_search", "thread_search+fused_energy"])
def test_batch_recovers_from_a_list_overflow(torch_cuda, search_mode, energy_mode):
    """A list that outgrows its capacity reports NB_ERR_CAPACITY, leaves the
    device state sound, and the resubmitted batch is correct.

    The batch's list capacity is sized for the tuning in force when it is
    created (max_entries 4096: about one item per (cluster, shift) run).
    Switching to max_entries 4 afterwards splits every run into items of four
    entries, several times more items than that capacity holds."""
    torch = torch_cuda
    stream = torch.cuda.Stream()
    ctx = nb.nb_ctx_create(0, stream, 0)
    systems = _systems()[:3]
    p = wb.params_rf()
    handles = []
    try:
        nb.nb_ctx_set_tuning(ctx, 4096, 3, search_mode, energy_mode)
        for s in systems:
            h = nb.nb_sys_create(ctx, p, s.n, s.box)
            nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
            nb.nb_sys_set_coords(h, s.xq(), s.type)
            handles.append(h)
        b = nb.nb_batch_create(ctx, handles)
        try:
            nb.nb_ctx_set_tuning(ctx, 4, 3, search_mode, energy_mode)
            t = nb.nb_batch_submit(b, FLAGS)
            with pytest.raises(nb.NbError) as ei:
                nb.nb_batch_poll(b, t, 10_000_000)
            assert ei.value.status == 9  # NB_ERR_CAPACITY, buffers grown
            t = nb.nb_batch_submit(b, FLAGS)
            assert nb.nb_batch_poll(b, t, 10_000_000)
            for h, s in zip(handles, systems):
                f = np.zeros((s.n, 3), dtype=np.float32)
                e = np.zeros(2)
                v = np.zeros(9)
                nb.nb_sys_results(h, f, e, v)
                ref = oracle.energy_virial(s, p)
                assert rel_rms(f, oracle.forces(s, p)) < 1e-5
                assert abs(e[0] - ref["e_lj"]) <= 1e-6 * abs(ref["e_lj"])
                assert abs(e[1] - ref["e_coul"]) <= 1e-6 * abs(ref["e_coul"])
        finally:
            nb.nb_batch_destroy(b)
    finally:
        for h in handles:
            nb.nb_sys_destroy(h)
        nb.nb_ctx_destroy(ctx)


def test_batch_with_reaction_field_exclusion_correction(torch_cuda):
    """The modifiers go through the batched path too (one launch per stage
    for all systems, the excluded-pair correction included)."""
    torch = torch_cuda
    stream = torch.cuda.Stream()
    ctx = nb.nb_ctx_create(0, stream, 0)
    try:
        systems = _systems()[:3]
        p = wb.Params(coul=wb.COUL_RF, modifiers=nb.NB_MOD_LJ_SHIFT | nb.NB_MOD_RF_EXCL)
        runs = _run_batch(ctx, systems, p, submits=1)
        for k, s in enumerate(systems):
            f, e, v = runs[0][k]
            ref = oracle.energy_virial(s, p)
            assert rel_rms(f, oracle.forces(s, p)) < 1e-5
            assert abs(e[0] - ref["e_lj"]) <= 1e-6 * abs(ref["e_lj"])
            assert abs(e[1] - ref["e_coul"]) <= 1e-6 * abs(ref["e_coul"])
            vr = ref["virial"].reshape(-1)
            assert np.abs(v - vr).max() <= 1e-6 * np.linalg.norm(vr)
    finally:
        nb.nb_ctx_destroy(ctx)
