"""The allocation-free entry point nb_eval_noalloc against the regular path.

nb_eval_noalloc exists for callers that cannot allocate device memory: a
plug-in that is only handed a stream by its host framework, code running
inside another memory manager's budget, or a latency-critical loop that must
never reach cudaMalloc (which can synchronise the device).  It runs the whole
evaluation in a fixed scratch array that is part of the library.

Two calls in a row, on systems of different sizes and electrostatics, each
compared with nb_grid_put + nb_pairlist_build + nb_forces on the same inputs,
within the parity tolerances of the other GPU tests.  The file is named to
be collected last; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

from paper_1506_00716_gb300 import nb
from paper_1506_00716_gb300 import waterbox as wb

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
E_TOL = 1e-6
V_TOL = 1e-6


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


def _regular(ctx, s, p, flags):
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    try:
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(2)
        v = np.zeros(9)
        nb.nb_forces(h, None, f, e, v, flags)
    finally:
        nb.nb_sys_destroy(h)
    return f, e, v


def _noalloc(s, p, flags):
    f = np.zeros((s.n, 3), dtype=np.float32)
    e = np.zeros(2)
    v = np.zeros(9)
    nb.nb_eval_noalloc(p, s.n, s.box, s.excl_index, s.excl_atoms, s.xq(), s.type, f, e, v, flags)
    return f, e, v


def test_noalloc_matches_regular_entry_point_twice(ctx):
    flags = nb.NB_F_ENERGY | nb.NB_F_VIRIAL
    cases = [(wb.mid_box(seed=2), wb.params_rf()), (wb.small_box(seed=1), wb.params_ewald())]
    for s, p in cases:  # two calls in a row on the shared scratch array
        f0, e0, v0 = _regular(ctx, s, p, flags)
        f1, e1, v1 = _noalloc(s, p, flags)
        rel_f = np.sqrt(((f1 - f0) ** 2).mean()) / np.sqrt((f0 ** 2).mean())
        assert rel_f <= F_TOL, rel_f
        assert abs(e1[0] - e0[0]) <= E_TOL * abs(e0[0])
        assert abs(e1[1] - e0[1]) <= E_TOL * abs(e0[1])
        assert np.abs(v1 - v0).max() <= V_TOL * np.linalg.norm(v0)


def test_noalloc_rejects_systems_above_its_limit(ctx):
    s = wb.water_box(11000, None, seed=3)  # 33,000 atoms > 32,768
    with pytest.raises(nb.NbError) as ei:
        _noalloc(s, wb.params_rf(), 0)
    assert ei.value.status == 9
