"""Parity of the long-range (PME) part on the GPU with the FP64 oracle.

The oracle (oracle/pme.py) spreads with the same mesh and B-spline order, so
the comparison measures the implementation, not PME's own error: forces
within RMS(dF)/RMS(F) <= 1e-5, each energy part (E_rec, E_self, E_excl)
within 1e-6 relative, every virial component within 1e-6 of the sum of the
Frobenius norms of its parts.  The reciprocal and excluded-pair virials
cancel in part (their sum is about a third of the reciprocal one in water),
and each part carries the error of its own arithmetic (the float32 mesh and
transforms: a few 1e-7 of the reciprocal virial's norm), so the bound of the
sum is the sum of the parts' bounds.  Meshes cover every radix of the
transform (16, 4, 2, 3, 5), one-stage and many-stage transforms, odd mesh
sizes (an odd z length and an odd number of z lines), ragged transform tiles,
all three spline orders, and triclinic cells (rhombic dodecahedra).
"""
import numpy as np
import pytest

import oracle
from oracle import pme as opme
from paper_1506_00716_gb300 import nb
from paper_1506_00716_gb300 import waterbox as wb
from _support import rel_rms

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
E_TOL = 1e-6
V_TOL = 1e-6
EV = nb.NB_F_ENERGY | nb.NB_F_VIRIAL


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


BOXES = {"small": lambda: wb.small_box(seed=1), "mid": lambda: wb.mid_box(seed=2)}


def _system(ctx, s, p, grid, order):
    h = nb.nb_sys_create(ctx, p, s.n, s.box, getattr(s, "skew", None))
    nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
    nb.nb_grid_put(h, np.ascontiguousarray(s.xq()), np.ascontiguousarray(s.type))
    nb.nb_pairlist_build(h)
    nb.nb_pme_init(h, grid, order)
    return h


def _gpu_lr(ctx, s, p, grid, order, flags=EV):
    h = _system(ctx, s, p, grid, order)
    try:
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(3)
        v = np.zeros(9)
        nb.nb_pme_forces(h, None, f, e, v, flags)
    finally:
        nb.nb_sys_destroy(h)
    return f, e, v.reshape(3, 3)


def _oracle_lr(s, p, grid, order, sel=None):
    """Forces, (E_rec, E_self, E_excl), virial and the virial's error scale
    (the sum of the Frobenius norms of the reciprocal and excluded-pair parts)."""
    rec = opme.pme(s, p, grid=grid, order=order, sel=sel)
    ex = opme.ewald_exclusions(s, p)
    fex = ex["forces"] if sel is None else ex["forces"][sel]
    return (rec["forces"] + fex, np.array([rec["energy"], opme.ewald_self(s, p), ex["energy"]]),
            rec["virial"] + ex["virial"], np.linalg.norm(rec["virial"]) + np.linalg.norm(ex["virial"]))


def _check(f, e, v, rf, re, rv, vscale):
    assert rel_rms(f, rf) <= F_TOL, rel_rms(f, rf)
    for k in range(3):
        assert abs(e[k] - re[k]) <= E_TOL * abs(re[k]), (k, e[k], re[k])
    assert np.abs(v - rv).max() <= V_TOL * vscale, np.abs(v - rv).max() / vscale


@pytest.mark.parametrize("name,grid,order", [
    ("small", (24, 24, 24), 4),      # radices 4, 2, 3
    ("small", (25, 27, 45), 6),      # 5, 3 only; odd z length, odd number of z lines
    ("small", (32, 30, 20), 8),      # mixed per axis, order 8
    ("small", (16, 8, 16), 4),       # single-stage transforms (16) on x and z, 4 x 2 on y
    ("mid", (54, 50, 60), 4),        # 2 3 3 3 / 2 5 5 / 4 3 5
    ("mid", (64, 64, 64), 6),
])
def test_long_range_matches_oracle(ctx, name, grid, order):
    s = BOXES[name]()
    p = wb.params_ewald()
    f, e, v = _gpu_lr(ctx, s, p, grid, order)
    _check(f, e, v, *_oracle_lr(s, p, grid, order))


def test_far_excluded_pairs(ctx):
    """Exclusions between atoms of different molecules at any distance up to
    half the box (beta r >= 1 takes the float64 library erf in the kernel,
    beta r < 1 the series), listed under one atom only."""
    s = BOXES["small"]()
    p = wb.params_ewald()
    n_mol = s.n // 3
    extra = {3 * m: 3 * ((m * 7 + 5) % n_mol) + 1 for m in range(0, n_mol, 4)}
    lists = [list(s.excl_atoms[s.excl_index[i]:s.excl_index[i + 1]]) for i in range(s.n)]
    for a, b in extra.items():
        if b != a and b not in lists[a]:
            lists[a].append(b)
    idx = np.zeros(s.n + 1, dtype=np.int32)
    idx[1:] = np.cumsum([len(x) for x in lists])
    at = np.array([b for x in lists for b in x], dtype=np.int32)
    s2 = wb.System(**{**s.__dict__})
    s2.excl_index, s2.excl_atoms = idx, at
    f, e, v = _gpu_lr(ctx, s2, p, (24, 24, 24), 4)
    _check(f, e, v, *_oracle_lr(s2, p, (24, 24, 24), 4))


TRI = {"rd_small": lambda: wb.rhombic_dodecahedron_box(648, seed=5),    # 2,100 atoms, d = 3.11 nm
       "rd_mid": lambda: wb.rhombic_dodecahedron_box(7744, seed=6)}    # 23,232 atoms, d = 6.83 nm


@pytest.mark.parametrize("name,grid,order", [
    ("rd_small", (24, 30, 18), 4),   # even meshes: Nyquist mirrors with their own G in the skewed cell
    ("rd_small", (16, 20, 12), 6),   # coarse, so that those terms matter
    ("rd_small", (25, 27, 15), 4),   # odd sizes: no Nyquist index
    ("rd_mid", (60, 60, 40), 4),
])
def test_triclinic_long_range_matches_oracle(ctx, name, grid, order):
    """Rhombic dodecahedra (box rows a = (d,0,0), b = (0,d,0),
    c = (d/2, d/2, d sqrt(2)/2))."""
    s = TRI[name]()
    p = wb.params_ewald()
    f, e, v = _gpu_lr(ctx, s, p, grid, order)
    _check(f, e, v, *_oracle_lr(s, p, grid, order))


def test_triclinic_combined_with_short_range(ctx):
    s = TRI["rd_small"]()
    p = wb.params_ewald()
    grid = (24, 30, 18)
    h = _system(ctx, s, p, grid, 4)
    try:
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(2)
        v = np.zeros(9)
        nb.nb_forces(h, None, f, e, v, EV | nb.NB_F_PME)
    finally:
        nb.nb_sys_destroy(h)
    lf, le, lv, lscale = _oracle_lr(s, p, grid, 4)
    ev = oracle.energy_virial(s, p)
    rf = oracle.forces(s, p) + lf
    assert rel_rms(f, rf) <= F_TOL, rel_rms(f, rf)
    e_c = ev["e_coul"] + le.sum()
    assert abs(e[1] - e_c) <= E_TOL * (abs(ev["e_coul"]) + np.abs(le).sum())
    rv = ev["virial"] + lv
    assert np.abs(v.reshape(3, 3) - rv).max() <= V_TOL * (np.linalg.norm(ev["virial"]) + lscale)


def test_forces_only_flags(ctx):
    s = BOXES["small"]()
    p = wb.params_ewald()
    f0, _, _ = _gpu_lr(ctx, s, p, (24, 24, 24), 4, flags=0)
    f1, _, _ = _gpu_lr(ctx, s, p, (24, 24, 24), 4, flags=EV)
    assert rel_rms(f0, f1) <= F_TOL


@pytest.mark.parametrize("name,grid", [("small", (24, 24, 24)), ("mid", (60, 60, 60))])
def test_combined_with_short_range(ctx, name, grid):
    """nb_forces with NB_F_PME: short-range + long-range sums."""
    s = BOXES[name]()
    p = wb.params_ewald()
    h = _system(ctx, s, p, grid, 4)
    try:
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(2)
        v = np.zeros(9)
        nb.nb_forces(h, None, f, e, v, EV | nb.NB_F_PME)
    finally:
        nb.nb_sys_destroy(h)
    lf, le, lv, lscale = _oracle_lr(s, p, grid, 4)
    ev = oracle.energy_virial(s, p)
    rf = oracle.forces(s, p) + lf
    assert rel_rms(f, rf) <= F_TOL, rel_rms(f, rf)
    assert e[0] == pytest.approx(ev["e_lj"], rel=E_TOL)
    # sums of separately computed parts: the bound is the sum of the parts' bounds
    e_c = ev["e_coul"] + le.sum()
    assert abs(e[1] - e_c) <= E_TOL * (abs(ev["e_coul"]) + np.abs(le).sum())
    rv = ev["virial"] + lv
    assert np.abs(v.reshape(3, 3) - rv).max() <= V_TOL * (np.linalg.norm(ev["virial"]) + lscale)


def test_new_coordinates(ctx):
    """nb_pme_forces(x_new): moved atoms, some across the box faces."""
    s = BOXES["small"]()
    p = wb.params_ewald()
    h = _system(ctx, s, p, (24, 24, 24), 4)
    rng = np.random.default_rng(7)
    x_new = (s.x.astype(np.float64) + rng.normal(scale=0.01, size=s.x.shape)).astype(np.float32)
    try:
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(3)
        v = np.zeros(9)
        nb.nb_pme_forces(h, np.ascontiguousarray(x_new), f, e, v, EV)
    finally:
        nb.nb_sys_destroy(h)
    moved = wb.System(**{**s.__dict__})
    moved.x = x_new
    _check(f, e, v.reshape(3, 3), *_oracle_lr(moved, p, (24, 24, 24), 4))


def test_device_buffers(ctx):
    import torch

    s = BOXES["small"]()
    p = wb.params_ewald()
    h = _system(ctx, s, p, (24, 24, 24), 4)
    try:
        fh = np.zeros((s.n, 3), dtype=np.float32)
        eh = np.zeros(3)
        vh = np.zeros(9)
        nb.nb_pme_forces(h, None, fh, eh, vh, EV)
        fd = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
        ed = torch.zeros(3, dtype=torch.float64, device="cuda")
        vd = torch.zeros(9, dtype=torch.float64, device="cuda")
        nb.nb_pme_forces(h, None, fd, ed, vd, EV)
        torch.cuda.synchronize()
    finally:
        nb.nb_sys_destroy(h)
    # the spread's float32 atomics sum in a different order on every run
    assert rel_rms(fd.cpu().numpy(), fh) <= F_TOL
    assert np.allclose(ed.cpu().numpy(), eh, rtol=E_TOL)
    assert np.allclose(vd.cpu().numpy(), vh, rtol=0, atol=V_TOL * np.abs(vh).max())


def test_reinit_mesh_and_memory_accounting(ctx):
    """A second nb_pme_init replaces the mesh (new size and order take effect);
    the budget accounting returns to its start when the system is destroyed."""
    s = BOXES["small"]()
    p = wb.params_ewald()
    used0, _ = nb.nb_ctx_memory(ctx)
    h = _system(ctx, s, p, (24, 24, 24), 4)
    used1, _ = nb.nb_ctx_memory(ctx)
    try:
        nb.nb_pme_init(h, (32, 30, 20), 6)
        used2, _ = nb.nb_ctx_memory(ctx)
        # the mesh grows from 24^3 to 32 x 30 x 20 (real + half spectrum)
        assert used2 > used1
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(3)
        v = np.zeros(9)
        nb.nb_pme_forces(h, None, f, e, v, EV)
    finally:
        nb.nb_sys_destroy(h)
    _check(f, e, v.reshape(3, 3), *_oracle_lr(s, p, (32, 30, 20), 6))
    used3, _ = nb.nb_ctx_memory(ctx)
    assert used3 == used0


def test_validation(ctx):
    s = BOXES["small"]()
    p = wb.params_ewald()
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    try:
        for grid, order, status in (((24, 24, 7), 4, 1), ((24, 24, 28), 4, 1), ((24, 24, 1030), 4, 1),
                                    ((24, 24, 24), 5, 1), ((24, 24, 12), 8, 1)):
            with pytest.raises(nb.NbError) as ei:
                nb.nb_pme_init(h, grid, order)
            assert ei.value.status == status
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_grid_put(h, np.ascontiguousarray(s.xq()), np.ascontiguousarray(s.type))
        nb.nb_pairlist_build(h)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_forces(h, None, None, None, None, nb.NB_F_PME)
        assert ei.value.status == 8
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pme_forces(h, None, None, None, None, 0)
        assert ei.value.status == 8
    finally:
        nb.nb_sys_destroy(h)
    hr = nb.nb_sys_create(ctx, wb.params_rf(), s.n, s.box)
    try:
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pme_init(hr, (24, 24, 24), 4)
        assert ei.value.status == 1
    finally:
        nb.nb_sys_destroy(hr)


def test_full_size_3M_atoms(ctx):
    """The 3,000,000-atom box with a 256^3 mesh, order 4 (0.12 nm spacing):
    energies and virial in full, forces on 192 sampled atoms."""
    s = wb.large_box(seed=3)
    p = wb.params_ewald()
    grid = (256, 256, 256)
    f, e, v = _gpu_lr(ctx, s, p, grid, 4)
    sel = np.sort(np.random.default_rng(31).choice(s.n, size=192, replace=False))
    _check(f[sel], e, v, *_oracle_lr(s, p, grid, 4, sel=sel))
