"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the pair list covers the oracle's interacting pairs exactly
(integer set equality) and every pair inside rlist; forces within
RMS(dF)/RMS(F) <= 1e-5; E_LJ, E_C within 1e-6 relative; every virial
component within 1e-6 of the virial's Frobenius norm.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1506_00716_gb300 import nb
from paper_1506_00716_gb300 import waterbox as wb
from _support import expand_pairs, export_list, gpu_eval, rel_rms

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
    c = nb.nb_ctx_create(0, None, 0)
    yield c
    nb.nb_ctx_destroy(c)


BOXES = {
    "small": lambda: wb.small_box(seed=1),
    "mid": lambda: wb.mid_box(seed=2),
    # triclinic: a rhombic dodecahedron of 700 waters (d = 3.11 nm)
    "rd_small": lambda: wb.rhombic_dodecahedron_box(648, seed=5),
}


@pytest.fixture(params=[(1, 0, 8, None), (2, 0, 8, None), (1, 1, 8, None),
                        (1, 0, 4, None), (2, 0, 4, None), (1, 1, 4, None), (2, 0, 4, 1), (1, 0, 4, 4)],
                ids=["warp_search+energy_kernel", "thread_search+energy_kernel", "warp_search+fused_energy",
                     "8x4+warp_search+energy_kernel", "8x4+thread_search+energy_kernel",
                     "8x4+warp_search+fused_energy", "8x4+thread_search+screening_energy_kernel",
                     "8x4+warp_search+energy_kernel+96_registers"])
def search_mode(request, ctx):
    """Both search kernels (a warp per i-cluster, a thread per i-cluster),
    whatever the size would choose, both energy paths (fused into the force
    kernel, or the separate energy kernel, queuing from the force kernel's
    marks or, at the register budget of one block per SM, screening the
    slots itself) and both cluster geometries (8 x 8, 8 x 4), and the force
    kernel's register budgets; the tuning is restored afterwards."""
    old = nb.nb_ctx_get_tuning(ctx)
    sm, em, jc, mb = request.param
    nb.nb_ctx_set_tuning(ctx, old["max_entries"], mb or old["force_min_blocks"], sm, em, jc)
    yield request.param
    nb.nb_ctx_set_tuning(ctx, old["max_entries"], old["force_min_blocks"], old["search_mode"], old["energy_mode"],
                         old["jcluster"])


@pytest.mark.parametrize("name", ["small", "mid", "rd_small"])
def test_pairlist_covers_oracle_pairs_exactly(ctx, name, search_mode):
    s = BOXES[name]()
    p = wb.params_rf()
    _, _, _, h = gpu_eval(ctx, s, p, flags=0, keep=True)
    try:
        info, perm, items, jslot, mask = export_list(h)
    finally:
        nb.nb_sys_destroy(h)
    assert sorted(perm[perm >= 0].tolist()) == list(range(s.n))
    got, occurrences = expand_pairs(s, perm, items, jslot, mask, p.rc)
    ref = oracle.pairs(s, p.rc)
    assert occurrences == got.shape[0], "a pair appears twice inside rc (double counting)"
    assert np.array_equal(got, ref)
    got_l, _ = expand_pairs(s, perm, items, jslot, mask, p.rlist)
    ref_l = oracle.pairs(s, p.rlist)
    assert np.isin(ref_l, got_l).all(), "a pair inside rlist is missing from the list"
    assert info["n_entries"] <= info["n_entries_raw"]


def _check(s, p, f, e, v, f_tol=F_TOL, e_tol=E_TOL, v_tol=V_TOL):
    ref_f = oracle.forces(s, p)
    ref = oracle.energy_virial(s, p)
    errs = {
        "f": rel_rms(f, ref_f),
        "e_lj": abs(e[0] - ref["e_lj"]) / abs(ref["e_lj"]),
        "e_coul": abs(e[1] - ref["e_coul"]) / abs(ref["e_coul"]),
        "virial": float(np.abs(v - ref["virial"].reshape(-1)).max() / np.linalg.norm(ref["virial"])),
    }
    print(errs)
    assert errs["f"] <= f_tol, errs
    assert errs["e_lj"] <= e_tol, errs
    assert errs["e_coul"] <= e_tol, errs
    assert errs["virial"] <= v_tol, errs
    return errs


@pytest.mark.parametrize("name", ["small", "mid", "rd_small"])
@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_forces_energies_virial(ctx, name, coul, search_mode):
    s = BOXES[name]()
    p = wb.Params(coul=coul)
    f, e, v, _ = gpu_eval(ctx, s, p)
    _check(s, p, f, e, v)


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_interacting_pair_count_is_exact(ctx, coul):
    s = BOXES["mid"]()
    p = wb.Params(coul=coul)
    _, _, _, h = gpu_eval(ctx, s, p, keep=True)
    try:
        n = nb.nb_eval_info(h)["n_pairs"]
    finally:
        nb.nb_sys_destroy(h)
    assert n == oracle.energy_virial(s, p)["npairs"]


@pytest.mark.parametrize("flags", [0, nb.NB_F_ENERGY, nb.NB_F_VIRIAL])
def test_flag_variants_give_the_same_forces(ctx, flags):
    s = BOXES["small"]()
    p = wb.params_rf()
    f_all, e_all, v_all, _ = gpu_eval(ctx, s, p)
    f, e, v, _ = gpu_eval(ctx, s, p, flags=flags)
    assert rel_rms(f, f_all) < 1e-6
    if flags & nb.NB_F_ENERGY:
        assert np.allclose(e, e_all, rtol=1e-9, atol=0)
    if flags & nb.NB_F_VIRIAL:
        assert np.allclose(v, v_all, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("geometry", [8, 4], indirect=True, ids=["8x8", "8x4"])
def test_stale_list_evaluations(ctx, geometry):
    """24,000-atom box: list rebuilt every 10 evaluations, Gaussian moves
    between; both cluster geometries."""
    s = wb.mid_box(seed=2)
    p = wb.params_rf()
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
    rng = np.random.default_rng(99)
    try:
        for ev in range(12):
            if ev % 10 == 0:
                nb.nb_grid_put(h, s.xq(), s.type)
                nb.nb_pairlist_build(h)
                x_new = None
            else:
                s.x = (s.x.astype(np.float64) + rng.normal(0.0, 0.005, size=s.x.shape)).astype(np.float32)
                x_new = np.ascontiguousarray(s.x)
            if ev in (0, 5, 9, 11):
                f = np.zeros((s.n, 3), dtype=np.float32)
                e = np.zeros(2)
                v = np.zeros(9)
                nb.nb_forces(h, x_new, f, e, v, nb.NB_F_ENERGY | nb.NB_F_VIRIAL)
                _check(s, p, f, e, v)
            else:
                nb.nb_forces(h, x_new, None, None, None, 0)
    finally:
        nb.nb_sys_destroy(h)


@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
def test_caller_buffer_kinds(ctx, kind):
    """nb_forces with new coordinates and all outputs in pageable host
    memory (staged copies), pinned host memory (read and written by the
    kernels through its mapped address) or device memory."""
    torch = pytest.importorskip("torch")
    s = wb.small_box(seed=1)
    p = wb.params_rf()
    rng = np.random.default_rng(7)
    x1 = (s.x.astype(np.float64) + rng.normal(0.0, 0.005, size=s.x.shape)).astype(np.float32)
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    try:
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)
        if kind == "pageable":
            x, f, e, v = np.ascontiguousarray(x1), np.zeros((s.n, 3), np.float32), np.zeros(2), np.zeros(9)
        else:
            mk = (lambda a: torch.from_numpy(a).pin_memory()) if kind == "pinned" else (lambda a: torch.from_numpy(a).cuda())
            x, f, e, v = mk(x1), mk(np.zeros((s.n, 3), np.float32)), mk(np.zeros(2)), mk(np.zeros(9))
        nb.nb_forces(h, x, f, e, v, nb.NB_F_ENERGY | nb.NB_F_VIRIAL)
        # the call has finished with host memory when it returns
        if kind != "pageable":
            f, e, v = (t.cpu().numpy() for t in (f, e, v))
    finally:
        nb.nb_sys_destroy(h)
    s.x = x1
    _check(s, p, f, e, v)


@pytest.fixture
def geometry(request, ctx):
    """The context's j-cluster size set to the test's parameter, restored after."""
    old = nb.nb_ctx_get_tuning(ctx)
    nb.nb_ctx_set_tuning(ctx, old["max_entries"], old["force_min_blocks"], old["search_mode"], old["energy_mode"],
                         request.param)
    yield request.param
    nb.nb_ctx_set_tuning(ctx, old["max_entries"], old["force_min_blocks"], old["search_mode"], old["energy_mode"],
                         old["jcluster"])


@pytest.mark.parametrize("geometry", [8, 4], indirect=True, ids=["8x8", "8x4"])
def test_dynamic_pruning(ctx, geometry):
    """Outer list at rlist = 1.3 nm built once; pruned out of place to an inner
    list at 1.1 nm every 5 evaluations while the atoms move (Gaussian, sigma
    0.005 nm per evaluation); every checked evaluation matches the oracle,
    interacting-pair count included.  Both cluster geometries (the inner
    list of an 8 x 4 list re-pairs the halves it keeps)."""
    s = wb.mid_box(seed=2)
    p = wb.Params(coul=wb.COUL_RF, rlist=1.3)
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
    rng = np.random.default_rng(123)
    try:
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pairlist_prune(h, 1.1)
        assert ei.value.status == 8  # NB_ERR_STATE: no list yet
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)
        for bad in (0.9, 1.4):
            with pytest.raises(nb.NbError) as ei:
                nb.nb_pairlist_prune(h, bad)
            assert ei.value.status == 1  # NB_ERR_ARG: outside [rc, rlist]
        x_new = None
        for ev in range(20):
            if ev > 0:
                s.x = (s.x.astype(np.float64) + rng.normal(0.0, 0.005, size=s.x.shape)).astype(np.float32)
                x_new = np.ascontiguousarray(s.x)
            if ev % 5 == 0:
                if x_new is not None:
                    nb.nb_forces(h, x_new, None, None, None, 0)  # coordinates of this evaluation
                nb.nb_pairlist_prune(h, 1.1)
                info = nb.nb_pairlist_info(h)
                assert info["n_entries_inner"] < info["n_entries"]
            if ev in (0, 4, 9, 14, 19):
                f = np.zeros((s.n, 3), dtype=np.float32)
                e = np.zeros(2)
                v = np.zeros(9)
                nb.nb_forces(h, x_new, f, e, v, nb.NB_F_ENERGY | nb.NB_F_VIRIAL)
                _check(s, p, f, e, v)
                assert nb.nb_eval_info(h)["n_pairs"] == oracle.energy_virial(s, p)["npairs"]
            else:
                nb.nb_forces(h, x_new, None, None, None, 0)
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)  # a new outer list discards the inner one
        info = nb.nb_pairlist_info(h)
        assert info["n_entries_inner"] == info["n_entries"]
    finally:
        nb.nb_sys_destroy(h)


def test_triclinic_mid_box_sampled_forces_and_stale_moves(ctx):
    """Rhombic dodecahedron of 7,744 waters (23,232 atoms), LJ + RF: forces of
    sampled atoms against the oracle's per-atom loop, before and after moves
    that carry atoms across the skewed faces (coordinates not re-wrapped), and
    the net force."""
    s = wb.rhombic_dodecahedron_box(8000, seed=6)
    p = wb.params_rf()
    h = nb.nb_sys_create(ctx, p, s.n, s.box, s.skew)
    nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
    rng = np.random.default_rng(61)
    sel = np.sort(rng.choice(s.n, size=256, replace=False)).astype(np.int32)
    try:
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)
        x_new = None
        for ev in range(6):
            if ev > 0:
                s.x = (s.x.astype(np.float64) + rng.normal(0.0, 0.01, size=s.x.shape)).astype(np.float32)
                x_new = np.ascontiguousarray(s.x)
            f = np.zeros((s.n, 3), dtype=np.float32)
            nb.nb_forces(h, x_new, f, None, None, 0)
            if ev in (0, 5):
                assert rel_rms(f[sel], oracle.forces(s, p, sel)) <= F_TOL
                rms = np.sqrt((f.astype(np.float64) ** 2).mean())
                assert np.linalg.norm(f.astype(np.float64).sum(0)) <= 1e-4 * np.sqrt(s.n) * rms
    finally:
        nb.nb_sys_destroy(h)


def test_triclinic_box_validation(ctx):
    p = wb.params_rf()
    d = 3.2
    rd = [d, 0, 0, 0, d, 0, d / 2, d / 2, d * 0.70710678]
    box3, skew = (rd[0], rd[4], rd[8]), (rd[3], rd[6], rd[7])
    h = nb.nb_sys_create(ctx, p, 100, box3, skew)  # a rhombic dodecahedron is admitted
    nb.nb_sys_destroy(h)
    bad = [((d, d, 3.0), (d * 0.3, d * 0.3, 0.0)),   # |bx| + |cx| > ax/2
           ((d, d, 3.0), (0.0, 0.0, d * 0.6)),       # |cy| > by/2
           ((2.0, d, 3.0), (0.0, 0.5, 0.0)),         # rlist > ax/2
           ((d, d, 1.05), (0.0, 0.2, 0.2))]          # rlist >= cz
    for box, sk in bad:
        with pytest.raises(nb.NbError) as ei:
            nb.nb_sys_create(ctx, p, 100, box, sk)
        assert ei.value.status == 2  # NB_ERR_BOX


def test_single_molecule_has_no_interactions(ctx):
    s = wb.water_box(1, 3.0, seed=5)
    f, e, v, _ = gpu_eval(ctx, s, wb.params_rf())
    assert np.all(f == 0) and np.all(e == 0) and np.all(v == 0)


def test_a_single_atom_and_no_atoms(ctx):
    """The degenerate sizes: one atom has no pairs at all (zero forces,
    energies, virial and pair count); no atoms is refused."""
    p = wb.params_ewald()
    h = nb.nb_sys_create(ctx, p, 1, [3.0, 3.0, 3.0])
    try:
        nb.nb_set_exclusions(h, np.zeros(2, np.int32), np.zeros(0, np.int32))
        nb.nb_grid_put(h, np.array([[1.0, 2.0, 0.5, -0.8]], np.float32), np.zeros(1, np.int32))
        nb.nb_pairlist_build(h)
        f = np.full((1, 3), 7.0, np.float32)
        e = np.full(2, 7.0)
        v = np.full(9, 7.0)
        nb.nb_forces(h, None, f, e, v, nb.NB_F_ENERGY | nb.NB_F_VIRIAL)
        assert np.all(f == 0) and np.all(e == 0) and np.all(v == 0)
        assert nb.nb_eval_info(h)["n_pairs"] == 0
    finally:
        nb.nb_sys_destroy(h)
    with pytest.raises(nb.NbError) as ei:
        nb.nb_sys_create(ctx, p, 0, [3.0, 3.0, 3.0])
    assert ei.value.status == 1


def test_two_atoms_across_the_boundary(ctx):
    L = wb.f32(2.5)
    s = wb.System(x=np.array([[0.05, 1.0, 1.0], [L - 0.25, 1.0, 1.0]], dtype=np.float32),
                  q=np.array([1.0, -1.0], dtype=np.float32), type=np.array([0, 0], dtype=np.int32),
                  box=np.array([L, L, L]), excl_index=np.zeros(3, dtype=np.int32),
                  excl_atoms=np.zeros(0, dtype=np.int32), n_mol=0, seed=0)
    p = wb.params_rf()
    f, e, v, _ = gpu_eval(ctx, s, p)
    _check(s, p, f, e, v, f_tol=1e-6, e_tol=1e-6, v_tol=1e-6)


def test_coordinates_outside_the_box_are_wrapped(ctx):
    s = BOXES["small"]()
    p = wb.params_rf()
    f0, e0, v0, _ = gpu_eval(ctx, s, p)
    L = np.float32(s.box[0])
    moved = wb.System(**{**s.__dict__})
    k = np.random.default_rng(3).integers(-2, 3, size=s.x.shape).astype(np.float32)
    moved.x = (s.x + k * L).astype(np.float32)
    f1, e1, v1, _ = gpu_eval(ctx, moved, p)
    # the library wraps x - L floor(x / L) in float32; for |k| <= 2 that is the
    # same rounding as numpy's, so the oracle sees exactly the wrapped inputs
    wrapped = wb.System(**{**moved.__dict__})
    w = (moved.x - L * np.floor(moved.x / L)).astype(np.float32)
    w[w >= L] = 0.0
    wrapped.x = w
    _check(wrapped, p, f1, e1, v1)


def test_box_of_exactly_two_list_radii(ctx):
    s = wb.water_box(300, 2.2, seed=8)
    p = wb.params_rf()
    f, e, v, _ = gpu_eval(ctx, s, p)
    _check(s, p, f, e, v)


MODIFIER_CASES = [
    (wb.COUL_RF, nb.NB_MOD_LJ_SHIFT),
    (wb.COUL_RF, nb.NB_MOD_RF_EXCL),
    (wb.COUL_RF, nb.NB_MOD_LJ_SHIFT | nb.NB_MOD_RF_EXCL),
    (wb.COUL_EWALD, nb.NB_MOD_EWALD_SHIFT),
    (wb.COUL_EWALD, nb.NB_MOD_LJ_SHIFT | nb.NB_MOD_EWALD_SHIFT),
]


@pytest.mark.parametrize("coul,mods", MODIFIER_CASES)
@pytest.mark.parametrize("name", ["small", "mid"])
def test_potential_modifiers(ctx, name, coul, mods, search_mode):
    """Potential-shift and excluded-pair reaction-field variants against the
    oracle with the same modifiers, at the standard tolerances."""
    s = BOXES[name]()
    p = wb.Params(coul=coul, modifiers=mods)
    f, e, v, _ = gpu_eval(ctx, s, p)
    _check(s, p, f, e, v)


def test_one_sided_exclusions_are_symmetrised(ctx):
    """Exclusions listed in one direction only, unsorted, with a self pair and
    a duplicate, give the same result as the canonical symmetric list: the
    library symmetrises what is not canonical and uses a canonical list as it
    is."""
    s = BOXES["small"]()
    p = wb.params_rf()
    n = s.n
    rows = []
    for a in range(n):
        m0 = 3 * (a // 3)
        partners = [b for b in range(m0, m0 + 3) if b > a][::-1]  # one direction, descending
        if a % 3 == 0:
            partners += [a, partners[0]]  # a self pair and a duplicate
        rows.append(partners)
    idx = np.zeros(n + 1, dtype=np.int32)
    idx[1:] = np.cumsum([len(r) for r in rows])
    atoms = np.array([b for r in rows for b in r], dtype=np.int32)
    one_sided = dataclasses.replace(s, excl_index=idx, excl_atoms=atoms)
    f0, e0, v0, _ = gpu_eval(ctx, s, p)
    f1, e1, v1, _ = gpu_eval(ctx, one_sided, p)
    assert rel_rms(f1, f0) < 1e-6
    assert np.allclose(e1, e0, rtol=1e-12, atol=0)
    assert np.abs(v1 - v0).max() <= 1e-7 * np.linalg.norm(v0)
    _check(s, p, f1, e1, v1)


def test_error_paths(ctx):
    p = wb.params_rf()
    with pytest.raises(nb.NbError) as ei:
        nb.nb_sys_create(ctx, p, 100, [1.5, 3.0, 3.0])
    assert ei.value.status == 2
    h = nb.nb_sys_create(ctx, p, 3, [3.0, 3.0, 3.0])
    try:
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pairlist_build(h)
        assert ei.value.status == 8
        with pytest.raises(nb.NbError) as ei:
            nb.nb_forces(h, None, None, None, None, 0)
        assert ei.value.status == 8
        with pytest.raises(nb.NbError) as ei:
            nb.nb_forces(h, None, None, None, None, 1)  # energy flag without a buffer
        assert ei.value.status == 1
    finally:
        nb.nb_sys_destroy(h)


def test_budget_refuses_without_allocating(ctx):
    c = nb.nb_ctx_create(0, None, 1 << 20)
    try:
        with pytest.raises(nb.NbError) as ei:
            nb.nb_sys_create(c, wb.params_rf(), 24000, [6.21] * 3)
        assert ei.value.status == 4
        assert nb.nb_ctx_memory(c)[0] == 0
    finally:
        nb.nb_ctx_destroy(c)


def test_device_erfc_two_atom_pairs(ctx):
    """The kernels' erfc on the device, one atom pair at a time: two unit
    charges without Lennard-Jones at distance r in (0.02, rc), Ewald real
    space.  The energy kernel's double-float V = f erfc(beta r) / r against
    the standard library's erfc at 2e-9 relative (its erfc, from the energy
    table, is good to 3e-11 absolute, see tests/test_ewald_energy_table_cpu.py),
    and the force kernel's float32 F = f (erfc(beta r)/r + 2 beta/sqrt(pi)
    exp(-beta^2 r^2)) / r against the same formula at 2e-6 relative (SFU rsqrt,
    the force table's 1e-7, see tests/test_ewald_table_cpu.py, and a few float32
    roundings)."""
    import math

    p = wb.params_ewald()
    p = dataclasses.replace(p, c6=np.zeros(4, dtype=np.float32), c12=np.zeros(4, dtype=np.float32))
    L = 2.4
    x0 = np.float32(0.7)
    worst_e = worst_f = 0.0
    for r_want in np.concatenate([np.geomspace(0.02, 0.2, 8), np.linspace(0.21, 0.999, 40)]):
        x1 = np.float32(x0 + np.float32(r_want))
        r = float(x1) - float(x0)  # exact: both coordinates are float32
        xq = np.array([[x0, 1.2, 1.2, 1.0], [x1, 1.2, 1.2, 1.0]], dtype=np.float32)
        s = wb.System(x=xq[:, :3].copy(), q=xq[:, 3].copy(), type=np.array([1, 1], dtype=np.int32),
                      box=np.array([L, L, L]), excl_index=np.zeros(3, dtype=np.int32),
                      excl_atoms=np.zeros(0, dtype=np.int32), n_mol=0, seed=0)
        f, e, v, _ = gpu_eval(ctx, s, p)
        br = p.beta * r
        v_ref = p.fcoul * math.erfc(br) / r
        f_ref = p.fcoul * (math.erfc(br) / r + 2.0 * p.beta / math.sqrt(math.pi) * math.exp(-br * br)) / r
        # the force on atom 0 points away from atom 1 (repulsion), along -x
        worst_e = max(worst_e, abs(e[1] - v_ref) / abs(v_ref))
        worst_f = max(worst_f, abs(-float(f[0, 0]) - f_ref) / f_ref, abs(float(f[1, 0]) - f_ref) / f_ref)
        assert e[0] == 0.0 and f[0, 1] == 0.0 and f[0, 2] == 0.0
    assert worst_e <= 2e-9, worst_e
    assert worst_f <= 2e-6, worst_f


def test_thread_search_grows_an_overflowing_list(ctx):
    """The thread-per-cluster search sized for one item split, then run with
    a finer one: its scan sees the list outgrow the buffers, writes no
    entries, the build grows the buffers and searches again; the forces are
    the oracle's."""
    s = BOXES["small"]()
    p = wb.params_rf()
    old = nb.nb_ctx_get_tuning(ctx)
    nb.nb_ctx_set_tuning(ctx, 4096, old["force_min_blocks"], 2)
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    try:
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)
        nb.nb_ctx_set_tuning(ctx, 4, old["force_min_blocks"], 2)
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)
        info = nb.nb_pairlist_info(h)
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(2)
        v = np.zeros(9)
        nb.nb_forces(h, None, f, e, v, nb.NB_F_ENERGY | nb.NB_F_VIRIAL)
        _check(s, p, f, e, v)
        assert info["n_items"] >= info["n_entries"] / 4
    finally:
        nb.nb_sys_destroy(h)
        nb.nb_ctx_set_tuning(ctx, old["max_entries"], old["force_min_blocks"], old["search_mode"],
                             old["energy_mode"])


def _three_type_box(seed):
    """The 1,944-atom box with every third oxygen made type 2: a Lennard-Jones
    table with three distinct nonzero parameter pairs (geometric mixing of
    sigma-epsilon pairs), which the kernels must look up per type pair."""
    s = wb.small_box(seed=seed)
    t = s.type.copy()
    o = np.nonzero(t == 0)[0]
    t[o[::3]] = 2
    s = dataclasses.replace(s, type=t)
    sig = np.array([0.3166, 0.0, 0.34])
    eps = np.array([0.650, 0.0, 0.45])
    c6 = np.zeros(9, dtype=np.float32)
    c12 = np.zeros(9, dtype=np.float32)
    for a in range(3):
        for b in range(3):
            sg = 0.5 * (sig[a] + sig[b])
            ep = np.sqrt(eps[a] * eps[b])
            c6[3 * a + b] = 4 * ep * sg**6
            c12[3 * a + b] = 4 * ep * sg**12
    return s, c6, c12


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_general_lennard_jones_table(ctx, coul):
    """A type-pair table that is not one parameter pair: the force kernel's
    table lookup, against the oracle."""
    s, c6, c12 = _three_type_box(seed=1)
    p = wb.Params(coul=coul, ntypes=3, c6=c6, c12=c12)
    f, e, v, _ = gpu_eval(ctx, s, p)
    _check(s, p, f, e, v)


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_lennard_jones_weights_match_the_table(ctx, coul):
    """Water (Lennard-Jones on oxygen only) takes the force kernel's weight
    path; the same water with an unused third type whose own pair is nonzero
    (so that the table is no longer one parameter pair) takes the table path.
    The pair terms are the same floats (Ewald adds one term in another
    order), so the forces agree to the rounding of their float atomic sums,
    whose order differs from run to run."""
    s = wb.small_box(seed=1)
    p = wb.Params(coul=coul)
    f1, e1, v1, _ = gpu_eval(ctx, s, p, flags=nb.NB_F_VIRIAL)
    c6 = np.zeros(9, dtype=np.float32)
    c12 = np.zeros(9, dtype=np.float32)
    c6[0], c12[0] = p.c6[0], p.c12[0]
    c6[8], c12[8] = 1e-3, 1e-6  # type 2: no atom has it
    q = wb.Params(coul=coul, ntypes=3, c6=c6, c12=c12)
    f2, e2, v2, _ = gpu_eval(ctx, s, q, flags=nb.NB_F_VIRIAL)
    assert rel_rms(f1, f2) <= 1e-6
    assert np.abs(v1 - v2).max() <= 1e-6 * np.linalg.norm(v1)
