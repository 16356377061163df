"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes one part of the oracle to something independent: a closed
form with a known value, a tabulated function, a conservation law, a
symmetry, a finite difference of the oracle's own energy (which ties the
force and virial code paths to the energy code path), or a brute-force
enumeration of all 27 periodic images.  A dropped term, a wrong sign, a
wrong factor or a broken minimum image in oracle/nb_oracle.c fails at least
one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1506_00716_gb300 import waterbox as wb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def _system(x, q, typ, L, excl=None):
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if excl is None:
        ei = np.zeros(n + 1, dtype=np.int32)
        ea = np.zeros(0, dtype=np.int32)
    else:
        ei, ea = excl
    return wb.System(x=x, q=np.asarray(q, dtype=np.float64), type=np.asarray(typ, dtype=np.int32),
                     box=np.array([L, L, L], dtype=np.float64), excl_index=ei, excl_atoms=ea,
                     n_mol=0, seed=0)


def _lj_params(coul=wb.COUL_RF, **kw):
    s, e = wb.SIGMA_O, wb.EPS_O
    c6 = np.array([4 * e * s**6, 0, 0, 0], dtype=np.float64)
    c12 = np.array([4 * e * s**12, 0, 0, 0], dtype=np.float64)
    return wb.Params(coul=coul, c6=c6, c12=c12, **kw)


def _two(r, q1=0.0, q2=0.0, t1=0, t2=0, L=5.0):
    return _system([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]], [q1, q2], [t1, t2], L)


# ---------------------------------------------------------------- closed forms

def test_lj_special_points():
    p = _lj_params()
    for r_s, v_e, f_se in _golden("lj_points.txt"):
        r = float(r_s) * wb.SIGMA_O
        sys = _two(r)
        ev = oracle.energy_virial(sys, p)
        assert ev["e_lj"] == pytest.approx(float(v_e) * wb.EPS_O, abs=1e-12)
        assert ev["e_coul"] == 0.0
        f = oracle.forces(sys, p)
        # force on atom 0 points away from atom 1 (along -x) when repulsive
        fr = -f[0, 0]
        assert fr == pytest.approx(float(f_se) * wb.EPS_O / wb.SIGMA_O, abs=1e-9)
        assert f[1, 0] == pytest.approx(-f[0, 0], abs=1e-12)


def test_erfc_table_and_ewald_pair():
    p = _lj_params(coul=wb.COUL_EWALD, beta=3.12)
    for x_s, erfc_s in _golden("erfc_table.txt"):
        x, ref = float(x_s), float(erfc_s)
        assert math.erfc(x) == pytest.approx(ref, rel=1e-14)
        r = x / p.beta
        sys = _two(r, q1=1.0, q2=-1.0, t1=1, t2=1)
        ev = oracle.energy_virial(sys, p)
        expect = -wb.ONE_4PI_EPS0 * ref / r
        assert ev["e_coul"] == pytest.approx(expect, rel=1e-13)


def test_rf_constants_from_energies():
    """k_rf and c_rf recovered from two pair energies match the closed forms."""
    g = {k: float(v) for k, v in _golden("rf_constants.txt")}
    p = _lj_params(coul=wb.COUL_RF, eps_rf=78.0, rc=1.0)
    vals = []
    for r in (0.4, 0.8):
        ev = oracle.energy_virial(_two(r, 1.0, 1.0, 1, 1), p)
        vals.append(ev["e_coul"] / wb.ONE_4PI_EPS0 - 1.0 / r)  # = k r^2 - c
    k = (vals[1] - vals[0]) / (0.8**2 - 0.4**2)
    c = k * 0.4**2 - vals[0]
    assert k == pytest.approx(g["k_rf"], rel=1e-12)
    assert c == pytest.approx(g["c_rf"], rel=1e-12)


def test_rf_is_zero_at_cutoff_and_conducting_force_vanishes():
    p = _lj_params(coul=wb.COUL_RF, eps_rf=78.0, rc=1.0)
    ev = oracle.energy_virial(_two(1.0 - 1e-9, 1.0, 1.0, 1, 1), p)
    assert abs(ev["e_coul"]) < 1e-6
    pc = _lj_params(coul=wb.COUL_RF, eps_rf=0.0, rc=1.0)  # eps_rf = infinity
    f = oracle.forces(_two(1.0 - 1e-9, 1.0, 1.0, 1, 1), pc)
    assert abs(f[0, 0]) < 1e-6
    # eps_rf = eps_r reduces to the cut-off-shifted Coulomb law f q q (1/r - 1/rc)
    pp = _lj_params(coul=wb.COUL_RF, eps_rf=1.0, rc=1.0)
    ev = oracle.energy_virial(_two(0.5, 1.0, 1.0, 1, 1), pp)
    assert ev["e_coul"] == pytest.approx(wb.ONE_4PI_EPS0 * (2.0 - 1.0), rel=1e-13)
    f = oracle.forces(_two(0.5, 1.0, 1.0, 1, 1), pp)
    assert -f[0, 0] == pytest.approx(wb.ONE_4PI_EPS0 / 0.25, rel=1e-13)


def test_cutoff_is_strict_and_minimum_image():
    p = _lj_params(coul=wb.COUL_RF, rc=1.0)
    L = 5.0
    # across the periodic boundary: separation 0.3 through the box face
    sys = _system([[0.1, 2.0, 2.0], [L - 0.2, 2.0, 2.0]], [0.0, 0.0], [0, 0], L)
    ev = oracle.energy_virial(sys, p)
    s, e = wb.SIGMA_O, wb.EPS_O
    assert ev["e_lj"] == pytest.approx(4 * e * ((s / 0.3) ** 12 - (s / 0.3) ** 6), rel=1e-10)
    f = oracle.forces(sys, p)
    assert f[0, 0] > 0  # repulsion pushes atom 0 away from its image neighbour at -0.2
    # exactly at rc (representable separation) there is no interaction
    sys = _system([[1.0, 2.0, 2.0], [2.0, 2.0, 2.0]], [1.0, 1.0], [0, 0], L)
    ev = oracle.energy_virial(sys, p)
    assert ev["npairs"] == 0 and ev["e_lj"] == 0.0 and ev["e_coul"] == 0.0


def test_excluded_pairs_contribute_nothing():
    box = wb.water_box(1, 3.0, seed=7)
    for coul in (wb.COUL_RF, wb.COUL_EWALD):
        p = wb.Params(coul=coul)
        ev = oracle.energy_virial(box, p)
        assert ev["npairs"] == 0 and ev["e_lj"] == 0.0 and ev["e_coul"] == 0.0
        assert np.all(oracle.forces(box, p) == 0.0)


# --------------------------------------------------- potential modifiers

def test_lj_potential_shift():
    p0 = _lj_params()
    p1 = _lj_params(modifiers=oracle.MOD_LJ_SHIFT)
    c6, c12, rc = p0.c6[0], p0.c12[0], p0.rc
    v_rc = c12 / rc**12 - c6 / rc**6  # the unshifted pair energy at the cut-off
    for r in (0.3, 0.5, 0.9):
        s = _two(r)
        e0, e1 = oracle.energy_virial(s, p0), oracle.energy_virial(s, p1)
        assert e1["e_lj"] == pytest.approx(e0["e_lj"] - v_rc, rel=1e-12, abs=1e-15)
        assert np.array_equal(oracle.forces(s, p0), oracle.forces(s, p1))
        assert np.array_equal(e0["virial"], e1["virial"])
    # the shifted potential is continuous at the cut-off
    assert abs(oracle.energy_virial(_two(rc - 1e-7), p1)["e_lj"]) < 1e-8
    assert oracle.energy_virial(_two(rc + 1e-7), p1)["e_lj"] == 0.0


def test_ewald_potential_shift():
    zero = np.zeros(4)
    p0 = wb.Params(coul=wb.COUL_EWALD, c6=zero, c12=zero)
    p1 = wb.Params(coul=wb.COUL_EWALD, c6=zero, c12=zero, modifiers=oracle.MOD_EWALD_SHIFT)
    q1, q2 = 0.6, -0.9
    shift = p0.fcoul * q1 * q2 * math.erfc(p0.beta * p0.rc) / p0.rc
    for r in (0.2, 0.6, 0.95):
        s = _two(r, q1, q2)
        e0, e1 = oracle.energy_virial(s, p0), oracle.energy_virial(s, p1)
        assert e1["e_coul"] == pytest.approx(e0["e_coul"] - shift, rel=1e-12, abs=1e-15)
        assert np.array_equal(oracle.forces(s, p0), oracle.forces(s, p1))
    assert abs(oracle.energy_virial(_two(p0.rc - 1e-7, q1, q2), p1)["e_coul"]) < 1e-7
    # the modifier leaves reaction field alone
    prf = wb.Params(c6=zero, c12=zero, modifiers=oracle.MOD_EWALD_SHIFT)
    s = _two(0.4, q1, q2)
    assert oracle.energy_virial(s, prf)["e_coul"] == oracle.energy_virial(s, wb.Params(c6=zero, c12=zero))["e_coul"]


def test_rf_exclusion_correction():
    zero = np.zeros(4)
    p = wb.Params(c6=zero, c12=zero, modifiers=oracle.MOD_RF_EXCL)
    q1, q2 = 0.6, -0.9
    rc, er, erf = p.rc, p.eps_r, p.eps_rf
    krf = (erf - er) / ((2 * erf + er) * rc**3)
    crf = 1 / rc + krf * rc**2
    excl = (np.array([0, 1, 2], dtype=np.int32), np.array([1, 0], dtype=np.int32))
    for r, inside in ((0.1, True), (0.97, True), (1.2, False)):
        s = _system([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]], [q1, q2], [0, 0], 5.0, excl)
        ev = oracle.energy_virial(s, p)
        f = oracle.forces(s, p)
        if inside:
            assert ev["e_coul"] == pytest.approx(p.fcoul * q1 * q2 * (krf * r * r - crf), rel=1e-13)
            # F_i = -dV/dx_i with V = f q1 q2 (k_rf r^2 - c_rf): -2 f q1 q2 k_rf (x_i - x_j)
            assert f[0, 0] == pytest.approx(2 * p.fcoul * q1 * q2 * krf * r, rel=1e-13)
            assert f[1, 0] == pytest.approx(-f[0, 0], rel=1e-15)
            # virial -1/2 d (x) F: xx = -1/2 (-r) (2 f qq k_rf r)
            assert ev["virial"][0, 0] == pytest.approx(p.fcoul * q1 * q2 * krf * r * r, rel=1e-13)
        else:
            assert ev["e_coul"] == 0.0 and np.all(f == 0.0)
        assert ev["npairs"] == 0  # excluded pairs are not interacting pairs
        # without the modifier the excluded pair contributes nothing
        s0 = oracle.energy_virial(s, wb.Params(c6=zero, c12=zero))
        assert s0["e_coul"] == 0.0


@pytest.mark.parametrize("mods,coul", [(1 | 4, wb.COUL_RF), (1 | 2, wb.COUL_EWALD)])
def test_modified_forces_are_minus_energy_gradient(mods, coul):
    sys = wb.small_box(seed=15)
    sys.x = sys.x.astype(np.float64)
    p = wb.Params(coul=coul, modifiers=mods)
    f = oracle.forces(sys, p)
    assert np.abs(f.sum(0)).max() <= 1e-9 * np.abs(f).sum()
    rng = np.random.default_rng(1)
    h = 1e-6
    checked = 0
    for a in rng.choice(sys.n, size=6, replace=False):
        for d in range(3):
            xp, xm = sys.x.copy(), sys.x.copy()
            xp[a, d] += h
            xm[a, d] -= h
            sp = wb.System(**{**sys.__dict__}); sp.x = xp
            sm = wb.System(**{**sys.__dict__}); sm.x = xm
            ep, npp = _etot(sp, p)
            em, nm = _etot(sm, p)
            if npp != nm:
                continue
            assert -(ep - em) / (2 * h) == pytest.approx(f[a, d], rel=2e-6, abs=2e-4)
            checked += 1
    assert checked >= 12


# ------------------------------------------------------ laws and symmetries

@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_newton_third_law(coul):
    sys = wb.small_box(seed=11)
    p = wb.Params(coul=coul)
    f = oracle.forces(sys, p)
    net = np.abs(f.sum(axis=0)).max()
    assert net <= 1e-10 * np.abs(f).sum()


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_translation_invariance(coul):
    sys = wb.small_box(seed=12)
    p = wb.Params(coul=coul)
    ev0, f0, pr0 = oracle.energy_virial(sys, p), oracle.forces(sys, p), oracle.pairs(sys, p.rc)
    L = float(sys.box[0])
    shift = np.array([0.731, -1.377, 2.113])
    moved = wb.System(**{**sys.__dict__})
    moved.x = np.mod(sys.x.astype(np.float64) + shift, L)
    ev1, f1, pr1 = oracle.energy_virial(moved, p), oracle.forces(moved, p), oracle.pairs(moved, p.rc)
    assert np.array_equal(pr0, pr1)
    for k in ("e_lj", "e_coul"):
        assert ev1[k] == pytest.approx(ev0[k], rel=1e-11)
    assert np.abs(f1 - f0).max() <= 1e-9 * np.abs(f0).max()


def test_axis_permutation():
    sys = wb.small_box(seed=13)
    p = wb.Params(coul=wb.COUL_RF)
    perm = [2, 0, 1]
    ev0, f0 = oracle.energy_virial(sys, p), oracle.forces(sys, p)
    rot = wb.System(**{**sys.__dict__})
    rot.x = sys.x[:, perm].copy()
    ev1, f1 = oracle.energy_virial(rot, p), oracle.forces(rot, p)
    assert ev1["e_lj"] == pytest.approx(ev0["e_lj"], rel=1e-12)
    assert ev1["e_coul"] == pytest.approx(ev0["e_coul"], rel=1e-12)
    assert np.abs(f1 - f0[:, perm]).max() <= 1e-10 * np.abs(f0).max()
    v0, v1 = ev0["virial"], ev1["virial"]
    assert np.abs(v1 - v0[np.ix_(perm, perm)]).max() <= 1e-10 * np.abs(v0).max()


# ----------------------------------------------------- finite differences

def _etot(sys, p):
    ev = oracle.energy_virial(sys, p)
    return ev["e_lj"] + ev["e_coul"], ev["npairs"]


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_forces_are_minus_energy_gradient(coul):
    sys = wb.small_box(seed=14)
    sys.x = sys.x.astype(np.float64)
    p = wb.Params(coul=coul)
    f = oracle.forces(sys, p)
    rng = np.random.default_rng(0)
    h = 1e-6
    checked = 0
    for a in rng.choice(sys.n, size=8, replace=False):
        for d in range(3):
            xp, xm = sys.x.copy(), sys.x.copy()
            xp[a, d] += h
            xm[a, d] -= h
            sp = wb.System(**{**sys.__dict__}); sp.x = xp
            sm = wb.System(**{**sys.__dict__}); sm.x = xm
            ep, npp = _etot(sp, p)
            em, nm = _etot(sm, p)
            if npp != nm:
                continue  # a pair crossed the cut-off: the energy jumps there
            fd = -(ep - em) / (2 * h)
            assert fd == pytest.approx(f[a, d], rel=2e-6, abs=2e-4)
            checked += 1
    assert checked >= 20


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_virial_from_box_deformation(coul):
    """2 Xi_ab = dE/d(eps) for x_a -> x_a + eps x_b (box deformed with the atoms).

    Diagonal components use a periodic water box scaled along one axis;
    off-diagonal ones use an isolated cluster (no pair crosses the box) that
    is sheared in place.
    """
    p = wb.Params(coul=coul)
    h = 1e-7
    sys = wb.small_box(seed=15)
    sys.x = sys.x.astype(np.float64)
    xi = oracle.energy_virial(sys, p)["virial"]
    for a in range(3):
        es = []
        for sgn in (+1, -1):
            s2 = wb.System(**{**sys.__dict__})
            scale = np.ones(3)
            scale[a] += sgn * h
            s2.x = sys.x * scale
            s2.box = sys.box * scale
            es.append(_etot(s2, p))
        assert es[0][1] == es[1][1]
        dE = (es[0][0] - es[1][0]) / (2 * h)
        assert dE == pytest.approx(2 * xi[a, a], rel=1e-5)
    # isolated cluster of molecules in a large box for the shear components
    cl = wb.water_box(64, 1.25, seed=16)
    big = wb.System(**{**cl.__dict__})
    big.x = cl.x.astype(np.float64) + 3.0
    big.box = np.array([9.0, 9.0, 9.0])
    xi = oracle.energy_virial(big, p)["virial"]
    for a, b in ((0, 1), (0, 2), (1, 2), (1, 0)):
        es = []
        for sgn in (+1, -1):
            s2 = wb.System(**{**big.__dict__})
            x2 = big.x.copy()
            x2[:, a] += sgn * h * (big.x[:, b] - 3.0)
            s2.x = x2
            es.append(_etot(s2, p))
        assert es[0][1] == es[1][1]
        dE = (es[0][0] - es[1][0]) / (2 * h)
        assert dE == pytest.approx(2 * xi[a, b], rel=1e-5, abs=1e-3)


def test_virial_identities():
    sys = wb.small_box(seed=17)
    p = wb.Params(coul=wb.COUL_RF)
    ev = oracle.energy_virial(sys, p)
    # for V = c12 r^-12 - c6 r^-6 the pair virial r.F equals 12 V12 - 6 V6
    assert ev["rdotf_lj"] == pytest.approx(12 * ev["e12"] - 6 * ev["e6"], rel=1e-12)
    assert ev["e_lj"] == pytest.approx(ev["e12"] - ev["e6"], rel=1e-12)
    tr = np.trace(ev["virial"])
    assert tr == pytest.approx(-0.5 * (ev["rdotf_lj"] + ev["rdotf_coul"]), rel=1e-12)
    assert np.allclose(ev["virial"], ev["virial"].T, rtol=0, atol=1e-12 * np.abs(tr))


# ------------------------------------------------------ brute-force pair set

def _pairs_27_images(sys, r_cut):
    """All non-excluded pairs i<j with some periodic image closer than r_cut."""
    x = sys.x.astype(np.float64)
    L = sys.box
    n = sys.n
    excl = set()
    for i in range(n):
        for k in range(sys.excl_index[i], sys.excl_index[i + 1]):
            j = int(sys.excl_atoms[k])
            excl.add((min(i, j), max(i, j)))
    best = np.full((n, n), np.inf)
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                d = x[:, None, :] - x[None, :, :] + np.array([sx, sy, sz]) * L
                best = np.minimum(best, (d * d).sum(-1))
    ii, jj = np.nonzero(np.triu(best < r_cut * r_cut, k=1))
    keys = [i * n + j for i, j in zip(ii.tolist(), jj.tolist()) if (i, j) not in excl]
    return np.array(sorted(keys), dtype=np.int64)


@pytest.mark.parametrize("seed", [21, 22])
def test_pair_set_matches_27_image_enumeration(seed):
    sys = wb.water_box(120, 2.3, seed=seed)
    for r_cut in (1.0, 1.1):
        assert np.array_equal(oracle.pairs(sys, r_cut), _pairs_27_images(sys, r_cut))


def test_pair_count_matches_density_estimate():
    """Half-pairs within rc of a uniform fluid are about N rho (4/3) pi rc^3 / 2."""
    sys = wb.small_box(seed=23)
    n_pairs = oracle.pairs(sys, 1.0).shape[0]
    rho = sys.n / float(sys.box[0]) ** 3
    est = sys.n * rho * 4.0 / 3.0 * math.pi / 2.0
    assert abs(n_pairs - est) / est < 0.02


# ------------------------------------------------------------ triclinic boxes

def _lattice_images(sys, r_cut, reach=2):
    """All non-excluded pairs i<j with some image under the lattice rows
    a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz) closer than r_cut, by brute
    force over |i|, |j|, |k| <= reach."""
    x = sys.x.astype(np.float64)
    ax, by, cz = sys.box
    bx, cx, cy = sys.skew
    a, b, c = np.array([ax, 0, 0]), np.array([bx, by, 0]), np.array([cx, cy, cz])
    n = sys.n
    excl = set()
    for i in range(n):
        for k in range(sys.excl_index[i], sys.excl_index[i + 1]):
            j = int(sys.excl_atoms[k])
            excl.add((min(i, j), max(i, j)))
    best = np.full((n, n), np.inf)
    rng = range(-reach, reach + 1)
    for i in rng:
        for j in rng:
            for k in rng:
                d = x[:, None, :] - x[None, :, :] + i * a + j * b + k * c
                best = np.minimum(best, (d * d).sum(-1))
    ii, jj = np.nonzero(np.triu(best < r_cut * r_cut, k=1))
    keys = [i * n + j for i, j in zip(ii.tolist(), jj.tolist()) if (i, j) not in excl]
    return np.array(sorted(keys), dtype=np.int64)


def test_triclinic_pair_set_matches_lattice_enumeration():
    sys = wb.rhombic_dodecahedron_box(120, seed=31)
    assert sys.skew[1] > 0 and sys.skew[2] > 0
    for r_cut in (1.0, 1.1):
        assert np.array_equal(oracle.pairs(sys, r_cut), _lattice_images(sys, r_cut))


def _rows_of(keys, n, sel):
    a, b = keys // n, keys % n
    return keys[np.isin(a, sel) | np.isin(b, sel)]


@pytest.mark.parametrize("seed", [21, 22])
def test_pairs_of_rows_are_rows_of_the_27_image_enumeration(seed):
    """The row-wise pair oracle (O(N) per selected atom, for boxes where the
    whole set is out of reach) against the brute-force enumeration: every
    pair touching a selected atom, and with all atoms selected the whole set."""
    sys = wb.water_box(120, 2.3, seed=seed)
    rng = np.random.default_rng(seed)
    for r_cut in (1.0, 1.1):
        ref = _pairs_27_images(sys, r_cut)
        sel = np.sort(rng.choice(sys.n, size=37, replace=False)).astype(np.int32)
        assert np.array_equal(oracle.pairs_of_rows(sys, r_cut, sel), _rows_of(ref, sys.n, sel))
        allrows = oracle.pairs_of_rows(sys, r_cut, np.arange(sys.n, dtype=np.int32))
        assert np.array_equal(allrows, ref)


def test_triclinic_pairs_of_rows_match_lattice_enumeration():
    sys = wb.rhombic_dodecahedron_box(120, seed=31)
    ref = _lattice_images(sys, 1.0)
    sel = np.arange(0, sys.n, 7, dtype=np.int32)
    assert np.array_equal(oracle.pairs_of_rows(sys, 1.0, sel), _rows_of(ref, sys.n, sel))


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_rectangular_lattice_in_triclinic_form(coul):
    """The rectangular lattice written with other rows (b' = a + b,
    c' = a + b + c) is the same lattice: the triclinic reduction must give
    the rectangular results."""
    sys = wb.small_box(seed=32)
    p = wb.Params(coul=coul)
    L = float(sys.box[0])
    ev0, f0 = oracle.energy_virial(sys, p), oracle.forces(sys, p)
    for skew in ([L, 0.0, 0.0], [0.0, L, L], [L, L, L]):
        tri = wb.System(**{**sys.__dict__, "skew": np.array(skew)})
        ev1, f1 = oracle.energy_virial(tri, p), oracle.forces(tri, p)
        assert ev1["npairs"] == ev0["npairs"]
        for k in ("e_lj", "e_coul"):
            assert ev1[k] == pytest.approx(ev0[k], rel=1e-12)
        assert np.abs(f1 - f0).max() <= 1e-10 * np.abs(f0).max()
        assert np.abs(ev1["virial"] - ev0["virial"]).max() <= 1e-10 * np.abs(ev0["virial"]).max()


@pytest.mark.parametrize("coul", [wb.COUL_RF, wb.COUL_EWALD])
def test_triclinic_translation_newton_and_gradient(coul):
    sys = wb.rhombic_dodecahedron_box(600, seed=33)
    sys.x = sys.x.astype(np.float64)
    p = wb.Params(coul=coul)
    ev0, f0, pr0 = oracle.energy_virial(sys, p), oracle.forces(sys, p), oracle.pairs(sys, p.rc)
    assert np.abs(f0.sum(0)).max() <= 1e-9 * np.abs(f0).sum()
    # translation (wrapped back into the cell with the lattice rows)
    moved = wb.System(**{**sys.__dict__})
    moved.x = wb.wrap_triclinic32(sys.x + np.array([1.37, -0.81, 2.9]), sys.box, sys.skew).astype(np.float64)
    shifted_back = moved.x - sys.x
    # the moved coordinates differ from x + t by lattice vectors and float32 rounding
    assert np.abs(shifted_back).max() > 0
    ev1 = oracle.energy_virial(moved, p)
    assert ev1["e_lj"] + ev1["e_coul"] == pytest.approx(ev0["e_lj"] + ev0["e_coul"], rel=1e-5)
    # forces are minus the energy gradient
    rng = np.random.default_rng(3)
    h = 1e-6
    checked = 0
    for a in rng.choice(sys.n, size=6, replace=False):
        for d in range(3):
            xp, xm = sys.x.copy(), sys.x.copy()
            xp[a, d] += h
            xm[a, d] -= h
            sp = wb.System(**{**sys.__dict__}); sp.x = xp
            sm = wb.System(**{**sys.__dict__}); sm.x = xm
            ep, npp = _etot(sp, p)
            em, nm = _etot(sm, p)
            if npp != nm:
                continue
            assert -(ep - em) / (2 * h) == pytest.approx(f0[a, d], rel=2e-6, abs=2e-4)
            checked += 1
    assert checked >= 12


def test_energy_virial_row_ranges_add_up_to_all_pairs():
    """The row-range sums (used to take the 3M-atom golden sums in pieces)
    cover every pair once: consecutive ranges add up to the full sums."""
    s = wb.small_box(seed=2)
    p = wb.params_ewald()
    full = oracle.energy_virial(s, p)
    cuts = [0, 1, 100, s.n // 2, s.n - 1, s.n]
    sums = np.zeros(15)
    npairs = 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        out, k = oracle.energy_virial_rows(s, p, a, b)
        sums += out
        npairs += k
    ev = oracle.ev_from_sums(sums, npairs)
    assert ev["npairs"] == full["npairs"]
    for key in ("e_lj", "e_coul", "e12", "e6"):
        assert abs(ev[key] - full[key]) <= 1e-12 * abs(full[key])
    assert np.allclose(ev["virial"], full["virial"], rtol=1e-12, atol=1e-9)
    with pytest.raises(RuntimeError):
        oracle.energy_virial_rows(s, p, 5, 3)
