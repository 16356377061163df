"""Pins of the long-range (PME) oracle against facts that do not come from it.

- The Madelung constant of rock salt: the real-space sum (written out here
  over explicit images), the oracle's exact reciprocal sum and its self term
  add up to the lattice energy of NaCl.
- A neutral pair of molecules far from its images: real space + reciprocal +
  self + excluded-pair correction equals the plain Coulomb energy and forces
  between the two molecules (up to the image dipole terms, O(mu^2 / L^3)).
- Coulomb's homogeneity: for the full Ewald sum, trace(virial) = -E / 2.
- Box deformation: each virial component of the reciprocal sum against a
  central difference of the reciprocal energy of the deformed (also sheared,
  triclinic) box; the sheared energy is written out here, not taken from the
  oracle.
- Smooth PME against the exact sum: the error falls as the grid refines and
  the spline order rises; PME forces are minus the gradient of PME energy.
- B-splines: partition of unity, the order-4 values at the integers, and the
  derivative relation.
"""
import math

import numpy as np
import pytest
from scipy.special import erfc, erf

from oracle import pme as opme
from paper_1506_00716_gb300 import waterbox as wb

MADELUNG_NACL = 1.747564594633182  # rock salt, per ion pair, in units of q^2 / d


def _system(x, q, L, excl=None):
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if excl is None:
        ei, ea = np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32)
    else:
        ei, ea = excl
    Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
    return wb.System(x=x, q=np.asarray(q, dtype=np.float64), type=np.zeros(n, dtype=np.int32), box=Lv,
                     excl_index=ei, excl_atoms=ea, n_mol=0, seed=0)


def _real_space(sys, p, r_cut, skip_excluded=True):
    """sum over pairs and periodic images of f qi qj erfc(beta r) / r within r_cut,
    with forces and the virial -1/2 sum d (x) F; written out over images."""
    x = sys.x.astype(np.float64)
    q = sys.q.astype(np.float64)
    L = sys.box
    f = p.fcoul / p.eps_r
    n = x.shape[0]
    excl = np.zeros((n, n), dtype=bool)
    for i in range(n):
        excl[i, sys.excl_atoms[sys.excl_index[i]:sys.excl_index[i + 1]]] = True
    reach = [int(math.ceil(r_cut / L[d])) + 1 for d in range(3)]
    e = 0.0
    F = np.zeros_like(x)
    W = np.zeros((3, 3))
    d0 = x[:, None, :] - x[None, :, :]
    for sx in range(-reach[0], reach[0] + 1):
        for sy in range(-reach[1], reach[1] + 1):
            for sz in range(-reach[2], reach[2] + 1):
                S = np.array([sx, sy, sz]) * L
                d = d0 + S
                r = np.sqrt((d * d).sum(-1))
                use = r < r_cut
                if sx == 0 and sy == 0 and sz == 0:
                    use &= ~np.eye(n, dtype=bool)
                    if skip_excluded:
                        use &= ~excl
                rr = np.where(use, r, 1.0)
                qq = f * q[:, None] * q[None, :]
                v = np.where(use, qq * erfc(p.beta * rr) / rr, 0.0)
                fr = np.where(use, qq * (erfc(p.beta * rr) / rr
                                         + 2 * p.beta / math.sqrt(math.pi) * np.exp(-(p.beta * rr) ** 2)) / rr ** 2, 0.0)
                e += 0.5 * v.sum()
                F += (fr[:, :, None] * d).sum(1)
                W += -0.25 * np.einsum("ij,ija,ijb->ab", fr, d, d)
    return e, F, W


def _nacl(cells, d):
    a = 2 * d
    base = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [0, 1, 1]], dtype=np.float64) * d
    na, cl = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                o = np.array([i, j, k]) * a
                na.extend(o + base)
                cl.extend(o + base + np.array([d, 0, 0]))
    x = np.array(na + cl) + 0.013
    q = np.array([1.0] * len(na) + [-1.0] * len(cl))
    return _system(x, q, cells * a)


def test_madelung_constant_of_rock_salt():
    d = 0.282
    sys = _nacl(2, d)
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    e_real, _, _ = _real_space(sys, p, r_cut=2.0)
    e_rec = opme.ewald_reciprocal_direct(sys, p, kmax=10)["energy"]
    e_self = opme.ewald_self(sys, p)
    n_pairs = sys.n // 2
    expect = -n_pairs * MADELUNG_NACL * p.fcoul / d
    assert e_real + e_rec + e_self == pytest.approx(expect, rel=1e-10)
    # the split does not depend on beta
    p2 = wb.Params(coul=wb.COUL_EWALD, beta=4.0)
    e2 = _real_space(sys, p2, r_cut=1.6)[0] + opme.ewald_reciprocal_direct(sys, p2, kmax=12)["energy"] + \
        opme.ewald_self(sys, p2)
    assert e2 == pytest.approx(expect, rel=1e-10)


def test_virial_trace_of_full_ewald_sum():
    rng = np.random.default_rng(3)
    n = 24
    L = 1.4
    x = rng.uniform(0, L, size=(n, 3))
    q = rng.normal(size=n)
    q -= q.mean()
    sys = _system(x, q, L)
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    e_real, f_real, w_real = _real_space(sys, p, r_cut=2.0)
    rec = opme.ewald_reciprocal_direct(sys, p, kmax=10)
    e = e_real + rec["energy"] + opme.ewald_self(sys, p)
    assert np.trace(w_real + rec["virial"]) == pytest.approx(-0.5 * e, rel=1e-9)
    # the total force is zero (a momentum check on the reciprocal forces)
    assert np.abs(rec["forces"].sum(0)).max() < 1e-9 * np.abs(rec["forces"]).max()


def _two_waters():
    w = wb.water_box(2, 1.0, seed=5)
    x = w.x.astype(np.float64)
    # molecule 2 moved 0.31 nm from molecule 1's oxygen, both in the middle of a 7 nm box
    x[3:] += (x[0] + np.array([0.31, 0.05, -0.02])) - x[3]
    x += 3.5 - x.mean(0)
    return _system(x, w.q, 7.0, (w.excl_index, w.excl_atoms))


def test_excluded_pair_correction_recovers_plain_coulomb():
    sys = _two_waters()
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    e_real, f_real, _ = _real_space(sys, p, r_cut=1.9)
    rec = opme.ewald_reciprocal_direct(sys, p, kmax=24)
    ex = opme.ewald_exclusions(sys, p)
    e = e_real + rec["energy"] + opme.ewald_self(sys, p) + ex["energy"]
    fe = f_real + rec["forces"] + ex["forces"]
    # plain Coulomb between the two molecules, no images
    f = p.fcoul
    e_ref = 0.0
    f_ref = np.zeros_like(sys.x)
    for i in range(3):
        for j in range(3, 6):
            dv = sys.x[i] - sys.x[j]
            r = np.linalg.norm(dv)
            e_ref += f * sys.q[i] * sys.q[j] / r
            fij = f * sys.q[i] * sys.q[j] / r ** 3 * dv
            f_ref[i] += fij
            f_ref[j] -= fij
    assert abs(e_ref) > 5.0
    assert e == pytest.approx(e_ref, abs=2e-3)
    assert np.abs(fe - f_ref).max() < 2e-3 * np.abs(f_ref).max()
    # without the correction it is far off
    assert abs(e - ex["energy"] - e_ref) > 100.0


def test_exclusion_forces_are_minus_gradient():
    sys = _two_waters()
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    ex = opme.ewald_exclusions(sys, p)
    h = 1e-6
    for a in range(sys.n):
        for d in range(3):
            sp, sm = _system(sys.x.copy(), sys.q, sys.box, (sys.excl_index, sys.excl_atoms)), \
                _system(sys.x.copy(), sys.q, sys.box, (sys.excl_index, sys.excl_atoms))
            sp.x[a, d] += h
            sm.x[a, d] -= h
            fd = -(opme.ewald_exclusions(sp, p)["energy"] - opme.ewald_exclusions(sm, p)["energy"]) / (2 * h)
            assert fd == pytest.approx(ex["forces"][a, d], rel=1e-6, abs=1e-5)
    # Xi = -1/2 sum d (x) F: the pair form against the atom form with a common origin
    w = -0.5 * np.einsum("ia,ib->ab", sys.x, ex["forces"])
    assert np.allclose(w, ex["virial"], atol=1e-9 * np.abs(w).max())


def _rec_energy_triclinic(x, q, rows, p, kmax):
    """Exact reciprocal energy for the lattice with rows a, b, c (written out
    here): m = k B^-T over the integer vectors k, V = det B."""
    B = np.asarray(rows, dtype=np.float64)
    V = abs(np.linalg.det(B))
    Binv_T = np.linalg.inv(B).T
    k = np.arange(-kmax, kmax + 1)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    K = K[np.any(K != 0, axis=1)]
    m = K @ Binv_T
    m2 = (m * m).sum(1)
    S = np.exp(2j * np.pi * (x @ m.T)) .T @ q
    f = p.fcoul / p.eps_r
    return float((f / (2 * np.pi * V) * np.exp(-np.pi ** 2 * m2 / p.beta ** 2) / m2 * np.abs(S) ** 2).sum())


def test_reciprocal_virial_from_box_deformation():
    rng = np.random.default_rng(8)
    n = 18
    L = np.array([1.3, 1.5, 1.4])
    x = rng.uniform(0, 1, size=(n, 3)) * L
    q = rng.normal(size=n)
    q -= q.mean()
    sys = _system(x, q, L)
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    rec = opme.ewald_reciprocal_direct(sys, p, kmax=10)
    e0 = _rec_energy_triclinic(x, q, np.diag(L), p, 10)
    assert e0 == pytest.approx(rec["energy"], rel=1e-12)
    h = 1e-6
    for a in range(3):
        for b in range(3):
            es = []
            for sgn in (+1, -1):
                D = np.eye(3)
                D[a, b] += sgn * h           # x_a -> x_a + eps x_b, for atoms and box rows alike
                es.append(_rec_energy_triclinic(x @ D.T, q, np.diag(L) @ D.T, p, 10))
            dE = (es[0] - es[1]) / (2 * h)
            assert dE == pytest.approx(2 * rec["virial"][a, b], rel=1e-6, abs=1e-6 * abs(e0))


def test_bsplines():
    for p in (3, 4, 5, 6, 8):
        u = np.linspace(0, 1, 17)
        s = sum(opme.bspline(u + j, p) for j in range(p))
        assert np.allclose(s, 1.0, atol=1e-14)
        ds = sum(opme.bspline_deriv(u + j, p) for j in range(p))
        assert np.allclose(ds, 0.0, atol=1e-13)
        # derivative by central difference
        h = 1e-6
        xs = np.linspace(0.1, p - 0.1, 23)
        fd = (opme.bspline(xs + h, p) - opme.bspline(xs - h, p)) / (2 * h)
        assert np.allclose(fd, opme.bspline_deriv(xs, p), atol=1e-8)
    # cubic B-spline at the integers: 1/6, 2/3, 1/6
    assert np.allclose(opme.bspline(np.array([1.0, 2.0, 3.0]), 4), [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    # moduli: B(0) = 1 (the weights sum to 1)
    assert opme.bspline_moduli(16, 4)[0] == pytest.approx(1.0, rel=1e-14)


def _small_neutral_box(seed=21):
    w = wb.water_box(64, 1.25, seed=seed)
    return _system(w.x.astype(np.float64), w.q.astype(np.float64), w.box, (w.excl_index, w.excl_atoms))


def test_pme_converges_to_exact_reciprocal_sum():
    sys = _small_neutral_box()
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    ref = opme.ewald_reciprocal_direct(sys, p, kmax=12)
    fref = np.sqrt((ref["forces"] ** 2).mean())
    errs = []
    for K, order in ((12, 4), (16, 4), (20, 6), (32, 8)):
        r = opme.pme(sys, p, grid=(K, K, K), order=order)
        errs.append((abs(r["energy"] - ref["energy"]) / abs(ref["energy"]),
                     np.sqrt(((r["forces"] - ref["forces"]) ** 2).mean()) / fref,
                     np.abs(r["virial"] - ref["virial"]).max() / np.abs(ref["virial"]).max()))
    errs = np.array(errs)
    assert np.all(np.diff(errs[:, 1]) < 0), errs
    assert errs[0, 1] < 5e-2
    assert errs[-1, 0] < 1e-8 and errs[-1, 1] < 1e-6 and errs[-1, 2] < 1e-6, errs


def test_pme_forces_are_minus_energy_gradient():
    sys = _small_neutral_box(seed=22)
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    r = opme.pme(sys, p, grid=(14, 14, 14), order=6)
    h = 1e-6
    rng = np.random.default_rng(1)
    for a in rng.choice(sys.n, size=5, replace=False):
        for d in range(3):
            es = []
            for sgn in (+1, -1):
                s2 = _system(sys.x.copy(), sys.q, sys.box)
                s2.x[a, d] += sgn * h
                es.append(opme.pme(s2, p, grid=(14, 14, 14), order=6)["energy"])
            fd = -(es[0] - es[1]) / (2 * h)
            assert fd == pytest.approx(r["forces"][a, d], rel=1e-6, abs=1e-5)
    # the PME virial along each axis against scaling the box and the atoms
    for a in range(3):
        es = []
        for sgn in (+1, -1):
            scale = np.ones(3)
            scale[a] += sgn * h
            s2 = _system(sys.x * scale, sys.q, sys.box * scale)
            es.append(opme.pme(s2, p, grid=(14, 14, 14), order=6)["energy"])
        dE = (es[0] - es[1]) / (2 * h)
        # the mesh charges depend on fractional coordinates only, so the PME
        # virial is the exact derivative of the PME energy
        assert dE == pytest.approx(2 * r["virial"][a, a], rel=1e-6, abs=1e-7 * abs(r["energy"]))


# ------------------------------------------------------------ triclinic boxes

def _tri_system(x, q, rows, excl=None):
    rows = np.asarray(rows, dtype=np.float64)
    assert rows[0, 1] == rows[0, 2] == rows[1, 2] == 0.0
    s = _system(x, q, np.array([rows[0, 0], rows[1, 1], rows[2, 2]]), excl)
    s.skew = np.array([rows[1, 0], rows[2, 0], rows[2, 1]])
    return s


def _real_space_lattice(sys, rows, p, r_cut, reach):
    """Real-space Ewald sum over explicit lattice images n1 a + n2 b + n3 c."""
    x = sys.x.astype(np.float64)
    q = sys.q.astype(np.float64)
    f = p.fcoul / p.eps_r
    n = x.shape[0]
    e = 0.0
    d0 = x[:, None, :] - x[None, :, :]
    for n1 in range(-reach, reach + 1):
        for n2 in range(-reach, reach + 1):
            for n3 in range(-reach, reach + 1):
                S = n1 * rows[0] + n2 * rows[1] + n3 * rows[2]
                r = np.sqrt(((d0 + S) ** 2).sum(-1))
                use = r < r_cut
                if n1 == n2 == n3 == 0:
                    use &= ~np.eye(n, dtype=bool)
                rr = np.where(use, r, 1.0)
                e += 0.5 * np.where(use, f * q[:, None] * q[None, :] * erfc(p.beta * rr) / rr, 0.0).sum()
    return e


def _fcc_primitive(d):
    """Rock salt as its two-ion primitive cell: the fcc vectors of cube edge
    2d, rotated into the lower-triangular box form (rows a, b, c)."""
    B0 = d * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    Qm, _ = np.linalg.qr(B0.T)
    rows = B0 @ Qm
    if rows[0, 0] < 0:
        rows[:, 0] *= -1
        Qm[:, 0] *= -1
    if rows[1, 1] < 0:
        rows[:, 1] *= -1
        Qm[:, 1] *= -1
    if rows[2, 2] < 0:
        rows[:, 2] *= -1
        Qm[:, 2] *= -1
    rows[np.abs(rows) < 1e-14] = 0.0
    x = np.array([[0.05, 0.02, 0.03], [0.05 + d, 0.02, 0.03]]) @ Qm
    return rows, x


def test_madelung_constant_in_a_triclinic_cell():
    d = 0.282
    rows, x = _fcc_primitive(d)
    sys = _tri_system(x, [1.0, -1.0], rows)
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    e_real = _real_space_lattice(sys, rows, p, r_cut=2.0, reach=10)
    e_rec = opme.ewald_reciprocal_direct(sys, p, kmax=8)["energy"]
    e_self = opme.ewald_self(sys, p)
    assert e_real + e_rec + e_self == pytest.approx(-MADELUNG_NACL * p.fcoul / d, rel=1e-10)


def test_reciprocal_sum_depends_on_the_lattice_not_the_basis():
    rng = np.random.default_rng(12)
    L = 1.4
    x = rng.uniform(0, L, size=(12, 3))
    q = rng.normal(size=12)
    q -= q.mean()
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    cube = _system(x, q, L)
    sheared = _tri_system(x, q, [[L, 0, 0], [L, L, 0], [L, L, L]])  # the same cubic lattice
    e0 = opme.ewald_reciprocal_direct(cube, p, kmax=10)
    e1 = opme.ewald_reciprocal_direct(sheared, p, kmax=24)
    assert e1["energy"] == pytest.approx(e0["energy"], rel=1e-11)
    assert np.allclose(e1["forces"], e0["forces"], rtol=0, atol=1e-9 * np.abs(e0["forces"]).max())
    assert np.allclose(e1["virial"], e0["virial"], rtol=0, atol=1e-9 * np.abs(e0["virial"]).max())


def _rd_small():
    rd = wb.rhombic_dodecahedron_box(80, seed=9)
    return rd


def test_triclinic_pme_converges_to_the_exact_sum():
    s = _rd_small()
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    ref = opme.ewald_reciprocal_direct(s, p, kmax=12)
    fref = np.sqrt((ref["forces"] ** 2).mean())
    errs = []
    for K, order in ((16, 4), (24, 6), (40, 8)):
        r = opme.pme(s, p, grid=(K, K, K), order=order)
        errs.append((abs(r["energy"] - ref["energy"]) / abs(ref["energy"]),
                     np.sqrt(((r["forces"] - ref["forces"]) ** 2).mean()) / fref,
                     np.abs(r["virial"] - ref["virial"]).max() / np.abs(ref["virial"]).max()))
    errs = np.array(errs)
    assert np.all(np.diff(errs[:, 1]) < 0), errs
    assert errs[-1, 0] < 1e-7 and errs[-1, 1] < 1e-5 and errs[-1, 2] < 1e-5, errs


def _tri_copy(s, x, rows):
    return _tri_system(x, s.q, rows, (s.excl_index, s.excl_atoms))


def test_triclinic_pme_forces_and_virial_are_energy_derivatives():
    s = _rd_small()
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    rows = opme._box_rows(s)
    x = s.x.astype(np.float64)
    grid = (14, 14, 12)
    r = opme.pme(s, p, grid=grid, order=6)
    h = 1e-6
    rng = np.random.default_rng(4)
    for a in rng.choice(s.n, size=4, replace=False):
        for dcomp in range(3):
            es = []
            for sgn in (+1, -1):
                x2 = x.copy()
                x2[a, dcomp] += sgn * h
                es.append(opme.pme(_tri_copy(s, x2, rows), p, grid=grid, order=6)["energy"])
            assert -(es[0] - es[1]) / (2 * h) == pytest.approx(r["forces"][a, dcomp], rel=1e-6, abs=1e-5)
    # x_a -> x_a + eps x_b for the atoms and the box rows, keeping the box
    # lower-triangular (b >= a): 2 Xi_ab = dE/deps
    for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)):
        es = []
        for sgn in (+1, -1):
            D = np.eye(3)
            D[a, b] += sgn * h
            es.append(opme.pme(_tri_copy(s, x @ D.T, rows @ D.T), p, grid=grid, order=6)["energy"])
        dE = (es[0] - es[1]) / (2 * h)
        assert dE == pytest.approx(2 * r["virial"][a, b], rel=1e-6, abs=1e-7 * abs(r["energy"]))


def test_triclinic_exclusions_use_the_minimum_image():
    s = _rd_small()
    p = wb.Params(coul=wb.COUL_EWALD, beta=3.12)
    ex = opme.ewald_exclusions(s, p)
    # the same molecules, each moved whole into the cell: nothing changes
    rows = opme._box_rows(s)
    x = s.x.astype(np.float64).reshape(-1, 3, 3)
    shift = np.array([1, -1, 0]) @ rows
    x2 = x.copy()
    x2[::2] += shift              # every other molecule by a lattice vector
    x2[1::3, 1] += rows[2]        # and some single atoms by another
    ex2 = opme.ewald_exclusions(_tri_copy(s, x2.reshape(-1, 3), rows), p)
    assert ex2["energy"] == pytest.approx(ex["energy"], rel=1e-12)
    assert np.allclose(ex2["forces"], ex["forces"], rtol=0, atol=1e-9 * np.abs(ex["forces"]).max())
