"""Seeded synthetic water boxes: the inputs shared by the CUDA path and the oracle.

This module holds input generation only.  It contains none of the
non-bonded arithmetic (no distances, no cut-off tests, no interactions), so
that the oracle and the CUDA path can both consume its output without
sharing any part of the method.

The paper measures on biomolecular systems (RNAse, GLIC and others, Sections
3.2-3.4) that are not available here.  Rigid three-site water boxes stand in
for them; the paper notes that water dominates such systems (Section 3.4).

Recipe (one molecule = consecutive atoms O, H1, H2):
  * cubic box of edge L, rounded to the nearest float32 so that both sides of
    every comparison use exactly the same box;
  * a simple-cubic lattice of n = ceil(n_mol**(1/3)) sites per edge, spacing
    L/n; n_mol of the n**3 sites are chosen by a seeded permutation;
  * O at the site plus a uniform jitter in [-0.02, 0.02] nm per coordinate;
  * H1, H2 at 0.1 nm from O with an H-O-H angle of 109.47 degrees, the
    molecule turned by a uniformly random rotation (random unit quaternion);
  * every coordinate wrapped into [0, L) and stored as float32;
  * charges O -0.8476 e, H +0.4238 e; Lennard-Jones on O only
    (sigma 0.3166 nm, epsilon 0.650 kJ/mol), given as a 2x2 type table
    c6 = 4 eps sigma^6, c12 = 4 eps sigma^12 (type 0 = O, type 1 = H);
  * the three intramolecular pairs of each molecule are excluded.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Water model (SPC/E-like charges, three sites).
Q_O = -0.8476
Q_H = 0.4238
SIGMA_O = 0.3166  # nm
EPS_O = 0.650  # kJ/mol
R_OH = 0.1  # nm
ANGLE_HOH_DEG = 109.47
JITTER = 0.02  # nm, uniform half-width
DENSITY_MOL = 33.4  # molecules / nm^3 for boxes sized from n_mol

COUL_RF = 0
COUL_EWALD = 1
ONE_4PI_EPS0 = 138.935458  # kJ mol^-1 nm e^-2


@dataclasses.dataclass
class Params:
    """Interaction parameters of a workload (units nm, kJ/mol, e)."""

    rc: float = 1.0
    rlist: float = 1.1
    coul: int = COUL_RF
    eps_r: float = 1.0
    eps_rf: float = 78.0
    beta: float = 3.12
    fcoul: float = ONE_4PI_EPS0
    ntypes: int = 2
    c6: np.ndarray = dataclasses.field(default_factory=lambda: lj_table()[0])
    c12: np.ndarray = dataclasses.field(default_factory=lambda: lj_table()[1])
    modifiers: int = 0  # potential-modifier bits (library: NB_MOD_*, oracle: MOD_*)


@dataclasses.dataclass
class System:
    """One periodic water box.  Arrays are in the caller's (original) atom order."""

    x: np.ndarray  # float32 [n, 3], wrapped into [0, L)
    q: np.ndarray  # float32 [n]
    type: np.ndarray  # int32 [n]
    box: np.ndarray  # float64 [3], each a float32-representable value
    excl_index: np.ndarray  # int32 [n + 1], CSR over atoms
    excl_atoms: np.ndarray  # int32 [nnz], the excluded partners (both directions)
    n_mol: int
    seed: int
    # off-diagonal box components (bx, cx, cy) of a triclinic box with rows
    # a = (ax, 0, 0), b = (bx, by, 0), c = (cx, cy, cz), box = (ax, by, cz);
    # zero for a rectangular box.  Coordinates then lie in the rectangle
    # [0, ax) x [0, by) x [0, cz), a unit cell of the same lattice.
    skew: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def xq(self) -> np.ndarray:
        """float32 [n, 4] = (x, y, z, q), the coordinate layout the library takes."""
        out = np.empty((self.n, 4), dtype=np.float32)
        out[:, :3] = self.x
        out[:, 3] = self.q
        return out


def lj_table() -> tuple[np.ndarray, np.ndarray]:
    """2x2 c6 / c12 tables (float32 values, row-major [ti * 2 + tj])."""
    c6 = np.zeros(4, dtype=np.float32)
    c12 = np.zeros(4, dtype=np.float32)
    c6[0] = 4.0 * EPS_O * SIGMA_O**6
    c12[0] = 4.0 * EPS_O * SIGMA_O**12
    return c6, c12


def f32(v: float) -> float:
    """Round a value to the nearest float32 and return it as a Python float."""
    return float(np.float32(v))


def box_for(n_mol: int) -> float:
    """Cubic box edge for n_mol molecules at the standard density."""
    return f32((n_mol / DENSITY_MOL) ** (1.0 / 3.0))


def _random_rotations(rng: np.random.Generator, m: int) -> np.ndarray:
    """m uniformly random rotation matrices from random unit quaternions."""
    qv = rng.standard_normal((m, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, a, b, c = qv[:, 0], qv[:, 1], qv[:, 2], qv[:, 3]
    r = np.empty((m, 3, 3))
    r[:, 0, 0] = 1 - 2 * (b * b + c * c)
    r[:, 0, 1] = 2 * (a * b - c * w)
    r[:, 0, 2] = 2 * (a * c + b * w)
    r[:, 1, 0] = 2 * (a * b + c * w)
    r[:, 1, 1] = 1 - 2 * (a * a + c * c)
    r[:, 1, 2] = 2 * (b * c - a * w)
    r[:, 2, 0] = 2 * (a * c - b * w)
    r[:, 2, 1] = 2 * (b * c + a * w)
    r[:, 2, 2] = 1 - 2 * (a * a + b * b)
    return r


def wrap32(x: np.ndarray, L: float) -> np.ndarray:
    """Wrap float64 coordinates into [0, L) and round to float32, keeping < L."""
    y = np.mod(x, L).astype(np.float32)
    Lf = np.float32(L)
    y[y >= Lf] = np.float32(0.0)
    y[y < 0] = np.float32(0.0)
    return y


def wrap_triclinic32(x: np.ndarray, box: np.ndarray, skew: np.ndarray) -> np.ndarray:
    """Wrap float64 coordinates into the unit cell [0, ax) x [0, by) x [0, cz) of
    the lattice a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz) (z by c first, then
    y by b, then x by a) and round to float32, keeping every value below its
    edge."""
    ax, by, cz = (float(v) for v in box)
    bx, cx, cy = (float(v) for v in skew)
    y = np.array(x, dtype=np.float64)
    k = np.floor(y[:, 2] / cz)
    y[:, 0] -= k * cx
    y[:, 1] -= k * cy
    y[:, 2] -= k * cz
    j = np.floor(y[:, 1] / by)
    y[:, 0] -= j * bx
    y[:, 1] -= j * by
    y[:, 0] -= np.floor(y[:, 0] / ax) * ax
    out = y.astype(np.float32)
    for d, edge in enumerate((ax, by, cz)):
        e = np.float32(edge)
        col = out[:, d]
        col[col >= e] = np.nextafter(e, np.float32(0.0))
        col[col < 0] = np.float32(0.0)
    return out


def water_box(n_mol: int, L: float | None = None, seed: int = 1) -> System:
    """A jittered-lattice water box of n_mol molecules (recipe in the module doc)."""
    if L is None:
        L = box_for(n_mol)
    L = f32(L)
    rng = np.random.default_rng(seed)
    n_side = int(math.ceil(round(n_mol ** (1.0 / 3.0), 9)))
    while n_side**3 < n_mol:
        n_side += 1
    spacing = L / n_side
    sites = rng.permutation(n_side**3)[:n_mol]
    ix = sites % n_side
    iy = (sites // n_side) % n_side
    iz = sites // (n_side * n_side)
    o = (np.stack([ix, iy, iz], axis=1) + 0.5) * spacing
    o = o + rng.uniform(-JITTER, JITTER, size=(n_mol, 3))
    half = math.radians(ANGLE_HOH_DEG) / 2.0
    local = np.array(
        [
            [R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
            [-R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
        ]
    )
    rot = _random_rotations(rng, n_mol)
    h = np.einsum("mij,kj->mki", rot, local)  # [m, 2, 3]
    pos = np.empty((n_mol, 3, 3))
    pos[:, 0] = o
    pos[:, 1] = o + h[:, 0]
    pos[:, 2] = o + h[:, 1]
    x = wrap32(pos.reshape(-1, 3), L)
    n = 3 * n_mol
    q = np.tile(np.array([Q_O, Q_H, Q_H], dtype=np.float32), n_mol)
    typ = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    excl_index = np.arange(0, 2 * n + 1, 2, dtype=np.int32)
    base = np.repeat(np.arange(n_mol, dtype=np.int32) * 3, 3)
    within = np.tile(np.array([[1, 2], [0, 2], [0, 1]], dtype=np.int32), (n_mol, 1))
    excl_atoms = (base[:, None] + within).reshape(-1).astype(np.int32)
    box = np.array([L, L, L], dtype=np.float64)
    return System(x=x, q=q, type=typ, box=box, excl_index=excl_index,
                  excl_atoms=excl_atoms, n_mol=n_mol, seed=seed)


def _waters_at(o: np.ndarray, rng: np.random.Generator):
    """Atoms (O, H, H per molecule) of water molecules with O at o [m, 3] in
    random orientations, and their charges, types and exclusions."""
    n_mol = o.shape[0]
    half = math.radians(ANGLE_HOH_DEG) / 2.0
    local = np.array([[R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
                      [-R_OH * math.sin(half), 0.0, R_OH * math.cos(half)]])
    rot = _random_rotations(rng, n_mol)
    h = np.einsum("mij,kj->mki", rot, local)
    pos = np.empty((n_mol, 3, 3))
    pos[:, 0] = o
    pos[:, 1] = o + h[:, 0]
    pos[:, 2] = o + h[:, 1]
    n = 3 * n_mol
    q = np.tile(np.array([Q_O, Q_H, Q_H], dtype=np.float32), n_mol)
    typ = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    excl_index = np.arange(0, 2 * n + 1, 2, dtype=np.int32)
    base = np.repeat(np.arange(n_mol, dtype=np.int32) * 3, 3)
    within = np.tile(np.array([[1, 2], [0, 2], [0, 1]], dtype=np.int32), (n_mol, 1))
    excl_atoms = (base[:, None] + within).reshape(-1).astype(np.int32)
    return pos.reshape(-1, 3), q, typ, excl_index, excl_atoms


def rhombic_dodecahedron_box(n_mol: int, seed: int = 1) -> System:
    """Water in a rhombic dodecahedron (its xy-square form: a = (d, 0, 0),
    b = (0, d, 0), c = (d/2, d/2, d sqrt(2)/2)) at the standard density, with
    about n_mol molecules.  O sits on a jittered lattice of n x n x nz sites in
    the rectangle [0, d) x [0, d) x [0, cz), n even, so that c carries every
    site onto a site: the lattice continues across every face of the cell."""
    spacing = (1.0 / DENSITY_MOL) ** (1.0 / 3.0)
    d = (n_mol / DENSITY_MOL / (math.sqrt(2.0) / 2.0)) ** (1.0 / 3.0)
    n = max(2, 2 * int(round(d / spacing / 2.0)))
    d = f32(n * spacing)
    cz = f32(d * math.sqrt(2.0) / 2.0)
    nz = max(1, int(round(cz / spacing)))
    s_xy, s_z = d / n, cz / nz
    rng = np.random.default_rng(seed)
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(nz), indexing="ij")
    o = np.stack([(i.ravel() + 0.5) * s_xy, (j.ravel() + 0.5) * s_xy, (k.ravel() + 0.5) * s_z], axis=1)
    o = o + rng.uniform(-JITTER, JITTER, size=o.shape)
    pos, q, typ, ei, ea = _waters_at(o, rng)
    box = np.array([d, d, cz], dtype=np.float64)
    skew = np.array([0.0, d / 2.0, d / 2.0], dtype=np.float64)
    x = wrap_triclinic32(pos, box, skew)
    return System(x=x, q=q, type=typ, box=box, excl_index=ei, excl_atoms=ea, n_mol=o.shape[0], seed=seed,
                  skew=skew)


def perturb(sys: System, rng: np.random.Generator, sigma: float = 0.005) -> np.ndarray:
    """Cumulative Gaussian displacement of every coordinate (float32, wrapped)."""
    xn = sys.x.astype(np.float64) + rng.normal(0.0, sigma, size=sys.x.shape)
    sys.x = wrap32(xn, float(sys.box[0]))
    return sys.x


# ---------------------------------------------------------------------------
# The five workloads.
# ---------------------------------------------------------------------------

def params_rf() -> Params:
    return Params(coul=COUL_RF)


def params_ewald() -> Params:
    return Params(coul=COUL_EWALD)


def small_box(seed: int = 1) -> System:
    """648 waters (1,944 atoms) in L = 2.69 nm; LJ + reaction-field."""
    return water_box(648, 2.69, seed)


def mid_box(seed: int = 2) -> System:
    """8,000 waters (24,000 atoms) in L = 6.21 nm; LJ + reaction-field."""
    return water_box(8000, 6.21, seed)


def large_box(seed: int = 3) -> System:
    """1,000,000 waters (3,000,000 atoms) in L = 31.0 nm; LJ + Ewald real space."""
    return water_box(1_000_000, 31.0, seed)


def ensemble_sizes(count: int = 64, lo: int = 1000, hi: int = 32000, seed: int = 4) -> list[int]:
    """Molecule counts drawn log-uniformly from [lo, hi]."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    return [int(round(math.exp(v))) for v in u]


def ensemble(count: int = 64, lo: int = 1000, hi: int = 32000, seed: int = 4) -> list[System]:
    """Independent boxes of log-uniform size, each at 33.4 molecules/nm^3."""
    sizes = ensemble_sizes(count, lo, hi, seed)
    return [water_box(m, None, seed * 1000 + k) for k, m in enumerate(sizes)]


def request_stream(count: int, rate: float = 2000.0, lo: int = 1000, hi: int = 100000,
                   seed: int = 5) -> tuple[np.ndarray, list[int]]:
    """Poisson arrival times (s) and log-uniform molecule counts of a request stream."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    sizes = [int(round(math.exp(v))) for v in u]
    return t, sizes
