"""The seeded synthetic inputs: the workloads' recipe, checked on the host.

The water boxes stand in for the paper's biomolecular systems.  These tests
fix what both the oracle and the CUDA path rely on: determinism under a
seed, the sizes of the five workloads, the rigid three-site geometry, the
charges and exclusions, the wrapping into the cell, the density, and the
distributions of the ensemble and of the request stream.
"""
import math

import numpy as np
import pytest

from paper_1506_00716_gb300 import waterbox as wb


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_boxes_are_deterministic_per_seed():
    a, b, c = wb.water_box(300, None, seed=7), wb.water_box(300, None, seed=7), wb.water_box(300, None, seed=8)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.q, b.q)
    assert np.array_equal(a.excl_atoms, b.excl_atoms)
    assert not np.array_equal(a.x, c.x)


@pytest.mark.parametrize("make,n,L", [(wb.small_box, 1944, 2.69), (wb.mid_box, 24000, 6.21)])
def test_workload_sizes(make, n, L):
    s = make()
    assert s.n == n and s.x.dtype == np.float32
    assert np.allclose(s.box, np.float32(L))
    # the box edge is a float32 value, so that host and device see one box
    assert float(np.float32(s.box[0])) == s.box[0]


def test_large_box_size_and_density():
    s = wb.large_box()
    assert s.n == 3_000_000
    assert s.box[0] == np.float32(31.0)
    rho = s.n / np.prod(s.box)
    assert rho == pytest.approx(100.2, rel=0.01)  # atoms per nm^3


def test_water_geometry_charges_exclusions():
    s = wb.mid_box()
    x = s.x.astype(np.float64).reshape(-1, 3, 3)
    L = s.box[0]
    oh1 = _min_image(x[:, 1] - x[:, 0], L)
    oh2 = _min_image(x[:, 2] - x[:, 0], L)
    r1, r2 = np.linalg.norm(oh1, axis=1), np.linalg.norm(oh2, axis=1)
    # rigid geometry up to the float32 rounding of the coordinates
    assert np.allclose(r1, wb.R_OH, atol=2e-6) and np.allclose(r2, wb.R_OH, atol=2e-6)
    ang = np.degrees(np.arccos((oh1 * oh2).sum(1) / (r1 * r2)))
    assert np.allclose(ang, wb.ANGLE_HOH_DEG, atol=2e-3)
    # neutral molecules with the listed charges; LJ on O only
    q = s.q.reshape(-1, 3)
    assert np.allclose(q.sum(1), 0.0, atol=1e-6)
    assert np.all(s.type.reshape(-1, 3) == [0, 1, 1])
    # symmetric exclusions: each atom excludes the other two atoms of its molecule
    for i in (0, 1, 2, 3 * 4000 + 2, s.n - 1):
        m = i // 3
        got = sorted(s.excl_atoms[s.excl_index[i]:s.excl_index[i + 1]].tolist())
        assert got == sorted({3 * m, 3 * m + 1, 3 * m + 2} - {i})


def test_coordinates_are_wrapped_into_the_cell():
    for s in (wb.small_box(), wb.mid_box()):
        assert np.all(s.x >= 0.0) and np.all(s.x < np.float32(s.box[0]))
    rd = wb.rhombic_dodecahedron_box(648, seed=5)
    for d in range(3):
        assert np.all(rd.x[:, d] >= 0.0) and np.all(rd.x[:, d] < np.float32(rd.box[d]))


def test_rhombic_dodecahedron_lattice():
    rd = wb.rhombic_dodecahedron_box(8000, seed=6)
    ax, by, cz = rd.box
    bx, cx, cy = rd.skew
    # xy-square form: a = (d,0,0), b = (0,d,0), c = (d/2, d/2, d sqrt(2)/2)
    assert ax == by and bx == 0.0 and cx == ax / 2 and cy == ax / 2
    assert cz == pytest.approx(ax * math.sqrt(2.0) / 2.0, rel=1e-6)
    # all 12 face vectors (a, b, c, c - a, c - b, c - a - b and opposites) equally long
    a, b, c = np.array([ax, 0, 0]), np.array([bx, by, 0]), np.array([cx, cy, cz])
    faces = [a, b, c - a, c - b, c, c - a - b]
    lens = [np.linalg.norm(v) for v in faces]
    assert np.allclose(lens, ax, rtol=1e-6)
    rho = rd.n / (ax * by * cz)
    assert rho == pytest.approx(100.2, rel=0.03)


def test_ensemble_sizes_log_uniform():
    sizes = wb.ensemble_sizes()
    assert sizes == wb.ensemble_sizes()  # seeded
    assert len(sizes) == 64 and min(sizes) >= 1000 and max(sizes) <= 32000
    logs = np.log(sizes)
    # log-uniform on [log 1000, log 32000]: mean of the logs near the midpoint
    mid = 0.5 * (math.log(1000) + math.log(32000))
    assert abs(logs.mean() - mid) < 0.35


def test_request_stream_poisson():
    t, sizes = wb.request_stream(4096)
    t2, sizes2 = wb.request_stream(4096)
    assert np.array_equal(t, t2) and sizes == sizes2
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps of mean 1/2000 s: mean and coefficient of variation near 1
    assert gaps.mean() == pytest.approx(1 / 2000, rel=0.06)
    assert gaps.std() / gaps.mean() == pytest.approx(1.0, abs=0.06)
    assert min(sizes) >= 1000 and max(sizes) <= 100000
