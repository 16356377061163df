"""Pins of the Ewald force table that the force kernel interpolates.

The real-space Coulomb force of a pair is F/r = f qi qj G(r) / r^3 with
G(r) = erfc(beta r) + 2 beta r / sqrt(pi) exp(-beta^2 r^2): G / r^2 is minus
the r-derivative of the pair energy term erfc(beta r) / r (Section 3.2's
Ewald real-space interaction).  The force kernel reads G from a cubic Hermite
table on intervals of width h = 2^-n, which the library builds on the host
(nb_ewald_force_table, no GPU needed).  These tests check the table against
the standard library's erfc and exp only:

  * G as the table defines it is the derivative of the energy term (central
    differences of math.erfc(beta r) / r);
  * the interval ends hold G and h dG/dr exactly up to float32 rounding;
  * the cubics, evaluated in float64, are within the stated interpolation
    error of G everywhere on [0, rc] (1e-7 of G, G taken as at least 1e-7),
    plus the rounding of the float32 coefficients;
  * the kernel's float32 evaluation (interval index k = floor(r / h) by the
    1.5 * 2^23 constant and a round-down fused multiply-add, s = r / h - k by
    one more, Horner in float32) is within a few float32 roundings of that;
  * the table covers every beta rc up to 10 within 2048 intervals and the
    entry point rejects what lies outside.
"""
import math
import os
import shutil

import numpy as np
import pytest

from paper_1506_00716_gb300 import build as nbbuild
from paper_1506_00716_gb300 import nb

f32 = np.float32
ISQPI = 1.0 / math.sqrt(math.pi)


@pytest.fixture(scope="module")
def lib():
    if shutil.which(nbbuild.NVCC) is None and not os.path.exists(nbbuild.LIB):
        pytest.skip("nvcc not available")
    nbbuild.build()
    return nb.load()


def G(beta, r):
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    x = beta * r
    return np.array([math.erfc(v) for v in x]) + 2.0 * ISQPI * x * np.exp(-x * x)


def dG(beta, r):
    x = beta * np.asarray(r, dtype=np.float64)
    return -4.0 * ISQPI * beta * x * x * np.exp(-x * x)


def _cubic64(coef, h, r):
    u = np.asarray(r, dtype=np.float64) / h
    k = np.minimum(np.floor(u).astype(np.int64), len(coef) - 1)
    s = u - k
    c = coef.astype(np.float64)[k]
    return ((c[:, 3] * s + c[:, 2]) * s + c[:, 1]) * s + c[:, 0], c


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _kernel32(coef, h, r):
    """The force kernel's evaluation, in emulated float32 arithmetic."""
    magic = f32(12582912.0)  # 1.5 * 2^23: the float32 grid spacing there is 1
    invh = f32(1.0 / h)
    r = np.asarray(r, dtype=np.float32)
    # a fused multiply-add rounded down: magic + floor(r / h), the float32
    # grid spacing at magic being 1 (r / h < 2^22 is exact in float64)
    m = (np.float64(magic) + np.floor(r.astype(np.float64) * np.float64(invh))).astype(np.float32)
    s = fma32(r, invh, f32(magic - m))  # r / h - k, exact
    k = np.minimum(m.view(np.int32) - np.array([magic], dtype=np.float32).view(np.int32)[0], len(coef) - 1)
    c = coef[k]
    g = fma32(fma32(fma32(c[:, 3], s, c[:, 2]), s, c[:, 1]), s, c[:, 0])
    return g, k, s


@pytest.mark.parametrize("beta", [0.7, 3.12, 4.5])
def test_G_is_minus_r2_times_the_derivative_of_the_energy_term(beta):
    r = np.linspace(0.05, 1.2, 200)
    d = 1e-4
    e = lambda rr: np.array([math.erfc(beta * v) / v for v in rr])
    # five-point central difference: truncation error d^4 f^(5) / 30
    deriv = (-e(r + 2 * d) + 8 * e(r + d) - 8 * e(r - d) + e(r - 2 * d)) / (12 * d)
    assert np.allclose(-deriv * r * r, G(beta, r), rtol=1e-9, atol=1e-12)


def test_benchmark_parameters_table_shape(lib):
    coef, h = nb.nb_ewald_force_table(3.12, 1.0)
    assert h == 2.0**-8
    assert coef.shape == (257, 4)  # intervals reach rc (1 + 1e-4)
    # G(0) = 1 (erfc(0) = 1, the Gaussian term vanishes), b1(0) = 0
    assert coef[0, 0] == f32(1.0)
    assert coef[0, 1] == f32(0.0)


@pytest.mark.parametrize("beta,rc", [(3.12, 1.0), (3.47, 0.9), (3.12, 1.2), (0.5, 1.0), (4.0, 1.0), (6.0, 1.0),
                                     (10.0, 1.0), (2.9, 3.0)])
def test_interval_ends_hold_G_and_its_derivative(lib, beta, rc):
    coef, h = nb.nb_ewald_force_table(beta, rc)
    K = len(coef)
    assert 0 < K <= 2048 and K * h >= rc * (1 + 1e-4) and (K - 1) * h < rc * (1 + 1e-4)
    assert h == 2.0 ** round(math.log2(h))
    ends = np.arange(K) * h
    c = coef.astype(np.float64)
    g0, g1 = G(beta, ends), G(beta, ends + h)
    d0, d1 = h * dG(beta, ends), h * dG(beta, ends + h)
    ulp = 2.0**-24
    sub = 1e-44  # a few float32 subnormal steps (G < 1e-38 for beta r > 9.3)
    assert np.all(np.abs(c[:, 0] - g0) <= ulp * np.abs(g0) + sub)
    assert np.all(np.abs(c[:, 1] - d0) <= ulp * np.abs(d0) + sub)
    # the far end: b0 + b1 + b2 + b3 = G((k+1) h), b1 + 2 b2 + 3 b3 = h G'((k+1) h)
    tol = 4 * ulp * np.abs(c).sum(axis=1) + sub
    assert np.all(np.abs(c.sum(axis=1) - g1) <= tol + ulp * np.abs(g1))
    assert np.all(np.abs(c[:, 1] + 2 * c[:, 2] + 3 * c[:, 3] - d1) <= 3 * tol + ulp * np.abs(d1))


@pytest.mark.parametrize("beta,rc", [(3.12, 1.0), (3.47, 0.9), (4.0, 1.0), (6.0, 1.0), (10.0, 1.0), (1.0, 2.5)])
def test_cubics_meet_the_stated_error(lib, beta, rc):
    coef, h = nb.nb_ewald_force_table(beta, rc)
    r = np.linspace(0.0, rc * (1 + 1e-4), 40001)
    got, c = _cubic64(coef, h, r)
    ref = G(beta, r)
    k = np.minimum(np.floor(r / h).astype(np.int64), len(coef) - 1)
    far = G(beta, (k + 1) * h)
    bound = 1e-7 * np.maximum(far, 1e-7) + 2.0**-24 * np.abs(c).sum(axis=1)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)
    # relative to G where G matters: the float32 rounding of G itself
    big = ref > 1e-4
    assert np.max(np.abs(got[big] / ref[big] - 1.0)) < 4e-7


def test_interpolation_error_is_not_trivially_small(lib):
    """The step is the largest power of two meeting 1e-7: twice the step
    would break it (the bound is not met by a needlessly fine table)."""
    beta, rc = 3.12, 1.0
    coef, h = nb.nb_ewald_force_table(beta, rc)
    # Hermite cubics with twice the step, built here from G and G' directly
    H2 = 2 * h
    r = np.linspace(0.0, rc, 20001)
    k = np.floor(r / H2)
    s = r / H2 - k
    a, b = k * H2, (k + 1) * H2
    g0, g1 = G(beta, a), G(beta, b)
    d0, d1 = H2 * dG(beta, a), H2 * dG(beta, b)
    h00, h10, h01, h11 = 2 * s**3 - 3 * s**2 + 1, s**3 - 2 * s**2 + s, -2 * s**3 + 3 * s**2, s**3 - s**2
    coarse = h00 * g0 + h10 * d0 + h01 * g1 + h11 * d1
    rel = np.abs(coarse - G(beta, r)) / np.maximum(G(beta, b), 1e-7)
    assert rel.max() > 1e-7


@pytest.mark.parametrize("beta,rc", [(3.12, 1.0), (3.47, 0.9), (6.0, 1.0)])
def test_kernel_float32_evaluation(lib, beta, rc):
    coef, h = nb.nb_ewald_force_table(beta, rc)
    rng = np.random.default_rng(5)
    r = np.concatenate([rng.uniform(0.0, rc, 200000), np.arange(len(coef)) * h,
                        np.arange(1, len(coef)) * h * (1 - 2.0**-24)]).astype(np.float32)
    r = r[r <= rc * (1 + 1e-4)]
    g, k, s = _kernel32(coef, h, r)
    rr = r.astype(np.float64)
    u = rr / h
    assert np.all(k == np.minimum(np.floor(u), len(coef) - 1))
    assert np.all(k + s.astype(np.float64) == u)  # s exact
    assert np.all((s >= 0) & (s < 1.0 + (u >= len(coef))))
    ref = G(beta, rr)
    c = coef.astype(np.float64)[k]
    far = G(beta, (k + 1) * h)
    # the interpolation error, plus about six float32 roundings of the Horner steps
    bound = 1e-7 * np.maximum(far, 1e-7) + 8 * 2.0**-24 * np.abs(c).sum(axis=1)
    err = np.abs(g.astype(np.float64) - ref)
    assert np.all(err <= bound), np.max(err / bound)
    big = ref > 1e-4
    assert np.max(err[big] / ref[big]) < 6e-7


def test_every_beta_rc_up_to_ten_fits(lib):
    for rc in (0.5, 0.75, 1.0, 1.3, 2.0):
        for br in (0.5, 2.0, 3.0, 4.0, 5.0, 7.5, 10.0):
            coef, h = nb.nb_ewald_force_table(br / rc, rc)
            assert 0 < len(coef) <= 2048


@pytest.mark.parametrize("beta,rc", [(10.5, 1.0), (0.0, 1.0), (-1.0, 1.0), (3.0, 0.0), (float("nan"), 1.0)])
def test_rejects_out_of_range_parameters(lib, beta, rc):
    with pytest.raises(nb.NbError):
        nb.nb_ewald_force_table(beta, rc)


def test_rejects_a_short_buffer(lib):
    import ctypes
    n = ctypes.c_int()
    h = ctypes.c_double()
    buf = np.zeros((10, 4), dtype=np.float32)
    st = lib.nb_ewald_force_table(3.12, 1.0, buf.ctypes.data_as(ctypes.c_void_p), 10, ctypes.byref(n),
                                  ctypes.byref(h))
    assert st == 1  # NB_ERR_ARG
