"""Pins of the Ewald energy table that the energy kernels interpolate.

The real-space Coulomb energy of a pair is f qi qj erfc(beta r) / r (Section
3.2's pair interaction with Ewald electrostatics).  The energy kernels take
erfc(beta r) from a table of quartics in s = r / h - k on intervals of width
h = 2^-n, which the library builds on the host (nb_ewald_energy_table, no GPU
needed), and evaluate the constant and linear terms in double-float, the
rest in float32.  These tests check the table against the standard library's
math.erfc and against printed values of erfc:

  * the quartics, evaluated in float64 from the stored float32 coefficients
    (a0 and a1 as hi + lo sums), are within the interpolation bound 1e-12
    plus the float32 rounding of a2..a4 (5e-12 in all) of erfc(beta r) on
    [0, rc (1 + 1e-4)], for several beta and rc, and reproduce the
    tabulated erfc(x) at x = 0.5, 1, 2, 3 (tests/golden/erfc_table.txt);
  * the low parts of a0 and a1 matter: without them the error reaches
    1e-9, so a table stored in plain float32 would not pass;
  * the kernels' evaluation (interval index by a round-down fused
    multiply-add onto 1.5 * 2^23, s = sh + sl, a0 + a1 s in double-float,
    s^2 (a2 + s (a3 + s a4)) in float32, a final fast two-sum), emulated
    step by step in float32, is within 3e-11 of erfc(beta r) for r given as
    a double-float value;
  * every beta rc up to 10 fits within 2048 intervals, and out-of-range
    parameters and short buffers are refused.

The float32 arithmetic is emulated with numpy: a product of two float32
values is exact in float64, so a fused multiply-add is formed in float64 and
rounded once to float32 (a double rounding that can move a result by one
float32 ulp in rare cases; the bounds leave room for it).
"""
import math
import os
import shutil

import numpy as np
import pytest

from paper_1506_00716_gb300 import build as nbbuild
from paper_1506_00716_gb300 import nb

f32 = np.float32
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "erfc_table.txt")


@pytest.fixture(scope="module")
def lib():
    if shutil.which(nbbuild.NVCC) is None and not os.path.exists(nbbuild.LIB):
        pytest.skip("nvcc not available")
    nbbuild.build()
    return nb.load()


def erfc64(x):
    return np.array([math.erfc(v) for v in np.atleast_1d(np.asarray(x, dtype=np.float64))])


def _quartic64(coef, h, r, with_lo=True):
    u = np.asarray(r, dtype=np.float64) / h
    k = np.minimum(np.floor(u).astype(np.int64), len(coef) - 1)
    s = u - k
    c = coef.astype(np.float64)[k]
    a0 = c[:, 0] + (c[:, 1] if with_lo else 0.0)
    a1 = c[:, 2] + (c[:, 3] if with_lo else 0.0)
    return a0 + s * (a1 + s * (c[:, 4] + s * (c[:, 5] + s * c[:, 6])))


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def two_prod(a, b):
    p = f32(a * b)
    return p, fma32(a, b, -p)


def _kernel_dd(coef, h, rh, rl):
    """The energy kernels' erfc(beta r) for r = rh + rl, in emulated float32."""
    magic = f32(12582912.0)  # 1.5 * 2^23: the float32 grid spacing there is 1
    invh = f32(1.0 / h)
    rh = np.asarray(rh, dtype=np.float32)
    rl = np.asarray(rl, dtype=np.float32)
    # round-down fused multiply-add: magic + floor(rh / h) (rh / h < 2^22)
    m = (np.float64(magic) + np.floor(rh.astype(np.float64) * np.float64(invh))).astype(np.float32)
    sh = fma32(rh, invh, f32(magic - m))
    sl = f32(rl * invh)
    k = np.minimum(m.view(np.int32) - np.array([magic], dtype=np.float32).view(np.int32)[0], len(coef) - 1)
    c = coef[k]
    t = fma32(c[:, 6], sh, c[:, 5])
    t = fma32(t, sh, c[:, 4])
    q = f32(f32(t * sh) * fma32(f32(2.0), sl, sh))
    p, pe = two_prod(c[:, 2], sh)
    low = fma32(c[:, 2], sl, fma32(c[:, 3], sh, pe))
    p2, e1 = two_sum(p, q)
    vh, e2 = two_sum(c[:, 0], p2)
    vl = f32(f32(e1 + e2) + f32(low + c[:, 1]))
    eh = f32(vh + vl)
    el = f32(vl - f32(eh - vh))
    return eh, el, k, sh


def test_benchmark_parameters_table_shape(lib):
    coef, h = nb.nb_ewald_energy_table(3.12, 1.0)
    assert h == 1.0 / 256
    assert len(coef) == 257  # reaches rc (1 + 1e-4)
    assert np.all(coef[:, 7] == 0.0)
    assert np.abs(coef[:, 4]).max() <= 1e-4  # the float32 quadratic term


@pytest.mark.parametrize("beta,rc", [(3.12, 1.0), (3.47, 0.9), (0.7, 1.2), (6.0, 1.0), (10.0, 1.0)])
def test_quartics_meet_the_stated_error(lib, beta, rc):
    coef, h = nb.nb_ewald_energy_table(beta, rc)
    r = np.linspace(0.0, rc * (1 + 1e-4), 200001)
    err = np.abs(_quartic64(coef, h, r) - erfc64(beta * r))
    # the interpolation bound 1e-12, plus the float32 rounding of a2..a4
    bound = 1e-12 + 2.0**-24 * np.abs(coef[:, 4:7].astype(np.float64)).sum(axis=1).max()
    assert err.max() <= bound, (err.max(), bound)
    assert err.max() <= 5e-12


def test_low_parts_are_needed(lib):
    coef, h = nb.nb_ewald_energy_table(3.12, 1.0)
    r = np.linspace(0.0, 1.0, 100001)
    err = np.abs(_quartic64(coef, h, r, with_lo=False) - erfc64(3.12 * r))
    assert err.max() > 1e-9


def test_reproduces_the_printed_erfc_values(lib):
    rows = [tuple(map(float, l.split())) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    # beta = 2 nm^-1, rc = 1.6 nm: r = x / 2 covers x up to 3.2
    beta, rc = 2.0, 1.6
    coef, h = nb.nb_ewald_energy_table(beta, rc)
    for x, ref in rows:
        got = _quartic64(coef, h, np.array([x / beta]))[0]
        assert abs(got - ref) <= 5e-12, (x, got, ref)


@pytest.mark.parametrize("beta,rc", [(3.12, 1.0), (3.47, 0.9), (6.0, 1.0)])
def test_kernel_double_float_evaluation(lib, beta, rc):
    coef, h = nb.nb_ewald_energy_table(beta, rc)
    rng = np.random.default_rng(11)
    r = np.concatenate([rng.uniform(0.05, rc * (1 + 1e-5), 200000), np.arange(1, len(coef) - 1) * h,
                        np.arange(1, len(coef) - 1) * h * (1 - 2.0**-23)])
    rh = r.astype(np.float32)
    rl = (r - rh.astype(np.float64)).astype(np.float32)
    rr = rh.astype(np.float64) + rl.astype(np.float64)
    eh, el, k, sh = _kernel_dd(coef, h, rh, rl)
    u = rh.astype(np.float64) / h
    assert np.all(k == np.minimum(np.floor(u), len(coef) - 1))
    assert np.all(k + sh.astype(np.float64) == u)  # sh exact
    got = eh.astype(np.float64) + el.astype(np.float64)
    err = np.abs(got - erfc64(beta * rr))
    assert err.max() <= 3e-11, err.max()


def test_every_beta_rc_up_to_ten_fits(lib):
    for rc in (0.5, 0.75, 1.0, 1.3, 2.0):
        for br in (0.5, 2.0, 3.0, 4.0, 5.0, 7.5, 10.0):
            coef, h = nb.nb_ewald_energy_table(br / rc, rc)
            assert 0 < len(coef) <= 2048
            assert len(coef) * h >= rc * (1 + 1e-4)


@pytest.mark.parametrize("beta,rc", [(10.5, 1.0), (0.0, 1.0), (-1.0, 1.0), (3.0, 0.0), (float("nan"), 1.0)])
def test_rejects_out_of_range_parameters(lib, beta, rc):
    with pytest.raises(nb.NbError):
        nb.nb_ewald_energy_table(beta, rc)


def test_rejects_a_short_buffer(lib):
    import ctypes
    n = ctypes.c_int()
    h = ctypes.c_double()
    buf = np.zeros((10, 8), dtype=np.float32)
    st = lib.nb_ewald_energy_table(3.12, 1.0, buf.ctypes.data_as(ctypes.c_void_p), 10, ctypes.byref(n),
                                   ctypes.byref(h))
    assert st == 1  # NB_ERR_ARG
