"""Pins of the erfc and 2^f fits that the Ewald energy kernel evaluates.

The energy kernel takes erfc(x) = exp(-x^2) R(u), t = 1 / (1 + P x),
u = UA t + UB, with R a least-squares polynomial fitted by csrc/fit_erfc.py,
and 2^f on [-0.5, 0.5] as a fitted polynomial.  These tests read the
coefficients exactly as csrc/erfc_fit.cuh stores them and check them against
the standard library's erfc and 2^f (math.erfc, math.exp; not scipy, which
the fitter used):

  * the fits with the stored coefficients, evaluated exactly in float64,
    meet the errors the header states;
  * the kernel's double-float evaluation (error-free two-sum and two-product
    steps, compensated Horner for the head terms, exact range reduction of
    2^a) reaches erfc to 1e-9 relative (the fit's 4.4e-11 plus the float32
    tail terms of its two polynomials).

The float32 arithmetic is emulated with numpy: a product of two float32
values is exact in float64, so a fused multiply-add is formed in float64 and
rounded once more to float32 (a double rounding that can move a result by
one float32 ulp in rare cases; the bounds below leave room for it).  The
kernel refines its SFU reciprocal by a residual step and uses no SFU 2^x, so
the emulation is faithful.  The force kernel uses no erfc fit: its table of
the force factor is pinned in tests/test_ewald_table_cpu.py.  These pins need
no GPU; the same quantities are checked on the device through the library in
tests/test_gpu_parity.py.
"""
import math
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1506_00716_gb300",
                   "csrc", "erfc_fit.cuh")
f32 = np.float32


def _header():
    src = open(HDR).read()

    def scal(name):
        return f32(float(re.search(r"constexpr float %s = ([^;]+?)f;" % name, src).group(1)))

    def arr(name):
        body = re.search(r"%s\[[A-Z0-9_]+\] = \{([^}]*)\}" % name, src).group(1)
        return np.array([float(v.strip().rstrip("f")) for v in body.split(",")], dtype=np.float32)

    h = {n: scal(n) for n in ("EF_P", "EF_XMAX", "EF_UA", "EF_UB")}
    for n in ("EF_EN_HI", "EF_EN_LO", "EX2_HI", "EX2_LO"):
        h[n] = arr(n)
    h["stated"] = [float(v) for v in re.findall(r"\(([0-9.e+-]+) with the", src)]
    return h


H = _header()


def erfc_ref(x):
    return np.array([math.erfc(float(v)) for v in np.ravel(x)])


def erfcx_ref(x):
    return np.array([math.erfc(float(v)) * math.exp(float(v) * float(v)) for v in np.ravel(x)])


def _horner64(c, u):
    r = np.zeros_like(u)
    for k in range(len(c) - 1, -1, -1):
        r = r * u + float(c[k])
    return r


def _mapping64(x):
    t = 1.0 / (1.0 + float(H["EF_P"]) * x)
    return float(H["EF_UA"]) * t + float(H["EF_UB"])


X = np.linspace(0.0, float(H["EF_XMAX"]), 6001)


# ------------------------------------------------------- the stored fits


def test_header_states_the_stored_coefficients_error():
    assert len(H["stated"]) == 1  # energy


def test_energy_fit_with_stored_coefficients():
    c = H["EF_EN_HI"].astype(np.float64) + H["EF_EN_LO"].astype(np.float64)
    r = _horner64(c, _mapping64(X))
    err = np.abs(r / erfcx_ref(X) - 1.0).max()
    assert err <= 1.05 * H["stated"][0], err
    assert err < 5e-11


def test_exp2_fit_with_stored_coefficients():
    f = np.linspace(-0.5, 0.5, 4001)
    c = H["EX2_HI"].astype(np.float64) + H["EX2_LO"].astype(np.float64)
    ref = np.array([math.exp(v * math.log(2.0)) for v in f])
    err = np.abs(_horner64(c, f) / ref - 1.0).max()
    assert err < 2e-15, err


def test_fit_reduces_to_erfc_at_zero():
    # erfc(0) = 1: R(u(0)) = 1
    u0 = _mapping64(np.array([0.0]))
    c = H["EF_EN_HI"].astype(np.float64) + H["EF_EN_LO"].astype(np.float64)
    assert abs(_horner64(c, u0)[0] - 1.0) < 5e-11


# ---------------------------------------------- float32 arithmetic emulation


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


def split(v):
    hi = f32(v)
    return hi, f32(np.float64(v) - np.float64(hi))


def _horner_dd(hi, lo, k1, uh, ul, ph, pl):
    for k in range(k1, -1, -1):
        m, me = two_prod(ph, uh)
        cross = fma32(ph, ul, f32(pl * uh))
        s, se = two_sum(m, np.full_like(m, hi[k]))
        ph = s
        pl = f32(f32(f32(f32(me + se) + cross)) + lo[k])
    return ph, pl


def erfc_energy_dd(xh, xl, ah, al):
    """The energy kernel's erfc in double-float: returns (eh, el)."""
    big = xh > H["EF_XMAX"]
    xh = np.where(big, H["EF_XMAX"], xh).astype(np.float32)
    xl = np.where(big, f32(0.0), xl).astype(np.float32)
    P, UA, UB = H["EF_P"], H["EF_UA"], H["EF_UB"]
    m, me = two_prod(np.full_like(xh, P), xh)
    dh, de = two_sum(np.full_like(xh, 1.0), m)
    dl = f32(de + fma32(P, xl, me))
    th = f32(f32(1.0) / dh)  # SFU reciprocal, then one Newton step as the kernel does
    th = f32(th * fma32(-dh, th, f32(2.0)))
    r = fma32(-dh, th, f32(1.0))
    r = fma32(-dl, th, r)
    tl = f32(th * r)
    uh, ue = two_prod(np.full_like(th, UA), th)
    sh, se = two_sum(uh, np.full_like(uh, UB))
    ul = f32(se + fma32(UA, tl, ue))
    uh = sh
    eh_, el_ = H["EF_EN_HI"], H["EF_EN_LO"]
    ph = np.full_like(uh, eh_[-1])
    for k in range(len(eh_) - 2, 4, -1):  # float32 tail, k = 11 .. 5
        ph = fma32(ph, uh, eh_[k])
    pl = np.zeros_like(ph)
    ph, pl = _horner_dd(eh_, el_, 4, uh, ul, ph, pl)
    ah = np.maximum(ah, f32(-120.0)).astype(np.float32)
    n = np.rint(ah).astype(np.float32)
    fh = f32(ah - n)
    qh_, ql_ = H["EX2_HI"], H["EX2_LO"]
    qh = np.full_like(fh, qh_[-1])
    for k in range(len(qh_) - 2, 3, -1):  # float32 tail, k = 9 .. 4
        qh = fma32(qh, fh, qh_[k])
    ql = np.zeros_like(qh)
    qh, ql = _horner_dd(qh_, ql_, 3, fh, al, qh, ql)
    scale = np.ldexp(np.float32(1.0), n.astype(np.int32)).astype(np.float32)
    ch, ce = two_prod(ph, qh)
    cl = f32(ce + fma32(ph, ql, f32(pl * qh)))
    return f32(ch * scale), f32(cl * scale)


@pytest.mark.parametrize("lo,hi", [(0.0, 0.5), (0.5, 3.2), (3.2, 6.0)])
def test_energy_kernel_double_float_erfc(lo, hi):
    x = np.linspace(lo, hi, 2001)
    xh, xl = split(x)
    a = -(x * x) / math.log(2.0)  # -x^2 log2(e), as the kernel forms it in double-float
    ah, al = split(a)
    eh, el = erfc_energy_dd(xh, xl, ah, al)
    got = eh.astype(np.float64) + el.astype(np.float64)
    xx = xh.astype(np.float64) + xl.astype(np.float64)
    err = np.abs(got / erfc_ref(xx) - 1.0).max()
    # the fit's 4.4e-11, plus the tail terms of both polynomials, which the
    # kernel evaluates in plain float32 (R: k >= 5; 2^f: k >= 4): each rounds
    # at 2^-24 of a partial sum of size ~1e-3 relative to the result, up to
    # about 5e-10 at the ends of the range.  The double-float head steps add
    # about 1e-13.
    assert err < 1e-9, err
