#!/usr/bin/env python3
"""Fit the erfc approximation used by the Ewald energy kernel; writes erfc_fit.cuh.

Form: erfc(x) = exp(-x^2) R(u), with t = 1 / (1 + P x) on x in [0, XMAX]
and u = UA t + UB mapping t's range onto [-1, 1].  R is a polynomial in u
fitted by least squares to the scaled complementary error function
erfcx(x) = exp(x^2) erfc(x) (scipy.special.erfcx, double precision) at
M Chebyshev nodes in u, in the Chebyshev basis (well conditioned), and
then converted to the power basis for Horner evaluation.  The fitted
R stays smooth and close to 1, and the power-basis coefficients sum to
about 1 in magnitude, so a float32 Horner evaluation adds only a few
roundings.

The fit is of degree 12 (max relative error ~4e-11), with every
coefficient split into a float32 head and a float32 tail so that the
rounding of the coefficients does not bias the energy.  A second fit, of
2^f on [-0.5, 0.5] (degree 10, head + tail), gives the energy kernel an
exponential free of the SFU's approximation error.  (The force kernel
takes the Ewald force from a table built by the library at run time.)

Run: python fit_erfc.py  (needs numpy and scipy; the output is committed)
"""
import os

import numpy as np
from scipy.special import erfcx

# The constants are rounded to float32 first and the fit is made for the
# rounded values, so that the kernels' float32 mapping x -> t -> u is the
# fitted one and only the (unbiased) rounding of each operation remains.
P = float(np.float32(0.4))
XMAX = 6.0
M = 4000
T0 = 1.0 / (1.0 + P * XMAX)
UA = float(np.float32(2.0 / (1.0 - T0)))
UB = float(np.float32(-2.0 * T0 / (1.0 - T0) - 1.0))
U_LO, U_HI = UA * T0 + UB, UA + UB


def fit(deg: int) -> np.ndarray:
    v = np.cos(np.pi * (np.arange(M) + 0.5) / M)
    u = 0.5 * (U_LO + U_HI) + 0.5 * (U_HI - U_LO) * v
    t = (u - UB) / UA
    x = (1.0 / t - 1.0) / P
    series = np.polynomial.Chebyshev.fit(u, erfcx(x), deg, domain=[U_LO, U_HI])
    return series.convert(kind=np.polynomial.Polynomial).coef


def fit_exp2(deg: int) -> np.ndarray:
    """2^f on f in [-0.5, 0.5] by least squares at Chebyshev nodes (power basis in f)."""
    v = np.cos(np.pi * (np.arange(M) + 0.5) / M)
    f = 0.5 * v
    series = np.polynomial.Chebyshev.fit(f, np.exp2(f), deg, domain=[-0.5, 0.5])
    return series.convert(kind=np.polynomial.Polynomial).coef


def max_rel_error(a: np.ndarray) -> float:
    x = np.linspace(0.0, XMAX, 400001)
    t = 1.0 / (1.0 + P * x)
    u = UA * t + UB
    r = np.polynomial.polynomial.polyval(u, a)
    return float(np.abs(r / erfcx(x) - 1.0).max())


def fmt(v: float) -> str:
    return f"{np.float32(v)!r}".replace("np.float32(", "").rstrip(")") + "f"


def main():
    ae = fit(12)
    ae_hi = ae.astype(np.float32)
    ae_lo = (ae - ae_hi.astype(np.float64)).astype(np.float32)
    a2 = fit_exp2(10)
    ff = np.linspace(-0.5, 0.5, 200001)
    e2 = float(np.abs(np.polynomial.polynomial.polyval(ff, a2) / np.exp2(ff) - 1.0).max())
    a2_hi = a2.astype(np.float32)
    a2_lo = (a2 - a2_hi.astype(np.float64)).astype(np.float32)
    # the error of the coefficients as stored (float32 head + float32 tail),
    # evaluated exactly in float64
    ae_st = ae_hi.astype(np.float64) + ae_lo.astype(np.float64)
    lines = [
        "// erfc_fit.cuh -- generated by fit_erfc.py; do not edit.",
        "// erfc(x) = exp(-x^2) R(u), t = 1/(1 + EF_P x), u = EF_UA t + EF_UB, x in [0, EF_XMAX].",
        f"// energy fit: degree {len(ae) - 1}, max relative error {max_rel_error(ae):.2e}"
        f" ({max_rel_error(ae_st):.2e} with the head + tail coefficients below)",
        "#pragma once",
        "namespace nbgb {",
        f"constexpr float EF_P = {fmt(P)};",
        f"constexpr float EF_XMAX = {fmt(XMAX)};",
        f"constexpr float EF_UA = {fmt(UA)};",
        f"constexpr float EF_UB = {fmt(UB)};",
        f"constexpr int EF_NE = {len(ae)};",
        "__device__ constexpr float EF_EN_HI[EF_NE] = {" + ", ".join(fmt(v) for v in ae_hi) + "};",
        "__device__ constexpr float EF_EN_LO[EF_NE] = {" + ", ".join(fmt(v) for v in ae_lo) + "};",
        f"// 2^f on [-0.5, 0.5]: degree {len(a2) - 1}, max relative error {e2:.2e}",
        f"constexpr int EX2_N = {len(a2)};",
        "__device__ constexpr float EX2_HI[EX2_N] = {" + ", ".join(fmt(v) for v in a2_hi) + "};",
        "__device__ constexpr float EX2_LO[EX2_N] = {" + ", ".join(fmt(v) for v in a2_lo) + "};",
        "}  // namespace nbgb",
        "",
    ]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "erfc_fit.cuh")
    with open(out, "w") as fh:
        fh.write("\n".join(lines))
    print(out)
    print(lines[2])


if __name__ == "__main__":
    main()
