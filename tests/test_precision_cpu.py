"""Why the energy kernel evaluates pair energies in double-float.

The energy and virial tolerance is 1e-6 relative.  A box of neutral,
randomly oriented waters cancels its Coulomb energy strongly: on the
1,944-atom box |E_C| is about 330 kJ/mol while the pair terms, up to ~100
kJ/mol each, add up to millions in absolute value.  This test evaluates the
reaction-field pair energies of the 1,944- and 24,000-atom boxes with every
operation rounded to float32 (what a float32 pair kernel does before it even
accumulates), sums those terms exactly, and finds the total off by more than
1e-6 on at least one of the seeded boxes; and it evaluates the same terms
exactly and rounds each once to float32 (the best any float32 pair term can
be), which stays within 1e-6 but with less than a 10x margin on some box.
Only the pair evaluation is float32 here; a kernel's float32 partial sums
would add their own rounding on top.
"""
import math

import numpy as np

import oracle
from paper_1506_00716_gb300 import waterbox as wb

f32 = np.float32


def _rf_terms(s, p):
    keys = oracle.pairs(s, p.rc)
    i, j = keys // s.n, keys % s.n
    L = float(s.box[0])
    d = s.x[i].astype(np.float64) - s.x[j].astype(np.float64)
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(1))
    krf = (p.eps_rf - p.eps_r) / ((2 * p.eps_rf + p.eps_r) * p.rc**3)
    crf = 1.0 / p.rc + krf * p.rc**2
    qq = p.fcoul / p.eps_r * s.q[i].astype(np.float64) * s.q[j].astype(np.float64)
    exact = qq * (1.0 / r + krf * r * r - crf)
    # every operation in float32 (d itself is exact: both coordinates are
    # float32 and the minimum-image shift is a multiple of the float32 box)
    d32 = d.astype(np.float32)
    r2 = f32(f32(f32(d32[:, 0] * d32[:, 0]) + f32(d32[:, 1] * d32[:, 1])) + f32(d32[:, 2] * d32[:, 2]))
    rinv = f32(f32(1.0) / np.sqrt(r2).astype(np.float32))
    arith = f32(qq.astype(np.float32) * f32(f32(rinv + f32(f32(krf) * r2)) - f32(crf)))
    return exact, arith


def test_float32_pair_energies_miss_the_energy_tolerance():
    p = wb.params_rf()
    err_arith, err_rounded = [], []
    for s in (wb.small_box(seed=1), wb.small_box(seed=2), wb.mid_box(seed=1), wb.mid_box(seed=2)):
        exact, arith = _rf_terms(s, p)
        e = math.fsum(exact.tolist())
        ref = oracle.energy_virial(s, p)["e_coul"]
        assert abs(e - ref) <= 1e-12 * abs(ref)  # the restated terms are the oracle's
        err_arith.append(abs(math.fsum(arith.astype(np.float64).tolist()) - e) / abs(e))
        rounded = exact.astype(np.float32).astype(np.float64)
        err_rounded.append(abs(math.fsum(rounded.tolist()) - e) / abs(e))
    assert max(err_arith) > 1e-6, err_arith
    assert max(err_rounded) < 1e-6, err_rounded
    assert max(err_rounded) > 1e-7, err_rounded
