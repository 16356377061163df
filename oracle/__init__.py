"""Python access to the FP64 oracle (nb_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only callers.  The CUDA library neither imports nor
calls anything here.

Each function takes the float32 inputs that the CUDA path receives and
promotes them exactly to float64 before calling the C code.

Pins (tests/test_oracle_pins.py): every function here is checked against the
two-particle closed forms, Newton's third law, translation and axis
permutation invariance, central finite differences of its own energy
(forces and all six virial components via box deformation), the
Lennard-Jones and Coulomb virial identities, tabulated erfc values, and a
brute-force 27-image pair enumeration on small boxes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libnb_oracle.so")
_lib = None

RF = 0
EWALD = 1
# potential modifiers (bits of Params.modifiers; nb_oracle.c documents them)
MOD_LJ_SHIFT = 1
MOD_EWALD_SHIFT = 2
MOD_RF_EXCL = 4


def build(force: bool = False) -> str:
    """Compile nb_oracle.c with gcc (OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-ffp-contract=off",
           "-D_GNU_SOURCE",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lp = ctypes.POINTER(ctypes.c_longlong)
    common = [ctypes.c_int, dp, dp, ip, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, ip, ip, ctypes.c_int]
    lib.or_energy_virial.argtypes = common + [dp, lp]
    lib.or_energy_virial.restype = ctypes.c_int
    lib.or_energy_virial_rows.argtypes = common + [ctypes.c_int, ctypes.c_int, dp, lp]
    lib.or_energy_virial_rows.restype = ctypes.c_int
    lib.or_forces.argtypes = common + [ctypes.c_int, ip, dp]
    lib.or_forces.restype = ctypes.c_int
    lib.or_pairs.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ip, ip, lp, ip]
    lib.or_pairs.restype = ctypes.c_longlong
    lib.or_pairs_rows.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ip, ip, ctypes.c_int, ip, lp, ip]
    lib.or_pairs_rows.restype = ctypes.c_longlong
    lib.or_num_threads.argtypes = []
    lib.or_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _box6(sys):
    """(ax, by, cz, bx, cx, cy): the box and the off-diagonal components of a
    triclinic box (zeros for a rectangular one)."""
    skew = getattr(sys, "skew", None)
    skew = np.zeros(3) if skew is None else np.asarray(skew, dtype=np.float64)
    return _d(np.concatenate([np.asarray(sys.box, dtype=np.float64), skew]))


def _common(sys, params):
    x, xp = _d(sys.x.astype(np.float64))
    q, qp = _d(sys.q.astype(np.float64))
    t, tp = _i(sys.type)
    b, bp = _box6(sys)
    c6, c6p = _d(np.asarray(params.c6, dtype=np.float64))
    c12, c12p = _d(np.asarray(params.c12, dtype=np.float64))
    ei, eip = _i(sys.excl_index)
    ea, eap = _i(sys.excl_atoms)
    keep = (x, q, t, b, c6, c12, ei, ea)
    args = [sys.n, xp, qp, tp, bp, float(params.rc), int(params.coul), float(params.eps_r),
            float(params.eps_rf), float(params.beta), float(params.fcoul), int(params.ntypes),
            c6p, c12p, eip, eap, int(getattr(params, "modifiers", 0))]
    return keep, args


def energy_virial(sys, params) -> dict:
    """E_LJ, E_C (kJ/mol), virial 3x3 and diagnostic sums over all pairs."""
    lib = _load()
    keep, args = _common(sys, params)
    out = np.zeros(15, dtype=np.float64)
    npairs = ctypes.c_longlong(0)
    rc = lib.or_energy_virial(*args, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              ctypes.byref(npairs))
    if rc != 0:
        raise RuntimeError("oracle energy_virial failed")
    del keep
    return _ev_dict(out, npairs.value)


def energy_virial_rows(sys, params, i0: int, i1: int) -> tuple:
    """The raw sums of energy_virial over the pairs (i, j), i0 <= i < i1, j > i:
    (float64 [15] in the C layout, pair count).  Sums over consecutive row
    ranges covering [0, n) add up to energy_virial's (see ev_from_sums)."""
    lib = _load()
    keep, args = _common(sys, params)
    out = np.zeros(15, dtype=np.float64)
    npairs = ctypes.c_longlong(0)
    rc = lib.or_energy_virial_rows(*args, int(i0), int(i1), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(npairs))
    if rc != 0:
        raise RuntimeError("oracle energy_virial_rows failed")
    del keep
    return out, int(npairs.value)


def ev_from_sums(out, npairs: int) -> dict:
    """energy_virial's dictionary from summed raw sums of energy_virial_rows."""
    return _ev_dict(np.asarray(out, dtype=np.float64), npairs)


def _ev_dict(out, npairs: int) -> dict:
    return {"e_lj": out[0], "e_coul": out[1], "virial": out[2:11].reshape(3, 3).copy(),
            "e12": out[11], "e6": out[12], "rdotf_lj": out[13], "rdotf_coul": out[14],
            "npairs": int(npairs)}


def forces(sys, params, sel=None) -> np.ndarray:
    """Total force (float64 [k, 3]) on each selected atom (all atoms if sel is None)."""
    lib = _load()
    keep, args = _common(sys, params)
    if sel is None:
        nsel, s, sp = sys.n, None, None
    else:
        s, sp = _i(np.asarray(sel))
        nsel = int(s.shape[0])
    f = np.zeros((nsel, 3), dtype=np.float64)
    rc = lib.or_forces(*args, nsel, sp, f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError("oracle forces failed")
    del keep, s
    return f


def pairs(sys, r_cut: float) -> np.ndarray:
    """Sorted int64 keys i * n + j of all non-excluded pairs i < j with r < r_cut."""
    lib = _load()
    x, xp = _d(sys.x.astype(np.float64))
    b, bp = _box6(sys)
    ei, eip = _i(sys.excl_index)
    ea, eap = _i(sys.excl_atoms)
    counts = np.zeros(sys.n, dtype=np.int64)
    cp = counts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    total = lib.or_pairs(sys.n, xp, bp, float(r_cut), eip, eap, cp, None)
    if total < 0:
        raise RuntimeError("oracle pairs failed")
    out = np.zeros((max(total, 1), 2), dtype=np.int32)
    got = lib.or_pairs(sys.n, xp, bp, float(r_cut), eip, eap, cp,
                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if got != total:
        raise RuntimeError("oracle pairs count mismatch")
    out = out[:total].astype(np.int64)
    return out[:, 0] * sys.n + out[:, 1]


def pairs_of_rows(sys, r_cut: float, sel) -> np.ndarray:
    """Sorted unique int64 keys min(i,j) * n + max(i,j) of every non-excluded pair
    with r < r_cut that has at least one atom in `sel` (O(N) per selected atom)."""
    lib = _load()
    x, xp = _d(sys.x.astype(np.float64))
    b, bp = _box6(sys)
    ei, eip = _i(sys.excl_index)
    ea, eap = _i(sys.excl_atoms)
    s, sp = _i(np.asarray(sel))
    nsel = int(s.shape[0])
    counts = np.zeros(max(nsel, 1), dtype=np.int64)
    cp = counts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    total = lib.or_pairs_rows(sys.n, xp, bp, float(r_cut), eip, eap, nsel, sp, cp, None)
    if total < 0:
        raise RuntimeError("oracle pairs_of_rows failed")
    out = np.zeros((max(total, 1), 2), dtype=np.int32)
    got = lib.or_pairs_rows(sys.n, xp, bp, float(r_cut), eip, eap, nsel, sp, cp,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if got != total:
        raise RuntimeError("oracle pairs_of_rows count mismatch")
    out = out[:total].astype(np.int64)
    return np.unique(out[:, 0] * sys.n + out[:, 1])


def num_threads() -> int:
    return int(_load().or_num_threads())
