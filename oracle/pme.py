"""Long-range (reciprocal-space) Ewald electrostatics for the oracle.

TEST INFRASTRUCTURE ONLY: the tests and the smoke check are the only
callers.  The CUDA library neither imports nor calls anything here, and
nothing here is shared with it.

The paper runs the long-range part of the electrostatics with particle-mesh
Ewald (PME) next to the short-range pair kernel (the multi-level parallelism
figure and the long-range discussion of the introduction) without stating its
equations.  The reading taken here is the smooth PME of the standard
literature, for a periodic cell with lattice vectors as the rows of B
(a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz); diagonal for a rectangular box
of edges L) and Gaussian splitting parameter beta (the same beta as the
real-space erfc term).  Wave vectors are m = k B^-T for integer k (k / L in a
rectangular box), V = det B, and the mesh coordinates of a position x are
u = x B^-1 diag(K):

  reciprocal energy (exact Ewald sum, `ewald_reciprocal_direct`):
    E_rec = f / (2 pi V) sum_{m != 0} exp(-pi^2 m^2 / beta^2) / m^2 |S(m)|^2,
    S(m) = sum_j q_j exp(2 pi i m . r_j);
  PME (`pme`): the structure factor from charges spread on a K1 x K2 x K3
    grid with cardinal B-splines M_p of order p,
      Q(n) = sum_j q_j prod_d M_p(u_jd - n_d),  u_j = x_j B^-1 diag(K) (periodic),
    E_rec ~ 1/2 sum_m B(m) C(m) |DFT(Q)(m)|^2 with C(m) the summand above
    without |S|^2 (C(0) = 0) and B(m) = prod_d |b_d(m_d)|^2 the B-spline
    moduli, |b(k)|^-2 = |sum_{j=0}^{p-2} M_p(j + 1) exp(2 pi i k j / K)|^2;
    forces F_j = -dE_rec/dr_j = -q_j (dE/du_j) diag(K) B^-T through the
    splines' derivatives; the mesh index K/2 of an even mesh is the signed
    frequency +K/2;
  self energy   E_self = -f beta / sqrt(pi) sum_j q_j^2;
  excluded pairs (inside a molecule; the reciprocal sum includes them):
    E_excl = -f sum_{excluded i<j} q_i q_j erf(beta r) / r, with its forces;
  virial (Xi = -1/2 sum r (x) F convention of the short-range part):
    Xi_rec = -1/2 sum_m E_m (delta - 2 (1 + pi^2 m^2 / beta^2) m m / m^2),
    E_m the energy of wave vector m.

Everything is float64; the DFT is numpy's (a library primitive).  Pins in
tests/test_pme_oracle.py: the Madelung constant of rock salt (real space +
exact reciprocal sum + self term), two molecules far from their images
against plain Coulomb (which needs the excluded-pair term), the homogeneity
identity trace(virial) = -E/2 of the full Ewald sum, every virial component
against the energy of a deformed (sheared) box, convergence of PME to the
exact sum as the grid refines and the order rises, PME forces and virial
against finite differences of the PME energy, and B-spline identities; for
triclinic cells, the Madelung constant of rock salt in its two-ion primitive
(fcc) cell, the reciprocal sum unchanged under a change of basis of the same
lattice, PME convergence and derivatives in a rhombic dodecahedron, and the
minimum image of excluded pairs.
"""
from __future__ import annotations

import math

import numpy as np


def _box_rows(sys) -> np.ndarray:
    """The lattice vectors as rows: a = (ax, 0, 0), b = (bx, by, 0), c = (cx, cy, cz);
    rectangular when the system has no skew."""
    L = np.asarray(sys.box, dtype=np.float64)
    sk = np.asarray(getattr(sys, "skew", np.zeros(3)), dtype=np.float64)
    return np.array([[L[0], 0.0, 0.0], [sk[0], L[1], 0.0], [sk[1], sk[2], L[2]]])


def _is_rectangular(sys) -> bool:
    return not np.any(np.asarray(getattr(sys, "skew", np.zeros(3))) != 0.0)


def _mesh_matrix(sys, K) -> np.ndarray:
    """M with u = x M the mesh coordinates of a position x (row vector):
    M = B^-1 diag(K), B the box rows; diag(K / L) for a rectangular box."""
    K = np.asarray(K, dtype=np.float64)
    if _is_rectangular(sys):
        return np.diag(K / np.asarray(sys.box, dtype=np.float64))
    return np.linalg.inv(_box_rows(sys)) * K[None, :]


def _recip(sys) -> np.ndarray:
    """B^-1: a wave vector of integer indices k (row) is m = k B^-T."""
    if _is_rectangular(sys):
        return np.diag(1.0 / np.asarray(sys.box, dtype=np.float64))
    return np.linalg.inv(_box_rows(sys))


def bspline(x: np.ndarray, p: int) -> np.ndarray:
    """Cardinal B-spline M_p(x) (support (0, p)) by the recursion
    M_n(x) = x/(n-1) M_{n-1}(x) + (n-x)/(n-1) M_{n-1}(x-1), M_2(x) = 1 - |x - 1|."""
    x = np.asarray(x, dtype=np.float64)
    if p == 2:
        return np.where((x >= 0) & (x <= 2), 1.0 - np.abs(x - 1.0), 0.0)
    return x / (p - 1) * bspline(x, p - 1) + (p - x) / (p - 1) * bspline(x - 1.0, p - 1)


def bspline_deriv(x: np.ndarray, p: int) -> np.ndarray:
    """dM_p/dx = M_{p-1}(x) - M_{p-1}(x - 1)."""
    return bspline(x, p - 1) - bspline(np.asarray(x) - 1.0, p - 1)


def bspline_moduli(K: int, p: int) -> np.ndarray:
    """|b(k)|^2 for k = 0..K-1."""
    j = np.arange(p - 1)
    w = bspline(j + 1.0, p)
    k = np.arange(K)[:, None]
    den = (w[None, :] * np.exp(2j * np.pi * k * j[None, :] / K)).sum(1)
    return 1.0 / np.abs(den) ** 2


def _signed(K: int) -> np.ndarray:
    """Signed frequency of mesh index k: k for k <= K/2, k - K above (the
    index K/2 of an even mesh is +K/2)."""
    k = np.arange(K)
    return np.where(k <= K // 2, k, k - K).astype(np.float64)


def pme(sys, params, grid=(32, 32, 32), order: int = 4, sel=None) -> dict:
    """Reciprocal energy, forces [n, 3] (of the atoms sel only, if given) and
    virial (3x3) by smooth PME.

    Even orders only: for odd p the modulus sum vanishes at k = K/2 (even K),
    where |b|^2 has a pole."""
    if order % 2:
        raise ValueError("PME order must be even")
    x = sys.x.astype(np.float64)
    q = sys.q.astype(np.float64)
    K = np.asarray(grid, dtype=np.int64)
    f = params.fcoul / params.eps_r
    beta = params.beta
    p = order
    M = _mesh_matrix(sys, K)
    u = x @ M                              # mesh coordinates, periodic modulo K
    u = u - K * np.floor(u / K)
    base = np.floor(u).astype(np.int64)
    frac = u - base
    j = np.arange(p)
    # grid point base - j carries weight M_p(frac + j)
    w = np.stack([bspline(frac[:, d, None] + j[None, :], p) for d in range(3)], axis=1)      # [n, 3, p]
    dw = np.stack([bspline_deriv(frac[:, d, None] + j[None, :], p) for d in range(3)], axis=1)
    idx = np.stack([np.mod(base[:, d, None] - j[None, :], K[d]) for d in range(3)], axis=1)  # [n, 3, p]
    Q = np.zeros(int(np.prod(K)))
    for a in range(p):
        for b in range(p):
            for c in range(p):
                flat = (idx[:, 0, a] * K[1] + idx[:, 1, b]) * K[2] + idx[:, 2, c]
                Q += np.bincount(flat, weights=q * w[:, 0, a] * w[:, 1, b] * w[:, 2, c], minlength=Q.size)
    Q = Q.reshape(tuple(K))
    F = np.fft.fftn(Q)
    kx, ky, kz = np.meshgrid(_signed(K[0]), _signed(K[1]), _signed(K[2]), indexing="ij")
    R = _recip(sys)
    # m = k B^-T: m_a = sum_d k_d (B^-1)[a, d]
    mx = kx * R[0, 0] + ky * R[0, 1] + kz * R[0, 2]
    my = kx * R[1, 0] + ky * R[1, 1] + kz * R[1, 2]
    mz = kx * R[2, 0] + ky * R[2, 1] + kz * R[2, 2]
    m2 = mx * mx + my * my + mz * mz
    V = float(abs(np.linalg.det(_box_rows(sys))))
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.where(m2 > 0, f * np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * V * m2), 0.0)
    B = (bspline_moduli(K[0], p)[:, None, None] * bspline_moduli(K[1], p)[None, :, None]
         * bspline_moduli(K[2], p)[None, None, :])
    G = B * C
    Em = 0.5 * G * np.abs(F) ** 2
    energy = float(Em.sum())
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(m2 > 0, 2.0 * (1.0 + np.pi ** 2 * m2 / beta ** 2) / m2, 0.0)
    mv = (mx, my, mz)
    W = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            W[a, b] = float((Em * ((1.0 if a == b else 0.0) - s * mv[a] * mv[b])).sum())
    virial = -0.5 * W
    phi = np.prod(K) * np.real(np.fft.ifftn(G * F))   # dE/dQ(n)
    if sel is not None:
        sel = np.asarray(sel)
        q, w, dw, idx = q[sel], w[sel], dw[sel], idx[sel]
    # dE/du_d per atom, then F = -q (dE/du) M^T
    g = np.zeros((q.shape[0], 3))
    for a in range(p):
        for b in range(p):
            for c in range(p):
                ph = phi[idx[:, 0, a], idx[:, 1, b], idx[:, 2, c]]
                g[:, 0] += ph * dw[:, 0, a] * w[:, 1, b] * w[:, 2, c]
                g[:, 1] += ph * w[:, 0, a] * dw[:, 1, b] * w[:, 2, c]
                g[:, 2] += ph * w[:, 0, a] * w[:, 1, b] * dw[:, 2, c]
    forces = -(q[:, None] * g) @ M.T
    return {"energy": energy, "forces": forces, "virial": virial}


def ewald_reciprocal_direct(sys, params, kmax: int) -> dict:
    """The exact Ewald reciprocal sum over |k_d| <= kmax (m = k B^-T, k integer)."""
    x = sys.x.astype(np.float64)
    q = sys.q.astype(np.float64)
    f = params.fcoul / params.eps_r
    beta = params.beta
    V = float(abs(np.linalg.det(_box_rows(sys))))
    k = np.arange(-kmax, kmax + 1)
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    keep = (kx != 0) | (ky != 0) | (kz != 0)
    kv = np.stack([kx[keep], ky[keep], kz[keep]], axis=1).astype(np.float64)
    m = kv @ _recip(sys).T                                                    # [M, 3], m = k B^-T
    m2 = (m * m).sum(1)
    c = f * np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * V * m2)           # [M]
    energy = 0.0
    forces = np.zeros_like(x)
    W = np.zeros((3, 3))
    s = 2.0 * (1.0 + np.pi ** 2 * m2 / beta ** 2) / m2
    for lo in range(0, m.shape[0], 512):
        mm = m[lo:lo + 512]
        arg = 2.0 * np.pi * (x @ mm.T)                                       # [n, b]
        cs, sn = np.cos(arg), np.sin(arg)
        Sr, Si = q @ cs, q @ sn                                              # [b]
        cc = c[lo:lo + 512]
        Em = 0.5 * cc * (Sr * Sr + Si * Si)
        energy += float(Em.sum())
        # dE/dr_j = sum_m c q_j 2 pi m (-sin Sr + cos Si)
        g = q[:, None] * (-sn * Sr[None, :] + cs * Si[None, :]) * (2.0 * np.pi) * cc[None, :]
        forces -= g @ mm
        ss = s[lo:lo + 512]
        for a in range(3):
            for b in range(3):
                W[a, b] += float((Em * ((1.0 if a == b else 0.0) - ss * mm[:, a] * mm[:, b])).sum())
    return {"energy": energy, "forces": forces, "virial": -0.5 * W}


def ewald_self(sys, params) -> float:
    """-f beta / sqrt(pi) sum q^2."""
    q = sys.q.astype(np.float64)
    return float(-params.fcoul / params.eps_r * params.beta / math.sqrt(math.pi) * (q * q).sum())


def ewald_exclusions(sys, params) -> dict:
    """Energy, forces and virial of -f q_i q_j erf(beta r) / r over the excluded
    pairs (each unordered pair once; minimum image of the box)."""
    x = sys.x.astype(np.float64)
    q = sys.q.astype(np.float64)
    L = np.asarray(sys.box, dtype=np.float64)
    f = params.fcoul / params.eps_r
    beta = params.beta
    counts = np.diff(np.asarray(sys.excl_index, dtype=np.int64))
    i = np.repeat(np.arange(sys.n), counts)
    j = np.asarray(sys.excl_atoms, dtype=np.int64)[: i.shape[0]]
    # each unordered pair once, whether the list names it under one atom or both
    pairs = np.unique(np.stack([np.minimum(i, j), np.maximum(i, j)], axis=1)[i != j], axis=0)
    i, j = pairs[:, 0], pairs[:, 1]
    d = x[i] - x[j]
    if _is_rectangular(sys):
        d -= L * np.round(d / L)
    else:
        # reduce by c, b, a, then the shortest of the 27 neighbouring images
        B = _box_rows(sys)
        for row in (2, 1, 0):
            d -= np.round(d[:, row] / B[row, row])[:, None] * B[row]
        best = d.copy()
        for s1 in (-1, 0, 1):
            for s2 in (-1, 0, 1):
                for s3 in (-1, 0, 1):
                    cand = d + s1 * B[0] + s2 * B[1] + s3 * B[2]
                    better = (cand * cand).sum(1) < (best * best).sum(1)
                    best[better] = cand[better]
        d = best
    r = np.sqrt((d * d).sum(1))
    qq = f * q[i] * q[j]
    erf_br = np.array([math.erf(v) for v in beta * r])
    energy = float(-(qq * erf_br / r).sum())
    # V = -qq erf(br)/r; dV/dr = -qq (2b/sqrt(pi) exp(-b^2 r^2) / r - erf(br)/r^2); F_i = -dV/dr d / r
    dvdr = -qq * (2.0 * beta / math.sqrt(math.pi) * np.exp(-beta * beta * r * r) / r - erf_br / (r * r))
    fi = -(dvdr / r)[:, None] * d
    forces = np.zeros_like(x)
    for c in range(3):
        forces[:, c] = np.bincount(i, weights=fi[:, c], minlength=sys.n) - \
            np.bincount(j, weights=fi[:, c], minlength=sys.n)
    virial = -0.5 * np.einsum("pa,pb->ab", d, fi)
    return {"energy": energy, "forces": forces, "virial": virial}
