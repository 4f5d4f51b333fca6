"""Algorithm 2 (TEFMM-II) tables of the reaction derivatives (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.2 builds the layered M2L from derivatives of the reaction components
computed not by complex images but from Sommerfeld integrals precomputed on a
grid and interpolated (eq. ``symmetricdetable``), with the in-plane
derivatives taken in the symmetric form of eq. ``sysdifferential``.  Here the
same idea serves the Cartesian derivative tables of Algorithm 1's M2L (Sec.
3.2-3.3).  A same-layer term tau of layer l, in the image-distance form of
``Medium.same_layer_terms`` (zeta = sz z + szp z' + c), is

    F_tau(X, Y, zeta) = (1/k) int_0^inf k_rho J_0(k_rho rho) e^{i k_z zeta} s_tau(k_rho) / k_z dk_rho,

rho = |(X, Y)|.  With D+- = d_x +- i d_y the identities of Sec. 4.2,
D+^a J_0(k rho) = (-k)^a J_a(k rho) e^{i a phi} and D-^b (J_a e^{i a phi}) =
k^b J_{a-b} e^{i (a-b) phi}, give D+^a D-^b J_0 = (-1)^a k^{a+b} J_{a-b} e^{i(a-b)phi}.
Writing d_x = (D+ + D-)/2, d_y = (D+ - D-)/(2i),

    a_g = D^g F / g! = (1/g!) sum_{a1 <= g1, a2 <= g2} c(a1, a2) (-1)^a e^{i (a-b) phi} T_{g1+g2, a-b, g3}(rho, zeta),
    c(a1, a2) = 2^-g1 (2i)^-g2 C(g1, a1) C(g2, a2) (-1)^(g2-a2),  a = a1 + a2,  b = g1 + g2 - a,
    T_{m, nu, n}(rho, zeta) = (1/k) int k_rho^{m+1} J_nu(k_rho rho) (i k_z)^n e^{i k_z zeta} s_tau / k_z dk_rho,

with T_{m,-nu,n} = (-1)^nu T_{m,nu,n}.  A table holds T_{m,nu,n} for
m <= 2p, 0 <= nu <= m (nu = m mod 2), n <= 2p - m on a uniform n x n grid
over rho in [0, rho_max] and zeta in [zeta_lo, zeta_hi], each value by the
contour quadrature of ``oracle.sommerfeld`` (the pinned path); a_g at a point
uses tensor-product Lagrange interpolation of degree 7 in each direction, the
stencil the 8 grid points around the point, shifted inside the grid at its
edges.  Each term of a layer has its own table.

Grid ranges (the "domain of interest" of Sec. 4.2): for the terms of layer l,
rho_max is the largest horizontal offset of the layer's same-layer M2L pairs
(all levels) and [zeta_lo, zeta_hi] the range of the term's image distance
over those pairs, computed from the box indices as the M2L tables do.  The
integral converges only for zeta > 0, and box centres of coarse levels can lie
beyond the layer's particle slab: a key whose image distance is below the
term's smallest one over the slab (zeta_min, the DCIM shift) keeps the images
of Algorithm 1 and stays out of the ranges.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from scipy.special import jv

from .medium import Medium, kz_branch
from .sommerfeld import contour_nodes
from .derivs import multi_indices

DEG = 7          # Lagrange degree per direction


def table_index(P2):
    """List of (m, nu, n) held by a table of order P2 = 2p, in storage order."""
    out = []
    for m in range(P2 + 1):
        for nu in range(m % 2, m + 1, 2):
            for n in range(P2 - m + 1):
                out.append((m, nu, n))
    return out


def quadrature_T(k, kmax, s, P2, rhos, zeta):
    """T_{m,nu,n}(rho, zeta) for every (m, nu, n) of table_index(P2) and every
    rho of rhos (one contour for the row), by quadrature; s(k_rho) is the term's
    s_tau.  Returns an array (len(rhos), len(table_index(P2)))."""
    rhos = np.atleast_1d(np.asarray(rhos, float))
    k = complex(k)
    nodes, weights = contour_nodes(kmax, zeta, max(float(rhos.max()), 1e-3), nd=P2 + 2)
    kz = kz_branch(k, nodes)
    ez = np.exp(1j * kz * zeta)
    with np.errstate(over='ignore', invalid='ignore'):
        sv = np.asarray(s(nodes), dtype=complex)
    # far out on the path a term's s_tau can come out as 0 * inf (an underflowed
    # density times an overflowed e^{-i k_z D}); there e^{i k_z zeta} k_rho^(P2+1)
    # is negligible, which is checked before those nodes are dropped
    bad = ~np.isfinite(sv)
    if bad.any():
        if np.max(np.abs(ez[bad]) * np.abs(nodes[bad]) ** (P2 + 1)) > 1e-30:
            raise FloatingPointError("s_tau not finite where the integrand is not negligible")
        sv[bad] = 0.0
    base = weights * nodes * sv * ez / kz / k
    idx = table_index(P2)
    out = np.zeros((len(rhos), len(idx)), dtype=complex)
    kzp = [(1j * kz) ** n for n in range(P2 + 1)]
    krp = [nodes ** m for m in range(P2 + 1)]
    for r, rho in enumerate(rhos):
        J = [jv(nu, nodes * rho) for nu in range(P2 + 1)]
        for e, (m, nu, n) in enumerate(idx):
            out[r, e] = np.sum(base * krp[m] * J[nu] * kzp[n])
    return out


def medium_T(med: Medium, l, tag, P2):
    """The T function of a same-layer term of layer l, for Alg2Table."""
    kmax = float(np.max(med.k.real))
    return lambda rhos, zeta: quadrature_T(med.k[l], kmax, lambda kr: med.s_tau(l, tag, kr), P2, rhos, zeta)


def grid(lo, hi, n):
    """The n uniform grid points lo + i (hi - lo) / (n - 1)."""
    step = (hi - lo) / (n - 1)
    return lo + step * np.arange(n)


def stencil(lo, hi, n, x):
    """First index and Lagrange weights of the DEG + 1 grid points around x."""
    step = (hi - lo) / (n - 1)
    i0 = int(math.floor((x - lo) / step)) - DEG // 2
    i0 = min(max(i0, 0), n - DEG - 1)
    xs = lo + step * np.arange(i0, i0 + DEG + 1)
    w = np.ones(DEG + 1)
    for a in range(DEG + 1):
        for b in range(DEG + 1):
            if a != b:
                w[a] *= (x - xs[b]) / (xs[a] - xs[b])
    return i0, w


class Alg2Table:
    """The grid of T_{m,nu,n} of one term (Algorithm 2's precomputed table).

    T_at(rhos, zeta) -> (len(rhos), n_entries) gives the values at grid points."""

    def __init__(self, T_at, P2, rho_max, zeta_lo, zeta_hi, n=64):
        if n < DEG + 1:
            raise ValueError("table needs at least 8 points per direction")
        self.P2 = P2
        self.idx = table_index(P2)
        self.pos = {t: i for i, t in enumerate(self.idx)}
        self.n = n
        self.rho_max, self.zeta_lo, self.zeta_hi = float(rho_max), float(zeta_lo), float(zeta_hi)
        self.rho = grid(0.0, self.rho_max, n)
        self.zeta = grid(self.zeta_lo, self.zeta_hi, n)
        self.T = np.zeros((n, n, len(self.idx)), dtype=complex)   # [i_rho][j_zeta][entry]
        for j, z in enumerate(self.zeta):
            self.T[:, j] = T_at(self.rho, z)

    def interp(self, rho, zeta):
        """All T_{m,nu,n} at (rho, zeta) by tensor-product Lagrange interpolation."""
        i0, wr = stencil(0.0, self.rho_max, self.n, rho)
        j0, wz = stencil(self.zeta_lo, self.zeta_hi, self.n, zeta)
        blk = self.T[i0:i0 + DEG + 1, j0:j0 + DEG + 1]
        return np.einsum('i,j,ijk->k', wr, wz, blk)

    def derivatives(self, X, Y, zeta, Tvals=None):
        """a_g = D^g F / g!, |g| <= 2p, at (X, Y, zeta) in the graded multi-index
        order, from interpolated (or given) T values."""
        if Tvals is None:
            Tvals = self.interp(math.hypot(X, Y), zeta)
        return assemble(self.P2, Tvals, math.atan2(Y, X))


@lru_cache(maxsize=None)
def assembly_terms(P2):
    """The sum defining a_g, as flat arrays over all (g, a1, a2): the index of
    g in the graded order, the T entry (m, |nu|, g3), nu, and the factor
    c(a1, a2) (-1)^a [(-1)^nu if nu < 0] / g!."""
    pos = {t: i for i, t in enumerate(table_index(P2))}
    gi, ti, nus, cs = [], [], [], []
    for i, (g1, g2, g3) in enumerate(multi_indices(P2)):
        g1, g2, g3 = int(g1), int(g2), int(g3)
        m = g1 + g2
        inv_fact = 1.0 / (math.factorial(g1) * math.factorial(g2) * math.factorial(g3))
        for a1 in range(g1 + 1):
            for a2 in range(g2 + 1):
                a = a1 + a2
                nu = a - (m - a)
                c = (0.5 ** g1) * (0.5 / 1j) ** g2 * math.comb(g1, a1) * math.comb(g2, a2) * \
                    (-1.0) ** (g2 - a2) * (-1.0) ** a
                if nu < 0:
                    c *= (-1.0) ** nu
                gi.append(i)
                ti.append(pos[(m, abs(nu), g3)])
                nus.append(nu)
                cs.append(c * inv_fact)
    return np.array(gi), np.array(ti), np.array(nus, float), np.array(cs, complex)


def assemble(P2, Tvals, phi):
    """Cartesian a_g = D^g F / g! from T_{m,nu,n} at one point (azimuth phi)."""
    gi, ti, nus, cs = assembly_terms(P2)
    out = np.zeros(len(multi_indices(P2)), dtype=complex)
    np.add.at(out, gi, cs * np.exp(1j * nus * phi) * np.asarray(Tvals)[ti])
    return out


def layer_ranges(med: Medium, l, keys, floor):
    """Grid ranges of the terms of layer l from its same-layer M2L keys.

    keys: iterable of (h, dix, diy, diz, zsum) per translation, zsum the sum of
    the two box centres' z.  ud/du terms use zeta = sz dz + c (dz = diz h),
    uu/dd zeta = sz zsum + c.  floor: {tag: the term's smallest image distance
    over the layer's particle slab (its DCIM shift zeta_min)}; a key below it
    (box centres beyond the slab, where the integral may diverge) is left to
    the images and does not count.  Returns (rho_max, {tag: (zeta_lo,
    zeta_hi)}) over the keys that use the tables."""
    rho_max = 0.0
    rng = {}
    for h, dix, diy, diz, zsum in keys:
        rho = math.hypot(dix * h, diy * h)
        for tag, sz, szp, c in med.same_layer_terms(l):
            zeta = sz * (diz * h) + c if tag in ('ud', 'du') else sz * zsum + c
            if not zeta >= floor[tag]:
                continue
            rho_max = max(rho_max, rho)
            lo, hi = rng.get(tag, (math.inf, -math.inf))
            rng[tag] = (min(lo, zeta), max(hi, zeta))
    if rho_max == 0.0:
        rho_max = 1.0
    for tag, (lo, hi) in rng.items():
        if hi == lo:
            rng[tag] = (lo, lo + 1.0)
    return rho_max, rng
