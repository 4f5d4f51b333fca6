"""Contour quadrature of the Sommerfeld integrals (oracle truth for u^up/u^down).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 2.1 (eq. ``greenfuncomponent`` and ``totaldensity``), with the
factor i k_l / (4 pi) omitted as in Sec. 3.1, so that

    u^up_{l l'}(r, r')   = (1/k_l) int_0^inf k_rho J0(k_rho rho) e^{ i k_lz (z - d_l)} / k_lz * sigma~^up(k_rho, z')   dk_rho
    u^down_{l l'}(r, r') = (1/k_l) int_0^inf k_rho J0(k_rho rho) e^{-i k_lz (z - d_l)} / k_lz * sigma~^down(k_rho, z') dk_rho

with sigma~^up = S2 sigma^{uu} + S1 sigma^{ud}, sigma~^down = S2 sigma^{du} +
S1 sigma^{dd}, S1 = e^{i k_l'z (d_{l'-1} - z')}, S2 = e^{i k_l'z (z' - d_l')}.

Derivatives (Sec. 3.3 and Sec. 4.2): d/dz acts on the target exponential,
d/dz' on S1, S2 (eq. ``layermediumdensity``), and the in-plane operator uses
(d/dx + i d/dy)^s J0(k_rho rho) = (-k_rho)^s J_s(k_rho rho) e^{i s theta}.

Path: a semi-ellipse in the fourth quadrant of the k_rho plane from 0 to 2a,
beyond every branch point Re k_m, followed by the real axis [2a, K_max] where
the integrand decays like e^{-k_rho h} (h = total vertical travel distance).
Gauss-Legendre panels on both pieces.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import jv

from .medium import Medium, kz_branch


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def contour_nodes(kmax_re, h, rho, n_ell_panels=48, n_nodes=24, depth=0.6,
                  extra_decades=40.0, nd=0):
    """Nodes and weights (complex) along the deformed Sommerfeld path."""
    a = 0.5 * kmax_re + 0.75
    b = depth
    xg, wg = _gl(n_nodes)
    nodes, weights = [], []
    edges = np.linspace(0.0, math.pi, n_ell_panels + 1)
    for lo, hi in zip(edges[:-1], edges[1:]):
        t = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
        wt = 0.5 * (hi - lo) * wg
        kr = a * (1 - np.cos(t)) - 1j * b * np.sin(t)
        dk = a * np.sin(t) - 1j * b * np.cos(t)
        nodes.append(kr)
        weights.append(wt * dk)
    k0 = 2 * a
    h = max(h, 1e-3)
    # e^{-K h} K^nd below 1e-40 relative to the peak
    kend = k0 + (extra_decades * math.log(10) + nd * math.log(max(nd, 1) / h + 10.0) + 10.0) / h
    width = min(0.5, 1.0 / max(rho, 1e-6), 0.5 / h)
    npan = int(math.ceil((kend - k0) / width))
    edges = k0 + width * np.arange(npan + 1)
    for lo, hi in zip(edges[:-1], edges[1:]):
        t = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
        nodes.append(t.astype(complex))
        weights.append((0.5 * (hi - lo) * wg).astype(complex))
    return np.concatenate(nodes), np.concatenate(weights)


def reaction_derivative(med: Medium, l, lp, r, rp, s=0, k3=0, k3p=0, part='both',
                        **path_kw):
    """(d_x + i d_y)^s d_z^k3 d_z'^k3p u_{l l'}^{part} / (s! k3! k3p!) by quadrature.

    ``part`` is 'up', 'down' or 'both' (the full reaction field u^up + u^down).
    Returns a complex number in the paper's normalisation (i k_l/4pi omitted).
    """
    r = np.asarray(r, float)
    rp = np.asarray(rp, float)
    dx, dy = r[0] - rp[0], r[1] - rp[1]
    rho = math.hypot(dx, dy)
    theta = math.atan2(dy, dx)
    z, zp = r[2], rp[2]
    L = med.L
    d = med.d
    # total vertical distances of the exponentials (decay rate on the real tail)
    hs = []
    parts = []
    if part in ('up', 'both') and l < L:
        parts.append('up')
    if part in ('down', 'both') and l > 0:
        parts.append('down')
    for pt in parts:
        zt = (z - d[l]) if pt == 'up' else (d[l - 1] - z)
        if lp > 0:
            hs.append(zt + d[lp - 1] - zp)
        if lp < L:
            hs.append(zt + zp - d[lp])
    h = min(hs)
    kmax = float(np.max(med.k.real))
    nodes, weights = contour_nodes(kmax, h, rho, nd=s + k3 + k3p + 2, **path_kw)
    sig = med.densities(lp, nodes, basis='solve')
    kzl = kz_branch(med.k[l], nodes)
    kzp = kz_branch(med.k[lp], nodes)
    total = np.zeros(nodes.shape, dtype=complex)
    for pt in parts:
        if pt == 'up':
            tgt_exp = 1j * kzl * (z - d[l])
            tgt_fac = (1j * kzl) ** k3
            keys = (('uu', 'S2'), ('ud', 'S1'))
        else:
            # solve basis: down-going wave referenced to the top interface
            tgt_exp = -1j * kzl * (z - d[l - 1])
            tgt_fac = (-1j * kzl) ** k3
            keys = (('du', 'S2'), ('dd', 'S1'))
        for tag, src in keys:
            key = (l, tag)
            if key not in sig:
                continue
            if src == 'S1':
                if lp == 0:
                    continue
                sexp = 1j * kzp * (d[lp - 1] - zp)
                sfac = (-1j * kzp) ** k3p
            else:
                if lp == L:
                    continue
                sexp = 1j * kzp * (zp - d[lp])
                sfac = (1j * kzp) ** k3p
            total = total + tgt_fac * sfac * np.exp(tgt_exp + sexp) * sig[key]
    radial = nodes * (-nodes) ** s * jv(s, nodes * rho) / kzl
    val = np.sum(weights * radial * total) / med.k[l]
    val *= np.exp(1j * s * theta)
    val /= math.factorial(s) * math.factorial(k3) * math.factorial(k3p)
    return complex(val)


def free_space_by_quadrature(k, r, rp, **path_kw):
    """h0(k|r - r'|) = (1/k) int k_rho J0(k_rho rho) e^{i k_z |z - z'|}/k_z dk_rho.

    The Sommerfeld identity of Sec. 3.3, evaluated numerically (homogeneous
    medium check of the quadrature path).
    """
    r = np.asarray(r, float)
    rp = np.asarray(rp, float)
    rho = math.hypot(r[0] - rp[0], r[1] - rp[1])
    h = abs(r[2] - rp[2])
    nodes, weights = contour_nodes(float(np.real(k)), h, rho, **path_kw)
    kz = kz_branch(k, nodes)
    val = np.sum(weights * nodes * jv(0, nodes * rho) * np.exp(1j * kz * h) / kz) / k
    return complex(val)


def h0(kR):
    """Spherical Hankel function of the first kind, order 0: e^{iz}/(iz)."""
    return np.exp(1j * kR) / (1j * kR)
