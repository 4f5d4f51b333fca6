"""Two-level discrete complex image fits (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 3.3, Steps 1-3 (eqs. ``compleximageapp`` and
``closedformgreen``):

* Step 1: sample the density on two paths in the k_lz plane,
      C_ap1: k_lz = i k_l (T0 + t),          0 <= t <= T1   (1st level)
      C_ap2: k_lz = k_l (1 - t/T0 + i t),     0 <= t <= T0   (2nd level)
  with T0 = sqrt(((max_m Re k_m + 0.8)/Re k_l)^2 - 1), T1 = 10 and 101
  samples per level (Sec. 3.3, the Table 3.1 set-up).
* Step 2: approximate the samples by sum_j A_j e^{-i k_lz Z_j} with the
  generalized pencil-of-function method (GPOF; Hua & Sarkar 1989): first level
  on C_ap1, then (reading: the standard two-level procedure) the first-level
  images are subtracted from the C_ap2 samples and the rest is fitted there.
* Step 3: the Sommerfeld identity turns every image into a free-space Hankel
  function at a complex distance, A_j h0(k_l sqrt(rho^2 + (w - Z_j)^2)).

Same-layer reading: the reaction field of u_ll splits into terms tau with a
real image distance zeta_tau (see ``Medium.same_layer_terms``); each term is
fitted once, as F_tau(k_z) = s_tau(k_rho) e^{i k_z zeta_min,tau}, so that

    u_tau(r, r') ~= sum_j A_j h0(k_l sqrt(rho^2 + (zeta_tau(z,z') - zeta_min,tau - Z_j)^2)).

GPOF parameters (the paper does not state them): pencil parameter N/2, model
order = number of singular values above ``rel_tol`` * sigma_max, capped per
level; the images of both levels together are at most ``n_images``; images
with Re Z >= 0 are dropped (see ``fit_two_level``).
"""
from __future__ import annotations

import math

import numpy as np

from .medium import Medium, kz_branch


def default_T0(med: Medium, l):
    kmax = float(np.max(med.k.real))
    kl = float(med.k[l].real)
    return math.sqrt(max(((kmax + 0.8) / kl) ** 2 - 1.0, 1e-6))


ABS_TOL = 1e-14


CANCEL = 1e4     # largest image term on the sampled paths / largest sample


def _hankel_svd(y):
    y = np.asarray(y, dtype=complex)
    N = y.size
    Lp = N // 2
    Y = np.array([y[i:i + Lp + 1] for i in range(N - Lp)])     # (N-Lp) x (Lp+1)
    _, S, Vh = np.linalg.svd(Y)
    return S, Vh.conj().T


def _poles(V, m):
    Vm = V[:, :m]                                              # (Lp+1) x m
    V1, V2 = Vm[:-1, :], Vm[1:, :]
    return np.linalg.eigvals(V2.conj().T @ np.linalg.pinv(V1.conj().T))


def gpof(y, m_max, rel_tol=1e-12, decaying=False, keep=None, accept=None, score=None):
    """Generalized pencil of function: y_n ~= sum_j b_j z_j^n.

    Returns (z, b).  Largest model order: the number of singular values of the
    Hankel data matrix above max(rel_tol * sigma_0, ABS_TOL * N) (the sampled
    functions are O(1), so anything below the absolute floor is rounding
    noise), at most m_max.  With ``decaying`` only poles with |z| < 1 are kept
    (images that decay along the first-level path); ``keep(z)`` (a boolean
    mask) drops further poles before the amplitudes are fitted.  ``accept(z,
    b)`` may reject a model order.  Without ``score`` the largest accepted
    order is returned; with it, every order from the largest down to 1 is
    tried and the accepted one with the smallest ``score(z, b)`` wins (ties:
    the larger order).
    """
    y = np.asarray(y, dtype=complex)
    N = y.size
    S, V = _hankel_svd(y)
    m = int(min(m_max, np.count_nonzero(S > max(rel_tol * S[0], ABS_TOL * N))))
    best, best_s = None, np.inf
    while m > 0:
        z = _poles(V, m)
        if decaying:
            z = z[np.abs(z) < 1.0]
        if keep is not None and z.size:
            z = z[keep(z)]
        if z.size:
            vand = z[None, :] ** np.arange(N)[:, None]
            b, *_ = np.linalg.lstsq(vand, y, rcond=None)
            if accept is None or accept(z, b):
                if score is None:
                    return z, b
                sc = score(z, b)
                if sc < best_s:
                    best, best_s = (z, b), sc
        m -= 1
    if best is not None:
        return best
    return np.zeros(0, complex), np.zeros(0, complex)


def sample_paths(k, T0, T1, n):
    """k_lz samples on C_ap1 and C_ap2 and their steps (Step 1)."""
    t1 = np.linspace(0.0, T1, n)
    t2 = np.linspace(0.0, T0, n)
    kz1 = 1j * k * (T0 + t1)
    kz2 = k * (1.0 - t2 / T0 + 1j * t2)
    return kz1, kz2, T1 / (n - 1), T0 / (n - 1)


def fit_two_level(F, k, T0, T1=10.0, n=101, n_images=8, m1=None, rel_tol=1e-12):
    """Fit F(k_z) ~= sum_j A_j e^{-i k_z Z_j} (Steps 1-2).  Returns (A, Z, info)."""
    k = complex(k)
    kz1, kz2, dt1, dt2 = sample_paths(k, T0, T1, n)
    y1 = F(kz1)
    y2 = F(kz2)
    if m1 is None:
        m1 = n_images // 2
    # Only images with Re Z < 0 are kept: the Sommerfeld identity that turns an
    # image into h0 at the complex distance W - W_min - Z needs Re(W - W_min - Z)
    # > 0 for every W >= W_min.  A model order is accepted only if no image term
    # exceeds CANCEL times the sampled data on either path: the image sums then
    # lose at most four digits to cancellation, so two FP64 evaluations of the
    # same images agree to ~1e-12 (with 1e6 they differed by 1e-10); among the
    # accepted orders the one with
    # the smallest sample residual is taken (level 1: on C_ap1; level 2: of all
    # images on both paths), since an ill-conditioned pencil at a high order
    # can give a poor fit.  These are readings; the paper does not discuss
    # GPOF's model order.
    scale = max(np.max(np.abs(y1)), np.max(np.abs(y2)), 1e-300)

    def small_terms(A, Z):
        t1 = np.abs(np.exp(-1j * kz1[:, None] * Z[None, :]) * A[None, :])
        t2 = np.abs(np.exp(-1j * kz2[:, None] * Z[None, :]) * A[None, :])
        return bool(np.all(np.isfinite(t1)) and np.all(np.isfinite(t2)) and
                    max(np.max(t1), np.max(t2)) <= CANCEL * scale)

    # level 1: e^{-i kz Z} = e^{k T0 Z} (e^{k dt1 Z})^n
    c1 = k * dt1
    conv1 = lambda z, b: (np.log(z) / c1, b * np.exp(-k * T0 * np.log(z) / c1))
    def resid1(z, b):
        Z, A = conv1(z, b)
        return float(np.max(np.abs(np.exp(-1j * kz1[:, None] * Z[None, :]) @ A - y1)))
    z1, b1 = gpof(y1, m1, rel_tol, decaying=True,
                  keep=lambda z: (np.log(z) / c1).real < 0,
                  accept=lambda z, b: small_terms(*conv1(z, b)[::-1]), score=resid1)
    Z1, A1 = conv1(z1, b1) if z1.size else (np.zeros(0, complex), np.zeros(0, complex))
    # level 2 on the residual: e^{-i kz Z} = e^{-i k Z} (e^{-i k (i - 1/T0) dt2 Z})^n
    res2 = y2 - (np.exp(-1j * kz2[:, None] * Z1[None, :]) @ A1 if A1.size else 0.0)
    c = -1j * k * (1j - 1.0 / T0) * dt2
    conv2 = lambda z, b: (np.log(z) / c, b * np.exp(1j * k * np.log(z) / c))
    def resid_all(z, b):
        Z, A = conv2(z, b)
        Z, A = np.concatenate([Z1, Z]), np.concatenate([A1, A])
        r1 = np.max(np.abs(np.exp(-1j * kz1[:, None] * Z[None, :]) @ A - y1))
        r2 = np.max(np.abs(np.exp(-1j * kz2[:, None] * Z[None, :]) @ A - y2))
        return float(max(r1, r2))
    z2, b2 = gpof(res2, n_images - A1.size, rel_tol, keep=lambda z: (np.log(z) / c).real < 0,
                  accept=lambda z, b: small_terms(*conv2(z, b)[::-1]), score=resid_all)
    Z2, A2 = conv2(z2, b2) if z2.size else (np.zeros(0, complex), np.zeros(0, complex))
    A = np.concatenate([A1, A2])
    Z = np.concatenate([Z1, Z2])
    approx1 = np.exp(-1j * kz1[:, None] * Z[None, :]) @ A
    approx2 = np.exp(-1j * kz2[:, None] * Z[None, :]) @ A
    info = {
        'resid1': float(np.max(np.abs(approx1 - y1))),
        'resid2': float(np.max(np.abs(approx2 - y2))),
        'scale': float(max(np.max(np.abs(y1)), np.max(np.abs(y2)))),
        'n1': int(A1.size), 'n2': int(A2.size),
    }
    return A, Z, info


class ImageTable:
    """Same-layer DCIM images of one medium (one fit per (layer, term)).

    ``terms[l]`` is a list of dicts with keys tag, sz, szp, c, zeta_min, A, Z.
    The 'ud' and 'du' terms of an interior layer have the same s_tau and the
    same zeta_min, so they share one fit.
    """

    def __init__(self, med: Medium, zext, n_images=8, T1=10.0, n_samples=101,
                 T0=None, m1=None, rel_tol=1e-12):
        self.med = med
        self.zext = [tuple(map(float, e)) for e in zext]
        self.terms = []
        for l in range(med.n_layers):
            lst = []
            zlo, zhi = self.zext[l]
            shared = None
            for tag, sz, szp, c in med.same_layer_terms(l):
                if tag == 'uu':
                    zmin = 2.0 * zlo + c
                elif tag == 'dd':
                    zmin = c - 2.0 * zhi
                else:
                    zmin = (zlo - zhi) + c
                kl = med.k[l]
                t0 = default_T0(med, l) if T0 is None else T0
                if tag in ('ud', 'du') and shared is not None:
                    A, Z, info = shared
                else:
                    def F(kz, tag=tag, l=l, zmin=zmin, kl=kl):
                        krho = np.sqrt(kl * kl - kz * kz)
                        return self.med.s_tau(l, tag, krho) * np.exp(1j * kz * zmin)
                    A, Z, info = fit_two_level(F, kl, t0, T1, n_samples, n_images, m1, rel_tol)
                    if tag in ('ud', 'du'):
                        shared = (A, Z, info)
                lst.append(dict(tag=tag, sz=sz, szp=szp, c=c, zeta_min=zmin, A=A, Z=Z, info=info))
            self.terms.append(lst)

    def reaction(self, l, x, y, z, xp, yp, zp):
        """Same-layer DCIM reaction field sum_tau sum_j A_j h0(k R_j) (vectorised)."""
        kl = self.med.k[l]
        rho2 = (x - xp) ** 2 + (y - yp) ** 2
        out = np.zeros(np.broadcast(x, xp).shape, dtype=complex)
        for t in self.terms[l]:
            zeta = t['sz'] * z + t['szp'] * zp + t['c']
            for A, Z in zip(t['A'], t['Z']):
                w = zeta - t['zeta_min'] - Z
                R = np.sqrt(rho2 + w * w)
                out = out + A * np.exp(1j * kl * R) / (1j * kl * R)
        return out

    def flat(self):
        """Flattened arrays (layer, term, A, Z, sz, szp, c, zeta_min) of all images."""
        rows = []
        for l, lst in enumerate(self.terms):
            for ti, t in enumerate(lst):
                for A, Z in zip(t['A'], t['Z']):
                    rows.append((l, ti, A, Z, t['sz'], t['szp'], t['c'], t['zeta_min']))
        return rows
