"""Cross-layer reaction components (target layer l != source layer l'), oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 3.2-3.3 of the paper for a component whose source and target lie in
different layers:

* the z'-derivatives of the density, eq. ``layermediumdensity``:
  d^{k3'}_{z'} sigma~(k_rho, z') / k3'! with the source exponentials
  S1 = e^{i k_l'z (d_{l'-1} - z')}, S2 = e^{i k_l'z (z' - d_l')};
* Theta^{k3'}(k_rho, z') = e^{i k_lz W_min} d^{k3'}_{z'} sigma~ / k3'!, fitted
  by the two-level DCIM in the target layer's variable k_lz (Steps 1-2), one fit
  per source z-centre and k3' (the "2^H (p+1)" precomputed approximations at the
  end of Sec. 3.3);
* d^{k3'}_{z'} u / k3'! ~= sum_j A_j h0(k_l sqrt(rho^2 + (W - W_min - Z_j)^2)),
  eq. ``closedformgreen``, with the target distance W = z - d_l for the up-going
  part and W = d_{l-1} - z for the down-going part (W > 0 in layer l).

Down-going waves of an interior target layer use the top-interface reference
(``Medium.densities(basis='solve')``), so W = d_{l-1} - z and every amplitude is
bounded; the bottom layer's reference is d_{L-1}.
"""
from __future__ import annotations

import math

import numpy as np

from .medium import Medium, kz_branch
from .dcim import fit_two_level, default_T0


def directions(med: Medium, l):
    """Reaction parts present in target layer l: 'up' if l < L, 'down' if l > 0."""
    out = []
    if l < med.L:
        out.append('up')
    if l > 0:
        out.append('down')
    return out


def W_of(med: Medium, l, direction, z):
    """Target distance W: z - d_l (up) or d_{l-1} - z (down)."""
    if direction == 'up':
        return np.asarray(z) - med.d[l]
    return med.d[l - 1] - np.asarray(z)


def W_min(med: Medium, l, direction, zext):
    zlo, zhi = zext[l]
    return (zlo - med.d[l]) if direction == 'up' else (med.d[l - 1] - zhi)


def source_part(med: Medium, l, lp, direction, zp, k3p, krho):
    """d^{k3'}_{z'} [S2 sigma^{.u} + S1 sigma^{.d}] / k3'! at z' = zp (eq. layermediumdensity)."""
    sig = med.densities(lp, krho, basis='solve')
    kzp = kz_branch(med.k[lp], krho)
    L = med.L
    t = 'u' if direction == 'up' else 'd'
    out = np.zeros(np.shape(krho), dtype=complex)
    if lp < L:       # S2 = e^{i kz' (z' - d_l')}
        out = out + (1j * kzp) ** k3p * np.exp(1j * kzp * (zp - med.d[lp])) * sig[(l, t + 'u')]
    if lp > 0:       # S1 = e^{i kz' (d_{l'-1} - z')}
        out = out + (-1j * kzp) ** k3p * np.exp(1j * kzp * (med.d[lp - 1] - zp)) * sig[(l, t + 'd')]
    return out / math.factorial(k3p)


RETRY_RESID = 1e-2


def source_distance(med: Medium, lp, zc):
    """Distance from z' = zc to the nearest interface of the source layer l'."""
    ds = []
    if lp > 0:
        ds.append(med.d[lp - 1] - zc)
    if lp < med.L:
        ds.append(zc - med.d[lp])
    return min(ds)


def extended_T1(k, T0, k3p, d_eff):
    """First-level path length reaching past the peak of |k_z|^{k3'} e^{-|k_z| d_eff}
    (at |k_z| = k3'/d_eff) by five decay lengths: |k| (T0 + T1) = (k3' + 5) / d_eff."""
    return (k3p + 5.0) / d_eff / abs(k) - T0


def fit_cross(med: Medium, l, lp, direction, zc, k3p, wmin, n_images=8, T1=10.0, n_samples=101,
              T0=None, m1=None, rel_tol=1e-12):
    """Images (A, Z, info) of Theta^{k3'} for source z-centre zc (Steps 1-2).

    Reading: when the fit on the given paths leaves a residual above
    RETRY_RESID of the largest sample, the first-level path is lengthened to
    extended_T1 and the fit repeated.  Theta^{k3'} grows like |k_z|^{k3'}
    e^{-|k_z| d_eff} along C_ap1 (d_eff = W_min + the source's distance to its
    nearest interface); with a large k3' and a small d_eff the fixed path ends
    before the function has peaked and no image set fits the samples.
    """
    kl = med.k[l]
    t0 = default_T0(med, l) if T0 is None else T0

    def F(kz):
        krho = np.sqrt(kl * kl - kz * kz)
        return source_part(med, l, lp, direction, zc, k3p, krho) * np.exp(1j * kz * wmin)
    A, Z, info = fit_two_level(F, kl, t0, T1, n_samples, n_images, m1, rel_tol)
    if max(info['resid1'], info['resid2']) > RETRY_RESID * info['scale']:
        T1x = extended_T1(kl, t0, k3p, wmin + source_distance(med, lp, zc))
        if T1x > T1:
            A, Z, info = fit_two_level(F, kl, t0, T1x, n_samples, n_images, m1, rel_tol)
            info['T1'] = T1x
    return A, Z, info


def image_sum(med: Medium, l, direction, A, Z, wmin, x, y, z, xp, yp):
    """sum_j A_j h0(k_l sqrt(rho^2 + (W(z) - W_min - Z_j)^2)) (Step 3)."""
    kl = med.k[l]
    rho2 = (np.asarray(x) - xp) ** 2 + (np.asarray(y) - yp) ** 2
    Wd = W_of(med, l, direction, z) - wmin
    out = np.zeros(np.broadcast(rho2, Wd).shape, dtype=complex)
    for a, zz in zip(A, Z):
        w = Wd - zz
        R = np.sqrt(rho2 + w * w)
        out = out + a * np.exp(1j * kl * R) / (1j * kl * R)
    return out


class CrossDirect:
    """Cross-layer reaction field by per-source-point fits (k3' = 0 at z' = z_j).

    The plain definition the FMM's cross-layer tables approximate: every source
    point gets its own DCIM fit of its exact z', so nothing is expanded in z'.
    """

    def __init__(self, med: Medium, zext, n_images=8, **fit_kw):
        self.med = med
        self.zext = zext
        self.n_images = n_images
        self.fit_kw = fit_kw
        self.cache = {}

    def images(self, l, lp, direction, zp):
        key = (l, lp, direction, float(zp))
        if key not in self.cache:
            wmin = W_min(self.med, l, direction, self.zext)
            A, Z, _ = fit_cross(self.med, l, lp, direction, zp, 0, wmin, self.n_images, **self.fit_kw)
            self.cache[key] = (A, Z, wmin)
        return self.cache[key]

    def potential(self, src, q, tgt):
        """Cross-layer part of Phi at the targets (all layer pairs l != l')."""
        med = self.med
        ls_ = med.layer_of(src[:, 2])
        lt_ = med.layer_of(tgt[:, 2])
        out = np.zeros(len(tgt), dtype=complex)
        for j in range(len(src)):
            lp = ls_[j]
            for l in range(med.n_layers):
                if l == lp:
                    continue
                sel = np.nonzero(lt_ == l)[0]
                if sel.size == 0:
                    continue
                for direction in directions(med, l):
                    A, Z, wmin = self.images(l, lp, direction, src[j, 2])
                    out[sel] += q[j] * image_sum(med, l, direction, A, Z, wmin, tgt[sel, 0], tgt[sel, 1],
                                                 tgt[sel, 2], src[j, 0], src[j, 1])
        return out
