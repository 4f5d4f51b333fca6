"""Layered medium, k_z branch and reflection/transmission densities (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed:
* Sec. 2.1, medium: L+1 layers, interfaces z = d_0 > d_1 > ... > d_{L-1};
  layer l is d_l < z < d_{l-1}; Helmholtz with wavenumber k_l.
* Sec. 2.1, transmission conditions: u continuous, k_{l-1} du/dz = k_l du/dz
  (the k-weighted flux) at every interface; decay at z -> +-inf.
* Sec. 2.1, k_lz = sqrt(k_l^2 - k_rho^2); the branch with Im k_lz >= 0 is used.
* Sec. 2.1, eq. ``updownspectraldoamin`` and the sigma definitions: the
  reaction field in layer l is theta * (a e^{-i k_lz (z - d_l)} +
  b e^{i k_lz (z - d_l)}) / k_lz, with a = sigma^{dd} S1 + sigma^{du} S2,
  b = sigma^{ud} S1 + sigma^{uu} S2, S1 = e^{i k_l'z (d_{l'-1} - z')},
  S2 = e^{i k_l'z (z' - d_l')}.
* Appendix A, three layers, source in the middle layer (eq.
  ``densitythreelayer2``): closed forms used only as an independent check of
  the numeric solve here.

The densities are obtained by a direct numeric solve of the interface
conditions for every k_rho, not from the closed forms.  To keep the linear
system free of growing exponentials, the down-going amplitude of an interior
layer is referenced to its top interface inside the solve and converted to the
paper's bottom-interface reference afterwards (multiply by e^{i k_lz D_l}).

Reading for the bottom layer L: the paper writes its down-going wave as
e^{-i k_Lz z}; here it is referenced to its own interface, e^{-i k_Lz (z -
d_{L-1})}.  For d_{L-1} = 0 the two agree; otherwise sigma_{L.} differs from the
paper's by the factor e^{i k_Lz d_{L-1}}, and u^down_L is the same function.
"""
from __future__ import annotations

import numpy as np


def kz_branch(k, krho):
    """k_z = sqrt(k^2 - k_rho^2) with Im k_z >= 0 (real part >= 0 when real)."""
    s = np.sqrt(np.asarray(k, dtype=complex) ** 2 - np.asarray(krho, dtype=complex) ** 2)
    return np.where(s.imag < 0, -s, s)


class Medium:
    """L+1 layers (``n_layers`` = L+1), interfaces ``d`` (strictly decreasing)."""

    def __init__(self, d, k):
        self.d = np.asarray(d, dtype=float).reshape(-1)
        self.k = np.asarray(k, dtype=complex).reshape(-1)
        if self.k.size != self.d.size + 1:
            raise ValueError("need len(k) == len(d) + 1")
        if np.any(np.diff(self.d) >= 0):
            raise ValueError("interfaces must be strictly decreasing")
        self.n_layers = self.k.size
        self.L = self.n_layers - 1

    def layer_of(self, z):
        """Layer index l with d_l < z < d_{l-1}; -1 for a point on an interface."""
        z = np.asarray(z, dtype=float)
        lay = np.zeros(z.shape, dtype=np.int64)
        bad = np.zeros(z.shape, dtype=bool)
        for dm in self.d:
            lay += (z < dm)
            bad |= (z == dm)
        return np.where(bad, -1, lay)

    def thickness(self, l):
        return self.d[l - 1] - self.d[l]

    # ------------------------------------------------------------------
    def densities(self, src_layer, krho, basis='paper'):
        """All densities for a source in layer ``src_layer`` at the given k_rho.

        ``basis='paper'`` gives the paper's sigma (down-going waves of an
        interior layer referenced to its bottom interface d_l).  ``basis='solve'``
        returns the same amplitudes with the down-going wave of an interior layer
        referenced to its top interface d_{l-1} (sigma * e^{-i k_lz D_l}); every
        amplitude is then bounded on the whole Sommerfeld path.

        Returns a dict  (l, tag) -> array, tag in {'uu','ud','du','dd'} with the
        paper's convention: b_l = sigma^{ud} S1 + sigma^{uu} S2 (up-going part
        of layer l), a_l = sigma^{dd} S1 + sigma^{du} S2 (down-going part).
        Entries that do not exist (no up-going wave in layer L, no down-going
        wave in layer 0, no S1 for a source in layer 0, no S2 for layer L) are
        omitted.
        """
        krho = np.atleast_1d(np.asarray(krho, dtype=complex))
        L = self.L
        n = krho.size
        kz = [kz_branch(self.k[m], krho) for m in range(L + 1)]
        # unknown ordering: b_0, (a_1, b_1), ..., (a_{L-1}, b_{L-1}), a_L
        def ia(m):
            return 2 * m - 1
        def ib(m):
            return 2 * m
        nu = 2 * L
        A = np.zeros((n, nu, nu), dtype=complex)
        # Basis inside the solve:
        #   layer 0:        b_0 e^{i kz (z-d_0)} / kz
        #   layer 0<m<L:    a_m e^{-i kz (z-d_{m-1})} / kz + b_m e^{i kz (z-d_m)} / kz
        #   layer L:        a_L e^{-i kz (z-d_{L-1})} / kz
        # value and z-derivative of each basis function at z = d_j:
        def basis_at(m, which, j):
            """(value, derivative) of the a- or b-basis of layer m at z = d_j."""
            kzm = kz[m]
            if which == 'b':
                ref = self.d[m] if m < L else None
                ex = np.exp(1j * kzm * (self.d[j] - ref))
                return ex / kzm, 1j * ex
            else:
                ref = self.d[m - 1]
                ex = np.exp(-1j * kzm * (self.d[j] - ref))
                return ex / kzm, -1j * ex
        for j in range(L):                  # interface d_j between layer j (above) and j+1
            up, lo = j, j + 1
            r_c, r_f = 2 * j, 2 * j + 1
            for m, sgn in ((up, 1.0), (lo, -1.0)):
                kw = self.k[m]
                for which in ('a', 'b'):
                    if which == 'a' and m == 0:
                        continue
                    if which == 'b' and m == L:
                        continue
                    col = ia(m) if which == 'a' else ib(m)
                    v, dv = basis_at(m, which, j)
                    A[:, r_c, col] += sgn * v
                    A[:, r_f, col] += sgn * kw * dv
        out = {}
        lp = src_layer
        for src in ('S1', 'S2'):
            if src == 'S1' and lp == 0:
                continue
            if src == 'S2' and lp == L:
                continue
            rhs = np.zeros((n, nu), dtype=complex)
            kzs = kz[lp]
            kw = self.k[lp]
            # free part e^{i kz |z - z'|}/kz of the source layer, normalised so
            # that it equals S/kz at the interface it hits (S = 1 here).
            if src == 'S1':
                j = lp - 1                      # interface above the source: source below it
                # at z = d_j: value 1/kz, derivative +i (wave e^{i kz (z - z')})
                val, der = 1.0 / kzs, 1j * np.ones(n)
                # equations: up-side minus low-side = 0; free part on the low side
                rhs[:, 2 * j] += val
                rhs[:, 2 * j + 1] += kw * der
            else:
                j = lp                          # interface below the source: source above it
                val, der = 1.0 / kzs, -1j * np.ones(n)
                rhs[:, 2 * j] -= val
                rhs[:, 2 * j + 1] -= kw * der
            x = np.linalg.solve(A, rhs[..., None])[..., 0]
            tag2 = 'd' if src == 'S1' else 'u'
            for m in range(L + 1):
                if m < L:
                    out[(m, 'u' + tag2)] = x[:, ib(m)]
                if m > 0:
                    a = x[:, ia(m)]
                    if m < L and basis == 'paper':
                        a = a * np.exp(1j * kz[m] * self.thickness(m))
                    out[(m, 'd' + tag2)] = a
        return out

    # ------------------------------------------------------------------
    def same_layer_terms(self, l):
        """Reaction terms of u_ll in the image-distance form.

        Each term tau has u_tau(r, r') = (1/k_l) int k_rho J0(k_rho rho)
        e^{i k_lz zeta_tau}/k_lz s_tau(k_rho) dk_rho with zeta_tau = sz*z +
        sz'*z' + c_tau (a real distance that is > 0 inside the layer) and s_tau
        holding only the multiple-reflection part of the density:

          'uu': zeta = z + z' - 2 d_l,          s = sigma^{uu}
          'dd': zeta = 2 d_{l-1} - z - z',      s = sigma^{dd} e^{-i kz D}
          'ud': zeta = z - z' + 2D,             s = sigma^{ud} e^{-i kz D}
          'du': zeta = z' - z + 2D,             s = sigma^{du} e^{-2i kz D}

        (top layer: only 'uu'; bottom layer: only 'dd' with s = sigma^{dd}).
        Returns a list of (tag, sz, szp, c).
        """
        L = self.L
        terms = []
        if L == 0:
            return terms
        if l < L:
            terms.append(('uu', 1.0, 1.0, -2.0 * self.d[l]))
        if l > 0:
            terms.append(('dd', -1.0, -1.0, 2.0 * self.d[l - 1]))
        if 0 < l < L:
            D = self.thickness(l)
            terms.append(('ud', 1.0, -1.0, 2.0 * D))
            terms.append(('du', -1.0, 1.0, 2.0 * D))
        return terms

    def s_tau(self, l, tag, krho):
        """The reflection factor s_tau(k_rho) of ``same_layer_terms``."""
        sig = self.densities(l, krho)
        kz = kz_branch(self.k[l], krho)
        L = self.L
        if tag == 'uu':
            return sig[(l, 'uu')]
        if tag == 'dd':
            if l == L:
                return sig[(l, 'dd')]
            return sig[(l, 'dd')] * np.exp(-1j * kz * self.thickness(l))
        D = self.thickness(l)
        if tag == 'ud':
            return sig[(l, 'ud')] * np.exp(-1j * kz * D)
        if tag == 'du':
            return sig[(l, 'du')] * np.exp(-2j * kz * D)
        raise ValueError(tag)


def three_layer_middle_closed_form(k, d, krho):
    """Appendix A, source in the middle layer of three: sigma_11^{uu,ud,du,dd}.

    Interfaces at 0 and -d.  Uses kappa_11, kappa_12 of eq. ``kappa1112`` and
    the common denominator k0 k0z kappa_11 - i k1 k1z kappa_12.
    """
    k0, k1, k2 = [complex(x) for x in k]
    krho = np.asarray(krho, dtype=complex)
    k0z, k1z, k2z = kz_branch(k0, krho), kz_branch(k1, krho), kz_branch(k2, krho)
    e2 = np.exp(2j * d * k1z)
    e1 = np.exp(1j * d * k1z)
    kap11 = (k1 * k1z - k2 * k2z) / 2 * e2 + (k1 * k1z + k2 * k2z) / 2
    kap12 = 1j * ((k2 * k2z - k1 * k1z) / 2 * e2 + (k1 * k1z + k2 * k2z) / 2)
    den = k0 * k0z * kap11 - 1j * k1 * k1z * kap12
    uu = (k1 * k1z - k2 * k2z) / den * (k1 * k1z + k0 * k0z) / 2
    ud = (k1 * k1z - k2 * k2z) / den * (k1 * k1z - k0 * k0z) / 2 * e1
    du = (k1 * k1z - k0 * k0z) * e1 / den * (k1 * k1z - k2 * k2z) / 2 * e1
    dd = (k1 * k1z - k0 * k0z) * e1 / den * (k1 * k1z + k2 * k2z) / 2
    return {'uu': uu, 'ud': ud, 'du': du, 'dd': dd}, den
