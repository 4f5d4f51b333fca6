"""Taylor coefficients of e^{ikR}/R at a complex point (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.3, eq. ``recurrsion``: with x = r - r' (third component possibly
complex, an image point), phi = e^{ikR}/R, psi = e^{ikR}, R = sqrt(x.x)
(principal branch), a_k = D^k phi / k!, b_k = D^k psi / k!.

The printed recurrence has wrong coefficients and an undefined psi.  Re-derived
from R^2 d_i phi + x_i phi = i k x_i psi and d_i psi = i k x_i phi by matching
Taylor coefficients and summing over i, it reads

    |k| R^2 a_k + (2|k|-1) sum_i x_i a_{k-e_i} + (|k|-1) sum_i a_{k-2e_i}
                                   = i k sum_i (x_i b_{k-e_i} + b_{k-2e_i}),
    |k| b_k = i k sum_i (x_i a_{k-e_i} + a_{k-2e_i}),

(coefficients with a negative index are zero), a_0 = e^{ikR}/R, b_0 = e^{ikR}.
The Taylor coefficients of h0(kR) = e^{ikR}/(ikR) are a_k/(ik).

Multi-index order used everywhere in the oracle ("graded, k1 descending"):
for n = 0..P, for k1 = n..0, for k2 = n-k1..0, k3 = n-k1-k2.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def multi_indices(P):
    out = []
    for n in range(P + 1):
        for k1 in range(n, -1, -1):
            for k2 in range(n - k1, -1, -1):
                out.append((k1, k2, n - k1 - k2))
    return np.array(out, dtype=np.int64)


@lru_cache(maxsize=None)
def index_map(P):
    return {tuple(int(v) for v in m): i for i, m in enumerate(multi_indices(P))}


def n_coeffs(P):
    return (P + 1) * (P + 2) * (P + 3) // 6


def taylor_phi(X, Y, W, k, P):
    """a[..., idx(k)] = D^k (e^{ikR}/R) / k!  at x = (X, Y, W), |k| <= P.

    X, Y real or complex arrays, W complex array (broadcast together).
    """
    X, Y, W = np.broadcast_arrays(np.asarray(X, complex), np.asarray(Y, complex),
                                  np.asarray(W, complex))
    x = (X, Y, W)
    R2 = X * X + Y * Y + W * W
    R = np.sqrt(R2)
    k = complex(k)
    T = len(multi_indices(P))
    # coefficient index first (row T is a zero row standing for a coefficient
    # with a negative index); order n needs orders n-1 and n-2 only, so all
    # coefficients of one order are computed together
    a = np.zeros((T + 1,) + X.shape, dtype=complex)
    b = np.zeros((T + 1,) + X.shape, dtype=complex)
    e = np.exp(1j * k * R)
    a[0] = e / R
    b[0] = e
    for n in range(1, P + 1):
        ts, J1, J2 = _order_links(P, n)
        sa1 = x[0][None] * a[J1[0]] + x[1][None] * a[J1[1]] + x[2][None] * a[J1[2]]
        sa2 = a[J2[0]] + a[J2[1]] + a[J2[2]]
        sbr = x[0][None] * b[J1[0]] + x[1][None] * b[J1[1]] + x[2][None] * b[J1[2]] + \
            b[J2[0]] + b[J2[1]] + b[J2[2]]
        b[ts] = 1j * k * (sa1 + sa2) / n
        a[ts] = (1j * k * sbr - (2 * n - 1) * sa1 - (n - 1) * sa2) / (n * R2[None])
    return np.moveaxis(a[:T], 0, -1)


@lru_cache(maxsize=None)
def _order_links(P, n):
    """Indices of the order-n multi-indices k (in the order-P list) and, per
    axis i, of k - e_i (J1[i]) and k - 2 e_i (J2[i]); T (a zero row) where
    that index is negative."""
    mi = multi_indices(P)
    im = index_map(P)
    T = len(mi)
    ts = np.nonzero(mi.sum(1) == n)[0]
    J1 = np.full((3, len(ts)), T, dtype=np.int64)
    J2 = np.full((3, len(ts)), T, dtype=np.int64)
    for c, t in enumerate(ts):
        for i in range(3):
            if mi[t][i] >= 1:
                km = mi[t].copy()
                km[i] -= 1
                J1[i, c] = im[tuple(int(v) for v in km)]
            if mi[t][i] >= 2:
                km = mi[t].copy()
                km[i] -= 2
                J2[i, c] = im[tuple(int(v) for v in km)]
    return ts, J1, J2


def taylor_h0(X, Y, W, k, P):
    """D^k h0(kR)/k! = a_k/(ik)."""
    return taylor_phi(X, Y, W, k, P) / (1j * complex(k))
