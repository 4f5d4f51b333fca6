"""Pins of the derivative recurrence (Sec. 3.3, corrected eq. ``recurrsion``).

Independent references: the closed-form Taylor series on the z axis, an
independent truncated multivariate power-series evaluation of e^{ikR}/R
(Taylor-mode differentiation), the Helmholtz equation satisfied by the
coefficients, and central finite differences.
"""
import math

import numpy as np
import pytest
from scipy.signal import convolve

from oracle.derivs import taylor_phi, taylor_h0, multi_indices, index_map


def _series_phi(x, k, P):
    """Taylor coefficients of e^{ikR}/R at x by truncated power-series algebra."""
    sh = (P + 1,) * 3
    deg = np.add.outer(np.add.outer(np.arange(P + 1), np.arange(P + 1)), np.arange(P + 1))
    mask = deg <= P

    def mul(a, b):
        return (convolve(a, b)[:P + 1, :P + 1, :P + 1]) * mask

    R2 = np.zeros(sh, complex)
    R2[0, 0, 0] = sum(xi * xi for xi in x)
    for i, xi in enumerate(x):
        e = [0, 0, 0]
        e[i] = 1
        R2[tuple(e)] += 2 * xi
        e[i] = 2
        R2[tuple(e)] += 1.0
    R0sq = R2[0, 0, 0]
    R0 = np.sqrt(R0sq)
    u = R2 / R0sq
    u[0, 0, 0] = 0.0
    # (1+u)^{1/2} and (1+u)^{-1/2} by binomial series
    def powser(alpha):
        out = np.zeros(sh, complex)
        out[0, 0, 0] = 1.0
        term = np.zeros(sh, complex)
        term[0, 0, 0] = 1.0
        c = 1.0
        for n in range(1, P + 1):
            term = mul(term, u)
            c *= (alpha - n + 1) / n
            out += c * term
        return out
    sq = powser(0.5)
    isq = powser(-0.5)
    dR = R0 * sq
    dR[0, 0, 0] = 0.0
    # exp(i k dR) by power series in dR
    ex = np.zeros(sh, complex)
    ex[0, 0, 0] = 1.0
    term = ex.copy()
    for n in range(1, P + 1):
        term = mul(term, 1j * k * dR) / n
        ex += term
    phi = np.exp(1j * k * R0) / R0 * mul(ex, isq)
    mi = multi_indices(P)
    return np.array([phi[tuple(m)] for m in mi])


@pytest.mark.parametrize("x,k", [((0.3, -0.7, 1.1 + 0.6j), 1.7 + 0.05j),
                                 ((1.2, 0.4, -0.9), 2.0),
                                 ((-0.5, 0.8, 2.5 - 1.5j), 3.0 + 0.01j)])
def test_recurrence_matches_power_series(x, k):
    P = 8
    a = taylor_phi(*x, k, P)
    s = _series_phi(x, k, P)
    assert np.max(np.abs(a - s) / (np.abs(s) + 1e-300 + np.max(np.abs(s)) * 1e-13)) < 1e-9


def test_axis_closed_form():
    k, w, P = 1.7 + 0.05j, 0.9 - 0.4j, 14
    a = taylor_phi(0.0, 0.0, w, k, P)
    im = index_map(P)
    for n in range(P + 1):
        c = np.exp(1j * k * w) * sum((1j * k) ** m / math.factorial(m) * (-1) ** (n - m) / w ** (n - m + 1)
                                     for m in range(n + 1))
        assert abs(a[im[(0, 0, n)]] - c) <= 1e-13 * abs(c)


def test_helmholtz_equation():
    k, P = 2.3 + 0.02j, 12
    a = taylor_phi(0.4, -0.2, 1.3 + 0.7j, k, P)
    mi, im = multi_indices(P), index_map(P)
    for t, g in enumerate(mi):
        if g.sum() > P - 2:
            continue
        s = k * k * a[t]
        for i in range(3):
            gg = g.copy()
            gg[i] += 2
            s += (g[i] + 1) * (g[i] + 2) * a[im[tuple(int(v) for v in gg)]]
        assert abs(s) <= 1e-11 * max(abs(a[t]), 1e-30) + 1e-14


def test_first_and_second_derivatives_finite_difference():
    k = 1.4
    x = np.array([0.7, -0.3, 0.5])

    def phi(v):
        R = np.sqrt(np.sum(v * v))
        return np.exp(1j * k * R) / R
    a = taylor_phi(*x, k, 2)
    im = index_map(2)
    h = 1e-4
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        d1 = (phi(x + e) - phi(x - e)) / (2 * h)
        d2 = (phi(x + e) - 2 * phi(x) + phi(x - e)) / (h * h) / 2
        m1 = [0, 0, 0]
        m1[i] = 1
        m2 = [0, 0, 0]
        m2[i] = 2
        assert abs(a[im[tuple(m1)]] - d1) < 1e-7
        assert abs(a[im[tuple(m2)]] - d2) < 1e-5


def test_reflection_and_swap_symmetry():
    """D^g / g! of a function of (x^2 + y^2, z): reflecting x (or y) flips the
    sign of the entries with odd g1 (g2), swapping x and y swaps g1 and g2.
    The device path builds one table per class of keys related by these maps
    and copies the rest."""
    P = 8
    k = 2.0 + 0.3j
    X, Y, W = 0.7, -0.4, 0.9 - 0.35j
    mi = multi_indices(P)
    im = index_map(P)
    T = taylor_h0(X, Y, W, k, P)
    g1, g2 = mi[:, 0], mi[:, 1]
    for sx in (1, -1):
        for sy in (1, -1):
            R = taylor_h0(sx * X, sy * Y, W, k, P)
            assert np.allclose(R, T * sx ** g1 * sy ** g2, rtol=1e-13, atol=0)
            S = taylor_h0(sx * Y, sy * X, W, k, P)
            perm = [im[(int(b), int(a), int(c))] for a, b, c in mi]
            assert np.allclose(S, T[perm] * sx ** g1 * sy ** g2, rtol=1e-13, atol=0)
