"""Pins of the Algorithm 2 oracle (Sec. 4.2: tables of Sommerfeld integrals,
eq. ``symmetricdetable``, interpolated, with the symmetric derivatives of
eq. ``sysdifferential``).

* unit density: with s_tau = 1 the Sommerfeld identity makes F = h0(kR), so
  the quadrature T_{m,nu,n} must equal (-1)^a e^{-i nu phi} D+^a D-^b d_z^n
  h0, written here from the Cartesian Taylor coefficients of
  ``derivs.taylor_h0`` (pinned on its own) through the binomial expansion of
  D+- = d_x +- i d_y;
* the Cartesian assembly maps those T back to taylor_h0 at a point off the
  x axis (the inverse expansion, so a dropped term, a wrong sign or a
  transposed index fails);
* the interpolation error at points between the grid nodes falls with the
  grid size (degree 7 Lagrange, order-8 convergence);
* a medium's reaction term: the table derivatives agree with the DCIM image
  recurrence of Algorithm 1 to within the fit's own accuracy;
* ranges: keys below the term's smallest image distance over the particle
  slab stay with the images and out of the table ranges;
* end to end: the oracle TE-FMM with Algorithm 2 tables matches the direct
  sum to the error of Algorithm 1.
"""
import math

import numpy as np
import pytest

from oracle import alg2 as A2
from oracle.derivs import multi_indices, taylor_h0
from oracle.medium import Medium
from oracle.dcim import ImageTable
from oracle.direct import direct_sum
from oracle.tefmm import TEFMM
from paper_1902_05875_gb300 import workloads as W


def cart_derivs(X, Y, Z, k, P2):
    """{(g1, g2, g3): D^g h0(kR)} at one point, from the Taylor coefficients."""
    c = taylor_h0(np.array([X]), np.array([Y]), np.array([Z], dtype=complex), k, P2)[0]
    return {tuple(int(v) for v in g): c[i] * math.factorial(g[0]) * math.factorial(g[1]) * math.factorial(g[2])
            for i, g in enumerate(multi_indices(P2))}


def T_closed(k, P2, rhos, zeta):
    """T_{m,nu,n}(rho, zeta) of the unit density at phi = 0 (X = rho, Y = 0):
    (-1)^a D+^a D-^b d_z^n h0 with a = (m + nu)/2, b = (m - nu)/2, expanding
    (d_x + i d_y)^a (d_x - i d_y)^b binomially into Cartesian derivatives."""
    out = np.zeros((len(rhos), len(A2.table_index(P2))), dtype=complex)
    for r, rho in enumerate(rhos):
        D = cart_derivs(rho, 0.0, zeta, k, P2)
        for e, (m, nu, n) in enumerate(A2.table_index(P2)):
            a, b = (m + nu) // 2, (m - nu) // 2
            acc = 0j
            for j in range(a + 1):
                for l in range(b + 1):
                    acc += math.comb(a, j) * math.comb(b, l) * (1j) ** j * (-1j) ** l * D[(m - j - l, j + l, n)]
            out[r, e] = (-1.0) ** a * acc
    return out


def test_unit_density_quadrature_is_h0():
    k, P2 = 1.5, 6
    rhos = [0.0, 0.4, 1.3]
    for zeta in (0.6, 1.7):
        T = A2.quadrature_T(k, 2.0, lambda kr: np.ones_like(kr), P2, rhos, zeta)
        ref = T_closed(k, P2, rhos, zeta)
        err = np.abs(T - ref).max() / np.abs(ref).max()
        assert err < 1e-10, (zeta, err)


def test_assembly_inverts_the_symmetric_derivatives():
    k, P2 = 2.0, 8
    X, Y, zeta = 0.7, -0.45, 0.9
    rho, phi = math.hypot(X, Y), math.atan2(Y, X)
    # T at azimuth phi equals T at phi = 0 (F depends on rho only)
    T = T_closed(k, P2, [rho], zeta)[0]
    a = A2.assemble(P2, T, phi)
    ref = taylor_h0(np.array([X]), np.array([Y]), np.array([zeta], dtype=complex), k, P2)[0]
    assert np.abs(a - ref).max() / np.abs(ref).max() < 1e-12


def test_interpolation_converges_with_the_grid():
    k, P2 = 1.5, 6
    pts = [(0.31, 0.22, 0.93), (1.17, -0.4, 1.61), (0.05, 0.02, 0.71)]
    errs = []
    for n in (10, 16, 28):
        tab = A2.Alg2Table(lambda rhos, z: T_closed(k, P2, rhos, z), P2, 1.6, 0.6, 2.0, n)
        e = 0.0
        for X, Y, z in pts:
            ref = taylor_h0(np.array([X]), np.array([Y]), np.array([z], dtype=complex), k, P2)[0]
            e = max(e, np.abs(tab.derivatives(X, Y, z) - ref).max() / np.abs(ref).max())
        errs.append(e)
    print(errs)
    assert errs[0] > errs[1] > errs[2]
    # order-8 convergence, (27/15)^8 ~ 110; the slowest point lies in the grid's
    # first cell at distance 0.71 from the singularity of h0 (5.9e-5 at n = 28)
    assert errs[1] / errs[2] > 20
    assert errs[2] < 2e-4


@pytest.mark.parametrize("tag,tol", [("ud", 1e-6), ("uu", 1e-4)])
def test_medium_term_matches_dcim_recurrence(tag, tol):
    """Quadrature T of a reaction term of the middle layer, assembled, against
    the 16-image DCIM sum of Algorithm 1 (sum_j A_j D^g h0(k R_j) / g!), at a
    point at distance ~1.3 from the term's nearest image.  The tolerance is
    the images' own accuracy for the term (the up-down term fits to ~1e-8, the
    up-up term to ~1e-5 in the highest derivatives)."""
    w = W.cfg_small()
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=16)
    l, P2 = 1, 8
    t = [tt for tt in img.terms[l] if tt['tag'] == tag][0]
    X, Y, zeta = 0.3, -0.2, t['zeta_min'] + 1.2
    T = A2.medium_T(med, l, tag, P2)([math.hypot(X, Y)], zeta)[0]
    a_q = A2.assemble(P2, T, math.atan2(Y, X))
    A, Z = np.asarray(t['A']), np.asarray(t['Z'])
    a_d = (A[:, None] * taylor_h0(np.full(len(A), X), np.full(len(A), Y), zeta - t['zeta_min'] - Z,
                                  med.k[l], P2)).sum(0)
    err = np.abs(a_q - a_d).max() / np.abs(a_d).max()
    print(tag, err)
    assert err < tol, err


def test_ranges_leave_keys_below_the_slab_to_the_images():
    med = Medium([0.0, -1.2], [1.2, 1.5, 2.0])
    # uu of the middle layer: zeta = z + z' + 2.4; a particle slab [-1.1, -0.1]
    # gives zeta_min = 0.2; a key with centres summing to -2.4 (zeta = 0) is left out
    floor = {'uu': 0.2, 'dd': 0.2, 'ud': 1.4, 'du': 1.4}
    keys = [(0.5, 2, 0, 0, -1.0), (0.5, 3, 1, 0, -2.4)]
    rho_max, rng = A2.layer_ranges(med, 1, keys, floor)
    assert rng['uu'] == (1.4, 2.4)          # zeta_hi widened from a single value
    assert abs(rng['dd'][0] - 1.0) < 1e-15 and abs(rng['ud'][0] - 2.4) < 1e-15
    assert rho_max == math.hypot(1.5, 0.5)     # the second key still serves dd, ud, du
    rho_max, rng = A2.layer_ranges(med, 1, keys[1:], {'uu': 0.2, 'dd': 9.0, 'ud': 9.0, 'du': 9.0})
    assert rng == {} and rho_max == 1.0


def test_fmm_with_tables_matches_direct_sum():
    """p = 3, 16 images, 12 x 12 tables: Algorithm 2's error against the
    direct sum equals Algorithm 1's (truncation dominates; the two derivative
    sources differ by the images' fit error, ~1e-8 here); a sign planted in
    one term's table breaks the match."""
    w = W.middle_layer_uniform(300, 3, 20, seed=4)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=16)
    ref = direct_sum(med, img, w.src, w.q, w.src)
    err = {}
    for alg in (1, 2):
        f = TEFMM(med, img, w.p, w.leaf_cap, algorithm=alg, table_n=12, n_images=16).setup(w.src, w.src)
        phi = f.evaluate(w.q)
        err[alg] = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    print(err)
    assert set(f.alg2[1]) == {'uu', 'dd', 'ud', 'du'}
    assert abs(err[2] - err[1]) <= 0.01 * err[1], err
    f.alg2[1]['du'].T *= -1
    planted = np.linalg.norm(f.evaluate(w.q) - ref) / np.linalg.norm(ref)
    assert planted > 10 * err[1], planted
