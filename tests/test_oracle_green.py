"""Pins of the oracle's Green's-function chain (no GPU).

* Tables 3.1/3.2 (Sec. 3.3): quadrature of the derivatives of u^up_11 must
  reproduce the paper's "direct quadrature" column (tests/golden).
* Appendix A closed forms (two layers; three layers, source in the middle):
  the numeric interface solve must reproduce them.
* Homogeneous medium: no reflection, unit transmission; the Sommerfeld identity
  (Sec. 3.3) must give h0.
* GPOF recovers a known sum of exponentials; the DCIM image sum approaches
  the quadrature truth as the number of images grows (Sec. 3.3, Steps 1-3).
* Reciprocity inside one layer: u(r, r') = u(r', r).
"""
import math
import os

import numpy as np
import pytest

from oracle.medium import Medium, kz_branch, three_layer_middle_closed_form
from oracle.sommerfeld import reaction_derivative, free_space_by_quadrature, h0
from oracle.dcim import ImageTable, gpof

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table_3_1_3_2.txt")


def test_table_3_1_3_2_quadrature():
    med = Medium([0.0, -2.0], [0.8, 1.5, 2.0])
    rows = np.loadtxt(GOLD)
    for row in rows:
        r, rp = row[0:3], row[3:6]
        k3, k3p, s = int(row[6]), int(row[7]), int(row[8])
        want = row[9] + 1j * row[10]
        got = reaction_derivative(med, 1, 1, r, rp, s=s, k3=k3, k3p=k3p, part='up')
        # the paper prints 15 significant digits; 1e-11 leaves room for the last one
        assert abs(got.real - want.real) <= 1e-11 * abs(want.real) + 1e-17, (row, got)
        assert abs(got.imag - want.imag) <= 1e-11 * abs(want.imag) + 1e-17, (row, got)


def test_table_values_detect_dropped_reflection_term():
    """A mistake planted in the oracle (dropping sigma^{ud}) must fail the pin."""
    med = Medium([0.0, -2.0], [0.8, 1.5, 2.0])
    orig = med.densities

    def broken(lp, krho, basis='paper'):
        d = orig(lp, krho, basis)
        d[(1, 'ud')] = 0 * d[(1, 'ud')]
        return d
    med.densities = broken
    row = np.loadtxt(GOLD)[0]
    got = reaction_derivative(med, 1, 1, row[0:3], row[3:6], part='up')
    assert abs(got.real - row[9]) > 1e-6


@pytest.mark.parametrize("krho", [0.3, 1.0 + 0.2j, 2.5 - 0.3j, 7.0, 0.1 - 0.5j, 30.0])
def test_three_layer_middle_source_closed_form(krho):
    k, d = [0.8, 1.5, 2.0], 2.0
    med = Medium([0.0, -d], k)
    sig = med.densities(1, np.array([krho]))
    cf, _ = three_layer_middle_closed_form(k, d, np.array([krho]))
    for t in ('uu', 'ud', 'du', 'dd'):
        assert abs(sig[(1, t)][0] - cf[t][0]) <= 1e-13 * max(1.0, abs(cf[t][0])), t


def test_two_layer_closed_forms():
    k0, k1 = 1.3, 2.1 + 0.05j
    med = Medium([0.0], [k0, k1])
    kr = np.array([0.2, 1.7, 3.0 - 0.4j, 9.0])
    k0z, k1z = kz_branch(k0, kr), kz_branch(k1, kr)
    den = k0 * k0z + k1 * k1z
    s0 = med.densities(0, kr)
    assert np.allclose(s0[(0, 'uu')], (k0 * k0z - k1 * k1z) / den, rtol=1e-13)
    assert np.allclose(s0[(1, 'du')], 2 * k0 * k1z / den, rtol=1e-13)
    s1 = med.densities(1, kr)
    assert np.allclose(s1[(0, 'ud')], 2 * k1 * k0z / den, rtol=1e-13)
    assert np.allclose(s1[(1, 'dd')], (k1 * k1z - k0 * k0z) / den, rtol=1e-13)


def test_appendix_common_denominator_identity():
    """k2 k2z kappa31 - i k1 k1z kappa32 = k0 k0z kappa11 - i k1 k1z kappa12."""
    k0, k1, k2, d = 0.8, 1.5, 2.0, 2.0
    for kr in (0.4, 1.9 - 0.3j, 5.0):
        k0z, k1z, k2z = kz_branch(k0, kr), kz_branch(k1, kr), kz_branch(k2, kr)
        e2 = np.exp(2j * d * k1z)
        k31 = (k1 * k1z - k0 * k0z) / 2 * e2 + (k1 * k1z + k0 * k0z) / 2
        k32 = 1j * ((k0 * k0z - k1 * k1z) / 2 * e2 + (k0 * k0z + k1 * k1z) / 2)
        _, den = three_layer_middle_closed_form([k0, k1, k2], d, np.array([kr]))
        assert abs(k2 * k2z * k31 - 1j * k1 * k1z * k32 - den[0]) < 1e-13 * abs(den[0])


def test_homogeneous_medium_no_reflection():
    med = Medium([0.0, -1.0], [1.7, 1.7, 1.7])
    kr = np.array([0.5, 1.6, 2.5, 4.0 - 0.2j])
    sig = med.densities(1, kr)
    for t in ('uu', 'ud', 'du', 'dd'):
        assert np.max(np.abs(sig[(1, t)])) < 1e-14
    # transmission up through a homogeneous interface stack: unit amplitude
    # relative to the source wave (b_0 = S1 e^{i kz (d_0 - d_0)})
    assert np.allclose(sig[(0, 'ud')], 1.0, atol=1e-14)


def test_sommerfeld_identity():
    for k, r, rp in ((1.5, (0.1, 0.2, 0.3), (0.5, -0.1, -0.2)),
                     (2.0 + 0.1j, (0.0, 0.0, 0.9), (0.7, 0.2, 0.1))):
        R = math.dist(r, rp)
        assert abs(free_space_by_quadrature(k, r, rp) - h0(k * R)) < 1e-12


def test_gpof_recovers_exponentials():
    n = np.arange(101)
    zt = np.array([0.9 * np.exp(0.3j), 0.5 - 0.2j, 0.99])
    bt = np.array([1.0, 2 - 1j, 0.3j])
    y = (zt[None, :] ** n[:, None]) @ bt
    z, b = gpof(y, 8)
    assert len(z) == 3
    o = np.argsort(np.abs(z))
    oz = np.argsort(np.abs(zt))
    assert np.allclose(z[o], zt[oz], atol=1e-10)
    assert np.allclose(b[o], bt[oz], atol=1e-9)


@pytest.fixture(scope="module")
def cfg_medium():
    return Medium([0.0, -1.2], [1.2, 1.5, 2.0]), [(0.1, 1.1), (-1.1, -0.1), (-2.3, -1.3)]


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        r = np.r_[rng.uniform(-1, 1, 2), rng.uniform(-1.1, -0.1)]
        rp = np.r_[rng.uniform(-1, 1, 2), rng.uniform(-1.1, -0.1)]
        out.append((r, rp))
    return out


def test_dcim_image_sum_vs_quadrature(cfg_medium):
    """G~ (DCIM) against the Sommerfeld quadrature; error falls with M."""
    med, zext = cfg_medium
    pairs = _pairs(40, 11)
    truth = [reaction_derivative(med, 1, 1, r, rp, part='both') for r, rp in pairs]
    errs = {}
    for M in (8, 16, 24):
        tab = ImageTable(med, zext, n_images=M)
        e = max(abs(tab.reaction(1, *r, *rp) - t) / abs(t) for (r, rp), t in zip(pairs, truth))
        errs[M] = e
    assert errs[8] < 5e-3
    assert errs[16] < 2e-5
    assert errs[24] < 1e-7
    assert errs[24] < errs[16] < errs[8]


def test_reaction_reciprocity_same_layer(cfg_medium):
    med, _ = cfg_medium
    for r, rp in _pairs(4, 3):
        a = reaction_derivative(med, 1, 1, r, rp, part='both')
        b = reaction_derivative(med, 1, 1, rp, r, part='both')
        assert abs(a - b) < 1e-12 * abs(a)


def test_point_on_interface_flagged(cfg_medium):
    med, _ = cfg_medium
    assert list(med.layer_of(np.array([0.5, 0.0, -0.6, -1.2, -5.0]))) == [0, -1, 1, -1, 2]
