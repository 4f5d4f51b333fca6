"""Pins of the CPU TE-FMM oracle (Sec. 3, Algorithm 1 and the component loop).

* brute force: at N = 500 the FMM matches the FP64 direct sum with an error
  that falls as p rises (p = 2, 4, 6, 8);
* homogeneous medium (all k equal): the reaction field vanishes and the FMM
  is the free-space FMM of the whole particle set;
* polynomial exactness of M2M and L2L (Sec. 3.1 translations are exact shifts);
* the interaction lists partition the (target, source) pairs: every pair is
  covered exactly once by a V pair of an ancestor or a P2P entry, V pairs are
  never adjacent, P2P pairs of U type are adjacent;
* the direct sum's reaction part matches Sommerfeld quadrature;
* a per-target evaluation equals the full evaluation.
"""
import math
import numpy as np
import pytest

from oracle.medium import Medium
from oracle.dcim import ImageTable
from oracle.tefmm import TEFMM, Trees, build_lists, Ops
from oracle.direct import direct_sum
from oracle.sommerfeld import reaction_derivative
from paper_1902_05875_gb300 import workloads as W


@pytest.fixture(scope="module")
def small():
    w = W.middle_layer_uniform(500, 4, 20, seed=3)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=8)
    ref = direct_sum(med, img, w.src, w.q, w.src)
    return w, med, img, ref


def test_fmm_error_falls_with_p(small):
    w, med, img, ref = small
    errs = []
    for p in (2, 4, 6, 8):
        phi = TEFMM(med, img, p, 20).setup(w.src, w.src).evaluate(w.q)
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 2e-6, errs


def test_fmm_detects_planted_sign_error(small):
    """A sign flip planted in the oracle's M2L must break the brute-force match."""
    w, med, img, ref = small
    f = TEFMM(med, img, 6, 20).setup(w.src, w.src)
    f.ops.s3p = -f.ops.s3p
    phi = f.evaluate(w.q)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) > 1e-3


def test_homogeneous_medium_is_free_space():
    rng = np.random.default_rng(7)
    src = rng.uniform([-1, -1, -1.0], [1, 1, -0.2], size=(400, 3))
    q = rng.uniform(0, 1, 400) + 1j * rng.uniform(0, 1, 400)
    med = Medium([0.0, -1.2], [1.5, 1.5, 1.5])
    img = ImageTable(med, [(0.1, 1.1), (-1.1, -0.1), (-2.3, -1.3)], n_images=8)
    for lst in img.terms:
        for t in lst:
            assert np.max(np.abs(t['A']), initial=0.0) < 1e-12
    phi = TEFMM(med, img, 8, 16).setup(src, src).evaluate(q)
    d = src[:, None, :] - src[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, 1.0)
    G = np.exp(1.5j * r) / (1.5j * r)
    np.fill_diagonal(G, 0.0)
    ref = G @ q
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-6


def test_m2m_l2l_polynomial_exactness():
    ops = Ops(5)
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.2, 0.2, size=(30, 3))
    q = rng.normal(size=30) + 1j * rng.normal(size=30)
    c_child = np.array([0.05, -0.03, 0.02])
    c_par = np.array([0.0, 0.0, 0.0])
    a_child = ops.p2m(pts, q, c_child)
    a_par = ops.m2m(a_child, c_child - c_par)
    assert np.allclose(a_par, ops.p2m(pts, q, c_par), rtol=1e-12, atol=1e-14)
    beta = rng.normal(size=ops.np_) + 1j * rng.normal(size=ops.np_)
    lam = ops.l2l(beta, c_child - c_par)
    x = rng.uniform(-0.1, 0.1, size=(10, 3)) + c_child
    assert np.allclose(ops.l2p(lam, x, c_child), ops.l2p(beta, x, c_par), rtol=1e-12, atol=1e-13)


def test_lists_partition_all_pairs(small):
    w, med, img, _ = small
    tr = Trees(med, w.src, w.src, 20)
    V, P2P = build_lists(tr, 1, 1)
    ns = len(w.src)
    cover = np.zeros((ns, ns), dtype=np.int64)   # [sorted target, sorted source]
    for t, lst in V.items():
        for s in lst:
            assert not tr.adjacent(t, s)
            assert tr.level[t] == tr.level[s]
            cover[tr.t0[t]:tr.t1[t], tr.s0[s]:tr.s1[s]] += 1
    for t, lst in P2P.items():
        assert tr.is_leaf[t]
        for s in lst:
            cover[tr.t0[t]:tr.t1[t], tr.s0[s]:tr.s1[s]] += 1
    assert np.all(cover == 1)


def test_direct_sum_reaction_matches_quadrature():
    med = Medium([0.0, -1.2], [1.2, 1.5, 2.0])
    img = ImageTable(med, [(0.1, 1.1), (-1.1, -0.1), (-2.3, -1.3)], n_images=24)
    rng = np.random.default_rng(4)
    src = rng.uniform([-1, -1, -1.1], [1, 1, -0.1], size=(3, 3))
    tgt = rng.uniform([-1, -1, -1.1], [1, 1, -0.1], size=(2, 3))
    q = np.array([1.0, 0.5 - 0.2j, -0.3j])
    got = direct_sum(med, img, src, q, tgt, include_free=False)
    for i in range(2):
        want = sum(q[j] * reaction_derivative(med, 1, 1, tgt[i], src[j], part='both') for j in range(3))
        assert abs(got[i] - want) < 1e-7 * abs(want)


def test_sampled_targets_equal_full(small):
    w, med, img, _ = small
    f = TEFMM(med, img, 4, 20).setup(w.src, w.src)
    phi = f.evaluate(w.q)
    sel = np.array([0, 5, 77, 311, 499])
    assert np.max(np.abs(f.evaluate(w.q, sel) - phi[sel])) < 1e-12 * np.max(np.abs(phi))


def _axis_shift(coef, p, d, ax, up):
    """One axis of a Taylor shift by d on graded coefficients (dict k -> value):
    up (M2M): out_k = sum_{j_ax <= k_ax} C(k_ax, j_ax) d^{k_ax - j_ax} in_{k: k_ax = j_ax};
    down (L2L): out_k = sum_{j_ax >= k_ax, |j| <= p} C(j_ax, k_ax) d^{j_ax - k_ax} in_{k: k_ax = j_ax}."""
    out = {}
    for k in coef:
        s = 0.0
        if up:
            js = range(0, k[ax] + 1)
        else:
            js = range(k[ax], p - (sum(k) - k[ax]) + 1)
        for j in js:
            m = list(k)
            m[ax] = j
            n, r = (k[ax], j) if up else (j, k[ax])
            s += math.comb(n, r) * d ** (n - r) * coef[tuple(m)]
        out[k] = s
    return out


@pytest.mark.parametrize("up", [True, False], ids=["m2m", "l2l"])
def test_separable_shift_equals_multi_index_shift(up):
    """The device's M2M and L2L apply the shift axis by axis (x, then y, then z);
    the product form C(k, k') d^{k-k'} = prod_a C(k_a, k'_a) d_a^{k_a - k'_a} makes
    that equal to the oracle's multi-index shift, truncated at total degree p."""
    p = 7
    ops = Ops(p)
    rng = np.random.default_rng(5)
    x = rng.normal(size=ops.np_) + 1j * rng.normal(size=ops.np_)
    dc = np.array([0.31, -0.22, 0.17])
    ref = ops.m2m(x, dc) if up else ops.l2l(x, dc)
    coef = {tuple(int(v) for v in k): x[t] for t, k in enumerate(ops.mi)}
    for ax in range(3):
        coef = _axis_shift(coef, p, dc[ax], ax, up)
    got = np.array([coef[tuple(int(v) for v in k)] for k in ops.mi])
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_wavenumber_rule_refines_coarse_levels():
    """Taylor translations between boxes with k h near 4 converge slowly; the
    opt-in rule kh_max refines the pairs of split boxes on such levels instead
    of translating them.  Free space, k = 4, a 4 x 4 x 1 slab (the coarsest
    translating level has k h = 4): at p = 4 the rule lowers the error
    against the brute-force sum more than fivefold, and the lists still cover
    every pair exactly once."""
    rng = np.random.default_rng(5)
    n = 400
    src = rng.uniform([-2, -2, -0.5], [2, 2, 0.5], size=(n, 3))
    q = rng.uniform(size=n) + 1j * rng.uniform(size=n)
    med = Medium([], [4.0])
    img = ImageTable(med, [(-0.5, 0.5)], n_images=4)
    d = src[:, None, :] - src[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, 1.0)
    G = np.exp(4j * r) / (4j * r)
    np.fill_diagonal(G, 0.0)
    ref = G @ q
    err = {}
    for kh in (None, 3.5):
        phi = TEFMM(med, img, 4, 8, kh_max=kh).setup(src, src).evaluate(q)
        err[kh] = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err[3.5] < err[None] / 5, err
    tr = Trees(med, src, src, 8, kh_max=3.5)
    V, P2P = build_lists(tr, 0, 0)
    cover = np.zeros((n, n), dtype=np.int64)
    for t, lst in V.items():
        for s in lst:
            if not (tr.is_leaf[t] or tr.is_leaf[s]):   # split pairs are not translated above the bound
                assert tr.kmax * tr.side / float(1 << int(tr.level[t])) <= 3.5
            cover[tr.t0[t]:tr.t1[t], tr.s0[s]:tr.s1[s]] += 1
    for t, lst in P2P.items():
        for s in lst:
            cover[tr.t0[t]:tr.t1[t], tr.s0[s]:tr.s1[s]] += 1
    assert np.all(cover == 1)


def test_far_of_near_keeps_the_error():
    """The far-of-near reading moves the images of adjacent same-level leaf
    pairs with -Re Z >= 10^(10/(p+1)) sqrt(3) h out of the direct sum and into
    M2L; at p = 8 on a three-slab case with small leaves (so that such images
    exist) the error against the direct sum stays that of the plain form
    (within 1.5x plus 1e-9), and images and pairs were moved."""
    from oracle.tefmm import fon_threshold
    from oracle.direct import direct_sum, cross_sum
    w = W.three_layer_slabs(900, 8, 6, seed=6, n_images=16, half_width=0.4)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images)
    idx = np.random.default_rng(2).choice(len(w.src), 30, replace=False)
    ref = direct_sum(med, img, w.src, w.q, w.src[idx]) + cross_sum(med, w.zext, w.src, w.q, w.src[idx], 16)
    err, moved = {}, 0
    for fon in (False, True):
        f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images, far_of_near=fon).setup(w.src, w.src)
        phi = f.evaluate(w.q, target_index=idx)
        err[fon] = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
        if fon:
            tr = f.tr
            for (lt, ls), (_, P2P) in f.lists.items():
                if lt != ls:
                    continue
                for t, lst in P2P.items():
                    thr = fon_threshold(w.p, tr.side, int(tr.level[t]))
                    nfar = sum(int(np.sum(-np.real(tt['Z']) >= thr)) for tt in img.terms[lt])
                    moved += nfar * sum(1 for s in lst if tr.level[s] == tr.level[t])
    print(err, moved)
    assert moved > 0
    assert err[True] <= 1.5 * err[False] + 1e-9, err


def test_far_of_near_mixed_levels_keeps_the_error():
    """Adaptive tree (clusters): near-list pairs of different levels take the
    far-of-near reading at the coarser level l* through the anchors (T*, S*)
    of ``fon_anchor`` (the level-l* boxes holding them, adjacent): one M2L per
    anchor, the pair sums without those images.  The error against the
    direct sum stays that of the plain form (within 1.5x plus 1e-9), with
    anchors of both kinds (T* split, S* split) present; every anchor is a pair
    of adjacent same-level boxes, one of them a leaf of the pair."""
    from oracle.tefmm import fon_anchor
    w = W.clustered(1500, p=8, leaf_cap=8, seed=2, n_clusters=4, n_images=16)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images)
    idx = np.random.default_rng(3).choice(len(w.src), 40, replace=False)
    ref = direct_sum(med, img, w.src, w.q, w.src[idx])
    err = {}
    for fon in (False, True):
        f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images, far_of_near=fon).setup(w.src, w.src)
        err[fon] = np.linalg.norm(f.evaluate(w.q, target_index=idx) - ref) / np.linalg.norm(ref)
    tr = f.tr
    kinds = set()
    for t, lst in f.lists[(1, 1)][1].items():
        for s in lst:
            a = fon_anchor(tr, t, s)
            if a is None:
                continue
            l, T, S = a
            assert tr.level[T] == tr.level[S] == l and (T == t or S == s)
            kinds.add((T == t, S == s))
    print(err, kinds)
    assert {(True, False), (False, True), (True, True)} <= kinds
    assert err[True] <= 1.5 * err[False] + 1e-9, err
