"""Pins of the oracle's cross-layer components (Sec. 3.2-3.3, target layer l differs
from source layer l').

What fixes them independently of the oracle's own formulas:

* homogeneous medium (every k_l equal): the transmitted field of a source in
  another layer is the free-space field, so u_{l l'} = e^{ikR}/(ikR) exactly
  (closed form; checked on the Sommerfeld quadrature, on the per-point DCIM
  sum and on the whole TE-FMM);
* reciprocity of the transmission problem: with the k-weighted flux condition
  the weak form sum_l k_l int (grad u . grad v - k_l^2 u v) is symmetric, which
  gives k_l' G(r'; r) = k_l G(r; r'); the potentials here omit i k_l / 4pi of
  the target layer, hence  k_l^2 u_{l l'}(r; r') = k_l'^2 u_{l' l}(r'; r);
* the DCIM fits of d^{k3'}_{z'} u / k3'! (every k3') against the Sommerfeld
  quadrature of the same derivative: within 1e-7 when the target layer has
  the larger |k| (the fits the product uses; 4.2e-8 at worst here), within
  5e-6 when it has the smaller one (layer 2 seen from layer 0 reaches 2e-6;
  the product takes those components through reciprocity instead);
* brute force: the TE-FMM with all nine components against the direct sum
  (same-layer images + per-source-point cross-layer fits), with an error that
  falls as p rises; a planted sign error in the down-going cross-layer tables
  is detected;
* which layer holds a component's images: against the Sommerfeld quadrature,
  fits whose images live in the layer of the larger |k| are accurate to about
  1e-8, fits in the smaller-|k| layer only to 1e-6 .. 4e-4; the cross-layer
  direct sum built on that choice (``cross_sum``) matches the quadrature sum
  to 2e-7, and its binned z'-Taylor part matches per-source fits to 2e-8;
* the cross-layer split rule and the stacked cross-layer admissibility rule:
  no cross-layer pair is left to the near field, and the lists still cover
  every (target, source) pair exactly once; on slabs 0.1 from the interfaces
  the admissibility rule lowers the cross-layer error by two orders.
"""
import numpy as np
import pytest

from oracle.medium import Medium
from oracle.dcim import ImageTable
from oracle.cross import CrossDirect, directions, fit_cross, image_sum, W_min
from oracle.direct import (direct_sum, cross_sum, cross_sum_binned, cross_sum_by_reciprocity,
                           images_in_source_layer)
from oracle.sommerfeld import reaction_derivative
from oracle.tefmm import TEFMM, Trees, build_lists
from paper_1902_05875_gb300 import workloads as W

R_A = np.r_[0.3, -0.2, 0.7]      # layer 0
R_B = np.r_[-0.1, 0.4, -0.7]     # layer 1
R_C = np.r_[0.2, 0.1, -2.0]      # layer 2


def test_quadrature_homogeneous_cross_layer_is_free_space():
    med = Medium(W.CROSS_D, [3.0, 3.0, 3.0])
    for (a, la), (b, lb) in [((R_A, 0), (R_B, 1)), ((R_A, 0), (R_C, 2)), ((R_C, 2), (R_B, 1))]:
        u = reaction_derivative(med, la, lb, a, b)
        R = np.linalg.norm(a - b)
        ref = np.exp(3j * R) / (3j * R)
        assert abs(u - ref) <= 1e-12 * abs(ref), (la, lb, u, ref)


def test_quadrature_reciprocity():
    med = Medium(W.CROSS_D, W.CROSS_K)
    k = med.k
    for (a, la), (b, lb) in [((R_A, 0), (R_B, 1)), ((R_A, 0), (R_C, 2)), ((R_B, 1), (R_C, 2))]:
        u1 = reaction_derivative(med, la, lb, a, b)
        u2 = reaction_derivative(med, lb, la, b, a)
        lhs, rhs = k[la] ** 2 * u1, k[lb] ** 2 * u2
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (la, lb, lhs, rhs)


@pytest.mark.parametrize("l,lp,part,k3p", [(0, 1, 'up', 0), (0, 2, 'up', 0), (0, 2, 'up', 3),
                                           (1, 0, 'down', 6), (2, 1, 'down', 3), (1, 2, 'up', 6),
                                           (1, 0, 'up', 2), (2, 0, 'down', 5)])
def test_cross_fit_matches_quadrature(l, lp, part, k3p):
    med = Medium(W.CROSS_D, W.CROSS_K)
    zext = W.CROSS_ZEXT
    zc = float(np.mean(zext[lp]))
    wmin = W_min(med, l, part, zext)
    A, Z, _ = fit_cross(med, l, lp, part, zc, k3p, wmin, n_images=16)
    r = np.r_[0.3, -0.2, np.mean(zext[l]) + 0.1]
    rp = np.r_[-0.1, 0.4, zc]
    ref = reaction_derivative(med, l, lp, r, rp, k3p=k3p, part=part)
    got = image_sum(med, l, part, A, Z, wmin, *r, rp[0], rp[1])
    tol = 1e-7 if abs(med.k[l]) > abs(med.k[lp]) else 5e-6
    assert abs(got - ref) <= tol * abs(ref), (got, ref, tol)


def test_cross_direct_homogeneous_is_free_space():
    med = Medium(W.CROSS_D, [3.0, 3.0, 3.0])
    src = np.array([R_B, R_C])
    tgt = np.array([R_A, R_A + 0.05, R_C + np.r_[0.3, 0.0, 0.1]])
    q = np.array([1.0 + 0.5j, -0.3 + 0.2j])
    got = CrossDirect(med, W.CROSS_ZEXT, n_images=16).potential(src, q, tgt)
    ref = np.zeros(len(tgt), complex)
    lay_s, lay_t = med.layer_of(src[:, 2]), med.layer_of(tgt[:, 2])
    for i in range(len(tgt)):
        for j in range(len(src)):
            if lay_s[j] != lay_t[i]:
                R = np.linalg.norm(tgt[i] - src[j])
                ref[i] += q[j] * np.exp(3j * R) / (3j * R)
    assert np.max(np.abs(got - ref)) <= 1e-8 * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def slabs():
    w = W.cross_layer_slabs(120, 0, 5, seed=0)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images)
    ref = direct_sum(med, img, w.src, w.q, w.src) + \
        cross_sum(med, w.zext, w.src, w.q, w.src, n_images=w.n_images)
    return w, med, img, ref


def test_cross_layer_fmm_error_falls_with_p(slabs):
    w, med, img, ref = slabs
    errs = []
    for p in (2, 4, 6):
        f = TEFMM(med, img, p, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src)
        assert any(a != b for (a, b) in f.lists), "workload has no cross-layer component"
        phi = f.evaluate(w.q)
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
    assert all(b < 0.2 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 2e-3, errs


def test_cross_layer_fmm_detects_planted_sign_error(slabs, monkeypatch):
    """Drop the (-1)^{g3} of the down-going cross-layer tables: the error grows."""
    w, med, img, ref = slabs
    import oracle.tefmm as T
    good = TEFMM(med, img, 4, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src).evaluate(w.q)
    e_good = np.linalg.norm(good - ref) / np.linalg.norm(ref)
    real_tables = T.TEFMM._cross_tables

    def planted(self, lt, ls, lev, keys):
        tab = real_tables(self, lt, ls, lev, keys)
        # undo the (-1)^{g3} of the down-going part by recomputing it without the sign
        import oracle.cross as xl
        from oracle.derivs import taylor_h0, multi_indices
        tr, p = self.tr, self.p
        h = tr.side / float(1 << lev)
        mi2 = multi_indices(2 * p)
        odd3 = (-1.0) ** mi2[:, 2]
        if 'down' in xl.directions(self.med, lt):
            wmin = xl.W_min(self.med, lt, 'down', self.zext)
            for i, (dix, diy, izt, izs) in enumerate(np.asarray(keys).reshape(-1, 4)):
                W0 = float(xl.W_of(self.med, lt, 'down', self.cross_centre(lt, lev, int(izt))))
                for k3p in range(p + 1):
                    A, Z = self.cross_image(lt, ls, 'down', lev, int(izs), k3p)
                    if len(A) == 0:
                        continue
                    t = taylor_h0(np.full(len(A), dix * h), np.full(len(A), diy * h),
                                  W0 - wmin - np.asarray(Z), self.med.k[lt], 2 * p)
                    s = (np.asarray(A)[:, None] * t).sum(0)
                    tab[i, k3p] += s - odd3 * s
        return tab
    monkeypatch.setattr(T.TEFMM, "_cross_tables", planted)
    bad = TEFMM(med, img, 4, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src).evaluate(w.q)
    e_bad = np.linalg.norm(bad - ref) / np.linalg.norm(ref)
    assert e_bad > 20 * e_good, (e_bad, e_good)


def test_homogeneous_multi_layer_fmm_is_free_space():
    w = W.cross_layer_slabs(60, 0, 5, seed=2, k=[3.0, 3.0, 3.0])
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images)
    pts = w.src
    d = pts[:, None, :] - pts[None, :, :]
    R = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(R, 1.0)
    G = np.exp(3j * R) / (3j * R)
    np.fill_diagonal(G, 0.0)
    ref = G @ w.q
    errs = []
    for p in (3, 6):
        phi = TEFMM(med, img, p, w.leaf_cap, n_images=w.n_images).setup(pts, pts).evaluate(w.q)
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
    assert errs[1] < 0.1 * errs[0] and errs[1] < 1e-3, errs


@pytest.mark.parametrize("case", ["wide_gaps", "slabs_near_interfaces"])
def test_cross_split_rule_lists_partition_pairs(case):
    """The lists cover every (target, source) pair once; with slabs 0.1 from
    the interfaces the stacked cross-layer admissibility rule is active (HX = 0.8
    < the box size at levels 0-2) and must keep that property."""
    if case == "wide_gaps":
        w = W.cross_layer_slabs(80, 0, 5, seed=1)
    else:
        w = W.three_layer_slabs(300, 0, 8, seed=3, half_width=0.5)
    med = Medium(w.interfaces, w.k)
    tr = Trees(med, w.src, w.src, w.leaf_cap, zext=w.zext)
    if case != "wide_gaps":
        assert abs(tr.HX - 0.8) < 1e-12
        assert any(tr.cross_colleague(a, b) for a in range(tr.n_nodes) for b in range(tr.n_nodes)
                   if tr.level[a] == tr.level[b] and tr.level[a] <= 2)
    ns = len(w.src)
    cover = np.zeros((ns, ns), dtype=np.int64)
    for lt in range(3):
        for ls in range(3):
            V, P = build_lists(tr, lt, ls)
            if lt != ls:
                assert not P, "cross-layer pair left to the near field"
            for t, lst in V.items():
                for s in lst:
                    assert not tr.adjacent(t, s) and not tr.cross_colleague(t, s)
                    cover[np.ix_(tr.tperm[tr.t0[t]:tr.t1[t]], tr.sperm[tr.s0[s]:tr.s1[s]])] += 1
            for t, lst in P.items():
                for s in lst:
                    cover[np.ix_(tr.tperm[tr.t0[t]:tr.t1[t]], tr.sperm[tr.s0[s]:tr.s1[s]])] += 1
    assert np.all(cover == 1), (cover.min(), cover.max())


def test_cross_sum_by_reciprocity_matches_per_source_fits():
    """One fit per target (reciprocity) and one fit per source give the same
    cross-layer field (up to the fits' accuracy)."""
    w = W.cross_layer_slabs(25, 0, 5, seed=5)
    med = Medium(w.interfaces, w.k)
    tgt = w.src[::4]
    a = CrossDirect(med, w.zext, n_images=16).potential(w.src, w.q, tgt)
    b = cross_sum_by_reciprocity(med, w.zext, w.src, w.q, tgt, n_images=16)
    assert np.linalg.norm(a - b) <= 2e-6 * np.linalg.norm(a), np.linalg.norm(a - b) / np.linalg.norm(a)


@pytest.mark.slow
def test_stacked_cross_pairs_rule_improves_accuracy():
    """Slabs 0.1 from the interfaces, p = 3: taking stacked coarse cross-layer
    pairs as translations (HX = inf) vs pairing their children (HX = 0.8)."""
    import oracle.tefmm as T
    w = W.three_layer_slabs(180, 3, 8, seed=4, half_width=0.5)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=16)
    ref = direct_sum(med, img, w.src, w.q, w.src) + \
        cross_sum(med, w.zext, w.src, w.q, w.src, n_images=16)
    errs = {}
    for name, lim in (("rule", None), ("no_rule", np.inf)):
        f = TEFMM(med, img, 3, w.leaf_cap, n_images=16)
        if lim is not None:
            orig = T.cross_box_limit
            T.cross_box_limit = lambda med_, zext_: lim
            try:
                f.setup(w.src, w.src)
            finally:
                T.cross_box_limit = orig
        else:
            f.setup(w.src, w.src)
        phi = f.evaluate(w.q)
        errs[name] = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    print(errs)
    assert errs["rule"] < 0.2 * errs["no_rule"], errs


def _slab_medium():
    w = W.cfg_mixed_200k()
    return Medium(w.interfaces, w.k), w.zext


@pytest.mark.parametrize("l,lp", [(2, 0), (0, 2), (2, 1), (1, 2), (0, 1)])
def test_images_in_larger_k_layer_match_quadrature(l, lp):
    """Medium k = (2, 3, 4 + 0.01i), slabs 0.1 from the interfaces: a target
    and a source each 0.1 from the interfaces, horizontal offsets 0 .. 4.  The
    component u_{l l'} with its images in the larger-|k| layer (target layer,
    or the source layer by reciprocity) matches the quadrature to 2e-7; with
    the images in the other layer it misses by more than 1e-6 somewhere."""
    med, zext = _slab_medium()
    zt = zext[l][1] if l > lp else zext[l][0]
    zs = zext[lp][0] if l > lp else zext[lp][1]
    good, bad = [], []
    for rho in (0.0, 0.7, 2.0, 4.0):
        r, rp = np.r_[rho, 0.0, zt], np.r_[0.0, 0.0, zs]
        ref = sum(reaction_derivative(med, l, lp, r, rp, part=pt) for pt in directions(med, l))
        tgt_form = 0
        for pt in directions(med, l):
            wm = W_min(med, l, pt, zext)
            A, Z, _ = fit_cross(med, l, lp, pt, zs, 0, wm, n_images=16)
            tgt_form += image_sum(med, l, pt, A, Z, wm, *r, rp[0], rp[1])
        src_form = 0
        for pt in directions(med, lp):
            wm = W_min(med, lp, pt, zext)
            A, Z, _ = fit_cross(med, lp, l, pt, zt, 0, wm, n_images=16)
            src_form += image_sum(med, lp, pt, A, Z, wm, *rp, r[0], r[1])
        src_form *= (med.k[lp] / med.k[l]) ** 2
        if images_in_source_layer(med, l, lp):
            good.append(abs(src_form - ref) / abs(ref))
            bad.append(abs(tgt_form - ref) / abs(ref))
        else:
            good.append(abs(tgt_form - ref) / abs(ref))
            bad.append(abs(src_form - ref) / abs(ref))
    assert max(good) <= 2e-7, good
    assert max(bad) > 1e-6, bad


@pytest.fixture(scope="module")
def small_slabs():
    w = W.three_layer_slabs(150, 4, 16, seed=3, n_images=16, name="small_slabs")
    med = Medium(w.interfaces, w.k)
    tgt = w.src[np.random.default_rng(7).choice(len(w.src), 40, replace=False)]
    return w, med, tgt


def test_cross_sum_binned_matches_per_source_fits(small_slabs):
    """The binned z'-Taylor form (fits at bin centres, order 6) against one fit
    per source point at its exact z' (``CrossDirect``), on the layer pairs where
    the images are in the target layer."""
    w, med, tgt = small_slabs
    nr = lambda l, lp: not images_in_source_layer(med, l, lp)
    got = cross_sum_binned(med, w.zext, w.src, w.q, tgt, 16, pairs=nr)
    tl, sl = med.layer_of(tgt[:, 2]), med.layer_of(w.src[:, 2])
    ref = np.zeros(len(tgt), complex)
    for lp in range(med.n_layers):
        m = sl == lp
        part = CrossDirect(med, w.zext, n_images=16).potential(w.src[m], w.q[m], tgt)
        sel = np.array([tl[i] != lp and nr(tl[i], lp) for i in range(len(tgt))])
        ref[sel] += part[sel]
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(got - ref) <= 2e-8 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_cross_sum_matches_quadrature(small_slabs):
    """The cross-layer direct sum (``cross_sum``) against the pairwise
    Sommerfeld quadrature at 3 targets in each layer: within 2e-7, while
    either single representation (all images in the source layer, or all in
    the target layer) misses by more than 5e-6."""
    w, med, tgt = small_slabs
    lay = med.layer_of(tgt[:, 2])
    tgt = np.concatenate([tgt[lay == l][:3] for l in range(3)])
    src, q = w.src[::3], w.q[::3]
    tl, sl = med.layer_of(tgt[:, 2]), med.layer_of(src[:, 2])
    assert len(set(tl)) == 3
    truth = np.zeros(len(tgt), complex)
    for i in range(len(tgt)):
        for j in range(len(src)):
            if tl[i] != sl[j]:
                truth[i] += q[j] * sum(reaction_derivative(med, tl[i], sl[j], tgt[i], src[j], part=pt)
                                       for pt in directions(med, tl[i]))
    err = lambda v: np.linalg.norm(v - truth) / np.linalg.norm(truth)
    assert err(cross_sum(med, w.zext, src, q, tgt, 16)) <= 2e-7
    assert err(cross_sum_by_reciprocity(med, w.zext, src, q, tgt, 16)) > 5e-6
    assert err(CrossDirect(med, w.zext, n_images=16).potential(src, q, tgt)) > 5e-6
