"""Cross-layer components on the GPU (target layer != source layer), ``-m gpu``.

* the octree with the cross-layer split rule and the merged V / near lists
  bit-exact against the oracle's;
* the FP64 form within 1e-11 of the oracle's TE-FMM with the same images:
  the plan's same-layer images and cross-layer fits are replaced by the
  oracle's (``set_images``, ``set_cross_images``), so the oracle never takes a
  value the device computed;
* the device cross-layer fits against Sommerfeld quadrature of the same
  z'-derivative;
* the whole product (device fits, p = 8) against the oracle's direct sum;
* the mixed form against the FP64 form; the fit cache (no refit for the same
  root cube, refit when it changes).
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm
from oracle.tefmm import TEFMM
from oracle.cross import image_sum, W_min
from oracle.direct import direct_sum, cross_sum
from oracle.sommerfeld import reaction_derivative

from _helpers import (need_gpu, oracle_images, push_images, push_cross_fits, make_plan, gpu_eval,
                      oracle_lists_csr)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


def _w(p=4, n=120, seed=0):
    return W.cross_layer_slabs(n, p, 5, seed=seed)


def test_cross_tree_and_lists_bit_exact():
    torch = need_gpu()
    w = _w()
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    gpu_eval(plan, torch, w.src, w.q)
    g = plan.export_tree()
    f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src)
    tr = f.tr
    assert g["n_nodes"] == tr.n_nodes
    for key, ref in (("layer", tr.layer), ("level", tr.level), ("ix", tr.ix), ("iy", tr.iy),
                     ("iz", tr.iz), ("parent", tr.parent), ("s0", tr.s0), ("s1", tr.s1),
                     ("t0", tr.t0), ("t1", tr.t1)):
        assert np.array_equal(g[key].astype(np.int64), np.asarray(ref, dtype=np.int64)), key
    assert np.array_equal(g["perm_s"], tr.sperm)
    vp, vs, npp, ns_ = plan.export_lists()
    (rvp, rvs), (rnp, rns) = oracle_lists_csr(tr, f.lists, tr.n_nodes)
    assert np.array_equal(vp, rvp) and np.array_equal(vs, rvs)
    assert np.array_equal(npp, rnp) and np.array_equal(ns_, rns)
    assert any(a != b for (a, b) in f.lists)
    assert plan.stats()["n_cross_tables"] > 0


def test_cross_fp64_matches_oracle_fmm():
    torch = need_gpu()
    w = _w()
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    gpu_eval(plan, torch, w.src, w.q)
    f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src)
    keys = push_cross_fits(plan, f)
    phi = gpu_eval(plan, torch, w.src, w.q)
    assert plan.stats()["n_cross_fits_last"] == 0        # every fit came from the oracle
    alpha = f.upward(w.q)
    beta = f.downward(alpha)
    assert sorted(f.cross_images) == keys, "the oracle and the plan use different fits"
    ga, gb = plan.export_expansions()
    for n in range(f.tr.n_nodes):
        if f.tr.nt(n) > 0:
            scale = np.max(np.abs(beta[n])) + 1e-300
            assert np.max(np.abs(gb[n] - beta[n])) <= 1e-10 * scale, n
    ref = f.evaluate(w.q)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    print(f'cross-layer FP64 form vs oracle TE-FMM: {err:.3e}')
    assert err <= FP64_TOL, err


def test_cross_device_fits_against_quadrature():
    torch = need_gpu()
    w = _w()
    med, img = oracle_images(w)
    plan = make_plan(w)
    gpu_eval(plan, torch, w.src, w.q)
    xi = plan.cross_images()
    g = plan.export_tree()
    lo = w.src.min(axis=0)
    side = float(np.max(w.src.max(axis=0) - lo))
    keys = sorted(xi)
    rng = np.random.default_rng(0)
    worst = 0.0
    for i in rng.choice(len(keys), min(12, len(keys)), replace=False):
        lt, ls, part, lev, izs, k3p = keys[i]
        A, Z = xi[keys[i]]
        zc = min(max(lo[2] + (izs + 0.5) * side / 2 ** lev, w.zext[ls][0]), w.zext[ls][1])
        wmin = W_min(med, lt, part, w.zext)
        r = np.r_[0.3, -0.2, np.mean(w.zext[lt])]
        rp = np.r_[-0.1, 0.2, zc]
        ref = reaction_derivative(med, lt, ls, r, rp, k3p=k3p, part=part)
        got = image_sum(med, lt, part, A, Z, wmin, *r, rp[0], rp[1])
        worst = max(worst, abs(got - ref) / abs(ref))
    print(f'device cross-layer fits vs quadrature: worst {worst:.2e}')
    assert worst < 5e-6, worst
    assert g["n_nodes"] > 0


def test_cross_fmm_against_direct_sum():
    torch = need_gpu()
    w = _w(p=8)
    med, img = oracle_images(w)
    plan = make_plan(w)
    phi = gpu_eval(plan, torch, w.src, w.q)
    ref = direct_sum(med, img, w.src, w.q, w.src) + \
        cross_sum(med, w.zext, w.src, w.q, w.src, n_images=w.n_images)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    print(f'cross-layer product (device fits, p=8) vs direct sum: {err:.3e}')
    assert err < 1e-4, err


def test_cross_mixed_close_to_fp64_form():
    torch = need_gpu()
    w = _w(p=6)
    med, img = oracle_images(w)
    p64 = make_plan(w)
    push_images(p64, img)
    pmx = make_plan(w, precision=tefmm.MIXED)
    push_images(pmx, img)
    a = gpu_eval(p64, torch, w.src, w.q)
    b = gpu_eval(pmx, torch, w.src, w.q)
    err = np.linalg.norm(a - b) / np.linalg.norm(a)
    print(f'cross-layer mixed vs fp64 form: {err:.3e}')
    assert err < 1.5e-6, err      # measured 7.2e-7


def test_cross_fit_cache():
    torch = need_gpu()
    w = _w()
    plan = make_plan(w)
    a = gpu_eval(plan, torch, w.src, w.q)
    s1 = plan.stats()
    assert s1["n_cross_fits_last"] == s1["n_cross_fits"] > 0
    b = gpu_eval(plan, torch, w.src, w.q)
    s2 = plan.stats()
    assert s2["n_cross_fits_last"] == 0 and s2["n_cross_fits"] == s1["n_cross_fits"]
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
    # a larger root cube (x extent 3.5 > z extent 3.2) moves every source
    # z-centre: everything is refitted
    src = np.concatenate([w.src, [[3.0, 0.2, 0.6]]])
    q = np.concatenate([w.q, [0.5 + 0.5j]])
    gpu_eval(plan, torch, src, q)
    s3 = plan.stats()
    assert s3["n_cross_fits_last"] > 0


def test_stacked_cross_rule_tree_lists_and_fp64_parity():
    """Slabs 0.1 from the interfaces (HX = 0.8): the stacked cross-layer
    admissibility rule is active; trees and lists stay bit-exact and the FP64
    form, run on the oracle's cross-layer fits, matches the oracle's TE-FMM."""
    torch = need_gpu()
    w = W.three_layer_slabs(240, 3, 8, seed=4, half_width=0.5, n_images=16)
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    gpu_eval(plan, torch, w.src, w.q)
    f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src)
    push_cross_fits(plan, f)
    phi = gpu_eval(plan, torch, w.src, w.q)
    tr = f.tr
    assert abs(tr.HX - 0.8) < 1e-12
    g = plan.export_tree()
    assert g["n_nodes"] == tr.n_nodes
    for key, ref in (("layer", tr.layer), ("level", tr.level), ("ix", tr.ix), ("iy", tr.iy),
                     ("iz", tr.iz), ("parent", tr.parent), ("s0", tr.s0), ("t1", tr.t1)):
        assert np.array_equal(g[key].astype(np.int64), np.asarray(ref, dtype=np.int64)), key
    vp, vs, npp, ns_ = plan.export_lists()
    (rvp, rvs), (rnp, rns) = oracle_lists_csr(tr, f.lists, tr.n_nodes)
    assert np.array_equal(vp, rvp) and np.array_equal(vs, rvs)
    assert np.array_equal(npp, rnp) and np.array_equal(ns_, rns)
    ref = f.evaluate(w.q)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    print(f'stacked cross rule, FP64 form vs oracle TE-FMM: {err:.3e}')
    assert err <= FP64_TOL, err
