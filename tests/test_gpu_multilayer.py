"""General media and the irregular-domain workload on the GPU, ``-m gpu``.

* 4- and 5-layer media (interfaces 0, -1, -2, ..; k = 1.5, 2.0, 2.5, ..):
  trees and lists bit-exact against the oracle's, and the FP64 form within
  1e-11 of the oracle's TE-FMM when both use the oracle's same-layer images
  and cross-layer fits (every one of the L(L-1) cross-layer components, both
  directions of reciprocity, present);
* the paper's Example 2 (particles in the irregular domains of its Sec. 5,
  three layers): the FP64 form against the oracle's TE-FMM as above, and the
  mixed form at 60k points against the oracle's direct sum at sampled targets.
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm
from oracle.tefmm import TEFMM
from oracle.direct import direct_sum, cross_sum

from _helpers import need_gpu, oracle_images, push_images, push_cross_fits, make_plan, gpu_eval, oracle_lists_csr

pytestmark = pytest.mark.gpu


def _parity(w):
    torch = need_gpu()
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    gpu_eval(plan, torch, w.src, w.q)
    f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src)
    push_cross_fits(plan, f)
    phi = gpu_eval(plan, torch, w.src, w.q)
    assert plan.stats()["n_cross_fits_last"] == 0
    g = plan.export_tree()
    tr = f.tr
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
    return err, f


@pytest.mark.parametrize("n_layers", [4, 5])
def test_multi_layer_fp64_matches_oracle(n_layers):
    w = W.multi_layer_slabs(60, n_layers, 4, 16, seed=1)
    err, f = _parity(w)
    pairs = {(lt, ls) for (lt, ls) in f.lists if lt != ls}
    print(f"{n_layers} layers: FP64 form vs oracle TE-FMM {err:.2e}, cross-layer components {len(pairs)}")
    assert len(pairs) == n_layers * (n_layers - 1)
    assert err <= 1e-11, err


def test_irregular_domains_fp64_matches_oracle():
    w = W.irregular_domains(450, 3, p=4, leaf_cap=16, seed=1)
    err, _ = _parity(w)
    print(f"irregular domains: FP64 form vs oracle TE-FMM {err:.2e}")
    assert err <= 1e-11, err


def test_irregular_domains_mixed_against_direct_sum():
    torch = need_gpu()
    w = W.irregular_domains(60000, 3, p=8, leaf_cap=64, seed=2)
    med, img = oracle_images(w)
    plan = make_plan(w, precision=tefmm.MIXED)
    phi = gpu_eval(plan, torch, w.src, w.q)
    idx = np.random.default_rng(3).choice(len(w.src), 40, replace=False)
    ref = direct_sum(med, img, w.src, w.q, w.src[idx]) + \
        cross_sum(med, w.zext, w.src, w.q, w.src[idx], n_images=w.n_images)
    err = np.linalg.norm(phi[idx] - ref) / np.linalg.norm(ref)
    print(f"irregular domains, 60k points, p=8, mixed form vs direct sum at 40 targets: {err:.2e}")
    assert err <= 1e-5, err


def test_clustered_deep_tree_fp64_matches_oracle():
    """32 Gaussian clusters (sigma 0.05) in the middle layer: an adaptive tree
    several levels deeper in the clusters than between them, with W and X
    pairs; trees, lists and the FP64 form against the oracle as above."""
    w = W.clustered(1500, p=4, leaf_cap=12, seed=3, n_clusters=8)
    err, f = _parity(w)
    depth = int(f.tr.level.max())
    print(f"clustered: depth {depth}, FP64 form vs oracle TE-FMM {err:.2e}")
    assert depth >= 5
    assert err <= 1e-11, err
