"""Parity at the configuration the benchmark times, ``-m gpu``.

The 2M three-slab workload's geometry and medium (slabs 0.1 from the
interfaces, k = (2, 3, 4 + 0.01i), 16 images per fit, leaf cap 64) at p = 10,
with 3000 points: every rule of the benchmark is active on it -- the
wavenumber admissibility (level 2 has k_max h = 4 > 3.5, its split boxes are
paired), the stacked cross-layer rule (HX = 0.8), cross-layer keys in both
directions (a target layer with the smaller |k| uses the transposed matrix of
its mirror pair), three output slices of the tensor-core M2L (2 n_p = 572
columns) and the order-20 derivative tables.

The device runs on the oracle's images (same-layer and cross-layer, imported),
and its potentials are compared element by element with the oracle's TE-FMM
at 24 sampled targets: the FP64 form within 1e-11, the mixed form within
2e-6 (its FP32/TF32 rounding; measured values printed).
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm
from oracle.tefmm import TEFMM

from _helpers import need_gpu, oracle_images, push_images, push_cross_fits, make_plan, gpu_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    w = W.three_layer_slabs(3000, 10, 64, seed=0, n_images=16, name="three_layer_slabs_n3000_p10")
    med, img = oracle_images(w)
    f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src)
    idx = np.random.default_rng(1).choice(len(w.src), 24, replace=False)
    return w, med, img, f, idx


def _run(case, precision):
    torch = need_gpu()
    w, med, img, f, idx = case
    plan = make_plan(w, precision=precision)
    push_images(plan, img)
    gpu_eval(plan, torch, w.src, w.q)
    push_cross_fits(plan, f)
    phi = gpu_eval(plan, torch, w.src, w.q)
    st = plan.stats()
    assert st["n_cross_fits_last"] == 0
    return phi, st


def test_bench_config_fp64_matches_oracle(case):
    w, med, img, f, idx = case
    phi, st = _run(case, tefmm.FP64)
    assert f.tr.kh_max is not None and f.tr.kmax * f.tr.side / 4 > f.tr.kh_max   # level 2 is coarse
    assert abs(f.tr.HX - 0.8) < 1e-12
    assert st["n_cross_tables"] > 0 and st["n_tables_built"] < st["n_tables"]
    ref = f.evaluate(w.q, target_index=idx)
    err = np.linalg.norm(phi[idx] - ref) / np.linalg.norm(ref)
    worst = np.max(np.abs(phi[idx] - ref) / np.abs(ref))
    print(f"p=10 three-slab, FP64 form vs oracle TE-FMM at {len(idx)} targets: "
          f"rel L2 {err:.2e}, max rel {worst:.2e}")
    assert err <= 1e-11, err


def test_bench_config_mixed_matches_oracle(case):
    w, med, img, f, idx = case
    phi, st = _run(case, tefmm.MIXED)
    ref = f.evaluate(w.q, target_index=idx)
    err = np.linalg.norm(phi[idx] - ref) / np.linalg.norm(ref)
    worst = np.max(np.abs(phi[idx] - ref) / np.abs(ref))
    print(f"p=10 three-slab, mixed form vs oracle TE-FMM at {len(idx)} targets: "
          f"rel L2 {err:.2e}, max rel {worst:.2e}")
    assert err <= 2e-6, err


def test_far_of_near_changes_the_fp64_form_below_its_bound(case):
    """The device's far-of-near path (far images of near pairs through the
    M2L of their anchors) against every image in P2P, FP64 form, same images:
    the two agree far below the method's error (1e-8), and pairs were moved.
    The near field's count of (pair, image term) evaluations is pairs x images
    per target layer without the reading and smaller with it."""
    torch = need_gpu()
    w, med, img, f, idx = case
    out, terms = {}, {}
    for fon in (True, False):
        plan = make_plan(w, far_of_near=fon)
        push_images(plan, img)
        out[fon] = gpu_eval(plan, torch, w.src, w.q)
        st = plan.stats()
        terms[fon] = st["n_near_img_terms"]
        if fon:
            assert st["n_fon_pairs"] > 0
        else:
            per_layer = [sum(len(t["A"]) for t in plan.images() if t["layer"] == l) for l in range(len(w.k))]
            assert terms[False] == sum(int(p) * m for p, m in zip(st["n_p2p_pairs_layer"], per_layer))
    assert 0 < terms[True] < terms[False], terms
    err = np.linalg.norm(out[True] - out[False]) / np.linalg.norm(out[False])
    print(f"far-of-near on vs off (FP64 form, p=10): {err:.2e}")
    assert err <= 1e-8, err
