"""GPU path against the CPU oracle, through the C-ABI (``-m gpu``).

* integer work (Morton sort, octree, V lists, near-field lists) bit-exact;
* FP64 moments, locals and potentials within 1e-11 relative of the oracle's
  TE-FMM fed the same DCIM images;
* the device DCIM fits approach the Sommerfeld quadrature truth;
* edge cases: empty inputs, single points, ragged leaves, distinct targets,
  points on an interface or outside their layer's range.
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from oracle.tefmm import TEFMM, build_lists, Trees
from oracle.direct import direct_sum

from _helpers import need_gpu, oracle_images, push_images, make_plan, gpu_eval, oracle_lists_csr

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


def _cases():
    return [
        W.cfg_small(),                                              # 2000 pts, p 6, cap 60
        W.middle_layer_uniform(3001, 5, 17, seed=4, name="ragged"),  # many leaves, ragged tail
    ]


@pytest.mark.parametrize("w", _cases(), ids=lambda w: w.name)
def test_tree_and_lists_bit_exact(w):
    torch = need_gpu()
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    gpu_eval(plan, torch, w.src, w.q)
    g = plan.export_tree()
    f = TEFMM(med, img, w.p, w.leaf_cap).setup(w.src, w.src)
    tr = f.tr
    assert g["n_nodes"] == tr.n_nodes
    for key, ref in (("layer", tr.layer), ("level", tr.level), ("ix", tr.ix), ("iy", tr.iy),
                     ("iz", tr.iz), ("parent", tr.parent), ("s0", tr.s0), ("s1", tr.s1),
                     ("t0", tr.t0), ("t1", tr.t1)):
        assert np.array_equal(g[key].astype(np.int64), np.asarray(ref, dtype=np.int64)), key
    assert np.array_equal(g["perm_s"], tr.sperm)
    assert np.array_equal(g["perm_t"], tr.tperm)
    vp, vs, npp, ns_ = plan.export_lists()
    (rvp, rvs), (rnp, rns) = oracle_lists_csr(tr, f.lists, tr.n_nodes)
    assert np.array_equal(vp, rvp) and np.array_equal(vs, rvs)
    assert np.array_equal(npp, rnp) and np.array_equal(ns_, rns)


@pytest.mark.parametrize("w", _cases(), ids=lambda w: w.name)
def test_fp64_fmm_matches_oracle_fmm(w):
    torch = need_gpu()
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    phi = gpu_eval(plan, torch, w.src, w.q)
    f = TEFMM(med, img, w.p, w.leaf_cap).setup(w.src, w.src)
    alpha = f.upward(w.q)
    beta = f.downward(alpha)
    ga, gb = plan.export_expansions()
    sel = [n for n in range(f.tr.n_nodes) if f.tr.ns(n) > 0]
    assert np.max(np.abs(ga[sel] - alpha[sel])) <= FP64_TOL * np.max(np.abs(alpha[sel]))
    selt = [n for n in range(f.tr.n_nodes) if f.tr.nt(n) > 0]
    for n in selt:   # locals, per node, relative to the node's largest coefficient
        scale = np.max(np.abs(beta[n])) + 1e-300
        assert np.max(np.abs(gb[n] - beta[n])) <= 1e-10 * scale, n
    ref = f.evaluate(w.q)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err <= FP64_TOL, err
    # most tables come from a reflected or swapped key's table (x <-> -x, y <-> -y, x <-> y)
    st = plan.stats()
    assert 0 < st["n_tables_built"] < st["n_tables"], st


def test_distinct_targets_and_ragged_sizes():
    torch = need_gpu()
    w = W.middle_layer_uniform(1500, 4, 23, seed=9)
    rng = np.random.default_rng(10)
    tgt = rng.uniform([-1, -1, -1.1], [1, 1, -0.1], size=(977, 3))
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    phi = gpu_eval(plan, torch, w.src, w.q, tgt)
    f = TEFMM(med, img, w.p, w.leaf_cap).setup(w.src, tgt)
    ref = f.evaluate(w.q)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) <= FP64_TOL
    g = plan.export_tree()
    assert np.array_equal(g["perm_t"], f.tr.tperm)
    assert np.array_equal(g["t0"], f.tr.t0) and np.array_equal(g["s1"], f.tr.s1)


def test_fmm_close_to_direct_sum():
    torch = need_gpu()
    w = W.cfg_small()
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    phi = gpu_eval(plan, torch, w.src, w.q)
    ref = direct_sum(med, img, w.src, w.q, w.src)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err      # TE truncation at p = 6


def test_device_fit_against_quadrature():
    """Images fitted on the device reproduce the Sommerfeld-integral truth."""
    torch = need_gpu()
    from oracle.sommerfeld import reaction_derivative
    from oracle.dcim import ImageTable
    w = W.middle_layer_uniform(64, 4, 16, seed=2, n_images=16)
    plan = make_plan(w)
    med, _ = oracle_images(w)
    # evaluate the device images with the oracle's image-sum formula
    tab = ImageTable.__new__(ImageTable)
    tab.med = med
    tab.terms = [[] for _ in range(med.n_layers)]
    for t in plan.images():
        tab.terms[t['layer']].append(dict(tag=t['tag'], sz=t['sz'], szp=t['szp'], c=t['c'],
                                          zeta_min=t['zeta_min'], A=t['A'], Z=t['Z']))
    rng = np.random.default_rng(12)
    worst = 0.0
    for _ in range(12):
        r = np.r_[rng.uniform(-1, 1, 2), rng.uniform(-1.1, -0.1)]
        rp = np.r_[rng.uniform(-1, 1, 2), rng.uniform(-1.1, -0.1)]
        q = reaction_derivative(med, 1, 1, r, rp, part='both')
        worst = max(worst, abs(tab.reaction(1, *r, *rp) - q) / abs(q))
    assert worst < 5e-5, worst
    assert plan.stats()["fit_max_resid"] < 1e-3


def test_device_fit_close_to_oracle_fit():
    torch = need_gpu()
    w = W.cfg_small()
    plan = make_plan(w)
    med, img = oracle_images(w)
    dev = plan.images()
    for t in dev:
        o = [x for x in img.terms[t['layer']] if x['tag'] == {0: 'uu', 1: 'dd', 2: 'ud', 3: 'du'}[t['tag']]][0]
        assert len(t['A']) == len(o['A']), (t['tag'], len(t['A']), len(o['A']))
    # the two image sets approximate the same function to DCIM accuracy
    rng = np.random.default_rng(3)
    from oracle.dcim import ImageTable
    tab = ImageTable.__new__(ImageTable)
    tab.med = med
    tab.terms = [[] for _ in range(med.n_layers)]
    for t in dev:
        tab.terms[t['layer']].append(dict(tag=t['tag'], sz=t['sz'], szp=t['szp'], c=t['c'],
                                          zeta_min=t['zeta_min'], A=t['A'], Z=t['Z']))
    a = rng.uniform([-1, -1, -1.1], [1, 1, -0.1], size=(200, 3))
    b = rng.uniform([-1, -1, -1.1], [1, 1, -0.1], size=(200, 3))
    u_dev = tab.reaction(1, a[:, 0], a[:, 1], a[:, 2], b[:, 0], b[:, 1], b[:, 2])
    u_ora = img.reaction(1, a[:, 0], a[:, 1], a[:, 2], b[:, 0], b[:, 1], b[:, 2])
    assert np.max(np.abs(u_dev - u_ora)) / np.max(np.abs(u_ora)) < 1e-6


def test_edge_cases():
    torch = need_gpu()
    from paper_1902_05875_gb300 import tefmm
    w = W.middle_layer_uniform(10, 3, 4, seed=5)
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    dev = "cuda:0"
    e = torch.empty(0, dtype=torch.float64, device=dev)
    eq = torch.empty(0, dtype=torch.complex128, device=dev)
    # no sources: zeros
    tx = torch.tensor(w.src[:, 0], device=dev)
    ty = torch.tensor(w.src[:, 1], device=dev)
    tz = torch.tensor(w.src[:, 2], device=dev)
    out = plan.eval(e, e, e, eq, tx, ty, tz)
    assert torch.all(out == 0)
    # no targets
    out = plan.eval(tx, ty, tz, torch.tensor(w.q, device=dev), e, e, e)
    assert out.numel() == 0
    # one point: no free-space self term, only its own reaction field
    one = w.src[:1]
    phi = gpu_eval(plan, torch, one, w.q[:1])
    ref = direct_sum(med, img, one, w.q[:1], one)
    assert abs(phi[0] - ref[0]) <= 1e-12 * abs(ref[0])
    # two coincident points: free-space pair skipped for identical coordinates
    two = np.repeat(w.src[:1], 2, axis=0)
    phi = gpu_eval(plan, torch, two, w.q[:2])
    ref = direct_sum(med, img, two, w.q[:2], two)
    assert np.max(np.abs(phi - ref)) <= 1e-12 * np.max(np.abs(ref))
    # all points exact (tiny N, whole tree is near field)
    phi = gpu_eval(plan, torch, w.src, w.q)
    ref = direct_sum(med, img, w.src, w.q, w.src)
    assert np.max(np.abs(phi - ref)) <= 1e-10 * np.max(np.abs(ref))
    # a point exactly on an interface
    bad = w.src.copy()
    bad[3, 2] = -1.2
    with pytest.raises(tefmm.TefmmError) as ei:
        gpu_eval(plan, torch, bad, w.q)
    assert ei.value.status == -2
    # a point in the middle layer but outside its declared particle range
    bad = w.src.copy()
    bad[3, 2] = -0.05
    with pytest.raises(tefmm.TefmmError) as ei:
        gpu_eval(plan, torch, bad, w.q)
    assert ei.value.status == -3


def test_eval_host_matches_device():
    torch = need_gpu()
    w = W.middle_layer_uniform(1200, 4, 30, seed=6)
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    a = gpu_eval(plan, torch, w.src, w.q)
    b = plan.eval_host(w.src, w.q)
    # M2L accumulates with atomics, so the summation order (last bits) may differ
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_full_size_200k_sampled_targets():
    """The 200k-point, p = 8 workload at the bench's launch configuration:
    sampled targets against the oracle's per-target TE-FMM (same images) and
    against the direct sum."""
    torch = need_gpu()
    w = W.cfg_fp64_200k()
    med, img = oracle_images(w)
    plan = make_plan(w)
    push_images(plan, img)
    phi = gpu_eval(plan, torch, w.src, w.q)
    rng = np.random.default_rng(1)
    sel = rng.choice(len(w.src), size=6, replace=False)
    f = TEFMM(med, img, w.p, w.leaf_cap).setup(w.src, w.src)
    ref = f.evaluate(w.q, sel)
    assert np.max(np.abs(phi[sel] - ref) / np.abs(ref)) <= FP64_TOL
    sel2 = rng.choice(len(w.src), size=40, replace=False)
    d = direct_sum(med, img, w.src, w.q, w.src[sel2])
    err = np.linalg.norm(phi[sel2] - d) / np.linalg.norm(d)
    assert err < 1e-5, err
