"""Batched evaluation of independent instances and the leaf-cap autotuner (``-m gpu``).

* ``tefmm_eval_batched`` gives each instance the same potentials as its own
  ``tefmm_eval`` (instances run concurrently on several streams);
* one instance of the batch against the oracle's FP64 direct sum (same-layer
  images plus the cross-layer field by one fit per target) at sampled targets,
  in the FP64 and the mixed form;
* a plan made with leaf_cap = 0 picks one of the autotuner's caps and then
  evaluates exactly like a plan made with that cap.
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm
from oracle.medium import Medium
from oracle.dcim import ImageTable
from oracle.direct import direct_sum, cross_sum

from _helpers import need_gpu, make_plan, gpu_eval, to_dev

pytestmark = pytest.mark.gpu


def _batch(n=6, p=5, leaf_cap=40, seed=11):
    return W.batched_instances(n, p=p, seed=seed, n_min=1000, n_max=4000, leaf_cap=leaf_cap)


@pytest.mark.parametrize("precision,tol", [(tefmm.FP64, 1e-12), (tefmm.MIXED, 1e-6)], ids=["fp64", "mixed"])
def test_batched_equals_individual_evaluations(precision, tol):
    """FP64: same to rounding of the FP64 atomics; mixed: the FP32 tensor-core
    accumulators are summed in an order that varies between runs."""
    torch = need_gpu()
    ws = _batch()
    plans = [make_plan(w, precision=precision) for w in ws]
    inst = []
    for w in ws:
        x, y, z = [to_dev(torch, w.src[:, i]) for i in range(3)]
        q = to_dev(torch, np.asarray(w.q, dtype=np.complex128))
        inst.append((x, y, z, q, torch.empty(len(w.src), dtype=torch.complex128, device="cuda:0")))
    status = tefmm.eval_batched(plans, inst, n_workers=4)
    torch.cuda.synchronize()
    assert status == [0] * len(ws)
    for w, pl, (_, _, _, _, out) in zip(ws, plans, inst):
        ref = gpu_eval(make_plan(w, precision=precision), torch, w.src, w.q)
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), w.name


@pytest.mark.parametrize("precision", [tefmm.FP64, tefmm.MIXED], ids=["fp64", "mixed"])
def test_batch_instance_against_direct_sum(precision):
    torch = need_gpu()
    w = _batch(n=3, p=6, seed=12)[2]
    plan = make_plan(w, precision=precision)
    phi = gpu_eval(plan, torch, w.src, w.q)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images)
    sel = np.random.default_rng(0).choice(len(w.src), 40, replace=False)
    ref = direct_sum(med, img, w.src, w.q, w.src[sel])
    if len(w.k) > 1:
        ref = ref + cross_sum(med, w.zext, w.src, w.q, w.src[sel], n_images=w.n_images)
    err = np.linalg.norm(phi[sel] - ref) / np.linalg.norm(ref)
    print(f'{w.name} ({len(w.k)} layers, p=6) vs direct sum: {err:.2e}')
    assert err < 5e-3, err


def test_autotuned_leaf_cap():
    torch = need_gpu()
    w = _batch(n=1, p=5, seed=13, leaf_cap=0)[0]
    plan = make_plan(w)
    a = gpu_eval(plan, torch, w.src, w.q)
    st = plan.stats()
    assert st["leaf_cap_used"] in (16, 32, 64, 128, 256) and st["ms_autotune"] > 0
    b = gpu_eval(make_plan(w, leaf_cap=st["leaf_cap_used"]), torch, w.src, w.q)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
