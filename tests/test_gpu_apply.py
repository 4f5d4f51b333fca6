"""Geometry once, charges many times: tefmm_set_points + tefmm_apply (``-m gpu``).

* apply(q) on a plan whose points were set equals a fresh tefmm_eval(points, q)
  (FP64 form to the rounding of its atomics, mixed form to its FP32
  accumulation order), for sources = targets and for distinct targets, with
  cross-layer components;
* a plan left by tefmm_eval applies new charges on those points, and the
  apply builds no trees or tables;
* apply before any points is an error, not a device call.
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm

from _helpers import need_gpu, make_plan, gpu_eval, to_dev

pytestmark = pytest.mark.gpu


def _w():
    return W.cross_layer_slabs(300, 5, 24, seed=7)


@pytest.mark.parametrize("precision,tol", [(tefmm.FP64, 1e-12), (tefmm.MIXED, 2e-6)], ids=["fp64", "mixed"])
def test_apply_equals_eval(precision, tol):
    torch = need_gpu()
    w = _w()
    rng = np.random.default_rng(3)
    q2 = rng.uniform(size=len(w.src)) + 1j * rng.uniform(size=len(w.src))
    plan = make_plan(w, precision=precision)
    x, y, z = [to_dev(torch, w.src[:, i]) for i in range(3)]
    plan.set_points(x, y, z)
    for q in (w.q, q2):
        got = plan.apply(to_dev(torch, np.asarray(q, dtype=np.complex128))).cpu().numpy()
        ref = gpu_eval(make_plan(w, precision=precision), torch, w.src, q)
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_apply_distinct_targets_and_after_eval():
    torch = need_gpu()
    w = _w()
    rng = np.random.default_rng(4)
    tgt = w.src[rng.choice(len(w.src), 250, replace=False)].copy()   # inside the layers' ranges
    tgt[:, :2] += rng.uniform(-1e-2, 1e-2, size=(250, 2))            # distinct from the sources
    plan = make_plan(w)
    x, y, z = [to_dev(torch, w.src[:, i]) for i in range(3)]
    tx, ty, tz = [to_dev(torch, tgt[:, i]) for i in range(3)]
    plan.set_points(x, y, z, tx, ty, tz)
    got = plan.apply(to_dev(torch, np.asarray(w.q, dtype=np.complex128))).cpu().numpy()
    ref = gpu_eval(make_plan(w), torch, w.src, w.q, tgt)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # a plan left by eval applies new charges on the eval's points
    plan2 = make_plan(w)
    gpu_eval(plan2, torch, w.src, w.q)
    q2 = np.conj(w.q)
    got2 = plan2.apply(to_dev(torch, np.asarray(q2, dtype=np.complex128))).cpu().numpy()
    ref2 = gpu_eval(make_plan(w), torch, w.src, q2)
    assert np.max(np.abs(got2 - ref2)) <= 1e-12 * np.max(np.abs(ref2))
    st = plan2.stats()
    assert st["ms_tables"] < 0.05 and st["ms_tree"] < 0.5, st


def test_apply_without_points_is_an_error():
    torch = need_gpu()
    w = _w()
    plan = make_plan(w)
    q = to_dev(torch, np.asarray(w.q, dtype=np.complex128))
    out = torch.empty_like(q)
    with pytest.raises(tefmm.TefmmError) as e:
        plan.apply(q, out=out)                    # the library itself refuses
    assert e.value.status == tefmm.ERR_INVALID_ARG
