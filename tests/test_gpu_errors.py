"""Error paths on the GPU, ``-m gpu``, made on the host (no device fault):

* an injected device-allocation failure (``tefmm_debug_inject``) surfaces as
  TEFMM_ERR_OOM wherever in the evaluation it falls, and the next evaluation
  of the same plan succeeds with the normal result;
* an injected DCIM fit failure surfaces as TEFMM_ERR_FIT_FAILED from plan
  creation (same-layer fits) and from an evaluation (cross-layer fits), and
  the plan recovers once the injection is cleared;
* a bounded device wait that nothing completes runs out after its limit and
  is reported as TEFMM_ERR_TIMEOUT, and the context stays usable.
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm

from _helpers import need_gpu, make_plan, gpu_eval

pytestmark = pytest.mark.gpu


def _status(fn):
    try:
        fn()
    except tefmm.TefmmError as e:
        return e.status
    return tefmm.OK


def test_injected_allocation_failure_reports_oom_and_recovers():
    torch = need_gpu()
    w = W.cross_layer_slabs(80, 4, 8, seed=3)
    ref = gpu_eval(make_plan(w), torch, w.src, w.q)
    seen = set()
    try:
        for n in (1, 5, 12, 25, 40, 60):
            plan = make_plan(w)
            tefmm.debug_inject(tefmm.INJECT_ALLOC, n)
            st = _status(lambda: gpu_eval(plan, torch, w.src, w.q))
            tefmm.debug_inject(0)
            seen.add(st)
            assert st in (tefmm.OK, tefmm.ERR_OOM), (n, st)
            phi = gpu_eval(plan, torch, w.src, w.q)        # the same plan, no injection
            assert np.max(np.abs(phi - ref)) <= 1e-12 * np.max(np.abs(ref)), n
    finally:
        tefmm.debug_inject(0)
    assert tefmm.ERR_OOM in seen


def test_injected_fit_failure_reports_fit_failed_and_recovers():
    torch = need_gpu()
    w = W.cross_layer_slabs(60, 4, 8, seed=4)
    try:
        tefmm.debug_inject(tefmm.INJECT_FIT, 1)
        assert _status(lambda: make_plan(w)) == tefmm.ERR_FIT_FAILED      # same-layer fits
        tefmm.debug_inject(0)
        plan = make_plan(w)
        tefmm.debug_inject(tefmm.INJECT_FIT, 1)
        assert _status(lambda: gpu_eval(plan, torch, w.src, w.q)) == tefmm.ERR_FIT_FAILED   # cross-layer fits
        tefmm.debug_inject(0)
        phi = gpu_eval(plan, torch, w.src, w.q)
        ref = gpu_eval(make_plan(w), torch, w.src, w.q)
        assert np.max(np.abs(phi - ref)) <= 1e-12 * np.max(np.abs(ref))
    finally:
        tefmm.debug_inject(0)


def test_bounded_wait_runs_out_and_context_stays_usable():
    torch = need_gpu()
    w = W.middle_layer_uniform(400, 4, 32, seed=2)
    plan = make_plan(w)
    lib = tefmm.load()
    st = lib.tefmm_debug_wait_probe(plan.h, 20, tefmm._stream_handle(None))
    assert st == tefmm.ERR_TIMEOUT, st
    phi = gpu_eval(plan, torch, w.src, w.q)                 # the next evaluation runs normally
    assert np.all(np.isfinite(phi))
    plan.status()
