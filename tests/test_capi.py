"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/tefmm.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tefmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tefmm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1902_05875_gb300 import _build, tefmm
    lib = ctypes.CDLL(_build.build())
    names = _declared()
    assert "tefmm_eval" in names and "tefmm_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(tefmm.EXPORTED) | {"tefmm_plan_image_counts"}


def test_status_strings_without_gpu():
    from paper_1902_05875_gb300 import tefmm
    lib = tefmm.load()
    assert lib.tefmm_status_string(0) == b"ok"
    assert b"interface" in lib.tefmm_status_string(-2)


def test_default_options_without_gpu():
    from paper_1902_05875_gb300 import tefmm
    lib = tefmm.load()
    o = tefmm.Options()
    assert lib.tefmm_default_options(ctypes.byref(o)) == 0
    assert (o.p, o.leaf_cap, o.n_images, o.n_samples) == (6, 64, 8, 101)
    assert lib.tefmm_default_options(None) == -1


def test_built_for_sm103a():
    from paper_1902_05875_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_apply_binding_checks_arguments_without_gpu():
    """set_points / apply refuse host tensors before calling the library."""
    torch = pytest.importorskip("torch")
    from paper_1902_05875_gb300 import tefmm
    plan = object.__new__(tefmm.Plan)          # argument checks only: no device plan
    x = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        tefmm.Plan.set_points(plan, x, x, x)
    with pytest.raises(ValueError):
        tefmm.Plan.apply(plan, torch.zeros(4, dtype=torch.complex128))


class _FakeCuda:
    """Stands in for a contiguous CUDA tensor (dtype, length) so that the
    binding's argument checks run on a machine without a GPU."""

    def __init__(self, dtype, n):
        self.dtype, self.n, self.is_cuda, self.device = dtype, n, True, "cuda:0"

    def is_contiguous(self):
        return True

    def numel(self):
        return self.n

    def data_ptr(self):
        raise AssertionError("the library must not be called")


def test_eval_and_apply_refuse_wrong_lengths_without_gpu():
    """eval() and apply() check that q has one entry per source and out one
    per target before the library is called (a short array would be read or
    written past its end on the device)."""
    torch = pytest.importorskip("torch")
    from paper_1902_05875_gb300 import tefmm
    plan = object.__new__(tefmm.Plan)
    f64 = lambda n: _FakeCuda(torch.float64, n)
    c128 = lambda n: _FakeCuda(torch.complex128, n)
    with pytest.raises(ValueError):
        tefmm.Plan.eval(plan, f64(5), f64(5), f64(5), c128(4))                     # short q
    with pytest.raises(ValueError):
        tefmm.Plan.eval(plan, f64(5), f64(5), f64(5), c128(5), out=c128(4))        # short out
    with pytest.raises(ValueError):
        tefmm.Plan.eval(plan, f64(5), f64(5), f64(5), c128(5), f64(3), f64(3), f64(2))
    with pytest.raises(RuntimeError):
        tefmm.Plan.apply(plan, c128(5))                                            # no points yet
    plan._n_sources, plan._n_targets = 5, 3
    with pytest.raises(ValueError):
        tefmm.Plan.apply(plan, c128(4))                                            # short q
    with pytest.raises(ValueError):
        tefmm.Plan.apply(plan, c128(5), out=c128(5))                               # out of the wrong length


def test_fault_injection_hook_arguments_without_gpu():
    """The error-path test hook takes its arguments and clears without a GPU."""
    from paper_1902_05875_gb300 import tefmm
    lib = tefmm.load()
    assert lib.tefmm_debug_inject(0, 0) == 0
    assert lib.tefmm_debug_inject(tefmm.INJECT_ALLOC, 0) == tefmm.ERR_INVALID_ARG
    assert lib.tefmm_debug_inject(7, 1) == tefmm.ERR_INVALID_ARG
    assert lib.tefmm_debug_inject(tefmm.INJECT_FIT, 3) == 0
    assert lib.tefmm_debug_inject(0, 0) == 0
    assert lib.tefmm_status_string(tefmm.ERR_TIMEOUT) == b"a bounded device wait ran out"
