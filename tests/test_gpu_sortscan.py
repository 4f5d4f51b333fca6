"""The library's own radix sort and prefix sums (csrc/sortscan.cu) on the GPU,
through their test hooks, against numpy: the sort against a stable argsort
(keys with many duplicates, most digits equal in every key so that the sort
skips their passes, 10% of them the all-ones key, values = input positions,
so stability is checked exactly), the scans against cumulative sums; sizes
around the tile lengths (4096 keys, 2048 values) and empty input."""
import ctypes

import numpy as np
import pytest

from _helpers import need_gpu

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1902_05875_gb300 import tefmm
    return tefmm.load(build_if_needed=False)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else None


@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 4097, 1_000_003])
def test_sort_is_a_stable_argsort(n):
    torch = need_gpu()
    rng = np.random.default_rng(n + 7)
    # high and low bits both vary; few distinct keys, so runs of equal keys are long
    keys = (rng.integers(0, 64, n).astype(np.uint64) << np.uint64(58)) | \
        rng.integers(0, 8, n).astype(np.uint64) | (rng.integers(0, 4, n).astype(np.uint64) << np.uint64(29))
    # the M2L builder's "no item" key ~0 among them (it must sort last although
    # most digits of the other keys are equal)
    keys[rng.random(n) < 0.1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    vals = np.arange(n, dtype=np.int32)
    kin = torch.tensor(keys.view(np.int64), device="cuda")
    vin = torch.tensor(vals, device="cuda")
    kout = torch.empty_like(kin)
    vout = torch.empty_like(vin)
    r = _lib().tefmm_debug_sort_u64(_ptr(kin), _ptr(kout), _ptr(vin), _ptr(vout), n, None)
    assert r == 0, r
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kout.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vout.cpu().numpy(), vals[order])
    assert np.array_equal(kin.cpu().numpy().view(np.uint64), keys)      # input untouched
    # keys only
    kout2 = torch.empty_like(kin)
    assert _lib().tefmm_debug_sort_u64(_ptr(kin), _ptr(kout2), None, None, n, None) == 0
    assert np.array_equal(kout2.cpu().numpy().view(np.uint64), keys[order])


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 5_000_001])
@pytest.mark.parametrize("inclusive", [0, 1])
def test_scan_is_a_cumulative_sum(n, inclusive):
    torch = need_gpu()
    rng = np.random.default_rng(n)
    v = rng.integers(0, 300, n).astype(np.int32)
    din = torch.tensor(v, device="cuda")
    dout = torch.empty_like(din)
    assert _lib().tefmm_debug_scan_i32(_ptr(din), _ptr(dout), n, inclusive, None) == 0
    c = np.cumsum(v, dtype=np.int64)
    ref = c if inclusive else np.concatenate([[0], c[:-1]]) if n else c
    assert np.array_equal(dout.cpu().numpy().astype(np.int64), ref)
