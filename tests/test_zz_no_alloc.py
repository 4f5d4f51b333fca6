"""The allocation-free fit entry point, through the C-ABI (``-m gpu``).

``tefmm_fit_images_noalloc`` serves callers that cannot allocate device memory
when they need a medium's images (inside a stream capture, under a pre-sized
pool allocator, on latency-critical paths).  It must return the same images as
the allocating path (``tefmm_plan_create`` + ``tefmm_plan_get_images``), on
two calls in a row (its fixed scratch array is reused by every call).
This file is collected last so that a failure here stops a ``-x`` run only
after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_1902_05875_gb300 import tefmm, workloads as W

from _helpers import need_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _noalloc(lib, w, opt):
    nL = len(w.k)
    k = np.asarray(w.k, dtype=complex)
    d = np.ascontiguousarray(np.asarray(w.interfaces, dtype=np.float64))
    kre = np.ascontiguousarray(k.real)
    kim = np.ascontiguousarray(k.imag)
    nt = ctypes.c_int(0)
    lay = np.zeros(4 * nL, np.int32)
    tag = np.zeros(4 * nL, np.int32)
    cnt = np.zeros(4 * nL, np.int32)
    A = np.zeros(2 * 32 * 4 * nL, np.float64)
    Z = np.zeros(2 * 32 * 4 * nL, np.float64)
    st = lib.tefmm_fit_images_noalloc(nL, tefmm._dptr(d), tefmm._dptr(kre), tefmm._dptr(kim),
                                      ctypes.byref(opt), ctypes.c_void_p(0), ctypes.byref(nt),
                                      tefmm._iptr(lay), tefmm._iptr(tag), tefmm._iptr(cnt),
                                      tefmm._dptr(A), tefmm._dptr(Z))
    assert st == 0, lib.tefmm_status_string(st)
    out = []
    for t in range(nt.value):
        j = np.arange(cnt[t])
        a = A[2 * (32 * t + j)] + 1j * A[2 * (32 * t + j) + 1]
        z = Z[2 * (32 * t + j)] + 1j * Z[2 * (32 * t + j) + 1]
        out.append((int(lay[t]), int(tag[t]), a, z))
    return out


@pytest.mark.parametrize("n_images", [8, 16])
def test_noalloc_fit_matches_plan_fit_twice(n_images):
    need_gpu()
    w = W.cfg_small()
    lib = tefmm.load()
    plan = tefmm.Plan(w.interfaces, w.k, p=w.p, leaf_cap=w.leaf_cap, n_images=n_images, zext=w.zext)
    ref = plan.images()
    opt = tefmm.Options()
    lib.tefmm_default_options(ctypes.byref(opt))
    opt.p, opt.leaf_cap, opt.n_images = w.p, w.leaf_cap, n_images
    for l, (a, b) in enumerate(w.zext):
        opt.zext[2 * l] = a
        opt.zext[2 * l + 1] = b
    for _ in range(2):
        got = _noalloc(lib, w, opt)
        assert len(got) == len(ref)
        for (lay, tag, a, z), r in zip(got, ref):
            assert (lay, tag) == (r['layer'], r['tag'])
            assert len(a) == len(r['A']) > 0
            assert np.max(np.abs(a - r['A'])) <= TOL * np.max(np.abs(r['A']))
            assert np.max(np.abs(z - r['Z'])) <= TOL * np.max(np.abs(r['Z']))


def test_noalloc_rejects_oversized_request():
    need_gpu()
    w = W.cfg_small()
    lib = tefmm.load()
    opt = tefmm.Options()
    lib.tefmm_default_options(ctypes.byref(opt))
    opt.n_samples = 200          # beyond the fixed per-fit sample buffers
    k = np.asarray(w.k, dtype=complex)
    d = np.ascontiguousarray(np.asarray(w.interfaces, dtype=np.float64))
    kre, kim = np.ascontiguousarray(k.real), np.ascontiguousarray(k.imag)
    nt = ctypes.c_int(0)
    cnt = np.zeros(12, np.int32)
    A = np.zeros(2 * 32 * 12)
    Z = np.zeros(2 * 32 * 12)
    st = lib.tefmm_fit_images_noalloc(3, tefmm._dptr(d), tefmm._dptr(kre), tefmm._dptr(kim),
                                      ctypes.byref(opt), ctypes.c_void_p(0), ctypes.byref(nt), None,
                                      None, tefmm._iptr(cnt), tefmm._dptr(A), tefmm._dptr(Z))
    assert st == -1
