"""Mixed-precision form (``precision=MIXED``) against the FP64 oracle (``-m gpu``).

The mixed form evaluates the near-field pairs in FP32 (FP64 per-target
accumulation, the images' constant part in FP64) and the M2L contractions on
the tensor cores in 3xTF32 with FP32 accumulation (highest orders first);
tables, P2M/M2M/L2L and L2P stay in FP64.  Measured rounding of the mixed form
on GB300: 8e-8 (2000 points, p = 6) and 1.8e-7 (3001 points, p = 5) against
the FP64 form; at the 20k sampled targets 2.5e-7 against the direct sum (FP64
form 1.8e-7), almost all of it from the FP32 accumulation of the M2L
contractions.
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm
from oracle.direct import direct_sum

from _helpers import need_gpu, oracle_images, push_images, make_plan, gpu_eval

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w", [W.cfg_small(), W.middle_layer_uniform(3001, 5, 17, seed=4)],
                         ids=lambda w: w.name)
def test_mixed_close_to_fp64_form(w):
    torch = need_gpu()
    med, img = oracle_images(w)
    p64 = make_plan(w)
    push_images(p64, img)
    pmx = make_plan(w, precision=tefmm.MIXED)
    push_images(pmx, img)
    a = gpu_eval(p64, torch, w.src, w.q)
    b = gpu_eval(pmx, torch, w.src, w.q)
    err = np.linalg.norm(a - b) / np.linalg.norm(a)
    print(f'mixed vs fp64 form ({w.name}): {err:.3e}')
    assert err < 5e-7, err


def test_mixed_vs_direct_sum_at_sampled_targets():
    torch = need_gpu()
    w = W.middle_layer_uniform(20000, 8, 64, seed=7)
    med, img = oracle_images(w)
    pmx = make_plan(w, precision=tefmm.MIXED)
    push_images(pmx, img)
    p64 = make_plan(w)
    push_images(p64, img)
    b = gpu_eval(pmx, torch, w.src, w.q)
    a = gpu_eval(p64, torch, w.src, w.q)
    sel = np.random.default_rng(0).choice(len(w.src), 300, replace=False)
    d = direct_sum(med, img, w.src, w.q, w.src[sel])
    e64 = np.linalg.norm(a[sel] - d) / np.linalg.norm(d)
    emx = np.linalg.norm(b[sel] - d) / np.linalg.norm(d)
    print(f'vs direct sum: mixed {emx:.3e}  fp64 {e64:.3e}')
    # split the mixed-form error: L2P of the local differences (tensor-core M2L)
    # against the rest (FP32 near field)
    g = pmx.export_tree()
    _, bmx = pmx.export_expansions()
    _, b64 = p64.export_expansions()
    from oracle.derivs import multi_indices
    mi = multi_indices(w.p)
    lo = w.src.min(axis=0)
    side = float(np.max(w.src.max(axis=0) - lo))
    inv = np.empty_like(g["perm_t"])
    inv[g["perm_t"]] = np.arange(len(inv))
    leaf = np.full(len(w.src), -1)
    for n in range(g["n_nodes"]):
        if g["t1"][n] > g["t0"][n]:
            leaf[g["t0"][n]:g["t1"][n]] = n      # deepest node wins (level-major order)
    dm2l = np.zeros(len(sel), complex)
    for i, t in enumerate(sel):
        n = leaf[inv[t]]
        hh = side / 2 ** g["level"][n]
        c = lo + (np.array([g["ix"][n], g["iy"][n], g["iz"][n]]) + 0.5) * hh
        d = w.src[t] - c
        mono = d[0] ** mi[:, 0] * d[1] ** mi[:, 1] * d[2] ** mi[:, 2]
        dm2l[i] = mono @ (bmx[n] - b64[n])
    e_m2l = np.linalg.norm(dm2l) / np.linalg.norm(a[sel])
    e_tot = np.linalg.norm(b[sel] - a[sel]) / np.linalg.norm(a[sel])
    e_near = np.linalg.norm(b[sel] - a[sel] - dm2l) / np.linalg.norm(a[sel])
    print(f'mixed - fp64 at samples: total {e_tot:.3e}, from M2L {e_m2l:.3e}, near field {e_near:.3e}')
    assert emx < e64 + 3e-7, (emx, e64)


@pytest.mark.parametrize("w", [W.cfg_small(), W.middle_layer_uniform(20000, 8, 64, seed=7)],
                         ids=lambda w: w.name)
def test_tensor_core_m2l_locals(w):
    """Locals after the tensor-core M2L (3xTF32, scaled) against the FP64 form's."""
    torch = need_gpu()
    med, img = oracle_images(w)
    p64 = make_plan(w)
    push_images(p64, img)
    pmx = make_plan(w, precision=tefmm.MIXED)
    push_images(pmx, img)
    gpu_eval(p64, torch, w.src, w.q)
    gpu_eval(pmx, torch, w.src, w.q)
    a64, b64 = p64.export_expansions()
    amx, bmx = pmx.export_expansions()
    assert np.array_equal(a64, amx)          # the upward pass is FP64 in both forms
    worst = 0.0
    for n in range(b64.shape[0]):
        s = np.max(np.abs(b64[n]))
        if s > 0:
            worst = max(worst, np.max(np.abs(bmx[n] - b64[n])) / s)
    print(f'tensor-core locals ({w.name}): worst relative {worst:.3e}')
    assert worst < 2e-5, worst
    assert pmx.stats()["n_v_pairs"] == p64.stats()["n_v_pairs"]
