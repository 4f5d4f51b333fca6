"""Near-field work items: a leaf whose near sources exceed one item (4096
sources) is split over several CTAs that add into its outputs.  Large leaves
(leaf cap 400) on clustered points give 68 such leaves with up to 20 000
near sources.  At targets in those leaves and at random ones, the FP64 form
equals the oracle TE-FMM (to 1e-11; a lost or doubled chunk would be off
by about 10%), and the mixed form stays within 1e-5 of it (FP32 pair sums
over up to 20 000 sources per target)."""
import numpy as np
import pytest

from _helpers import need_gpu, oracle_images, push_images, make_plan, gpu_eval

pytestmark = pytest.mark.gpu


def test_split_leaves_match_oracle():
    torch = need_gpu()
    from paper_1902_05875_gb300 import tefmm
    from paper_1902_05875_gb300 import workloads as W
    from oracle.tefmm import TEFMM
    w = W.clustered(20000, p=4, leaf_cap=400, seed=7, n_clusters=4, n_images=8)
    med, img = oracle_images(w)
    f = TEFMM(med, img, w.p, w.leaf_cap, n_images=w.n_images).setup(w.src, w.src)
    tr = f.tr
    near = f.lists[(1, 1)][1]
    big = [t for t, lst in near.items() if sum(int(tr.s1[s] - tr.s0[s]) for s in lst) > 4096]
    assert len(big) > 10
    idx = np.concatenate([np.concatenate([tr.tperm[tr.t0[t]:tr.t0[t] + 5] for t in big[:3]]),
                          np.random.default_rng(1).choice(len(w.src), 15, replace=False)])
    ref = f.evaluate(w.q, target_index=idx)
    for prec, tol in ((tefmm.FP64, 1e-11), (tefmm.MIXED, 1e-5)):
        plan = make_plan(w, precision=prec)
        push_images(plan, img)
        phi = gpu_eval(plan, torch, w.src, w.q)[idx]
        err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
        print(f"split leaves, precision {prec}: rel L2 vs oracle {err:.2e}")
        assert err <= tol, (prec, err)
