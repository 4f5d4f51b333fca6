"""Batched form as one launch, ``-m gpu``: the charge phases of several
independent media (two- and three-layer instances of the batched workload)
captured into one CUDA graph (``tefmm_batch_graph_create``) and replayed.

* the graph's potentials equal each instance's own ``tefmm_eval`` (mixed form;
  the FP32 output atomics may sum in another order: within 1e-6);
* the charges are rewritten in place and the graph replayed: it follows the
  new charges;
* ``tefmm_apply`` itself no longer waits for the host after the first call on
  a geometry, so a plain stream capture of it also works;
* no device error is flagged (``tefmm_plan_status``).
"""
import numpy as np
import pytest

from paper_1902_05875_gb300 import workloads as W
from paper_1902_05875_gb300 import tefmm

from _helpers import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def _instances(n=6):
    ws = W.batched_instances(n, n_min=1000, n_max=6000, leaf_cap=64)
    return ws


def test_batch_graph_matches_eval_and_follows_new_charges():
    torch = need_gpu()
    ws = _instances()
    plans, qs, phis, pts = [], [], [], []
    for w in ws:
        pl = tefmm.Plan(w.interfaces, w.k, p=w.p, leaf_cap=w.leaf_cap, n_images=w.n_images, zext=w.zext,
                        precision=tefmm.MIXED)
        x, y, z = [to_dev(torch, w.src[:, i]) for i in range(3)]
        pl.set_points(x, y, z)
        plans.append(pl)
        pts.append((x, y, z))
        qs.append(to_dev(torch, np.asarray(w.q, dtype=np.complex128)))
        phis.append(torch.zeros(len(w.src), dtype=torch.complex128, device="cuda"))
    g = tefmm.BatchGraph(plans, qs, phis)
    for rnd in range(2):
        if rnd == 1:                              # new charges, written in place
            rng = np.random.default_rng(11)
            for q in qs:
                q.copy_(torch.tensor(rng.uniform(size=q.numel()) + 1j * rng.uniform(size=q.numel()),
                                     device="cuda"))
        g.launch()
        torch.cuda.synchronize()
        for pl, (x, y, z), q, phi, w in zip(plans, pts, qs, phis, ws):
            pl.status()
            ref_plan = tefmm.Plan(w.interfaces, w.k, p=w.p, leaf_cap=w.leaf_cap, n_images=w.n_images,
                                  zext=w.zext, precision=tefmm.MIXED)
            ref = ref_plan.eval(x, y, z, q).cpu().numpy()
            got = phi.cpu().numpy()
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= 1e-6, (rnd, len(w.src), err)
    g.close()


def test_apply_can_be_captured_in_a_cuda_graph():
    torch = need_gpu()
    w = _instances(1)[0]
    pl = tefmm.Plan(w.interfaces, w.k, p=w.p, leaf_cap=w.leaf_cap, n_images=w.n_images, zext=w.zext,
                    precision=tefmm.MIXED)
    x, y, z = [to_dev(torch, w.src[:, i]) for i in range(3)]
    q = to_dev(torch, np.asarray(w.q, dtype=np.complex128))
    out = torch.zeros(len(w.src), dtype=torch.complex128, device="cuda")
    ref = pl.eval(x, y, z, q).clone()
    pl.apply(q, out=out)                          # first apply on the geometry: sizes the buffers
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
        pl.apply(q, out=out, stream=s)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    pl.status()
    err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
    assert err <= 1e-6, err
