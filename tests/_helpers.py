"""Shared helpers of the GPU parity tests (inputs and oracle plumbing only)."""
import numpy as np
import pytest

TAGS = {0: 'uu', 1: 'dd', 2: 'ud', 3: 'du'}


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def oracle_images(w, n_images=None):
    from oracle.medium import Medium
    from oracle.dcim import ImageTable
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images if n_images is None else n_images)
    return med, img


def push_images(plan, img):
    """Give the plan the oracle's images, term by term ((layer, tag) matched)."""
    per = []
    for t in plan.images():
        mine = [o for o in img.terms[t['layer']] if o['tag'] == TAGS[t['tag']]]
        assert len(mine) == 1
        o = mine[0]
        assert abs(o['zeta_min'] - t['zeta_min']) < 1e-14 and o['sz'] == t['sz'] and o['szp'] == t['szp']
        per.append((o['A'], o['Z']))
    plan.set_images(per)


def make_plan(w, **kw):
    from paper_1902_05875_gb300 import tefmm
    args = dict(p=w.p, leaf_cap=w.leaf_cap, n_images=w.n_images, zext=w.zext)
    args.update(kw)
    return tefmm.Plan(w.interfaces, w.k, **args)


def to_dev(torch, arr):
    return torch.tensor(np.ascontiguousarray(arr), device="cuda:0")


def gpu_eval(plan, torch, src, q, tgt=None):
    x, y, z = [to_dev(torch, src[:, i]) for i in range(3)]
    qq = to_dev(torch, np.asarray(q, dtype=np.complex128))
    if tgt is None:
        phi = plan.eval(x, y, z, qq)
    else:
        tx, ty, tz = [to_dev(torch, tgt[:, i]) for i in range(3)]
        phi = plan.eval(x, y, z, qq, tx, ty, tz)
    torch.cuda.synchronize()
    return phi.cpu().numpy()


def oracle_lists_csr(tr, lists_by_pair, n_nodes):
    """Combine the oracle's per-(target layer, source layer) lists into CSR."""
    V = {}
    N = {}
    for (lt, ls), (v, p) in lists_by_pair.items():
        for t, l in v.items():
            V.setdefault(t, []).extend(l)
        for t, l in p.items():
            N.setdefault(t, []).extend(l)

    def csr(D):
        ptr = np.zeros(n_nodes + 1, np.int64)
        src = []
        for t in range(n_nodes):
            lst = sorted(D.get(t, []))
            ptr[t + 1] = ptr[t] + len(lst)
            src.extend(lst)
        return ptr, np.array(src, dtype=np.int64)
    return csr(V), csr(N)


def push_cross_fits(plan, oracle_fmm):
    """Replace the plan's cross-layer fits by the oracle's: every key the plan
    holds (after an evaluation) is fitted by the oracle's TE-FMM object
    (``cross_image``, the oracle's own DCIM fit at the same clamped source
    z-centre) and imported with ``set_cross_images``.  Returns the keys."""
    keys = sorted(plan.cross_images())
    fits = {k: oracle_fmm.cross_image(*k) for k in keys}
    plan.set_cross_images(fits)
    return keys
