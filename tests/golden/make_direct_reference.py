"""Writes the FP64 direct-sum reference of a bench workload at sampled targets:
the 2M three-slab workload at 1000 targets
(``direct_three_layer_slabs_n2M_1000.txt``) and the clustered 16M workload
at 20 targets (``direct_clustered_n16M_p8_20.txt``).

The values come from the oracle alone (``oracle.direct``: same-layer part by
the DCIM images of ``oracle.dcim``, cross-layer part by ``cross_sum``, every
layer pair with its images in the layer of the larger |k|); the workload is
the seeded input generator's.  The sample is n targets drawn without
replacement by numpy ``default_rng(1)``.  Each output line is ``index re im``
(17 significant digits).  Run from the repository root:

    python tests/golden/make_direct_reference.py [n_targets] [workload]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))


def workload(name):
    from paper_1902_05875_gb300 import workloads
    if name == "three_layer_slabs_n2M_p10":
        return workloads.cfg_mixed_2m(), os.path.join(HERE, "direct_three_layer_slabs_n2M_{n}.txt")
    if name == "clustered_n16M_p8":
        return (workloads.clustered(16_000_000, 8, 64, seed=0, n_images=16, name=name),
                os.path.join(HERE, "direct_clustered_n16M_p8_{n}.txt"))
    raise ValueError(name)


def main(n=1000, name="three_layer_slabs_n2M_p10"):
    from oracle.medium import Medium
    from oracle.dcim import ImageTable
    from oracle.direct import direct_sum, cross_sum
    w, OUT = workload(name)
    idx = np.random.default_rng(1).choice(len(w.src), n, replace=False)
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images)
    tgt = w.src[idx]
    t0 = time.perf_counter()
    phi = direct_sum(med, img, w.src, w.q, tgt)
    if med.n_layers > 1:
        phi = phi + cross_sum(med, w.zext, w.src, w.q, tgt, n_images=w.n_images)
    dt = time.perf_counter() - t0
    with open(OUT.format(n=n), "w") as f:
        f.write(f"# FP64 direct sum (oracle) of {w.name} at {n} targets, default_rng(1); "
                f"index re im; {dt:.0f} s on {os.cpu_count()} cores\n")
        for i, v in zip(idx, phi):
            f.write(f"{int(i)} {v.real:.17g} {v.imag:.17g}\n")
    print(OUT.format(n=n), f"{dt:.1f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1000,
         sys.argv[2] if len(sys.argv) > 2 else "three_layer_slabs_n2M_p10")
