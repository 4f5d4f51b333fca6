"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Shared by the tests, the bench and the oracle-facing test code.  Every
generator draws positions first, then charges, with ``numpy.random.
default_rng(seed)``; particles of several layers are drawn layer by layer, top
to bottom.  The media and particle recipes follow the workloads of the paper's
Sec. 5 (uniform particles in slabs inside the layers of a two- or three-layer
medium) at the sizes this library is measured on.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    interfaces: list            # d_0 > d_1 > ... (len = n_layers - 1)
    k: list                     # complex wavenumber per layer
    zext: list                  # per layer (zlo, zhi) of the particle slab (DCIM zeta_min)
    src: np.ndarray             # (N, 3) float64
    q: np.ndarray               # (N,) complex128
    p: int
    leaf_cap: int
    n_images: int = 8
    tgt: np.ndarray = None      # None: targets are the sources
    extra: dict = field(default_factory=dict)

    @property
    def targets(self):
        return self.src if self.tgt is None else self.tgt


THREE_LAYER_D = [0.0, -1.2]
THREE_LAYER_K = [1.2, 1.5, 2.0]
THREE_LAYER_ZEXT = [(0.1, 1.1), (-1.1, -0.1), (-2.3, -1.3)]


def _charges(rng, n):
    re = rng.uniform(0.0, 1.0, n)
    im = rng.uniform(0.0, 1.0, n)
    return re + 1j * im


def middle_layer_uniform(n, p, leaf_cap, seed=0, n_images=8, name=None):
    """Three layers (interfaces 0, -1.2; k = 1.2, 1.5, 2.0); n uniform points in
    [-1,1]^2 x [-1.1,-0.1] (middle layer); charges re, im ~ U[0,1]."""
    rng = np.random.default_rng(seed)
    src = rng.uniform([-1.0, -1.0, -1.1], [1.0, 1.0, -0.1], size=(n, 3))
    q = _charges(rng, n)
    return Workload(name or f"middle_layer_uniform_n{n}_p{p}", THREE_LAYER_D, THREE_LAYER_K,
                    THREE_LAYER_ZEXT, src, q, p, leaf_cap, n_images)


def three_layer_slabs(n, p, leaf_cap, seed=0, n_images=8, k=(2.0, 3.0, 4.0 + 0.01j),
                      half_width=2.0, name=None):
    """Three layers (interfaces 0, -1.2), n points split equally over the three
    slabs [-w,w]^2 x {[0.1,1.1], [-1.1,-0.1], [-2.3,-1.3]}, top layer first."""
    rng = np.random.default_rng(seed)
    counts = [n // 3 + (1 if i < n % 3 else 0) for i in range(3)]
    parts = []
    for (zlo, zhi), c in zip(THREE_LAYER_ZEXT, counts):
        parts.append(rng.uniform([-half_width, -half_width, zlo], [half_width, half_width, zhi],
                                 size=(c, 3)))
    src = np.concatenate(parts, 0)
    q = _charges(rng, n)
    return Workload(name or f"three_layer_slabs_n{n}_p{p}", THREE_LAYER_D, list(k),
                    THREE_LAYER_ZEXT, src, q, p, leaf_cap, n_images)


CROSS_D = [0.0, -1.4]
CROSS_K = [2.0, 3.0, 4.0 + 0.01j]
CROSS_ZEXT = [(0.5, 0.9), (-1.0, -0.4), (-2.3, -1.9)]


def cross_layer_slabs(n_per_layer, p, leaf_cap, seed=0, n_images=16, k=None, name=None):
    """Three layers (interfaces 0, -1.4; k = 2, 3, 4 + 0.01i unless given),
    n_per_layer uniform points in each slab [-0.5,0.5]^2 x {[0.5,0.9],
    [-1.0,-0.4], [-2.3,-1.9]}, top layer first.  Small enough for the oracle's
    cross-layer direct sum (one DCIM fit per source point)."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform([-0.5, -0.5, a], [0.5, 0.5, b], size=(n_per_layer, 3)) for a, b in CROSS_ZEXT]
    src = np.concatenate(parts, 0)
    q = _charges(rng, len(src))
    kk = list(CROSS_K if k is None else k)
    return Workload(name or f"cross_layer_slabs_n{3 * n_per_layer}_p{p}", CROSS_D, kk, CROSS_ZEXT,
                    src, q, p, leaf_cap, n_images)


def cfg_small():
    """2000 points in the middle layer, p = 6, leaf cap 60, 8 images per term."""
    return middle_layer_uniform(2000, 6, 60, seed=0, n_images=8,
                                name="three_layer_middle_n2000_p6")


def cfg_fp64_200k():
    """200k points in the middle layer, p = 8, leaf cap 64."""
    return middle_layer_uniform(200_000, 8, 64, seed=0, n_images=8,
                                name="three_layer_middle_n200k_p8")


def cfg_mixed_2m():
    """2M points over three layers, k = (2, 3, 4 + 0.01i), p = 10, leaf cap 64,
    16 images per fit (the cross-layer fits need them for ~1e-7 accuracy)."""
    return three_layer_slabs(2_000_000, 10, 64, seed=0, n_images=16,
                             name="three_layer_slabs_n2M_p10")


def cfg_mixed_200k():
    """The 2M workload's geometry and medium at 200k points (a profiling case)."""
    return three_layer_slabs(200_000, 10, 64, seed=0, n_images=16,
                             name="three_layer_slabs_n200k_p10")


def batched_instances(n_inst, p=6, seed=2, n_min=1000, n_max=64000, n_images=8, leaf_cap=0):
    """Independent two- or three-layer instances (the batched workload): layer
    count 2 or 3 with equal probability; interface depths uniform in [-2, 0],
    sorted, a middle layer at least 0.3 thick (rejection); real k per layer
    uniform in [1, 4]; N log-uniform in [n_min, n_max], split equally over the
    layers, uniform in [-1,1]^2 x slabs 0.1 inside each layer (outer slabs 1.0
    thick); complex charges.  leaf_cap = 0 asks the library's autotuner."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        nl = int(rng.integers(2, 4))
        while True:
            d = np.sort(rng.uniform(-2.0, 0.0, nl - 1))[::-1]
            if nl == 2 or d[0] - d[1] >= 0.3:
                break
        k = list(rng.uniform(1.0, 4.0, nl))
        n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        zext = []
        for l in range(nl):
            top = d[l - 1] - 0.1 if l > 0 else d[0] + 1.1
            bot = d[l] + 0.1 if l < nl - 1 else d[-1] - 1.1
            zext.append((float(bot), float(top)))
        counts = [n // nl + (1 if l < n % nl else 0) for l in range(nl)]
        src = np.concatenate([rng.uniform([-1.0, -1.0, a], [1.0, 1.0, b], size=(c, 3))
                              for (a, b), c in zip(zext, counts)], 0)
        q = _charges(rng, len(src))
        out.append(Workload(f"batch{i}_L{nl}_n{n}", list(map(float, d)), k, zext, src, q, p, leaf_cap,
                            n_images))
    return out


def multi_layer_slabs(n_per_layer, n_layers, p, leaf_cap, seed=0, n_images=16, name=None):
    """n_layers layers (2..8) with interfaces at 0, -1, -2, ..., real
    wavenumbers 1.5, 2.0, 2.5, ... from the top; n_per_layer uniform points per
    layer in [-0.6,0.6]^2 x a slab 0.2 inside each interface (outer slabs 0.6
    thick), top layer first."""
    rng = np.random.default_rng(seed)
    d = [0.0] + [-float(m) for m in range(1, n_layers - 1)]
    k = [1.5 + 0.5 * l for l in range(n_layers)]
    zext = []
    for l in range(n_layers):
        top = d[l - 1] - 0.2 if l > 0 else d[0] + 0.8
        bot = d[l] + 0.2 if l < n_layers - 1 else d[-1] - 0.8
        zext.append((float(bot), float(top)))
    src = np.concatenate([rng.uniform([-0.6, -0.6, a], [0.6, 0.6, b], size=(n_per_layer, 3))
                          for (a, b) in zext], 0)
    q = _charges(rng, len(src))
    return Workload(name or f"multi_layer{n_layers}_n{len(src)}_p{p}", d, k, zext, src, q, p, leaf_cap,
                    n_images)


# Example 2 of the paper's Sec. 5: irregular domains
# r(theta) = 0.5 - a + (a / 8) (35 cos^4 theta - 30 cos^2 theta + 3)
# shifted to centres (0, 0, 1), (0, 0, -1) (two layers, interface z = 0) and
# (0, 0, -3) (three layers, interfaces 0, -2), a = 0.1, 0.15, 0.05.
IRREGULAR_CENTRES = [1.0, -1.0, -3.0]
IRREGULAR_A = [0.1, 0.15, 0.05]


def irregular_domains(n, n_layers=3, p=6, leaf_cap=64, seed=0, n_images=16, k=(0.8, 1.5, 2.0), name=None):
    """Particles uniform inside the irregular domains of Example 2 (rejection
    from the cube of side 1 around each domain centre), n split equally over
    the n_layers (2 or 3) domains, top layer first.  The paper does not state
    the wavenumbers of Sec. 5; k defaults to those of its Sec. 3.3 example."""
    assert n_layers in (2, 3)
    rng = np.random.default_rng(seed)
    d = [0.0] if n_layers == 2 else [0.0, -2.0]
    counts = [n // n_layers + (1 if l < n % n_layers else 0) for l in range(n_layers)]
    parts, zext = [], []
    for l in range(n_layers):
        c, a, need = IRREGULAR_CENTRES[l], IRREGULAR_A[l], counts[l]
        got = []
        while need > 0:
            x = rng.uniform([-0.5, -0.5, c - 0.5], [0.5, 0.5, c + 0.5], size=(max(2 * need, 64), 3))
            rel = x - np.array([0.0, 0.0, c])
            r = np.sqrt(np.sum(rel * rel, 1))
            ct = np.divide(rel[:, 2], r, out=np.zeros_like(r), where=r > 0)
            keep = x[r < 0.5 - a + a / 8.0 * (35 * ct ** 4 - 30 * ct ** 2 + 3)][:need]
            got.append(keep)
            need -= len(keep)
        parts.append(np.concatenate(got, 0))
        zext.append((c - 0.5, c + 0.5))
    src = np.concatenate(parts, 0)
    q = _charges(rng, len(src))
    return Workload(name or f"irregular_domains{n_layers}_n{n}_p{p}", d, list(k)[:n_layers], zext, src, q,
                    p, leaf_cap, n_images)


def clustered(n, p=8, leaf_cap=64, seed=0, n_images=16, n_clusters=32, sigma=0.05, name=None):
    """n points from n_clusters Gaussian clusters (standard deviation sigma,
    centres uniform in the middle slab [-1,1]^2 x [-1.1,-0.1] of the
    three-layer medium of the small workload, points clipped to the slab):
    an adaptive octree many levels deep in the clusters and shallow between them."""
    rng = np.random.default_rng(seed)
    lo, hi = np.array([-1.0, -1.0, -1.1]), np.array([1.0, 1.0, -0.1])
    centres = rng.uniform(lo, hi, size=(n_clusters, 3))
    which = rng.integers(0, n_clusters, n)
    src = np.clip(centres[which] + sigma * rng.standard_normal((n, 3)), lo, hi)
    q = _charges(rng, n)
    return Workload(name or f"clustered_n{n}_p{p}", THREE_LAYER_D, THREE_LAYER_K, THREE_LAYER_ZEXT, src, q, p,
                    leaf_cap, n_images)
