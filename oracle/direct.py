"""Python side of the C direct-sum oracle (``oracle/direct.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  ``build()`` compiles the C
file with gcc (-O2, OpenMP, no FMA contraction) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_direct.so")
_lib = None


def build(force=False):
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "direct.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared",
                               "-fPIC", "-o", _SO, src, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _lib.oracle_direct_sum.restype = None
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def direct_sum(med, images, src, q, tgt, include_free=True, include_reaction=True):
    """Phi at the targets.  src/tgt: (n, 3) float arrays; q complex (n,).

    ``images``: an ``oracle.dcim.ImageTable`` (same-layer terms) or None.
    """
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.float64)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    qi = np.ascontiguousarray(np.stack([np.real(q), np.imag(q)], -1).reshape(-1), dtype=np.float64)
    slay = np.ascontiguousarray(med.layer_of(src[:, 2]), dtype=np.int32)
    tlay = np.ascontiguousarray(med.layer_of(tgt[:, 2]), dtype=np.int32)
    if np.any(slay < 0) or np.any(tlay < 0):
        raise ValueError("point on an interface")
    rows = images.flat() if (images is not None and include_reaction) else []
    nimg = len(rows)
    f64 = lambda v: np.ascontiguousarray(np.array(v, dtype=np.float64).reshape(-1))
    il = np.ascontiguousarray(np.array([r[0] for r in rows], dtype=np.int32).reshape(-1))
    A = np.array([r[2] for r in rows], dtype=complex).reshape(-1)
    Z = np.array([r[3] for r in rows], dtype=complex).reshape(-1)
    arrs = [f64([r[4] for r in rows]), f64([r[5] for r in rows]), f64([r[6] for r in rows]),
            f64([r[7] for r in rows]), f64(A.real), f64(A.imag), f64(Z.real), f64(Z.imag)]
    kre = f64(med.k.real)
    kim = f64(med.k.imag)
    phi = np.zeros(2 * tgt.shape[0], dtype=np.float64)
    sx, sy, sz = [np.ascontiguousarray(src[:, i]) for i in range(3)]
    tx, ty, tz = [np.ascontiguousarray(tgt[:, i]) for i in range(3)]
    D = ctypes.POINTER(ctypes.c_double)
    Ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_direct_sum(
        ctypes.c_int64(src.shape[0]), _p(sx, ctypes.c_double), _p(sy, ctypes.c_double),
        _p(sz, ctypes.c_double), _p(qi, ctypes.c_double), _p(slay, ctypes.c_int),
        ctypes.c_int64(tgt.shape[0]), _p(tx, ctypes.c_double), _p(ty, ctypes.c_double),
        _p(tz, ctypes.c_double), _p(tlay, ctypes.c_int), _p(kre, ctypes.c_double),
        _p(kim, ctypes.c_double), ctypes.c_int(nimg), _p(il, ctypes.c_int),
        *[_p(a, ctypes.c_double) for a in arrs],
        ctypes.c_int(1 if include_free else 0), ctypes.c_int(1 if include_reaction else 0),
        _p(phi, ctypes.c_double))
    return phi[0::2] + 1j * phi[1::2]


def images_in_source_layer(med, l, lp):
    """A cross-layer component (target layer l, source layer l') has its DCIM
    images in the layer of the larger |k|: those fits match Sommerfeld
    quadrature to about 1e-8, fits in the smaller-|k| layer only to 1e-6 .. 4e-4
    (branch points of the spectral function near the sampling paths).  True
    when that layer is the source layer (reciprocity form)."""
    return abs(complex(med.k[lp])) > abs(complex(med.k[l]))


def cross_sum(med, zext, src, q, tgt, n_images=16, zbin=0.02, K=6, **fit_kw):
    """Cross-layer part of Phi at the targets, every layer pair with its images
    in the layer of the larger |k| (``images_in_source_layer``): by reciprocity
    with one fit per target where that is the source layer, else with the
    images in the target layer and fits per narrow source z'-bin (width at most
    ``zbin``, z'-Taylor order ``K``; ``cross_sum_binned``)."""
    out = cross_sum_by_reciprocity(med, zext, src, q, tgt, n_images,
                                   pairs=lambda l, lp: images_in_source_layer(med, l, lp), **fit_kw)
    return out + cross_sum_binned(med, zext, src, q, tgt, n_images, zbin, K,
                                  pairs=lambda l, lp: not images_in_source_layer(med, l, lp), **fit_kw)


def cross_sum_binned(med, zext, src, q, tgt, n_images=16, zbin=0.02, K=6, pairs=None, **fit_kw):
    """Cross-layer part of Phi with the images in the target layer: the sources
    of layer l' are grouped in equal z'-bins of width <= zbin over the layer's
    particle slab, each bin centre zc gets the fits of Theta^{k3'}, k3' = 0..K
    (Sec. 3.3, ``oracle.cross.fit_cross``), and a source at zc + delta adds
    sum_{k3'} delta^{k3'} (image sum of fit k3') (``oracle_cross_sum_binned``).
    pairs(l, l') selects the layer pairs (default: all)."""
    from .cross import directions, fit_cross, W_min
    lib = _load()
    lib.oracle_cross_sum_binned.restype = None
    src = np.ascontiguousarray(src, dtype=np.float64)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    qi = np.ascontiguousarray(np.stack([np.real(q), np.imag(q)], -1).reshape(-1), dtype=np.float64)
    slay = np.ascontiguousarray(med.layer_of(src[:, 2]), dtype=np.int32)
    tlay = np.ascontiguousarray(med.layer_of(tgt[:, 2]), dtype=np.int32)
    if np.any(slay < 0) or np.any(tlay < 0):
        raise ValueError("point on an interface")
    nl = med.n_layers
    use = np.zeros((nl, nl), dtype=np.int32)
    for l in set(int(v) for v in tlay):
        for lp in set(int(v) for v in slay):
            if lp != l and (pairs is None or pairs(l, lp)):
                use[l, lp] = 1
    # bins: per source layer, equal widths over its particle slab; global numbering
    nb = [max(1, int(math.ceil((zext[l][1] - zext[l][0]) / zbin - 1e-9))) for l in range(nl)]
    b0 = np.concatenate([[0], np.cumsum(nb)]).astype(np.int64)
    nbin = int(b0[-1])
    sbin = np.zeros(len(src), dtype=np.int32)
    sdelta = np.zeros(len(src), dtype=np.float64)
    zc_of = np.zeros(nbin)
    for l in range(nl):
        w = (zext[l][1] - zext[l][0]) / nb[l]
        zc_of[b0[l]:b0[l + 1]] = zext[l][0] + (np.arange(nb[l]) + 0.5) * w
        m = slay == l
        b = np.clip(np.floor((src[m, 2] - zext[l][0]) / w).astype(np.int64), 0, nb[l] - 1)
        sbin[m] = (b0[l] + b).astype(np.int32)
        sdelta[m] = src[m, 2] - zc_of[b0[l] + b]
    counts = np.zeros(nl * nbin * 2 * (K + 1), dtype=np.int64)
    A_all, Z_all = [], []
    chunks = {}
    for l in range(nl):
        for lp in range(nl):
            if not use[l, lp]:
                continue
            for part in directions(med, l):
                wm = W_min(med, l, part, zext)
                pi = 0 if part == 'up' else 1
                for b in range(b0[lp], b0[lp + 1]):
                    for k3p in range(K + 1):
                        A, Z, _ = fit_cross(med, l, lp, part, float(zc_of[b]), k3p, wm, n_images, **fit_kw)
                        f = ((l * nbin + b) * 2 + pi) * (K + 1) + k3p
                        chunks[f] = (np.asarray(A, complex), np.asarray(Z, complex))
                        counts[f] = len(A)
    img_first = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    A_all = np.zeros(int(img_first[-1]), dtype=complex)
    Z_all = np.zeros(int(img_first[-1]), dtype=complex)
    for f, (A, Z) in chunks.items():
        A_all[img_first[f]:img_first[f + 1]] = A
        Z_all[img_first[f]:img_first[f + 1]] = Z
    wmin = np.zeros(2 * nl)
    for l in range(nl):
        for part in directions(med, l):
            wmin[2 * l + (0 if part == 'up' else 1)] = W_min(med, l, part, zext)
    f64 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
    are, aim, zre, zim = f64(A_all.real), f64(A_all.imag), f64(Z_all.real), f64(Z_all.imag)
    kre, kim = f64(med.k.real), f64(med.k.imag)
    dd = f64(np.concatenate([med.d, [0.0]]))
    wmin = f64(wmin)
    use_f = np.ascontiguousarray(use.reshape(-1))
    phi = np.zeros(2 * tgt.shape[0], dtype=np.float64)
    sx, sy = [np.ascontiguousarray(src[:, i]) for i in range(2)]
    tx, ty, tz = [np.ascontiguousarray(tgt[:, i]) for i in range(3)]
    D, L, Ci = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    lib.oracle_cross_sum_binned(
        ctypes.c_int64(src.shape[0]), _p(sx, D), _p(sy, D), _p(qi, D), _p(slay, Ci), _p(sbin, Ci),
        _p(sdelta, D), ctypes.c_int64(tgt.shape[0]), _p(tx, D), _p(ty, D), _p(tz, D), _p(tlay, Ci),
        ctypes.c_int(nl), _p(use_f, Ci), ctypes.c_int(nbin), ctypes.c_int(K), _p(img_first, L),
        _p(are, D), _p(aim, D), _p(zre, D), _p(zim, D), _p(wmin, D), _p(kre, D), _p(kim, D), _p(dd, D),
        _p(phi, D))
    return phi[0::2] + 1j * phi[1::2]


def cross_sum_by_reciprocity(med, zext, src, q, tgt, n_images=16, pairs=None, **fit_kw):
    """Cross-layer part of Phi at the targets, one DCIM fit per target
    (``oracle_cross_sum`` in ``direct.c``), its images in the source layer:
    the plain definition for large source counts, where one fit per source
    point is out of reach.  pairs(l, l') selects the (target layer, source
    layer) pairs (default: all)."""
    from .cross import directions, fit_cross, W_min
    lib = _load()
    lib.oracle_cross_sum.restype = None
    src = np.ascontiguousarray(src, dtype=np.float64)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    qi = np.ascontiguousarray(np.stack([np.real(q), np.imag(q)], -1).reshape(-1), dtype=np.float64)
    slay = np.ascontiguousarray(med.layer_of(src[:, 2]), dtype=np.int32)
    tlay = med.layer_of(tgt[:, 2])
    if np.any(slay < 0) or np.any(tlay < 0):
        raise ValueError("point on an interface")
    present = set(int(v) for v in np.unique(slay))
    fit_first = [0]
    fl, fp, fw, fre, fim, img_first, A_all, Z_all = [], [], [], [], [], [0], [], []
    for i in range(len(tgt)):
        l = int(tlay[i])
        for lp in sorted(present):
            if lp == l or (pairs is not None and not pairs(l, lp)):
                continue
            for part in directions(med, lp):
                wmin = W_min(med, lp, part, zext)
                A, Z, _ = fit_cross(med, lp, l, part, float(tgt[i, 2]), 0, wmin, n_images, **fit_kw)
                fac = (med.k[lp] / med.k[l]) ** 2
                fl.append(lp)
                fp.append(0 if part == 'up' else 1)
                fw.append(wmin)
                fre.append(fac.real)
                fim.append(fac.imag)
                A_all.extend(A)
                Z_all.extend(Z)
                img_first.append(len(A_all))
        fit_first.append(len(fl))
    i64 = lambda v: np.ascontiguousarray(np.array(v, dtype=np.int64))
    i32 = lambda v: np.ascontiguousarray(np.array(v, dtype=np.int32))
    f64 = lambda v: np.ascontiguousarray(np.array(v, dtype=np.float64).reshape(-1))
    A_all = np.array(A_all, dtype=complex)
    Z_all = np.array(Z_all, dtype=complex)
    arrs = dict(ff=i64(fit_first), fl=i32(fl), fp=i32(fp), fw=f64(fw), fre=f64(fre), fim=f64(fim),
                imf=i64(img_first), are=f64(A_all.real), aim=f64(A_all.imag), zre=f64(Z_all.real),
                zim=f64(Z_all.imag), kre=f64(med.k.real), kim=f64(med.k.imag),
                d=f64(np.concatenate([med.d, [0.0]])))
    phi = np.zeros(2 * tgt.shape[0], dtype=np.float64)
    sx, sy, sz = [np.ascontiguousarray(src[:, i]) for i in range(3)]
    tx, ty = [np.ascontiguousarray(tgt[:, i]) for i in range(2)]
    D, L = ctypes.c_double, ctypes.c_int64
    lib.oracle_cross_sum(
        ctypes.c_int64(src.shape[0]), _p(sx, D), _p(sy, D), _p(sz, D), _p(qi, D),
        _p(slay, ctypes.c_int), ctypes.c_int64(tgt.shape[0]), _p(tx, D), _p(ty, D),
        _p(arrs['ff'], L), _p(arrs['fl'], ctypes.c_int), _p(arrs['fp'], ctypes.c_int),
        _p(arrs['fw'], D), _p(arrs['fre'], D), _p(arrs['fim'], D), _p(arrs['imf'], L),
        _p(arrs['are'], D), _p(arrs['aim'], D), _p(arrs['zre'], D), _p(arrs['zim'], D),
        _p(arrs['kre'], D), _p(arrs['kim'], D), _p(arrs['d'], D), _p(phi, D))
    return phi[0::2] + 1j * phi[1::2]
