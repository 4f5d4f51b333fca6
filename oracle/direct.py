"""Python side of the C direct-sum oracle (``oracle/direct.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  ``build()`` compiles the C
file with gcc (-O2, OpenMP, no FMA contraction) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
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
