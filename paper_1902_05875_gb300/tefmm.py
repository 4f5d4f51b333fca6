"""Python binding of libtefmm (include/tefmm.h): argument marshalling only.

Every step of the matrix-vector product runs in the library's CUDA kernels;
this module passes device pointers of torch tensors (or host numpy arrays for
``eval_host``) through ctypes.  There is no fallback: if the library cannot be
built or loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -4
ERR_FIT_FAILED = -6
ERR_NOT_IMPLEMENTED = -8
ERR_TIMEOUT = -10
INJECT_ALLOC = 1
INJECT_FIT = 2
_STATUS = {}

FP64 = 0
MIXED = 1


class Options(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("leaf_cap", ctypes.c_int), ("max_level", ctypes.c_int),
                ("precision", ctypes.c_int), ("n_images", ctypes.c_int), ("n_samples", ctypes.c_int),
                ("T1", ctypes.c_double), ("T0", ctypes.c_double), ("zext", ctypes.c_double * 32),
                ("kh_max", ctypes.c_double), ("algorithm", ctypes.c_int), ("split", ctypes.c_int),
                ("far_of_near", ctypes.c_int), ("scale_output", ctypes.c_int), ("table_n", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("n_v_pairs", ctypes.c_int64), ("n_p2p_pairs", ctypes.c_int64),
                ("n_tables", ctypes.c_int), ("n_images_total", ctypes.c_int),
                ("ms_tree", ctypes.c_double), ("ms_upward", ctypes.c_double),
                ("ms_tables", ctypes.c_double), ("ms_m2l", ctypes.c_double),
                ("ms_downward", ctypes.c_double), ("ms_near", ctypes.c_double),
                ("fit_max_resid", ctypes.c_double), ("n_launches", ctypes.c_int64),
                ("n_cross_tables", ctypes.c_int), ("n_cross_fits", ctypes.c_int),
                ("n_cross_fits_last", ctypes.c_int), ("ms_cross_fit", ctypes.c_double),
                ("fit_max_resid_cross", ctypes.c_double), ("ms_cross_tables", ctypes.c_double),
                ("ms_cross_m2l", ctypes.c_double), ("leaf_cap_used", ctypes.c_int),
                ("ms_autotune", ctypes.c_double), ("n_tables_built", ctypes.c_int),
                ("n_m2l_items", ctypes.c_int64), ("n_m2l_items_cross", ctypes.c_int64),
                ("ms_m2l_kernel", ctypes.c_double), ("n_m2l_kernel_launches", ctypes.c_int),
                ("n_p2p_pairs_layer", ctypes.c_int64 * 8), ("n_fon_pairs", ctypes.c_int64),
                ("n_alg2_tables", ctypes.c_int), ("ms_alg2_build", ctypes.c_double),
                ("n_alg2_image_keys", ctypes.c_int), ("n_near_img_terms", ctypes.c_int64)]


EXPORTED = [
    "tefmm_default_options", "tefmm_plan_create", "tefmm_plan_destroy", "tefmm_eval",
    "tefmm_eval_host", "tefmm_get_stats", "tefmm_status_string", "tefmm_plan_image_counts",
    "tefmm_plan_get_images", "tefmm_plan_set_images", "tefmm_export_tree", "tefmm_export_lists",
    "tefmm_export_expansions", "tefmm_fit_images_noalloc", "tefmm_plan_cross_images",
    "tefmm_eval_batched", "tefmm_set_points", "tefmm_apply", "tefmm_plan_set_cross_images",
    "tefmm_plan_status", "tefmm_batch_graph_create", "tefmm_batch_graph_launch", "tefmm_batch_graph_destroy",
    "tefmm_debug_inject", "tefmm_debug_wait_probe", "tefmm_plan_get_alg2_table",
    "tefmm_debug_sort_u64", "tefmm_debug_scan_i32",
]

_lib = None


def library_path():
    return _build.LIB


def load(build_if_needed=True):
    """Load libtefmm.so (building it first if sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libtefmm.so is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    I64 = ctypes.POINTER(ctypes.c_int64)
    i64 = ctypes.c_int64
    lib.tefmm_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.tefmm_plan_create.argtypes = [ctypes.c_int, D, D, D, ctypes.POINTER(Options), P,
                                      ctypes.POINTER(P)]
    lib.tefmm_plan_destroy.argtypes = [P]
    lib.tefmm_eval.argtypes = [P, i64, P, P, P, P, i64, P, P, P, P, P]
    lib.tefmm_eval_host.argtypes = [P, i64, D, D, D, D, i64, D, D, D, D, P]
    lib.tefmm_set_points.argtypes = [P, i64, P, P, P, i64, P, P, P, P]
    lib.tefmm_apply.argtypes = [P, P, P, P]
    lib.tefmm_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.tefmm_status_string.argtypes = [ctypes.c_int]
    lib.tefmm_status_string.restype = ctypes.c_char_p
    lib.tefmm_plan_image_counts.argtypes = [P, I, I]
    lib.tefmm_plan_get_images.argtypes = [P, I, I, I, I, D, D, D]
    lib.tefmm_plan_set_images.argtypes = [P, I, D, D]
    lib.tefmm_export_tree.argtypes = [P, I, I64, I64] + [I] * 12
    lib.tefmm_export_lists.argtypes = [P, I64, I64, I, I, I, I]
    lib.tefmm_export_expansions.argtypes = [P, D, D]
    lib.tefmm_plan_set_cross_images.argtypes = [P, ctypes.c_int, I, I, D, D]
    lib.tefmm_plan_status.argtypes = [P, P]
    lib.tefmm_plan_get_alg2_table.argtypes = [P, ctypes.c_int, ctypes.c_int, I, I, D, D]
    lib.tefmm_debug_sort_u64.argtypes = [P, P, P, P, i64, P]
    lib.tefmm_debug_scan_i32.argtypes = [P, P, i64, ctypes.c_int, P]
    lib.tefmm_debug_inject.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.tefmm_debug_wait_probe.argtypes = [P, ctypes.c_int, P]
    lib.tefmm_batch_graph_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                             P, ctypes.POINTER(P)]
    lib.tefmm_batch_graph_launch.argtypes = [P, P]
    lib.tefmm_batch_graph_destroy.argtypes = [P]
    lib.tefmm_eval_batched.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(BatchItem), ctypes.c_int, P, I]
    lib.tefmm_fit_images_noalloc.argtypes = [ctypes.c_int, D, D, D, ctypes.POINTER(Options), P,
                                             I, I, I, I, D, D]
    for name in EXPORTED:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    lib.tefmm_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


class TefmmError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = load(False).tefmm_status_string(status).decode()
        super().__init__(f"{what}: {msg} ({status})")


def _check(status, what):
    if status != OK:
        raise TefmmError(status, what)


def _dptr(a):
    return ctypes.cast(a.ctypes.data, ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return ctypes.cast(a.ctypes.data, ctypes.POINTER(ctypes.c_int))


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class BatchItem(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int64), ("sx", ctypes.c_void_p), ("sy", ctypes.c_void_p),
                ("sz", ctypes.c_void_p), ("q", ctypes.c_void_p), ("nt", ctypes.c_int64),
                ("tx", ctypes.c_void_p), ("ty", ctypes.c_void_p), ("tz", ctypes.c_void_p),
                ("phi", ctypes.c_void_p)]


def eval_batched(plans, instances, n_workers=8, stream=None):
    """``tefmm_eval_batched``: plans[i] evaluates instances[i] = (sx, sy, sz, q, out),
    contiguous CUDA tensors (float64 coordinates, complex128 charges and output;
    targets are the sources).  Returns the per-instance status list."""
    lib = load()
    n = len(plans)
    items = (BatchItem * max(n, 1))()
    keep = []
    for i, (sx, sy, sz, q, out) in enumerate(instances):
        for a in (sx, sy, sz):
            if not (a.is_cuda and a.is_contiguous()):
                raise ValueError("coordinates must be contiguous CUDA tensors")
        vp = lambda t: t.data_ptr()
        items[i] = BatchItem(sx.numel(), vp(sx), vp(sy), vp(sz), vp(q), sx.numel(), None, None, None,
                             vp(out))
        keep.append((sx, sy, sz, q, out))
    hs = (ctypes.c_void_p * max(n, 1))(*[pl.h.value for pl in plans])
    st = (ctypes.c_int * max(n, 1))()
    _check(lib.tefmm_eval_batched(n, hs, items, int(n_workers), _stream_handle(stream), st),
           "tefmm_eval_batched")
    for pl, (sx, *_rest) in zip(plans, instances):     # the plans now hold these points
        pl._n_sources = pl._n_targets = sx.numel()
    return list(st[:n])


class BatchGraph:
    """``tefmm_batch_graph_create``: the charge phases (apply) of several plans,
    each on the points of its last set_points / eval, captured into one CUDA
    graph; ``launch()`` replays the whole batch with one graph launch.  qs[i]
    and phis[i] are contiguous complex128 CUDA tensors that stay bound to the
    graph: write new charges into qs[i] in place between launches."""

    def __init__(self, plans, qs, phis, stream=None):
        import torch
        self.lib = load()
        n = len(plans)
        for q, phi, pl in zip(qs, phis, plans):
            for t in (q, phi):
                if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
                    raise ValueError("charges and potentials must be contiguous complex128 CUDA tensors")
            if q.numel() != getattr(pl, "_n_sources", None) or phi.numel() != getattr(pl, "_n_targets", None):
                raise ValueError("q and phi must match the plan's last set_points() / eval()")
        self._keep = (list(plans), list(qs), list(phis))
        hp = (ctypes.c_void_p * n)(*[pl.h.value for pl in plans])
        hq = (ctypes.c_void_p * n)(*[q.data_ptr() for q in qs])
        hphi = (ctypes.c_void_p * n)(*[phi.data_ptr() for phi in phis])
        h = ctypes.c_void_p()
        _check(self.lib.tefmm_batch_graph_create(n, hp, hq, hphi, _stream_handle(stream), ctypes.byref(h)),
               "tefmm_batch_graph_create")
        self.h = h

    def launch(self, stream=None):
        _check(self.lib.tefmm_batch_graph_launch(self.h, _stream_handle(stream)), "tefmm_batch_graph_launch")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tefmm_batch_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A layered medium plus its DCIM images (``tefmm_plan_create``)."""

    def __init__(self, interfaces, k, p=6, leaf_cap=64, max_level=20, precision=FP64,
                 n_images=8, n_samples=101, T1=10.0, T0=0.0, zext=None, kh_max=3.5,
                 far_of_near=True, scale_output=False, algorithm=1, table_n=0, stream=None):
        lib = load()
        self.lib = lib
        k = np.asarray(k, dtype=complex).reshape(-1)
        d = np.ascontiguousarray(np.asarray(interfaces, dtype=np.float64).reshape(-1))
        kre = np.ascontiguousarray(k.real.astype(np.float64))
        kim = np.ascontiguousarray(k.imag.astype(np.float64))
        opt = Options()
        lib.tefmm_default_options(ctypes.byref(opt))
        opt.p, opt.leaf_cap, opt.max_level = int(p), int(leaf_cap), int(max_level)
        opt.precision = int(precision)
        opt.n_images, opt.n_samples = int(n_images), int(n_samples)
        opt.T1, opt.T0 = float(T1), float(T0)
        opt.kh_max = 0.0 if kh_max is None else float(kh_max)
        opt.scale_output = 1 if scale_output else 0
        opt.far_of_near = 1 if far_of_near else 0
        opt.algorithm = int(algorithm)
        opt.table_n = int(table_n)
        if zext is not None:
            for l, (a, b) in enumerate(zext):
                opt.zext[2 * l] = float(a)
                opt.zext[2 * l + 1] = float(b)
        self.n_layers = k.size
        self.p = int(p)
        self.np = (p + 1) * (p + 2) * (p + 3) // 6
        h = ctypes.c_void_p()
        st = _stream_handle(stream) if stream is not None else ctypes.c_void_p(0)
        _check(lib.tefmm_plan_create(k.size, _dptr(d) if d.size else None, _dptr(kre), _dptr(kim),
                                     ctypes.byref(opt), st, ctypes.byref(h)), "tefmm_plan_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tefmm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- evaluation ----------------------------------------------------------
    def eval(self, sx, sy, sz, q, tx=None, ty=None, tz=None, out=None, stream=None):
        """Device evaluation.  sx.. are contiguous float64 CUDA tensors, q a
        complex128 CUDA tensor; targets default to the sources.  Returns the
        complex128 potentials (``out`` if given)."""
        import torch
        shared = tx is None
        if shared:
            tx, ty, tz = sx, sy, sz
        for a in (sx, sy, sz, tx, ty, tz):
            if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous():
                raise ValueError("coordinates must be contiguous float64 CUDA tensors")
        if q.dtype != torch.complex128 or not q.is_cuda or not q.is_contiguous():
            raise ValueError("q must be a contiguous complex128 CUDA tensor")
        ns, nt = sx.numel(), tx.numel()
        if sy.numel() != ns or sz.numel() != ns or ty.numel() != nt or tz.numel() != nt:
            raise ValueError("coordinate arrays of one point set must have equal lengths")
        if q.numel() != ns:
            raise ValueError("q must have one entry per source")
        if out is None:
            out = torch.empty(nt, dtype=torch.complex128, device=sx.device)
        elif out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous() or out.numel() != nt:
            raise ValueError("out must be a contiguous complex128 CUDA tensor with one entry per target")
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        _check(self.lib.tefmm_eval(self.h, ns, vp(sx), vp(sy), vp(sz), vp(q), nt, vp(tx), vp(ty),
                                   vp(tz), vp(out), _stream_handle(stream)), "tefmm_eval")
        self._n_sources, self._n_targets = ns, nt
        return out

    def set_points(self, sx, sy, sz, tx=None, ty=None, tz=None, stream=None):
        """``tefmm_set_points``: build the charge-independent part (trees, lists,
        keys, fits, tables) for these points; targets default to the sources."""
        import torch
        shared = tx is None
        if shared:
            tx, ty, tz = sx, sy, sz
        for a in (sx, sy, sz, tx, ty, tz):
            if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous():
                raise ValueError("coordinates must be contiguous float64 CUDA tensors")
        ns, nt = sx.numel(), tx.numel()
        if sy.numel() != ns or sz.numel() != ns or ty.numel() != nt or tz.numel() != nt:
            raise ValueError("coordinate arrays of one point set must have equal lengths")
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        self._n_sources = self._n_targets = None      # unknown until the call succeeds
        _check(self.lib.tefmm_set_points(self.h, ns, vp(sx), vp(sy), vp(sz), nt, vp(tx),
                                         vp(ty), vp(tz), _stream_handle(stream)), "tefmm_set_points")
        self._n_sources, self._n_targets = ns, nt

    def apply(self, q, out=None, stream=None):
        """``tefmm_apply``: potentials of charges q (contiguous complex128 CUDA
        tensor, source order) on the points of the last set_points / eval."""
        import torch
        if q.dtype != torch.complex128 or not q.is_cuda or not q.is_contiguous():
            raise ValueError("q must be a contiguous complex128 CUDA tensor")
        n = getattr(self, "_n_targets", None)
        ns = getattr(self, "_n_sources", None)
        if ns is not None and q.numel() != ns:
            raise ValueError("q must have one entry per source of the last set_points() / eval()")
        if out is None:
            if n is None:
                raise RuntimeError("apply() needs a successful set_points() or eval() first")
            out = torch.empty(n, dtype=torch.complex128, device=q.device)
        elif out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous() or \
                (n is not None and out.numel() != n):
            raise ValueError("out must be a contiguous complex128 CUDA tensor with one entry per target")
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        _check(self.lib.tefmm_apply(self.h, vp(q), vp(out), _stream_handle(stream)), "tefmm_apply")
        return out

    def eval_host(self, src, q, tgt=None, stream=None):
        """Host evaluation through ``tefmm_eval_host`` (copies inside)."""
        src = np.asarray(src, dtype=np.float64)
        sx, sy, sz = [np.ascontiguousarray(src[:, i]) for i in range(3)]
        qi = np.ascontiguousarray(np.stack([np.real(q), np.imag(q)], -1).astype(np.float64))
        if tgt is None:
            tx, ty, tz, nt = sx, sy, sz, len(sx)
        else:
            tgt = np.asarray(tgt, dtype=np.float64)
            tx, ty, tz = [np.ascontiguousarray(tgt[:, i]) for i in range(3)]
            nt = len(tx)
        phi = np.zeros(2 * nt, dtype=np.float64)
        st = _stream_handle(stream) if stream is not None else ctypes.c_void_p(0)
        _check(self.lib.tefmm_eval_host(self.h, len(sx), _dptr(sx), _dptr(sy), _dptr(sz), _dptr(qi),
                                        nt, _dptr(tx), _dptr(ty), _dptr(tz), _dptr(phi), st),
               "tefmm_eval_host")
        return phi[0::2] + 1j * phi[1::2]

    def status(self, stream=None):
        """``tefmm_plan_status``: raises if the plan's device work so far flagged an error."""
        _check(self.lib.tefmm_plan_status(self.h, _stream_handle(stream)), "tefmm_plan_status")

    # -- inspection ----------------------------------------------------------
    def stats(self):
        s = Stats()
        _check(self.lib.tefmm_get_stats(self.h, ctypes.byref(s)), "tefmm_get_stats")
        out = {f: getattr(s, f) for f, _ in Stats._fields_}
        out["n_p2p_pairs_layer"] = list(s.n_p2p_pairs_layer)
        return out

    def images(self):
        nt_ = ctypes.c_int()
        ni = ctypes.c_int()
        _check(self.lib.tefmm_plan_image_counts(self.h, ctypes.byref(nt_), ctypes.byref(ni)), "counts")
        n, m = nt_.value, ni.value
        lay = np.zeros(n, np.int32)
        tag = np.zeros(n, np.int32)
        first = np.zeros(n, np.int32)
        cnt = np.zeros(n, np.int32)
        geom = np.zeros(4 * n, np.float64)
        A = np.zeros(2 * max(m, 1), np.float64)
        Z = np.zeros(2 * max(m, 1), np.float64)
        _check(self.lib.tefmm_plan_get_images(self.h, _iptr(lay), _iptr(tag), _iptr(first), _iptr(cnt),
                                              _dptr(geom), _dptr(A), _dptr(Z)), "get_images")
        out = []
        for i in range(n):
            a, b = first[i], first[i] + cnt[i]
            out.append(dict(layer=int(lay[i]), tag=int(tag[i]), sz=geom[4 * i], szp=geom[4 * i + 1],
                            c=geom[4 * i + 2], zeta_min=geom[4 * i + 3],
                            A=A[2 * a:2 * b:2] + 1j * A[2 * a + 1:2 * b:2],
                            Z=Z[2 * a:2 * b:2] + 1j * Z[2 * a + 1:2 * b:2]))
        return out

    def set_images(self, per_term):
        """per_term: list (same order as images()) of (A, Z) complex arrays."""
        cnt = np.array([len(a) for a, _ in per_term], dtype=np.int32)
        A = np.concatenate([np.asarray(a, complex) for a, _ in per_term]) if cnt.sum() else np.zeros(1, complex)
        Z = np.concatenate([np.asarray(z, complex) for _, z in per_term]) if cnt.sum() else np.zeros(1, complex)
        Ai = np.ascontiguousarray(np.stack([A.real, A.imag], -1).reshape(-1))
        Zi = np.ascontiguousarray(np.stack([Z.real, Z.imag], -1).reshape(-1))
        _check(self.lib.tefmm_plan_set_images(self.h, _iptr(cnt), _dptr(Ai), _dptr(Zi)), "set_images")

    def export_tree(self):
        nn = ctypes.c_int()
        ns = ctypes.c_int64()
        nt = ctypes.c_int64()
        nul = [None] * 12
        _check(self.lib.tefmm_export_tree(self.h, ctypes.byref(nn), ctypes.byref(ns), ctypes.byref(nt),
                                          *nul), "export_tree")
        n = nn.value
        arrs = {k: np.zeros(max(n, 1), np.int32) for k in
                ("layer", "level", "ix", "iy", "iz", "parent", "s0", "s1", "t0", "t1")}
        perm_s = np.zeros(max(ns.value, 1), np.int32)
        perm_t = np.zeros(max(nt.value, 1), np.int32)
        _check(self.lib.tefmm_export_tree(
            self.h, None, None, None, *[_iptr(arrs[k]) for k in
                                        ("layer", "level", "ix", "iy", "iz", "parent", "s0", "s1", "t0", "t1")],
            _iptr(perm_s), _iptr(perm_t)), "export_tree")
        out = {k: v[:n] for k, v in arrs.items()}
        out["perm_s"] = perm_s[:ns.value]
        out["perm_t"] = perm_t[:nt.value]
        out["n_nodes"] = n
        return out

    def export_lists(self):
        nv = ctypes.c_int64()
        nn_ = ctypes.c_int64()
        _check(self.lib.tefmm_export_lists(self.h, ctypes.byref(nv), ctypes.byref(nn_), None, None, None,
                                           None), "export_lists")
        n_nodes = self.stats()["n_nodes"]
        vp = np.zeros(n_nodes + 1, np.int32)
        npp = np.zeros(n_nodes + 1, np.int32)
        vs = np.zeros(max(nv.value, 1), np.int32)
        ns_ = np.zeros(max(nn_.value, 1), np.int32)
        _check(self.lib.tefmm_export_lists(self.h, None, None, _iptr(vp), _iptr(vs), _iptr(npp),
                                           _iptr(ns_)), "export_lists")
        return vp, vs[:nv.value], npp, ns_[:nn_.value]

    def cross_images(self):
        """Cached cross-layer fits: {(l, l', 'up'|'down', level, iz_s, k3'): (A, Z)}."""
        n = ctypes.c_int()
        _check(self.lib.tefmm_plan_cross_images(self.h, ctypes.byref(n), None, None, None, None),
               "cross_images")
        m = n.value
        keys = np.zeros(6 * max(m, 1), np.int32)
        cnt = np.zeros(max(m, 1), np.int32)
        A = np.zeros(2 * 32 * max(m, 1), np.float64)
        Z = np.zeros(2 * 32 * max(m, 1), np.float64)
        _check(self.lib.tefmm_plan_cross_images(self.h, ctypes.byref(n), _iptr(keys), _iptr(cnt),
                                                _dptr(A), _dptr(Z)), "cross_images")
        out = {}
        for i in range(m):
            lt, ls, d, lev, izs, k3p = (int(v) for v in keys[6 * i:6 * i + 6])
            j = 32 * i + np.arange(cnt[i])
            out[(lt, ls, 'up' if d == 0 else 'down', lev, izs, k3p)] = (
                A[2 * j] + 1j * A[2 * j + 1], Z[2 * j] + 1j * Z[2 * j + 1])
        return out

    def alg2_table(self, layer, tag, values=True):
        """One Algorithm 2 table (``tefmm_plan_get_alg2_table``): (rho_max,
        zeta_lo, zeta_hi, T) with T complex of shape (n, n, entries) indexed
        [i_rho, j_zeta, entry], or None for T when values is False."""
        n, ne = ctypes.c_int(), ctypes.c_int()
        rng = np.zeros(3)
        _check(self.lib.tefmm_plan_get_alg2_table(self.h, int(layer), int(tag), ctypes.byref(n), ctypes.byref(ne),
                                                  _dptr(rng), None), "tefmm_plan_get_alg2_table")
        T = None
        if values:
            buf = np.zeros(2 * n.value * n.value * ne.value)
            _check(self.lib.tefmm_plan_get_alg2_table(self.h, int(layer), int(tag), ctypes.byref(n),
                                                      ctypes.byref(ne), _dptr(rng), _dptr(buf)),
                   "tefmm_plan_get_alg2_table")
            T = buf.view(np.complex128).reshape(n.value, n.value, ne.value)
        return float(rng[0]), float(rng[1]), float(rng[2]), T

    def set_cross_images(self, fits):
        """``tefmm_plan_set_cross_images``: fits {(l, l', 'up'|'down', level, iz_s, k3'): (A, Z)}
        (the layout of cross_images()) replace or join the plan's cached cross-layer fits."""
        items = list(fits.items())
        m = len(items)
        keys = np.zeros(6 * max(m, 1), np.int32)
        cnt = np.zeros(max(m, 1), np.int32)
        A = np.zeros(2 * 32 * max(m, 1), np.float64)
        Z = np.zeros(2 * 32 * max(m, 1), np.float64)
        for i, ((lt, ls, d, lev, izs, k3p), (a, z)) in enumerate(items):
            a = np.asarray(a, complex)
            z = np.asarray(z, complex)
            if len(a) != len(z) or len(a) > 32:
                raise ValueError("at most 32 images per fit, A and Z of equal length")
            keys[6 * i:6 * i + 6] = (lt, ls, 0 if d == 'up' else 1, lev, izs, k3p)
            cnt[i] = len(a)
            j = 32 * i + np.arange(len(a))
            A[2 * j], A[2 * j + 1] = a.real, a.imag
            Z[2 * j], Z[2 * j + 1] = z.real, z.imag
        _check(self.lib.tefmm_plan_set_cross_images(self.h, m, _iptr(keys), _iptr(cnt), _dptr(A), _dptr(Z)),
               "set_cross_images")

    def export_expansions(self):
        n = self.stats()["n_nodes"]
        a = np.zeros(2 * n * self.np, np.float64)
        b = np.zeros(2 * n * self.np, np.float64)
        _check(self.lib.tefmm_export_expansions(self.h, _dptr(a), _dptr(b)), "export_expansions")
        return (a[0::2] + 1j * a[1::2]).reshape(n, self.np), (b[0::2] + 1j * b[1::2]).reshape(n, self.np)


def debug_inject(kind, n=1):
    """``tefmm_debug_inject`` (test hook): the n-th device allocation (INJECT_ALLOC)
    or DCIM fit batch (INJECT_FIT) from now on fails once; kind 0 clears."""
    _check(load().tefmm_debug_inject(int(kind), int(n)), "tefmm_debug_inject")
