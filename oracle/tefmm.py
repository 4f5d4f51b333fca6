"""CPU Taylor-expansion FMM in layered media, FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 3 of the paper:
* Sec. 3.1 (free space): source-box TE alpha_k = sum_j q_j (r_j - r_c)^k
  (eq. ``taylorexpfarxcfree``), target-box TE beta_k (eq.
  ``taylorexplocxclfree``), M2M by the binomial shift (eqs. ``LETOLEmat``,
  ``TETartoTETar``), L2L (eq. ``freeletole``), and the box-to-box translation
  L_k^{k'} = D_r^k D_{r'}^{k'} h0 / (k! k'!).
* Sec. 3.2 (layered media): the same M2M/L2L, and the layered M2L of eq.
  ``tesourceboxtotargetbox`` with D_r^k D_{r'}^{k'} u / (k! k'!).
* Sec. 3.3: DCIM images and the derivative recurrence (``oracle.derivs``).
* Algorithm 1 (upward pass, downward pass with L2L and M2L, L2P, near-field
  direct sum) and the component loop of the heterogeneous algorithm that
  follows it (free space for l = l', up/down reaction components).

Readings where the paper is silent (all stated the same way for the CUDA path):
* One octree per layer, all in one root cube: lo = min over all points per
  axis, side = max over axes of (max - min) (1 if zero).  Integer box
  coordinates i = min(floor(((x - lo) / side) * 2^20), 2^20 - 1) with plain
  IEEE double operations (no fused multiply-add); 60-bit Morton keys with bit
  3b+2 = bit b of ix, 3b+1 = iy, 3b = iz.  Points are sorted by (layer, key,
  input index).  Box centre of coordinate i at level l: lo + (i + 0.5) *
  (side / 2^l).
* A box is split while max(#sources, #targets) > leaf_cap, or while it is
  adjacent to a box of the same level in another layer's tree, and level <
  max_level; only children holding a point exist.  Nodes are numbered
  level-major: by (level, layer, Morton prefix).  The second rule (a reading)
  keeps leaves of different layers apart, so that every cross-layer
  interaction is an M2L (V-list) pair.
* Cross-layer admissibility (a reading): two split boxes of different layers
  at a level where the box size exceeds HX (= 4 min over interfaces of the
  summed gaps between the particle slabs and the interface), horizontally
  within one box of each other (|dx|, |dy| <= 1), are not translated but
  treated like adjacent boxes (their children are paired).  Such vertically
  stacked pairs have expansion centres far (relative to the box size) from
  the closest particles through the interface; taking their translation
  costs 100x in accuracy on slabs 0.1 from the interfaces.
* Interaction lists: a dual-tree traversal of (target tree, source tree),
  which for one tree is the classic adaptive U/V/W/X construction
  (Carrier-Greengard-Rokhlin).  V pairs go through M2L; U, W and X pairs are
  evaluated directly (P2P) -- W/X boxes are whole subtrees.
* Same-layer reaction terms are written in the image-distance form of
  ``Medium.same_layer_terms``; with W = sz z + szp z' + c,
  D_r^k D_r'^k' f / (k! k'!) = (-1)^{k1'+k2'} sz^{k3} szp^{k3'} C(k+k', k) a_{k+k'}
  where a_g = D^g f / g!, C(k+k', k) = prod_i (k_i+k'_i)!/(k_i! k'_i!).
  Offsets of M2L pairs are taken from integer box coordinates:
  X0 = di_x * (side / 2^l), and zt_c + zs_c = 2 lo_z + (i_t + i_s + 1) * (side / 2^l).
* Cross-layer components (target layer l != source layer l', Sec. 3.2-3.3): per
  source z-centre z_c and k3' = 0..p the images of Theta^{k3'} (``oracle.cross``)
  give d^{k3'}_{z'} u / k3'! as image Hankel functions of (X, Y, W), W = z - d_l
  (up) or d_{l-1} - z (down); hence
  D_r^k D_r'^k' u / (k! k'!) = (-1)^{k1'+k2'} C(k1+k1',k1) C(k2+k2',k2)
                               sz^{k3} T^{(k3')}_{(k1+k1', k2+k2', k3)},
  T^{(k3')}_g = sum_j A_j D^g h0(k_l R_j) / g! at (X0, Y0, W(z_t) - W_min - Z_j),
  sz = +1 (up), -1 (down).  Reading: the z-centres z_c (source) and z_t
  (target) of a cross-layer translation are the box centres clamped to the
  layer's particle slab; the source moments are shifted there exactly (M2M
  in z) and the resulting local expansion is shifted back to the box centre
  (L2L in z).  A box of one layer's tree can have its centre outside the
  layer (it straddles an interface); at such a z_c the fitted function grows
  like e^{|k_z| (z_c - d)} along the first DCIM path and cannot be fitted.  Cross-layer near-field pairs are not supported
  (leaves must be small enough that boxes of different layers are never
  adjacent).
* Far-of-near (a reading of the precision pattern the method is built for):
  for a pair of adjacent leaves of one level l, an image j of a same-layer
  term whose depth satisfies -Re Z_j >= kappa_p sqrt(3) h_l, kappa_p =
  10^(10/(p+1)), is far from both leaves (their points lie within sqrt(3) h_l
  of each other's centres in the combined displacement), so its part of the
  pair's field is a smooth function that a Taylor translation of order p
  carries to about kappa_p^-(p+1) = 1e-10 of itself.  Those images go through
  M2L between the two leaves (tables of the far images only, no free-space
  term); the free-space term and the nearer images stay in the direct sum.
  Pairs of leaves of different levels (and W/X pairs) keep every image direct.
* Which layer holds the images of a cross-layer component (a reading): the
  DCIM fit of Sec. 3.3 is accurate to about 1e-8 against Sommerfeld quadrature
  when its images live in the layer of the larger |k|, but only to 1e-6 .. 4e-4
  in the layer of the smaller |k| (branch points k_rho = k_other of the
  spectral function then lie close to the sampling paths).  So a component
  whose target layer l has the smaller |k| is evaluated through reciprocity,
  k_l^2 u_{l l'}(r; r') = k_l'^2 u_{l' l}(r'; r): its M2L matrix between a
  target box t and a source box s is (k_l' / k_l)^2 times the transpose of the
  M2L matrix of component (l', l) from box t to box s, whose fits have their
  images in layer l' (the z-Taylor order of the target plays the role of k3').
"""
from __future__ import annotations

import math

import numpy as np

from .derivs import multi_indices, index_map, n_coeffs, taylor_h0
from . import cross as xl
from . import alg2 as a2

NBITS = 20
# wavenumber admissibility bound (see Trees): on levels where k_max h > KH_MAX,
# split boxes are paired instead of translated; None turns the rule off
KH_MAX = 3.5


def morton_encode(ix, iy, iz):
    key = np.zeros(ix.shape, dtype=np.uint64)
    for b in range(NBITS):
        key |= ((ix >> b) & 1).astype(np.uint64) << np.uint64(3 * b + 2)
        key |= ((iy >> b) & 1).astype(np.uint64) << np.uint64(3 * b + 1)
        key |= ((iz >> b) & 1).astype(np.uint64) << np.uint64(3 * b)
    return key


def morton_decode(prefix, level):
    ix = np.zeros(np.shape(prefix), dtype=np.int64)
    iy = np.zeros_like(ix)
    iz = np.zeros_like(ix)
    p = np.asarray(prefix, dtype=np.uint64)
    for b in range(level):
        iz |= ((p >> np.uint64(3 * b)) & np.uint64(1)).astype(np.int64) << b
        iy |= ((p >> np.uint64(3 * b + 1)) & np.uint64(1)).astype(np.int64) << b
        ix |= ((p >> np.uint64(3 * b + 2)) & np.uint64(1)).astype(np.int64) << b
    return ix, iy, iz


def fon_threshold(p, side, lev):
    """Depth beyond which an image is far for a pair of adjacent leaves of
    level lev (see the far-of-near reading): kappa_p sqrt(3) h."""
    return 10.0 ** (10.0 / (p + 1)) * math.sqrt(3.0) * (side / float(1 << lev))


def fon_anchor(tr, t, s):
    """Far-of-near anchor of a near-list pair (target box t, source box s):
    l* = the coarser of the two levels, T* and S* the boxes of level l* that
    hold t and s.  When T* and S* are adjacent, the far images (-Re Z >=
    fon_threshold(l*)) of every particle pair under (T*, S*) go through one M2L
    from S* to T*, and the pair sum of (t, s) leaves them out.  Returns
    (l*, T*, S*), or None when T* and S* are not adjacent (all images in P2P)."""
    ls = min(int(tr.level[t]), int(tr.level[s]))
    T, S = t, s
    while tr.level[T] > ls:
        T = tr.parent[T]
    while tr.level[S] > ls:
        S = tr.parent[S]
    if max(abs(int(tr.ix[T]) - int(tr.ix[S])), abs(int(tr.iy[T]) - int(tr.iy[S])),
           abs(int(tr.iz[T]) - int(tr.iz[S]))) > 1:
        return None
    return ls, int(T), int(S)


def cross_box_limit(med, zext):
    """HX = 4 min over interfaces of (gap of the slab above + gap of the slab below),
    the gaps between the particle slabs (zext) and the interface; interfaces with
    no gap are skipped; +inf when no interface counts (or no zext)."""
    if zext is None or med.n_layers < 2:
        return np.inf
    g = []
    for m in range(med.L):
        gm = (float(zext[m][0]) - float(med.d[m])) + (float(med.d[m]) - float(zext[m + 1][1]))
        if gm > 0.0:
            g.append(gm)
    return 4.0 * min(g) if g else np.inf


def root_cube(points):
    lo = points.min(axis=0)
    hi = points.max(axis=0)
    side = float(np.max(hi - lo))
    if side == 0.0:
        side = 1.0
    return lo.astype(np.float64), side


def int_coords(xyz, lo, side):
    t = (xyz - lo[None, :]) / side
    t = t * float(1 << NBITS)
    i = np.floor(t).astype(np.int64)
    return np.clip(i, 0, (1 << NBITS) - 1)


class Trees:
    """Per-layer octrees in a common root cube (see module docstring)."""

    def __init__(self, med, src, tgt, leaf_cap, max_level=NBITS, cube=None, zext=None, kh_max=KH_MAX):
        self.med = med
        allp = np.concatenate([src, tgt], 0)
        self.lo, self.side = root_cube(allp) if cube is None else cube
        self.HX = cross_box_limit(med, zext)
        # wavenumber admissibility (kh_max None or <= 0: off): on levels whose box
        # size h has k_max h > kh_max, pairs of split boxes are refined, not translated
        self.kh_max = kh_max
        self.kmax = max(abs(complex(k)) for k in med.k)
        self.leaf_cap = leaf_cap
        self.max_level = max_level
        self.slay = med.layer_of(src[:, 2])
        self.tlay = med.layer_of(tgt[:, 2])
        if np.any(self.slay < 0) or np.any(self.tlay < 0):
            raise ValueError("point on an interface")
        si = int_coords(src, self.lo, self.side)
        ti = int_coords(tgt, self.lo, self.side)
        self.skey = morton_encode(si[:, 0], si[:, 1], si[:, 2])
        self.tkey = morton_encode(ti[:, 0], ti[:, 1], ti[:, 2])
        self.sperm = np.lexsort((np.arange(len(src)), self.skey, self.slay))
        self.tperm = np.lexsort((np.arange(len(tgt)), self.tkey, self.tlay))
        sk = self.skey[self.sperm]
        tk = self.tkey[self.tperm]
        sl = self.slay[self.sperm]
        tl = self.tlay[self.tperm]
        nodes = []      # (layer, level, prefix, parent, s0, s1, t0, t1)
        children = []
        self.root = {}
        frontier = []
        for l in range(med.n_layers):
            s0, s1 = np.searchsorted(sl, l, 'left'), np.searchsorted(sl, l, 'right')
            t0, t1 = np.searchsorted(tl, l, 'left'), np.searchsorted(tl, l, 'right')
            if s1 - s0 + t1 - t0 == 0:
                continue
            self.root[l] = len(nodes)
            nodes.append([l, 0, 0, -1, s0, s1, t0, t1])
            children.append([])
            frontier.append(self.root[l])
        # level-major: all level-(l+1) nodes after all level-l nodes; within a
        # level parents are visited in (layer, prefix) order and children in
        # child-index order, so a level is ordered by (layer, prefix).
        while frontier:
            nxt = []
            # boxes of this level by layer, for the cross-layer adjacency rule
            coords = {}
            for nid in frontier:
                l, lev, pre = nodes[nid][0], nodes[nid][1], nodes[nid][2]
                a, b, c = morton_decode(np.uint64(pre), lev)
                coords[nid] = (l, int(a), int(b), int(c))

            def cross_adjacent(nid):
                l, a, b, c = coords[nid]
                for o, (lo_, a2, b2, c2) in coords.items():
                    if lo_ != l and abs(a - a2) <= 1 and abs(b - b2) <= 1 and abs(c - c2) <= 1:
                        return True
                return False
            for nid in frontier:
                l, lev, pre, _, a0, a1, b0, b1 = nodes[nid]
                if lev >= max_level:
                    continue
                if max(a1 - a0, b1 - b0) <= leaf_cap and not cross_adjacent(nid):
                    continue
                shift = np.uint64(3 * (NBITS - lev - 1))
                sc = (sk[a0:a1] >> shift) & np.uint64(7)
                tc = (tk[b0:b1] >> shift) & np.uint64(7)
                for c in range(8):
                    cs0 = a0 + np.searchsorted(sc, c, 'left')
                    cs1 = a0 + np.searchsorted(sc, c, 'right')
                    ct0 = b0 + np.searchsorted(tc, c, 'left')
                    ct1 = b0 + np.searchsorted(tc, c, 'right')
                    if cs1 - cs0 + ct1 - ct0 == 0:
                        continue
                    cid = len(nodes)
                    nodes.append([l, lev + 1, (pre << 3) | c, nid, cs0, cs1, ct0, ct1])
                    children.append([])
                    children[nid].append(cid)
                    nxt.append(cid)
            frontier = nxt
        self.n_nodes = len(nodes)
        self.layer = np.array([n[0] for n in nodes], dtype=np.int64)
        self.level = np.array([n[1] for n in nodes], dtype=np.int64)
        self.prefix = np.array([n[2] for n in nodes], dtype=np.uint64)
        self.parent = np.array([n[3] for n in nodes], dtype=np.int64)
        self.s0 = np.array([n[4] for n in nodes], dtype=np.int64)
        self.s1 = np.array([n[5] for n in nodes], dtype=np.int64)
        self.t0 = np.array([n[6] for n in nodes], dtype=np.int64)
        self.t1 = np.array([n[7] for n in nodes], dtype=np.int64)
        self.children = children
        self.is_leaf = np.array([len(c) == 0 for c in children])
        ix, iy, iz = [], [], []
        for n in nodes:
            a, b, c = morton_decode(np.uint64(n[2]), n[1])
            ix.append(int(a)); iy.append(int(b)); iz.append(int(c))
        self.ix = np.array(ix, dtype=np.int64)
        self.iy = np.array(iy, dtype=np.int64)
        self.iz = np.array(iz, dtype=np.int64)

    def ns(self, n):
        return self.s1[n] - self.s0[n]

    def nt(self, n):
        return self.t1[n] - self.t0[n]

    def center(self, n):
        h = self.side / float(1 << int(self.level[n]))
        return np.array([self.lo[0] + (self.ix[n] + 0.5) * h,
                         self.lo[1] + (self.iy[n] + 0.5) * h,
                         self.lo[2] + (self.iz[n] + 0.5) * h])

    def cross_colleague(self, a, b):
        """Same-level boxes of different layers, both split, stacked (|dx|, |dy| <= 1)
        and larger than HX: their translation is not taken, their children are paired."""
        la = int(self.level[a])
        if (self.layer[a] == self.layer[b] or la != int(self.level[b]) or self.is_leaf[a] or
                self.is_leaf[b]):
            return False
        if not (self.side / float(1 << la) > self.HX):
            return False
        return max(abs(int(self.ix[a]) - int(self.ix[b])), abs(int(self.iy[a]) - int(self.iy[b]))) <= 1

    def coarse_colleague(self, a, b):
        """Same-level split boxes on a level where the Taylor expansions would
        span k_max h > kh_max: their children are paired instead (no translation)."""
        if self.kh_max is None or self.kh_max <= 0:
            return False
        la = int(self.level[a])
        if la != int(self.level[b]) or self.is_leaf[a] or self.is_leaf[b]:
            return False
        return self.kmax * self.side / float(1 << la) > self.kh_max

    def adjacent(self, a, b):
        la, lb = int(self.level[a]), int(self.level[b])
        if la > lb:
            a, b, la, lb = b, a, lb, la
        s = lb - la
        for ca, cb in ((self.ix[a], self.ix[b]), (self.iy[a], self.iy[b]), (self.iz[a], self.iz[b])):
            lo_ = int(ca) << s
            hi_ = ((int(ca) + 1) << s) - 1
            if int(cb) < lo_ - 1 or int(cb) > hi_ + 1:
                return False
        return True


def build_lists(tr: Trees, lt, ls):
    """Dual-tree traversal of target tree ``lt`` against source tree ``ls``.

    Returns (V, P2P): dicts target node -> sorted list of source nodes; P2P
    only has target leaves, and already folds U, W and the X entries of every
    ancestor-or-self.
    """
    if lt not in tr.root or ls not in tr.root:
        return {}, {}
    rt, rs = tr.root[lt], tr.root[ls]
    if tr.nt(rt) == 0 or tr.ns(rs) == 0:
        return {}, {}
    U, V, W, X = {}, {}, {}, {}

    def add(D, a, b):
        D.setdefault(a, []).append(b)

    def ch_t(n):
        return [c for c in tr.children[n] if tr.nt(c) > 0]

    def ch_s(n):
        return [c for c in tr.children[n] if tr.ns(c) > 0]

    def leaf_target(t, c):
        if tr.is_leaf[c]:
            add(U, t, c)
            return
        for cc in ch_s(c):
            if tr.adjacent(t, cc):
                leaf_target(t, cc)
            else:
                add(W, t, cc)

    def leaf_source(c, s):
        if tr.is_leaf[c]:
            add(U, c, s)
            return
        for cc in ch_t(c):
            if tr.adjacent(cc, s):
                leaf_source(cc, s)
            else:
                add(X, cc, s)

    stack = [(rt, rs)]
    while stack:
        t, s = stack.pop()
        lt_, ls_ = tr.is_leaf[t], tr.is_leaf[s]
        if lt_ and ls_:
            add(U, t, s)
        elif lt_:
            for c in ch_s(s):
                if tr.adjacent(t, c):
                    leaf_target(t, c)
                else:
                    add(W, t, c)
        elif ls_:
            for c in ch_t(t):
                if tr.adjacent(c, s):
                    leaf_source(c, s)
                else:
                    add(X, c, s)
        else:
            for ct in ch_t(t):
                for cs in ch_s(s):
                    if tr.adjacent(ct, cs) or tr.cross_colleague(ct, cs) or tr.coarse_colleague(ct, cs):
                        stack.append((ct, cs))
                    else:
                        add(V, ct, cs)
    P2P = {}
    leaves = [n for n in range(tr.n_nodes) if tr.layer[n] == lt and tr.is_leaf[n] and tr.nt(n) > 0]
    for t in leaves:
        lst = list(U.get(t, [])) + list(W.get(t, []))
        a = t
        while a >= 0:
            lst += X.get(a, [])
            a = tr.parent[a]
        if lst:
            P2P[t] = sorted(lst)
    V = {t: sorted(v) for t, v in V.items()}
    return V, P2P


# ----------------------------------------------------------------------------
# Taylor-expansion operators (Sec. 3.1)

class Ops:
    def __init__(self, p):
        self.p = p
        self.mi = multi_indices(p)
        self.np_ = len(self.mi)
        im2 = index_map(2 * p)
        mi = self.mi
        n = self.np_
        self.g = np.zeros((n, n), dtype=np.int64)        # index of k + k' in the order-2p list
        self.mult = np.zeros((n, n))                     # prod_i C(k_i + k'_i, k_i)
        self.sxy = np.zeros((n, n))                      # (-1)^{k1' + k2'}
        self.s3p = np.zeros((n, n))                      # (-1)^{k3'}
        self.s3g = np.zeros((n, n))                      # (-1)^{k3 + k3'}
        for a in range(n):
            for b in range(n):
                gg = mi[a] + mi[b]
                self.g[a, b] = im2[tuple(int(v) for v in gg)]
                self.mult[a, b] = np.prod([math.comb(int(gg[i]), int(mi[a][i])) for i in range(3)])
                self.sxy[a, b] = (-1.0) ** (mi[b][0] + mi[b][1])
                self.s3p[a, b] = (-1.0) ** mi[b][2]
                self.s3g[a, b] = (-1.0) ** (mi[a][2] + mi[b][2])
        # binomial tables for M2M / L2L: C(k, k') for k' <= k componentwise
        self.binom = np.zeros((n, n))
        self.dpow = np.zeros((n, n), dtype=np.int64)     # index of k - k'
        self.valid = np.zeros((n, n), dtype=bool)
        im = index_map(p)
        for a in range(n):
            for b in range(n):
                d = mi[a] - mi[b]
                if np.all(d >= 0):
                    self.valid[a, b] = True
                    self.binom[a, b] = np.prod([math.comb(int(mi[a][i]), int(mi[b][i])) for i in range(3)])
                    self.dpow[a, b] = im[tuple(int(v) for v in d)]

    def monomials(self, d):
        """d: (..., 3) -> (..., n_p) with d^k."""
        d = np.asarray(d)
        out = np.ones(d.shape[:-1] + (self.np_,), dtype=d.dtype if np.iscomplexobj(d) else float)
        for t, k in enumerate(self.mi):
            out[..., t] = d[..., 0] ** k[0] * d[..., 1] ** k[1] * d[..., 2] ** k[2]
        return out

    def p2m(self, pts, q, c):
        """alpha_k = sum_j q_j (r_j - c)^k."""
        return q @ self.monomials(pts - c[None, :])

    def shift_matrix(self, dc):
        """B[k, k'] = C(k, k') dc^{k-k'} for k' <= k componentwise (else 0); the
        same few offsets recur (8 child positions per level), so B is kept."""
        key = tuple(float(v) for v in dc)
        cache = self.__dict__.setdefault('_shift_cache', {})
        if key not in cache:
            m = self.monomials(np.asarray(dc, dtype=float)[None, :])[0]
            cache[key] = np.where(self.valid, self.binom * m[self.dpow], 0.0)
        return cache[key]

    def m2m(self, alpha_child, dc):
        """Parent moments from a child's, dc = child centre - parent centre:
        gamma_k = sum_{k' <= k} C(k, k') dc^{k-k'} alpha_{k'}."""
        return self.shift_matrix(dc) @ alpha_child

    def l2l(self, beta_parent, dc):
        """Child local from the parent's, dc = child centre - parent centre:
        lambda_k = sum_{k' >= k} C(k', k) dc^{k'-k} beta_{k'}."""
        return self.shift_matrix(dc).T @ beta_parent

    def l2p(self, beta, pts, c):
        return self.monomials(pts - c[None, :]) @ beta

    def cross_maps(self):
        """Index (into the order-2p list) and coefficient of the cross-layer M2L:
        gx[k,k'] = idx(k1+k1', k2+k2', k3), cx[k,k'] = (-1)^{k1'+k2'} C(k1+k1',k1) C(k2+k2',k2),
        k3p[k'] = k3'."""
        if not hasattr(self, 'gx'):
            im2 = index_map(2 * self.p)
            mi = self.mi
            n = self.np_
            self.gx = np.zeros((n, n), dtype=np.int64)
            self.cx = np.zeros((n, n))
            for a in range(n):
                for b in range(n):
                    g = (int(mi[a][0] + mi[b][0]), int(mi[a][1] + mi[b][1]), int(mi[a][2]))
                    self.gx[a, b] = im2[g]
                    self.cx[a, b] = ((-1.0) ** (mi[b][0] + mi[b][1]) *
                                     math.comb(g[0], int(mi[a][0])) * math.comb(g[1], int(mi[a][1])))
            self.k3p = mi[:, 2].copy()
        return self.gx, self.cx, self.k3p

    def m2l_matrix(self, A, B):
        """M2L matrix from the combined derivative tables (see module docstring):
        H[k,k'] = C(k+k',k) (-1)^{k1'+k2'} (A_{k+k'} + (-1)^{k3'} B_{k+k'})."""
        return self.mult * self.sxy * (A[self.g] + self.s3p * B[self.g])


class TEFMM:
    """Algorithm 1 + the component loop, for every (target layer, source layer)."""

    def __init__(self, med, images, p, leaf_cap, max_level=NBITS, cube=None, zext=None,
                 cross_images=None, n_images=None, kh_max=KH_MAX, far_of_near=True,
                 algorithm=1, table_n=64):
        self.med = med
        self.kh_max = kh_max
        # Algorithm 2 (Sec. 4.2): same-layer reaction derivatives of the V
        # pairs from interpolated tables of Sommerfeld integrals (oracle.alg2)
        # instead of complex images; the near field keeps the images, and so
        # do the far-of-near translations (their far images only)
        self.algorithm = algorithm
        self.table_n = table_n
        self.alg2 = {}
        self.far_of_near = far_of_near
        self.images = images
        self.zext = zext if zext is not None else (images.zext if images is not None else None)
        # cross-layer images: dict (lt, ls, direction, level, izs, k3p) -> (A, Z);
        # missing entries are fitted with oracle.cross.fit_cross
        self.cross_images = {} if cross_images is None else cross_images
        self.n_images = n_images if n_images is not None else 8
        self.p = p
        self.leaf_cap = leaf_cap
        self.max_level = max_level
        self.cube = cube
        self.ops = Ops(p)

    def setup(self, src, tgt):
        self.src = np.asarray(src, float)
        self.tgt = np.asarray(tgt, float)
        self.tr = Trees(self.med, self.src, self.tgt, self.leaf_cap, self.max_level, self.cube,
                        self.zext, kh_max=self.kh_max)
        self.lists = {}
        for lt in range(self.med.n_layers):
            for ls in range(self.med.n_layers):
                V, P = build_lists(self.tr, lt, ls)
                if V or P:
                    if lt != ls and P:
                        raise NotImplementedError("cross-layer near-field pairs")
                    self.lists[(lt, ls)] = (V, P)
        return self

    # -- upward pass --------------------------------------------------------
    def upward(self, q):
        tr, ops = self.tr, self.ops
        sp = self.src[tr.sperm]
        qs = np.asarray(q)[tr.sperm]
        alpha = np.zeros((tr.n_nodes, ops.np_), dtype=complex)
        order = np.argsort(-tr.level, kind='stable')
        for n in order:
            if tr.ns(n) == 0:
                continue
            c = tr.center(n)
            if tr.is_leaf[n]:
                a, b = tr.s0[n], tr.s1[n]
                alpha[n] = ops.p2m(sp[a:b], qs[a:b], c)
            else:
                for ch in tr.children[n]:
                    if tr.ns(ch) > 0:
                        alpha[n] += ops.m2m(alpha[ch], tr.center(ch) - c)
        return alpha

    # -- derivative tables (Sec. 3.3) ---------------------------------------
    def _tables(self, l, lev, keysB, keysA, far_thr=None):
        """Combined tables per key at one level of layer l.

        keysB: (n, 3) integer offsets (dix, diy, diz) -> B = free + ud + (-1)^{g3} du
        keysA: (n, 3) (dix, diy, izt + izs)           -> A = uu + (-1)^{g3} dd
        With far_thr (far-of-near pairs): no free-space term, and only the
        images with -Re Z >= far_thr.
        """
        tr = self.tr
        P2 = 2 * self.p
        k = self.med.k[l]
        h = tr.side / float(1 << lev)
        mi2 = multi_indices(P2)
        odd3 = (-1.0) ** mi2[:, 2]
        terms = {t['tag']: t for t in self.images.terms[l]} if self.images is not None else {}
        if self.algorithm == 2 and far_thr is None:
            return self._tables_alg2(l, h, keysB, keysA, odd3)
        TB = np.zeros((len(keysB), len(mi2)), dtype=complex)
        TA = np.zeros((len(keysA), len(mi2)), dtype=complex)
        if len(keysB):
            X0 = keysB[:, 0] * h
            Y0 = keysB[:, 1] * h
            dz = keysB[:, 2] * h
            if far_thr is None:
                TB += taylor_h0(X0, Y0, dz.astype(complex), k, P2)
            for tag, sgn in (('ud', None), ('du', odd3)):
                if tag not in terms:
                    continue
                t = terms[tag]
                W0 = t['sz'] * dz + t['c']          # sz z_t + szp z_s + c with szp = -sz
                for A, Z in zip(t['A'], t['Z']):
                    if far_thr is not None and not (-Z.real >= far_thr):
                        continue
                    tab = A * taylor_h0(X0, Y0, W0 - t['zeta_min'] - Z, k, P2)
                    TB += tab if sgn is None else tab * sgn[None, :]
        if len(keysA):
            X0 = keysA[:, 0] * h
            Y0 = keysA[:, 1] * h
            zsum = 2.0 * tr.lo[2] + (keysA[:, 2] + 1) * h
            for tag, sgn in (('uu', None), ('dd', odd3)):
                if tag not in terms:
                    continue
                t = terms[tag]
                W0 = t['sz'] * zsum + t['c']        # sz = szp for these terms
                for A, Z in zip(t['A'], t['Z']):
                    if far_thr is not None and not (-Z.real >= far_thr):
                        continue
                    tab = A * taylor_h0(X0, Y0, W0 - t['zeta_min'] - Z, k, P2)
                    TA += tab if sgn is None else tab * sgn[None, :]
        return TB, TA

    def alg2_ranges(self, l):
        """Grid ranges of the Algorithm 2 tables of layer l over all its
        same-layer M2L pairs: (rho_max, {tag: (zeta_lo, zeta_hi)}), or None."""
        tr = self.tr
        V = self.lists[(l, l)][0] if (l, l) in self.lists else {}
        keys = []
        for t, lst in V.items():
            for s in lst:
                lev = int(tr.level[t])
                h = tr.side / float(1 << lev)
                keys.append((h, int(tr.ix[t] - tr.ix[s]), int(tr.iy[t] - tr.iy[s]), int(tr.iz[t] - tr.iz[s]),
                             2.0 * tr.lo[2] + (int(tr.iz[t] + tr.iz[s]) + 1) * h))
        floor = {t['tag']: t['zeta_min'] for t in self.images.terms[l]}
        return a2.layer_ranges(self.med, l, keys, floor) if keys else None

    def alg2_tables(self, l):
        """The Algorithm 2 tables of layer l, {tag: Alg2Table}, over the grid
        ranges of all the layer's same-layer M2L pairs (built once)."""
        if l not in self.alg2:
            tabs = {}
            r = self.alg2_ranges(l)
            if r is not None:
                rho_max, rng = r
                for tag, (lo, hi) in rng.items():
                    tabs[tag] = a2.Alg2Table(a2.medium_T(self.med, l, tag, 2 * self.p), 2 * self.p,
                                             rho_max, lo, hi, self.table_n)
            self.alg2[l] = tabs
        return self.alg2[l]

    def _tables_alg2(self, l, h, keysB, keysA, odd3):
        """_tables with the reaction part from the Algorithm 2 tables: the
        same combinations (B = free + ud + (-1)^{g3} du, A = uu + (-1)^{g3} dd)
        with each term's D^g F / g! interpolated at its image distance; a key
        below the term's zeta_min (box centres beyond the particle slab) keeps
        the term's images."""
        P2 = 2 * self.p
        k = self.med.k[l]
        tabs = self.alg2_tables(l)
        terms = {t['tag']: t for t in self.images.terms[l]}
        n = len(multi_indices(P2))
        TB = np.zeros((len(keysB), n), dtype=complex)
        TA = np.zeros((len(keysA), n), dtype=complex)
        for T, keys, tags in ((TB, keysB, ('ud', 'du')), (TA, keysA, ('uu', 'dd'))):
            if not len(keys):
                continue
            X0 = keys[:, 0] * h
            Y0 = keys[:, 1] * h
            if T is TB:
                zarg = keys[:, 2] * h
                T += taylor_h0(X0, Y0, zarg.astype(complex), k, P2)
            else:
                zarg = 2.0 * self.tr.lo[2] + (keys[:, 2] + 1) * h
            for tag in tags:
                if tag not in terms:
                    continue
                t = terms[tag]
                sgn = odd3 if tag in ('du', 'dd') else 1.0
                for i in range(len(keys)):
                    zeta = t['sz'] * zarg[i] + t['c']
                    if zeta >= t['zeta_min']:
                        T[i] += tabs[tag].derivatives(float(X0[i]), float(Y0[i]), zeta) * sgn
                    else:
                        for A, Z in zip(t['A'], t['Z']):
                            T[i] += A * taylor_h0(X0[i:i + 1], Y0[i:i + 1], np.array([zeta - t['zeta_min'] - Z]),
                                                  k, P2)[0] * sgn
        return TB, TA

    # -- downward pass -------------------------------------------------------
    def downward(self, alpha, only_targets=None):
        """Local expansions of every target node (or only the ancestors of the
        given target leaves)."""
        tr, ops = self.tr, self.ops
        beta = np.zeros((tr.n_nodes, ops.np_), dtype=complex)
        need = None
        if only_targets is not None:
            need = set()
            for n in only_targets:
                a = n
                while a >= 0:
                    need.add(a)
                    a = tr.parent[a]
        for (lt, ls), (V, P2P) in self.lists.items():
            if lt != ls:
                self._cross_m2l(lt, ls, V, alpha, beta, need)
                continue
            # group V pairs by level; far-of-near pairs (the anchors of the
            # near-list pairs, see fon_anchor) translate their far images only
            pairs = [(t, s) for t, lst in V.items() for s in lst if need is None or t in need]
            self._same_layer_m2l(lt, pairs, alpha, beta, None)
            if self.far_of_near and self.images is not None:
                fon = sorted({a[1:] for t, lst in P2P.items() for s in lst
                              for a in [fon_anchor(tr, t, s)] if a is not None})
                fon = [(T, S) for T, S in fon if need is None or T in need]
                self._same_layer_m2l(lt, fon, alpha, beta, True)
        order = np.argsort(tr.level, kind='stable')
        for n in order:
            par = tr.parent[n]
            if par < 0 or tr.nt(n) == 0:
                continue
            if need is not None and n not in need:
                continue
            beta[n] += ops.l2l(beta[par], tr.center(n) - tr.center(par))
        return beta

    def _same_layer_m2l(self, l, pairs, alpha, beta, fon):
        """M2L of same-layer box pairs, grouped by level and key; fon: the
        far-of-near tables (far images only) of adjacent leaf pairs."""
        tr, ops = self.tr, self.ops
        if pairs:
            pairs = np.array(pairs, dtype=np.int64)
            for lev in np.unique(tr.level[pairs[:, 0]]):
                sel = pairs[tr.level[pairs[:, 0]] == lev]
                t, s = sel[:, 0], sel[:, 1]
                kB = np.stack([tr.ix[t] - tr.ix[s], tr.iy[t] - tr.iy[s], tr.iz[t] - tr.iz[s]], 1)
                kA = np.stack([tr.ix[t] - tr.ix[s], tr.iy[t] - tr.iy[s], tr.iz[t] + tr.iz[s]], 1)
                uB, invB = np.unique(kB, axis=0, return_inverse=True)
                uA, invA = np.unique(kA, axis=0, return_inverse=True)
                thr = fon_threshold(self.p, tr.side, int(lev)) if fon else None
                TB, TA = self._tables(l, int(lev), uB, uA, far_thr=thr)
                zero = np.zeros(TB.shape[1], dtype=complex)
                invB = invB.reshape(-1)
                invA = invA.reshape(-1)
                contrib = np.zeros((len(t), ops.np_), dtype=complex)
                for i in range(len(uB)):
                    m = invB == i
                    contrib[m] += alpha[s[m]] @ ops.m2l_matrix(zero, TB[i]).T
                for i in range(len(uA)):
                    m = invA == i
                    contrib[m] += alpha[s[m]] @ ops.m2l_matrix(TA[i], zero).T
                np.add.at(beta, t, contrib)

    def cross_centre(self, layer, lev, iz):
        """z of a box's cross-layer expansion centre: its centre clamped to the
        layer's particle slab (zlo, zhi)."""
        h = self.tr.side / float(1 << lev)
        zc = self.tr.lo[2] + (iz + 0.5) * h
        zlo, zhi = self.zext[layer]
        return min(max(zc, zlo), zhi)

    def cross_image(self, lt, ls, direction, lev, izs, k3p):
        key = (lt, ls, direction, lev, izs, k3p)
        if key not in self.cross_images:
            zc = self.cross_centre(ls, lev, izs)
            wmin = xl.W_min(self.med, lt, direction, self.zext)
            A, Z, _ = xl.fit_cross(self.med, lt, ls, direction, zc, k3p, wmin, self.n_images)
            self.cross_images[key] = (A, Z)
        return self.cross_images[key]

    def _cross_tables(self, lt, ls, lev, keys):
        """T^{(k3')} of cross keys (dix, diy, izt, izs) at one level, shape
        (n_keys, p+1, n_{2p}): T^{(k3')}_g = sum over parts and images of
        A_j D^g h0(k_l R_j) / g! at (dix h, diy h, W(z_t) - W_min - Z_j).  The
        recurrence runs once over all (key, image) points of a (part, k3')."""
        tr, p = self.tr, self.p
        keys = np.asarray(keys, dtype=np.int64).reshape(-1, 4)
        h = tr.side / float(1 << lev)
        X0, Y0 = keys[:, 0] * h, keys[:, 1] * h
        zt = np.array([self.cross_centre(lt, lev, int(i)) for i in keys[:, 2]])
        mi2 = multi_indices(2 * p)
        odd3 = (-1.0) ** mi2[:, 2]
        T = np.zeros((len(keys), p + 1, len(mi2)), dtype=complex)
        k = self.med.k[lt]
        for direction in xl.directions(self.med, lt):
            wmin = xl.W_min(self.med, lt, direction, self.zext)
            W0 = xl.W_of(self.med, lt, direction, zt)
            sgn = 1.0 if direction == 'up' else odd3
            for k3p in range(p + 1):
                idx, A, Z = [], [], []
                for i, izs in enumerate(keys[:, 3]):
                    a, z = self.cross_image(lt, ls, direction, lev, int(izs), k3p)
                    idx.extend([i] * len(a))
                    A.extend(a)
                    Z.extend(z)
                idx, A, Z = np.array(idx, dtype=np.int64), np.array(A, complex), np.array(Z, complex)
                # slice k3' needs the derivatives of order <= 2p - k3' only
                P2 = 2 * p - k3p
                nP = n_coeffs(P2)
                sg = sgn if np.isscalar(sgn) else sgn[:nP]
                for c0 in range(0, len(idx), 2048):
                    sl = slice(c0, c0 + 2048)
                    tab = taylor_h0(X0[idx[sl]], Y0[idx[sl]], W0[idx[sl]] - wmin - Z[sl], k, P2)
                    vals = sg * (A[sl, None] * tab)
                    # the images of a key are consecutive: sum each key's run
                    ii = idx[sl]
                    starts = np.nonzero(np.r_[True, ii[1:] != ii[:-1]])[0]
                    T[ii[starts], k3p, :nP] += np.add.reduceat(vals, starts, axis=0)
        return T

    def _cross_m2l(self, lt, ls, V, alpha, beta, need):
        tr, ops = self.tr, self.ops
        gx, cx, k3p = ops.cross_maps()
        pairs = [(t, s) for t, lst in V.items() for s in lst if need is None or t in need]
        groups = {}
        for t, s in pairs:
            key = (int(tr.level[t]), int(tr.ix[t] - tr.ix[s]), int(tr.iy[t] - tr.iy[s]),
                   int(tr.iz[t]), int(tr.iz[s]))
            groups.setdefault(key, []).append((t, s))
        # images in the layer of the larger |k| (see the module docstring): a target
        # layer with the smaller |k| uses reciprocity, k_l^2 u_{l l'}(r; r') =
        # k_l'^2 u_{l' l}(r'; r), i.e. the transposed matrix of the mirror pair
        # (target box <-> source box) of component (l', l), times (k_l' / k_l)^2
        rev = abs(self.med.k[ls]) > abs(self.med.k[lt])
        by_level = {}
        for g in groups:
            by_level.setdefault(g[0], []).append(g)
        for lev, gl in by_level.items():
            if rev:
                Ts = self._cross_tables(ls, lt, lev, [(-dx, -dy, zs, zt) for (_, dx, dy, zt, zs) in gl])
            else:
                Ts = self._cross_tables(lt, ls, lev, [(dx, dy, zt, zs) for (_, dx, dy, zt, zs) in gl])
            for (_, dix, diy, izt, izs), T in zip(gl, Ts):
                lst = groups[(lev, dix, diy, izt, izs)]
                H = cx * T[k3p[None, :], gx]
                if rev:
                    H = (self.med.k[ls] / self.med.k[lt]) ** 2 * H.T
                t = np.array([a for a, _ in lst])
                s_ = np.array([b for _, b in lst])
                # moments about the source's cross-layer centre, M2L into locals
                # about the target's cross-layer centre, re-expanded at the box centre
                zs, zsc = tr.center(s_[0])[2], self.cross_centre(ls, lev, izs)
                zt, ztc = tr.center(t[0])[2], self.cross_centre(lt, lev, izt)
                a_sh = alpha[s_] @ ops.shift_matrix(np.array([0.0, 0.0, zs - zsc])).T
                loc = a_sh @ H.T
                np.add.at(beta, t, loc @ ops.shift_matrix(np.array([0.0, 0.0, zt - ztc])))

    # -- near field ----------------------------------------------------------
    def _kernel_same_layer(self, l, tpts, spts, far_thr=None):
        """free h0 (skip identical coordinates) + DCIM images, (nt, ns) matrix;
        with far_thr (a far-of-near pair) the images with -Re Z >= far_thr are
        left out (they went through M2L)."""
        k = self.med.k[l]
        dx = tpts[:, None, 0] - spts[None, :, 0]
        dy = tpts[:, None, 1] - spts[None, :, 1]
        dz = tpts[:, None, 2] - spts[None, :, 2]
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        same = (tpts[:, None, 0] == spts[None, :, 0]) & (tpts[:, None, 1] == spts[None, :, 1]) & \
            (tpts[:, None, 2] == spts[None, :, 2])
        with np.errstate(divide='ignore', invalid='ignore'):
            G = np.where(same, 0.0, np.exp(1j * k * r) / (1j * k * np.where(same, 1.0, r)))
        if self.images is not None and far_thr is None:
            G = G + self.images.reaction(l, tpts[:, None, 0], tpts[:, None, 1], tpts[:, None, 2],
                                         spts[None, :, 0], spts[None, :, 1], spts[None, :, 2])
        elif self.images is not None:
            rho2 = dx * dx + dy * dy
            for t in self.images.terms[l]:
                zeta = t['sz'] * tpts[:, None, 2] + t['szp'] * spts[None, :, 2] + t['c']
                for A, Z in zip(t['A'], t['Z']):
                    if -Z.real >= far_thr:
                        continue
                    w = zeta - t['zeta_min'] - Z
                    R = np.sqrt(rho2 + w * w)
                    G = G + A * np.exp(1j * k * R) / (1j * k * R)
        return G

    def evaluate(self, q, target_index=None):
        """Phi at all targets (input order), or at the given target indices."""
        tr, ops = self.tr, self.ops
        q = np.asarray(q, dtype=complex)
        alpha = self.upward(q)
        tp = self.tgt[tr.tperm]
        sp = self.src[tr.sperm]
        qs = q[tr.sperm]
        inv_t = np.empty_like(tr.tperm)
        inv_t[tr.tperm] = np.arange(len(tr.tperm))
        if target_index is None:
            want_sorted = np.arange(len(tp))
        else:
            want_sorted = inv_t[np.asarray(target_index)]
        # leaf of every sorted target
        leaf_of = np.full(len(tp), -1, dtype=np.int64)
        for n in range(tr.n_nodes):
            if tr.is_leaf[n] and tr.nt(n) > 0:
                leaf_of[tr.t0[n]:tr.t1[n]] = n
        leaves = np.unique(leaf_of[want_sorted])
        beta = self.downward(alpha, only_targets=None if target_index is None else leaves)
        phi_sorted = np.zeros(len(tp), dtype=complex)
        wanted = np.zeros(len(tp), dtype=bool)
        wanted[want_sorted] = True
        for t in leaves:
            a, b = tr.t0[t], tr.t1[t]
            idx = np.arange(a, b)[wanted[a:b]]
            pts = tp[idx]
            val = ops.l2p(beta[t], pts, tr.center(t))
            l = int(tr.layer[t])
            for (lt, ls), (_, P2P) in self.lists.items():
                if lt != l or t not in P2P:
                    continue
                for s in P2P[t]:
                    s0, s1 = tr.s0[s], tr.s1[s]
                    anc = fon_anchor(tr, t, s) if self.far_of_near else None
                    thr = fon_threshold(self.p, tr.side, anc[0]) if anc is not None else None
                    G = self._kernel_same_layer(l, pts, sp[s0:s1], far_thr=thr)
                    val = val + G @ qs[s0:s1]
            phi_sorted[idx] = val
        out = np.zeros(len(tp), dtype=complex)
        out[tr.tperm] = phi_sorted
        if target_index is None:
            return out
        return out[np.asarray(target_index)]
