// Morton keys, sort, per-layer octrees and interaction lists.
//
// Tree rule (the paper's adaptive tree, Algorithm 1, with the details it
// leaves open fixed as follows): one octree per layer inside one common root
// cube; integer coordinates i = min(floor(((x - lo)/side) * 2^20), 2^20 - 1)
// with correctly rounded double operations (no FMA); 60-bit Morton codes with
// the layer in bits 60..63; a box is split while max(#sources, #targets) >
// leaf_cap, or while a box of the same level in another layer's tree is
// adjacent to it (so that boxes of different layers never meet in a near-field
// list); only boxes that hold a point exist; nodes are numbered level-major,
// by (level, layer, Morton prefix).
//
// Lists: the dual-tree traversal of (target tree, source tree) that for a
// single tree is the classic adaptive U/V/W/X construction; V pairs go to M2L,
// U/W/X pairs to the near field.  Built level by level from per-node sets
//   C(t): same-level adjacent source boxes reached by the traversal,
//   D(t): coarser adjacent source leaves handed down to t,
//   X(t): source leaves not adjacent to t handed down from its parent,
//   V(t): children of C(parent) boxes that are not adjacent to t.

#include <string.h>

#include <algorithm>

#include "internal.cuh"
#include "ops_common.cuh"

namespace {

struct Geo {
    double d[TEFMM_MAX_LAYERS];
    double zlo[TEFMM_MAX_LAYERS], zhi[TEFMM_MAX_LAYERS];
    double lo[3];
    double side;
    int nL;
};

__device__ __forceinline__ unsigned long long ord_of(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}
__host__ __device__ __forceinline__ double double_of(unsigned long long o) {
    unsigned long long u = (o >> 63) ? (o & 0x7fffffffffffffffULL) : ~o;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}

__global__ void k_bbox(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, unsigned long long *bb) {
    unsigned long long mn[3] = {~0ULL, ~0ULL, ~0ULL}, mx[3] = {0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long o[3] = {ord_of(x[i]), ord_of(y[i]), ord_of(z[i])};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mn[d] = o[d] < mn[d] ? o[d] : mn[d];
            mx[d] = o[d] > mx[d] ? o[d] : mx[d];
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[d], off);
            unsigned long long b = __shfl_xor_sync(0xffffffffu, mx[d], off);
            mn[d] = a < mn[d] ? a : mn[d];
            mx[d] = b > mx[d] ? b : mx[d];
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bb[d], mn[d]);
            atomicMax(&bb[3 + d], mx[d]);
        }
    }
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0xfffffULL;   // 20 bits
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

__device__ __forceinline__ int icoord(double v, double lo, double side) {
    double t = __dsub_rn(v, lo);
    t = __ddiv_rn(t, side);
    t = __dmul_rn(t, 1048576.0);
    double f = floor(t);
    long long i = (long long)f;
    if (i < 0) i = 0;
    if (i > (1 << TEFMM_NBITS) - 1) i = (1 << TEFMM_NBITS) - 1;
    return (int)i;
}

__global__ void k_keys(int64_t nitems, int64_t ns, const double *__restrict__ sx,
                       const double *__restrict__ sy, const double *__restrict__ sz,
                       const double *__restrict__ tx, const double *__restrict__ ty,
                       const double *__restrict__ tz, Geo g, uint64_t *__restrict__ keys,
                       int *__restrict__ vals, int *flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    double x, y, z;
    if (i < ns) {
        x = sx[i]; y = sy[i]; z = sz[i];
    } else {
        x = tx[i - ns]; y = ty[i - ns]; z = tz[i - ns];
    }
    int lay = 0;
    bool on = false;
    for (int m = 0; m < g.nL - 1; ++m) {
        lay += (z < g.d[m]) ? 1 : 0;
        on |= (z == g.d[m]);
    }
    if (on) atomicOr(flags, FLAG_ON_INTERFACE);
    else if (z < g.zlo[lay] || z > g.zhi[lay]) atomicOr(flags, FLAG_OUT_OF_DOMAIN);
    uint64_t key = spread3(icoord(x, g.lo[0], g.side)) << 2 | spread3(icoord(y, g.lo[1], g.side)) << 1 |
                   spread3(icoord(z, g.lo[2], g.side));
    keys[i] = ((uint64_t)lay << 60) | key;
    vals[i] = (int)i;
}

// sorted items -> sorted source / target arrays and their counting scans
__global__ void k_is_src(int64_t nitems, int64_t ns, const int *__restrict__ vals,
                         int *__restrict__ is_src) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nitems) is_src[i] = vals[i] < ns ? 1 : 0;
}

__global__ void k_gather(int64_t nitems, int64_t ns, bool shared, const int *__restrict__ vals,
                         const int *__restrict__ cnt_s, const double *__restrict__ sx,
                         const double *__restrict__ sy, const double *__restrict__ sz,
                         const double *__restrict__ q, const double *__restrict__ tx,
                         const double *__restrict__ ty, const double *__restrict__ tz,
                         double *osx, double *osy, double *osz, double *oq, double *otx,
                         double *oty, double *otz, int *perm_s, int *perm_t) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    int v = vals[i];
    if (v < ns) {
        int64_t pos = shared ? i : cnt_s[i];
        osx[pos] = sx[v];
        osy[pos] = sy[v];
        osz[pos] = sz[v];
        if (q) {                      // no charges when only the geometry is built
            oq[2 * pos] = q[2 * v];
            oq[2 * pos + 1] = q[2 * v + 1];
        }
        perm_s[pos] = v;
    } else {
        int64_t pos = i - cnt_s[i];
        int w = (int)(v - ns);
        otx[pos] = tx[w];
        oty[pos] = ty[w];
        otz[pos] = tz[w];
        perm_t[pos] = w;
    }
}

__device__ __forceinline__ uint64_t prefix_at(uint64_t key, int l) {
    // layer bits and the Morton prefix of level l
    uint64_t lay = key >> 60;
    uint64_t m = key & 0x0fffffffffffffffULL;
    return (lay << 60) | (m >> (3 * (TEFMM_NBITS - l)));
}

__global__ void k_mark(int64_t nitems, int l, const uint64_t *__restrict__ keys,
                       const int *__restrict__ item_node, const int *__restrict__ n_i0,
                       const int *__restrict__ n_split, int *__restrict__ flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    int f = 0;
    if (l == 0) {
        f = (i == 0) || ((keys[i] >> 60) != (keys[i - 1] >> 60));
    } else {
        int pn = item_node[i];
        if (pn >= 0 && n_split[pn]) {
            f = (i == n_i0[pn]) || (prefix_at(keys[i], l) != prefix_at(keys[i - 1], l));
        }
    }
    flag[i] = f;
}

__global__ void k_make_nodes(int64_t nitems, int l, int off, const uint64_t *__restrict__ keys,
                             const int *__restrict__ flag, const int *__restrict__ scan,
                             int *__restrict__ item_node, int *n_layer, int *n_level, int *n_ix,
                             int *n_iy, int *n_iz, int *n_parent, int *n_i0, int *n_nchild,
                             int *n_cfirst, int *n_split) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    int pn = (l == 0) ? 0 : item_node[i];
    bool inside = (l == 0) || (pn >= 0 && n_split[pn]);
    if (!inside) {
        item_node[i] = -1;
        return;
    }
    int c = off + scan[i] - 1;     // inclusive scan
    if (flag[i]) {
        uint64_t key = keys[i];
        uint64_t m = key & 0x0fffffffffffffffULL;
        uint64_t pre = (l == 0) ? 0 : (m >> (3 * (TEFMM_NBITS - l)));
        int ix = 0, iy = 0, iz = 0;
        for (int b = 0; b < l; ++b) {
            iz |= (int)((pre >> (3 * b)) & 1) << b;
            iy |= (int)((pre >> (3 * b + 1)) & 1) << b;
            ix |= (int)((pre >> (3 * b + 2)) & 1) << b;
        }
        n_layer[c] = (int)(key >> 60);
        n_level[c] = l;
        n_ix[c] = ix;
        n_iy[c] = iy;
        n_iz[c] = iz;
        n_parent[c] = (l == 0) ? -1 : pn;
        n_i0[c] = (int)i;
        n_nchild[c] = 0;
        n_cfirst[c] = -1;
        n_split[c] = 0;
    }
    item_node[i] = c;
}

__global__ void k_node_ranges(int off, int cnt, int64_t nitems, int l, int leaf_cap, int max_level,
                              const int *__restrict__ n_i0, const int *__restrict__ n_parent,
                              const int *__restrict__ cnt_s, const int *__restrict__ cnt_t,
                              bool shared, int *n_i1, int *n_s0, int *n_s1, int *n_t0,
                              int *n_t1, int *n_split, int *n_cfirst, int *n_nchild,
                              int *nsplit_count) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    int c = off + j;
    int par = n_parent[c];
    int i1;
    if (j + 1 < cnt && n_parent[c + 1] == par) i1 = n_i0[c + 1];
    else i1 = (l == 0) ? (int)nitems : n_i1[par];
    int i0 = n_i0[c];
    n_i1[c] = i1;
    int s0, s1, t0, t1;
    if (shared) {
        s0 = t0 = i0;
        s1 = t1 = i1;
    } else {
        s0 = cnt_s[i0];
        s1 = cnt_s[i1];
        t0 = i0 - s0;
        t1 = i1 - s1;
    }
    n_s0[c] = s0;
    n_s1[c] = s1;
    n_t0[c] = t0;
    n_t1[c] = t1;
    int nmax = max(s1 - s0, t1 - t0);
    int sp = (nmax > leaf_cap && l < max_level) ? 1 : 0;
    n_split[c] = sp;
    if (sp) atomicAdd(nsplit_count, 1);
    if (par >= 0) {
        if (j == 0 || n_parent[c - 1] != par) n_cfirst[par] = c;
        atomicAdd(&n_nchild[par], 1);
    }
}

// Cross-layer split rule: a box that is not split by the leaf-size rule is
// still split while a box of another layer's tree at the same level is
// adjacent to it (and level < max_level).  Level nodes are ordered by
// (layer, prefix); n_key holds (layer << 60 | prefix) for a binary search.
__global__ void k_level_keys(int off, int cnt, int l, const int *__restrict__ n_i0,
                             const uint64_t *__restrict__ keys, uint64_t *__restrict__ nkey) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    nkey[j] = prefix_at(keys[n_i0[off + j]], l);
}

__device__ __forceinline__ bool find_key(const uint64_t *nkey, int cnt, uint64_t k) {
    int lo = 0, hi = cnt;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (nkey[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo < cnt && nkey[lo] == k;
}

__device__ __forceinline__ uint64_t morton3(int ix, int iy, int iz, int l) {
    uint64_t m = 0;
    for (int b = 0; b < l; ++b) {
        m |= (uint64_t)((ix >> b) & 1) << (3 * b + 2);
        m |= (uint64_t)((iy >> b) & 1) << (3 * b + 1);
        m |= (uint64_t)((iz >> b) & 1) << (3 * b);
    }
    return m;
}

__global__ void k_cross_split(int off, int cnt, int l, int nL, int max_level,
                              const uint64_t *__restrict__ nkey, const int *__restrict__ n_layer,
                              const int *__restrict__ n_ix, const int *__restrict__ n_iy,
                              const int *__restrict__ n_iz, int *n_split, int *nsplit_count) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt || l >= max_level) return;
    int c = off + j;
    if (n_split[c]) return;
    int lay = n_layer[c], ix = n_ix[c], iy = n_iy[c], iz = n_iz[c];
    int side = 1 << l;
    for (int ob = 0; ob < nL; ++ob) {
        if (ob == lay) continue;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    int x = ix + dx, y = iy + dy, z = iz + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) continue;
                    uint64_t k = ((uint64_t)ob << 60) | morton3(x, y, z, l);
                    if (find_key(nkey, cnt, k)) {
                        n_split[c] = 1;
                        atomicAdd(nsplit_count, 1);
                        return;
                    }
                }
    }
}

// ---------------------------------------------------------------- lists
struct NodeView {
    const int *layer, *level, *ix, *iy, *iz, *parent, *cfirst, *nchild, *s0, *s1, *t0, *t1, *split;
};

// Per-level rows of the C (colleague) and V (M2L) work lists: node t of level l
// owns cap[l] entries at base[l] + (t - off[l]) * cap[l].  Coarse levels of the
// wavenumber rule pair every split box of a level, so their rows (and the V rows
// of the level below) are as wide as the level; the others stay neighbourhood-sized.
struct ListLayout {
    int off[TEFMM_NBITS + 2];
    int ccap[TEFMM_NBITS + 1], vcap[TEFMM_NBITS + 1];
    long long cbase[TEFMM_NBITS + 1], vbase[TEFMM_NBITS + 1];
};
__device__ __forceinline__ long long c_row(const ListLayout &Ly, int l, int t) {
    return Ly.cbase[l] + (long long)(t - Ly.off[l]) * Ly.ccap[l];
}
__device__ __forceinline__ long long v_row(const ListLayout &Ly, int l, int t) {
    return Ly.vbase[l] + (long long)(t - Ly.off[l]) * Ly.vcap[l];
}

__device__ __forceinline__ bool adjacent(const NodeView &N, int a, int b) {
    int la = N.level[a], lb = N.level[b];
    int ax = N.ix[a], ay = N.iy[a], az = N.iz[a];
    int bx = N.ix[b], by = N.iy[b], bz = N.iz[b];
    if (la > lb) {
        int t;
        t = la; la = lb; lb = t;
        t = ax; ax = bx; bx = t;
        t = ay; ay = by; by = t;
        t = az; az = bz; bz = t;
    }
    int s = lb - la;
    int lo, hi;
    lo = ax << s; hi = ((ax + 1) << s) - 1;
    if (bx < lo - 1 || bx > hi + 1) return false;
    lo = ay << s; hi = ((ay + 1) << s) - 1;
    if (by < lo - 1 || by > hi + 1) return false;
    lo = az << s; hi = ((az + 1) << s) - 1;
    if (bz < lo - 1 || bz > hi + 1) return false;
    return true;
}

__device__ __forceinline__ void isort(int *a, int n) {
    for (int i = 1; i < n; ++i) {
        int v = a[i], j = i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

// level 0: C(root_t) = every root that holds sources
__global__ void k_lists_root(int nroots, NodeView N, ListLayout Ly, int *C_list, int *C_cnt, int *D_cnt,
                             int *X_cnt, int *V_cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nroots) return;
    int n = 0;
    if (N.t1[t] > N.t0[t]) {
        for (int s = 0; s < nroots; ++s)
            if (N.s1[s] > N.s0[s]) C_list[c_row(Ly, 0, t) + n++] = s;
    }
    C_cnt[t] = n;
    D_cnt[t] = 0;
    X_cnt[t] = 0;
    V_cnt[t] = 0;
}

// Cross-layer admissibility: at a level whose box size exceeds HX (coarse != 0),
// two split boxes of different layers stacked within one box horizontally are
// paired like adjacent boxes (their children are paired) instead of translated.
__device__ __forceinline__ bool cross_colleague(const NodeView &N, int t, int c, int coarse) {
    if (!coarse || N.layer[t] == N.layer[c] || !N.split[t] || !N.split[c]) return false;
    return abs(N.ix[t] - N.ix[c]) <= 1 && abs(N.iy[t] - N.iy[c]) <= 1;
}

// Wavenumber admissibility: on a level whose Taylor expansions would span
// k_max h > kh_max (kcoarse != 0), two split boxes are not translated; their
// children are paired instead, whatever their distance.
__device__ __forceinline__ bool coarse_colleague(const NodeView &N, int t, int c, int kcoarse) {
    return kcoarse && N.split[t] && N.split[c];
}

__global__ void k_lists_level(int off, int cnt, int l, NodeView N, ListLayout Ly, int *C_list, int *C_cnt,
                              int *D_list, int *D_cnt, int capD, int *X_list, int *X_cnt, int capX,
                              int *V_list, int *V_cnt, int *flags, int coarse, int kcoarse) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    int t = off + j;
    int nc = 0, nd = 0, nx = 0, nv = 0;
    if (N.t1[t] > N.t0[t]) {
        const int capC = Ly.ccap[l], capV = Ly.vcap[l];
        int P = N.parent[t];
        int *Cl = C_list + c_row(Ly, l, t);
        int *Dl = D_list + (int64_t)t * capD;
        int *Xl = X_list + (int64_t)t * capX;
        int *Vl = V_list + v_row(Ly, l, t);
        bool ovf = false;
        const int *CP = C_list + c_row(Ly, l - 1, P);
        for (int a = 0; a < C_cnt[P]; ++a) {
            int s = CP[a];
            if (N.split[s]) {
                int c0 = N.cfirst[s], c1 = c0 + N.nchild[s];
                for (int c = c0; c < c1; ++c) {
                    if (N.s1[c] <= N.s0[c]) continue;
                    if (adjacent(N, t, c) || cross_colleague(N, t, c, coarse) ||
                        coarse_colleague(N, t, c, kcoarse)) {
                        if (nc < capC) Cl[nc++] = c; else ovf = true;
                    } else {
                        if (nv < capV) Vl[nv++] = c; else ovf = true;
                    }
                }
            } else {
                if (adjacent(N, t, s)) {
                    if (nd < capD) Dl[nd++] = s; else ovf = true;
                } else {
                    if (nx < capX) Xl[nx++] = s; else ovf = true;
                }
            }
        }
        const int *DP = D_list + (int64_t)P * capD;
        for (int a = 0; a < D_cnt[P]; ++a) {
            int s = DP[a];
            if (adjacent(N, t, s)) {
                if (nd < capD) Dl[nd++] = s; else ovf = true;
            } else {
                if (nx < capX) Xl[nx++] = s; else ovf = true;
            }
        }
        isort(Dl, nd);
        isort(Xl, nx);
        if (ovf) atomicOr(flags, FLAG_LIST_OVERFLOW);
    }
    C_cnt[t] = nc;
    D_cnt[t] = nd;
    X_cnt[t] = nx;
    V_cnt[t] = nv;
}

// near-field list of a target leaf: U (leaves of C(t), D(t), the adjacent
// leaves found below the non-leaf boxes of C(t)), W (non-adjacent boxes found
// there) and X of t and of every ancestor.  Two passes: with out == nullptr
// only the count is written; otherwise the list is written at out[ptr[t]..]
// and sorted.
__global__ void k_near(int off, int cnt, int l, NodeView N, ListLayout Ly, const int *C_list, const int *C_cnt,
                       const int *D_list, const int *D_cnt, int capD, const int *X_list,
                       const int *X_cnt, int capX, const int *ptr, int *out, int *near_cnt,
                       int *flags) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    int t = off + j;
    int n = 0;
    if (N.t1[t] > N.t0[t] && !N.split[t]) {
        int *L = out ? out + ptr[t] : nullptr;
        bool ovf = false;
        int stack[160];
        int sp = 0;
        const int *Cl = C_list + c_row(Ly, l, t);
        for (int a = 0; a < C_cnt[t]; ++a) {
            int s = Cl[a];
            if (!N.split[s]) {
                if (L) L[n] = s;
                ++n;
            } else {
                if (sp < 160) stack[sp++] = s; else ovf = true;
                while (sp > 0) {
                    int u = stack[--sp];
                    int c0 = N.cfirst[u], c1 = c0 + N.nchild[u];
                    for (int c = c0; c < c1; ++c) {
                        if (N.s1[c] <= N.s0[c]) continue;
                        if (adjacent(N, t, c) && N.split[c]) {
                            if (sp < 160) stack[sp++] = c; else ovf = true;
                        } else {
                            if (L) L[n] = c;
                            ++n;
                        }
                    }
                }
            }
        }
        const int *Dl = D_list + (int64_t)t * capD;
        for (int a = 0; a < D_cnt[t]; ++a) {
            if (L) L[n] = Dl[a];
            ++n;
        }
        for (int a = t; a >= 0; a = N.parent[a]) {
            const int *Xl = X_list + (int64_t)a * capX;
            for (int b = 0; b < X_cnt[a]; ++b) {
                if (L) L[n] = Xl[b];
                ++n;
            }
        }
        if (L) isort(L, n);
        if (ovf) atomicOr(flags, FLAG_LIST_OVERFLOW);
    }
    if (!out) near_cnt[t] = n;
}

__global__ void k_csr_fill(int off, int cnt, int l, ListLayout Ly, const int *__restrict__ vcnt,
                           const int *__restrict__ tmp, const int *__restrict__ ptr,
                           int *__restrict__ out, int *__restrict__ out_t) {
    int j = blockIdx.x;
    if (j >= cnt) return;
    int t = off + j;
    int c = vcnt[t], base = ptr[t];
    const int *row = tmp + v_row(Ly, l, t);
    for (int a = threadIdx.x; a < c; a += blockDim.x) {
        out[base + a] = row[a];
        out_t[base + a] = t;
    }
}

// near-field particle pairs: out[0] in all, out[1 + l] with targets in layer l
__global__ void k_count_pairs(int n_nodes, const int *__restrict__ near_ptr,
                              const int *__restrict__ near_src, const int *__restrict__ s0,
                              const int *__restrict__ s1, const int *__restrict__ t0,
                              const int *__restrict__ t1, const int *__restrict__ layer,
                              unsigned long long *out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    unsigned long long acc = 0;
    int nt = t1[t] - t0[t];
    for (int a = near_ptr[t]; a < near_ptr[t + 1]; ++a) {
        int s = near_src[a];
        acc += (unsigned long long)nt * (unsigned long long)(s1[s] - s0[s]);
    }
    if (acc) {
        atomicAdd(out, acc);
        atomicAdd(out + 1 + (layer[t] & 7), acc);
    }
}

// Far-of-near anchors.  For the near-list entry (target box t, source box s)
// let l* be the coarser of their levels and T*, S* the boxes of level l* that
// hold them.  When T* and S* are adjacent, the far images (-Re Z >= thr[l*])
// of every particle pair under (T*, S*) go through one M2L from S* to T* (all
// those pairs are near-list pairs with the same anchor: one of T*, S* is t or
// s itself, a leaf, so no V pair covers them), and the entry's pair sum leaves
// them out.  Per entry: fl = l* (or -1: not adjacent, all images in P2P) and
// the anchor key (T* << 32 | S*, or ~0 for none).
__global__ void k_fon_anchor(int n_nodes, const int *__restrict__ level, const int *__restrict__ parent,
                             const int *__restrict__ ix, const int *__restrict__ iy, const int *__restrict__ iz,
                             const int *__restrict__ ptr, const int *__restrict__ src,
                             int *__restrict__ fl, unsigned long long *__restrict__ akey) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    for (int a = ptr[t]; a < ptr[t + 1]; ++a) {
        const int s = src[a];
        const int ls = min(level[t], level[s]);
        int T = t, S = s;
        for (int guard = 0; level[T] > ls && guard < 32; ++guard) T = parent[T];
        for (int guard = 0; level[S] > ls && guard < 32; ++guard) S = parent[S];
        const bool adj = level[T] == ls && level[S] == ls && abs(ix[T] - ix[S]) <= 1 &&
                         abs(iy[T] - iy[S]) <= 1 && abs(iz[T] - iz[S]) <= 1;
        fl[a] = adj ? ls : -1;
        akey[a] = adj ? (((unsigned long long)(unsigned)T << 32) | (unsigned)S) : ~0ULL;
    }
}

// unique anchors of the sorted keys -> (pair_t, pair_s) after the V pairs
__global__ void k_fon_heads(int64_t n, const unsigned long long *__restrict__ k, int *__restrict__ head) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    head[i] = k[i] != ~0ULL && (i == 0 || k[i] != k[i - 1]);
}
__global__ void k_fon_fill(int64_t n, const unsigned long long *__restrict__ k, const int *__restrict__ head,
                           const int *__restrict__ pos, int64_t base, int *__restrict__ pair_t,
                           int *__restrict__ pair_s) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !head[i]) return;
    const int64_t o = base + pos[i];
    pair_t[o] = (int)(k[i] >> 32);
    pair_s[o] = (int)(k[i] & 0xffffffffULL);
}

// Image terms the near-field kernels evaluate: per entry, its particle pairs
// times the images of the target layer's terms that are near at the entry's
// far-of-near level (all images when it has none).  c[l][lv] = that image
// count for layer l at level lv, c[l][NBITS + 1] = all of the layer's images.
struct NearImgCount {
    int c[TEFMM_MAX_LAYERS][TEFMM_NBITS + 2];
};
__global__ void k_near_img_terms(int n_nodes, const int *__restrict__ layer, const int *__restrict__ t0,
                                 const int *__restrict__ t1, const int *__restrict__ s0,
                                 const int *__restrict__ s1, const int *__restrict__ ptr,
                                 const int *__restrict__ src, const int *__restrict__ fl, NearImgCount nc,
                                 unsigned long long *out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    const unsigned long long nt = (unsigned long long)(t1[t] - t0[t]);
    const int l = layer[t] & 7;
    unsigned long long acc = 0;
    for (int a = ptr[t]; a < ptr[t + 1]; ++a) {
        const int lv = fl ? fl[a] : -1;
        const int nimg = nc.c[l][lv >= 0 ? lv : TEFMM_NBITS + 1];
        acc += nt * (unsigned long long)(s1[src[a]] - s0[src[a]]) * (unsigned long long)nimg;
    }
    if (acc) atomicAdd(out, acc);
}

// Near-field work items: the near sources of a target leaf, taken in list
// order, are cut into chunks of NEAR_CHUNK; each chunk is one CTA of the
// near-field kernels, so that a leaf beside a dense region (W-type entries of
// 10^5 sources) is spread over many CTAs instead of one.
__global__ void k_near_items_count(int n_nodes, const int *__restrict__ split, const int *__restrict__ t0,
                                   const int *__restrict__ t1, const int *__restrict__ s0,
                                   const int *__restrict__ s1, const int *__restrict__ ptr,
                                   const int *__restrict__ src, int *__restrict__ cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    int parts = 0;
    if (!split[t] && t1[t] > t0[t]) {
        int64_t ns = 0;
        for (int a = ptr[t]; a < ptr[t + 1]; ++a) ns += s1[src[a]] - s0[src[a]];
        parts = (int)max((int64_t)1, (ns + NEAR_CHUNK - 1) / NEAR_CHUNK);
    }
    cnt[t] = parts;
}
__global__ void k_near_items_fill(int n_nodes, const int *__restrict__ cnt, const int *__restrict__ pos,
                                  int *__restrict__ item_node, int *__restrict__ item_part,
                                  int *__restrict__ item_np) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    const int n = cnt[t], o = pos[t];
    for (int j = 0; j < n; ++j) {
        item_node[o + j] = t;
        item_part[o + j] = j;
        item_np[o + j] = n;
    }
}

__global__ void k_layer_mismatch(int n_nodes, const int *__restrict__ layer,
                                 const int *__restrict__ ptr, const int *__restrict__ src,
                                 int *flags) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    for (int a = ptr[t]; a < ptr[t + 1]; ++a)
        if (layer[src[a]] != layer[t]) {
            atomicOr(flags, FLAG_CROSS_LAYER);
            return;
        }
}

int scan_excl(tefmm_plan_s *P, const int *in, int *out, int64_t n, cudaStream_t st) {
    return dev_scan_i32(P, in, out, n, false, st);
}
int scan_incl(tefmm_plan_s *P, const int *in, int *out, int64_t n, cudaStream_t st) {
    return dev_scan_i32(P, in, out, n, true, st);
}

// grow node arrays keeping their contents
int grow_nodes(tefmm_plan_s *P, int64_t need, int64_t have, cudaStream_t st) {
    DBuf *arrs[] = {&P->n_layer, &P->n_level, &P->n_ix, &P->n_iy, &P->n_iz, &P->n_parent,
                    &P->n_cfirst, &P->n_nchild, &P->n_s0, &P->n_s1, &P->n_t0, &P->n_t1,
                    &P->n_i0, &P->n_i1, &P->n_split};
    for (DBuf *b : arrs) {
        if (b->cap >= (size_t)need * sizeof(int)) continue;
        size_t ncap = (size_t)(need * 2) * sizeof(int);
        void *np_ = nullptr;
        if (inject_alloc_failure()) return TEFMM_ERR_OOM;
        CUDA_TRY(cudaMalloc(&np_, ncap));
        if (have > 0 && b->p) CUDA_TRY(cudaMemcpyAsync(np_, b->p, have * sizeof(int), cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (b->p) cudaFree(b->p);
        b->p = np_;
        b->cap = ncap;
    }
    return TEFMM_OK;
}

NodeView node_view(tefmm_plan_s *P) {
    NodeView N;
    N.layer = dp<int>(P->n_layer);
    N.level = dp<int>(P->n_level);
    N.ix = dp<int>(P->n_ix);
    N.iy = dp<int>(P->n_iy);
    N.iz = dp<int>(P->n_iz);
    N.parent = dp<int>(P->n_parent);
    N.cfirst = dp<int>(P->n_cfirst);
    N.nchild = dp<int>(P->n_nchild);
    N.s0 = dp<int>(P->n_s0);
    N.s1 = dp<int>(P->n_s1);
    N.t0 = dp<int>(P->n_t0);
    N.t1 = dp<int>(P->n_t1);
    N.split = dp<int>(P->n_split);
    return N;
}

}  // namespace

int check_flags(tefmm_plan_s *P, cudaStream_t st) {
    int f = 0;
    CUDA_TRY(cudaMemcpyAsync(&f, P->flags.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (f & FLAG_ON_INTERFACE) return TEFMM_ERR_POINT_ON_INTERFACE;
    if (f & FLAG_OUT_OF_DOMAIN) return TEFMM_ERR_OUT_OF_DOMAIN;
    if (f & FLAG_LIST_OVERFLOW) return TEFMM_ERR_LIST_OVERFLOW;
    if (f & FLAG_CROSS_LAYER) return TEFMM_ERR_NOT_IMPLEMENTED;
    if (f & FLAG_TIMEOUT) return TEFMM_ERR_TIMEOUT;
    if (f & FLAG_CHECK) return TEFMM_ERR_DEVICE_CHECK;
    return TEFMM_OK;
}

int tree_build(tefmm_plan_s *P, const double *sx, const double *sy, const double *sz,
               const double *q, const double *tx, const double *ty, const double *tz,
               cudaStream_t st) {
    const int64_t ns = P->ns, nt = P->nt;
    const bool shared = P->shared_pts;
    const int64_t nitems = shared ? ns : ns + nt;
    P->nitems = nitems;
    TRY(dbuf_ensure(P->flags, 64));
    CUDA_TRY(cudaMemsetAsync(P->flags.p, 0, 64, st));

    // bounding box of all points
    TRY(dbuf_ensure(P->bbox, 6 * sizeof(unsigned long long)));
    unsigned long long init[6] = {~0ULL, ~0ULL, ~0ULL, 0, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(P->bbox.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
    k_bbox<<<grid_for(ns, 256) > 1024 ? 1024 : grid_for(ns, 256), 256, 0, st>>>(
        ns, sx, sy, sz, dp<unsigned long long>(P->bbox));
    P->launches++;
    if (!shared) {
        k_bbox<<<grid_for(nt, 256) > 1024 ? 1024 : grid_for(nt, 256), 256, 0, st>>>(
            nt, tx, ty, tz, dp<unsigned long long>(P->bbox));
        P->launches++;
    }
    unsigned long long bb[6];
    CUDA_TRY(cudaMemcpyAsync(bb, P->bbox.p, sizeof(bb), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = double_of(bb[d]);
        hi[d] = double_of(bb[3 + d]);
    }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = hi[d] - lo[d];
        if (e > side) side = e;
    }
    if (side == 0.0) side = 1.0;
    for (int d = 0; d < 3; ++d) P->lo[d] = lo[d];
    P->side = side;

    Geo g;
    for (int m = 0; m < TEFMM_MAX_LAYERS; ++m) {
        g.d[m] = m < P->nL - 1 ? P->d[m] : 0.0;
        g.zlo[m] = P->opt.zext[2 * m];
        g.zhi[m] = P->opt.zext[2 * m + 1];
    }
    for (int d = 0; d < 3; ++d) g.lo[d] = lo[d];
    g.side = side;
    g.nL = P->nL;

    // keys and stable sort (layer, Morton key, input index)
    TRY(dbuf_ensure(P->keys_in, nitems * 8));
    TRY(dbuf_ensure(P->keys_out, nitems * 8));
    TRY(dbuf_ensure(P->vals_in, nitems * 4));
    TRY(dbuf_ensure(P->vals_out, nitems * 4));
    k_keys<<<grid_for(nitems, 256), 256, 0, st>>>(nitems, ns, sx, sy, sz, tx, ty, tz, g,
                                                  dp<uint64_t>(P->keys_in), dp<int>(P->vals_in),
                                                  dp<int>(P->flags));
    P->launches++;
    TRY(dev_sort_u64(P, dp<uint64_t>(P->keys_in), dp<uint64_t>(P->keys_out), dp<int>(P->vals_in),
                     dp<int>(P->vals_out), nitems, st));
    const uint64_t *keys = dp<uint64_t>(P->keys_out);

    // counting scans and sorted particle arrays
    TRY(dbuf_ensure(P->cnt_s, (nitems + 1) * 4));
    TRY(dbuf_ensure(P->item_flag, (nitems + 1) * 4));
    if (!shared) {
        CUDA_TRY(cudaMemsetAsync(P->item_flag.p, 0, (nitems + 1) * 4, st));
        k_is_src<<<grid_for(nitems, 256), 256, 0, st>>>(nitems, ns, dp<int>(P->vals_out),
                                                        dp<int>(P->item_flag));
        P->launches++;
        TRY(scan_excl(P, dp<int>(P->item_flag), dp<int>(P->cnt_s), nitems + 1, st));
    }
    TRY(dbuf_ensure(P->sx, ns * 8));
    TRY(dbuf_ensure(P->sy, ns * 8));
    TRY(dbuf_ensure(P->sz, ns * 8));
    TRY(dbuf_ensure(P->sq, ns * 16));
    TRY(dbuf_ensure(P->perm_s, ns * 4 + 4));
    if (!shared) {
        TRY(dbuf_ensure(P->tx, nt * 8));
        TRY(dbuf_ensure(P->ty, nt * 8));
        TRY(dbuf_ensure(P->tz, nt * 8));
        TRY(dbuf_ensure(P->perm_t, nt * 4 + 4));
    }
    k_gather<<<grid_for(nitems, 256), 256, 0, st>>>(
        nitems, ns, shared, dp<int>(P->vals_out), dp<int>(P->cnt_s), sx, sy, sz, q, tx, ty, tz,
        dp<double>(P->sx), dp<double>(P->sy), dp<double>(P->sz), dp<double>(P->sq),
        shared ? nullptr : dp<double>(P->tx), shared ? nullptr : dp<double>(P->ty),
        shared ? nullptr : dp<double>(P->tz), dp<int>(P->perm_s),
        shared ? nullptr : dp<int>(P->perm_t));
    P->launches++;

    // level-by-level octree
    TRY(dbuf_ensure(P->item_node, nitems * 4));
    TRY(dbuf_ensure(P->item_scan, nitems * 4));
    TRY(dbuf_ensure(P->counters, 64));
    P->level_off.clear();
    P->level_off.push_back(0);
    int64_t total = 0;
    int max_level = P->opt.max_level;
    for (int l = 0; l <= max_level; ++l) {
        k_mark<<<grid_for(nitems, 256), 256, 0, st>>>(nitems, l, keys, dp<int>(P->item_node),
                                                      dp<int>(P->n_i0), dp<int>(P->n_split),
                                                      dp<int>(P->item_flag));
        P->launches++;
        TRY(scan_incl(P, dp<int>(P->item_flag), dp<int>(P->item_scan), nitems, st));
        int cnt = 0;
        CUDA_TRY(cudaMemcpyAsync(&cnt, dp<int>(P->item_scan) + nitems - 1, 4,
                                 cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (cnt == 0) break;
        TRY(grow_nodes(P, total + cnt, total, st));
        k_make_nodes<<<grid_for(nitems, 256), 256, 0, st>>>(
            nitems, l, (int)total, keys, dp<int>(P->item_flag), dp<int>(P->item_scan),
            dp<int>(P->item_node), dp<int>(P->n_layer), dp<int>(P->n_level), dp<int>(P->n_ix),
            dp<int>(P->n_iy), dp<int>(P->n_iz), dp<int>(P->n_parent), dp<int>(P->n_i0),
            dp<int>(P->n_nchild), dp<int>(P->n_cfirst), dp<int>(P->n_split));
        P->launches++;
        CUDA_TRY(cudaMemsetAsync(P->counters.p, 0, 4, st));
        k_node_ranges<<<grid_for(cnt, 256), 256, 0, st>>>(
            (int)total, cnt, nitems, l, P->leaf_cap_eff, max_level, dp<int>(P->n_i0),
            dp<int>(P->n_parent), dp<int>(P->cnt_s), nullptr, shared, dp<int>(P->n_i1),
            dp<int>(P->n_s0), dp<int>(P->n_s1), dp<int>(P->n_t0), dp<int>(P->n_t1),
            dp<int>(P->n_split), dp<int>(P->n_cfirst), dp<int>(P->n_nchild),
            dp<int>(P->counters));
        P->launches++;
        if (P->nL > 1) {
            TRY(dbuf_ensure(P->n_key, (size_t)cnt * 8));
            k_level_keys<<<grid_for(cnt, 256), 256, 0, st>>>((int)total, cnt, l, dp<int>(P->n_i0), keys,
                                                             dp<uint64_t>(P->n_key));
            P->launches++;
            k_cross_split<<<grid_for(cnt, 128), 128, 0, st>>>(
                (int)total, cnt, l, P->nL, max_level, dp<uint64_t>(P->n_key), dp<int>(P->n_layer),
                dp<int>(P->n_ix), dp<int>(P->n_iy), dp<int>(P->n_iz), dp<int>(P->n_split),
                dp<int>(P->counters));
            P->launches++;
        }
        int nsplit = 0;
        CUDA_TRY(cudaMemcpyAsync(&nsplit, P->counters.p, 4, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        total += cnt;
        P->level_off.push_back((int)total);
        if (nsplit == 0) break;
    }
    P->n_nodes = (int)total;
    P->n_levels = (int)P->level_off.size() - 1;
    return TEFMM_OK;
}

// level l is coarse for the wavenumber rule when k_max h_l > kh_max (kh_max > 0)
static bool kh_coarse(const tefmm_plan_s *P, int l) {
    return P->opt.kh_max > 0.0 && P->kmax * (P->side / (double)(1 << l)) > P->opt.kh_max;
}

int lists_build(tefmm_plan_s *P, cudaStream_t st) {
    const int nn = P->n_nodes;
    const int NL = P->n_levels;
    // stacked cross-layer colleagues (at most 128 per other layer) and their
    // children in the V lists; overflow is reported (LIST_OVERFLOW)
    const bool xrule = P->nL > 1 && P->HX < INFINITY;
    const int capC_near = 27 * P->nL + (xrule ? 128 * (P->nL - 1) : 0);
    P->cap_D = 128;
    P->cap_X = 27 * P->nL + 128;
    ListLayout Ly;
    memset(&Ly, 0, sizeof(Ly));
    long long ctot = 0, vtot = 0;
    for (int l = 0; l <= NL; ++l) Ly.off[l] = P->level_off[l];
    for (int l = 0; l < NL; ++l) {
        const int cnt = P->level_off[l + 1] - P->level_off[l];
        Ly.ccap[l] = (l == 0 || kh_coarse(P, l)) ? cnt : std::min(cnt, capC_near);
        Ly.vcap[l] = l == 0 ? 0 : std::min(cnt, 8 * Ly.ccap[l - 1]);
        Ly.cbase[l] = ctot;
        Ly.vbase[l] = vtot;
        ctot += (long long)cnt * Ly.ccap[l];
        vtot += (long long)cnt * Ly.vcap[l];
    }
    TRY(dbuf_ensure(P->C_list, (size_t)ctot * 4));
    TRY(dbuf_ensure(P->C_cnt, (size_t)nn * 4));
    TRY(dbuf_ensure(P->D_list, (size_t)nn * P->cap_D * 4));
    TRY(dbuf_ensure(P->D_cnt, (size_t)nn * 4));
    TRY(dbuf_ensure(P->X_list, (size_t)nn * P->cap_X * 4));
    TRY(dbuf_ensure(P->X_cnt, (size_t)nn * 4));
    TRY(dbuf_ensure(P->V_tmp, (size_t)vtot * 4));
    TRY(dbuf_ensure(P->V_cnt, (size_t)(nn + 1) * 4));
    TRY(dbuf_ensure(P->near_cnt, (size_t)(nn + 1) * 4));
    CUDA_TRY(cudaMemsetAsync(P->V_cnt.p, 0, (size_t)(nn + 1) * 4, st));
    CUDA_TRY(cudaMemsetAsync(P->near_cnt.p, 0, (size_t)(nn + 1) * 4, st));
    // the first translating level below a coarse level l pairs boxes up to
    // 2^(l+1) - 1 apart; the M2L keys hold offsets up to 15
    for (int l = 1; l + 1 < NL; ++l)
        if (kh_coarse(P, l) && (1 << (l + 1)) - 1 > 15) return TEFMM_ERR_NOT_IMPLEMENTED;
    NodeView N = node_view(P);
    int nroots = P->level_off[1];
    k_lists_root<<<1, 32, 0, st>>>(nroots, N, Ly, dp<int>(P->C_list), dp<int>(P->C_cnt), dp<int>(P->D_cnt),
                                   dp<int>(P->X_cnt), dp<int>(P->V_cnt));
    P->launches++;
    for (int l = 1; l < NL; ++l) {
        int off = P->level_off[l], cnt = P->level_off[l + 1] - off;
        k_lists_level<<<grid_for(cnt, 128), 128, 0, st>>>(
            off, cnt, l, N, Ly, dp<int>(P->C_list), dp<int>(P->C_cnt), dp<int>(P->D_list),
            dp<int>(P->D_cnt), P->cap_D, dp<int>(P->X_list), dp<int>(P->X_cnt), P->cap_X,
            dp<int>(P->V_tmp), dp<int>(P->V_cnt), dp<int>(P->flags),
            (P->nL > 1 && P->side / (double)(1 << l) > P->HX) ? 1 : 0, kh_coarse(P, l) ? 1 : 0);
        P->launches++;
    }
    for (int l = 0; l < NL; ++l) {
        int off = P->level_off[l], cnt = P->level_off[l + 1] - off;
        k_near<<<grid_for(cnt, 64), 64, 0, st>>>(
            off, cnt, l, N, Ly, dp<int>(P->C_list), dp<int>(P->C_cnt), dp<int>(P->D_list),
            dp<int>(P->D_cnt), P->cap_D, dp<int>(P->X_list), dp<int>(P->X_cnt), P->cap_X, nullptr,
            nullptr, dp<int>(P->near_cnt), dp<int>(P->flags));
        P->launches++;
    }
    // CSR
    TRY(dbuf_ensure(P->v_ptr, (size_t)(nn + 1) * 4));
    TRY(dbuf_ensure(P->near_ptr, (size_t)(nn + 1) * 4));
    TRY(scan_excl(P, dp<int>(P->V_cnt), dp<int>(P->v_ptr), nn + 1, st));
    TRY(scan_excl(P, dp<int>(P->near_cnt), dp<int>(P->near_ptr), nn + 1, st));
    int tot[2];
    CUDA_TRY(cudaMemcpyAsync(&tot[0], dp<int>(P->v_ptr) + nn, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&tot[1], dp<int>(P->near_ptr) + nn, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    P->n_v = tot[0];
    P->n_near = tot[1];
    // V pairs, then (at most one per near entry) the far-of-near pairs
    TRY(dbuf_ensure(P->v_src, (size_t)(P->n_v + P->n_near + 1) * 4));
    TRY(dbuf_ensure(P->pair_t, (size_t)(P->n_v + P->n_near + 1) * 4));
    TRY(dbuf_ensure(P->near_src, (size_t)(P->n_near + 1) * 4));
    for (int l = 0; l < NL; ++l) {
        int off = P->level_off[l], cnt = P->level_off[l + 1] - off;
        k_near<<<grid_for(cnt, 64), 64, 0, st>>>(
            off, cnt, l, N, Ly, dp<int>(P->C_list), dp<int>(P->C_cnt), dp<int>(P->D_list),
            dp<int>(P->D_cnt), P->cap_D, dp<int>(P->X_list), dp<int>(P->X_cnt), P->cap_X,
            dp<int>(P->near_ptr), dp<int>(P->near_src), nullptr, dp<int>(P->flags));
        P->launches++;
    }
    for (int l = 1; l < NL; ++l) {
        int off = P->level_off[l], cnt = P->level_off[l + 1] - off;
        if (cnt == 0) continue;
        k_csr_fill<<<cnt, 64, 0, st>>>(off, cnt, l, Ly, dp<int>(P->V_cnt), dp<int>(P->V_tmp),
                                       dp<int>(P->v_ptr), dp<int>(P->v_src), dp<int>(P->pair_t));
        P->launches++;
    }
    if (nn > 0) {
        k_layer_mismatch<<<grid_for(nn, 128), 128, 0, st>>>(nn, dp<int>(P->n_layer),
                                                            dp<int>(P->near_ptr),
                                                            dp<int>(P->near_src), dp<int>(P->flags));
        P->launches++;
    }
    TRY(dbuf_ensure(P->counters, 128));
    CUDA_TRY(cudaMemsetAsync(P->counters.p, 0, 72, st));
    if (nn > 0) {
        k_count_pairs<<<grid_for(nn, 128), 128, 0, st>>>(
            nn, dp<int>(P->near_ptr), dp<int>(P->near_src), dp<int>(P->n_s0), dp<int>(P->n_s1),
            dp<int>(P->n_t0), dp<int>(P->n_t1), dp<int>(P->n_layer), dp<unsigned long long>(P->counters));
        P->launches++;
    }
    P->n_fon = 0;
    if (P->opt.far_of_near && P->n_near > 0) {
        const int64_t ne = P->n_near;
        TRY(dbuf_ensure(P->near_fl, (size_t)ne * 4));
        TRY(dbuf_ensure(P->fon_key, (size_t)ne * 8));
        TRY(dbuf_ensure(P->fon_key_sorted, (size_t)ne * 8));
        TRY(dbuf_ensure(P->fon_cnt, (size_t)(ne + 1) * 4));
        TRY(dbuf_ensure(P->fon_ptr, (size_t)(ne + 1) * 4));
        k_fon_anchor<<<grid_for(nn, 128), 128, 0, st>>>(nn, dp<int>(P->n_level), dp<int>(P->n_parent),
                                                        dp<int>(P->n_ix), dp<int>(P->n_iy), dp<int>(P->n_iz),
                                                        dp<int>(P->near_ptr), dp<int>(P->near_src),
                                                        dp<int>(P->near_fl), dp<unsigned long long>(P->fon_key));
        P->launches++;
        TRY(dev_sort_u64(P, dp<uint64_t>(P->fon_key), dp<uint64_t>(P->fon_key_sorted), nullptr, nullptr, ne, st));
        k_fon_heads<<<grid_for(ne, 256), 256, 0, st>>>(ne, dp<unsigned long long>(P->fon_key_sorted),
                                                       dp<int>(P->fon_cnt));
        P->launches++;
        CUDA_TRY(cudaMemsetAsync(dp<int>(P->fon_cnt) + ne, 0, 4, st));
        TRY(scan_excl(P, dp<int>(P->fon_cnt), dp<int>(P->fon_ptr), ne + 1, st));
        int nf = 0;
        CUDA_TRY(cudaMemcpyAsync(&nf, dp<int>(P->fon_ptr) + ne, 4, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        P->n_fon = nf;
        if (nf > 0) {
            k_fon_fill<<<grid_for(ne, 256), 256, 0, st>>>(ne, dp<unsigned long long>(P->fon_key_sorted),
                                                          dp<int>(P->fon_cnt), dp<int>(P->fon_ptr), P->n_v,
                                                          dp<int>(P->pair_t), dp<int>(P->v_src));
            P->launches++;
        }
    }
    // image terms the near field evaluates (for the near kernels' work figure)
    {
        NearImgCount nc{};
        const FonThr ft = fon_thresholds(P);
        for (const TermDesc &td : P->terms)
            for (int j = td.first; j < td.first + td.count; ++j) {
                const double depth = -P->Z[j].x;
                for (int lv = 0; lv <= TEFMM_NBITS; ++lv)
                    nc.c[td.layer][lv] += !(depth >= ft.thr[lv]);
                nc.c[td.layer][TEFMM_NBITS + 1] += 1;
            }
        CUDA_TRY(cudaMemsetAsync(dp<unsigned long long>(P->counters) + 9, 0, 8, st));
        if (nn > 0) {
            k_near_img_terms<<<grid_for(nn, 128), 128, 0, st>>>(
                nn, dp<int>(P->n_layer), dp<int>(P->n_t0), dp<int>(P->n_t1), dp<int>(P->n_s0), dp<int>(P->n_s1),
                dp<int>(P->near_ptr), dp<int>(P->near_src),
                (P->opt.far_of_near && P->n_near > 0) ? dp<int>(P->near_fl) : nullptr, nc,
                dp<unsigned long long>(P->counters) + 9);
            P->launches++;
        }
    }
    // near-field work items
    {
        TRY(dbuf_ensure(P->nitem_cnt, (size_t)(P->n_nodes + 1) * 4));
        TRY(dbuf_ensure(P->nitem_pos, (size_t)(P->n_nodes + 1) * 4));
        CUDA_TRY(cudaMemsetAsync(dp<int>(P->nitem_cnt) + P->n_nodes, 0, 4, st));
        if (P->n_nodes > 0) {
            k_near_items_count<<<grid_for(P->n_nodes, 128), 128, 0, st>>>(
                P->n_nodes, dp<int>(P->n_split), dp<int>(P->n_t0), dp<int>(P->n_t1), dp<int>(P->n_s0),
                dp<int>(P->n_s1), dp<int>(P->near_ptr), dp<int>(P->near_src), dp<int>(P->nitem_cnt));
            P->launches++;
        }
        TRY(scan_excl(P, dp<int>(P->nitem_cnt), dp<int>(P->nitem_pos), P->n_nodes + 1, st));
        int ni = 0;
        CUDA_TRY(cudaMemcpyAsync(&ni, dp<int>(P->nitem_pos) + P->n_nodes, 4, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        P->n_near_items = ni;
        TRY(dbuf_ensure(P->nitem_node, (size_t)(ni + 1) * 4));
        TRY(dbuf_ensure(P->nitem_part, (size_t)(ni + 1) * 4));
        TRY(dbuf_ensure(P->nitem_np, (size_t)(ni + 1) * 4));
        if (ni > 0) {
            k_near_items_fill<<<grid_for(P->n_nodes, 128), 128, 0, st>>>(
                P->n_nodes, dp<int>(P->nitem_cnt), dp<int>(P->nitem_pos), dp<int>(P->nitem_node),
                dp<int>(P->nitem_part), dp<int>(P->nitem_np));
            P->launches++;
        }
    }
    unsigned long long np2p[10] = {};
    CUDA_TRY(cudaMemcpyAsync(np2p, P->counters.p, 80, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    P->n_p2p_pairs = (int64_t)np2p[0];
    for (int l = 0; l < 8; ++l) P->p2p_by_layer[l] = (int64_t)np2p[1 + l];
    P->n_near_img_terms = (int64_t)np2p[9];
    return TEFMM_OK;
}
