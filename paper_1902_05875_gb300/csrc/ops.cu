// Taylor-expansion operators of Sec. 3.1 and the near field (FP64 form).
//
//   P2M   alpha_k = sum_j q_j (r_j - c)^k                          (eq. taylorexpfar3layers)
//   M2M   gamma_k = sum_{k'<=k} C(k,k') (c - c')^{k-k'} alpha_k'    (eqs. LETOLEmat, TETartoTETar)
//   M2L   beta_k += sum_k' alpha_k' D_r^k D_r'^k' u / (k! k'!)     (eq. tesourceboxtotargetbox)
//   L2L   lambda_k = sum_{k'>=k} C(k',k) (c~ - c)^{k'-k} beta_k'   (eq. freeletole)
//   L2P   Phi(r) += sum_k beta_k (r - c)^k                         (eq. taylorexploc2ld)
//   P2P   free-space h0 plus the DCIM image sum (Sec. 3.3, eq. closedformgreen)
//
// M2L follows the per-key batching of Sec. 3.2 (the derivative tables depend
// only on the box centres): V pairs are grouped by a key, one derivative table
// a_g = D^g f / g!, |g| <= 2p, is built per key with the recurrence of eq.
// ``recurrsion`` (corrected form, see the derivative-table kernel), and each
// pair contracts H[k][k'] = C(k+k',k) (-1)^{k1'+k2'} (A_{k+k'} + (-1)^{k3'} B_{k+k'})
// with its source moments.  For a same-layer term with image distance
// W = sz z + szp z' + c one has D_r^k D_r'^k' f = (-1)^{k1'+k2'} sz^{k3} szp^{k3'}
// D^{k+k'} f, so the terms split into
//   B (sz*szp = -1): free space, up-down, down-up; key (level, layer, dx, dy, dz)
//   A (sz*szp = +1): up-up, down-down;             key (level, layer, dx, dy, iz_t+iz_s)
// with (-1)^{g3} folded into the down-up and down-down images.

#include "ops_common.cuh"
#include "alg2.cuh"

namespace {

constexpr int CH = 16;          // pairs per M2L work chunk

// ------------------------------------------------------------------ P2M
__global__ void k_p2m(int nn, TreeArrays T, Cube cb, int p, int np, const int *__restrict__ mi,
                      const double *__restrict__ sx, const double *__restrict__ sy,
                      const double *__restrict__ sz, const double *__restrict__ sq,
                      cplx *__restrict__ alpha) {
    int node = blockIdx.x;
    if (node >= nn || T.split[node]) return;
    int s0 = T.s0[node], s1 = T.s1[node];
    if (s1 <= s0) return;
    extern __shared__ double sm[];
    const int TILE = 64;
    const int P1 = p + 1;
    double *pw = sm;                       // [TILE][3][P1]
    cplx *qq = (cplx *)(pw + TILE * 3 * P1);
    int l = T.level[node];
    double h = box_h(cb.side, l);
    double cx = centre(cb.lo[0], T.ix[node], h);
    double cy = centre(cb.lo[1], T.iy[node], h);
    double cz = centre(cb.lo[2], T.iz[node], h);
    const int R = 4;                       // up to 4 coefficients per thread (np <= 4*blockDim)
    cplx acc[R];
    int kk[R][3];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[r] = mkc(0, 0);
        int k = threadIdx.x + r * blockDim.x;
        if (k < np) {
            kk[r][0] = mi[3 * k];
            kk[r][1] = mi[3 * k + 1];
            kk[r][2] = mi[3 * k + 2];
        } else {
            kk[r][0] = kk[r][1] = kk[r][2] = 0;
        }
    }
    for (int base = s0; base < s1; base += TILE) {
        int cnt = min(TILE, s1 - base);
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            double d[3] = {sx[base + j] - cx, sy[base + j] - cy, sz[base + j] - cz};
            for (int a = 0; a < 3; ++a) {
                double v = 1.0;
                for (int e = 0; e < P1; ++e) {
                    pw[(j * 3 + a) * P1 + e] = v;
                    v *= d[a];
                }
            }
            qq[j] = mkc(sq[2 * (base + j)], sq[2 * (base + j) + 1]);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int k = threadIdx.x + r * blockDim.x;
            if (k >= np) continue;
            for (int j = 0; j < cnt; ++j) {
                double m = pw[(j * 3 + 0) * P1 + kk[r][0]] * pw[(j * 3 + 1) * P1 + kk[r][1]] *
                           pw[(j * 3 + 2) * P1 + kk[r][2]];
                acc[r].x += qq[j].x * m;
                acc[r].y += qq[j].y * m;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int k = threadIdx.x + r * blockDim.x;
        if (k < np) alpha[(int64_t)node * np + k] = acc[r];
    }
}

// ------------------------------------------------------------------ M2M / L2L
// A Taylor shift by an offset d factors over the three axes,
//   C(k, j) d^{k - j} = prod_a C(k_a, j_a) d_a^{k_a - j_a},
// so the multi-index shift is three one-dimensional shifts, applied one axis
// after the other (each of at most p + 1 terms per coefficient); the
// intermediate coefficients keep total degree <= p.
constexpr int SH_KPT = 2;   // coefficients per thread (256 threads, n_p <= 512)

// cw[(a * (p + 1) + n) * (p + 1) + j] = C(n, j) d_a^{n - j}, 0 <= j <= n <= p
__device__ __forceinline__ void shift_coeffs(double *cw, int p, double d0, double d1, double d2) {
    const int P1 = p + 1;
    for (int t = threadIdx.x; t < 3 * P1; t += blockDim.x) {
        const int ax = t / P1, n = t % P1;
        const double d = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
        double c = 1.0, pw = 1.0;            // C(n, j), d^{n - j}, from j = n down
        for (int j = n; j >= 0; --j) {
            cw[(ax * P1 + n) * P1 + j] = c * pw;
            c = c * (double)j / (double)(n - j + 1);
            pw *= d;
        }
    }
}

// one axis of the upward shift: out_k = sum_{j_a <= k_a} C(k_a, j_a) d_a^{k_a - j_a} in_{k with k_a = j_a}
__device__ __forceinline__ cplx shift_up_axis(int ax, const int kk[3], const double *cw, int P1, const cplx *in) {
    cplx acc = mkc(0, 0);
    int m[3] = {kk[0], kk[1], kk[2]};
    const double *row = cw + (ax * P1 + kk[ax]) * P1;
    for (int j = 0; j <= kk[ax]; ++j) {
        m[ax] = j;
        const double c = row[j];
        const cplx x = in[midx(m[0], m[1], m[2])];
        acc.x += c * x.x;
        acc.y += c * x.y;
    }
    return acc;
}

// one axis of the downward shift: out_k = sum_{j_a >= k_a, |m| <= p} C(j_a, k_a) d_a^{j_a - k_a} in_{k with k_a = j_a}
__device__ __forceinline__ cplx shift_down_axis(int ax, const int kk[3], const double *cw, int p, const cplx *in) {
    const int P1 = p + 1;
    cplx acc = mkc(0, 0);
    int m[3] = {kk[0], kk[1], kk[2]};
    const int jmax = p - (kk[0] + kk[1] + kk[2] - kk[ax]);
    for (int j = kk[ax]; j <= jmax; ++j) {
        m[ax] = j;
        const double c = cw[(ax * P1 + j) * P1 + kk[ax]];
        const cplx x = in[midx(m[0], m[1], m[2])];
        acc.x += c * x.x;
        acc.y += c * x.y;
    }
    return acc;
}

// gamma_k = sum_children sum_{k' <= k} C(k,k') (c_child - c_parent)^{k-k'} alpha^child_k'
__global__ void k_m2m(int off, int cnt, TreeArrays T, Cube cb, int p, int np, const int *__restrict__ mi,
                      cplx *__restrict__ alpha) {
    int node = off + blockIdx.x;
    if (blockIdx.x >= cnt || !T.split[node] || T.s1[node] <= T.s0[node]) return;
    extern __shared__ double sm[];
    const int P1 = p + 1;
    cplx *s0 = (cplx *)sm, *s1 = s0 + np;
    double *cw = (double *)(s1 + np);                 // [3][p+1][p+1]
    const int l = T.level[node];
    const double h = box_h(cb.side, l), hc = box_h(cb.side, l + 1);
    const double c0 = centre(cb.lo[0], T.ix[node], h), c1 = centre(cb.lo[1], T.iy[node], h),
                 c2 = centre(cb.lo[2], T.iz[node], h);
    int kk[SH_KPT][3];
    cplx acc[SH_KPT];
#pragma unroll
    for (int i = 0; i < SH_KPT; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        for (int ax = 0; ax < 3; ++ax) kk[i][ax] = k < np ? mi[3 * k + ax] : 0;
        acc[i] = mkc(0, 0);
    }
    const int cf0 = T.cfirst[node], nch = T.nchild[node];
    for (int c = 0; c < nch; ++c) {
        const int ch = cf0 + c;
        if (T.s1[ch] <= T.s0[ch]) continue;
        __syncthreads();                              // the previous child is done with s0, cw
        for (int k = threadIdx.x; k < np; k += blockDim.x) s0[k] = alpha[(int64_t)ch * np + k];
        shift_coeffs(cw, p, centre(cb.lo[0], T.ix[ch], hc) - c0, centre(cb.lo[1], T.iy[ch], hc) - c1,
                     centre(cb.lo[2], T.iz[ch], hc) - c2);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SH_KPT; ++i) {
            const int k = threadIdx.x + i * blockDim.x;
            if (k < np) s1[k] = shift_up_axis(0, kk[i], cw, P1, s0);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SH_KPT; ++i) {
            const int k = threadIdx.x + i * blockDim.x;
            if (k < np) s0[k] = shift_up_axis(1, kk[i], cw, P1, s1);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SH_KPT; ++i) {
            const int k = threadIdx.x + i * blockDim.x;
            if (k < np) {
                const cplx v = shift_up_axis(2, kk[i], cw, P1, s0);
                acc[i].x += v.x;
                acc[i].y += v.y;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < SH_KPT; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k < np) alpha[(int64_t)node * np + k] = acc[i];
    }
}

// ------------------------------------------------------------------ L2L
// lambda_k += sum_{k' >= k} C(k',k) (c_child - c_parent)^{k'-k} beta^parent_k'
__global__ void k_l2l(int off, int cnt, TreeArrays T, Cube cb, int p, int np, const int *__restrict__ mi,
                      cplx *__restrict__ beta) {
    int node = off + blockIdx.x;
    if (blockIdx.x >= cnt || T.t1[node] <= T.t0[node]) return;
    int par = T.parent[node];
    if (par < 0) return;
    extern __shared__ double sm[];
    cplx *s0 = (cplx *)sm, *s1 = s0 + np;
    double *cw = (double *)(s1 + np);
    const int l = T.level[node];
    const double h = box_h(cb.side, l), hp = box_h(cb.side, l - 1);
    for (int k = threadIdx.x; k < np; k += blockDim.x) s0[k] = beta[(int64_t)par * np + k];
    shift_coeffs(cw, p, centre(cb.lo[0], T.ix[node], h) - centre(cb.lo[0], T.ix[par], hp),
                 centre(cb.lo[1], T.iy[node], h) - centre(cb.lo[1], T.iy[par], hp),
                 centre(cb.lo[2], T.iz[node], h) - centre(cb.lo[2], T.iz[par], hp));
    int kk[SH_KPT][3];
#pragma unroll
    for (int i = 0; i < SH_KPT; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        for (int ax = 0; ax < 3; ++ax) kk[i][ax] = k < np ? mi[3 * k + ax] : 0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SH_KPT; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k < np) s1[k] = shift_down_axis(0, kk[i], cw, p, s0);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SH_KPT; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k < np) s0[k] = shift_down_axis(1, kk[i], cw, p, s1);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SH_KPT; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k < np) {
            const cplx v = shift_down_axis(2, kk[i], cw, p, s0);
            cplx b = beta[(int64_t)node * np + k];
            beta[(int64_t)node * np + k] = mkc(b.x + v.x, b.y + v.y);
        }
    }
}

// ------------------------------------------------------------------ M2L keys
// (layout and field accessors in ops_common.cuh)
// has_A[16]: a layer with up-up or down-down images; fonB / fonA [16][21]: a
// layer with far images of its B' / A' terms at a level (far-of-near pairs
// e >= nv_v come after the V pairs)
__global__ void k_m2l_items(int64_t nv, int64_t nv_v, TreeArrays T, const int *__restrict__ pair_t,
                            const int *__restrict__ v_src, const int *__restrict__ has_A,
                            const cplx *__restrict__ kl, uint64_t *__restrict__ keys,
                            int *__restrict__ vals, int *flags) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nv) return;
    int t = pair_t[e], s = v_src[e];
    int l = T.level[t], lay = T.layer[t], lays = T.layer[s];
    int dx = T.ix[t] - T.ix[s], dy = T.iy[t] - T.iy[s], dz = T.iz[t] - T.iz[s];
    vals[2 * e] = (int)(2 * e);
    vals[2 * e + 1] = (int)(2 * e + 1);
    if (e >= nv_v) {                   // far-of-near pair of adjacent leaves of level l
        const int *fonB = has_A + TEFMM_MAX_LAYERS, *fonA = fonB + TEFMM_MAX_LAYERS * (TEFMM_NBITS + 1);
        const int li = lay * (TEFMM_NBITS + 1) + l;
        if (abs(dx) > 1 || abs(dy) > 1 || abs(dz) > 1 || lay != lays) {
            atomicOr(flags, FLAG_CHECK);
            keys[2 * e] = keys[2 * e + 1] = ~0ULL;
            return;
        }
        keys[2 * e] = fonB[li] ? fon_key(l, lay, dx, dy, 0, (uint64_t)(dz + KEY_OFF)) : ~0ULL;
        keys[2 * e + 1] = fonA[li] ? fon_key(l, lay, dx, dy, 1, (uint64_t)(T.iz[t] + T.iz[s])) : ~0ULL;
        return;
    }
    // offsets must fit the keys' fields (a V pair lies within the neighbourhood of
    // its parent's colleagues; wavenumber-coarse levels widen that neighbourhood)
    if (abs(dx) > KEY_OFF || abs(dy) > KEY_OFF || (lay == lays && abs(dz) > KEY_OFF)) {
        atomicOr(flags, FLAG_CHECK);
        keys[2 * e] = keys[2 * e + 1] = ~0ULL;
    } else if (lay != lays) {          // cross-layer component: one table per (z_t, z_s)
        // images in the layer of the larger |k| (their DCIM fits are the accurate
        // ones): a target layer with the smaller |k| takes its mirror pair's key
        const double kt = hypot(kl[lay].x, kl[lay].y), ks = hypot(kl[lays].x, kl[lays].y);
        keys[2 * e] = ks > kt ? xkey(l, lays, lay, -dx, -dy, T.iz[s], T.iz[t], 1)
                              : xkey(l, lay, lays, dx, dy, T.iz[t], T.iz[s], 0);
        keys[2 * e + 1] = ~0ULL;
    } else {
        keys[2 * e] = m2l_key(0, l, lay, dx, dy, (uint64_t)(dz + KEY_OFF));
        keys[2 * e + 1] = has_A[lay] ? m2l_key(1, l, lay, dx, dy, (uint64_t)(T.iz[t] + T.iz[s])) : ~0ULL;
    }
}

__global__ void k_heads(int64_t n, const uint64_t *__restrict__ keys, int *__restrict__ head,
                        int *__restrict__ nvalid) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool valid = keys[i] != ~0ULL;
    head[i] = valid && (i == 0 || keys[i] != keys[i - 1]);
    // invalid keys sort last: the first invalid position is the valid count
    if (!valid && (i == 0 || keys[i - 1] != ~0ULL)) *nvalid = (int)i;
}

__global__ void k_seg_start(int64_t n, const int *__restrict__ head, const int *__restrict__ seg_incl,
                            const uint64_t *__restrict__ keys, int *__restrict__ seg_start,
                            uint64_t *__restrict__ table_key) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !head[i]) return;
    int s = seg_incl[i] - 1;
    seg_start[s] = (int)i;
    table_key[s] = keys[i];
}

// Symmetry of the derivative tables.  A table takes D^g / g! of a function of
// (x^2 + y^2, z) at (X, Y) = (dx h, dy h); the key's other fields do not
// involve dx, dy.  Hence for signs sx, sy:
//   T(sx X, sy Y)[g1, g2, g3] = sx^g1 sy^g2 T(X, Y)[g1, g2, g3],
//   T(Y, X)[g1, g2, g3]       = T(X, Y)[g2, g1, g3].
// Of the (up to eight) keys that differ only by these maps, the first in key
// order (its representative) is computed by the recurrence and the others are
// copied from it.  A reversed cross-layer key (rev bit) has the table of its
// rev = 0 twin, so cross keys search sixteen variants.  rep_code[i] = rep * 8 + code, code bit 0: sx = -1, bit 1:
// sy = -1, bit 2: swapped, so that T_i[g] = sx^g1 sy^g2 T_rep[g or (g2, g1, g3)].
// The sign flips reproduce the recurrence's own result bit for bit; the swap
// changes its rounding only (the x and y terms are summed in the other order).
__global__ void k_table_rep(int ntab, const uint64_t *__restrict__ keys, int *__restrict__ rep_code,
                            int *__restrict__ nrep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntab) return;
    const uint64_t key = keys[i];
    const int dx = key_dx(key), dy = key_dy(key);
    // a reversed cross key uses the table of the same key with rev = 0
    const int nvar = key_is_cross(key) ? 16 : 8;
    int rep = i, rdx = dx, rdy = dy;
    for (int v = 1; v < nvar; ++v) {
        int a = (v & 4) ? dy : dx, b = (v & 4) ? dx : dy;
        if (v & 1) a = -a;
        if (v & 2) b = -b;
        uint64_t kv = key_with_dxdy(key, a, b);
        if (v & 8) kv ^= 1ULL << 43;
        int lo = 0, hi = rep;   // keys are sorted: search the ones before the current representative
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (keys[mid] < kv) lo = mid + 1;
            else hi = mid;
        }
        if (lo < rep && keys[lo] == kv) {
            rep = lo;
            rdx = a;
            rdy = b;
        }
    }
    int code;
    if (abs(dx) == abs(rdx) && abs(dy) == abs(rdy)) code = (dx != rdx) | ((dy != rdy) << 1);
    else code = 4 | (dx != rdy) | ((dy != rdx) << 1);
    rep_code[i] = rep * 8 + code;
    if (rep == i) atomicAdd(nrep, 1);
}

// copy the tables [first, first + ntab) that are not representatives from
// their representative: grid (ntab, slices), slice s holds ncoef(2p - s) entries
__global__ void k_table_expand(int ntab, int first, const int *__restrict__ rep_code,
                               const int *__restrict__ mi, int p, cplx *__restrict__ tabs, int64_t stride) {
    const int t = blockIdx.x, s = blockIdx.y;
    if (t >= ntab) return;
    const int rc = rep_code[first + t];
    const int rep = (rc >> 3) - first, code = rc & 7;
    if (rep == t) return;
    const int n = ncoef(2 * p - s), off = slice_off(p, s);
    const cplx *src = tabs + (int64_t)rep * stride + off;
    cplx *dst = tabs + (int64_t)t * stride + off;
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
        const int g1 = mi[3 * g], g2 = mi[3 * g + 1], g3 = mi[3 * g + 2];
        const cplx v = src[(code & 4) ? midx(g2, g1, g3) : g];
        const bool neg = ((code & 1) && (g1 & 1)) != ((code & 2) && (g2 & 1));
        dst[g] = neg ? mkc(-v.x, -v.y) : v;
    }
}

__global__ void k_chunk_heads(int64_t n, const uint64_t *__restrict__ keys,
                              const int *__restrict__ seg_incl, const int *__restrict__ seg_start,
                              int *__restrict__ chead, int chsize) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f = 0;
    if (keys[i] != ~0ULL) {
        int s = seg_incl[i] - 1;
        f = ((i - seg_start[s]) % chsize) == 0;
    }
    chead[i] = f;
}

__global__ void k_chunks(int64_t n, int64_t nvalid, const int *__restrict__ chead,
                         const int *__restrict__ cscan, const int *__restrict__ seg_incl,
                         int *__restrict__ chunk_start, int *__restrict__ chunk_table,
                         int *__restrict__ chunk_cnt, int nchunks) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !chead[i]) return;
    int c = cscan[i] - 1;
    chunk_start[c] = (int)i;
    chunk_table[c] = seg_incl[i] - 1;
    (void)nchunks;
    (void)nvalid;
}

__global__ void k_chunk_cnt(int nchunks, int64_t nvalid, const int *__restrict__ chunk_start,
                            const int *__restrict__ chunk_table, int *__restrict__ chunk_cnt,
                            int chsize) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    int end = (c + 1 < nchunks) ? chunk_start[c + 1] : (int)nvalid;
    int cnt = end - chunk_start[c];
    chunk_cnt[c] = cnt < chsize ? cnt : chsize;
}

__global__ void __launch_bounds__(256, 4) k_tables(int ntab, const uint64_t *__restrict__ table_key, Cube cb, int P2, int np2,
                         ImgView im, FonThr fon, int a2_on, const int *__restrict__ rep_code, cplx *__restrict__ tables) {
    int tb = blockIdx.x;
    if (tb >= ntab || (rep_code[tb] >> 3) != tb) return;   // copied by symmetry
    extern __shared__ double sm[];
    const int cmax = tri(P2 + 1);            // entries of the largest order
    cplx *a = (cplx *)sm;                    // [3][cmax] ring of orders
    cplx *b = a + 3 * cmax;
    cplx *acc = tables + (int64_t)tb * np2;  // the table accumulates in place
    for (int g = threadIdx.x; g < np2; g += blockDim.x) acc[g] = mkc(0, 0);
    __syncthreads();
    uint64_t key = table_key[tb];
    int kind = key_kind(key);
    int l = key_level(key);
    int lay = key_layer(key);
    int dx = key_dx(key);
    int dy = key_dy(key);
    int w = (int)key_w(key);
    double h = box_h(cb.side, l);
    double X = (double)dx * h, Y = (double)dy * h;
    cplx k = im.k[lay];
    int tf = im.lt_first[lay], tc = im.lt_count[lay];
    if (kind == 0) {
        double dz = (double)(w - KEY_OFF) * h;
        recur_accumulate(P2, cmax, k, X, Y, mkc(dz, 0), mkc(1, 0), false, a, b, acc);
        for (int ti = tf; ti < tf + tc; ++ti) {
            DevTerm t = im.terms[ti];
            if (t.tag != 2 && t.tag != 3) continue;
            double W0 = __dadd_rn(__dmul_rn(t.sz, dz), t.c);
            if (a2_on && W0 >= t.zmin) continue;   // Algorithm 2: added by k_tables_a2
            for (int j = t.first; j < t.first + t.count; ++j) {
                cplx Wj = mkc(W0 - t.zmin - im.Z[j].x, -im.Z[j].y);
                recur_accumulate(P2, cmax, k, X, Y, Wj, im.A[j], t.tag == 3, a, b, acc);
            }
        }
    } else if (kind == 1) {
        double zsum = __dadd_rn(2.0 * cb.lo[2], __dmul_rn((double)(w + 1), h));
        for (int ti = tf; ti < tf + tc; ++ti) {
            DevTerm t = im.terms[ti];
            if (t.tag != 0 && t.tag != 1) continue;
            double W0 = __dadd_rn(__dmul_rn(t.sz, zsum), t.c);
            if (a2_on && W0 >= t.zmin) continue;
            for (int j = t.first; j < t.first + t.count; ++j) {
                cplx Wj = mkc(W0 - t.zmin - im.Z[j].x, -im.Z[j].y);
                recur_accumulate(P2, cmax, k, X, Y, Wj, im.A[j], t.tag == 1, a, b, acc);
            }
        }
    } else {
        // far-of-near (kind 2): the far images only, no free-space term
        const int sub = (int)((key >> 43) & 1);
        const int ww = (int)(key_w(key) & ((1ULL << 43) - 1));
        const double thr = fon.thr[l];
        if (sub == 0) {
            double dz = (double)(ww - KEY_OFF) * h;
            for (int ti = tf; ti < tf + tc; ++ti) {
                DevTerm t = im.terms[ti];
                if (t.tag != 2 && t.tag != 3) continue;
                double W0 = __dadd_rn(__dmul_rn(t.sz, dz), t.c);
                for (int j = t.first; j < t.first + t.count; ++j) {
                    if (!(-im.Z[j].x >= thr)) continue;
                    cplx Wj = mkc(W0 - t.zmin - im.Z[j].x, -im.Z[j].y);
                    recur_accumulate(P2, cmax, k, X, Y, Wj, im.A[j], t.tag == 3, a, b, acc);
                }
            }
        } else {
            double zsum = __dadd_rn(2.0 * cb.lo[2], __dmul_rn((double)(ww + 1), h));
            for (int ti = tf; ti < tf + tc; ++ti) {
                DevTerm t = im.terms[ti];
                if (t.tag != 0 && t.tag != 1) continue;
                double W0 = __dadd_rn(__dmul_rn(t.sz, zsum), t.c);
                for (int j = t.first; j < t.first + t.count; ++j) {
                    if (!(-im.Z[j].x >= thr)) continue;
                    cplx Wj = mkc(W0 - t.zmin - im.Z[j].x, -im.Z[j].y);
                    recur_accumulate(P2, cmax, k, X, Y, Wj, im.A[j], t.tag == 1, a, b, acc);
                }
            }
        }
    }
}

// Algorithm 2: the reaction terms of the same-layer keys of kinds 0 and 1 from
// their Sommerfeld-integral tables, added to the tables k_tables started
// (free-space part); the image distance as in k_tables.
__global__ void __launch_bounds__(256) k_tables_a2(int ntab, const uint64_t *__restrict__ table_key, Cube cb,
                                                   int np2, ImgView im, A2View a2,
                                                   const int *__restrict__ rep_code, cplx *__restrict__ tables) {
    const int tb = blockIdx.x;
    if (tb >= ntab || (rep_code[tb] >> 3) != tb) return;
    const uint64_t key = table_key[tb];
    const int kind = key_kind(key);
    if (kind > 1) return;
    extern __shared__ double sm[];
    const int l = key_level(key), lay = key_layer(key);
    const int w = (int)key_w(key);
    const double h = box_h(cb.side, l);
    const double X = (double)key_dx(key) * h, Y = (double)key_dy(key) * h;
    const double zarg = kind == 0 ? (double)(w - KEY_OFF) * h
                                  : __dadd_rn(2.0 * cb.lo[2], __dmul_rn((double)(w + 1), h));
    const int tf = im.lt_first[lay], tc = im.lt_count[lay];
    for (int ti = tf; ti < tf + tc; ++ti) {
        const DevTerm t = im.terms[ti];
        if (kind == 0 ? t.tag < 2 : t.tag > 1) continue;
        const double W0 = __dadd_rn(__dmul_rn(t.sz, zarg), t.c);
        if (!(W0 >= t.zmin)) continue;      // below the slab's image distances: the images (k_tables)
        alg2_accumulate(a2, a2.t[lay][t.tag], X, Y, W0, t.tag == 1 || t.tag == 3, (cplx *)sm, np2,
                        tables + (int64_t)tb * np2);
    }
}

// ------------------------------------------------------------------ M2L apply (FP64)
__global__ void k_m2l_fp64(int nchunks, const int *__restrict__ chunk_start,
                           const int *__restrict__ chunk_table, const int *__restrict__ chunk_cnt,
                           const uint64_t *__restrict__ table_key, const cplx *__restrict__ tables,
                           const int *__restrict__ sorted_vals, const int *__restrict__ pair_t,
                           const int *__restrict__ v_src, int np, int np2,
                           const unsigned short *__restrict__ G, const double *__restrict__ cB,
                           const double *__restrict__ cA, const cplx *__restrict__ alpha,
                           cplx *__restrict__ beta) {
    int c = blockIdx.x;
    if (c >= nchunks) return;
    extern __shared__ double sm[];
    cplx *tab = (cplx *)sm;                  // [np2]
    cplx *al = tab + np2;                    // [CH][np]
    __shared__ int tgt[CH];
    int tb = chunk_table[c];
    int cnt = chunk_cnt[c];
    int st = chunk_start[c];
    const double *coef = key_is_B(table_key[tb]) ? cB : cA;
    for (int g = threadIdx.x; g < np2; g += blockDim.x) tab[g] = tables[(int64_t)tb * np2 + g];
    for (int q = 0; q < cnt; ++q) {
        int item = sorted_vals[st + q];
        int e = item >> 1;
        int s = v_src[e];
        if (threadIdx.x == 0) tgt[q] = pair_t[e];
        for (int k = threadIdx.x; k < np; k += blockDim.x) al[q * np + k] = alpha[(int64_t)s * np + k];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        cplx acc[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) acc[q] = mkc(0, 0);
        for (int kp = 0; kp < np; ++kp) {
            double cf = coef[(int64_t)kp * np + k];
            cplx hv = tab[G[(int64_t)kp * np + k]];
            hv.x *= cf;
            hv.y *= cf;
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                if (q < cnt) {
                    cplx a = al[q * np + kp];
                    acc[q].x += hv.x * a.x - hv.y * a.y;
                    acc[q].y += hv.x * a.y + hv.y * a.x;
                }
            }
        }
        for (int q = 0; q < cnt; ++q) {
            double *dst = (double *)&beta[(int64_t)tgt[q] * np + k];
            atomicAdd(dst, acc[q].x);
            atomicAdd(dst + 1, acc[q].y);
        }
    }
}

// ------------------------------------------------------------------ near field (FP64)
__device__ __forceinline__ cplx eikr_over_r(cplx ik, cplx R) {
    // e^{ikR}/R
    cplx e = cexp_(cmul(ik, R));
    return cdiv(e, R);
}

__global__ void k_near_fp64(int n_items, NearArgs a) {
    // one work item: near sources [src_lo, src_hi) of the leaf's list; chunk 0 also adds the L2P
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int node = a.item_node[it], part = a.item_part[it], nparts = a.item_np[it];
    const int64_t src_lo = (int64_t)part * NEAR_CHUNK, src_hi = src_lo + NEAR_CHUNK;
    const TreeArrays &T = a.T;
    if (T.split[node]) return;
    int t0 = T.t0[node], t1 = T.t1[node];
    int nt = t1 - t0;
    if (nt <= 0) return;
    const int TILE = 128;
    __shared__ double xs[TILE], ys[TILE], zs[TILE];
    __shared__ cplx qs[TILE];
    __shared__ cplx red[128];
    __shared__ cplx imgA[TEFMM_MAX_TERMS * TEFMM_MAX_IMG], imgZ[TEFMM_MAX_TERMS * TEFMM_MAX_IMG];
    __shared__ double tgeo[TEFMM_MAX_TERMS][4];
    __shared__ int tcnt[TEFMM_MAX_TERMS];
    int lay = T.layer[node];
    cplx k = a.im.k[lay];
    cplx ik = mkc(-k.y, k.x);
    cplx inv_ik = cdiv(mkc(1, 0), ik);
    int tf = a.im.lt_first[lay], ntm = a.im.lt_count[lay];
    if (threadIdx.x < ntm) {
        DevTerm t = a.im.terms[tf + threadIdx.x];
        tgeo[threadIdx.x][0] = t.sz;
        tgeo[threadIdx.x][1] = t.szp;
        tgeo[threadIdx.x][2] = t.c;
        tgeo[threadIdx.x][3] = t.zmin;
        tcnt[threadIdx.x] = t.count;
    }
    for (int ti = 0; ti < ntm; ++ti) {
        DevTerm t = a.im.terms[tf + ti];
        for (int j = threadIdx.x; j < t.count; j += blockDim.x) {
            imgA[ti * TEFMM_MAX_IMG + j] = cmul(a.im.A[t.first + j], inv_ik);
            imgZ[ti * TEFMM_MAX_IMG + j] = a.im.Z[t.first + j];
        }
    }
    // thread layout: nslice threads per target
    int ntp = 1;
    while (ntp < nt && ntp < 128) ntp <<= 1;
    int nslice = 128 / ntp;
    int my_t = threadIdx.x % ntp, slice = threadIdx.x / ntp;
    int l = T.level[node];
    double h = box_h(a.cb.side, l);
    double cx = centre(a.cb.lo[0], T.ix[node], h), cy = centre(a.cb.lo[1], T.iy[node], h),
           cz = centre(a.cb.lo[2], T.iz[node], h);
    int nb0 = a.near_ptr[node], nb1 = a.near_ptr[node + 1];
    for (int tbase = 0; tbase < nt; tbase += ntp) {
        int ti = tbase + my_t;
        bool active = ti < nt;
        double xt = 0, yt = 0, zt = 0;
        if (active) {
            xt = a.tx[t0 + ti];
            yt = a.ty[t0 + ti];
            zt = a.tz[t0 + ti];
        }
        cplx accf = mkc(0, 0);     // sum q e^{ikr}/r (free)
        cplx acci = mkc(0, 0);     // sum q A/(ik) e^{ikR}/R (images)
        __syncthreads();
        int64_t off = 0;           // near sources of the list before entry nb
        for (int nb = nb0; nb < nb1 && off < src_hi; ++nb) {
            int s = a.near_src[nb];
            int s0 = T.s0[s], s1 = T.s1[s];
            const int64_t ns_e = s1 - s0;
            const int b0 = (int)(s0 + max((int64_t)0, src_lo - off));
            const int b1 = (int)(s0 + min(ns_e, src_hi - off));
            off += ns_e;
            if (b0 >= b1) continue;
            s0 = b0;
            s1 = b1;
            // an entry with a far-of-near anchor: its far images went through M2L
            const int fl = a.fon.on ? a.near_fl[nb] : -1;
            const double thr = fl >= 0 ? a.fon.thr[fl] : INFINITY;
            for (int base = s0; base < s1; base += TILE) {
                int cnt = min(TILE, s1 - base);
                __syncthreads();
                for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
                    xs[j] = a.sx[base + j];
                    ys[j] = a.sy[base + j];
                    zs[j] = a.sz[base + j];
                    qs[j] = mkc(a.sq[2 * (base + j)], a.sq[2 * (base + j) + 1]);
                }
                __syncthreads();
                if (active) {
                    for (int j = slice; j < cnt; j += nslice) {
                        double dx = xt - xs[j], dy = yt - ys[j], dz = zt - zs[j];
                        double rho2 = dx * dx + dy * dy;
                        cplx q = qs[j];
                        if (!(xt == xs[j] && yt == ys[j] && zt == zs[j])) {
                            double r = sqrt(rho2 + dz * dz);
                            cplx g = eikr_over_r(ik, mkc(r, 0));
                            accf = cadd(accf, cmul(q, g));
                        }
                        cplx gi = mkc(0, 0);
                        for (int tm = 0; tm < ntm; ++tm) {
                            double zeta = tgeo[tm][0] * zt + tgeo[tm][1] * zs[j] + tgeo[tm][2] - tgeo[tm][3];
                            for (int m = 0; m < tcnt[tm]; ++m) {
                                cplx Z = imgZ[tm * TEFMM_MAX_IMG + m];
                                if (-Z.x >= thr) continue;
                                cplx w = mkc(zeta - Z.x, -Z.y);
                                cplx R = csqrt_p(mkc(rho2 + w.x * w.x - w.y * w.y, 2.0 * w.x * w.y));
                                gi = cadd(gi, cmul(imgA[tm * TEFMM_MAX_IMG + m], eikr_over_r(ik, R)));
                            }
                        }
                        acci = cadd(acci, cmul(q, gi));
                    }
                }
            }
        }
        cplx tot = cadd(cmul(accf, inv_ik), acci);
        __syncthreads();
        red[threadIdx.x] = tot;
        __syncthreads();
        if (slice == 0 && active) {
            for (int sl = 1; sl < nslice; ++sl) tot = cadd(tot, red[sl * ntp + my_t]);
            // L2P
            double d[3] = {xt - cx, yt - cy, zt - cz};
            double pw[3][13];
            for (int e = 0; e < 3; ++e) {
                double v = 1.0;
                for (int q = 0; q <= a.p; ++q) {
                    pw[e][q] = v;
                    v *= d[e];
                }
            }
            const cplx *bt = a.beta + (int64_t)node * a.np;
            cplx loc = mkc(0, 0);
            for (int kk = 0; part == 0 && kk < a.np; ++kk) {
                double m = pw[0][a.mi[3 * kk]] * pw[1][a.mi[3 * kk + 1]] * pw[2][a.mi[3 * kk + 2]];
                cplx b = bt[kk];
                loc.x += b.x * m;
                loc.y += b.y * m;
            }
            tot = cadd(tot, loc);
            if (a.scale) tot = cmul(tot, mkc(-k.y / (4.0 * M_PI), k.x / (4.0 * M_PI)));   // i k / (4 pi)
            int out = a.perm_t[t0 + ti];
            if (nparts == 1) {
                a.phi[2 * out] = tot.x;
                a.phi[2 * out + 1] = tot.y;
            } else {                  // chunks of one leaf add into zeroed outputs
                atomicAdd(&a.phi[2 * out], tot.x);
                atomicAdd(&a.phi[2 * out + 1], tot.y);
            }
        }
    }
}

// zero the outputs of the leaves whose near field is split over several work items
__global__ void k_near_zero(int n_items, NearArgs a) {
    const int it = blockIdx.x;
    if (it >= n_items || a.item_part[it] != 0 || a.item_np[it] < 2) return;
    const int node = a.item_node[it];
    for (int t = a.T.t0[node] + threadIdx.x; t < a.T.t1[node]; t += blockDim.x) {
        const int out = a.perm_t[t];
        a.phi[2 * out] = 0.0;
        a.phi[2 * out + 1] = 0.0;
    }
}

int scan_i(tefmm_plan_s *P, const int *in, int *out, int64_t n, bool inclusive, cudaStream_t st) {
    return dev_scan_i32(P, in, out, n, inclusive, st);
}

}  // namespace

int near_zero_split(tefmm_plan_s *P, const NearArgs &a, cudaStream_t st) {
    k_near_zero<<<P->n_near_items, 64, 0, st>>>(P->n_near_items, a);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}


// ---------------------------------------------------------------- host side
int upward_pass(tefmm_plan_s *P, cudaStream_t st) {
    const int nn = P->n_nodes, np = P->np, p = P->p;
    TRY(dbuf_ensure(P->alpha, (size_t)nn * np * sizeof(cplx)));
    CUDA_TRY(cudaMemsetAsync(P->alpha.p, 0, (size_t)nn * np * sizeof(cplx), st));
    TreeArrays T = tree_arrays(P);
    Cube cb = cube_of(P);
    size_t sm_p2m = 64 * 3 * (p + 1) * sizeof(double) + 64 * sizeof(cplx);
    k_p2m<<<nn, 128, sm_p2m, st>>>(nn, T, cb, p, np, dp<int>(P->d_mi), dp<double>(P->sx),
                                   dp<double>(P->sy), dp<double>(P->sz), dp<double>(P->sq),
                                   dp<cplx>(P->alpha));
    P->launches++;
    if (np > SH_KPT * 256) return TEFMM_ERR_INVALID_ARG;
    const size_t sm_m2m = 2 * (size_t)np * sizeof(cplx) + 3 * (size_t)(p + 1) * (p + 1) * sizeof(double);
    TRY(smem_optin(k_m2m));
    for (int l = P->n_levels - 2; l >= 0; --l) {
        int off = P->level_off[l], cnt = P->level_off[l + 1] - off;
        if (cnt > 0) {
            k_m2m<<<cnt, 256, sm_m2m, st>>>(off, cnt, T, cb, p, np, dp<int>(P->d_mi), dp<cplx>(P->alpha));
            P->launches++;
        }
    }
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

int m2l_prepare(tefmm_plan_s *P, cudaStream_t st) {
    const int64_t nv = P->n_v + P->n_fon;
    P->n_tables = 0;
    P->n_tables_built = 0;
    P->n_chunks = 0;
    P->x_first_table = 0;
    P->x_first_chunk = 0;
    if (nv == 0) return TEFMM_OK;
    const int64_t ni = 2 * nv;
    TRY(dbuf_ensure(P->pair_slot, ni * 8));
    TRY(dbuf_ensure(P->pair_slot_sorted, ni * 8));
    TRY(dbuf_ensure(P->pair_idx, ni * 4));
    TRY(dbuf_ensure(P->pair_idx_sorted, ni * 4));
    // has_A per layer: any up-up or down-down term with images; per (layer,
    // level): far images of the B' (up-down, down-up) and A' terms
    constexpr int NLV = TEFMM_NBITS + 1;
    std::vector<int> flagsA(TEFMM_MAX_LAYERS * (1 + 2 * NLV), 0);
    int *hasA = flagsA.data(), *fonB = hasA + TEFMM_MAX_LAYERS, *fonA = fonB + TEFMM_MAX_LAYERS * NLV;
    const FonThr ft = fon_thresholds(P);
    for (auto &t : P->terms) {
        if ((t.tag == 0 || t.tag == 1) && t.count > 0) hasA[t.layer] = 1;
        for (int lv = 0; lv < NLV; ++lv)
            for (int j = t.first; j < t.first + t.count; ++j)
                if (-P->Z[j].x >= ft.thr[lv]) (t.tag >= 2 ? fonB : fonA)[t.layer * NLV + lv] = 1;
    }
    TRY(dbuf_ensure(P->seg_tmp, flagsA.size() * sizeof(int)));
    CUDA_TRY(cudaMemcpyAsync(P->seg_tmp.p, flagsA.data(), flagsA.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    TreeArrays T = tree_arrays(P);
    k_m2l_items<<<grid_for(nv, 256), 256, 0, st>>>(nv, P->n_v, T, dp<int>(P->pair_t), dp<int>(P->v_src),
                                                   dp<int>(P->seg_tmp), dp<cplx>(P->d_k),
                                                   dp<uint64_t>(P->pair_slot),
                                                   dp<int>(P->pair_idx), dp<int>(P->flags));
    P->launches++;
    TRY(dev_sort_u64(P, dp<uint64_t>(P->pair_slot), dp<uint64_t>(P->pair_slot_sorted), dp<int>(P->pair_idx),
                     dp<int>(P->pair_idx_sorted), ni, st));
    const uint64_t *keys = dp<uint64_t>(P->pair_slot_sorted);
    // heads and segments (reuse item buffers as scratch)
    TRY(dbuf_ensure(P->item_flag, (ni + 1) * 4));
    TRY(dbuf_ensure(P->item_scan, (ni + 1) * 4));
    TRY(dbuf_ensure(P->item_node, (ni + 1) * 4));
    int *head = dp<int>(P->item_flag), *seg = dp<int>(P->item_scan), *chead = dp<int>(P->item_node);
    TRY(dbuf_ensure(P->counters, 64));
    int ni_int = (int)ni;
    CUDA_TRY(cudaMemcpyAsync(P->counters.p, &ni_int, 4, cudaMemcpyHostToDevice, st));
    k_heads<<<grid_for(ni, 256), 256, 0, st>>>(ni, keys, head, dp<int>(P->counters));
    P->launches++;
    TRY(scan_i(P, head, seg, ni, true, st));
    int nseg = 0;
    CUDA_TRY(cudaMemcpyAsync(&nseg, seg + ni - 1, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    P->n_tables = nseg;
    TRY(dbuf_ensure(P->keyslot_flag, (size_t)(nseg + 1) * 4));      // segment start
    TRY(dbuf_ensure(P->table_slot, (size_t)(nseg + 1) * 8));        // table key
    k_seg_start<<<grid_for(ni, 256), 256, 0, st>>>(ni, head, seg, keys, dp<int>(P->keyslot_flag),
                                                   dp<uint64_t>(P->table_slot));
    P->launches++;
    TRY(dbuf_ensure(P->table_rep, (size_t)(nseg + 1) * 4));
    CUDA_TRY(cudaMemsetAsync(dp<int>(P->counters) + 2, 0, 4, st));
    k_table_rep<<<grid_for(nseg, 256), 256, 0, st>>>(nseg, dp<uint64_t>(P->table_slot),
                                                     dp<int>(P->table_rep), dp<int>(P->counters) + 2);
    P->launches++;
    P->chunk_pairs = (P->opt.precision == TEFMM_MIXED) ? 128 * TC_MT : CH;
    k_chunk_heads<<<grid_for(ni, 256), 256, 0, st>>>(ni, keys, seg, dp<int>(P->keyslot_flag), chead,
                                                     P->chunk_pairs);
    P->launches++;
    TRY(dbuf_ensure(P->keyslot_table, (ni + 1) * 4));
    TRY(scan_i(P, chead, dp<int>(P->keyslot_table), ni, true, st));
    int nch = 0, nvalid_i = 0;
    CUDA_TRY(cudaMemcpyAsync(&nch, dp<int>(P->keyslot_table) + ni - 1, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&nvalid_i, P->counters.p, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&P->n_tables_built, dp<int>(P->counters) + 2, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    P->n_chunks = nch;
    TRY(dbuf_ensure(P->chunk_start, (size_t)(nch + 1) * 4));
    TRY(dbuf_ensure(P->chunk_key, (size_t)(nch + 1) * 4));
    TRY(dbuf_ensure(P->chunk_cnt, (size_t)(nch + 1) * 4));
    k_chunks<<<grid_for(ni, 256), 256, 0, st>>>(ni, ni, chead, dp<int>(P->keyslot_table), seg,
                                                dp<int>(P->chunk_start), dp<int>(P->chunk_key),
                                                dp<int>(P->chunk_cnt), nch);
    P->launches++;
    const int64_t nvalid = nvalid_i;
    P->n_items = nvalid;
    P->n_items_cross = 0;
    k_chunk_cnt<<<grid_for(nch, 256), 256, 0, st>>>(nch, nvalid, dp<int>(P->chunk_start),
                                                    dp<int>(P->chunk_key), dp<int>(P->chunk_cnt),
                                                    P->chunk_pairs);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    P->x_first_table = P->n_tables;     // narrowed by cross_prepare when cross keys exist
    P->x_first_chunk = P->n_chunks;
    // the tensor-core M2L launches key batches by chunk ranges: their host copy
    // is taken here, once per geometry, so that later applies need no host wait
    P->chunk_key_host.clear();
    if (P->opt.precision == TEFMM_MIXED && nch > 0) {
        P->chunk_key_host.resize(nch);
        CUDA_TRY(cudaMemcpyAsync(P->chunk_key_host.data(), P->chunk_key.p, (size_t)nch * 4,
                                 cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    return TEFMM_OK;
}

int m2l_tables(tefmm_plan_s *P, cudaStream_t st) {
    const int ntab = P->x_first_table;        // same-layer tables (cross-layer ones follow)
    if (ntab == 0) return TEFMM_OK;
    const int np2 = P->np2;
    TRY(dbuf_ensure(P->tables, (size_t)ntab * np2 * sizeof(cplx)));
    const size_t sm = 6 * (size_t)tri(2 * P->p + 1) * sizeof(cplx);
    TRY(smem_optin(k_tables));
    const A2View a2 = a2_view(P);
    k_tables<<<ntab, 256, sm, st>>>(ntab, dp<uint64_t>(P->table_slot), cube_of(P), 2 * P->p, np2,
                                    img_view(P), fon_thresholds(P), a2.on, dp<int>(P->table_rep), dp<cplx>(P->tables));
    P->launches++;
    if (a2.on) {
        const size_t sm2 = (size_t)a2_smem_cplx(a2.P2, a2.ne) * sizeof(cplx);
        TRY(smem_optin(k_tables_a2));
        k_tables_a2<<<ntab, 256, sm2, st>>>(ntab, dp<uint64_t>(P->table_slot), cube_of(P), np2, img_view(P), a2,
                                            dp<int>(P->table_rep), dp<cplx>(P->tables));
        P->launches++;
    }
    CUDA_TRY(cudaGetLastError());
    return tables_expand(P, 0, ntab, 1, dp<cplx>(P->tables), np2, st);
}

int tables_expand(tefmm_plan_s *P, int first, int ntab, int nslices, cplx *tabs, int64_t stride,
                  cudaStream_t st) {
    if (ntab == 0) return TEFMM_OK;
    k_table_expand<<<dim3((unsigned)ntab, (unsigned)nslices), 256, 0, st>>>(
        ntab, first, dp<int>(P->table_rep), dp<int>(P->d_mi), P->p, tabs, stride);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

int m2l_apply(tefmm_plan_s *P, cudaStream_t st) {
    const int nn = P->n_nodes, np = P->np;
    TRY(dbuf_ensure(P->beta, (size_t)nn * np * sizeof(cplx)));
    CUDA_TRY(cudaMemsetAsync(P->beta.p, 0, (size_t)nn * np * sizeof(cplx), st));
    const int nch = (int)P->x_first_chunk;    // same-layer chunks (cross-layer ones follow)
    if (nch == 0) return TEFMM_OK;
    size_t sm = (size_t)P->np2 * sizeof(cplx) + (size_t)CH * np * sizeof(cplx);
    TRY(smem_optin(k_m2l_fp64));
    k_m2l_fp64<<<nch, 256, sm, st>>>(
        nch, dp<int>(P->chunk_start), dp<int>(P->chunk_key), dp<int>(P->chunk_cnt),
        dp<uint64_t>(P->table_slot), dp<cplx>(P->tables), dp<int>(P->pair_idx_sorted),
        dp<int>(P->pair_t), dp<int>(P->v_src), np, P->np2, dp<unsigned short>(P->d_m2l_g),
        dp<double>(P->d_m2l_cB), dp<double>(P->d_m2l_cA), dp<cplx>(P->alpha), dp<cplx>(P->beta));
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

int downward_pass(tefmm_plan_s *P, cudaStream_t st) {
    TreeArrays T = tree_arrays(P);
    Cube cb = cube_of(P);
    if (P->np > SH_KPT * 256) return TEFMM_ERR_INVALID_ARG;
    const size_t sm = 2 * (size_t)P->np * sizeof(cplx) + 3 * (size_t)(P->p + 1) * (P->p + 1) * sizeof(double);
    for (int l = 1; l < P->n_levels; ++l) {
        int off = P->level_off[l], cnt = P->level_off[l + 1] - off;
        if (cnt > 0) {
            k_l2l<<<cnt, 256, sm, st>>>(off, cnt, T, cb, P->p, P->np, dp<int>(P->d_mi), dp<cplx>(P->beta));
            P->launches++;
        }
    }
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

int near_field(tefmm_plan_s *P, double *phi, cudaStream_t st) {
    NearArgs a;
    a.T = tree_arrays(P);
    a.cb = cube_of(P);
    a.p = P->p;
    a.np = P->np;
    a.mi = dp<int>(P->d_mi);
    a.near_ptr = dp<int>(P->near_ptr);
    a.near_src = dp<int>(P->near_src);
    a.sx = dp<double>(P->sx);
    a.sy = dp<double>(P->sy);
    a.sz = dp<double>(P->sz);
    a.sq = dp<double>(P->sq);
    a.tx = P->shared_pts ? a.sx : dp<double>(P->tx);
    a.ty = P->shared_pts ? a.sy : dp<double>(P->ty);
    a.tz = P->shared_pts ? a.sz : dp<double>(P->tz);
    a.perm_t = P->shared_pts ? dp<int>(P->perm_s) : dp<int>(P->perm_t);
    a.beta = dp<cplx>(P->beta);
    a.im = img_view(P);
    a.fon = fon_thresholds(P);
    a.near_fl = dp<int>(P->near_fl);
    a.item_node = dp<int>(P->nitem_node);
    a.item_part = dp<int>(P->nitem_part);
    a.item_np = dp<int>(P->nitem_np);
    a.scale = P->opt.scale_output;
    a.phi = phi;
    if (P->n_near_items > 0) {
        TRY(near_zero_split(P, a, st));
        k_near_fp64<<<P->n_near_items, 128, 0, st>>>(P->n_near_items, a);
        P->launches++;
    }
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}
