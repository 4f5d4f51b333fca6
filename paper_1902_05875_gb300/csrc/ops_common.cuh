// Structures and helpers shared by the operator translation units.
#pragma once

#include "internal.cuh"

struct TreeArrays {
    const int *layer, *level, *ix, *iy, *iz, *parent, *cfirst, *nchild, *s0, *s1, *t0, *t1, *split;
};

inline TreeArrays tree_arrays(tefmm_plan_s *P) {
    TreeArrays T;
    T.layer = dp<int>(P->n_layer);
    T.level = dp<int>(P->n_level);
    T.ix = dp<int>(P->n_ix);
    T.iy = dp<int>(P->n_iy);
    T.iz = dp<int>(P->n_iz);
    T.parent = dp<int>(P->n_parent);
    T.cfirst = dp<int>(P->n_cfirst);
    T.nchild = dp<int>(P->n_nchild);
    T.s0 = dp<int>(P->n_s0);
    T.s1 = dp<int>(P->n_s1);
    T.t0 = dp<int>(P->n_t0);
    T.t1 = dp<int>(P->n_t1);
    T.split = dp<int>(P->n_split);
    return T;
}

struct Cube {
    double lo[3];
    double side;
};

// box centre lo + (i + 0.5) * (side / 2^l), no contraction
__device__ __forceinline__ double centre(double lo, int i, double h) {
    return __dadd_rn(lo, __dmul_rn((double)i + 0.5, h));
}
__device__ __forceinline__ double box_h(double side, int l) { return side / (double)(1 << l); }

__device__ __forceinline__ double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

struct ImgView {
    const DevTerm *terms;
    const cplx *A, *Z;
    const int *lt_first, *lt_count;   // per layer: term range
    const cplx *k;
};

struct NearArgs {
    TreeArrays T;
    Cube cb;
    int p, np;
    const int *mi;
    const int *near_ptr, *near_src;
    const double *sx, *sy, *sz, *sq, *tx, *ty, *tz;
    const int *perm_t;
    const cplx *beta;
    ImgView im;
    double *phi;
};

inline ImgView img_view(tefmm_plan_s *P) {
    ImgView im;
    im.terms = dp<DevTerm>(P->d_terms);
    im.A = dp<cplx>(P->d_A);
    im.Z = dp<cplx>(P->d_Z);
    im.k = dp<cplx>(P->d_k);
    im.lt_first = dp<int>(P->d_k) == nullptr ? nullptr : (const int *)(dp<cplx>(P->d_k) + TEFMM_MAX_LAYERS);
    im.lt_count = im.lt_first + TEFMM_MAX_LAYERS;
    return im;
}

inline Cube cube_of(tefmm_plan_s *P) {
    Cube c;
    for (int d = 0; d < 3; ++d) c.lo[d] = P->lo[d];
    c.side = P->side;
    return c;
}


// offset of slice k3' in a packed cross-layer table (slice k3' holds the
// ncoef(2p - k3') derivatives of order <= 2p - k3'); a same-layer table is slice 0
__host__ __device__ inline int slice_off(int p, int k3p) {
    int o = 0;
    for (int j = 0; j < k3p; ++j) o += ncoef(2 * p - j);
    return o;
}

// Cross-layer M2L key (kind 2): level(5) lt(4) dx+3(3) dy+3(3) ls(4) iz_t(20) iz_s(20).
// Same-layer keys (kinds 0 and 1) sort before it.
__host__ __device__ inline uint64_t xkey(int l, int lt, int ls, int dx, int dy, int izt, int izs) {
    return (2ULL << 62) | ((uint64_t)l << 57) | ((uint64_t)lt << 53) | ((uint64_t)(dx + 3) << 50) |
           ((uint64_t)(dy + 3) << 47) | ((uint64_t)ls << 40) | ((uint64_t)izt << 20) | (uint64_t)izs;
}
struct XKey {
    int level, lt, ls, dx, dy, izt, izs;
};
__host__ __device__ inline XKey xkey_decode(uint64_t k) {
    XKey x;
    x.level = (int)((k >> 57) & 31);
    x.lt = (int)((k >> 53) & 15);
    x.dx = (int)((k >> 50) & 7) - 3;
    x.dy = (int)((k >> 47) & 7) - 3;
    x.ls = (int)((k >> 40) & 15);
    x.izt = (int)((k >> 20) & 0xFFFFF);
    x.izs = (int)(k & 0xFFFFF);
    return x;
}

// ------------------------------------------------------------------ derivative tables
// One derivative table per key: sum over the key's images of
// A_j D^g h0(k R_j) / g!, |g| <= 2p, by the recurrence (Sec. 3.2)
//   |g| R^2 a_g + (2|g|-1) sum_i x_i a_{g-e_i} + (|g|-1) sum_i a_{g-2e_i}
//       = i k sum_i (x_i b_{g-e_i} + b_{g-2e_i}),
//   |g| b_g = i k sum_i (x_i a_{g-e_i} + a_{g-2e_i}),
// a_0 = e^{ikR}/R, b_0 = e^{ikR}, D^g h0 / g! = a_g / (ik).
__device__ inline void recur_accumulate(int P2, int np2, const int *mi, cplx k, double X, double Y, cplx W,
                                 cplx coef, bool flip3, cplx *a, cplx *b, cplx *acc) {
    if (threadIdx.x == 0) {
        cplx R2 = mkc(X * X + Y * Y + W.x * W.x - W.y * W.y, 2.0 * W.x * W.y);
        cplx R = csqrt_p(R2);
        cplx ikR = cmul(mkc(-k.y, k.x), R);
        cplx e = cexp_(ikR);
        a[0] = cdiv(e, R);
        b[0] = e;
    }
    __syncthreads();
    cplx R2 = mkc(X * X + Y * Y + W.x * W.x - W.y * W.y, 2.0 * W.x * W.y);
    cplx ik = mkc(-k.y, k.x);
    const cplx iR2 = cdiv(mkc(1, 0), R2);
    for (int n = 1; n <= P2; ++n) {
        const double inv_n = 1.0 / n;
        int first = n * (n + 1) * (n + 2) / 6, last = (n + 1) * (n + 2) * (n + 3) / 6;
        for (int g = first + threadIdx.x; g < last; g += blockDim.x) {
            int kk[3] = {mi[3 * g], mi[3 * g + 1], mi[3 * g + 2]};
            cplx xs[3] = {mkc(X, 0), mkc(Y, 0), W};
            cplx sa1 = mkc(0, 0), sa2 = mkc(0, 0), sb = mkc(0, 0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (kk[i] >= 1) {
                    int m[3] = {kk[0], kk[1], kk[2]};
                    m[i] -= 1;
                    int j = midx(m[0], m[1], m[2]);
                    sa1 = cadd(sa1, cmul(xs[i], a[j]));
                    sb = cadd(sb, cmul(xs[i], b[j]));
                }
                if (kk[i] >= 2) {
                    int m[3] = {kk[0], kk[1], kk[2]};
                    m[i] -= 2;
                    int j = midx(m[0], m[1], m[2]);
                    sa2 = cadd(sa2, a[j]);
                    sb = cadd(sb, b[j]);
                }
            }
            cplx bg = cscale(cmul(ik, cadd(sa1, sa2)), inv_n);
            cplx num = csub(csub(cmul(ik, sb), cscale(sa1, 2.0 * n - 1.0)), cscale(sa2, n - 1.0));
            cplx ag = cscale(cmul(num, iR2), inv_n);
            a[g] = ag;
            b[g] = bg;
        }
        __syncthreads();
    }
    // acc += coef * a / (ik) * (-1)^{g3 if flip3}
    cplx c2 = cdiv(coef, ik);
    for (int g = threadIdx.x; g < np2; g += blockDim.x) {
        cplx v = cmul(c2, a[g]);
        if (flip3 && (mi[3 * g + 2] & 1)) v = mkc(-v.x, -v.y);
        acc[g] = cadd(acc[g], v);
    }
    __syncthreads();
}

