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

// Far-of-near reading: for a pair of adjacent leaves of level l, image j of a
// same-layer term is "far" when -Re Z_j >= thr[l] = kappa_p sqrt(3) h_l,
// kappa_p = 10^(10/(p+1)) (the combined displacement of target and source from
// their leaf centres is at most sqrt(3) h_l, so a Taylor expansion of that
// image term to order p errs by about kappa_p^-(p+1) = 1e-10 of it).  Far
// images of such pairs go through M2L (key kind 2), the others through P2P.
struct FonThr {
    double thr[TEFMM_NBITS + 1];
    int on;
};

inline FonThr fon_thresholds(const tefmm_plan_s *P) {
    FonThr f{};
    f.on = P->opt.far_of_near ? 1 : 0;
    const double kap = pow(10.0, 10.0 / (double)(P->p + 1));
    for (int l = 0; l <= TEFMM_NBITS; ++l)
        f.thr[l] = f.on ? kap * sqrt(3.0) * (P->side / (double)(1 << l)) : INFINITY;
    return f;
}

struct NearArgs {
    TreeArrays T;
    Cube cb;
    int p, np;
    const int *mi;
    const int *near_ptr, *near_src;
    const int *near_fl;        // far-of-near level l* per near entry (-1: none); read when fon.on
    const int *item_node, *item_part, *item_np;   // near-field work items (leaf, chunk, chunks of the leaf)
    const double *sx, *sy, *sz, *sq, *tx, *ty, *tz;
    const int *perm_t;
    const cplx *beta;
    ImgView im;
    FonThr fon;
    int scale;                 // multiply each potential by i k_l / (4 pi) of its layer
    double *phi;
};

int near_zero_split(tefmm_plan_s *P, const NearArgs &a, cudaStream_t st);

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

// M2L keys (64 bits): kind(2) level(5) target layer(3) dx+15(5) dy+15(5) w(44).
//   kind 0 = B (same layer; w = dz + 15),
//   kind 1 = A (same layer; w = iz_t + iz_s),
//   kind 2 = far-of-near pair of adjacent leaves of one level: w = sub(1) at
//            bit 43 and, for sub 0 (B': far images of the up-down and down-up
//            terms) dz + 15, for sub 1 (A': far images of up-up and down-down)
//            iz_t + iz_s,
//   kind 3 = cross layer (w = rev(1) source layer(3) iz_t(20) iz_s(20)); sorts last.
// dx, dy, dz are the target-minus-source box offsets of a V pair.  With
// wavenumber admissibility the first translating level can pair boxes up to
// 2^level - 1 apart, so the offset fields hold |d| <= KEY_OFF.
#define KEY_OFF 15
__host__ __device__ inline uint64_t m2l_key(int kind, int l, int lay, int dx, int dy, uint64_t w) {
    return ((uint64_t)kind << 62) | ((uint64_t)l << 57) | ((uint64_t)lay << 54) |
           ((uint64_t)(dx + KEY_OFF) << 49) | ((uint64_t)(dy + KEY_OFF) << 44) | w;
}
__host__ __device__ inline int key_kind(uint64_t k) { return (int)(k >> 62); }
__host__ __device__ inline int key_level(uint64_t k) { return (int)((k >> 57) & 31); }
__host__ __device__ inline int key_layer(uint64_t k) { return (int)((k >> 54) & 7); }
__host__ __device__ inline int key_dx(uint64_t k) { return (int)((k >> 49) & 31) - KEY_OFF; }
__host__ __device__ inline int key_dy(uint64_t k) { return (int)((k >> 44) & 31) - KEY_OFF; }
__host__ __device__ inline uint64_t key_w(uint64_t k) { return k & ((1ULL << 44) - 1); }
__host__ __device__ inline bool key_is_cross(uint64_t k) { return key_kind(k) == 3; }
// the key's table is a B table (free space, up-down, down-up; or B'), else an A table
__host__ __device__ inline bool key_is_B(uint64_t k) {
    const int c = key_kind(k);
    return c == 0 || (c == 2 && !((k >> 43) & 1));
}
__host__ __device__ inline uint64_t fon_key(int l, int lay, int dx, int dy, int sub, uint64_t w) {
    return m2l_key(2, l, lay, dx, dy, ((uint64_t)sub << 43) | w);
}
// the same key with other horizontal offsets
__host__ __device__ inline uint64_t key_with_dxdy(uint64_t k, int dx, int dy) {
    return (k & ~(1023ULL << 44)) | ((uint64_t)(dx + KEY_OFF) << 49) | ((uint64_t)(dy + KEY_OFF) << 44);
}

// Cross-layer M2L key: kind 3, w = rev(1) ls(3) iz_t(20) iz_s(20).  The fields
// describe the component (lt <- ls) whose fits and table the key uses.  rev = 0:
// the V pairs of the key translate from a source box of layer ls into a target
// box of layer lt.  rev = 1 (the pair's target layer has the smaller |k|): the
// pairs run the other way, target box (layer ls, z-index izs) from source box
// (layer lt, izt, offset -dx, -dy), and use the transposed matrix of the key's
// component scaled by (k_lt / k_ls)^2 (reciprocity).
__host__ __device__ inline uint64_t xkey(int l, int lt, int ls, int dx, int dy, int izt, int izs, int rev = 0) {
    return m2l_key(3, l, lt, dx, dy,
                   ((uint64_t)rev << 43) | ((uint64_t)ls << 40) | ((uint64_t)izt << 20) | (uint64_t)izs);
}
__host__ __device__ inline int xkey_rev(uint64_t k) { return (int)((k >> 43) & 1); }
struct XKey {
    int level, lt, ls, dx, dy, izt, izs;
};
__host__ __device__ inline XKey xkey_decode(uint64_t k) {
    XKey x;
    x.level = key_level(k);
    x.lt = key_layer(k);
    x.dx = key_dx(k);
    x.dy = key_dy(k);
    x.ls = (int)((k >> 40) & 7);
    x.izt = (int)((k >> 20) & 0xFFFFF);
    x.izs = (int)(k & 0xFFFFF);
    return x;
}

// ------------------------------------------------------------------ derivative tables
// One derivative table per key: sum over the key's images of
// A_j D^g h0(k R_j) / g!, |g| <= P2, by the recurrence (Sec. 3.3)
//   |g| R^2 a_g + (2|g|-1) sum_i x_i a_{g-e_i} + (|g|-1) sum_i a_{g-2e_i}
//       = i k sum_i (x_i b_{g-e_i} + b_{g-2e_i}),
//   |g| b_g = i k sum_i (x_i a_{g-e_i} + a_{g-2e_i}),
// a_0 = e^{ikR}/R, b_0 = e^{ikR}, D^g h0 / g! = a_g / (ik).
// Order n needs orders n-1 and n-2 only, so a and b live in shared memory as
// a ring of three orders (slot n mod 3, each ncoef-level wide: cmax entries).
// Within order n the graded index of g = (k1, k2, k3) is
// loc(g) = T(k2 + k3) + k3, T(x) = x (x + 1) / 2 (so g = n(n+1)(n+2)/6 + loc(g)).
// The thread that computes a_g adds coef a_g / (ik) (times (-1)^{g3} if flip3)
// to the table entry dst[g] itself: the table is the accumulator.
__host__ __device__ inline int tri(int x) { return x * (x + 1) / 2; }

__device__ inline void recur_accumulate(int P2, int cmax, cplx k, double X, double Y, cplx W, cplx coef,
                                        bool flip3, cplx *a, cplx *b, cplx *dst) {
    const cplx ik = mkc(-k.y, k.x);
    const cplx c2 = cdiv(coef, ik);
    if (threadIdx.x == 0) {
        cplx R2 = mkc(X * X + Y * Y + W.x * W.x - W.y * W.y, 2.0 * W.x * W.y);
        cplx R = csqrt_p(R2);
        cplx ikR = cmul(ik, R);
        cplx e = cexp_(ikR);
        const cplx a0 = cdiv(e, R);
        a[0] = a0;
        b[0] = e;
        dst[0] = cadd(dst[0], cmul(c2, a0));
    }
    __syncthreads();
    const cplx R2 = mkc(X * X + Y * Y + W.x * W.x - W.y * W.y, 2.0 * W.x * W.y);
    const cplx iR2 = cdiv(mkc(1, 0), R2);
    for (int n = 1; n <= P2; ++n) {
        const double inv_n = 1.0 / n;
        const int first = n * (n + 1) * (n + 2) / 6, cnt = tri(n + 1);
        cplx *an = a + (n % 3) * cmax, *bn = b + (n % 3) * cmax;
        const cplx *a1 = a + ((n + 2) % 3) * cmax, *b1 = b + ((n + 2) % 3) * cmax;   // order n - 1
        const cplx *a2 = a + ((n + 1) % 3) * cmax, *b2 = b + ((n + 1) % 3) * cmax;   // order n - 2
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            // (k1, k2, k3) of local index i: i = T(s) + k3 with s = k2 + k3
            int s = (int)((sqrtf(8.f * (float)i + 1.f) - 1.f) * 0.5f);
            while (tri(s + 1) <= i) ++s;
            while (tri(s) > i) --s;
            const int k3 = i - tri(s), k2 = s - k3, k1 = n - s;
            const int kk[3] = {k1, k2, k3};
            cplx sa1 = mkc(0, 0), sa2 = mkc(0, 0), sb = mkc(0, 0);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (kk[d] >= 1) {
                    int m2 = kk[1] - (d == 1), m3 = kk[2] - (d == 2);
                    const int j = tri(m2 + m3) + m3;
                    if (d < 2) {   // x and y offsets are real: scale instead of a complex product
                        const double xd = d == 0 ? X : Y;
                        sa1 = cadd(sa1, cscale(a1[j], xd));
                        sb = cadd(sb, cscale(b1[j], xd));
                    } else {
                        sa1 = cadd(sa1, cmul(W, a1[j]));
                        sb = cadd(sb, cmul(W, b1[j]));
                    }
                }
                if (kk[d] >= 2) {
                    int m2 = kk[1] - 2 * (d == 1), m3 = kk[2] - 2 * (d == 2);
                    const int j = tri(m2 + m3) + m3;
                    sa2 = cadd(sa2, a2[j]);
                    sb = cadd(sb, b2[j]);
                }
            }
            const cplx bg = cscale(cmul(ik, cadd(sa1, sa2)), inv_n);
            const cplx num = csub(csub(cmul(ik, sb), cscale(sa1, 2.0 * n - 1.0)), cscale(sa2, n - 1.0));
            const cplx ag = cscale(cmul(num, iR2), inv_n);
            an[i] = ag;
            bn[i] = bg;
            cplx v = cmul(c2, ag);
            if (flip3 && (k3 & 1)) v = mkc(-v.x, -v.y);
            dst[first + i] = cadd(dst[first + i], v);
        }
        __syncthreads();
    }
}

