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

