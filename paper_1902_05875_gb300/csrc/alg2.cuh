// Algorithm 2 lookup (Sec. 4.2): interpolation of the Sommerfeld-integral
// tables T_{m,nu,n}(rho, zeta) of a same-layer term and assembly of the
// Cartesian derivatives a_g = D^g F / g! from them (see alg2.cu for the
// construction and the formulas).
#pragma once

#include "ops_common.cuh"

struct A2Tab {                 // one term's table on the device
    const cplx *T;             // [n][n][ne]
    double rho_max, zlo, zhi;
    int n;
};

struct A2View {
    int on, P2, ne;
    const int *mi;             // multi-indices of order <= P2, graded order
    A2Tab t[TEFMM_MAX_LAYERS][4];
};

A2View a2_view(tefmm_plan_s *P);

// first index and weights of the degree-7 Lagrange stencil of x on the grid
// lo + i (hi - lo) / (n - 1), shifted inside the grid at its edges
__device__ inline void a2_stencil(double lo, double hi, int n, double x, int *i0, double *w) {
    const double step = (hi - lo) / (double)(n - 1);
    int i = (int)floor((x - lo) / step) - 3;
    i = i < 0 ? 0 : (i > n - 8 ? n - 8 : i);
    *i0 = i;
    double xs[8];
    for (int a = 0; a < 8; ++a) xs[a] = lo + step * (double)(i + a);
    for (int a = 0; a < 8; ++a) {
        double v = 1.0;
        for (int b = 0; b < 8; ++b)
            if (b != a) v *= (x - xs[b]) / (xs[a] - xs[b]);
        w[a] = v;
    }
}

// shared memory (complex units) that alg2_accumulate needs
__host__ __device__ inline int a2_smem_cplx(int P2, int ne) { return ne + 2 * P2 + 1 + 9; }

// dst[g] += a_g of the term at (X, Y, zeta), g over the np2 multi-indices of
// order <= P2, odd z-orders negated when flip3.  Block-wide (every thread of
// the block calls it with the same arguments); sm: a2_smem_cplx complex.
__device__ inline void alg2_accumulate(const A2View &v, const A2Tab &tb, double X, double Y, double zeta,
                                       bool flip3, cplx *sm, int np2, cplx *dst) {
    const int P2 = v.P2, ne = v.ne;
    cplx *Tv = sm, *E = sm + ne;
    double *wr = (double *)(E + 2 * P2 + 1), *wz = wr + 8;
    int *ij = (int *)(wz + 8);
    __syncthreads();                       // sm and dst may still be in use by the caller
    if (threadIdx.x == 0) {
        const double rho = hypot(X, Y), phi = atan2(Y, X);
        a2_stencil(0.0, tb.rho_max, tb.n, rho, &ij[0], wr);
        a2_stencil(tb.zlo, tb.zhi, tb.n, zeta, &ij[1], wz);
        for (int nu = -P2; nu <= P2; ++nu) {
            double s, c;
            sincos((double)nu * phi, &s, &c);
            E[nu + P2] = mkc(c, s);
        }
    }
    __syncthreads();
    const int i0 = ij[0], j0 = ij[1];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        cplx acc = mkc(0, 0);
        for (int a = 0; a < 8; ++a) {
            const cplx *src = tb.T + ((int64_t)(i0 + a) * tb.n + j0) * ne + e;
            cplx row = mkc(0, 0);
            for (int b = 0; b < 8; ++b) row = cadd(row, cscale(src[(int64_t)b * ne], wz[b]));
            acc = cadd(acc, cscale(row, wr[a]));
        }
        Tv[e] = acc;
    }
    __syncthreads();
    for (int g = threadIdx.x; g < np2; g += blockDim.x) {
        const int g1 = v.mi[3 * g], g2 = v.mi[3 * g + 1], g3 = v.mi[3 * g + 2];
        const int m = g1 + g2;
        int base = 0;                      // entries of the orders below m
        for (int q = 0; q < m; ++q) base += (q / 2 + 1) * (P2 - q + 1);
        const int stride = P2 - m + 1;
        cplx acc = mkc(0, 0);
        double c1 = 1.0;                   // C(g1, a1)
        for (int a1 = 0; a1 <= g1; ++a1) {
            double c2 = 1.0;               // C(g2, a2)
            for (int a2 = 0; a2 <= g2; ++a2) {
                const int a = a1 + a2, nu = 2 * a - m, anu = nu < 0 ? -nu : nu;
                double c = c1 * c2;
                if ((g2 - a2 + a) & 1) c = -c;        // (-1)^(g2 - a2) (-1)^a
                if (nu < 0 && (anu & 1)) c = -c;      // T_{m,-nu} = (-1)^nu T_{m,nu}
                const cplx t = Tv[base + ((anu - (m & 1)) >> 1) * stride + g3];
                acc = cadd(acc, cscale(cmul(E[nu + P2], t), c));
                c2 = c2 * (double)(g2 - a2) / (double)(a2 + 1);
            }
            c1 = c1 * (double)(g1 - a1) / (double)(a1 + 1);
        }
        double f = ldexp(1.0, -m);        // 2^-(g1+g2) / g!
        for (int q = 2; q <= g1; ++q) f /= q;
        for (int q = 2; q <= g2; ++q) f /= q;
        for (int q = 2; q <= g3; ++q) f /= q;
        cplx r = cscale(acc, f);
        switch (g2 & 3) {                  // times (-i)^g2
            case 1: r = mkc(r.y, -r.x); break;
            case 2: r = mkc(-r.x, -r.y); break;
            case 3: r = mkc(-r.y, r.x); break;
            default: break;
        }
        if (flip3 && (g3 & 1)) r = mkc(-r.x, -r.y);
        dst[g] = cadd(dst[g], r);
    }
    __syncthreads();
}
