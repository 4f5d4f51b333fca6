// The layered medium's reaction densities at one spectral sample, shared by
// the DCIM fits (Sec. 3.3) and Algorithm 2's Sommerfeld-integral tables
// (Sec. 4.2): the k_z branch, the direct solve of the interface conditions of
// Sec. 2.1 and the multiple-reflection factor s_tau of a same-layer term (or
// the z'-derivative of a cross-layer density).
#pragma once

#include "internal.cuh"

namespace {

constexpr int MAXU = 16;         // unknowns of the interface solve (8 layers)

struct FitJob {
    int layer, tag, nL;
    double d[TEFMM_MAX_LAYERS];
    cplx k[TEFMM_MAX_LAYERS];
    double zmin, T0, T1;
    int n, n_images;
    // cross-layer mode (mode = 1): source layer, direction (0 up, 1 down),
    // source z-centre and z'-derivative order; zmin is then W_min
    int mode, src_layer, dir, k3p;
    double zc;
};

__host__ __device__ __forceinline__ cplx conjc(cplx a) { return mkc(a.x, -a.y); }
__host__ __device__ __forceinline__ double abs2(cplx a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs_(cplx a) { return hypot(a.x, a.y); }
__host__ __device__ __forceinline__ cplx clog_(cplx a) { return mkc(log(cabs_(a)), atan2(a.y, a.x)); }

__host__ __device__ cplx kz_of(cplx k, cplx krho2) {
    // sqrt(k^2 - k_rho^2) with Im >= 0
    cplx s = csqrt_p(csub(cmul(k, k), krho2));
    if (s.y < 0) s = mkc(-s.x, -s.y);
    return s;
}

// Interface solve at one sample: amplitudes of every layer for a unit source
// wave S1 (column 0) and S2 (column 1) of a source in layer lp.
// Unknowns: b_0, (a_1, b_1), ..., (a_{L-1}, b_{L-1}), a_L.
// Basis: up-going b e^{i kz (z - d_l)} / kz (bottom interface reference),
// down-going a e^{-i kz (z - d_{l-1})} / kz (top interface reference).
__host__ __device__ void interface_solve(const FitJob &J, int lp, const cplx *kz, cplx x[][2]) {
    const int L = J.nL - 1, nu = 2 * L;
    cplx A[MAXU][MAXU + 2];
    for (int r = 0; r < nu; ++r)
        for (int c = 0; c < nu + 2; ++c) A[r][c] = mkc(0, 0);
    for (int j = 0; j < L; ++j) {
        for (int side = 0; side < 2; ++side) {
            int m = j + side;
            double sg = side == 0 ? 1.0 : -1.0;
            cplx kw = J.k[m];
            if (m < L) {
                int col = 2 * m;
                cplx ex = cexp_(cmul(mkc(0, 1), cscale(kz[m], J.d[j] - J.d[m])));
                cplx v = cdiv(ex, kz[m]);
                cplx dv = cmul(mkc(0, 1), ex);
                A[2 * j][col] = cadd(A[2 * j][col], cscale(v, sg));
                A[2 * j + 1][col] = cadd(A[2 * j + 1][col], cscale(cmul(kw, dv), sg));
            }
            if (m > 0) {
                int col = 2 * m - 1;
                cplx ex = cexp_(cmul(mkc(0, -1), cscale(kz[m], J.d[j] - J.d[m - 1])));
                cplx v = cdiv(ex, kz[m]);
                cplx dv = cmul(mkc(0, -1), ex);
                A[2 * j][col] = cadd(A[2 * j][col], cscale(v, sg));
                A[2 * j + 1][col] = cadd(A[2 * j + 1][col], cscale(cmul(kw, dv), sg));
            }
        }
    }
    // right-hand sides: column nu = unit wave S1 (source below interface lp-1),
    // column nu+1 = unit wave S2 (source above interface lp)
    if (lp > 0) {
        int j = lp - 1;
        A[2 * j][nu] = cadd(A[2 * j][nu], cdiv(mkc(1, 0), kz[lp]));
        A[2 * j + 1][nu] = cadd(A[2 * j + 1][nu], cmul(J.k[lp], mkc(0, 1)));
    }
    if (lp < L) {
        int j = lp;
        A[2 * j][nu + 1] = csub(A[2 * j][nu + 1], cdiv(mkc(1, 0), kz[lp]));
        A[2 * j + 1][nu + 1] = csub(A[2 * j + 1][nu + 1], cmul(J.k[lp], mkc(0, -1)));
    }
    // Gaussian elimination with partial pivoting
    for (int c = 0; c < nu; ++c) {
        int piv = c;
        double best = abs2(A[c][c]);
        for (int r = c + 1; r < nu; ++r)
            if (abs2(A[r][c]) > best) {
                best = abs2(A[r][c]);
                piv = r;
            }
        if (piv != c)
            for (int q = 0; q < nu + 2; ++q) {
                cplx t = A[c][q];
                A[c][q] = A[piv][q];
                A[piv][q] = t;
            }
        cplx inv = cdiv(mkc(1, 0), A[c][c]);
        for (int r = c + 1; r < nu; ++r) {
            cplx f = cmul(A[r][c], inv);
            if (f.x == 0 && f.y == 0) continue;
            for (int q = c; q < nu + 2; ++q) A[r][q] = csub(A[r][q], cmul(f, A[c][q]));
        }
    }
    for (int r = nu - 1; r >= 0; --r)
        for (int h = 0; h < 2; ++h) {
            cplx s = A[r][nu + h];
            for (int q = r + 1; q < nu; ++q) s = csub(s, cmul(A[r][q], x[q][h]));
            x[r][h] = cdiv(s, A[r][r]);
        }
}

// The fitted function F(k_z) / e^{i k_z zmin} at one sample of layer J.layer.
// Same-layer mode: the multiple-reflection factor s_tau of the term.
// Cross-layer mode: d^{k3'}_{z'} [S2 sigma^{.u} + S1 sigma^{.d}] / k3'! at z' = zc
// (eq. ``layermediumdensity``), sigma read in the target layer J.layer.
__host__ __device__ cplx s_tau_sample(const FitJob &J, cplx kz_l) {
    const int L = J.nL - 1;
    cplx krho2 = csub(cmul(J.k[J.layer], J.k[J.layer]), cmul(kz_l, kz_l));
    cplx kz[TEFMM_MAX_LAYERS];
    for (int m = 0; m <= L; ++m) kz[m] = kz_of(J.k[m], krho2);
    cplx x[MAXU][2];
    const int l = J.layer;
    if (J.mode == 1) {
        const int lp = J.src_layer;
        interface_solve(J, lp, kz, x);
        const int row = J.dir == 0 ? 2 * l : 2 * l - 1;       // b_l (up) or a_l (down)
        cplx out = mkc(0, 0);
        double fact = 1.0;
        for (int i = 2; i <= J.k3p; ++i) fact *= i;
        cplx ikp = cmul(mkc(0, 1), kz[lp]);
        if (lp < L) {   // S2 = e^{i kz' (z' - d_l')}, d/dz' -> (i kz')
            cplx f = cexp_(cmul(mkc(0, 1), cscale(kz[lp], J.zc - J.d[lp])));
            for (int i = 0; i < J.k3p; ++i) f = cmul(f, ikp);
            out = cadd(out, cmul(f, x[row][1]));
        }
        if (lp > 0) {   // S1 = e^{i kz' (d_{l'-1} - z')}, d/dz' -> (-i kz')
            cplx f = cexp_(cmul(mkc(0, 1), cscale(kz[lp], J.d[lp - 1] - J.zc)));
            for (int i = 0; i < J.k3p; ++i) f = cmul(f, mkc(-ikp.x, -ikp.y));
            out = cadd(out, cmul(f, x[row][0]));
        }
        return cscale(out, 1.0 / fact);
    }
    interface_solve(J, l, kz, x);
    cplx eD = mkc(1, 0);
    if (l > 0 && l < L) eD = cexp_(cmul(mkc(0, -1), cscale(kz[l], J.d[l - 1] - J.d[l])));  // e^{-i kz D}
    switch (J.tag) {
        case 0: return x[2 * l][1];                       // up-up: b_l(S2)
        case 1: return x[2 * l - 1][0];                   // down-down: a_l(S1), top reference
        case 2: return cmul(x[2 * l][0], eD);             // up-down: b_l(S1) e^{-i kz D}
        default: return cmul(x[2 * l - 1][1], eD);        // down-up: a_l(S2) e^{-i kz D}
    }
}

}  // namespace
