// Plan-time DCIM fits on the device (Sec. 3.3, Steps 1-2), one CTA per fit.
//
// Step 1 samples, on the two paths of the k_lz plane
//   C_ap1: k_lz = i k_l (T0 + t), 0 <= t <= T1;   C_ap2: k_lz = k_l (1 - t/T0 + i t), 0 <= t <= T0,
// the function F(k_z) = s_tau(k_rho) e^{i k_z zeta_min} of one same-layer
// reaction term, where s_tau is the multiple-reflection factor of the term's
// density: the densities come from a direct solve of the interface conditions
// of Sec. 2.1 (u continuous, k-weighted flux continuous, decay at +-inf) at
// every sample.  Step 2 fits sum_j A_j e^{-i k_z Z_j} with the generalized
// pencil-of-function method (Hua & Sarkar): a Hankel data matrix, its SVD (a
// one-sided complex Jacobi method), the eigenvalues of the m x m pencil
// V2^H V1 (V1^H V1)^{-1} (Hessenberg reduction + shifted QR), and the
// amplitudes by Householder least squares.  The first level keeps only
// decaying poles; the second level fits what the first leaves on C_ap2.
#include <mutex>
#include <math.h>

#include "internal.cuh"
#include "density.cuh"

namespace {

constexpr int MAXN = 127;        // samples per level
constexpr int MAXC = 64;         // Hankel columns (pencil parameter + 1, even)
constexpr int MAXM = TEFMM_MAX_IMG;  // images per fit (both levels)
constexpr int MAXLS = 24;            // images per level
constexpr double REL_TOL = 1e-12;
constexpr double ABS_TOL = 1e-14;
constexpr double CANCEL = 1e4;     // largest image term / largest sample
constexpr double RETRY_RESID = 1e-2;   // cross-layer fit residual that triggers a longer path

// ---------------------------------------------------------------- GPOF
struct GpofSmem {
    union {
        cplx Y[MAXC][MAXC];          // column-major Hankel data (column c, row r)
        cplx Q[MAXN][MAXLS + 1];     // least-squares work (after the pencil step)
    };
    cplx V[MAXC][MAXC];      // right rotations (column c, row r)
    cplx y[MAXN];
    cplx res[MAXN];
    double sv[MAXC];
    int order[MAXC];
    int arr[MAXC];
    cplx H[MAXLS][MAXLS];
    cplx B2[MAXLS][MAXLS];
    cplx zp[MAXLS];
    cplx bb[MAXLS];
    int m;
    int nconv;
};

// one-sided Jacobi on the ncol (even) columns of Y, rows nrow; V accumulates.
__device__ void jacobi_svd(GpofSmem &S, int nrow, int ncol) {
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = threadIdx.x; c < ncol * ncol; c += blockDim.x) {
        int a = c / ncol, b = c % ncol;
        S.V[a][b] = mkc(a == b ? 1.0 : 0.0, 0.0);
    }
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) S.arr[c] = c;
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) S.nconv = 0;
        __syncthreads();
        for (int round = 0; round < ncol - 1; ++round) {
            for (int pi = warp; pi < ncol / 2; pi += nw) {
                int p = S.arr[pi], q = S.arr[ncol - 1 - pi];
                if (p > q) {
                    int t = p;
                    p = q;
                    q = t;
                }
                double al = 0, be = 0;
                cplx ga = mkc(0, 0);
                for (int r = lane; r < nrow; r += 32) {
                    cplx a = S.Y[p][r], b = S.Y[q][r];
                    al += abs2(a);
                    be += abs2(b);
                    ga = cadd(ga, cmul(conjc(a), b));
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
                    ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
                }
                double g = cabs_(ga);
                if (g > 1e-15 * sqrt(al * be) && g > 1e-300) {
                    if (lane == 0) atomicAdd(&S.nconv, 1);
                    double zeta = (be - al) / (2.0 * g);
                    double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    // rotate (y_p, e^{-i phi} y_q), whose inner product g is real
                    cplx ph = conjc(cscale(ga, 1.0 / g));   // e^{-i phi}
                    for (int r = lane; r < nrow; r += 32) {
                        cplx a = S.Y[p][r], b = S.Y[q][r];
                        cplx pb = cmul(ph, b);
                        S.Y[p][r] = csub(cscale(a, c), cscale(pb, s));
                        S.Y[q][r] = cadd(cscale(a, s), cscale(pb, c));
                    }
                    for (int r = lane; r < ncol; r += 32) {
                        cplx a = S.V[p][r], b = S.V[q][r];
                        cplx pb = cmul(ph, b);
                        S.V[p][r] = csub(cscale(a, c), cscale(pb, s));
                        S.V[q][r] = cadd(cscale(a, s), cscale(pb, c));
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int last = S.arr[ncol - 1];
                for (int i = ncol - 1; i > 1; --i) S.arr[i] = S.arr[i - 1];
                S.arr[1] = last;
            }
            __syncthreads();
        }
        if (S.nconv == 0) break;
        __syncthreads();
    }
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        double s = 0;
        for (int r = 0; r < nrow; ++r) s += abs2(S.Y[c][r]);
        S.sv[c] = sqrt(s);
    }
    __syncthreads();
}

// eigenvalues of the m x m complex matrix S.H (destroyed), single thread
__host__ __device__ void eig_small(GpofSmem &S, int n) {
    // Householder reduction to upper Hessenberg form
    for (int k = 0; k < n - 2; ++k) {
        double nx = 0;
        for (int i = k + 1; i < n; ++i) nx += abs2(S.H[i][k]);
        nx = sqrt(nx);
        if (nx == 0) continue;
        cplx x0 = S.H[k + 1][k];
        double a0 = cabs_(x0);
        cplx ph = a0 > 0 ? cscale(x0, 1.0 / a0) : mkc(1, 0);
        cplx alpha = cscale(ph, -nx);
        cplx v[MAXLS];
        for (int i = 0; i < n; ++i) v[i] = mkc(0, 0);
        for (int i = k + 1; i < n; ++i) v[i] = S.H[i][k];
        v[k + 1] = csub(v[k + 1], alpha);
        double nv = 0;
        for (int i = k + 1; i < n; ++i) nv += abs2(v[i]);
        nv = sqrt(nv);
        if (nv == 0) continue;
        for (int i = k + 1; i < n; ++i) v[i] = cscale(v[i], 1.0 / nv);
        // H = (I - 2 v v^H) H
        for (int j = 0; j < n; ++j) {
            cplx s = mkc(0, 0);
            for (int i = k + 1; i < n; ++i) s = cadd(s, cmul(conjc(v[i]), S.H[i][j]));
            for (int i = k + 1; i < n; ++i) S.H[i][j] = csub(S.H[i][j], cscale(cmul(v[i], s), 2.0));
        }
        // H = H (I - 2 v v^H)
        for (int i = 0; i < n; ++i) {
            cplx s = mkc(0, 0);
            for (int j = k + 1; j < n; ++j) s = cadd(s, cmul(S.H[i][j], v[j]));
            for (int j = k + 1; j < n; ++j) S.H[i][j] = csub(S.H[i][j], cscale(cmul(s, conjc(v[j])), 2.0));
        }
    }
    int hi = n - 1, iter = 0;
    double cs[MAXLS];
    cplx sn[MAXLS];
    while (hi >= 0) {
        if (hi == 0) {
            S.zp[0] = S.H[0][0];
            break;
        }
        int l = hi;
        for (; l > 0; --l) {
            double sc = cabs_(S.H[l][l]) + cabs_(S.H[l - 1][l - 1]);
            if (cabs_(S.H[l][l - 1]) <= 1e-16 * (sc > 0 ? sc : 1.0)) {
                S.H[l][l - 1] = mkc(0, 0);
                break;
            }
        }
        if (l == hi) {
            S.zp[hi] = S.H[hi][hi];
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 300) {       // give up: take the diagonal
            for (int i = l; i <= hi; ++i) S.zp[i] = S.H[i][i];
            hi = l - 1;
            iter = 0;
            continue;
        }
        cplx a = S.H[hi - 1][hi - 1], b = S.H[hi - 1][hi], c = S.H[hi][hi - 1], d = S.H[hi][hi];
        cplx mu;
        if (iter % 11 == 10) {
            mu = cadd(d, mkc(cabs_(c), 0));
        } else {
            cplx half = cscale(csub(a, d), 0.5);
            cplx disc = csqrt_p(cadd(cmul(half, half), cmul(b, c)));
            cplx m1 = cadd(cscale(cadd(a, d), 0.5), disc), m2 = csub(cscale(cadd(a, d), 0.5), disc);
            mu = cabs_(csub(m1, d)) < cabs_(csub(m2, d)) ? m1 : m2;
        }
        for (int i = l; i <= hi; ++i) S.H[i][i] = csub(S.H[i][i], mu);
        for (int k2 = l; k2 < hi; ++k2) {
            cplx x = S.H[k2][k2], y = S.H[k2 + 1][k2];
            double r = sqrt(abs2(x) + abs2(y));
            double c0;
            cplx s0;
            if (r == 0) {
                c0 = 1;
                s0 = mkc(0, 0);
            } else if (cabs_(x) == 0) {
                c0 = 0;
                s0 = cscale(conjc(y), 1.0 / r);
            } else {
                double ax = cabs_(x);
                c0 = ax / r;
                s0 = cscale(cmul(cscale(x, 1.0 / ax), conjc(y)), 1.0 / r);
            }
            cs[k2] = c0;
            sn[k2] = s0;
            for (int j = k2; j <= hi; ++j) {
                cplx u = S.H[k2][j], w = S.H[k2 + 1][j];
                S.H[k2][j] = cadd(cscale(u, c0), cmul(s0, w));
                S.H[k2 + 1][j] = csub(cscale(w, c0), cmul(conjc(s0), u));
            }
        }
        for (int k2 = l; k2 < hi; ++k2) {
            double c0 = cs[k2];
            cplx s0 = sn[k2];
            int top = k2 + 2 < hi ? k2 + 2 : hi;
            for (int i = l; i <= top; ++i) {
                cplx u = S.H[i][k2], w = S.H[i][k2 + 1];
                S.H[i][k2] = cadd(cscale(u, c0), cmul(conjc(s0), w));
                S.H[i][k2 + 1] = csub(cscale(w, c0), cmul(s0, u));
            }
        }
        for (int i = l; i <= hi; ++i) S.H[i][i] = cadd(S.H[i][i], mu);
    }
}

// least squares  min || sum_j b_j z_j^n - y_n ||, n < N, single thread (Householder)
__host__ __device__ void vandermonde_lsq(GpofSmem &S, int N, int m) {
    for (int n = 0; n < N; ++n) {
        for (int j = 0; j < m; ++j) {
            // z^n by repeated multiplication
            cplx v = mkc(1, 0);
            for (int e = 0; e < n; ++e) v = cmul(v, S.zp[j]);
            S.Q[n][j] = v;
        }
        S.Q[n][m] = S.res[n];
    }
    for (int j = 0; j < m; ++j) {
        double nx = 0;
        for (int i = j; i < N; ++i) nx += abs2(S.Q[i][j]);
        nx = sqrt(nx);
        if (nx == 0) continue;
        cplx x0 = S.Q[j][j];
        double a0 = cabs_(x0);
        cplx ph = a0 > 0 ? cscale(x0, 1.0 / a0) : mkc(1, 0);
        cplx alpha = cscale(ph, -nx);
        // v = x - alpha e1 stored in place below the diagonal (column j)
        cplx v0 = csub(x0, alpha);
        double nv = abs2(v0);
        for (int i = j + 1; i < N; ++i) nv += abs2(S.Q[i][j]);
        nv = sqrt(nv);
        if (nv == 0) continue;
        S.Q[j][j] = v0;
        for (int i = j; i < N; ++i) S.Q[i][j] = cscale(S.Q[i][j], 1.0 / nv);
        for (int c = j + 1; c <= m; ++c) {
            cplx s = mkc(0, 0);
            for (int i = j; i < N; ++i) s = cadd(s, cmul(conjc(S.Q[i][j]), S.Q[i][c]));
            for (int i = j; i < N; ++i) S.Q[i][c] = csub(S.Q[i][c], cscale(cmul(S.Q[i][j], s), 2.0));
        }
        S.Q[j][j] = alpha;   // R diagonal
        for (int i = j + 1; i < N; ++i) S.Q[i][j] = mkc(0, 0);
    }
    for (int j = m - 1; j >= 0; --j) {
        cplx s = S.Q[j][m];
        for (int c = j + 1; c < m; ++c) s = csub(s, cmul(S.Q[j][c], S.bb[c]));
        S.bb[j] = cdiv(s, S.Q[j][j]);
    }
}

// GPOF, first stage (all threads): Hankel data matrix of S.res[0..N), its SVD,
// singular values ordered; S.m = number above max(REL_TOL sigma_0, ABS_TOL N).
__device__ void gpof_svd(GpofSmem &S, int N) {
    const int Lp = N / 2;
    const int nrow = N - Lp, ncolr = Lp + 1;
    const int ncol = (ncolr + 1) & ~1;
    for (int e = threadIdx.x; e < ncol * MAXC; e += blockDim.x) {
        int c = e / MAXC, r = e % MAXC;
        S.Y[c][r] = (c < ncolr && r < nrow) ? S.res[r + c] : mkc(0, 0);
    }
    __syncthreads();
    jacobi_svd(S, nrow, ncol);
    if (threadIdx.x == 0) {
        for (int c = 0; c < ncol; ++c) S.order[c] = c;
        for (int i = 1; i < ncol; ++i) {      // sort by singular value, descending
            int v = S.order[i], j = i - 1;
            while (j >= 0 && S.sv[S.order[j]] < S.sv[v]) {
                S.order[j + 1] = S.order[j];
                --j;
            }
            S.order[j + 1] = v;
        }
        double smax = S.sv[S.order[0]];
        double thr = fmax(REL_TOL * smax, ABS_TOL * N);
        int m = 0;
        while (m < ncol && S.sv[S.order[m]] > thr) ++m;
        S.m = m;
    }
    __syncthreads();
}

// GPOF, second stage (one thread): poles and amplitudes for model order m.
// Pencil Zmat = V2^H V1 (V1^H V1)^{-1} (V1, V2: rows 0..Lp-1 and 1..Lp of the m
// leading right singular vectors); keeps |z| < 1 if ``decaying`` and poles with
// Re(log(z)/c) < 0 (images with Re Z < 0); amplitudes by least squares.
// Returns the number of poles kept (in S.zp, S.bb).
__host__ __device__ int gpof_order(GpofSmem &S, int N, int m, bool decaying, cplx c) {
    const int Lp = N / 2;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            cplx g = mkc(0, 0), h = mkc(0, 0);
            const cplx *va = S.V[S.order[a]], *vb = S.V[S.order[b]];
            for (int r = 0; r < Lp; ++r) {
                g = cadd(g, cmul(conjc(va[r]), vb[r]));
                h = cadd(h, cmul(conjc(va[r + 1]), vb[r]));
            }
            S.H[a][b] = g;   // V1^H V1
            S.B2[a][b] = h;  // V2^H V1
        }
    // solve (V1^H V1) X = V2^H V1 by Gauss-Jordan elimination, X -> H
    for (int cc = 0; cc < m; ++cc) {
        int piv = cc;
        for (int r = cc + 1; r < m; ++r)
            if (abs2(S.H[r][cc]) > abs2(S.H[piv][cc])) piv = r;
        for (int q = 0; q < m; ++q) {
            cplx t = S.H[cc][q];
            S.H[cc][q] = S.H[piv][q];
            S.H[piv][q] = t;
            t = S.B2[cc][q];
            S.B2[cc][q] = S.B2[piv][q];
            S.B2[piv][q] = t;
        }
        cplx inv = cdiv(mkc(1, 0), S.H[cc][cc]);
        for (int r = 0; r < m; ++r) {
            if (r == cc) continue;
            cplx f = cmul(S.H[r][cc], inv);
            for (int q = 0; q < m; ++q) {
                S.H[r][q] = csub(S.H[r][q], cmul(f, S.H[cc][q]));
                S.B2[r][q] = csub(S.B2[r][q], cmul(f, S.B2[cc][q]));
            }
        }
        for (int q = 0; q < m; ++q) S.B2[cc][q] = cmul(S.B2[cc][q], inv);
        for (int q = 0; q < m; ++q) S.H[cc][q] = cmul(S.H[cc][q], inv);
    }
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) S.H[a][b] = S.B2[a][b];
    eig_small(S, m);
    int w = 0;
    for (int j = 0; j < m; ++j) {
        cplx z = S.zp[j];
        if (decaying && !(cabs_(z) < 1.0)) continue;
        if (!(cdiv(clog_(z), c).x < 0.0)) continue;
        S.zp[w++] = z;
    }
    if (w > 0) vandermonde_lsq(S, N, w);
    return w;
}

__host__ __device__ __forceinline__ cplx path1(cplx k, double T0, double dt1, int i) {
    return cmul(mkc(0, 1), cscale(k, T0 + i * dt1));                  // C_ap1
}
__host__ __device__ __forceinline__ cplx path2(cplx k, double T0, double dt2, int i) {
    double t = i * dt2;
    return cmul(k, mkc(1.0 - t / T0, t));                              // C_ap2
}

__device__ __forceinline__ double finite_or_inf(double v) { return v <= 1.7e308 ? v : INFINITY; }

__device__ double block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < nw; ++w) r = fmax(r, red[w]);
    return r;
}

// Candidate images CA/CZ (nc) on top of fixed images FA/FZ (nf), every thread
// of the block: the largest candidate term on both paths (tmax) and the
// largest residual against the samples (rmax; path 1 only unless both_paths).
// A NaN or infinity anywhere gives +inf.
__device__ void cand_eval(const cplx *FA, const cplx *FZ, int nf, const cplx *CA, const cplx *CZ, int nc,
                          cplx k, double T0, double dt1, double dt2, int N, const cplx *y1,
                          const cplx *y2, bool both_paths, double *red, double &tmax, double &rmax) {
    double tm = 0.0, rm = 0.0;
    for (int n = threadIdx.x; n < 2 * N; n += blockDim.x) {
        const int lev = n / N, i = n % N;
        const cplx kz = lev == 0 ? path1(k, T0, dt1, i) : path2(k, T0, dt2, i);
        const cplx mikz = cmul(mkc(0, -1), kz);
        cplx ap = mkc(0, 0);
        for (int j = 0; j < nc; ++j) {
            cplx e = cmul(CA[j], cexp_(cmul(mikz, CZ[j])));
            tm = fmax(tm, finite_or_inf(cabs_(e)));
            ap = cadd(ap, e);
        }
        if (lev == 0 || both_paths) {
            for (int j = 0; j < nf; ++j) ap = cadd(ap, cmul(FA[j], cexp_(cmul(mikz, FZ[j]))));
            rm = fmax(rm, finite_or_inf(cabs_(csub(ap, lev == 0 ? y1[i] : y2[i]))));
        }
    }
    tmax = block_max(tm, red);
    rmax = block_max(rm, red);
}

__global__ void __launch_bounds__(512) k_fit(const FitJob *jobs, int njobs, cplx *outA, cplx *outZ, int *outN,
                      double *outRes) {
    int jb = blockIdx.x;
    if (jb >= njobs) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    GpofSmem &S = *reinterpret_cast<GpofSmem *>(smraw);
    const FitJob J = jobs[jb];
    const int N = J.n;
    const cplx k = J.k[J.layer];
    const double T0 = J.T0, T1 = J.T1;
    const double dt1 = T1 / (N - 1), dt2 = T0 / (N - 1);
    const cplx c1 = cscale(k, dt1);                                      // z = e^{c1 Z}
    const cplx c2 = cscale(cmul(cmul(mkc(0, -1), k), mkc(-1.0 / T0, 1.0)), dt2);   // -i k (i - 1/T0) dt2
    __shared__ cplx y1[MAXN], y2[MAXN], A1[MAXM], Z1[MAXM];
    __shared__ int n1;
    __shared__ double scale;
    // Step 1: samples
    for (int n = threadIdx.x; n < 2 * N; n += blockDim.x) {
        int lev = n / N, i = n % N;
        cplx kz = lev == 0 ? path1(k, T0, dt1, i) : path2(k, T0, dt2, i);
        cplx F = cmul(s_tau_sample(J, kz), cexp_(cmul(mkc(0, 1), cscale(kz, J.zmin))));
        if (lev == 0) y1[i] = F;
        else y2[i] = F;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sc = 1e-300;
        for (int i = 0; i < N; ++i) sc = fmax(sc, fmax(cabs_(y1[i]), cabs_(y2[i])));
        scale = sc;
    }
    // level 1: among the model orders whose image terms stay below CANCEL
    // times the samples on both paths, the one with the smallest residual on
    // C_ap1 (ties: the larger order)
    __shared__ cplx cA[MAXLS], cZ[MAXLS];
    __shared__ int cw, cap;
    __shared__ double bres, red[32];
    for (int i = threadIdx.x; i < N; i += blockDim.x) S.res[i] = y1[i];
    __syncthreads();
    gpof_svd(S, N);
    if (threadIdx.x == 0) {
        cap = min(S.m, min(J.n_images / 2, MAXLS));
        n1 = 0;
        bres = INFINITY;
    }
    __syncthreads();
    for (int m = cap; m >= 1; --m) {
        if (threadIdx.x == 0) {
            cw = gpof_order(S, N, m, true, c1);
            for (int j = 0; j < cw; ++j) {
                cZ[j] = cdiv(clog_(S.zp[j]), c1);                               // z = e^{k dt1 Z}
                cA[j] = cmul(S.bb[j], cexp_(cscale(cmul(k, cZ[j]), -T0)));      // A = b e^{-k T0 Z}
            }
        }
        __syncthreads();
        if (cw > 0) {
            double tmax, rmax;
            cand_eval(nullptr, nullptr, 0, cA, cZ, cw, k, T0, dt1, dt2, N, y1, y2, false, red, tmax, rmax);
            if (threadIdx.x == 0 && tmax <= CANCEL * scale && rmax < bres) {
                for (int j = 0; j < cw; ++j) {
                    A1[j] = cA[j];
                    Z1[j] = cZ[j];
                }
                n1 = cw;
                bres = rmax;
            }
        }
        __syncthreads();
    }
    // level 2 on the residual
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        cplx kz = path2(k, T0, dt2, i);
        cplx s = y2[i];
        for (int j = 0; j < n1; ++j)
            s = csub(s, cmul(A1[j], cexp_(cmul(mkc(0, -1), cmul(kz, Z1[j])))));
        S.res[i] = s;
    }
    __syncthreads();
    gpof_svd(S, N);
    // level 2: same rule, residual of all images on both paths
    __shared__ cplx bA[MAXLS], bZ[MAXLS];
    __shared__ int n2;
    if (threadIdx.x == 0) {
        cap = min(S.m, min(J.n_images - n1, MAXLS));
        n2 = 0;
        bres = INFINITY;
    }
    __syncthreads();
    for (int m = cap; m >= 1; --m) {
        if (threadIdx.x == 0) {
            cw = gpof_order(S, N, m, false, c2);
            for (int j = 0; j < cw; ++j) {
                cZ[j] = cdiv(clog_(S.zp[j]), c2);
                cA[j] = cmul(S.bb[j], cexp_(cmul(mkc(0, 1), cmul(k, cZ[j]))));   // A = b e^{ikZ}
            }
        }
        __syncthreads();
        if (cw > 0) {
            double tmax, rmax;
            cand_eval(A1, Z1, n1, cA, cZ, cw, k, T0, dt1, dt2, N, y1, y2, true, red, tmax, rmax);
            if (threadIdx.x == 0 && tmax <= CANCEL * scale && rmax < bres) {
                for (int j = 0; j < cw; ++j) {
                    bA[j] = cA[j];
                    bZ[j] = cZ[j];
                }
                n2 = cw;
                bres = rmax;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int j = 0; j < n1; ++j) {
            outA[jb * MAXM + tot] = A1[j];
            outZ[jb * MAXM + tot] = Z1[j];
            ++tot;
        }
        for (int j = 0; j < n2; ++j) {
            outA[jb * MAXM + tot] = bA[j];
            outZ[jb * MAXM + tot] = bZ[j];
            ++tot;
        }
        outN[jb] = tot;
        // residual on both paths, relative to the largest sample
        double res = 0;
        for (int lev = 0; lev < 2; ++lev)
            for (int i = 0; i < N; ++i) {
                cplx kz = lev == 0 ? path1(k, T0, dt1, i) : path2(k, T0, dt2, i);
                cplx sm = lev == 0 ? y1[i] : y2[i];
                cplx ap = mkc(0, 0);
                for (int j = 0; j < tot; ++j)
                    ap = cadd(ap, cmul(outA[jb * MAXM + j], cexp_(cmul(mkc(0, -1), cmul(kz, outZ[jb * MAXM + j])))));
                res = fmax(res, cabs_(csub(ap, sm)));
            }
        outRes[jb] = res / scale;
    }
}

}  // namespace

int plan_fit_images(tefmm_plan_s *P, cudaStream_t st) {
    P->A.clear();
    P->Z.clear();
    P->fit_max_resid = 0;
    if (P->terms.empty() || P->opt.n_images == 0) {
        for (auto &t : P->terms) t.first = t.count = 0;
        return TEFMM_OK;
    }
    if (P->nL > 8 || P->opt.n_samples > MAXN) return TEFMM_ERR_NOT_IMPLEMENTED;
    // one job per term; the down-up term reuses the up-down fit (same s_tau, zeta_min)
    std::vector<FitJob> jobs;
    std::vector<int> job_of(P->terms.size(), -1);
    double kmax = 0;
    for (int l = 0; l < P->nL; ++l) kmax = fmax(kmax, P->k[l].x);
    for (size_t i = 0; i < P->terms.size(); ++i) {
        const TermDesc &t = P->terms[i];
        if (t.tag == 3 && i > 0 && P->terms[i - 1].tag == 2 && P->terms[i - 1].layer == t.layer) {
            job_of[i] = job_of[i - 1];
            continue;
        }
        FitJob J{};
        J.mode = 0;
        J.layer = t.layer;
        J.tag = t.tag;
        J.nL = P->nL;
        for (int m = 0; m < TEFMM_MAX_LAYERS; ++m) {
            J.d[m] = m < P->nL - 1 ? P->d[m] : 0.0;
            J.k[m] = m < P->nL ? P->k[m] : mkc(1, 0);
        }
        J.zmin = t.zmin;
        double kl = P->k[t.layer].x;
        J.T0 = P->opt.T0 > 0 ? P->opt.T0 : sqrt(fmax(((kmax + 0.8) / kl) * ((kmax + 0.8) / kl) - 1.0, 1e-6));
        J.T1 = P->opt.T1;
        J.n = P->opt.n_samples;
        J.n_images = P->opt.n_images;
        job_of[i] = (int)jobs.size();
        jobs.push_back(J);
    }
    int nj = (int)jobs.size();
    FitJob *djobs = nullptr;
    cplx *dA = nullptr, *dZ = nullptr;
    int *dN = nullptr;
    double *dR = nullptr;
    CUDA_TRY(cudaMalloc(&djobs, nj * sizeof(FitJob)));
    CUDA_TRY(cudaMalloc(&dA, nj * MAXM * sizeof(cplx)));
    CUDA_TRY(cudaMalloc(&dZ, nj * MAXM * sizeof(cplx)));
    CUDA_TRY(cudaMalloc(&dN, nj * sizeof(int)));
    CUDA_TRY(cudaMalloc(&dR, nj * sizeof(double)));
    CUDA_TRY(cudaMemcpyAsync(djobs, jobs.data(), nj * sizeof(FitJob), cudaMemcpyHostToDevice, st));
    size_t sm = sizeof(GpofSmem);
    CUDA_TRY(cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_fit<<<nj, 512, sm, st>>>(djobs, nj, dA, dZ, dN, dR);
    CUDA_TRY(cudaGetLastError());
    std::vector<cplx> hA(nj * MAXM), hZ(nj * MAXM);
    std::vector<int> hN(nj);
    std::vector<double> hR(nj);
    CUDA_TRY(cudaMemcpyAsync(hA.data(), dA, nj * MAXM * sizeof(cplx), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hZ.data(), dZ, nj * MAXM * sizeof(cplx), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hN.data(), dN, nj * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hR.data(), dR, nj * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(djobs);
    cudaFree(dA);
    cudaFree(dZ);
    cudaFree(dN);
    cudaFree(dR);
    if (inject_fit_failure()) return TEFMM_ERR_FIT_FAILED;
    for (size_t i = 0; i < P->terms.size(); ++i) {
        int jb = job_of[i];
        TermDesc &t = P->terms[i];
        t.first = (int)P->A.size();
        t.count = hN[jb];
        for (int j = 0; j < hN[jb]; ++j) {
            P->A.push_back(hA[jb * MAXM + j]);
            P->Z.push_back(hZ[jb * MAXM + j]);
        }
        if (!(hR[jb] == hR[jb])) return TEFMM_ERR_FIT_FAILED;
        P->fit_max_resid = fmax(P->fit_max_resid, hR[jb]);
    }
    return TEFMM_OK;
}

// ---------------------------------------------------------------------------
// tefmm_fit_images_noalloc: the device DCIM fit without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need the images
// of a medium: frameworks that hand all device memory to their own pool
// allocator up front (a stray cudaMalloc can fail or fragment that pool), and
// latency-sensitive loops that must not hit the implicit device-wide
// synchronisation of an allocation.  This entry point runs the same fit kernel as
// tefmm_plan_create, with its job descriptors and per-fit results held in the
// fixed array below instead of freshly allocated scratch; the caller passes
// the medium in and receives the images in its own host arrays.
//
// The array lives in this library's module and is held by every device that
// loads the library until the process exits.  Its device address is looked up
// once per device (cudaGetSymbolAddress, with that device current, under a
// mutex so that concurrent first calls do not race on the lookup) on the
// first call made on that device; that first call should therefore come
// before any stream capture.  The address is kept for the process: a caller
// that resets the device (cudaDeviceReset) must not call this entry point on
// that device afterwards.  All calls share the array: two calls whose work
// overlaps on the GPU (different streams or host threads) race on it, so such
// calls must be serialised by the caller.
namespace {
constexpr int NOALLOC_MAX_FITS = 4 * 8;     // 8 layers x 4 reaction terms
struct NoAllocScratch {
    FitJob jobs[NOALLOC_MAX_FITS];
    cplx A[NOALLOC_MAX_FITS * MAXM];
    cplx Z[NOALLOC_MAX_FITS * MAXM];
    int N[NOALLOC_MAX_FITS];
    double R[NOALLOC_MAX_FITS];
};

struct NaTerm {
    int layer, tag;
    double zmin;
};

// the same-layer reaction terms of tefmm_plan_create, in the same order
int noalloc_terms(int nL, const double *d, const double *zext, NaTerm *out) {
    const int L = nL - 1;
    int n = 0;
    for (int l = 0; l <= L && L > 0; ++l) {
        double zlo = zext[2 * l], zhi = zext[2 * l + 1];
        if (l < L) out[n++] = NaTerm{l, 0, 2.0 * zlo - 2.0 * d[l]};
        if (l > 0) out[n++] = NaTerm{l, 1, 2.0 * d[l - 1] - 2.0 * zhi};
        if (l > 0 && l < L) {
            double D = d[l - 1] - d[l];
            out[n++] = NaTerm{l, 2, (zlo - zhi) + 2.0 * D};
            out[n++] = NaTerm{l, 3, (zlo - zhi) + 2.0 * D};
        }
    }
    return n;
}
}  // namespace

static __device__ __align__(256) unsigned char g_fit_scratch[sizeof(NoAllocScratch)];

static void *g_fit_scratch_addr[64];
static bool g_fit_scratch_ready[64];
static std::mutex g_fit_scratch_mutex;

extern "C" int tefmm_fit_images_noalloc(int n_layers, const double *interfaces, const double *k_re,
                                        const double *k_im, const tefmm_options *opt, void *stream,
                                        int *n_terms, int *term_layer, int *term_tag,
                                        int *term_count, double *A, double *Z) {
    // the argument checks of tefmm_plan_create
    if (n_layers < 1 || n_layers > 8 || !k_re || !k_im) return TEFMM_ERR_INVALID_ARG;
    if (n_layers > 1 && !interfaces) return TEFMM_ERR_INVALID_ARG;
    if (!n_terms || !term_count || !A || !Z) return TEFMM_ERR_INVALID_ARG;
    for (int m = 0; m + 1 < n_layers - 1; ++m)
        if (!(interfaces[m] > interfaces[m + 1])) return TEFMM_ERR_INVALID_ARG;
    for (int l = 0; l < n_layers; ++l)
        if (!(k_im[l] >= 0.0) || !(k_re[l] > 0.0)) return TEFMM_ERR_INVALID_ARG;
    tefmm_options o;
    if (opt) o = *opt;
    else tefmm_default_options(&o);
    if (o.n_images < 0 || o.n_images > TEFMM_MAX_IMG || o.n_samples < 8 || o.n_samples > MAXN ||
        !(o.T1 > 0))
        return TEFMM_ERR_INVALID_ARG;
    for (int l = 0; l < n_layers; ++l) {
        double top = (l == 0) ? (n_layers > 1 ? interfaces[0] + 1.0 : 1.0) : interfaces[l - 1];
        double bot = (l == n_layers - 1) ? (n_layers > 1 ? interfaces[n_layers - 2] - 1.0 : -1.0)
                                         : interfaces[l];
        if (isnan(o.zext[2 * l])) o.zext[2 * l] = bot;
        if (isnan(o.zext[2 * l + 1])) o.zext[2 * l + 1] = top;
        if (!(o.zext[2 * l] <= o.zext[2 * l + 1])) return TEFMM_ERR_INVALID_ARG;
        if (l > 0 && o.zext[2 * l + 1] > interfaces[l - 1]) return TEFMM_ERR_INVALID_ARG;
        if (l < n_layers - 1 && o.zext[2 * l] < interfaces[l]) return TEFMM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double d[TEFMM_MAX_LAYERS] = {0};
    cplx k[TEFMM_MAX_LAYERS];
    for (int m = 0; m < n_layers - 1; ++m) d[m] = interfaces[m];
    for (int l = 0; l < n_layers; ++l) k[l] = mkc(k_re[l], k_im[l]);
    NaTerm terms[NOALLOC_MAX_FITS];
    const int nterms = noalloc_terms(n_layers, d, o.zext, terms);
    *n_terms = nterms;
    for (int i = 0; i < nterms; ++i) {
        if (term_layer) term_layer[i] = terms[i].layer;
        if (term_tag) term_tag[i] = terms[i].tag;
        term_count[i] = 0;
    }
    if (nterms == 0 || o.n_images == 0) return TEFMM_OK;
    // one job per term; the down-up term of an interior layer reuses the
    // up-down fit, as in tefmm_plan_create
    FitJob jobs[NOALLOC_MAX_FITS];
    int job_of[NOALLOC_MAX_FITS];
    double kmax = 0;
    for (int l = 0; l < n_layers; ++l) kmax = fmax(kmax, k[l].x);
    int nj = 0;
    for (int i = 0; i < nterms; ++i) {
        if (terms[i].tag == 3 && i > 0 && terms[i - 1].tag == 2 && terms[i - 1].layer == terms[i].layer) {
            job_of[i] = job_of[i - 1];
            continue;
        }
        FitJob J{};
        J.mode = 0;
        J.layer = terms[i].layer;
        J.tag = terms[i].tag;
        J.nL = n_layers;
        for (int m = 0; m < TEFMM_MAX_LAYERS; ++m) {
            J.d[m] = m < n_layers - 1 ? d[m] : 0.0;
            J.k[m] = m < n_layers ? k[m] : mkc(1, 0);
        }
        J.zmin = terms[i].zmin;
        double kl = k[J.layer].x;
        J.T0 = o.T0 > 0 ? o.T0 : sqrt(fmax(((kmax + 0.8) / kl) * ((kmax + 0.8) / kl) - 1.0, 1e-6));
        J.T1 = o.T1;
        J.n = o.n_samples;
        J.n_images = o.n_images;
        job_of[i] = nj;
        jobs[nj++] = J;
    }
    // set-up, once per device: the device address of the fixed scratch array
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return TEFMM_ERR_INVALID_ARG;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_fit_scratch_mutex);
        if (!g_fit_scratch_ready[dev]) {
            void *ptr = nullptr;
            CUDA_TRY(cudaGetSymbolAddress(&ptr, g_fit_scratch));
            g_fit_scratch_addr[dev] = ptr;
            g_fit_scratch_ready[dev] = true;
        }
        scratch = g_fit_scratch_addr[dev];
    }
    NoAllocScratch *S = reinterpret_cast<NoAllocScratch *>(scratch);
    CUDA_TRY(cudaMemcpyAsync(S->jobs, jobs, nj * sizeof(FitJob), cudaMemcpyHostToDevice, st));
    // counts and residuals start at zero; images are written up to the counts
    CUDA_TRY(cudaMemsetAsync(S->N, 0, sizeof(S->N), st));
    CUDA_TRY(cudaMemsetAsync(S->R, 0, sizeof(S->R), st));
    size_t sm = sizeof(GpofSmem);
    CUDA_TRY(cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_fit<<<nj, 512, sm, st>>>(S->jobs, nj, S->A, S->Z, S->N, S->R);
    CUDA_TRY(cudaGetLastError());
    cplx hA[NOALLOC_MAX_FITS * MAXM], hZ[NOALLOC_MAX_FITS * MAXM];
    int hN[NOALLOC_MAX_FITS];
    double hR[NOALLOC_MAX_FITS];
    CUDA_TRY(cudaMemcpyAsync(hA, S->A, nj * MAXM * sizeof(cplx), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hZ, S->Z, nj * MAXM * sizeof(cplx), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hN, S->N, nj * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hR, S->R, nj * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < nterms; ++i) {
        int jb = job_of[i];
        if (!(hR[jb] == hR[jb])) return TEFMM_ERR_FIT_FAILED;
        term_count[i] = hN[jb];
        for (int j = 0; j < hN[jb]; ++j) {
            A[2 * (i * MAXM + j)] = hA[jb * MAXM + j].x;
            A[2 * (i * MAXM + j) + 1] = hA[jb * MAXM + j].y;
            Z[2 * (i * MAXM + j)] = hZ[jb * MAXM + j].x;
            Z[2 * (i * MAXM + j) + 1] = hZ[jb * MAXM + j].y;
        }
    }
    return TEFMM_OK;
}

// ---------------------------------------------------------------------------
// Cross-layer fits (Sec. 3.3: one DCIM fit per source z-centre and k3', for a
// component whose source and target layers differ).  Runs the fit kernel on
// the given jobs and appends the images to the plan's cross-layer pool.
int fit_cross_jobs(tefmm_plan_s *P, const std::vector<CrossFitKey> &keys, cudaStream_t st) {
    const int nj = (int)keys.size();
    if (nj == 0) return TEFMM_OK;
    if (P->nL > 8 || P->opt.n_samples > MAXN) return TEFMM_ERR_NOT_IMPLEMENTED;
    double kmax = 0;
    for (int l = 0; l < P->nL; ++l) kmax = fmax(kmax, P->k[l].x);
    std::vector<FitJob> jobs(nj);
    for (int i = 0; i < nj; ++i) {
        const CrossFitKey &c = keys[i];
        FitJob J{};
        J.mode = 1;
        J.layer = c.lt;
        J.src_layer = c.ls;
        J.dir = c.dir;
        J.k3p = c.k3p;
        J.nL = P->nL;
        for (int m = 0; m < TEFMM_MAX_LAYERS; ++m) {
            J.d[m] = m < P->nL - 1 ? P->d[m] : 0.0;
            J.k[m] = m < P->nL ? P->k[m] : mkc(1, 0);
        }
        // source z-centre: the box centre clamped to the source layer's slab
        double h = P->side / (double)(1 << c.level);
        double zc = P->lo[2] + ((double)c.izs + 0.5) * h;
        J.zc = fmin(fmax(zc, P->opt.zext[2 * c.ls]), P->opt.zext[2 * c.ls + 1]);
        J.zmin = cross_wmin(P, c.lt, c.dir);
        double kl = P->k[c.lt].x;
        J.T0 = P->opt.T0 > 0 ? P->opt.T0 : sqrt(fmax(((kmax + 0.8) / kl) * ((kmax + 0.8) / kl) - 1.0, 1e-6));
        J.T1 = P->opt.T1;
        J.n = P->opt.n_samples;
        J.n_images = P->opt.n_images;
        jobs[i] = J;
    }
    FitJob *djobs = nullptr;
    cplx *dA = nullptr, *dZ = nullptr;
    int *dN = nullptr;
    double *dR = nullptr;
    CUDA_TRY(cudaMalloc(&djobs, nj * sizeof(FitJob)));
    CUDA_TRY(cudaMalloc(&dA, (size_t)nj * MAXM * sizeof(cplx)));
    CUDA_TRY(cudaMalloc(&dZ, (size_t)nj * MAXM * sizeof(cplx)));
    CUDA_TRY(cudaMalloc(&dN, nj * sizeof(int)));
    CUDA_TRY(cudaMalloc(&dR, nj * sizeof(double)));
    CUDA_TRY(cudaMemcpyAsync(djobs, jobs.data(), nj * sizeof(FitJob), cudaMemcpyHostToDevice, st));
    size_t sm = sizeof(GpofSmem);
    CUDA_TRY(cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_fit<<<nj, 512, sm, st>>>(djobs, nj, dA, dZ, dN, dR);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    std::vector<cplx> hA((size_t)nj * MAXM), hZ((size_t)nj * MAXM);
    std::vector<int> hN(nj);
    std::vector<double> hR(nj);
    auto fetch = [&]() -> int {
        CUDA_TRY(cudaMemcpyAsync(hA.data(), dA, hA.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(hZ.data(), dZ, hZ.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(hN.data(), dN, nj * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(hR.data(), dR, nj * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return TEFMM_OK;
    };
    TRY(fetch());
    // Fits whose residual exceeds RETRY_RESID of the largest sample are
    // repeated on a first-level path that reaches past the peak of
    // |k_z|^{k3'} e^{-|k_z| d_eff}: |k| (T0 + T1) = (k3' + 5) / d_eff, with
    // d_eff = W_min + the source centre's distance to its nearest interface.
    std::vector<int> redo;
    for (int i = 0; i < nj; ++i) {
        if (!(hR[i] > RETRY_RESID)) continue;
        FitJob &J = jobs[i];
        double ds = 1e300;
        if (J.src_layer > 0) ds = fmin(ds, J.d[J.src_layer - 1] - J.zc);
        if (J.src_layer < J.nL - 1) ds = fmin(ds, J.zc - J.d[J.src_layer]);
        const cplx kl = J.k[J.layer];
        const double T1x = (J.k3p + 5.0) / (J.zmin + ds) / hypot(kl.x, kl.y) - J.T0;
        if (T1x > J.T1) {
            J.T1 = T1x;
            redo.push_back(i);
        }
    }
    if (!redo.empty()) {
        const int nr = (int)redo.size();
        std::vector<FitJob> rj(nr);
        for (int i = 0; i < nr; ++i) rj[i] = jobs[redo[i]];
        CUDA_TRY(cudaMemcpyAsync(djobs, rj.data(), nr * sizeof(FitJob), cudaMemcpyHostToDevice, st));
        k_fit<<<nr, 512, sm, st>>>(djobs, nr, dA, dZ, dN, dR);
        P->launches++;
        CUDA_TRY(cudaGetLastError());
        std::vector<cplx> rA((size_t)nr * MAXM), rZ((size_t)nr * MAXM);
        std::vector<int> rN(nr);
        std::vector<double> rR(nr);
        CUDA_TRY(cudaMemcpyAsync(rA.data(), dA, rA.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(rZ.data(), dZ, rZ.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(rN.data(), dN, nr * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(rR.data(), dR, nr * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < nr; ++i) {
            const int j = redo[i];
            for (int m = 0; m < MAXM; ++m) {
                hA[(size_t)j * MAXM + m] = rA[(size_t)i * MAXM + m];
                hZ[(size_t)j * MAXM + m] = rZ[(size_t)i * MAXM + m];
            }
            hN[j] = rN[i];
            hR[j] = rR[i];
        }
    }
    cudaFree(djobs);
    cudaFree(dA);
    cudaFree(dZ);
    cudaFree(dN);
    cudaFree(dR);
    if (inject_fit_failure()) return TEFMM_ERR_FIT_FAILED;
    for (int i = 0; i < nj; ++i) {
        if (!(hR[i] == hR[i])) return TEFMM_ERR_FIT_FAILED;
        CrossFitVal v;
        v.first = (int)P->xA.size();
        v.count = hN[i];
        for (int j = 0; j < hN[i]; ++j) {
            P->xA.push_back(hA[(size_t)i * MAXM + j]);
            P->xZ.push_back(hZ[(size_t)i * MAXM + j]);
        }
        P->xcache[keys[i]] = v;
        P->fit_max_resid_cross = fmax(P->fit_max_resid_cross, hR[i]);
    }
    return TEFMM_OK;
}
