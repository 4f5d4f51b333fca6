// Algorithm 2 (Sec. 4.2, TEFMM-II): the same-layer reaction derivatives of
// the M2L from precomputed tables of Sommerfeld integrals instead of complex
// images.
//
// A same-layer reaction term tau of layer l, with image distance
// zeta = sz z + sz' z' + c (> 0 inside the layer), is
//   F_tau(X, Y, zeta) = (1/k) int_0^inf k_rho J_0(k_rho rho) e^{i k_z zeta} s_tau(k_rho) / k_z dk_rho,
// rho = |(X, Y)|.  With D+- = d_x +- i d_y (eq. ``sysdifferential``),
// D+^a D-^b d_zeta^n F = (-1)^a e^{i (a-b) phi} T_{a+b, a-b, n}(rho, zeta) with
//   T_{m,nu,n}(rho, zeta) = (1/k) int k_rho^{m+1} J_nu(k_rho rho) (i k_z)^n e^{i k_z zeta} s_tau / k_z dk_rho
// (the integrals of eq. ``symmetricdetable`` for one term) and T_{m,-nu,n} =
// (-1)^nu T_{m,nu,n}.  One table per term holds T_{m,nu,n}, m + n <= 2p,
// nu = m mod 2 .. m step 2, on a uniform n x n grid of (rho, zeta) over the
// ranges of the layer's M2L keys ("the domain of interest").
//
// Table construction, one CTA per grid point: the integral along the paper's
// contour Gamma_1 = {k_rho = i t, -b <= t <= 0}, Gamma_2 = {k_rho = t - i b,
// t >= 0}, truncated where the integrand has decayed (Sec. 4.2), by composite
// 8-point Gauss-Legendre panels (fine panels up to max Re k + 1, where the
// branch points and guided-mode poles lie a distance b above the path).  The
// integrand factors into A_{m,nu}(k_rho) = k_rho^{m+1} J_nu(k_rho rho) and
// B_n(k_rho) = w (i k_z)^n e^{i k_z zeta} s_tau / (k_z k): per chunk of 32
// nodes, 32 threads evaluate A and B into shared memory and every thread
// accumulates its entries T = sum_nodes A B.  J_nu of complex argument:
// ascending series for |z| <= 2, Miller's backward recurrence normalised by
// e^{iz} = J_0 + 2 sum_n i^n J_n otherwise, and for |z| >= max(25, 2 nu_max + 5)
// Hankel's asymptotic expansion of J_0, J_1 (DLMF 10.17.3) with forward
// recurrence.  s_tau comes from the same interface solve as the DCIM fits.
//
// Lookup (in the derivative-table kernel): degree-7 Lagrange interpolation in
// FP64 in each direction (the 8 grid points around the point, shifted inside
// the grid at its edges), then the Cartesian coefficients
//   a_g = D^g F / g! = (1/g!) 2^-(g1+g2) (-i)^g2 sum_{a1<=g1, a2<=g2} C(g1,a1) C(g2,a2)
//         (-1)^(g2-a2) (-1)^a e^{i nu phi} T_{g1+g2, nu, g3},  a = a1 + a2, nu = 2a - g1 - g2,
// from d_x = (D+ + D-)/2 and d_y = (D+ - D-)/(2i).
#include <math.h>
#include <chrono>

#include "internal.cuh"
#include "ops_common.cuh"
#include "alg2.cuh"
#include "density.cuh"

namespace {

constexpr int A2_GL = 8;          // Gauss-Legendre nodes per panel
constexpr int A2_CHUNK = 32;      // contour nodes per shared-memory chunk
constexpr int A2_THREADS = 256;
constexpr int A2_OUT = 8;         // table entries per thread (entries <= 2048)
constexpr double A2_B = 0.4;      // depth of the contour below the real axis
constexpr double A2_WNEAR = 0.1;  // panel width up to max Re k + 1
constexpr double A2_DECAY = 44.0; // truncate Gamma_2 where the integrand fell by e^-44

__constant__ double c_gl_x[A2_GL], c_gl_w[A2_GL];

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n with
// the three-term recurrence (host, once per process)
void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

__host__ __device__ __forceinline__ cplx cexp_i(cplx z) {   // e^{i z}
    return cexp_(mkc(-z.y, z.x));
}

// J_0 .. J_nmax of complex z (nmax <= 24)
__host__ __device__ void bessel_j(cplx z, int nmax, cplx *J) {
    const double az = hypot(z.x, z.y);
    if (az == 0.0) {
        J[0] = mkc(1, 0);
        for (int n = 1; n <= nmax; ++n) J[n] = mkc(0, 0);
        return;
    }
    if (az <= 2.0) {
        // ascending series: J_nu = (z/2)^nu sum_k (-z^2/4)^k / (k! (nu + k)!)
        const cplx h = cscale(z, 0.5);
        const cplx q = cscale(cmul(h, h), -1.0);
        cplx lead = mkc(1, 0);                 // (z/2)^nu / nu!
        for (int nu = 0; nu <= nmax; ++nu) {
            if (nu > 0) lead = cscale(cmul(lead, h), 1.0 / nu);
            cplx term = lead, sum = lead;
            for (int k = 1; k < 60; ++k) {
                term = cscale(cmul(term, q), 1.0 / ((double)k * (double)(nu + k)));
                sum = cadd(sum, term);
                if (hypot(term.x, term.y) <= 1e-18 * hypot(sum.x, sum.y)) break;
            }
            J[nu] = sum;
        }
        return;
    }
    const double zasym = fmax(25.0, 2.0 * nmax + 5.0);
    const cplx iz = cdiv(mkc(1, 0), z);
    if (az >= zasym) {
        // Hankel's expansion, DLMF 10.17.3: J_nu ~ (2/(pi z))^(1/2) (P cos w - Q sin w),
        // w = z - nu pi/2 - pi/4, a_k(nu) = prod_{j<=k} (4nu^2 - (2j-1)^2) / (k! 8^k)
        const cplx pre = csqrt_p(cscale(iz, 2.0 / M_PI));
        for (int nu = 0; nu <= 1 && nu <= nmax; ++nu) {
            cplx P = mkc(1, 0), Q = mkc(0, 0), zk = mkc(1, 0);
            double a = 1.0, last = INFINITY;
            for (int k = 1; k < 80; ++k) {
                a *= (4.0 * nu * nu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
                zk = cmul(zk, iz);
                const cplx t = cscale(zk, a);
                const double mag = hypot(t.x, t.y);
                if (mag > last) break;          // the asymptotic series starts to grow
                last = mag;
                const double sg = ((k / 2) % 2) ? -1.0 : 1.0;   // (-1)^floor(k/2)
                if (k % 2 == 0) P = cadd(P, cscale(t, sg));
                else Q = cadd(Q, cscale(t, sg));
                if (mag < 1e-18) break;
            }
            const double ph = nu * M_PI * 0.5 + M_PI * 0.25;
            const cplx w = mkc(z.x - ph, z.y);
            double sr, cr;
            sincos(w.x, &sr, &cr);
            const double ch = cosh(w.y), sh = sinh(w.y);
            const cplx cw = mkc(cr * ch, -sr * sh), sw = mkc(sr * ch, cr * sh);
            J[nu] = cmul(pre, csub(cmul(P, cw), cmul(Q, sw)));
        }
        for (int n = 1; n < nmax; ++n)   // forward recurrence, stable for n < |z|
            J[n + 1] = csub(cmul(cscale(iz, 2.0 * n), J[n]), J[n - 1]);
        return;
    }
    // Miller: f_{n-1} = (2n/z) f_n - f_{n+1} from f_{N+1} = 0, f_N = 1e-30,
    // normalised by e^{i s z} = f_0 + 2 sum_{n>=1} (i s)^n f_n, s = 1 for Im z <= 0
    // and s = -1 otherwise (the side without cancellation)
    const double s = z.y <= 0.0 ? 1.0 : -1.0;
    int N = (int)(fmax(az, (double)nmax) + 30.0);
    N += N & 1;
    cplx fp = mkc(0, 0), f = mkc(1e-30, 0), sum = mkc(0, 0);
    for (int n = N; n >= 1; --n) {
        if (n <= nmax) J[n] = f;
        // (i s)^n: n mod 4 -> 1, i s, -1, -i s
        const int r = n & 3;
        const cplx ph = r == 0 ? mkc(1, 0) : r == 1 ? mkc(0, s) : r == 2 ? mkc(-1, 0) : mkc(0, -s);
        sum = cadd(sum, cscale(cmul(ph, f), 2.0));
        const cplx fm = csub(cmul(cscale(iz, 2.0 * n), f), fp);
        fp = f;
        f = fm;
        if (hypot(f.x, f.y) > 1e200) {          // rescale to stay in range
            f = cscale(f, 1e-200);
            fp = cscale(fp, 1e-200);
            sum = cscale(sum, 1e-200);
            for (int m = n; m <= nmax; ++m) J[m] = cscale(J[m], 1e-200);
        }
    }
    J[0] = f;
    sum = cadd(sum, f);
    const cplx norm = cdiv(cexp_i(cscale(z, s)), sum);
    for (int n = 0; n <= nmax; ++n) J[n] = cmul(J[n], norm);
}

}  // namespace

// ---------------------------------------------------------------- table build
namespace {

struct A2Build {
    FitJob J;                  // medium, layer and term (same-layer mode)
    cplx k;                    // the layer's wavenumber
    int P2, n, ne, nmv;
    double rho_max, zlo, zhi, kre_max;
    cplx *T;                   // [n][n][ne]
};

// grid (i_rho, j_zeta) = (blockIdx.x, blockIdx.y); shared memory:
// A[nmv][A2_CHUNK] then B[P2 + 1][A2_CHUNK], complex
__global__ void __launch_bounds__(A2_THREADS) k_alg2_build(A2Build B) {
    extern __shared__ double a2sm[];
    cplx *As = (cplx *)a2sm;
    cplx *Bs = As + B.nmv * A2_CHUNK;
    const int i = blockIdx.x, j = blockIdx.y, P2 = B.P2;
    const double rho = (B.rho_max / (double)(B.n - 1)) * (double)i;
    const double zeta = __dadd_rn(B.zlo, __dmul_rn((B.zhi - B.zlo) / (double)(B.n - 1), (double)j));

    // the entries this thread accumulates: (m, nu) pair index and n
    int o_mv[A2_OUT], o_n[A2_OUT];
    int nmine = 0;
    {
        int o = 0, mv = 0;
        for (int m = 0; m <= P2; ++m)
            for (int nu = m & 1; nu <= m; nu += 2, ++mv)
                for (int nn = 0; nn <= P2 - m; ++nn, ++o)
                    if (o % A2_THREADS == (int)threadIdx.x && nmine < A2_OUT) {
                        o_mv[nmine] = mv;
                        o_n[nmine] = nn;
                        ++nmine;
                    }
    }
    cplx acc[A2_OUT];
    for (int q = 0; q < A2_OUT; ++q) acc[q] = mkc(0, 0);

    // contour: Gamma_1 (2 panels), Gamma_2 fine panels up to tn, coarse to tmax
    const int NP1 = 2;
    const int NPn = (int)ceil((B.kre_max + 1.0) / A2_WNEAR);
    const double tn = NPn * A2_WNEAR;
    const double Pw = (double)(P2 + 1);
    const double tpk = Pw / zeta;
    double tmax = fmax(tpk, tn);
    for (int it = 0; it < 4000 && Pw * log(tmax / tpk) - (tmax - tpk) * zeta > -A2_DECAY; ++it)
        tmax += fmax(0.5, 0.05 * tmax);
    double wf = 1.0;
    if (rho > 0.0) wf = fmin(wf, 2.0 / rho);
    wf = fmin(wf, 2.0 / zeta);
    const int NPf = tmax > tn ? (int)ceil((tmax - tn) / wf) : 0;
    if (NPf > 0) wf = (tmax - tn) / NPf;
    const int nq = A2_GL * (NP1 + NPn + NPf);

    for (int q0 = 0; q0 < nq; q0 += A2_CHUNK) {
        if (threadIdx.x < A2_CHUNK) {
            const int t = threadIdx.x, q = q0 + t;
            if (q < nq) {
                const int pn = q / A2_GL, g = q % A2_GL;
                const double xg = 0.5 * (c_gl_x[g] + 1.0), wg = 0.5 * c_gl_w[g];
                cplx kr, w;
                if (pn < NP1) {                     // k_rho = -i u, u in [0, b]: dk_rho = -i du
                    const double hw = A2_B / NP1;
                    kr = mkc(0.0, -hw * (pn + xg));
                    w = mkc(0.0, -hw * wg);
                } else if (pn < NP1 + NPn) {        // k_rho = t - i b, t in [0, tn]
                    kr = mkc(A2_WNEAR * (pn - NP1 + xg), -A2_B);
                    w = mkc(A2_WNEAR * wg, 0.0);
                } else {                            // t in [tn, tmax]
                    kr = mkc(tn + wf * (pn - NP1 - NPn + xg), -A2_B);
                    w = mkc(wf * wg, 0.0);
                }
                const cplx kz = kz_of(B.k, cmul(kr, kr));
                const cplx s = s_tau_sample(B.J, kz);
                const cplx base = cdiv(cmul(cmul(w, s), cexp_i(cscale(kz, zeta))), cmul(kz, B.k));
                cplx Jv[25];
                bessel_j(cscale(kr, rho), P2, Jv);
                cplx pw = kr;                       // k_rho^{m+1}
                int mv = 0;
                for (int m = 0; m <= P2; ++m) {
                    for (int nu = m & 1; nu <= m; nu += 2, ++mv) As[mv * A2_CHUNK + t] = cmul(pw, Jv[nu]);
                    pw = cmul(pw, kr);
                }
                const cplx ikz = mkc(-kz.y, kz.x);
                cplx b = base;                      // base (i k_z)^n
                for (int nn = 0; nn <= P2; ++nn) {
                    Bs[nn * A2_CHUNK + t] = b;
                    b = cmul(b, ikz);
                }
            } else {
                for (int mv = 0; mv < B.nmv; ++mv) As[mv * A2_CHUNK + t] = mkc(0, 0);
                for (int nn = 0; nn <= P2; ++nn) Bs[nn * A2_CHUNK + t] = mkc(0, 0);
            }
        }
        __syncthreads();
        for (int q = 0; q < nmine; ++q) {
            const cplx *a = As + o_mv[q] * A2_CHUNK, *b = Bs + o_n[q] * A2_CHUNK;
            cplx s = acc[q];
#pragma unroll 8
            for (int t = 0; t < A2_CHUNK; ++t) s = cadd(s, cmul(a[t], b[t]));
            acc[q] = s;
        }
        __syncthreads();
    }
    cplx *out = B.T + ((int64_t)i * B.n + j) * B.ne;
    for (int q = 0; q < nmine; ++q) out[threadIdx.x + q * A2_THREADS] = acc[q];
}

}  // namespace

// ---------------------------------------------------------------- host side
int alg2_entries(int P2) {
    int ne = 0;
    for (int m = 0; m <= P2; ++m) ne += (m / 2 + 1) * (P2 - m + 1);
    return ne;
}

A2View a2_view(tefmm_plan_s *P) {
    A2View v{};
    v.on = P->opt.algorithm == TEFMM_ALG_TABLES ? 1 : 0;
    v.P2 = 2 * P->p;
    v.ne = alg2_entries(v.P2);
    v.mi = dp<int>(P->d_mi);
    for (const Alg2Table &t : P->a2) v.t[t.layer][t.tag] = A2Tab{t.T, t.rho_max, t.zlo, t.zhi, t.n};
    return v;
}

namespace {

int build_table(tefmm_plan_s *P, Alg2Table &t, cudaStream_t st) {
    // the quadrature rule goes to the current device's constant memory before
    // every build (128 bytes; no per-process flag that a device reset or a
    // second host thread could leave stale)
    {
        double x[A2_GL], w[A2_GL];
        gauss_legendre(A2_GL, x, w);
        CUDA_TRY(cudaMemcpyToSymbolAsync(c_gl_x, x, sizeof(x), 0, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyToSymbolAsync(c_gl_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    A2Build B{};
    B.J.mode = 0;
    B.J.layer = t.layer;
    B.J.tag = t.tag;
    B.J.nL = P->nL;
    for (int m = 0; m < TEFMM_MAX_LAYERS; ++m) {
        B.J.d[m] = m < P->nL - 1 ? P->d[m] : 0.0;
        B.J.k[m] = m < P->nL ? P->k[m] : mkc(1, 0);
    }
    B.k = P->k[t.layer];
    B.P2 = t.P2;
    B.n = t.n;
    B.ne = t.ne;
    B.nmv = 0;
    for (int m = 0; m <= t.P2; ++m) B.nmv += m / 2 + 1;
    B.rho_max = t.rho_max;
    B.zlo = t.zlo;
    B.zhi = t.zhi;
    B.kre_max = 0.0;
    for (int l = 0; l < P->nL; ++l) B.kre_max = fmax(B.kre_max, P->k[l].x);
    if (t.ne > A2_OUT * A2_THREADS) return TEFMM_ERR_NOT_IMPLEMENTED;
    const size_t bytes = (size_t)t.n * t.n * t.ne * sizeof(cplx);
    if (inject_alloc_failure()) return TEFMM_ERR_OOM;
    if (cudaMalloc(&t.T, bytes) != cudaSuccess) {
        cudaGetLastError();
        t.T = nullptr;
        return TEFMM_ERR_OOM;
    }
    B.T = t.T;
    const size_t sm = (size_t)(B.nmv + B.P2 + 1) * A2_CHUNK * sizeof(cplx);
    CUDA_TRY(cudaFuncSetAttribute(k_alg2_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_alg2_build<<<dim3((unsigned)t.n, (unsigned)t.n), A2_THREADS, sm, st>>>(B);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

}  // namespace

void alg2_release(tefmm_plan_s *P) {
    for (Alg2Table &t : P->a2) {
        bool shared = false;               // a down-up table may reuse the up-down buffer
        for (Alg2Table &o : P->a2)
            if (&o != &t && o.T == t.T && (o.layer < t.layer || (o.layer == t.layer && o.tag < t.tag)))
                shared = true;
        if (t.T && !shared) cudaFree(t.T);
    }
    P->a2.clear();
}

// Ranges of the same-layer keys per (layer, term), then the tables they need
// (kept when an earlier geometry already built them over the same ranges).
int alg2_prepare(tefmm_plan_s *P, cudaStream_t st) {
    if (P->opt.algorithm != TEFMM_ALG_TABLES) return TEFMM_OK;
    const int ntab = P->x_first_table;
    std::vector<uint64_t> keys(ntab);
    if (ntab > 0) {
        CUDA_TRY(cudaMemcpyAsync(keys.data(), P->table_slot.p, (size_t)ntab * 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    const int L = P->nL;
    std::vector<double> rmax(L, 0.0), lo(4 * L, INFINITY), hi(4 * L, -INFINITY);
    std::vector<char> has(4 * L, 0);
    int n_images = 0;
    for (uint64_t key : keys) {
        const int kind = key_kind(key);
        if (kind > 1) continue;            // far-of-near keys (kind 2) keep the images
        const int l = key_layer(key), lev = key_level(key);
        const double h = P->side / (double)(1 << lev);
        const double rho = hypot((double)key_dx(key) * h, (double)key_dy(key) * h);
        const int w = (int)key_w(key);
        for (int ti = P->layer_term_first[l]; ti < P->layer_term_first[l] + P->layer_term_count[l]; ++ti) {
            const TermDesc &td = P->terms[ti];
            double zeta;
            if (kind == 0 && td.tag >= 2) zeta = td.sz * ((double)(w - KEY_OFF) * h) + td.c;
            else if (kind == 1 && td.tag <= 1) zeta = td.sz * (2.0 * P->lo[2] + (double)(w + 1) * h) + td.c;
            else continue;
            // below the term's smallest image distance over the particle slab
            // (its DCIM shift: box centres beyond the slab) the key keeps the images
            if (!(zeta >= td.zmin)) {
                ++n_images;
                continue;
            }
            const int s = 4 * l + td.tag;
            has[s] = 1;
            lo[s] = fmin(lo[s], zeta);
            hi[s] = fmax(hi[s], zeta);
            rmax[l] = fmax(rmax[l], rho);
        }
    }
    P->n_alg2_image_keys = n_images;
    const int P2 = 2 * P->p, n = P->opt.table_n > 0 ? P->opt.table_n : 64;
    std::vector<Alg2Table> want;
    for (int l = 0; l < L; ++l)
        for (int tag = 0; tag < 4; ++tag) {
            const int s = 4 * l + tag;
            if (!has[s]) continue;
            Alg2Table t;
            t.layer = l;
            t.tag = tag;
            t.P2 = P2;
            t.n = n;
            t.ne = alg2_entries(P2);
            t.rho_max = rmax[l] > 0.0 ? rmax[l] : 1.0;
            t.zlo = lo[s];
            t.zhi = hi[s] > lo[s] ? hi[s] : lo[s] + 1.0;
            want.push_back(t);
        }
    auto same = [](const Alg2Table &a, const Alg2Table &b) {
        return a.P2 == b.P2 && a.n == b.n && a.rho_max == b.rho_max && a.zlo == b.zlo && a.zhi == b.zhi;
    };
    bool keep = want.size() == P->a2.size();
    for (size_t i = 0; keep && i < want.size(); ++i)
        keep = want[i].layer == P->a2[i].layer && want[i].tag == P->a2[i].tag && same(want[i], P->a2[i]);
    if (keep) return TEFMM_OK;
    alg2_release(P);
    const auto t0 = std::chrono::steady_clock::now();
    int err = TEFMM_OK;
    for (size_t i = 0; i < want.size() && err == TEFMM_OK; ++i) {
        Alg2Table &t = want[i];
        // the down-up factor equals the up-down one (reciprocity): share its table over the same ranges
        if (t.tag == 3 && i > 0 && want[i - 1].layer == t.layer && want[i - 1].tag == 2 && same(want[i - 1], t)) {
            t.T = want[i - 1].T;
            continue;
        }
        err = build_table(P, t, st);
    }
    P->a2 = want;
    if (err != TEFMM_OK) {
        alg2_release(P);
        return err;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    P->ms_alg2_build = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return TEFMM_OK;
}

extern "C" int tefmm_plan_get_alg2_table(tefmm_plan P, int layer, int tag, int *n, int *n_entries,
                                         double *range, double *T) {
    if (!P || !n || !n_entries || !range) return TEFMM_ERR_INVALID_ARG;
    for (const Alg2Table &t : P->a2) {
        if (t.layer != layer || t.tag != tag) continue;
        *n = t.n;
        *n_entries = t.ne;
        range[0] = t.rho_max;
        range[1] = t.zlo;
        range[2] = t.zhi;
        if (T) CUDA_TRY(cudaMemcpy(T, t.T, (size_t)t.n * t.n * t.ne * sizeof(cplx), cudaMemcpyDeviceToHost));
        return TEFMM_OK;
    }
    return TEFMM_ERR_INVALID_ARG;
}
