// Cross-layer reaction components (Sec. 3.2-3.3): target layer l != source layer l'.
//
// The component's z'-dependence cannot be folded into an image distance, so
// the paper expands it in z' about the source box centre z_c: for each source
// z-centre and each k3' = 0..p the density's k3'-th z'-derivative (divided by
// k3'!) is fitted by the two-level DCIM in the target layer's k_lz,
//   d^{k3'}_{z'} u / k3'! ~= sum_j A_j h0(k_l sqrt(rho^2 + (W - W_min - Z_j)^2)),
// with W = z - d_l for the up-going part (present for l < L) and
// W = d_{l-1} - z for the down-going part (present for l > 0).  The M2L of a cross pair is then
//   beta_k += sum_k' alpha_k' (-1)^{k1'+k2'} C(k1+k1',k1) C(k2+k2',k2)
//             sz^{k3} T^{(k3')}_{(k1+k1', k2+k2', k3)},
//   T^{(k3')}_g = sum_dir sum_j A_j D^g h0(k_l R_j) / g!   at (dx h, dy h, W(z_t) - W_min - Z_j),
// sz = +1 (up) / -1 (down, folded into the table as (-1)^{g3}).
// One table per key (level, l, l', dx, dy, iz_t, iz_s) holds T^{(k3')} for all
// k3' (orders 2p - k3'), packed slice after slice.
//
// The z-centres of a cross-layer translation are the box centres clamped to
// the layer's particle slab (a box of one layer's tree may straddle an
// interface, and at a source centre outside its layer the fitted function
// grows along the first DCIM path).  The source moments are shifted to the
// clamped centre exactly (a z-only M2M), the translation produces locals
// about the target's clamped centre, and these are re-expanded at the box
// centre (a z-only L2L) and added to the box's locals.
//
// The fits depend only on the geometry of the root cube (through z_c), so they
// are cached in the plan and refitted only when the cube's z-origin or side
// changes (the paper precomputes them once, 2^H (p+1) per component).
#include <chrono>
#include <set>

#include "ops_common.cuh"

namespace {

struct XGeom {
    double d[TEFMM_MAX_LAYERS];
    double wmin[2 * TEFMM_MAX_LAYERS];   // [layer][dir]
    double zlo[TEFMM_MAX_LAYERS], zhi[TEFMM_MAX_LAYERS];   // particle slab of each layer
    cplx k[TEFMM_MAX_LAYERS];
};

// cross-layer expansion centre in z: the box centre clamped to the layer's slab
__host__ __device__ inline double xcentre(double c, double zlo, double zhi) {
    return fmin(fmax(c, zlo), zhi);
}

// moments about the cross-layer centre: alpha*_k = sum_{j3<=k3} C(k3,j3) dz^{k3-j3}
// alpha_(k1,k2,j3), dz = box centre - cross-layer centre (exact shift in z)
__global__ void k_xshift_alpha(int nn, TreeArrays T, Cube cb, XGeom geo, int p, int np,
                               const int *__restrict__ mi, const cplx *__restrict__ alpha,
                               cplx *__restrict__ alpha_x) {
    int node = blockIdx.x;
    if (node >= nn) return;
    const int lay = T.layer[node];
    const double h = box_h(cb.side, T.level[node]);
    const double zc = centre(cb.lo[2], T.iz[node], h);
    const double dz = zc - xcentre(zc, geo.zlo[lay], geo.zhi[lay]);
    const cplx *a = alpha + (int64_t)node * np;
    cplx *o = alpha_x + (int64_t)node * np;
    if (dz == 0.0) {
        for (int k = threadIdx.x; k < np; k += blockDim.x) o[k] = a[k];
        return;
    }
    __shared__ double cw[32 * 32];   // cw[n * (p + 1) + j] = C(n, j) dz^{n-j}
    if (threadIdx.x <= p) {
        const int n = threadIdx.x;
        double c = 1.0;               // C(n, j), built from j = n down
        double pw = 1.0;              // dz^{n-j}
        for (int j = n; j >= 0; --j) {
            cw[n * (p + 1) + j] = c * pw;
            c = c * (double)j / (double)(n - j + 1);
            pw *= dz;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const int k1 = mi[3 * k], k2 = mi[3 * k + 1], k3 = mi[3 * k + 2];
        cplx s = mkc(0, 0);
        for (int j3 = 0; j3 <= k3; ++j3) {
            const double b = cw[k3 * (p + 1) + j3];
            const cplx x = a[midx(k1, k2, j3)];
            s.x += b * x.x;
            s.y += b * x.y;
        }
        o[k] = s;
    }
}

// locals about the cross-layer centre, re-expanded at the box centre and added:
// beta_k += sum_{j3>=k3} C(j3,k3) dz^{j3-k3} beta*_(k1,k2,j3), dz = box centre - cross centre
__global__ void k_xshift_beta(int nn, TreeArrays T, Cube cb, XGeom geo, int p, int np,
                              const int *__restrict__ mi, const cplx *__restrict__ beta_x,
                              cplx *__restrict__ beta) {
    int node = blockIdx.x;
    if (node >= nn || T.t1[node] <= T.t0[node]) return;
    const int lay = T.layer[node];
    const double h = box_h(cb.side, T.level[node]);
    const double zc = centre(cb.lo[2], T.iz[node], h);
    const double dz = zc - xcentre(zc, geo.zlo[lay], geo.zhi[lay]);
    const cplx *bx = beta_x + (int64_t)node * np;
    cplx *b = beta + (int64_t)node * np;
    if (dz == 0.0) {
        for (int k = threadIdx.x; k < np; k += blockDim.x) b[k] = cadd(b[k], bx[k]);
        return;
    }
    __shared__ double cw[32 * 32];   // cw[j * (p + 1) + n] = C(j, n) dz^{j-n}, j >= n
    if (threadIdx.x <= p) {
        const int j = threadIdx.x;
        double c = 1.0, pw = 1.0;
        for (int n = j; n >= 0; --n) {
            cw[j * (p + 1) + n] = c * pw;
            c = c * (double)n / (double)(j - n + 1);
            pw *= dz;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const int k1 = mi[3 * k], k2 = mi[3 * k + 1], k3 = mi[3 * k + 2];
        cplx s = mkc(0, 0);
        for (int j3 = k3; k1 + k2 + j3 <= p; ++j3) {
            const double w = cw[j3 * (p + 1) + k3];
            const cplx x = bx[midx(k1, k2, j3)];
            s.x += w * x.x;
            s.y += w * x.y;
        }
        b[k] = mkc(b[k].x + s.x, b[k].y + s.y);
    }
}

// first cross-layer table and first cross-layer chunk (keys are sorted, kind 3 last)
__global__ void k_first_cross(int ntab, const uint64_t *__restrict__ tkey, int64_t nch,
                              const int *__restrict__ chunk_table, int *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < ntab) {
        bool x = key_is_cross(tkey[i]), xp = i > 0 && key_is_cross(tkey[i - 1]);
        if (x && !xp) out[0] = (int)i;
    }
    if (i < nch) {
        bool x = key_is_cross(tkey[chunk_table[i]]);
        bool xp = i > 0 && key_is_cross(tkey[chunk_table[i - 1]]);
        if (x && !xp) out[1] = (int)i;
    }
}

// T^{(k3')} slice of one cross table: grid (tables, p + 1)
__global__ void __launch_bounds__(256, 4) k_xtables(int nx, const uint64_t *__restrict__ keys, Cube cb, int p, XGeom geo,
                          const int2 *__restrict__ xrange,
                          const cplx *__restrict__ xA, const cplx *__restrict__ xZ, int NX,
                          const int *__restrict__ rep_code, int first, cplx *__restrict__ xt) {
    int tb = blockIdx.x, k3p = blockIdx.y;
    if (tb >= nx || k3p > p) return;
    if ((rep_code[first + tb] >> 3) != first + tb) return;   // copied by symmetry
    const int P2 = 2 * p - k3p, n2 = ncoef(P2), cmax = tri(P2 + 1);
    extern __shared__ double sm[];
    cplx *a = (cplx *)sm;                                     // [3][cmax] ring of orders
    cplx *b = a + 3 * cmax;
    cplx *acc = xt + (int64_t)tb * NX + slice_off(p, k3p);   // the slice accumulates in place
    for (int g = threadIdx.x; g < n2; g += blockDim.x) acc[g] = mkc(0, 0);
    __syncthreads();
    const XKey x = xkey_decode(keys[tb]);
    const double h = box_h(cb.side, x.level);
    const double X = (double)x.dx * h, Y = (double)x.dy * h;
    const double zt = xcentre(centre(cb.lo[2], x.izt, h), geo.zlo[x.lt], geo.zhi[x.lt]);
    const cplx k = geo.k[x.lt];
    for (int dir = 0; dir < 2; ++dir) {
        int2 r = xrange[((int64_t)tb * 2 + dir) * (p + 1) + k3p];
        if (r.y == 0) continue;
        double W0 = dir == 0 ? zt - geo.d[x.lt] : geo.d[x.lt - 1] - zt;
        double Wr = W0 - geo.wmin[2 * x.lt + dir];
        for (int j = r.x; j < r.x + r.y; ++j) {
            cplx Wj = mkc(Wr - xZ[j].x, -xZ[j].y);
            recur_accumulate(P2, cmax, k, X, Y, Wj, xA[j], dir == 1, a, b, acc);
        }
    }
}

// Cross-layer M2L, FP64: one CTA per chunk of pairs of one cross key, one
// thread per output coefficient k; the k' sum walks the k3' slices.  A reversed
// key (xkey_rev) applies (k_lt / k_ls)^2 times the transposed matrix
// H^T[k][k'] = xcf[k][k'] T^{(k3)}[xg[k][k']]: thread k takes its whole sum from
// the slice of its own k3.
constexpr int CHX = 16;

__global__ void k_m2l_x(int c0, int nch, const int *__restrict__ chunk_start,
                        const int *__restrict__ chunk_table, const int *__restrict__ chunk_cnt,
                        int first_table, const cplx *__restrict__ xt, int NX,
                        const int *__restrict__ items, const int *__restrict__ pair_t,
                        const int *__restrict__ v_src, int p, int np,
                        const unsigned short *__restrict__ xg, const double *__restrict__ xcf,
                        const int *__restrict__ kp_order, const int *__restrict__ kp_grp,
                        const uint64_t *__restrict__ table_key, const int *__restrict__ mi,
                        const cplx *__restrict__ kl, const cplx *__restrict__ alpha,
                        cplx *__restrict__ beta) {
    int c = c0 + blockIdx.x;
    if (blockIdx.x >= nch) return;
    extern __shared__ double sm[];
    cplx *tab = (cplx *)sm;                       // [ncoef(2p)]
    cplx *al = tab + ncoef(2 * p);                // [CHX][np]
    __shared__ int tgt[CHX];
    const int tb = chunk_table[c] - first_table;
    const int cnt = chunk_cnt[c], st = chunk_start[c];
    const int k = threadIdx.x;
    const cplx *T = xt + (int64_t)tb * NX;
    const uint64_t key = table_key[chunk_table[c]];
    const bool rev = xkey_rev(key) != 0;
    cplx fac = mkc(1, 0);
    if (rev) {
        const XKey x = xkey_decode(key);
        const cplx r = cdiv(kl[x.lt], kl[x.ls]);
        fac = cmul(r, r);
    }
    const int k3 = k < np ? mi[3 * k + 2] : -1;
    for (int qb = 0; qb < cnt; qb += CHX) {
        const int nq = min(CHX, cnt - qb);
        __syncthreads();
        for (int q = 0; q < nq; ++q) {
            int e = items[st + qb + q] >> 1;
            if (threadIdx.x == 0) tgt[q] = pair_t[e];
            int s = v_src[e];
            for (int kk = threadIdx.x; kk < np; kk += blockDim.x) al[q * np + kk] = alpha[(int64_t)s * np + kk];
        }
        cplx acc[CHX];
#pragma unroll
        for (int q = 0; q < CHX; ++q) acc[q] = mkc(0, 0);
        int off = 0;
        for (int k3p = 0; k3p <= p; ++k3p) {
            const int n2 = ncoef(2 * p - k3p);
            __syncthreads();
            for (int g = threadIdx.x; g < n2; g += blockDim.x) tab[g] = T[off + g];
            __syncthreads();
            off += n2;
            if (k >= np) continue;
            if (!rev) {
                for (int i = kp_grp[k3p]; i < kp_grp[k3p + 1]; ++i) {
                    const int kp = kp_order[i];
                    const double cf = xcf[(int64_t)kp * np + k];
                    cplx hv = tab[xg[(int64_t)kp * np + k]];
                    hv.x *= cf;
                    hv.y *= cf;
#pragma unroll
                    for (int q = 0; q < CHX; ++q) {
                        if (q < nq) {
                            cplx a = al[q * np + kp];
                            acc[q].x += hv.x * a.x - hv.y * a.y;
                            acc[q].y += hv.x * a.y + hv.y * a.x;
                        }
                    }
                }
            } else if (k3 == k3p) {
                for (int kp = 0; kp < np; ++kp) {
                    const double cf = xcf[(int64_t)k * np + kp];
                    cplx hv = tab[xg[(int64_t)k * np + kp]];
                    hv.x *= cf;
                    hv.y *= cf;
#pragma unroll
                    for (int q = 0; q < CHX; ++q) {
                        if (q < nq) {
                            cplx a = al[q * np + kp];
                            acc[q].x += hv.x * a.x - hv.y * a.y;
                            acc[q].y += hv.x * a.y + hv.y * a.x;
                        }
                    }
                }
            }
        }
        if (k < np) {
#pragma unroll
            for (int q = 0; q < CHX; ++q) {
                if (q < nq) {
                    const cplx v = rev ? cmul(fac, acc[q]) : acc[q];
                    double *dst = (double *)&beta[(int64_t)tgt[q] * np + k];
                    atomicAdd(dst, v.x);
                    atomicAdd(dst + 1, v.y);
                }
            }
        }
    }
}

XGeom geometry(const tefmm_plan_s *P) {
    XGeom g{};
    for (int l = 0; l < TEFMM_MAX_LAYERS; ++l) {
        g.d[l] = l < P->nL - 1 ? P->d[l] : 0.0;
        g.k[l] = l < P->nL ? P->k[l] : mkc(1, 0);
        g.zlo[l] = l < P->nL ? P->opt.zext[2 * l] : 0.0;
        g.zhi[l] = l < P->nL ? P->opt.zext[2 * l + 1] : 0.0;
        for (int dir = 0; dir < 2; ++dir) {
            bool present = l < P->nL && (dir == 0 ? l < P->nL - 1 : l > 0);
            g.wmin[2 * l + dir] = present ? cross_wmin(P, l, dir) : 0.0;
        }
    }
    return g;
}

// cross-layer M2L maps: xg[k'][k] = index of (k1+k1', k2+k2', k3) within the
// k3' slice, xcf[k'][k] = (-1)^{k1'+k2'} C(k1+k1',k1) C(k2+k2',k2); k' ordered by k3'
int build_maps(tefmm_plan_s *P) {
    const int p = P->p, np = P->np;
    if (P->d_xG.p && P->d_xoff.p && P->d_xcf.cap >= (size_t)np * np * 8) return TEFMM_OK;
    std::vector<int> mi(3 * np);
    int t = 0;
    for (int n = 0; n <= p; ++n)
        for (int k1 = n; k1 >= 0; --k1)
            for (int k2 = n - k1; k2 >= 0; --k2) {
                mi[3 * t] = k1;
                mi[3 * t + 1] = k2;
                mi[3 * t + 2] = n - k1 - k2;
                ++t;
            }
    auto comb = [](int n, int k) {
        double r = 1.0;
        for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
        return r;
    };
    std::vector<unsigned short> G((size_t)np * np);
    std::vector<double> cf((size_t)np * np);
    for (int kp = 0; kp < np; ++kp)
        for (int k = 0; k < np; ++k) {
            int g1 = mi[3 * k] + mi[3 * kp], g2 = mi[3 * k + 1] + mi[3 * kp + 1], g3 = mi[3 * k + 2];
            G[(size_t)kp * np + k] = (unsigned short)midx(g1, g2, g3);
            double s = ((mi[3 * kp] + mi[3 * kp + 1]) & 1) ? -1.0 : 1.0;
            cf[(size_t)kp * np + k] = s * comb(g1, mi[3 * k]) * comb(g2, mi[3 * k + 1]);
        }
    std::vector<int> ord, grp(p + 2, 0);
    for (int k3p = 0; k3p <= p; ++k3p) {
        grp[k3p] = (int)ord.size();
        for (int kp = 0; kp < np; ++kp)
            if (mi[3 * kp + 2] == k3p) ord.push_back(kp);
    }
    grp[p + 1] = (int)ord.size();
    std::vector<int> og(ord);
    og.insert(og.end(), grp.begin(), grp.end());
    // tensor-core form: index into the packed slices and FP32 coefficients (exact)
    std::vector<unsigned short> Gs((size_t)np * np);
    std::vector<float> cf32((size_t)np * np);
    for (int kp = 0; kp < np; ++kp)
        for (int k = 0; k < np; ++k) {
            Gs[(size_t)kp * np + k] = (unsigned short)(slice_off(p, mi[3 * kp + 2]) + G[(size_t)kp * np + k]);
            cf32[(size_t)kp * np + k] = (float)cf[(size_t)kp * np + k];
        }
    TRY(dbuf_ensure(P->tc_xgs, Gs.size() * 2));
    TRY(dbuf_ensure(P->tc_xcf32, cf32.size() * 4));
    CUDA_TRY(cudaMemcpy(P->tc_xgs.p, Gs.data(), Gs.size() * 2, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->tc_xcf32.p, cf32.data(), cf32.size() * 4, cudaMemcpyHostToDevice));
    TRY(dbuf_ensure(P->d_xG, G.size() * 2));
    TRY(dbuf_ensure(P->d_xcf, cf.size() * 8));
    TRY(dbuf_ensure(P->d_xoff, og.size() * 4));
    CUDA_TRY(cudaMemcpy(P->d_xG.p, G.data(), G.size() * 2, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->d_xcf.p, cf.data(), cf.size() * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->d_xoff.p, og.data(), og.size() * 4, cudaMemcpyHostToDevice));
    return TEFMM_OK;
}

}  // namespace

double cross_wmin(const tefmm_plan_s *P, int lt, int dir) {
    const double zlo = P->opt.zext[2 * lt], zhi = P->opt.zext[2 * lt + 1];
    return dir == 0 ? zlo - P->d[lt] : P->d[lt - 1] - zhi;
}

int cross_prepare(tefmm_plan_s *P, cudaStream_t st) {
    P->n_xtables = 0;
    P->n_xfits_last = 0;
    P->ms_xfit = 0;
    if (P->nL < 2 || P->n_tables == 0) return TEFMM_OK;
    int h[2] = {P->n_tables, (int)P->n_chunks};
    TRY(dbuf_ensure(P->counters, 64));
    int *dcnt = dp<int>(P->counters) + 4;
    CUDA_TRY(cudaMemcpyAsync(dcnt, h, 8, cudaMemcpyHostToDevice, st));
    int64_t n = std::max<int64_t>(P->n_tables, P->n_chunks);
    k_first_cross<<<grid_for(n, 256), 256, 0, st>>>(P->n_tables, dp<uint64_t>(P->table_slot),
                                                    P->n_chunks, dp<int>(P->chunk_key), dcnt);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(h, dcnt, 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    P->x_first_table = h[0];
    P->x_first_chunk = h[1];
    const int nx = P->n_tables - h[0];
    if (nx == 0) return TEFMM_OK;
    if (P->x_first_chunk < P->n_chunks) {   // items from the first cross-layer chunk on are cross-layer
        int first_item = 0;
        CUDA_TRY(cudaMemcpy(&first_item, dp<int>(P->chunk_start) + P->x_first_chunk, 4, cudaMemcpyDeviceToHost));
        P->n_items_cross = P->n_items - first_item;
    }
    P->n_xtables = nx;
    std::vector<uint64_t> keys(nx);
    CUDA_TRY(cudaMemcpy(keys.data(), dp<uint64_t>(P->table_slot) + h[0], (size_t)nx * 8,
                        cudaMemcpyDeviceToHost));
    // the fits depend on the root cube through the source z-centres
    if (P->lo[2] != P->xgeo_lo || P->side != P->xgeo_side) {
        P->xcache.clear();
        P->xA.clear();
        P->xZ.clear();
        P->x_uploaded = 0;
        P->fit_max_resid_cross = 0;
        P->xgeo_lo = P->lo[2];
        P->xgeo_side = P->side;
    }
    const int p = P->p;
    std::vector<CrossFitKey> miss;
    std::set<CrossFitKey> pending;
    for (uint64_t key : keys) {
        XKey x = xkey_decode(key);
        for (int dir = 0; dir < 2; ++dir) {
            if (dir == 0 ? x.lt >= P->nL - 1 : x.lt == 0) continue;
            for (int k3p = 0; k3p <= p; ++k3p) {
                CrossFitKey c{x.lt, x.ls, dir, x.level, x.izs, k3p};
                if (P->xcache.count(c) || pending.count(c)) continue;
                pending.insert(c);
                miss.push_back(c);
            }
        }
    }
    auto t0 = std::chrono::steady_clock::now();
    const size_t BATCH = 4096;
    for (size_t i = 0; i < miss.size(); i += BATCH) {
        std::vector<CrossFitKey> part(miss.begin() + i, miss.begin() + std::min(miss.size(), i + BATCH));
        TRY(fit_cross_jobs(P, part, st));
    }
    P->n_xfits_last = (int)miss.size();
    P->ms_xfit = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (P->xA.size() != P->x_uploaded || !P->d_xA.p) {
        size_t ni = P->xA.size();
        TRY(dbuf_ensure(P->d_xA, (ni + 1) * sizeof(cplx)));
        TRY(dbuf_ensure(P->d_xZ, (ni + 1) * sizeof(cplx)));
        if (ni) {
            CUDA_TRY(cudaMemcpy(P->d_xA.p, P->xA.data(), ni * sizeof(cplx), cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(P->d_xZ.p, P->xZ.data(), ni * sizeof(cplx), cudaMemcpyHostToDevice));
        }
        P->x_uploaded = ni;
    }
    std::vector<int2> rng((size_t)nx * 2 * (p + 1), make_int2(0, 0));
    for (int tb = 0; tb < nx; ++tb) {
        XKey x = xkey_decode(keys[tb]);
        for (int dir = 0; dir < 2; ++dir) {
            if (dir == 0 ? x.lt >= P->nL - 1 : x.lt == 0) continue;
            for (int k3p = 0; k3p <= p; ++k3p) {
                auto it = P->xcache.find(CrossFitKey{x.lt, x.ls, dir, x.level, x.izs, k3p});
                if (it == P->xcache.end()) return TEFMM_ERR_FIT_FAILED;
                rng[((size_t)tb * 2 + dir) * (p + 1) + k3p] = make_int2(it->second.first, it->second.count);
            }
        }
    }
    TRY(dbuf_ensure(P->d_xrange, rng.size() * sizeof(int2)));
    CUDA_TRY(cudaMemcpy(P->d_xrange.p, rng.data(), rng.size() * sizeof(int2), cudaMemcpyHostToDevice));
    TRY(build_maps(P));
    P->NX = slice_off(p, p + 1);
    return TEFMM_OK;
}

int cross_tables(tefmm_plan_s *P, cudaStream_t st) {
    const int nx = P->n_xtables;
    if (nx == 0) return TEFMM_OK;
    TRY(dbuf_ensure(P->xtables, (size_t)nx * P->NX * sizeof(cplx)));
    const size_t sm = 6 * (size_t)tri(2 * P->p + 1) * sizeof(cplx);
    TRY(smem_optin(k_xtables));
    dim3 grid((unsigned)nx, (unsigned)(P->p + 1));
    k_xtables<<<grid, 256, sm, st>>>(nx, dp<uint64_t>(P->table_slot) + P->x_first_table, cube_of(P),
                                     P->p, geometry(P), dp<int2>(P->d_xrange),
                                     dp<cplx>(P->d_xA), dp<cplx>(P->d_xZ), P->NX,
                                     dp<int>(P->table_rep), P->x_first_table, dp<cplx>(P->xtables));
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return tables_expand(P, P->x_first_table, nx, P->p + 1, dp<cplx>(P->xtables), P->NX, st);
}

int cross_apply(tefmm_plan_s *P, cudaStream_t st) {
    const int nch = (int)(P->n_chunks - P->x_first_chunk);
    if (P->n_xtables == 0 || nch <= 0) return TEFMM_OK;
    const int np = P->np;
    const int nthr = (np + 31) / 32 * 32;
    size_t sm = (size_t)P->np2 * sizeof(cplx) + (size_t)CHX * np * sizeof(cplx);
    TRY(smem_optin(k_m2l_x));
    const int *og = dp<int>(P->d_xoff);
    const int nn = P->n_nodes;
    const size_t nb = (size_t)nn * np * sizeof(cplx);
    TRY(dbuf_ensure(P->xalpha, nb));
    TRY(dbuf_ensure(P->xbeta, nb));
    CUDA_TRY(cudaMemsetAsync(P->xbeta.p, 0, nb, st));
    const TreeArrays T = tree_arrays(P);
    const Cube cb = cube_of(P);
    const XGeom geo = geometry(P);
    k_xshift_alpha<<<nn, 128, 0, st>>>(nn, T, cb, geo, P->p, np, dp<int>(P->d_mi), dp<cplx>(P->alpha),
                                       dp<cplx>(P->xalpha));
    P->launches++;
    if (P->opt.precision == TEFMM_MIXED && (size_t)P->NX * sizeof(double) <= 200 * 1024) {
        // mixed form: the cross-layer contraction on the tensor cores (3xTF32)
        TRY(m2l_apply_tc_cross(P, st, dp<cplx>(P->xalpha), dp<cplx>(P->xbeta),
                               dp<unsigned short>(P->tc_xgs), dp<float>(P->tc_xcf32)));
    } else {
        k_m2l_x<<<nch, nthr, sm, st>>>((int)P->x_first_chunk, nch, dp<int>(P->chunk_start),
                                   dp<int>(P->chunk_key), dp<int>(P->chunk_cnt), P->x_first_table,
                                   dp<cplx>(P->xtables), P->NX, dp<int>(P->pair_idx_sorted),
                                   dp<int>(P->pair_t), dp<int>(P->v_src), P->p, np,
                                   dp<unsigned short>(P->d_xG), dp<double>(P->d_xcf), og, og + np,
                                   dp<uint64_t>(P->table_slot), dp<int>(P->d_mi), dp<cplx>(P->d_k),
                                   dp<cplx>(P->xalpha), dp<cplx>(P->xbeta));
        P->launches++;
    }
    k_xshift_beta<<<nn, 128, 0, st>>>(nn, T, cb, geo, P->p, np, dp<int>(P->d_mi), dp<cplx>(P->xbeta),
                                      dp<cplx>(P->beta));
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

void cross_release(tefmm_plan_s *P) {
    DBuf *b[] = {&P->d_xA, &P->d_xZ, &P->d_xrange, &P->d_tslot, &P->xtables, &P->d_xG,
                 &P->d_xcf, &P->d_xexp, &P->d_xoff, &P->tc_xcf, &P->xalpha, &P->xbeta,
                 &P->tc_xah, &P->tc_xal, &P->tc_xbt, &P->tc_xgs, &P->tc_xcf32, &P->tc_xW};
    for (DBuf *x : b) dbuf_free(*x);
}

extern "C" int tefmm_plan_cross_images(tefmm_plan P, int *n_fits, int *keys, int *counts, double *A,
                                       double *Z) {
    if (!P || !n_fits) return TEFMM_ERR_INVALID_ARG;
    *n_fits = (int)P->xcache.size();
    if (!keys && !counts && !A && !Z) return TEFMM_OK;
    int i = 0;
    for (const auto &e : P->xcache) {
        const CrossFitKey &c = e.first;
        const CrossFitVal &v = e.second;
        if (keys) {
            int *o = keys + 6 * i;
            o[0] = c.lt;
            o[1] = c.ls;
            o[2] = c.dir;
            o[3] = c.level;
            o[4] = c.izs;
            o[5] = c.k3p;
        }
        if (counts) counts[i] = v.count;
        for (int j = 0; j < v.count; ++j) {
            if (A) {
                A[2 * (TEFMM_MAX_IMG * i + j)] = P->xA[v.first + j].x;
                A[2 * (TEFMM_MAX_IMG * i + j) + 1] = P->xA[v.first + j].y;
            }
            if (Z) {
                Z[2 * (TEFMM_MAX_IMG * i + j)] = P->xZ[v.first + j].x;
                Z[2 * (TEFMM_MAX_IMG * i + j) + 1] = P->xZ[v.first + j].y;
            }
        }
        ++i;
    }
    return TEFMM_OK;
}

extern "C" int tefmm_plan_set_cross_images(tefmm_plan P, int n_fits, const int *keys, const int *counts,
                                           const double *A, const double *Z) {
    if (!P || n_fits < 0 || (n_fits > 0 && (!keys || !counts || !A || !Z))) return TEFMM_ERR_INVALID_ARG;
    for (int i = 0; i < n_fits; ++i) {
        const int *k = keys + 6 * i;
        const int lt = k[0], ls = k[1], dir = k[2], lev = k[3], izs = k[4], k3p = k[5];
        if (lt < 0 || lt >= P->nL || ls < 0 || ls >= P->nL || lt == ls || (dir != 0 && dir != 1) ||
            (dir == 0 && lt >= P->nL - 1) || (dir == 1 && lt == 0) || lev < 0 || lev > TEFMM_NBITS ||
            izs < 0 || izs >= (1 << lev) || k3p < 0 || k3p > P->p || counts[i] < 0 ||
            counts[i] > TEFMM_MAX_IMG)
            return TEFMM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n_fits; ++i) {
        const int *k = keys + 6 * i;
        CrossFitVal v{(int)P->xA.size(), counts[i]};
        for (int j = 0; j < counts[i]; ++j) {
            P->xA.push_back(mkc(A[2 * (TEFMM_MAX_IMG * i + j)], A[2 * (TEFMM_MAX_IMG * i + j) + 1]));
            P->xZ.push_back(mkc(Z[2 * (TEFMM_MAX_IMG * i + j)], Z[2 * (TEFMM_MAX_IMG * i + j) + 1]));
        }
        P->xcache[CrossFitKey{k[0], k[1], k[2], k[3], k[4], k[5]}] = v;
    }
    P->x_uploaded = (size_t)-1;   // the device pool is copied again by the next evaluation
    P->geom_ready = false;        // tables of the imported fits are built by the next evaluation
    return TEFMM_OK;
}
