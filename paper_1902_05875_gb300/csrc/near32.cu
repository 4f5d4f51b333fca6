// Near field of the mixed-precision form: L2P in FP64 and the pair sums of
// Algorithm 1's "local direct interactions" in FP32.
//
// For a target leaf, every source box of its near list contributes
//   q_j [ e^{ik r}/(ik r)  (free space, skipped for coincident points)
//       + sum_tau sum_m A_m e^{ik R_m}/(ik R_m) ]  (DCIM images, Sec. 3.3 Step 3)
// with R_m = sqrt(rho^2 + w_m^2), w_m = zeta_tau(z, z') - zeta_min - Z_m.
// Coordinates enter as FP32 offsets from the target leaf's centre (each
// offset formed in FP64); every pair is evaluated in FP32; the sum over one
// source box is kept in FP32 and added to an FP64 accumulator per target.
//
// An image distance w_m is complex and can be large, so e^{ik R_m} in plain
// FP32 would lose its phase and exponent to rounding.  Each image is therefore
// evaluated relative to a reference taken at the leaf centre for both points
// (rho = 0, w = w0_m, so R0 = w0_m): with dw = w - w0 (small, exact in FP32
// offsets), D = R^2 - R0^2 = rho^2 + dw (2 w0 + dw) and delta = R - R0 =
// D / (R + R0),
//   A_m e^{ik R}/(ik R) = E0_m e^{ik delta} / (1 + delta/R0),
//   E0_m = A_m e^{ik R0}/(ik R0)   (FP64, once per leaf and image).
// The image terms of a fit can cancel (terms up to 1e4 times their sum), so
// the constant part is split off:  sum_m E0_m g_m = sum_m E0_m + sum_m E0_m (g_m - 1)
// with g = e^{ik delta}/(1 + delta/R0).  The first sum times the near-field
// charge total is formed once per leaf in FP64; only g - 1 (small for the
// distant images) goes through FP32, written as
//   g - 1 = (e^{ik delta} - 1 - delta/R0) / (1 + delta/R0),
//   e^{a+ib} - 1 = expm1(a) cos b - 2 sin^2(b/2) + i e^a sin b,
// (one sincos of b/2: sin b = 2 sin(b/2) cos(b/2), cos b - 1 = -2 sin^2(b/2)),
// so that its rounding is relative to |g - 1|, not to 1.
// sin, cos, exp and expm1 are CUDA's accurate single-precision functions
// (their arguments here are small: k r within a near box pair and k delta).
// Pairs whose FP32 offsets coincide (r = 0) are skipped in the free-space sum.
#include "ops_common.cuh"

namespace {

struct f2 {
    float x, y;
};

__device__ __forceinline__ f2 csqrt32(float x, float y) {
    float r = sqrtf(x * x + y * y);
    if (r == 0.f) return f2{0.f, 0.f};
    if (x >= 0.f) {
        float t = sqrtf(0.5f * (r + x));
        return f2{t, 0.5f * y * __frcp_rn(t)};
    }
    float t = sqrtf(0.5f * (r - x));
    return f2{0.5f * fabsf(y) * __frcp_rn(t), copysignf(t, y)};
}

__global__ void __launch_bounds__(128) k_near_fp32(int n_items, NearArgs a) {
    // one work item: near sources [src_lo, src_hi) of the leaf's list; chunk 0
    // also adds the constant part and the L2P
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const int node = a.item_node[it], part = a.item_part[it], nparts = a.item_np[it];
    const int64_t src_lo = (int64_t)part * NEAR_CHUNK, src_hi = src_lo + NEAR_CHUNK;
    const TreeArrays &T = a.T;
    if (T.split[node]) return;
    int t0 = T.t0[node], t1 = T.t1[node];
    int nt = t1 - t0;
    if (nt <= 0) return;
    const int TILE = 256;
    constexpr int MI = TEFMM_MAX_TERMS * TEFMM_MAX_IMG;
    __shared__ float xs[TILE], ys[TILE], zs[TILE];
    __shared__ f2 qs[TILE];
    __shared__ double2 red[128];
    // per image: (w0, R0^2) and (1/R0, E0), FP32, two 16-byte loads per pair
    __shared__ float4 sWR[MI], sIE[MI];
    __shared__ float tsz[TEFMM_MAX_TERMS], tszp[TEFMM_MAX_TERMS];
    __shared__ int tcnt[TEFMM_MAX_TERMS];   // images per term
    // images of term ti with -Re Z < thr[lv] (the ones a pair sum with
    // far-of-near level lv evaluates), lv <= the leaf's level
    __shared__ int ncnt[TEFMM_MAX_TERMS][TEFMM_NBITS + 1];
    __shared__ int slot[MI];       // image j of term ti at slot[ti * MAX_IMG + j]: by -Re Z ascending
    // near-field charge totals: [lv] entries with far-of-near level lv, [NBITS + 1] entries without
    __shared__ double2 qlev[TEFMM_NBITS + 2];
    __shared__ double2 cq[1];      // the images' constant part times the charges it applies to
    int lay = T.layer[node];
    cplx k = a.im.k[lay];
    cplx ik = mkc(-k.y, k.x);
    cplx inv_ik = cdiv(mkc(1, 0), ik);
    int l = T.level[node];
    double h = box_h(a.cb.side, l);
    double cx = centre(a.cb.lo[0], T.ix[node], h), cy = centre(a.cb.lo[1], T.iy[node], h),
           cz = centre(a.cb.lo[2], T.iz[node], h);
    int tf = a.im.lt_first[lay], ntm = a.im.lt_count[lay];
    for (int i = threadIdx.x; i < TEFMM_NBITS + 2; i += blockDim.x) qlev[i] = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) cq[0] = make_double2(0.0, 0.0);
    if (threadIdx.x < ntm) {
        DevTerm t = a.im.terms[tf + threadIdx.x];
        tsz[threadIdx.x] = (float)t.sz;
        tszp[threadIdx.x] = (float)t.szp;
        tcnt[threadIdx.x] = t.count;
        // rank by depth -Re Z (ties by index; a NaN depth counts as near)
        for (int j = 0; j < t.count; ++j) {
            const double dj = -a.im.Z[t.first + j].x;
            const double kj = dj == dj ? dj : -INFINITY;
            int r = 0;
            for (int i = 0; i < t.count; ++i) {
                const double di = -a.im.Z[t.first + i].x;
                const double ki_ = di == di ? di : -INFINITY;
                r += (ki_ < kj) || (ki_ == kj && i < j);
            }
            slot[threadIdx.x * TEFMM_MAX_IMG + j] = r;
        }
        for (int lv = 0; lv <= l; ++lv) {
            const double thr = a.fon.on ? a.fon.thr[lv] : INFINITY;
            int c = 0;
            for (int j = 0; j < t.count; ++j) c += !(-a.im.Z[t.first + j].x >= thr);
            ncnt[threadIdx.x][lv] = c;
        }
    }
    __syncthreads();
    // near-field charge totals (FP64) by far-of-near level (chunk 0 only)
    for (int nb = a.near_ptr[node]; part == 0 && nb < a.near_ptr[node + 1]; ++nb) {
        const int sb = a.near_src[nb];
        const int fl = a.fon.on ? a.near_fl[nb] : -1;
        double qr = 0.0, qi = 0.0;
        bool any = false;
        for (int j = T.s0[sb] + threadIdx.x; j < T.s1[sb]; j += blockDim.x) {
            qr += a.sq[2 * j];
            qi += a.sq[2 * j + 1];
            any = true;
        }
        if (any) {
            double2 *dst = &qlev[fl >= 0 ? fl : TEFMM_NBITS + 1];
            atomicAdd(&dst->x, qr);
            atomicAdd(&dst->y, qi);
        }
    }
    __syncthreads();
    // per-image reference at the leaf centre (FP64); the constant part E0 times
    // the charge of the entries that evaluate the image
    for (int ti = 0; ti < ntm; ++ti) {
        DevTerm t = a.im.terms[tf + ti];
        for (int j = threadIdx.x; j < t.count; j += blockDim.x) {
            cplx Z = a.im.Z[t.first + j];
            cplx w0 = mkc((t.sz + t.szp) * cz + t.c - t.zmin - Z.x, -Z.y);
            cplx e = cexp_(cmul(ik, w0));                       // R0 = w0
            cplx E0 = cmul(cmul(a.im.A[t.first + j], inv_ik), cdiv(e, w0));
            cplx r0sq = cmul(w0, w0);
            cplx ir0 = cdiv(mkc(1, 0), w0);
            const int r = slot[ti * TEFMM_MAX_IMG + j];
            int s = ti * TEFMM_MAX_IMG + r;
            sWR[s] = make_float4((float)w0.x, (float)w0.y, (float)r0sq.x, (float)r0sq.y);
            sIE[s] = make_float4((float)ir0.x, (float)ir0.y, (float)E0.x, (float)E0.y);
            cplx qw = mkc(qlev[TEFMM_NBITS + 1].x, qlev[TEFMM_NBITS + 1].y);
            for (int lv = 0; lv <= l; ++lv)
                if (r < ncnt[ti][lv]) qw = cadd(qw, mkc(qlev[lv].x, qlev[lv].y));
            const cplx c = cmul(E0, qw);
            atomicAdd(&cq[0].x, c.x);
            atomicAdd(&cq[0].y, c.y);
        }
    }
    __syncthreads();

    const float kr = (float)k.x, ki = (float)k.y;
    const f2 iik = f2{(float)inv_ik.x, (float)inv_ik.y};
    // thread -> (target, source slice): ntp = min(nt, 128) targets at a time,
    // nslice = 128 / ntp slices of the sources; the 128 - ntp * nslice
    // remaining threads only help with the loads
    const int ntp = min(nt, 128);
    const int nslice = 128 / ntp;
    const int my_t = threadIdx.x % ntp, slice = threadIdx.x / ntp;
    const bool in_grid = slice < nslice;
    int nb0 = a.near_ptr[node], nb1 = a.near_ptr[node + 1];
    for (int tbase = 0; tbase < nt; tbase += ntp) {
        int ti = tbase + my_t;
        bool active = in_grid && ti < nt;
        double xt = 0, yt = 0, zt = 0;
        if (active) {
            xt = a.tx[t0 + ti];
            yt = a.ty[t0 + ti];
            zt = a.tz[t0 + ti];
        }
        const float xf = (float)(xt - cx), yf = (float)(yt - cy), zf = (float)(zt - cz);
        double accr = 0.0, acci = 0.0;
        __syncthreads();
        int64_t off = 0;           // near sources of the list before entry nb
        for (int nb = nb0; nb < nb1 && off < src_hi; ++nb) {
            int s = a.near_src[nb];
            int s0 = T.s0[s], s1 = T.s1[s];
            const int64_t ns_e = s1 - s0;
            // this item's part of the entry
            const int b0 = (int)(s0 + max((int64_t)0, src_lo - off));
            const int b1 = (int)(s0 + min(ns_e, src_hi - off));
            off += ns_e;
            if (b0 >= b1) continue;
            s0 = b0;
            s1 = b1;
            const int fl = a.fon.on ? a.near_fl[nb] : -1;   // far images of the anchor already in M2L
            for (int base = s0; base < s1; base += TILE) {
                int cnt = min(TILE, s1 - base);
                __syncthreads();
                for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
                    xs[j] = (float)(a.sx[base + j] - cx);
                    ys[j] = (float)(a.sy[base + j] - cy);
                    zs[j] = (float)(a.sz[base + j] - cz);
                    qs[j] = f2{(float)a.sq[2 * (base + j)], (float)a.sq[2 * (base + j) + 1]};
                }
                __syncthreads();
                if (!active) continue;
                float fr = 0.f, fi = 0.f;      // free space, times q
                float gr = 0.f, gi = 0.f;      // images, times q
                for (int j = slice; j < cnt; j += nslice) {
                    float dx = xf - xs[j], dy = yf - ys[j], dz = zf - zs[j];
                    float rho2 = dx * dx + dy * dy;
                    float r2 = rho2 + dz * dz;
                    f2 q = qs[j];
                    if (r2 > 0.f) {
                        float r = sqrtf(r2);
                        float sn, cs;
                        sincosf(kr * r, &sn, &cs);
                        float m = expf(-ki * r) * __frcp_rn(r);
                        float er = m * cs, ei = m * sn;
                        fr += q.x * er - q.y * ei;
                        fi += q.x * ei + q.y * er;
                    }
                    float hr = 0.f, hi = 0.f;
                    for (int tm = 0; tm < ntm; ++tm) {
                        const float dw = tsz[tm] * zf + tszp[tm] * zs[j];   // w - w0 (real)
                        const int lim = fl >= 0 ? ncnt[tm][fl] : tcnt[tm];
                        for (int m = 0; m < lim; ++m) {
                            const int sidx = tm * TEFMM_MAX_IMG + m;
                            const float4 wr = sWR[sidx];
                            const f2 w0 = f2{wr.x, wr.y}, r0s = f2{wr.z, wr.w};
                            // D = rho^2 + dw (2 w0 + dw)
                            float Dr = rho2 + dw * (2.f * w0.x + dw), Di = dw * 2.f * w0.y;
                            // R = sqrt(R0^2 + D) (principal), delta = D / (R + R0)
                            f2 R = csqrt32(r0s.x + Dr, r0s.y + Di);
                            float sr = R.x + w0.x, si = R.y + w0.y;
                            float isn = __frcp_rn(sr * sr + si * si);
                            float der = (Dr * sr + Di * si) * isn, dei = (Di * sr - Dr * si) * isn;
                            // e^{i k delta} - 1
                            float ph = kr * der - ki * dei, dec = -(kr * dei + ki * der);
                            // half-angle: sin ph = 2 s c, cos ph = 1 - 2 s^2 (one sincos)
                            float sh, ch;
                            sincosf(0.5f * ph, &sh, &ch);
                            const float sn = 2.f * sh * ch, cm1 = -2.f * sh * sh;   // cos ph - 1
                            float em1 = expm1f(dec);
                            float ur = em1 * (1.f + cm1) + cm1, ui = (1.f + em1) * sn;
                            // delta / R0 and g - 1 = (e^{ik delta} - 1 - delta/R0) / (1 + delta/R0)
                            const float4 ie = sIE[sidx];
                            float tr = der * ie.x - dei * ie.y, ti = der * ie.y + dei * ie.x;
                            float nr = ur - tr, ni = ui - ti;
                            float vr = 1.f + tr, vi = ti;
                            float iv = __frcp_rn(vr * vr + vi * vi);
                            float pr = (nr * vr + ni * vi) * iv, pi = (ni * vr - nr * vi) * iv;
                            hr += ie.z * pr - ie.w * pi;
                            hi += ie.z * pi + ie.w * pr;
                        }
                    }
                    gr += q.x * hr - q.y * hi;
                    gi += q.x * hi + q.y * hr;
                }
                // free part still needs the factor 1/(ik)
                float ur = iik.x * fr - iik.y * fi, ui = iik.x * fi + iik.y * fr;
                accr += (double)(ur + gr);
                acci += (double)(ui + gi);
            }
        }
        __syncthreads();
        red[threadIdx.x] = make_double2(accr, acci);
        __syncthreads();
        if (slice == 0 && active) {
            for (int sl = 1; sl < nslice; ++sl) {
                accr += red[sl * ntp + my_t].x;
                acci += red[sl * ntp + my_t].y;
            }
            if (part == 0) {
                accr += cq[0].x;       // the images' constant part times the charge total
                acci += cq[0].y;
                // L2P in FP64
                double d[3] = {xt - cx, yt - cy, zt - cz};
                double pw[3][13];
                for (int e = 0; e < 3; ++e) {
                    double v = 1.0;
                    for (int qq = 0; qq <= a.p; ++qq) {
                        pw[e][qq] = v;
                        v *= d[e];
                    }
                }
                const cplx *bt = a.beta + (int64_t)node * a.np;
                for (int kk = 0; kk < a.np; ++kk) {
                    double m = pw[0][a.mi[3 * kk]] * pw[1][a.mi[3 * kk + 1]] * pw[2][a.mi[3 * kk + 2]];
                    cplx b = bt[kk];
                    accr += b.x * m;
                    acci += b.y * m;
                }
            }
            if (a.scale) {                // i k / (4 pi)
                const double sr = -k.y / (4.0 * M_PI), si = k.x / (4.0 * M_PI);
                const double vr = accr * sr - acci * si, vi = accr * si + acci * sr;
                accr = vr;
                acci = vi;
            }
            int out = a.perm_t[t0 + ti];
            if (nparts == 1) {
                a.phi[2 * out] = accr;
                a.phi[2 * out + 1] = acci;
            } else {                  // chunks of one leaf add into zeroed outputs
                atomicAdd(&a.phi[2 * out], accr);
                atomicAdd(&a.phi[2 * out + 1], acci);
            }
        }
    }
}

}  // namespace

int near_field_fp32(tefmm_plan_s *P, double *phi, cudaStream_t st) {
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
        k_near_fp32<<<P->n_near_items, 128, 0, st>>>(P->n_near_items, a);
        P->launches++;
    }
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}
