// Plan lifetime, operator tables and image storage.
#include <math.h>
#include <string.h>

#include <atomic>

#include "internal.cuh"

// Fault injection for the tests of the error paths (tefmm_debug_inject):
// countdowns of device allocations and of DCIM fit batches; the one that
// reaches zero fails.  -1 / 0: nothing injected.
static std::atomic<int> g_inject_alloc{0}, g_inject_fit{0};

static bool countdown_hits(std::atomic<int> &c) {
    int v = c.load();
    while (v > 0) {
        if (c.compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}
bool inject_alloc_failure() { return countdown_hits(g_inject_alloc); }
bool inject_fit_failure() { return countdown_hits(g_inject_fit); }

extern "C" int tefmm_debug_inject(int kind, int n) {
    if (kind == 0) {
        g_inject_alloc = 0;
        g_inject_fit = 0;
        return TEFMM_OK;
    }
    if (n < 1) return TEFMM_ERR_INVALID_ARG;
    if (kind == TEFMM_INJECT_ALLOC) g_inject_alloc = n;
    else if (kind == TEFMM_INJECT_FIT) g_inject_fit = n;
    else return TEFMM_ERR_INVALID_ARG;
    return TEFMM_OK;
}

int dbuf_ensure(DBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return TEFMM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (inject_alloc_failure()) return TEFMM_ERR_OOM;
    size_t cap = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(&b.p, cap);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return TEFMM_ERR_OOM;
    }
    b.cap = cap;
    return TEFMM_OK;
}

void dbuf_free(DBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

// M2L coefficient tables: rows k and columns k' both in the graded order.
//   G[k'*np + k]  = index of k + k' in the order-2p list
//   cB[k'*np + k] = C(k+k', k) (-1)^{k1'+k2'} (-1)^{k3'}
//   cA[k'*np + k] = C(k+k', k) (-1)^{k1'+k2'}
// with C(k+k', k) = prod_i (k_i + k'_i)! / (k_i! k'_i!).
int plan_build_operator_tables(tefmm_plan_s *P) {
    const int p = P->p, np = ncoef(p), np2 = ncoef(2 * p);
    P->np = np;
    P->np2 = np2;
    std::vector<int> mi(3 * np2);
    int t = 0;
    for (int n = 0; n <= 2 * p; ++n)
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
    std::vector<double> cB((size_t)np * np), cA((size_t)np * np);
    for (int kp = 0; kp < np; ++kp)
        for (int k = 0; k < np; ++k) {
            int g1 = mi[3 * k] + mi[3 * kp], g2 = mi[3 * k + 1] + mi[3 * kp + 1],
                g3 = mi[3 * k + 2] + mi[3 * kp + 2];
            G[(size_t)kp * np + k] = (unsigned short)midx(g1, g2, g3);
            double m = comb(g1, mi[3 * k]) * comb(g2, mi[3 * k + 1]) * comb(g3, mi[3 * k + 2]);
            double sxy = ((mi[3 * kp] + mi[3 * kp + 1]) & 1) ? -1.0 : 1.0;
            double s3 = (mi[3 * kp + 2] & 1) ? -1.0 : 1.0;
            cA[(size_t)kp * np + k] = m * sxy;
            cB[(size_t)kp * np + k] = m * sxy * s3;
        }
    TRY(dbuf_ensure(P->d_mi, mi.size() * sizeof(int)));
    TRY(dbuf_ensure(P->d_m2l_g, G.size() * sizeof(unsigned short)));
    TRY(dbuf_ensure(P->d_m2l_cB, cB.size() * sizeof(double)));
    TRY(dbuf_ensure(P->d_m2l_cA, cA.size() * sizeof(double)));
    CUDA_TRY(cudaMemcpy(P->d_mi.p, mi.data(), mi.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->d_m2l_g.p, G.data(), G.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->d_m2l_cB.p, cB.data(), cB.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->d_m2l_cA.p, cA.data(), cA.size() * sizeof(double), cudaMemcpyHostToDevice));
    return TEFMM_OK;
}

// d_k layout: cplx k[16]; int term_first[16]; int term_count[16]
int plan_upload_images(tefmm_plan_s *P) {
    std::vector<DevTerm> dt(P->terms.size() + 1);
    for (int l = 0; l < TEFMM_MAX_LAYERS; ++l) {
        P->layer_term_first[l] = 0;
        P->layer_term_count[l] = 0;
    }
    for (size_t i = 0; i < P->terms.size(); ++i) {
        const TermDesc &t = P->terms[i];
        dt[i] = DevTerm{t.sz, t.szp, t.c, t.zmin, t.first, t.count, t.layer, t.tag};
        if (P->layer_term_count[t.layer] == 0) P->layer_term_first[t.layer] = (int)i;
        P->layer_term_count[t.layer]++;
    }
    size_t nimg = P->A.size();
    TRY(dbuf_ensure(P->d_terms, dt.size() * sizeof(DevTerm)));
    TRY(dbuf_ensure(P->d_A, (nimg + 1) * sizeof(cplx)));
    TRY(dbuf_ensure(P->d_Z, (nimg + 1) * sizeof(cplx)));
    TRY(dbuf_ensure(P->d_k, TEFMM_MAX_LAYERS * (sizeof(cplx) + 2 * sizeof(int))));
    CUDA_TRY(cudaMemcpy(P->d_terms.p, dt.data(), dt.size() * sizeof(DevTerm), cudaMemcpyHostToDevice));
    if (nimg) {
        CUDA_TRY(cudaMemcpy(P->d_A.p, P->A.data(), nimg * sizeof(cplx), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(P->d_Z.p, P->Z.data(), nimg * sizeof(cplx), cudaMemcpyHostToDevice));
    }
    char buf[TEFMM_MAX_LAYERS * (sizeof(cplx) + 2 * sizeof(int))];
    memcpy(buf, P->k, TEFMM_MAX_LAYERS * sizeof(cplx));
    memcpy(buf + TEFMM_MAX_LAYERS * sizeof(cplx), P->layer_term_first, TEFMM_MAX_LAYERS * sizeof(int));
    memcpy(buf + TEFMM_MAX_LAYERS * (sizeof(cplx) + sizeof(int)), P->layer_term_count,
           TEFMM_MAX_LAYERS * sizeof(int));
    CUDA_TRY(cudaMemcpy(P->d_k.p, buf, sizeof(buf), cudaMemcpyHostToDevice));
    return TEFMM_OK;
}

// Same-layer reaction terms of layer l (image-distance form):
//   up-up   (l < L):      zeta = z + z' - 2 d_l
//   down-down (l > 0):    zeta = 2 d_{l-1} - z - z'
//   up-down (0 < l < L):  zeta = z - z' + 2 D_l
//   down-up (0 < l < L):  zeta = z' - z + 2 D_l
// zeta_min is the smallest zeta over the layer's particle slab [zlo, zhi].
static void make_terms(tefmm_plan_s *P) {
    P->terms.clear();
    const int L = P->nL - 1;
    for (int l = 0; l <= L && L > 0; ++l) {
        double zlo = P->opt.zext[2 * l], zhi = P->opt.zext[2 * l + 1];
        if (l < L) P->terms.push_back(TermDesc{l, 0, 0, 0, 1.0, 1.0, -2.0 * P->d[l], 2.0 * zlo - 2.0 * P->d[l]});
        if (l > 0)
            P->terms.push_back(TermDesc{l, 1, 0, 0, -1.0, -1.0, 2.0 * P->d[l - 1], 2.0 * P->d[l - 1] - 2.0 * zhi});
        if (l > 0 && l < L) {
            double D = P->d[l - 1] - P->d[l];
            P->terms.push_back(TermDesc{l, 2, 0, 0, 1.0, -1.0, 2.0 * D, (zlo - zhi) + 2.0 * D});
            P->terms.push_back(TermDesc{l, 3, 0, 0, -1.0, 1.0, 2.0 * D, (zlo - zhi) + 2.0 * D});
        }
    }
}

extern "C" int tefmm_default_options(tefmm_options *opt) {
    if (!opt) return TEFMM_ERR_INVALID_ARG;
    memset(opt, 0, sizeof(*opt));
    opt->p = 6;
    opt->leaf_cap = 64;
    opt->max_level = TEFMM_NBITS;
    opt->precision = TEFMM_FP64;
    opt->n_images = 8;
    opt->n_samples = 101;
    opt->T1 = 10.0;
    opt->T0 = 0.0;
    for (int l = 0; l < TEFMM_MAX_LAYERS; ++l) {
        opt->zext[2 * l] = NAN;
        opt->zext[2 * l + 1] = NAN;
    }
    opt->kh_max = 3.5;
    opt->far_of_near = 1;
    opt->algorithm = TEFMM_ALG_RECURRENCE;
    opt->split = TEFMM_SPLIT_TF32X3;
    opt->scale_output = 0;
    opt->table_n = 0;
    return TEFMM_OK;
}

extern "C" int tefmm_plan_create(int n_layers, const double *interfaces, const double *k_re,
                                 const double *k_im, const tefmm_options *opt, void *stream,
                                 tefmm_plan *out) {
    if (!out || n_layers < 1 || n_layers > 8 || !k_re || !k_im) return TEFMM_ERR_INVALID_ARG;
    if (n_layers > 1 && !interfaces) return TEFMM_ERR_INVALID_ARG;
    for (int m = 0; m + 1 < n_layers - 1; ++m)
        if (!(interfaces[m] > interfaces[m + 1])) return TEFMM_ERR_INVALID_ARG;
    for (int l = 0; l < n_layers; ++l)
        if (!(k_im[l] >= 0.0) || !(k_re[l] > 0.0)) return TEFMM_ERR_INVALID_ARG;
    tefmm_options o;
    if (opt) o = *opt;
    else tefmm_default_options(&o);
    if (o.p < 1 || o.p > 12 || o.leaf_cap < 0 || o.max_level < 1 || o.max_level > TEFMM_NBITS ||
        o.n_images < 0 || o.n_images > TEFMM_MAX_IMG || o.n_samples < 8 || o.n_samples > 127 ||
        !(o.T1 > 0) || (o.precision != TEFMM_FP64 && o.precision != TEFMM_MIXED) ||
        isnan(o.kh_max) || (o.scale_output != 0 && o.scale_output != 1) ||
        (o.far_of_near != 0 && o.far_of_near != 1) ||
        (o.algorithm != TEFMM_ALG_RECURRENCE && o.algorithm != TEFMM_ALG_TABLES) ||
        (o.table_n != 0 && (o.table_n < 8 || o.table_n > 512)))
        return TEFMM_ERR_INVALID_ARG;
    if (o.split != TEFMM_SPLIT_TF32X3) return TEFMM_ERR_NOT_IMPLEMENTED;
    // default particle ranges: the whole layer (top/bottom: one unit beyond the interface)
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
    tefmm_plan_s *P = new tefmm_plan_s();
    P->leaf_cap_eff = o.leaf_cap;      // 0: chosen by the autotuner on the first evaluation
    // HX = 4 min over interfaces of (gap above + gap below) between the particle
    // slabs and the interface; interfaces without a gap do not count
    {
        double gmin = INFINITY;
        for (int m = 0; m + 1 < n_layers; ++m) {
            const double gm = (o.zext[2 * m] - interfaces[m]) + (interfaces[m] - o.zext[2 * (m + 1) + 1]);
            if (gm > 0.0 && gm < gmin) gmin = gm;
        }
        P->HX = gmin < INFINITY ? 4.0 * gmin : INFINITY;
    }
    P->nL = n_layers;
    for (int m = 0; m < n_layers - 1; ++m) P->d[m] = interfaces[m];
    for (int l = 0; l < n_layers; ++l) {
        P->k[l] = mkc(k_re[l], k_im[l]);
        P->kmax = fmax(P->kmax, hypot(k_re[l], k_im[l]));
    }
    P->opt = o;
    P->p = o.p;
    cudaGetDevice(&P->device);
    int r = plan_build_operator_tables(P);
    if (r == TEFMM_OK) {
        make_terms(P);
        r = plan_fit_images(P, (cudaStream_t)stream);
    }
    if (r == TEFMM_OK) r = plan_upload_images(P);
    if (r == TEFMM_OK)
        for (int i = 0; i < 12; ++i)
            if (cudaEventCreate(&P->ev[i]) != cudaSuccess) r = TEFMM_ERR_CUDA;
    if (r != TEFMM_OK) {
        tefmm_plan_destroy(P);
        return r;
    }
    *out = P;
    return TEFMM_OK;
}

extern "C" int tefmm_plan_destroy(tefmm_plan P) {
    if (!P) return TEFMM_OK;
    DBuf *all[] = {&P->d_terms, &P->d_A, &P->d_Z, &P->d_k, &P->d_mi, &P->d_m2l_g, &P->d_m2l_cB,
                   &P->d_m2l_cA, &P->keys_in, &P->keys_out, &P->vals_in,
                   &P->vals_out, &P->sort_tmp, &P->scan_tmp, &P->item_node, &P->item_flag,
                   &P->item_scan, &P->cnt_s, &P->cnt_t, &P->sx, &P->sy, &P->sz, &P->sq, &P->tx,
                   &P->ty, &P->tz, &P->perm_s, &P->perm_t, &P->n_layer, &P->n_level, &P->n_ix,
                   &P->n_iy, &P->n_iz, &P->n_parent, &P->n_cfirst, &P->n_nchild, &P->n_s0,
                   &P->n_s1, &P->n_t0, &P->n_t1, &P->n_i0, &P->n_i1, &P->n_split, &P->n_key, &P->bbox,
                   &P->flags, &P->counters, &P->C_list, &P->C_cnt, &P->D_list, &P->D_cnt,
                   &P->X_list, &P->X_cnt, &P->V_tmp, &P->V_cnt, &P->v_ptr, &P->v_src,
                   &P->near_ptr, &P->near_src, &P->near_tmp, &P->near_cnt, &P->alpha, &P->beta,
                   &P->keyslot_flag, &P->keyslot_table, &P->pair_t, &P->pair_s, &P->pair_slot,
                   &P->pair_slot_sorted, &P->pair_idx, &P->pair_idx_sorted, &P->chunk_key,
                   &P->chunk_start, &P->chunk_cnt, &P->tables, &P->table_slot, &P->seg_tmp, &P->table_rep,
                   &P->h_in, &P->h_out, &P->fon_cnt, &P->fon_ptr, &P->fon_key, &P->fon_key_sorted, &P->near_fl, &P->nitem_cnt, &P->nitem_pos, &P->nitem_node, &P->nitem_part, &P->nitem_np, &P->tc_ah, &P->tc_al, &P->tc_bt, &P->tc_cfA, &P->tc_cfB, &P->tc_W};
    for (DBuf *b : all) dbuf_free(*b);
    cross_release(P);
    alg2_release(P);
    for (int i = 0; i < 12; ++i)
        if (P->ev[i]) cudaEventDestroy(P->ev[i]);
    for (cudaEvent_t e : P->kev) cudaEventDestroy(e);
    delete P;
    return TEFMM_OK;
}

extern "C" int tefmm_plan_image_counts(tefmm_plan P, int *n_terms, int *n_images) {
    if (!P) return TEFMM_ERR_INVALID_ARG;
    if (n_terms) *n_terms = (int)P->terms.size();
    if (n_images) *n_images = (int)P->A.size();
    return TEFMM_OK;
}

extern "C" int tefmm_plan_get_images(tefmm_plan P, int *term_layer, int *term_tag, int *term_first,
                                     int *term_count, double *term_geom, double *A, double *Z) {
    if (!P) return TEFMM_ERR_INVALID_ARG;
    for (size_t i = 0; i < P->terms.size(); ++i) {
        const TermDesc &t = P->terms[i];
        if (term_layer) term_layer[i] = t.layer;
        if (term_tag) term_tag[i] = t.tag;
        if (term_first) term_first[i] = t.first;
        if (term_count) term_count[i] = t.count;
        if (term_geom) {
            term_geom[4 * i] = t.sz;
            term_geom[4 * i + 1] = t.szp;
            term_geom[4 * i + 2] = t.c;
            term_geom[4 * i + 3] = t.zmin;
        }
    }
    for (size_t j = 0; j < P->A.size(); ++j) {
        if (A) {
            A[2 * j] = P->A[j].x;
            A[2 * j + 1] = P->A[j].y;
        }
        if (Z) {
            Z[2 * j] = P->Z[j].x;
            Z[2 * j + 1] = P->Z[j].y;
        }
    }
    return TEFMM_OK;
}

extern "C" int tefmm_plan_set_images(tefmm_plan P, const int *term_count, const double *A,
                                     const double *Z) {
    if (!P || !term_count) return TEFMM_ERR_INVALID_ARG;
    int tot = 0;
    for (size_t i = 0; i < P->terms.size(); ++i) {
        if (term_count[i] < 0 || term_count[i] > TEFMM_MAX_IMG) return TEFMM_ERR_INVALID_ARG;
        tot += term_count[i];
    }
    if (tot > 0 && (!A || !Z)) return TEFMM_ERR_INVALID_ARG;
    P->geom_ready = false;      // the derivative tables depend on the images
    P->A.assign(tot, mkc(0, 0));
    P->Z.assign(tot, mkc(0, 0));
    int f = 0;
    for (size_t i = 0; i < P->terms.size(); ++i) {
        P->terms[i].first = f;
        P->terms[i].count = term_count[i];
        f += term_count[i];
    }
    for (int j = 0; j < tot; ++j) {
        P->A[j] = mkc(A[2 * j], A[2 * j + 1]);
        P->Z[j] = mkc(Z[2 * j], Z[2 * j + 1]);
    }
    return plan_upload_images(P);
}
