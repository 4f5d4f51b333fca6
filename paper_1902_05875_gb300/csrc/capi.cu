// C-ABI entry points: evaluation, statistics and inspection hooks.
#include <string.h>

#include "internal.cuh"

extern "C" const char *tefmm_status_string(int s) {
    switch (s) {
        case TEFMM_OK: return "ok";
        case TEFMM_ERR_INVALID_ARG: return "invalid argument";
        case TEFMM_ERR_POINT_ON_INTERFACE: return "a point lies exactly on an interface";
        case TEFMM_ERR_OUT_OF_DOMAIN: return "a point lies outside its layer's particle range";
        case TEFMM_ERR_OOM: return "device allocation failed";
        case TEFMM_ERR_CUDA: return "CUDA runtime error";
        case TEFMM_ERR_FIT_FAILED: return "DCIM fit failed";
        case TEFMM_ERR_LIST_OVERFLOW: return "interaction list capacity exceeded";
        case TEFMM_ERR_NOT_IMPLEMENTED: return "configuration not implemented";
        case TEFMM_ERR_DEVICE_CHECK: return "device-side check failed";
        case TEFMM_ERR_TIMEOUT: return "a bounded device wait ran out";
        default: return "unknown status";
    }
}

namespace {
__global__ void k_zero(int64_t n, double *a) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0.0;
}

// charges into the plan's source order: sq[pos] = q[perm_s[pos]]
__global__ void k_gather_q(int64_t ns, const int *__restrict__ perm_s, const double *__restrict__ q,
                           double *__restrict__ sq) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int64_t v = perm_s[i];
    sq[2 * i] = q[2 * v];
    sq[2 * i + 1] = q[2 * v + 1];
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}
}  // namespace

namespace {
int eval_once(tefmm_plan P, int64_t ns, const double *sx, const double *sy, const double *sz,
              const double *q, int64_t nt, const double *tx, const double *ty, const double *tz,
              double *phi, cudaStream_t st);
int geometry(tefmm_plan P, int64_t ns, const double *sx, const double *sy, const double *sz,
             const double *q, int64_t nt, const double *tx, const double *ty, const double *tz,
             cudaStream_t st);
int charge_phases(tefmm_plan P, double *phi, cudaStream_t st);
int tables(tefmm_plan P, cudaStream_t st);
int zero_output(int64_t nt, double *phi, cudaStream_t st, tefmm_plan P);
}

// Leaf-cap autotuner: with leaf_cap = 0 the first evaluation tries each cap of
// TUNE_CAPS (the trade between near-field pairs and M2L translations depends on
// p, the images per term, the precision and the particle distribution), times
// each trial with CUDA events, keeps the fastest for the plan's lifetime and
// evaluates once more with it.
extern "C" int tefmm_eval(tefmm_plan P, int64_t ns, const double *sx, const double *sy,
                          const double *sz, const double *q, int64_t nt, const double *tx,
                          const double *ty, const double *tz, double *phi, void *stream) {
    if (!P || ns < 0 || nt < 0 || ns > (1LL << 30) || nt > (1LL << 30)) return TEFMM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (P->leaf_cap_eff == 0 && ns > 0 && nt > 0) {
        static const int TUNE_CAPS[] = {16, 32, 64, 128, 256};
        float best = 1e30f;
        int best_cap = 64;
        for (int cap : TUNE_CAPS) {
            P->leaf_cap_eff = cap;
            float ms = 0.f;
            CUDA_TRY(cudaEventRecord(P->ev[9], st));
            int r = eval_once(P, ns, sx, sy, sz, q, nt, tx, ty, tz, phi, st);
            CUDA_TRY(cudaEventRecord(P->ev[10], st));
            CUDA_TRY(cudaEventSynchronize(P->ev[10]));
            CUDA_TRY(cudaEventElapsedTime(&ms, P->ev[9], P->ev[10]));
            if (r != TEFMM_OK) continue;       // e.g. a cap that leaves cross-layer near pairs
            P->ms_autotune += ms;
            if (ms < best) {
                best = ms;
                best_cap = cap;
            }
        }
        P->leaf_cap_eff = best_cap;
    }
    return eval_once(P, ns, sx, sy, sz, q, nt, tx, ty, tz, phi, st);
}

// Geometry once, charges many times (an iterative solver's matrix-vector
// products): set_points builds the trees, lists, M2L keys, cross-layer fits
// and derivative tables of the points; apply then runs only the phases that
// depend on the charges.  A plan made with leaf_cap = 0 uses the cap its
// autotuner chose in an earlier tefmm_eval, else 64.
extern "C" int tefmm_set_points(tefmm_plan P, int64_t ns, const double *sx, const double *sy,
                                const double *sz, int64_t nt, const double *tx, const double *ty,
                                const double *tz, void *stream) {
    if (!P || ns < 0 || nt < 0 || ns > (1LL << 30) || nt > (1LL << 30)) return TEFMM_ERR_INVALID_ARG;
    if (ns > 0 && (!sx || !sy || !sz)) return TEFMM_ERR_INVALID_ARG;
    if (nt > 0 && (!tx || !ty || !tz)) return TEFMM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (P->leaf_cap_eff == 0) P->leaf_cap_eff = 64;
    TRY(geometry(P, ns, sx, sy, sz, nullptr, nt, tx, ty, tz, st));
    if (ns == 0 || nt == 0) return TEFMM_OK;
    TRY(tables(P, st));
    P->geom_ready = true;
    return TEFMM_OK;
}

extern "C" int tefmm_apply(tefmm_plan P, const double *q, double *phi, void *stream) {
    if (!P || !P->geom_ready) return TEFMM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (P->ns == 0 || P->nt == 0) return zero_output(P->nt, phi, st, P);
    if (!q || !phi) return TEFMM_ERR_INVALID_ARG;
    CUDA_TRY(cudaEventRecord(P->ev[0], st));
    k_gather_q<<<grid_for(P->ns, 256), 256, 0, st>>>(P->ns, dp<int>(P->perm_s), q, dp<double>(P->sq));
    P->launches++;
    CUDA_TRY(cudaEventRecord(P->ev[1], st));
    TRY(upward_pass(P, st));
    // no tables to build: ev[2], ev[7] and ev[3] mark an empty phase
    CUDA_TRY(cudaEventRecord(P->ev[2], st));
    CUDA_TRY(cudaEventRecord(P->ev[7], st));
    CUDA_TRY(cudaEventRecord(P->ev[3], st));
    return charge_phases(P, phi, st);
}

namespace {
// tree, lists, M2L keys, cross-layer fits (ev[0] .. ev[1]); with q == nullptr
// the sorted charges are left alone (set_points)
int geometry(tefmm_plan P, int64_t ns, const double *sx, const double *sy, const double *sz,
             const double *q, int64_t nt, const double *tx, const double *ty, const double *tz,
             cudaStream_t st) {
    P->geom_ready = false;
    P->ns = ns;
    P->nt = nt;
    P->shared_pts = (tx == sx && ty == sy && tz == sz && nt == ns);
    if (ns == 0 || nt == 0) {
        P->geom_ready = true;
        return TEFMM_OK;
    }
    CUDA_TRY(cudaEventRecord(P->ev[0], st));
    TRY(tree_build(P, sx, sy, sz, q, tx, ty, tz, st));
    TRY(check_flags(P, st));
    TRY(lists_build(P, st));
    TRY(check_flags(P, st));
    TRY(m2l_prepare(P, st));
    TRY(alg2_prepare(P, st));
    TRY(cross_prepare(P, st));
    CUDA_TRY(cudaEventRecord(P->ev[1], st));
    return TEFMM_OK;
}

// derivative tables (ev[2] .. ev[3], cross-layer from ev[7])
int tables(tefmm_plan P, cudaStream_t st) {
    CUDA_TRY(cudaEventRecord(P->ev[2], st));
    TRY(m2l_tables(P, st));
    CUDA_TRY(cudaEventRecord(P->ev[7], st));
    TRY(cross_tables(P, st));
    CUDA_TRY(cudaEventRecord(P->ev[3], st));
    return TEFMM_OK;
}

// M2L, L2L, L2P and near field for the sorted charges (ev[3] .. ev[6]), then
// the device flags of the whole evaluation
int charge_phases(tefmm_plan P, double *phi, cudaStream_t st) {
    P->kev_used = 0;
    if (P->opt.precision == TEFMM_MIXED) TRY(m2l_apply_tc(P, st));
    else TRY(m2l_apply(P, st));
    CUDA_TRY(cudaEventRecord(P->ev[8], st));
    TRY(cross_apply(P, st));
    CUDA_TRY(cudaEventRecord(P->ev[4], st));
    TRY(downward_pass(P, st));
    CUDA_TRY(cudaEventRecord(P->ev[5], st));
    if (P->opt.precision == TEFMM_MIXED) TRY(near_field_fp32(P, phi, st));
    else TRY(near_field(P, phi, st));
    CUDA_TRY(cudaEventRecord(P->ev[6], st));
    CUDA_TRY(cudaGetLastError());
    // flags raised after the list checks (M2L key range, bounded waits of the
    // tensor-core kernel) are reported by this call, before the next one resets
    // them; work queued into a stream capture cannot wait for them, and
    // tefmm_plan_status reads them after the graph has run
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return TEFMM_OK;
    return check_flags(P, st);
}

int zero_output(int64_t nt, double *phi, cudaStream_t st, tefmm_plan P) {
    if (nt > 0) {
        k_zero<<<grid_for(2 * nt, 256), 256, 0, st>>>(2 * nt, phi);
        P->launches++;
    }
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

int eval_once(tefmm_plan P, int64_t ns, const double *sx, const double *sy, const double *sz,
              const double *q, int64_t nt, const double *tx, const double *ty, const double *tz,
              double *phi, cudaStream_t st) {
    if (nt > 0 && !phi) return TEFMM_ERR_INVALID_ARG;
    if (ns > 0 && (!sx || !sy || !sz || !q)) return TEFMM_ERR_INVALID_ARG;
    if (nt > 0 && (!tx || !ty || !tz)) return TEFMM_ERR_INVALID_ARG;
    TRY(geometry(P, ns, sx, sy, sz, q, nt, tx, ty, tz, st));
    if (ns == 0 || nt == 0) return zero_output(nt, phi, st, P);
    TRY(upward_pass(P, st));
    TRY(tables(P, st));
    TRY(charge_phases(P, phi, st));
    P->geom_ready = true;
    return TEFMM_OK;
}
}  // namespace

extern "C" int tefmm_eval_host(tefmm_plan P, int64_t ns, const double *sx, const double *sy,
                               const double *sz, const double *q, int64_t nt, const double *tx,
                               const double *ty, const double *tz, double *phi, void *stream) {
    if (!P || ns < 0 || nt < 0) return TEFMM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    bool shared = (tx == sx && ty == sy && tz == sz && nt == ns);
    size_t nin = (size_t)ns * 5 + (shared ? 0 : (size_t)nt * 3);
    TRY(dbuf_ensure(P->h_in, nin * sizeof(double) + 64));
    TRY(dbuf_ensure(P->h_out, (size_t)nt * 2 * sizeof(double) + 64));
    double *d = dp<double>(P->h_in);
    double *dsx = d, *dsy = d + ns, *dsz = d + 2 * ns, *dq = d + 3 * ns;
    double *dtx = dsx, *dty = dsy, *dtz = dsz;
    if (ns > 0) {
        CUDA_TRY(cudaMemcpyAsync(dsx, sx, ns * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(dsy, sy, ns * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(dsz, sz, ns * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(dq, q, ns * 16, cudaMemcpyHostToDevice, st));
    }
    if (!shared && nt > 0) {
        dtx = d + 5 * ns;
        dty = dtx + nt;
        dtz = dty + nt;
        CUDA_TRY(cudaMemcpyAsync(dtx, tx, nt * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(dty, ty, nt * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(dtz, tz, nt * 8, cudaMemcpyHostToDevice, st));
    }
    TRY(tefmm_eval(P, ns, dsx, dsy, dsz, dq, nt, dtx, dty, dtz, dp<double>(P->h_out), stream));
    if (nt > 0) CUDA_TRY(cudaMemcpyAsync(phi, P->h_out.p, nt * 16, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return TEFMM_OK;
}

extern "C" int tefmm_get_stats(tefmm_plan P, tefmm_stats *o) {
    if (!P || !o) return TEFMM_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->n_nodes = P->n_nodes;
    o->n_levels = P->n_levels;
    o->n_v_pairs = P->n_v;
    o->n_p2p_pairs = P->n_p2p_pairs;
    o->n_tables = P->n_tables;
    o->n_images_total = (int)P->A.size();
    o->fit_max_resid = P->fit_max_resid;
    o->n_launches = P->launches;
    o->n_cross_tables = P->n_xtables;
    o->n_cross_fits = (int)P->xcache.size();
    o->n_cross_fits_last = P->n_xfits_last;
    o->ms_cross_fit = P->ms_xfit;
    o->fit_max_resid_cross = P->fit_max_resid_cross;
    if (P->n_nodes > 0 && cudaEventQuery(P->ev[6]) == cudaSuccess) {
        o->ms_tree = elapsed(P->ev[0], P->ev[1]);
        o->ms_upward = elapsed(P->ev[1], P->ev[2]);
        o->ms_tables = elapsed(P->ev[2], P->ev[3]);
        o->ms_m2l = elapsed(P->ev[3], P->ev[4]);
        o->ms_downward = elapsed(P->ev[4], P->ev[5]);
        o->ms_near = elapsed(P->ev[5], P->ev[6]);
        o->ms_cross_tables = elapsed(P->ev[7], P->ev[3]);
        o->ms_cross_m2l = elapsed(P->ev[8], P->ev[4]);
    }
    o->n_m2l_items = P->n_items - P->n_items_cross;
    o->n_m2l_items_cross = P->n_items_cross;
    o->n_m2l_kernel_launches = P->kev_used / 2;
    if (P->kev_used > 0 && cudaEventQuery(P->kev[P->kev_used - 1]) == cudaSuccess)
        for (int i = 0; i + 1 < P->kev_used; i += 2) o->ms_m2l_kernel += elapsed(P->kev[i], P->kev[i + 1]);
    for (int l = 0; l < 8; ++l) o->n_p2p_pairs_layer[l] = P->p2p_by_layer[l];
    o->n_fon_pairs = P->n_fon;
    o->n_alg2_tables = (int)P->a2.size();
    o->ms_alg2_build = P->ms_alg2_build;
    o->n_alg2_image_keys = P->n_alg2_image_keys;
    o->n_near_img_terms = P->n_near_img_terms;
    o->leaf_cap_used = P->leaf_cap_eff;
    o->ms_autotune = P->ms_autotune;
    o->n_tables_built = P->n_tables_built;
    return TEFMM_OK;
}

extern "C" int tefmm_export_tree(tefmm_plan P, int *n_nodes, int64_t *ns, int64_t *nt, int *layer,
                                 int *level, int *ix, int *iy, int *iz, int *parent, int *s0,
                                 int *s1, int *t0, int *t1, int *perm_s, int *perm_t) {
    if (!P) return TEFMM_ERR_INVALID_ARG;
    if (n_nodes) *n_nodes = P->n_nodes;
    if (ns) *ns = P->ns;
    if (nt) *nt = P->nt;
    const int nn = P->n_nodes;
    struct {
        int *h;
        DBuf *d;
    } m[] = {{layer, &P->n_layer}, {level, &P->n_level}, {ix, &P->n_ix}, {iy, &P->n_iy},
             {iz, &P->n_iz},       {parent, &P->n_parent}, {s0, &P->n_s0}, {s1, &P->n_s1},
             {t0, &P->n_t0},       {t1, &P->n_t1}};
    for (auto &e : m)
        if (e.h && nn > 0) CUDA_TRY(cudaMemcpy(e.h, e.d->p, nn * sizeof(int), cudaMemcpyDeviceToHost));
    if (perm_s && P->ns > 0) CUDA_TRY(cudaMemcpy(perm_s, P->perm_s.p, P->ns * 4, cudaMemcpyDeviceToHost));
    if (perm_t && P->nt > 0)
        CUDA_TRY(cudaMemcpy(perm_t, P->shared_pts ? P->perm_s.p : P->perm_t.p, P->nt * 4,
                            cudaMemcpyDeviceToHost));
    return TEFMM_OK;
}

extern "C" int tefmm_export_lists(tefmm_plan P, int64_t *n_v, int64_t *n_near, int *v_ptr,
                                  int *v_src, int *near_ptr, int *near_src) {
    if (!P) return TEFMM_ERR_INVALID_ARG;
    if (n_v) *n_v = P->n_v;
    if (n_near) *n_near = P->n_near;
    const int nn = P->n_nodes;
    if (v_ptr && nn > 0) CUDA_TRY(cudaMemcpy(v_ptr, P->v_ptr.p, (nn + 1) * 4, cudaMemcpyDeviceToHost));
    if (near_ptr && nn > 0)
        CUDA_TRY(cudaMemcpy(near_ptr, P->near_ptr.p, (nn + 1) * 4, cudaMemcpyDeviceToHost));
    if (v_src && P->n_v > 0) CUDA_TRY(cudaMemcpy(v_src, P->v_src.p, P->n_v * 4, cudaMemcpyDeviceToHost));
    if (near_src && P->n_near > 0)
        CUDA_TRY(cudaMemcpy(near_src, P->near_src.p, P->n_near * 4, cudaMemcpyDeviceToHost));
    return TEFMM_OK;
}

extern "C" int tefmm_export_expansions(tefmm_plan P, double *alpha, double *beta) {
    if (!P) return TEFMM_ERR_INVALID_ARG;
    size_t n = (size_t)P->n_nodes * P->np * sizeof(cplx);
    if (alpha && n) CUDA_TRY(cudaMemcpy(alpha, P->alpha.p, n, cudaMemcpyDeviceToHost));
    if (beta && n) CUDA_TRY(cudaMemcpy(beta, P->beta.p, n, cudaMemcpyDeviceToHost));
    return TEFMM_OK;
}

int kernel_event(tefmm_plan_s *P, cudaStream_t st) {
    if (P->kev_used == (int)P->kev.size()) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        P->kev.push_back(e);
    }
    CUDA_TRY(cudaEventRecord(P->kev[P->kev_used++], st));
    return TEFMM_OK;
}

extern "C" int tefmm_plan_status(tefmm_plan P, void *stream) {
    if (!P) return TEFMM_ERR_INVALID_ARG;
    if (!P->flags.p) return TEFMM_OK;
    return check_flags(P, (cudaStream_t)stream);
}

namespace {
// a bounded wait on an mbarrier that nothing completes: the wait runs out after
// `ms` milliseconds of device time (%globaltimer) and raises FLAG_TIMEOUT
__global__ void k_wait_probe(int *flags, unsigned long long ms) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;");
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     "selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(b) : "memory");
        if (ok) return;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > ms * 1000000ULL) break;
    }
    atomicOr(flags, FLAG_TIMEOUT);
}
}  // namespace

extern "C" int tefmm_debug_wait_probe(tefmm_plan P, int ms, void *stream) {
    if (!P || ms < 1 || ms > 2000) return TEFMM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(dbuf_ensure(P->flags, 64));
    CUDA_TRY(cudaMemsetAsync(P->flags.p, 0, 64, st));
    k_wait_probe<<<1, 32, 0, st>>>(dp<int>(P->flags), (unsigned long long)ms);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return check_flags(P, st);
}
