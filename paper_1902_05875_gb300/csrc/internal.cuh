// Internal declarations shared by the translation units of libtefmm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <stdio.h>

#include <map>
#include <vector>

#include "tefmm.h"

#define TEFMM_NBITS 20          // bits per axis of the Morton code (levels 0..20)
#define TEFMM_MAX_LAYERS 16
#define TEFMM_MAX_TERMS 4       // same-layer reaction terms per layer
#define TEFMM_MAX_IMG 32        // images per term

// device-side error flags (bit mask, OR-ed by kernels)
#define FLAG_ON_INTERFACE 1
#define FLAG_OUT_OF_DOMAIN 2
#define FLAG_LIST_OVERFLOW 4
#define FLAG_CROSS_LAYER 8
#define FLAG_CHECK 16
#define FLAG_TIMEOUT 32         // a bounded device wait ran out

// ---------------------------------------------------------------- complex
struct cplx {
    double x, y;
};

__host__ __device__ __forceinline__ cplx mkc(double x, double y) { return cplx{x, y}; }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cplx{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return cplx{a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return cplx{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return cplx{a.x * s, a.y * s}; }
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return cplx{(a.x + a.y * r) / den, (a.y - a.x * r) / den};
    } else {
        double r = b.x / b.y, den = b.x * r + b.y;
        return cplx{(a.x * r + a.y) / den, (a.y * r - a.x) / den};
    }
}
// principal square root (Re >= 0)
__host__ __device__ __forceinline__ cplx csqrt_p(cplx z) {
    double r = hypot(z.x, z.y);
    if (r == 0.0) return cplx{0.0, 0.0};
    if (z.x >= 0.0) {
        double t = sqrt(0.5 * (r + z.x));
        return cplx{t, z.y / (2.0 * t)};
    } else {
        double t = sqrt(0.5 * (r - z.x));
        return cplx{fabs(z.y) / (2.0 * t), copysign(t, z.y)};
    }
}
__host__ __device__ __forceinline__ cplx cexp_(cplx z) {
    double e = exp(z.x), s, c;
#ifdef __CUDA_ARCH__
    sincos(z.y, &s, &c);
#else
    s = sin(z.y);
    c = cos(z.y);
#endif
    return cplx{e * c, e * s};
}
// h0(kR) = e^{ikR}/(ikR)
__host__ __device__ __forceinline__ cplx h0c(cplx kR) {
    cplx ikr = cplx{-kR.y, kR.x};
    return cdiv(cexp_(ikr), ikr);
}

// ------------------------------------------------------------ multi-indices
// graded order: n = 0..P; k1 = n..0; k2 = n-k1..0; k3 = n-k1-k2
__host__ __device__ __forceinline__ int ncoef(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }
__host__ __device__ __forceinline__ int midx(int k1, int k2, int k3) {
    int n = k1 + k2 + k3;
    int a = n - k1;
    return n * (n + 1) * (n + 2) / 6 + a * (a + 1) / 2 + (a - k2);
}

// ------------------------------------------------------------ device buffers
struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
};
int dbuf_ensure(DBuf &b, size_t bytes);   // grow (contents not preserved)
// test hooks (tefmm_debug_inject): true when the next allocation / fit is to fail
bool inject_alloc_failure();
bool inject_fit_failure();
void dbuf_free(DBuf &b);

template <class T>
static inline T *dp(DBuf &b) { return reinterpret_cast<T *>(b.p); }

// ---------------------------------------------------------------- images
struct TermDesc {          // one same-layer reaction term of one layer
    int layer, tag;        // tag: 0 uu, 1 dd, 2 ud, 3 du
    int first, count;      // range in the image arrays
    double sz, szp, c, zmin;
};

struct Alg2Table {         // one Algorithm 2 table (host record of a device buffer)
    int layer = 0, tag = 0, P2 = 0, n = 0, ne = 0;
    double rho_max = 0, zlo = 0, zhi = 0;
    cplx *T = nullptr;     // device [n][n][ne]
};

struct DevTerm {           // POD copy for kernels
    double sz, szp, c, zmin;
    int first, count, layer, tag;
};

// cross-layer fit: (target layer, source layer, direction 0 up / 1 down,
// level, source z-index, k3') -> images in the plan's cross-layer pool
struct CrossFitKey {
    int lt, ls, dir, level, izs, k3p;
    bool operator<(const CrossFitKey &o) const {
        if (lt != o.lt) return lt < o.lt;
        if (ls != o.ls) return ls < o.ls;
        if (dir != o.dir) return dir < o.dir;
        if (level != o.level) return level < o.level;
        if (izs != o.izs) return izs < o.izs;
        return k3p < o.k3p;
    }
};
struct CrossFitVal {
    int first, count;
};

// ---------------------------------------------------------------- plan
struct tefmm_plan_s {
    int nL = 0;
    double d[TEFMM_MAX_LAYERS] = {0};
    cplx k[TEFMM_MAX_LAYERS] = {};
    tefmm_options opt{};
    int p = 0, np = 0, np2 = 0;
    int device = 0;
    int leaf_cap_eff = 64;        // leaf cap in use (0 until the autotuner has chosen one)
    double HX = INFINITY;         // box size above which stacked cross-layer boxes are paired, not translated
    double kmax = 0.0;            // max over layers of |k_l| (wavenumber admissibility)
    double ms_autotune = 0;       // time of the autotuner's trial evaluations

    // images (host mirror + device copy)
    std::vector<TermDesc> terms;
    std::vector<cplx> A, Z;
    int layer_term_first[TEFMM_MAX_LAYERS] = {0};
    int layer_term_count[TEFMM_MAX_LAYERS] = {0};
    DBuf d_terms, d_A, d_Z, d_k;
    double fit_max_resid = 0.0;

    // operator tables (device)
    DBuf d_mi;        // int [np2*3] multi-indices up to order 2p
    DBuf d_m2l_g;     // uint16 [np*np]  index of k+k' (layout [k'][k])
    DBuf d_m2l_cB;    // double [np*np]  C(k+k',k) (-1)^{k1'+k2'} (-1)^{k3'}  ([k'][k])
    DBuf d_m2l_cA;    // double [np*np]  C(k+k',k) (-1)^{k1'+k2'}            ([k'][k])

    // workspace of the last evaluation
    int64_t ns = 0, nt = 0, nitems = 0;
    bool shared_pts = false;
    bool geom_ready = false;   // tree, lists and tables match the last points (eval or set_points)
    DBuf keys_in, keys_out, vals_in, vals_out, sort_tmp, scan_tmp;
    DBuf item_node, item_flag, item_scan, cnt_s, cnt_t;
    DBuf sx, sy, sz, sq, tx, ty, tz, perm_s, perm_t;
    DBuf n_layer, n_level, n_ix, n_iy, n_iz, n_parent, n_cfirst, n_nchild, n_s0, n_s1, n_t0,
        n_t1, n_i0, n_i1, n_split, n_key;
    DBuf bbox, flags, counters;
    int n_nodes = 0, n_levels = 0;
    std::vector<int> level_off;   // node range per level: [level_off[l], level_off[l+1])
    double lo[3] = {0, 0, 0}, side = 1.0;

    // lists
    DBuf C_list, C_cnt, D_list, D_cnt, X_list, X_cnt, V_tmp, V_cnt;
    DBuf v_ptr, v_src, near_ptr, near_src, near_tmp, near_cnt;
    int64_t n_v = 0, n_near = 0, n_p2p_pairs = 0;
    int64_t n_fon = 0;            // far-of-near pairs (same-level adjacent leaves), after the V pairs
    DBuf fon_cnt, fon_ptr, fon_key, fon_key_sorted;
    DBuf near_fl;   // per near-list entry: far-of-near level l* of its anchor, or -1
    // near-field work items (one CTA each): target leaf, chunk index, chunks of that leaf
    DBuf nitem_cnt, nitem_pos, nitem_node, nitem_part, nitem_np;
    int n_near_items = 0;
    int64_t n_near_img_terms = 0;   // pair x image-term evaluations of the near field
    int cap_D = 64, cap_X = 0;

    // expansions
    DBuf alpha, beta;

    // M2L grouping and tables
    DBuf keyslot_flag, keyslot_table, pair_t, pair_s, pair_slot, pair_slot_sorted, pair_idx,
        pair_idx_sorted, chunk_key, chunk_start, chunk_cnt, tables, table_slot, seg_tmp;
    DBuf table_rep;           // per table: representative * 8 + symmetry code
    int n_tables = 0;
    int n_tables_built = 0;   // tables computed by the recurrence (the rest by symmetry)
    int64_t n_chunks = 0;
    std::vector<int> chunk_key_host;   // mixed form: chunk -> table, copied when the geometry is built
    int chunk_pairs = 16;     // pairs per M2L work chunk (FP64 SIMT: 16, tensor cores: 512)

    // Algorithm 2: one Sommerfeld-integral table per (layer, same-layer term),
    // [n][n][entries] complex, over the ranges of the last geometry's keys
    std::vector<Alg2Table> a2;
    double ms_alg2_build = 0.0;
    int n_alg2_image_keys = 0;   // (key, term) lookups of the last geometry left to the images

    // cross-layer components: fitted images (cached per root-cube geometry),
    // per-table image ranges and tables
    std::map<CrossFitKey, CrossFitVal> xcache;
    std::vector<cplx> xA, xZ;
    double xgeo_lo = 0.0, xgeo_side = -1.0;
    double fit_max_resid_cross = 0.0;
    DBuf d_xA, d_xZ, d_xrange, d_tslot, xtables, d_xG, d_xcf, d_xexp, d_xoff, tc_xcf;
    DBuf xalpha, xbeta;   // moments / locals about the cross-layer centres
    DBuf tc_xah, tc_xal, tc_xbt, tc_xgs, tc_xcf32, tc_xW;   // tensor-core cross-layer M2L
    int NX = 0, n_xtables = 0, n_xfits_last = 0;
    int x_first_table = 0;        // cross-layer tables are [x_first_table, n_tables)
    int64_t x_first_chunk = 0;    // cross-layer chunks are [x_first_chunk, n_chunks)
    size_t x_uploaded = 0;        // images of the pool on the device
    double ms_xfit = 0;           // host time of the cross-layer fits of the last eval

    // tensor-core M2L buffers (mixed form)
    DBuf tc_ah, tc_al, tc_bt, tc_cfA, tc_cfB, tc_W;   // tc_W: precomputed W^T blocks
    int tc_cf_np = 0;

    // host staging for tefmm_eval_host
    DBuf h_in, h_out;

    // timing
    cudaEvent_t ev[12] = {};
    std::vector<cudaEvent_t> kev;   // pairs of events around the tensor-core M2L launches
    int kev_used = 0;               // events recorded by the last evaluation
    int64_t n_items = 0, n_items_cross = 0;   // M2L items (one per translation matrix applied)
    int64_t p2p_by_layer[8] = {};             // near-field particle pairs per target layer
    double ms_tree = 0, ms_upward = 0, ms_tables = 0, ms_m2l = 0, ms_downward = 0, ms_near = 0;
    int64_t launches = 0;    // kernels of this library launched so far
};

// ---------------------------------------------------------------- helpers
#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess) {                                                          \
            fprintf(stderr, "tefmm: %s failed at %s:%d: %s\n", #expr, __FILE__, __LINE__,  \
                    cudaGetErrorString(_e));                                              \
            return (_e == cudaErrorMemoryAllocation) ? TEFMM_ERR_OOM : TEFMM_ERR_CUDA;    \
        }                                                                                 \
    } while (0)

#define TRY(expr)                         \
    do {                                  \
        int _r = (expr);                  \
        if (_r != TEFMM_OK) return _r;    \
    } while (0)

// Raise a kernel's dynamic shared-memory limit to the most the device allows
// beside the kernel's static shared memory.  Every call sets the same value,
// so plans evaluated concurrently from several host threads (batched
// evaluation) cannot lower the limit under one another's launches.
template <class F>
static inline int smem_optin(F *func) {
    int dev = 0, mx = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, (const void *)func) != cudaSuccess ||
        cudaFuncSetAttribute((const void *)func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             mx - (int)fa.sharedSizeBytes) != cudaSuccess)
        return TEFMM_ERR_CUDA;
    return TEFMM_OK;
}

static inline int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 2147483647LL) g = 2147483647LL;
    return (int)g;
}

// ------------------------------------------------------------ entry points
// tree.cu
int tree_build(tefmm_plan_s *P, const double *sx, const double *sy, const double *sz,
               const double *q, const double *tx, const double *ty, const double *tz,
               cudaStream_t st);
int lists_build(tefmm_plan_s *P, cudaStream_t st);
int check_flags(tefmm_plan_s *P, cudaStream_t st);
int kernel_event(tefmm_plan_s *P, cudaStream_t st);   // record the next timing event
// ops.cu
int upward_pass(tefmm_plan_s *P, cudaStream_t st);
int m2l_prepare(tefmm_plan_s *P, cudaStream_t st);
int m2l_tables(tefmm_plan_s *P, cudaStream_t st);
int m2l_apply(tefmm_plan_s *P, cudaStream_t st);
// m2l_tc.cu
int m2l_apply_tc(tefmm_plan_s *P, cudaStream_t st);
int m2l_apply_tc_cross(tefmm_plan_s *P, cudaStream_t st, const cplx *alpha_x, cplx *beta_x,
                       const unsigned short *xgs, const float *xcf);
size_t m2l_tc_smem(int np, int MT, int tab_entries);
void m2l_tc_geometry(int np, int MT, int *Kpad, int *Ncta, int *nsplit);
#define NEAR_CHUNK 4096   // near sources per near-field work item
#define TC_MT 1         // tiles of 128 pairs per pass, same-layer keys
#define TC_MT_CROSS 1   // cross-layer keys
int downward_pass(tefmm_plan_s *P, cudaStream_t st);
int near_field(tefmm_plan_s *P, double *phi, cudaStream_t st);
// near32.cu
int near_field_fp32(tefmm_plan_s *P, double *phi, cudaStream_t st);
// plan.cu
int plan_upload_images(tefmm_plan_s *P);
int plan_build_operator_tables(tefmm_plan_s *P);
// fit.cu
int plan_fit_images(tefmm_plan_s *P, cudaStream_t st);
int fit_cross_jobs(tefmm_plan_s *P, const std::vector<CrossFitKey> &keys, cudaStream_t st);
// cross.cu
double cross_wmin(const tefmm_plan_s *P, int lt, int dir);
int tables_expand(tefmm_plan_s *P, int first, int ntab, int nslices, cplx *tabs, int64_t stride,
                  cudaStream_t st);
int cross_prepare(tefmm_plan_s *P, cudaStream_t st);
int cross_tables(tefmm_plan_s *P, cudaStream_t st);
int cross_apply(tefmm_plan_s *P, cudaStream_t st);
void cross_release(tefmm_plan_s *P);
// sortscan.cu: int32 prefix sums and the stable radix sort of 64-bit keys
int dev_scan_i32(tefmm_plan_s *P, const int *in, int *out, int64_t n, bool inclusive, cudaStream_t st);
int dev_sort_u64(tefmm_plan_s *P, const uint64_t *kin, uint64_t *kout, const int *vin, int *vout, int64_t n,
                 cudaStream_t st);
// alg2.cu
int alg2_prepare(tefmm_plan_s *P, cudaStream_t st);
void alg2_release(tefmm_plan_s *P);
int alg2_entries(int P2);
