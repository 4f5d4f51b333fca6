/*
 * tefmm.h -- C ABI of the GB300 Taylor-expansion FMM for the 3-D Helmholtz
 * equation in layered media (Wang, Zhang, Cai: arXiv 1902.05875).
 *
 * The library computes the matrix-vector product of the paper's Sec. 3.2,
 * eq. ``totalinteraction``:
 *
 *   Phi_l(r_i) = sum_{j in layer l, r_j != r_i} q_j h0(k_l |r_i - r_j|)
 *              + sum_{l'} sum_{j in layer l'} q_j (u^up_{l l'} + u^down_{l l'})(r_i, r_j),
 *
 * with h0(z) = e^{iz}/(iz) and the factor i k_l / (4 pi) omitted (Sec. 3.1),
 * by the TE-FMM of Algorithm 1 applied to every component of the heterogeneous
 * loop that follows it (Sec. 3.3).  The reaction components are represented by
 * discrete complex images (Sec. 3.3, eq. ``closedformgreen``) fitted at plan
 * time.  Everything below these calls runs in this library's own CUDA kernels.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Medium: n_layers = L+1 layers numbered 0 (top) .. L (bottom); interfaces
 *   z = d_0 > d_1 > ... > d_{L-1}; layer l is d_l < z < d_{l-1} (Sec. 2.1).
 * - Complex numbers are interleaved (re, im) doubles.
 * - Return value: TEFMM_OK (0) or a negative TEFMM_ERR_* code; nothing is
 *   modified on an argument error.  tefmm_status_string() names the code.
 * - Streams: ``stream`` is a cudaStream_t (NULL = legacy default stream).
 *   Work is queued on it; calls that build trees read sizes back and so
 *   synchronise the stream internally.
 * - Memory: pointers named d_* are caller-owned DEVICE memory of the current
 *   CUDA device; h_* are caller-owned HOST memory.  The library never frees
 *   or retains caller memory.  A plan owns its tables and scratch, released by
 *   tefmm_plan_destroy().
 * - Threading: a plan may be used by one host thread at a time.
 */
#ifndef TEFMM_H
#define TEFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TEFMM_OK 0
#define TEFMM_ERR_INVALID_ARG (-1)        /* bad argument (sizes, ordering, NULL)        */
#define TEFMM_ERR_POINT_ON_INTERFACE (-2) /* some z equals an interface depth exactly    */
#define TEFMM_ERR_OUT_OF_DOMAIN (-3)      /* a point lies outside its layer's slab       */
#define TEFMM_ERR_OOM (-4)                /* device allocation failed                    */
#define TEFMM_ERR_CUDA (-5)               /* a CUDA runtime call failed                  */
#define TEFMM_ERR_FIT_FAILED (-6)         /* DCIM fit produced no usable images          */
#define TEFMM_ERR_LIST_OVERFLOW (-7)      /* an interaction list exceeded its capacity   */
#define TEFMM_ERR_NOT_IMPLEMENTED (-8)    /* configuration not supported by this build   */
#define TEFMM_ERR_DEVICE_CHECK (-9)       /* a device-side consistency check failed      */
#define TEFMM_ERR_TIMEOUT (-10)           /* a bounded device wait ran out (the kernel
                                             skipped its output and released its TMEM)  */

#define TEFMM_FP64 0   /* every step in FP64                                          */
#define TEFMM_MIXED 1  /* M2L on tensor cores and P2P in FP32; FP64 tables and sums   */

#define TEFMM_ALG_RECURRENCE 1 /* Algorithm 1: DCIM images + derivative recurrence (Sec. 3.3) */
#define TEFMM_ALG_TABLES 2     /* Algorithm 2/3 (Sec. 4.2): same-layer reaction derivatives from
                                  interpolated tables of Sommerfeld integrals               */

#define TEFMM_SPLIT_TF32X3 0   /* mixed form: FP32 operands split hi + lo in TF32, three products
                                  (hi*hi + hi*lo + lo*hi) with FP32 accumulation                */

typedef struct tefmm_plan_s *tefmm_plan;

typedef struct {
    int p;                 /* Taylor order (|k| <= p), 1..12                          */
    int leaf_cap;          /* split a box while max(#sources, #targets) > leaf_cap;
                              0: autotuned on the first evaluation (the fastest of
                              16, 32, 64, 128, 256 by CUDA-event timing)              */
    int max_level;         /* deepest octree level, 1..20                             */
    int precision;         /* TEFMM_FP64 or TEFMM_MIXED                               */
    int n_images;          /* DCIM images per fitted term (<= 32; <= 24 per level)    */
    int n_samples;         /* DCIM samples per level, 8..127 (Sec. 3.3 uses 101)     */
    double T1;             /* length of the first-level path (Sec. 3.3 uses 10)       */
    double T0;             /* second-level path; <= 0: sqrt(((max Re k + 0.8)/Re k_l)^2 - 1) */
    double zext[2 * 16];   /* per layer (zlo, zhi): z-range of the particles, used for
                              the DCIM shift zeta_min (Sec. 3.3, z_min); a point outside
                              its layer's range is TEFMM_ERR_OUT_OF_DOMAIN             */
    double kh_max;         /* wavenumber admissibility: on octree levels whose box size h
                              has max_l |k_l| h > kh_max, two split boxes are not
                              translated (M2L) but their children are paired, so every
                              translation spans k h <= kh_max (the truncated Taylor
                              series of e^{ikR}/R of Sec. 3.1 converges slowly for
                              large k h); <= 0 turns the rule off.  Default 3.5.  The
                              first translating level may pair boxes at most 15 apart:
                              a medium that needs more coarse levels returns
                              TEFMM_ERR_NOT_IMPLEMENTED from the evaluation.          */
    int algorithm;         /* TEFMM_ALG_RECURRENCE (default): every M2L derivative from
                              the DCIM images by the recurrence of Sec. 3.3.
                              TEFMM_ALG_TABLES (Sec. 4.2, eqs. ``sysdifferential`` and
                              ``symmetricdetable``): the same-layer reaction derivatives
                              D^g u_tau / g! from tables of the Sommerfeld integrals
                              T_{m,nu,n}(rho, zeta) = (1/k) int k_rho^{m+1} J_nu(k_rho rho)
                              (i k_z)^n e^{i k_z zeta} s_tau / k_z dk_rho  (m + n <= 2p,
                              nu = m, m-2, ..), one table per same-layer term tau, on a
                              uniform table_n x table_n grid over rho in [0, rho_max] and
                              the term's image distance zeta in [zeta_lo, zeta_hi], the
                              ranges of the layer's M2L pairs (built on the device by
                              contour quadrature when the geometry is set, rebuilt when a
                              new geometry leaves the ranges); FP64 degree-7 Lagrange
                              interpolation in each direction, assembled into Cartesian
                              derivatives through D+- = d_x +- i d_y.  The free-space part,
                              cross-layer components, the near field and the far-of-near
                              translations (far images only) keep Algorithm 1's images.
                              The integral converges for zeta > 0
                              only: a key whose image distance lies below the term's
                              smallest one over the layer's particle slab (zext; the
                              DCIM shift zeta_min), i.e. box centres of a coarse level
                              beyond the slab, keeps the images for that term and stays
                              out of the grid ranges.                                  */
    int split;             /* tensor-core split of the mixed form: TEFMM_SPLIT_TF32X3
                              (the only one built; others TEFMM_ERR_NOT_IMPLEMENTED)  */
    int far_of_near;       /* 1 (default): for a near-field pair of boxes (target t,
                              source s) let l* be the coarser of their levels and T*, S*
                              the level-l* boxes holding them; when T* and S* are
                              adjacent, the DCIM images far from both (-Re Z_j >=
                              10^(10/(p+1)) sqrt(3) h_{l*}) are translated by one M2L
                              from S* to T* (through the tensor cores in the mixed
                              form) instead of summed pair by pair; the free-space term
                              and the near images stay in P2P.  0: every image in P2P. */
    int scale_output;      /* 0 (default): potentials in the paper's normalisation
                              (Sec. 3.1: free term h0(k|r - r'|), factor i k_l/(4 pi)
                              omitted); 1: every potential multiplied by i k_l/(4 pi)
                              of its target's layer l                                  */
    int table_n;           /* TEFMM_ALG_TABLES: grid points per direction, 8..512;
                              0 (default) = 64                                         */
} tefmm_options;

typedef struct {
    int n_nodes;           /* octree nodes, all layers                                */
    int n_levels;          /* deepest level + 1                                       */
    int64_t n_v_pairs;     /* M2L (V-list) pairs, all components                      */
    int64_t n_p2p_pairs;   /* near-field (target, source) particle pairs              */
    int n_tables;          /* derivative tables built (distinct M2L keys)             */
    int n_images_total;    /* DCIM images held by the plan                            */
    double ms_tree;        /* last eval: keys, sort, tree, lists                      */
    double ms_upward;      /* P2M + M2M                                               */
    double ms_tables;      /* derivative tables                                       */
    double ms_m2l;         /* M2L contractions                                        */
    double ms_downward;    /* L2L                                                     */
    double ms_near;        /* L2P + P2P                                               */
    double fit_max_resid;  /* worst DCIM fit residual on the samples (relative)       */
    int64_t n_launches;    /* kernels of this library launched by this plan so far    */
    int n_cross_tables;    /* last eval: cross-layer derivative tables (l != l')      */
    int n_cross_fits;      /* cross-layer DCIM fits cached by the plan                */
    int n_cross_fits_last; /* cross-layer fits computed by the last eval (cache misses) */
    double ms_cross_fit;   /* host time of those fits                                 */
    double fit_max_resid_cross; /* worst cross-layer fit residual (relative)          */
    double ms_cross_tables; /* part of ms_tables spent on cross-layer tables          */
    double ms_cross_m2l;   /* part of ms_m2l spent on cross-layer translations        */
    int leaf_cap_used;     /* leaf cap of the last evaluation (the autotuner's choice
                              when the plan was made with leaf_cap = 0)               */
    double ms_autotune;    /* time of the autotuner's trial evaluations               */
    int n_tables_built;    /* last eval: tables computed by the recurrence; the other
                              n_tables - n_tables_built are copied from one of these by
                              the reflection x -> -x, y -> -y and swap x <-> y symmetry */
    int64_t n_m2l_items;   /* last eval: translation matrices applied, same-layer (up to
                              two per V pair: the B and the A table)                  */
    int64_t n_m2l_items_cross; /* ... cross-layer (one per cross-layer V pair)        */
    double ms_m2l_kernel;  /* mixed form: device time of the tensor-core contraction
                              kernels alone (CUDA events around each launch)          */
    int n_m2l_kernel_launches; /* ... and their number                               */
    int64_t n_p2p_pairs_layer[8]; /* near-field particle pairs by target layer        */
    int64_t n_fon_pairs;   /* last eval: leaf pairs whose far images went through M2L */
    int n_alg2_tables;     /* TEFMM_ALG_TABLES: Sommerfeld-integral tables held        */
    double ms_alg2_build;  /* ... host time of the last (re)build of those tables      */
    int n_alg2_image_keys; /* ... (key, term) derivatives of the last geometry taken from
                              the images instead (image distance below the slab's)   */
    int64_t n_near_img_terms; /* last geometry: near-field (particle pair, image term)
                              evaluations, after the far-of-near reading              */
} tefmm_stats;

/* Fill ``opt`` with defaults: p = 6, leaf_cap = 64, max_level = 20, FP64,
 * 8 images, 101 samples, T1 = 10, T0 = formula, zext = whole layers,
 * kh_max = 3.5, far_of_near = 1, algorithm 1, TF32x3 split, unscaled output. */
int tefmm_default_options(tefmm_options *opt);

/* Create a plan for a layered medium (Sec. 2.1) and fit its DCIM images
 * (Sec. 3.3, Steps 1-2) on the device.
 *   n_layers        1..8;
 *   interfaces      host array [n_layers-1], strictly decreasing;
 *   k_re, k_im      host arrays [n_layers], k_im >= 0;
 *   opt             host struct (NULL = defaults);
 *   stream          cudaStream_t used for the fits;
 *   out             receives the plan.
 * Errors: INVALID_ARG, OOM, CUDA, FIT_FAILED, NOT_IMPLEMENTED (algorithm or
 * split not built). */
int tefmm_plan_create(int n_layers, const double *interfaces, const double *k_re,
                      const double *k_im, const tefmm_options *opt, void *stream,
                      tefmm_plan *out);

/* Release a plan and everything it owns.  NULL is accepted. */
int tefmm_plan_destroy(tefmm_plan plan);

/* The matrix-vector product (Sec. 3.2, eq. ``totalinteraction``; Algorithm 1
 * for every component).  Builds the octrees and lists for the given points,
 * then runs the upward pass, the M2L translations, the downward pass, L2P and
 * the near field.
 *   ns, d_sx/d_sy/d_sz  source coordinates (device, ns doubles each);
 *   d_q                 source charges (device, 2*ns doubles, interleaved);
 *   nt, d_tx/d_ty/d_tz  target coordinates (device); passing the source
 *                       pointers with nt == ns selects the "targets are the
 *                       sources" case (self pairs skipped in free space only);
 *   d_phi               output potentials (device, 2*nt doubles), overwritten.
 * Errors: INVALID_ARG, POINT_ON_INTERFACE, OUT_OF_DOMAIN, OOM, CUDA,
 *         LIST_OVERFLOW, DEVICE_CHECK (an M2L pair offset outside the key
 *         range), TIMEOUT (a bounded device wait of the tensor-core M2L ran
 *         out), NOT_IMPLEMENTED (wavenumber rule needing offsets above 15).  The call returns
 *         when the result is complete on the stream, with any device-detected
 *         error of this evaluation.  ns == 0 or nt == 0 writes zeros. */
int tefmm_eval(tefmm_plan plan, int64_t ns, const double *d_sx, const double *d_sy,
               const double *d_sz, const double *d_q, int64_t nt, const double *d_tx,
               const double *d_ty, const double *d_tz, double *d_phi, void *stream);

/* Geometry once, charges many times: the repeated matrix-vector products of an
 * iterative solver (Sec. 1 motivates the FMM as the matvec of such solvers).
 * tefmm_set_points builds, for the given points, everything of tefmm_eval
 * that does not depend on the charges: trees, lists, M2L keys, cross-layer
 * fits and derivative tables (arguments as tefmm_eval without d_q and d_phi).
 * tefmm_apply then evaluates the potentials of charges d_q (device, 2*ns
 * doubles, interleaved, in the order of the set_points sources) into d_phi
 * (device, 2*nt doubles, target order), running only P2M, M2M, M2L, L2L, L2P
 * and the near field.  The points are not copied from the caller again; the
 * plan keeps its own sorted copy.  tefmm_eval also leaves the plan ready for
 * tefmm_apply on its points; tefmm_plan_set_images invalidates it.
 * Errors: as tefmm_eval; tefmm_apply returns INVALID_ARG when the plan has no
 * points.  A plan made with leaf_cap = 0 uses the cap its autotuner chose in
 * an earlier tefmm_eval, else 64.  No counterpart in the paper's code. */
int tefmm_set_points(tefmm_plan plan, int64_t ns, const double *d_sx, const double *d_sy,
                     const double *d_sz, int64_t nt, const double *d_tx, const double *d_ty,
                     const double *d_tz, void *stream);
int tefmm_apply(tefmm_plan plan, const double *d_q, double *d_phi, void *stream);

/* One instance of a batch: device arrays as for tefmm_eval; tx == NULL means
 * the targets are the sources (then nt, ty, tz are ignored). */
typedef struct {
    int64_t ns;
    const double *sx, *sy, *sz, *q;
    int64_t nt;
    const double *tx, *ty, *tz;
    double *phi;
} tefmm_batch_item;

/* Batched matrix-vector products of n independent instances (the batched
 * workload of many small layered media; the paper evaluates one medium at a
 * time).  plans[i] holds instance i's medium and options (distinct plans; a
 * plan may appear once), items[i] its particles and output.  The instances
 * run concurrently on n_workers (<= 0: 8) internal streams, each driven by a
 * host thread; the work is ordered after the caller's stream at entry and the
 * caller's stream waits for all of it at exit.  status (optional, host int[n])
 * receives each instance's result.  Returns the first error of any instance,
 * INVALID_ARG for bad arguments, CUDA for stream/event failures. */
int tefmm_eval_batched(int n, tefmm_plan *plans, const tefmm_batch_item *items, int n_workers,
                       void *stream, int *status);

/* Device-detected errors of the plan's work so far (reads the plan's device
 * flags, synchronising the stream): the status tefmm_eval / tefmm_apply would
 * have returned.  Work captured into a CUDA graph cannot report them when it
 * runs; read them with this call after the graph has run.  Flags accumulate
 * from the plan's last tefmm_eval / tefmm_set_points on.  No counterpart in
 * the paper. */
int tefmm_plan_status(tefmm_plan plan, void *stream);

/* Batch graph: the charge phases of n plans (tefmm_apply of plans[i] with
 * device charges q[i] and potentials phi[i], each plan on the points of its
 * last tefmm_set_points or tefmm_eval) captured once into one CUDA graph, each
 * plan a parallel branch, and replayed with one cudaGraphLaunch per batch:
 * the batched workload of many independent media run as a single launch.
 * create runs one tefmm_apply per plan on ``stream`` first (buffers are sized
 * outside the capture), then captures on ``stream`` (relaxed mode).  The
 * pointers q[i] and phi[i] are baked into the graph: write new charges into
 * the same buffers before each launch.  Plans must be distinct and must not be
 * used by other calls while the graph exists (tefmm_set_points or tefmm_eval
 * on one of them invalidates the graph).  Errors found on the device are read
 * with tefmm_plan_status.  No counterpart in the paper.
 * Errors: INVALID_ARG (n <= 0, NULL, a plan without points, a repeated plan),
 * CUDA, and the errors of tefmm_apply. */
typedef struct tefmm_batch_graph_s *tefmm_batch_graph;
int tefmm_batch_graph_create(int n, tefmm_plan *plans, const double *const *q, double *const *phi,
                             void *stream, tefmm_batch_graph *out);
int tefmm_batch_graph_launch(tefmm_batch_graph graph, void *stream);
int tefmm_batch_graph_destroy(tefmm_batch_graph graph);

/* Same as tefmm_eval with HOST arrays: copies the inputs to plan-owned device
 * buffers, evaluates, copies Phi back, and synchronises the stream. */
int tefmm_eval_host(tefmm_plan plan, int64_t ns, const double *h_sx, const double *h_sy,
                    const double *h_sz, const double *h_q, int64_t nt, const double *h_tx,
                    const double *h_ty, const double *h_tz, double *h_phi, void *stream);

/* Statistics and phase timings of the last evaluation (host struct). */
int tefmm_get_stats(tefmm_plan plan, tefmm_stats *out);

/* Human-readable name of a status code (static string). */
const char *tefmm_status_string(int status);

/* ---- inspection hooks (used by the parity tests) ------------------------
 * Images are described per (layer, term): term tags 0 = up-up, 1 = down-down,
 * 2 = up-down, 3 = down-up.  A same-layer reaction term is written with a real
 * image distance zeta = sz*z + szp*z' + c (> 0 inside the layer) and contributes
 * sum_j A_j h0(k_l sqrt(rho^2 + (zeta - zeta_min - Z_j)^2)) (Sec. 3.3, Step 3,
 * eq. ``closedformgreen`` with the density's reflection exponentials folded
 * into zeta).  For each term: sz, szp, c, zeta_min and its images (A_j, Z_j).
 */

/* Number of (layer, term) entries and of images held by the plan. */
int tefmm_plan_image_counts(tefmm_plan plan, int *n_terms, int *n_images);

/* Copy the plan's images to host arrays:
 *   term_layer[n_terms], term_tag[n_terms], term_first[n_terms], term_count[n_terms],
 *   term_geom[4*n_terms] = (sz, szp, c, zeta_min), A[2*n_images], Z[2*n_images]. */
int tefmm_plan_get_images(tefmm_plan plan, int *term_layer, int *term_tag, int *term_first,
                          int *term_count, double *term_geom, double *A, double *Z);

/* Replace the images of every term (same term layout as get_images: same
 * n_terms, per-term counts may change, total <= 32 * n_terms). */
int tefmm_plan_set_images(tefmm_plan plan, const int *term_count, const double *A,
                          const double *Z);

/* Tree of the last evaluation.  With all pointers NULL only the counts are
 * returned.  Node arrays (host, n_nodes each): layer, level, ix, iy, iz,
 * parent, s0, s1, t0, t1 (ranges in the sorted source / target order);
 * perm_s[ns], perm_t[nt]: sorted position -> input index. */
int tefmm_export_tree(tefmm_plan plan, int *n_nodes, int64_t *ns, int64_t *nt, int *layer,
                      int *level, int *ix, int *iy, int *iz, int *parent, int *s0, int *s1,
                      int *t0, int *t1, int *perm_s, int *perm_t);

/* Interaction lists of the last evaluation as CSR over target nodes:
 * V lists (M2L) and near-field lists (target leaves only; empty elsewhere).
 * With NULL arrays only the sizes are returned. */
int tefmm_export_lists(tefmm_plan plan, int64_t *n_v, int64_t *n_near, int *v_ptr, int *v_src,
                       int *near_ptr, int *near_src);

/* Moments (P2M/M2M) and locals (after L2L, before L2P) of the last
 * evaluation: host arrays [n_nodes * n_coeffs * 2] in graded multi-index order
 * (n = 0..p; k1 = n..0; k2 = n-k1..0; k3 = n-k1-k2).  NULL skips one. */
int tefmm_export_expansions(tefmm_plan plan, double *alpha, double *beta);

/* Cross-layer DCIM images held by the plan (Sec. 3.3: one fit of the
 * k3'-th z'-derivative density per target layer l, source layer l', part
 * (0 up-going, W = z - d_l; 1 down-going, W = d_{l-1} - z), octree level,
 * source z-box index iz_s and k3' = 0..p; the source z-centre is
 * lo_z + (iz_s + 1/2) side / 2^level of the last evaluation's root cube).
 * Fitted on demand by tefmm_eval and cached until the root cube's z-origin
 * or side changes.
 *   n_fits (out)        number of cached fits; with the other pointers all
 *                       NULL only this is returned;
 *   keys (out)          host int[6*n_fits]: (l, l', part, level, iz_s, k3');
 *   counts (out)        host int[n_fits]: images of each fit (<= 32);
 *   A, Z (out)          host double[2*32*n_fits]: image j of fit i at
 *                       [2*(32*i + j)] (real, imaginary).
 * Any of keys/counts/A/Z may be NULL.  Errors: INVALID_ARG. */
int tefmm_plan_cross_images(tefmm_plan plan, int *n_fits, int *keys, int *counts, double *A,
                            double *Z);

/* Replace or add cross-layer fits in the plan's cache (the inverse of
 * tefmm_plan_cross_images, same layouts): fit i with key keys[6*i..6*i+5] =
 * (l, l', part, level, iz_s, k3') takes the counts[i] images at
 * A[2*(32*i + j)], Z[2*(32*i + j)].  The fits describe the source z-centre of
 * the root cube of the plan's last evaluation (or set_points): an evaluation
 * with a different root cube z-origin or side discards the cache.  The next
 * tefmm_eval / tefmm_set_points rebuilds the cross-layer tables from them
 * (tefmm_apply is refused until then).  The parity tests use it to run the
 * device on the oracle's fits; the paper has no counterpart.
 * Errors: INVALID_ARG (a key outside the plan's layers, parts, p or levels, or
 * more than 32 images). */
int tefmm_plan_set_cross_images(tefmm_plan plan, int n_fits, const int *keys, const int *counts,
                                const double *A, const double *Z);

/* Read one Algorithm 2 table (Sec. 4.2, eq. ``symmetricdetable``) of a plan
 * made with TEFMM_ALG_TABLES, as built for its last geometry: the table of
 * same-layer term ``tag`` (0 up-up, 1 down-down, 2 up-down, 3 down-up) of
 * ``layer``.  Outputs (host): *n grid points per direction, *n_entries
 * entries per point (the T_{m,nu,n} in the order m = 0..2p, nu = m mod 2,
 * .., m step 2, n = 0..2p - m), range[3] = (rho_max, zeta_lo, zeta_hi) and,
 * unless T is NULL, T[2 * ((i * n + j) * n_entries + e)] (+1) = real (imag)
 * part of entry e at rho_i = i rho_max / (n - 1), zeta_j = zeta_lo + j
 * (zeta_hi - zeta_lo) / (n - 1).  Synchronous.
 * Errors: INVALID_ARG (no such table: other algorithm, no geometry, or the
 * layer has no M2L pairs or no such term), CUDA. */
int tefmm_plan_get_alg2_table(tefmm_plan plan, int layer, int tag, int *n, int *n_entries,
                              double *range, double *T);

/* ---- test hooks for the error paths --------------------------------------
 * No counterpart in the paper; used by the tests.
 * tefmm_debug_inject(kind, n): make the n-th (n >= 1) device allocation
 * (kind TEFMM_INJECT_ALLOC, returned as TEFMM_ERR_OOM) or the n-th batch of
 * DCIM fits (kind TEFMM_INJECT_FIT: plan creation's same-layer fits or an
 * evaluation's cross-layer fits, returned as TEFMM_ERR_FIT_FAILED) made by
 * the library from now on fail, once; kind 0 clears both.  Process-wide.
 * tefmm_debug_wait_probe(plan, ms, stream): one kernel waits, bounded by ms
 * milliseconds of device time (1..2000), on an mbarrier that nothing
 * completes; it raises the plan's timeout flag, and the call returns
 * TEFMM_ERR_TIMEOUT, the status a run-out wait of the tensor-core M2L gives.
 * Errors: INVALID_ARG. */
#define TEFMM_INJECT_ALLOC 1
#define TEFMM_INJECT_FIT 2
int tefmm_debug_inject(int kind, int n);
int tefmm_debug_wait_probe(tefmm_plan plan, int ms, void *stream);

/* The library's own primitives on caller DEVICE buffers, for their tests:
 * tefmm_debug_sort_u64 sorts n 64-bit keys (and, when d_vals_in is not NULL,
 * their int32 values) stably into d_keys_out / d_vals_out, leaving the inputs
 * unchanged; tefmm_debug_scan_i32 writes the exclusive (inclusive != 0:
 * inclusive) prefix sums of n int32 values.  Both allocate their scratch,
 * synchronise the stream and free it.  Errors: INVALID_ARG, OOM, CUDA. */
int tefmm_debug_sort_u64(const uint64_t *d_keys_in, uint64_t *d_keys_out, const int *d_vals_in,
                         int *d_vals_out, int64_t n, void *stream);
int tefmm_debug_scan_i32(const int *d_in, int *d_out, int64_t n, int inclusive, void *stream);

/* ---- fit without device allocation -------------------------------------
 * The paper has no counterpart to this call; it is a convenience of this
 * library.  It runs the same device DCIM fit as tefmm_plan_create (same
 * images, same order of terms as tefmm_plan_get_images) for callers that
 * cannot allocate device memory at that point: code whose device memory is
 * owned by a pre-sized pool allocator (where a stray cudaMalloc can fail or
 * fragment the pool), or latency-critical paths that must avoid an
 * allocation's implicit device synchronisation.  It calls no
 * cudaMalloc/cudaFree: its scratch is a fixed array of about 46 KB inside the
 * library, held by every device that loads the library until the process
 * exits.
 *   n_layers, interfaces, k_re, k_im, opt   as for tefmm_plan_create;
 *   stream                                  cudaStream_t for the fit; the call
 *                                           synchronises it before returning;
 *   n_terms (out)                           number of (layer, term) entries, <= 32;
 *   term_layer, term_tag (out, may be NULL) host int[4*n_layers];
 *   term_count (out)                        host int[4*n_layers], images per term;
 *   A, Z (out)                              host double[2*32*4*n_layers]: the images
 *                                           of term t at A[2*(32*t + j)], j < term_count[t].
 * The first call on a device looks up the array's device address and should
 * come before any stream capture; the address is kept for the process, so a
 * caller that resets the device (cudaDeviceReset) must not call this entry
 * point on that device afterwards.  Calls share the array: calls that overlap
 * on the GPU race and must be serialised by the caller.  Sizes beyond the
 * array (more than 32 fits, n_samples > 127, n_images > 32) return
 * TEFMM_ERR_INVALID_ARG; other errors as tefmm_plan_create. */
int tefmm_fit_images_noalloc(int n_layers, const double *interfaces, const double *k_re,
                             const double *k_im, const tefmm_options *opt, void *stream,
                             int *n_terms, int *term_layer, int *term_tag, int *term_count,
                             double *A, double *Z);

#ifdef __cplusplus
}
#endif
#endif /* TEFMM_H */
