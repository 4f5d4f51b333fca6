// M2L of the mixed-precision form on the 5th-generation tensor cores.
//
// Per key (a group of V pairs sharing one derivative table, see ops.cu) the
// translation of eq. ``tesourceboxtotargetbox`` is a complex matrix product
//   beta_t += H alpha_s,  H[k][k'] = C(k+k',k) (-1)^{k1'+k2'} (A_{k+k'} + (-1)^{k3'} B_{k+k'}),
// written here in real form  C^T (pairs x 2np) = X^T (pairs x 2np) . W^T  with
//   X^T[pair] = (Re alpha~_s, Im alpha~_s),  W = [[Re H, -Im H], [Im H, Re H]].
// Scaling by the box size h: alpha~_k = alpha_k / h^{|k|}, the table is used as
// T~_g = T_g h^{|g|}, and the result beta~_k = h^{|k|} beta_k.
//
// Precision: FP32 values split into TF32 hi/lo parts; three tcgen05.mma
// kind::tf32 products (hi.hi + hi.lo + lo.hi) accumulate in FP32 in TMEM.
//
// Kernel layout (k_wgen, k_m2l_tc below): k_wgen writes W^T per key and
// output slice in the MMA's shared-memory operand layout (TF32 hi and lo);
// k_m2l_tc takes one chunk of <= 128 pairs of one key (M = 128 rows of TMEM =
// pairs) and one slice of N <= 256 output columns, and walks K (2np, padded
// to 16) in stages of 8 through a 5-stage shared-memory ring filled by
// producer warps (bulk copy of the W^T block, 16-byte copies of the pairs'
// moment rows) and drained by one MMA-issuing thread.
// Operands are K-major without swizzle (8-row x 16-byte core matrices,
// LBO = 128 B between K-neighbours, SBO = 256 B between 8-row groups).
// Every wait is bounded; on a timeout the CTA raises a flag, skips its output
// and still releases its TMEM.
#include <algorithm>

#include "ops_common.cuh"

namespace {

constexpr int TM = 128;      // pairs per CTA (MMA M)
constexpr int KC = 8;        // K elements per pipeline stage (KC / 8 MMA K steps)
static_assert(KC % 8 == 0 && KC <= 32, "a stage holds whole MMA K steps of 8");
constexpr int NST = 5;       // pipeline stages (shared-memory buffers)
constexpr int NMAX = 256;    // widest output slice (the MMA's N for M = 128)
constexpr int NTHR = 256;
constexpr long SPIN_LIMIT = 4000000;
constexpr size_t W_BATCH_BYTES = (size_t)2 << 30;   // W^T blocks held at once, at most
constexpr size_t W_BATCH_MIN = (size_t)64 << 20;    // ... and at least (unless fewer are needed)

struct TcArgs {
    int nchunks;
    const int *chunk_start, *chunk_table, *chunk_cnt;
    const uint64_t *table_key;
    const cplx *tables;
    const int *items;            // sorted pair items (pair << 1 | kind)
    const int *pair_t, *v_src;
    const float *ah, *al;        // scaled moments, hi / lo, [node][Kpad]
    float *bt;                   // scaled locals accumulator [node][Ntot]
    const unsigned short *G;     // [k'][k]
    const float *cfA, *cfB;      // [k'][k] coefficients with signs
    const int *mi;
    int np, np2, Kpad, Ncta, Ntot, nblk;   // nblk: unused (1)
    double side;
    int *flags;
    // table of key tb: tables + (tb - tab_origin) * tab_stride; W^T blocks of the
    // keys tab_base.. of this launch (k_wgen); xmode: cross-layer tables (p + 1
    // slices of orders 2p - k3', entry scaled by h^{|g| + k3'})
    int tab_origin, tab_base, tab_stride, xmode, p;
    int MT;                      // tiles of 128 pairs per pass (MT * Ncta <= 512 TMEM columns)
    int nsplit;                  // column slices per chunk
    const float *W;              // precomputed W^T blocks (k_wgen)
    int tcols;                   // TMEM columns allocated (power of 2 >= MT * Ncta)
    const cplx *kl;              // wavenumber per layer (reversed cross keys)
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;   // LBO
    d |= (uint64_t)((8 * KC * 4) >> 4) << 32;   // SBO: 8 rows x KC 4-byte elements
    d |= (uint64_t)1 << 46;            // descriptor version
    return d;
}

// K order of the contraction (kcol): column 2j + part holds part (0 real, 1
// imaginary) of the source coefficient k' = n_p - 1 - j, i.e. the highest
// orders first.  The terms shrink with the order, so the FP32 accumulator
// collects the small terms before the large ones; this ordering measured
// 2.5x less accumulation error than the graded order.
//
// byte offset of (row r, k) in a K-major no-swizzle tile with KC columns:
// 8-row x 16-byte core matrices, LBO = 128 B between K-neighbouring core
// matrices, SBO = 32 KC B between 8-row groups; one MMA K step (8 values)
// spans two core matrices, so step s of a stage starts 256 s bytes in
__device__ __forceinline__ int koff(int r, int k) {
    return (r >> 3) * (32 * KC) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long it = 0; it < SPIN_LIMIT; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// W^T blocks of one key, one column slice and one K chunk: NC x KC TF32 hi
// values in the K-major core-matrix layout of koff(), then the lo values;
// block (key - tab_base, slice, ch) at W + ((tbl * nsplit + slice) * nk + ch) * 2 * NC * KC.
// One CTA per (key, slice): the scaled table T~_g = T_g h^{|g|} (cross-layer:
// h^{|g| + k3'} in slice k3') goes to shared memory in FP32 and every entry
// of the real form [[Re H, -Im H], [Im H, Re H]] of the slice is generated once.
__global__ void __launch_bounds__(NTHR) k_wgen(TcArgs a, int ntab, float *__restrict__ W) {
    const int tbl = blockIdx.x / a.nsplit, slice = blockIdx.x % a.nsplit;
    if (tbl >= ntab) return;
    const int tid = threadIdx.x;
    const int NC = a.Ncta, np = a.np, nk = a.Kpad / KC;
    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *tab = (float2 *)smem;
    const int tb = a.tab_base + tbl;
    const uint64_t key = a.table_key[tb];
    const int lev = key_level(key);
    const double h = a.side / (double)(1 << lev);
    const float *cf = key_is_B(key) ? a.cfB : a.cfA;
    // a reversed cross key: (k_lt / k_ls)^2 times the transposed matrix of its component
    const bool rev = a.xmode && xkey_rev(key);
    cplx fac = mkc(1, 0);
    if (rev) {
        const XKey x = xkey_decode(key);
        const cplx r = cdiv(a.kl[x.lt], a.kl[x.ls]);
        fac = cmul(r, r);
    }
    {
        const cplx *T = a.tables + (int64_t)(tb - a.tab_origin) * a.tab_stride;
        const int nsl = a.xmode ? a.p + 1 : 1;
        int off = 0;
        for (int k3p = 0; k3p < nsl; ++k3p) {
            const int n2 = a.xmode ? ncoef(2 * a.p - k3p) : a.np2;
            for (int g = tid; g < n2; g += NTHR) {
                int n = a.mi[3 * g] + a.mi[3 * g + 1] + a.mi[3 * g + 2] + (a.xmode ? k3p : 0);
                double s = 1.0;
                for (int i = 0; i < n; ++i) s *= h;
                cplx v = T[off + g];
                if (rev) v = cmul(fac, v);
                tab[off + g] = make_float2((float)(v.x * s), (float)(v.y * s));
            }
            off += n2;
        }
    }
    __syncthreads();
    // one thread per 16-byte chunk of the layout (row nl, K values 4 cg .. 4 cg + 3):
    // the chunk's two source coefficients k' (real and imaginary column each)
    // need two table lookups, and its hi and lo parts are one 16-byte store each
    const int n0 = slice * NC;
    for (int ch = 0; ch < nk; ++ch) {
        float *blk = W + (((int64_t)tbl * a.nsplit + slice) * nk + ch) * (2 * NC * KC);
        const int c0 = ch * KC;
        for (int j = tid; j < (KC / 4) * NC; j += NTHR) {
            const int cg = j / NC, nl = j - cg * NC;
            const int n = n0 + nl;
            float w[4] = {0.f, 0.f, 0.f, 0.f};
            if (n < 2 * np) {
                const int k = n < np ? n : n - np, po = n < np ? 0 : 1;
#pragma unroll
                for (int hp = 0; hp < 2; ++hp) {
                    const int col = c0 + 4 * cg + 2 * hp;          // real column of k'; col + 1 imaginary
                    if (col < 2 * np) {
                        const int kp = np - 1 - (col >> 1);         // K order: see kcol()
                        const int64_t o = rev ? (int64_t)k * np + kp : (int64_t)kp * np + k;
                        const float cfv = __ldg(cf + o);
                        const float2 t = tab[__ldg(a.G + o)];
                        const float hr = cfv * t.x, hi = cfv * t.y;
                        // row part po, column parts 0 and 1 of [[Re H, -Im H], [Im H, Re H]]
                        w[2 * hp] = po == 0 ? hr : hi;
                        w[2 * hp + 1] = po == 0 ? -hi : hr;
                    }
                }
            }
            float4 wh, wl;
            wh.x = tf32_rn(w[0]);
            wh.y = tf32_rn(w[1]);
            wh.z = tf32_rn(w[2]);
            wh.w = tf32_rn(w[3]);
            wl.x = tf32_rn(w[0] - wh.x);
            wl.y = tf32_rn(w[1] - wh.y);
            wl.z = tf32_rn(w[2] - wh.z);
            wl.w = tf32_rn(w[3] - wh.w);
            const int e = koff(nl, 4 * cg) >> 2;
            *(float4 *)(blk + e) = wh;
            *(float4 *)(blk + NC * KC + e) = wl;
        }
    }
}

// wait until at most n of this thread's cp.async groups are pending
__device__ __forceinline__ void cp_async_wait(int n) {
    if (n <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else if (n == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else asm volatile("cp.async.wait_group 3;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

// One CTA: one chunk of up to chunk_pairs pairs of one key, and one slice of
// NC output columns, taken in passes of MT tiles of TM = 128 pairs; TMEM holds
// one 128 x NC FP32 accumulator per tile (MT * NC <= 512 columns).  The K
// dimension runs through a ring of NST shared-memory stages of KC values,
// warp-specialised:
//  * warps 0-7 (producers): for stage g they wait until the MMAs that last
//    read the stage's buffer are done (empty[g % NST], committed by the MMA
//    warp), thread 0 starts the bulk copy of the W^T block (completing on
//    wbar), and every thread issues its two 16-byte copies of moment rows
//    (addresses fixed per pass).  LAG stages later the thread waits for its
//    own copies, fences them for the tensor core (async proxy) and arrives on
//    full[g % NST];
//  * warp 8, lane 0 (MMA issuer): waits full and wbar of stage g, issues the
//    3 MMAs per tile (hi.hi, hi.lo, lo.hi) and commits them to empty; after
//    the pass's last stage it also commits to done (one phase per pass).
// Warps 0-7 wait on done and move the accumulators out of TMEM (the
// epilogue).  Every wait is bounded; on a timeout the CTA raises a flag, skips
// its output, waits for its copies and MMAs in flight (again bounded) and
// releases its TMEM.
constexpr int NPROD = 256;              // producer / epilogue threads
constexpr int NTHR_TC = NPROD + 32;     // + the MMA warp
constexpr int LAG = 2;                  // stages a producer keeps in flight before arriving
static_assert(LAG < NST, "a producer must arrive for a stage before it waits for that stage's buffer");

__global__ void __launch_bounds__(NTHR_TC, 1) k_m2l_tc(TcArgs a) {
    // 1-D grid: the nsplit column slices of one chunk are adjacent blocks, so
    // they run together and share the chunk's moment rows through L2
    const int c = blockIdx.x / a.nsplit;
    const int slice = blockIdx.x % a.nsplit;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int MT = a.MT, NC = a.Ncta;
    extern __shared__ __align__(1024) unsigned char smem[];
    // layout: [NST stages][Xh (MT tiles) | Xl (MT tiles) | Wh | Wl]
    const int tbytes = TM * KC * 4;                 // one X tile
    const int xbytes = MT * tbytes;
    const int wbytes = NC * KC * 4;
    const int stbytes = 2 * xbytes + 2 * wbytes;
    __shared__ __align__(8) uint64_t full[NST], empty[NST], wbar[NST], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_src[4 * TM], s_tgt[4 * TM];
    __shared__ int s_fail, s_issued, s_committed;

    const int tb = a.chunk_table[c];
    const int cnt = a.chunk_cnt[c];
    const int st = a.chunk_start[c];
    const int nk = a.Kpad / KC;
    const float *Wkey = a.W + ((int64_t)(tb - a.tab_base) * a.nsplit + slice) * nk * (2 * NC * KC);

    if (tid == 0) {
        s_fail = 0;
        s_issued = 0;        // stages whose W^T copy was started
        s_committed = -1;    // last stage whose MMAs were committed
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&tmem_base)), "r"(a.tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&full[i])), "r"(NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&empty[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&wbar[i])));
        }
        // done: one phase per pass, completed by the commit after the pass's last MMAs
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NC >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);
    const int n0 = slice * NC;             // first output column of this CTA
    int gbase = 0;                         // global index of the pass's first K stage
    int npass = 0;                         // passes completed (phase of done)

    for (int pb = 0; pb < cnt; pb += MT * TM) {
        const int npair = min(MT * TM, cnt - pb);
        const int ntile = (npair + TM - 1) / TM;
        for (int r = tid; r < MT * TM; r += NTHR_TC) {
            if (r < npair) {
                int e = a.items[st + pb + r] >> 1;
                s_src[r] = a.v_src[e];
                s_tgt[r] = a.pair_t[e];
            } else {
                s_src[r] = -1;
                s_tgt[r] = -1;
            }
        }
        __syncthreads();
        if (warp < NPROD / 32) {
            // ---------------------------------------------------------- producers
            // thread t copies the 16-byte chunks (4 K values each) q, q + 2, .. (q = t & 1)
            // of row t >> 1 of every tile, hi and lo: source addresses advance by KC
            // floats per stage
            const int q = tid & 1, r = tid >> 1;
            bool okp = true;
            for (int kc = 0; kc < nk && okp; ++kc) {
                const int g = gbase + kc, sb = g % NST;
                if (g >= NST && !mbar_wait(su32(&empty[sb]), ((g - NST) / NST) & 1)) okp = false;
                if (!okp || *(volatile int *)&s_fail) {
                    okp = false;
                    break;
                }
                unsigned char *buf = smem + sb * stbytes;
                if (tid == 0) {
                    const uint32_t bytes = 2u * (uint32_t)wbytes;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 :: "r"(su32(&wbar[sb])), "r"(bytes) : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(su32(buf + 2 * xbytes)), "l"(Wkey + (int64_t)kc * (2 * NC * KC)),
                                    "r"(bytes), "r"(su32(&wbar[sb]))
                                 : "memory");
                    s_issued = g + 1;
                }
                for (int mt = 0; mt < ntile; ++mt) {
                    const int s = s_src[mt * TM + r];
                    const uint32_t sz = s >= 0 ? 16u : 0u;
#pragma unroll
                    for (int cq = q; cq < KC / 4; cq += 2) {
                        const int64_t so = (int64_t)(s >= 0 ? s : 0) * a.Kpad + kc * KC + 4 * cq;
                        const uint32_t dst = su32(buf + mt * tbytes + koff(r, 4 * cq));
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                     :: "r"(dst), "l"(a.ah + so), "r"(sz) : "memory");
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                     :: "r"(dst + (uint32_t)xbytes), "l"(a.al + so), "r"(sz) : "memory");
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (kc >= LAG) {
                    cp_async_wait(LAG);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(su32(&full[(g - LAG) % NST]));
                }
            }
            if (okp) {
                // the last LAG stages of the pass
                for (int kc = max(nk - LAG, 0); kc < nk; ++kc) {
                    cp_async_wait(nk - 1 - kc);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(su32(&full[(gbase + kc) % NST]));
                }
            } else {
                atomicExch(&s_fail, 1);
            }
        } else if (lane == 0) {
            // ----------------------------------------------------------- MMA issuer
            for (int kc = 0; kc < nk; ++kc) {
                const int g = gbase + kc, sb = g % NST;
                if (!mbar_wait(su32(&full[sb]), (g / NST) & 1) || !mbar_wait(su32(&wbar[sb]), (g / NST) & 1)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                unsigned char *buf = smem + sb * stbytes;
                for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t ko = 256u * (uint32_t)ks;       // K step ks of the stage
                const uint64_t dwh = sdesc(su32(buf + 2 * xbytes) + ko), dwl = sdesc(su32(buf + 2 * xbytes + wbytes) + ko);
                const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
                for (int mt = 0; mt < ntile; ++mt) {
                    const uint32_t d = tmem + (uint32_t)(mt * NC);
                    const uint64_t dxh = sdesc(su32(buf + mt * tbytes) + ko);
                    const uint64_t dxl = sdesc(su32(buf + xbytes + mt * tbytes) + ko);
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(d), "l"(dxh), "l"(dwh), "r"(idesc), "r"(acc0));
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(d), "l"(dxh), "l"(dwl), "r"(idesc), "r"(1u));
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(d), "l"(dxl), "l"(dwh), "r"(idesc), "r"(1u));
                }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(su32(&empty[sb])) : "memory");
                s_committed = g;
                if (kc == nk - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(su32(&done)) : "memory");
            }
        }
        __syncwarp();
        gbase += nk;
        if (warp < NPROD / 32) {
            // ------------------------------------------------------------ epilogue
            // the pass's last commit (to done) covers every MMA of the pass
            bool ok = !*(volatile int *)&s_fail && mbar_wait(su32(&done), npass & 1);
            if (!ok) atomicExch(&s_fail, 1);
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (ok) {
                // warp w reads TMEM lanes 32*(w%4).., column half w/4 of each tile
                const int row = (warp & 3) * 32 + lane;
                const int chalf = warp >> 2;
                const int colw = NC / 2;
                for (int mt = 0; mt < ntile; ++mt) {
                    const int t = s_tgt[mt * TM + row];
                    for (int cc = chalf * colw; cc < (chalf + 1) * colw; cc += 16) {
                        uint32_t v[16];
                        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(mt * NC + cc);
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                                       "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                                       "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                                     : "r"(taddr));
                        asm volatile("tcgen05.wait::ld.sync.aligned;");
                        if (t >= 0) {
                            float *dst = a.bt + (int64_t)t * a.Ntot + n0 + cc;
                            for (int qq = 0; qq < 16; qq += 4) {
                                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                                             :: "l"(dst + qq), "f"(__uint_as_float(v[qq])), "f"(__uint_as_float(v[qq + 1])),
                                                "f"(__uint_as_float(v[qq + 2])), "f"(__uint_as_float(v[qq + 3]))
                                             : "memory");
                            }
                        }
                    }
                }
            }
        }
        // TMEM reads of this pass done before the next pass's MMAs overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        ++npass;
        if (s_fail) break;
    }
    // nothing of this CTA may still be landing in its shared memory or running
    // on its TMEM: the moment-row copies, the W^T bulk copies, the MMAs
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (tid == 0) {
        const int gissued = s_issued;
        for (int sb = 0; sb < NST && sb < gissued; ++sb) {
            const int last = sb + (gissued - 1 - sb) / NST * NST;     // last stage that used buffer sb
            mbar_wait(su32(&wbar[sb]), (last / NST) & 1);
        }
        const int gc = s_committed;
        if (gc >= 0) mbar_wait(su32(&empty[gc % NST]), (gc / NST) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_fail && tid == 0) atomicOr(a.flags, FLAG_TIMEOUT);   // only a bounded wait sets s_fail
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(a.tcols));
    }
}

// alpha (FP64 complex, [node][np]) -> scaled FP32 TF32 hi/lo rows [node][Kpad]
__global__ void k_split_alpha(int nn, const int *__restrict__ level, double side, int np, int Kpad,
                              const int *__restrict__ mi, const cplx *__restrict__ alpha,
                              float *__restrict__ ah, float *__restrict__ al) {
    int node = blockIdx.x;
    if (node >= nn) return;
    double h = side / (double)(1 << level[node]);
    double ih = 1.0 / h;
    for (int c = threadIdx.x; c < Kpad; c += blockDim.x) {
        float v = 0.f;
        if (c < 2 * np) {
            int k = np - 1 - (c >> 1);                       // K order: see kcol()
            int n = mi[3 * k] + mi[3 * k + 1] + mi[3 * k + 2];
            double s = 1.0;
            for (int i = 0; i < n; ++i) s *= ih;
            cplx x = alpha[(int64_t)node * np + k];
            v = (float)(((c & 1) == 0 ? x.x : x.y) * s);
        }
        float hi = tf32_rn(v);
        ah[(int64_t)node * Kpad + c] = hi;
        al[(int64_t)node * Kpad + c] = tf32_rn(v - hi);
    }
}

// beta (FP64) += beta~ / h^{|k|}
__global__ void k_fold_beta(int nn, const int *__restrict__ level, double side, int np, int Ntot,
                            const int *__restrict__ mi, const float *__restrict__ bt,
                            cplx *__restrict__ beta) {
    int node = blockIdx.x;
    if (node >= nn) return;
    double h = side / (double)(1 << level[node]);
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int n = mi[3 * k] + mi[3 * k + 1] + mi[3 * k + 2];
        double s = 1.0;
        for (int i = 0; i < n; ++i) s *= h;
        double is = 1.0 / s;
        cplx v = beta[(int64_t)node * np + k];
        v.x += (double)bt[(int64_t)node * Ntot + k] * is;
        v.y += (double)bt[(int64_t)node * Ntot + np + k] * is;
        beta[(int64_t)node * np + k] = v;
    }
}

}  // namespace

// column geometry of the tensor-core M2L: K padded to 16; the 2 n_p output
// columns are cut into nsplit = ceil(2 n_p / NMAX) slices of Ncta columns
// (a multiple of 32, at most NMAX <= 256: the MMA's N, and 16-column TMEM
// loads per half of the epilogue warps)
void m2l_tc_geometry(int np, int MT, int *Kpad, int *Ncta, int *nsplit) {
    const int R = 2 * np;
    (void)MT;
    *Kpad = (R + 15) / 16 * 16;
    *nsplit = (R + NMAX - 1) / NMAX;
    *Ncta = ((R + *nsplit - 1) / *nsplit + 31) / 32 * 32;
}

namespace {

// launch: split moments, tensor-core contraction of chunks [c0, c0 + nch), fold into beta_out
int tc_launch(tefmm_plan_s *P, cudaStream_t st, int c0, int nch, const cplx *alpha, cplx *beta_out,
              const cplx *tables, int tab_origin, int tab_first, int ntab, int tab_stride, int xmode,
              const unsigned short *G, const float *cfA, const float *cfB, size_t tab_bytes,
              DBuf &ah, DBuf &al, DBuf &bt, DBuf &Wbuf, int MT) {
    const int nn = P->n_nodes, np = P->np;
    int Kpad, Ncta, nsplit;
    m2l_tc_geometry(np, MT, &Kpad, &Ncta, &nsplit);
    const int Ntot = Ncta * nsplit;
    // MMA shape M = 128, N = Ncta (multiple of 16, at most 256); MT accumulators in TMEM
    if (Ncta > 256 || Ncta % 32 != 0 || MT < 1 || MT > 4 || MT * Ncta > 512) return TEFMM_ERR_INVALID_ARG;
    int tcols = 32;
    while (tcols < MT * Ncta) tcols <<= 1;
    TRY(dbuf_ensure(ah, (size_t)nn * Kpad * 4));
    TRY(dbuf_ensure(al, (size_t)nn * Kpad * 4));
    TRY(dbuf_ensure(bt, (size_t)nn * Ntot * 4));
    CUDA_TRY(cudaMemsetAsync(bt.p, 0, (size_t)nn * Ntot * 4, st));
    k_split_alpha<<<nn, 128, 0, st>>>(nn, dp<int>(P->n_level), P->side, np, Kpad, dp<int>(P->d_mi),
                                      alpha, dp<float>(ah), dp<float>(al));
    P->launches++;
    TcArgs a;
    a.nchunks = nch;
    a.chunk_start = dp<int>(P->chunk_start) + c0;
    a.chunk_table = dp<int>(P->chunk_key) + c0;
    a.chunk_cnt = dp<int>(P->chunk_cnt) + c0;
    a.table_key = dp<uint64_t>(P->table_slot);
    a.tables = tables;
    a.items = dp<int>(P->pair_idx_sorted);
    a.pair_t = dp<int>(P->pair_t);
    a.v_src = dp<int>(P->v_src);
    a.ah = dp<float>(ah);
    a.al = dp<float>(al);
    a.bt = dp<float>(bt);
    a.G = G;
    a.cfA = cfA;
    a.cfB = cfB;
    a.mi = dp<int>(P->d_mi);
    a.np = np;
    a.np2 = P->np2;
    a.Kpad = Kpad;
    a.Ncta = Ncta;
    a.Ntot = Ntot;
    a.nblk = 1;
    a.MT = MT;
    a.side = P->side;
    a.flags = dp<int>(P->flags);
    a.tab_origin = tab_origin;
    a.tab_base = tab_first;
    a.tab_stride = tab_stride;
    a.xmode = xmode;
    a.p = P->p;
    a.nsplit = nsplit;
    a.tcols = tcols;
    a.kl = dp<cplx>(P->d_k);
    // keys in batches whose W^T blocks fit in W_BATCH_BYTES; chunks are sorted
    // by key, so a batch of keys is a contiguous range of chunks
    const int nk = Kpad / KC;
    const size_t wkey = (size_t)nsplit * nk * 2 * Ncta * KC * sizeof(float);
    // a quarter of what all keys need, within [W_BATCH_MIN, W_BATCH_BYTES]: large
    // problems take few batches, and many plans alive at once (batched
    // evaluation) do not each hold gigabytes
    const size_t wcap = std::min(W_BATCH_BYTES, std::max(W_BATCH_MIN, (size_t)ntab * wkey / 4));
    const int kb = (int)std::max<size_t>(1, std::min<size_t>((size_t)ntab, wcap / wkey));
    TRY(dbuf_ensure(Wbuf, (size_t)kb * wkey));
    a.W = dp<float>(Wbuf);
    if ((int64_t)P->chunk_key_host.size() < (int64_t)c0 + nch) return TEFMM_ERR_DEVICE_CHECK;
    const int *ctab = P->chunk_key_host.data() + c0;    // host copy made with the geometry
    TRY(smem_optin(k_wgen));
    const size_t sm = m2l_tc_smem(np, MT, 0);
    TRY(smem_optin(k_m2l_tc));
    int cb = 0;
    for (int t0 = tab_first; t0 < tab_first + ntab; t0 += kb) {
        const int t1 = std::min(t0 + kb, tab_first + ntab);
        int ce = cb;
        while (ce < nch && ctab[ce] < t1) ++ce;
        a.tab_base = t0;
        k_wgen<<<(unsigned)((int64_t)(t1 - t0) * nsplit), NTHR, tab_bytes, st>>>(a, t1 - t0, dp<float>(Wbuf));
        P->launches++;
        if (ce > cb) {
            TcArgs b = a;
            b.chunk_start = a.chunk_start + cb;
            b.chunk_table = a.chunk_table + cb;
            b.chunk_cnt = a.chunk_cnt + cb;
            b.nchunks = ce - cb;
            TRY(kernel_event(P, st));
            k_m2l_tc<<<(unsigned)((int64_t)(ce - cb) * nsplit), NTHR_TC, sm, st>>>(b);
            P->launches++;
            TRY(kernel_event(P, st));
        }
        cb = ce;
    }
    k_fold_beta<<<nn, 128, 0, st>>>(nn, dp<int>(P->n_level), P->side, np, Ntot, dp<int>(P->d_mi),
                                    dp<float>(bt), beta_out);
    P->launches++;
    CUDA_TRY(cudaGetLastError());
    return TEFMM_OK;
}

}  // namespace

// shared memory of the tensor-core M2L with MT tiles per pass and a table of
// tab_entries complex entries
size_t m2l_tc_smem(int np, int MT, int tab_entries) {
    int Kpad, Ncta, nsplit;
    m2l_tc_geometry(np, MT, &Kpad, &Ncta, &nsplit);
    return NST * (size_t)(2 * MT * TM * KC * 4 + 2 * Ncta * KC * 4) + (size_t)tab_entries * sizeof(float2);
}

int m2l_apply_tc_cross(tefmm_plan_s *P, cudaStream_t st, const cplx *alpha_x, cplx *beta_x,
                       const unsigned short *xgs, const float *xcf) {
    const int c0 = (int)P->x_first_chunk, nch = (int)(P->n_chunks - P->x_first_chunk);
    if (nch <= 0) return TEFMM_OK;
    return tc_launch(P, st, c0, nch, alpha_x, beta_x, dp<cplx>(P->xtables), P->x_first_table,
                     P->x_first_table, P->n_xtables, P->NX, 1, xgs, xcf, xcf, (size_t)P->NX * sizeof(float2),
                     P->tc_xah, P->tc_xal, P->tc_xbt, P->tc_xW, TC_MT_CROSS);
}

int m2l_apply_tc(tefmm_plan_s *P, cudaStream_t st) {
    const int nn = P->n_nodes, np = P->np;
    TRY(dbuf_ensure(P->beta, (size_t)nn * np * sizeof(cplx)));
    CUDA_TRY(cudaMemsetAsync(P->beta.p, 0, (size_t)nn * np * sizeof(cplx), st));
    const int nch = (int)P->x_first_chunk;    // same-layer chunks (cross-layer ones follow)
    if (nch == 0) return TEFMM_OK;
    TRY(dbuf_ensure(P->tc_cfA, (size_t)np * np * 4));
    TRY(dbuf_ensure(P->tc_cfB, (size_t)np * np * 4));
    if (P->tc_cf_np != np) {
        // FP32 copies of the M2L coefficients (exact: multinomials < 2^24 and signs)
        std::vector<double> a((size_t)np * np), b((size_t)np * np);
        CUDA_TRY(cudaMemcpy(a.data(), P->d_m2l_cA.p, a.size() * 8, cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(b.data(), P->d_m2l_cB.p, b.size() * 8, cudaMemcpyDeviceToHost));
        std::vector<float> fa(a.begin(), a.end()), fb(b.begin(), b.end());
        CUDA_TRY(cudaMemcpy(P->tc_cfA.p, fa.data(), fa.size() * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(P->tc_cfB.p, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice));
        P->tc_cf_np = np;
    }
    return tc_launch(P, st, 0, nch, dp<cplx>(P->alpha), dp<cplx>(P->beta), dp<cplx>(P->tables), 0, 0,
                     P->x_first_table, P->np2, 0, dp<unsigned short>(P->d_m2l_g), dp<float>(P->tc_cfA),
                     dp<float>(P->tc_cfB), (size_t)P->np2 * sizeof(float2), P->tc_ah, P->tc_al, P->tc_bt,
                     P->tc_W, TC_MT);
}
