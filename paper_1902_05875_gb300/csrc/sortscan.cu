// Prefix sums and the stable radix sort of the tree, list and M2L-key
// builders.
//
// Scan of int32 (exclusive or inclusive): tiles of SCAN_TILE values, one CTA
// each.  A CTA scans its tile (per-thread sequential sums, then a warp-shuffle
// scan of the thread totals) and writes the tile total.  The tile totals are
// scanned the same way (recursively while there is more than one tile), and a
// last kernel adds each tile's offset.
//
// Sort: least-significant-digit radix sort of 64-bit keys (optionally with an
// int32 value each), 4-bit digits, 16 passes, stable.  A pass:
// (1) every CTA counts the digits of its tile of SORT_TILE keys;
// (2) the counts, laid out digit-major ([digit][tile]), are scanned, giving
//     each (digit, tile) its first output position;
// (3) every CTA re-reads its tile and writes each key to that position plus
//     its rank among the tile's keys of the same digit.  The rank is the
//     key's order within its thread's consecutive run, plus the keys of that
//     digit held by the threads before it.  So equal digits keep their input
//     order, which makes every pass, and the sort, stable.  The tile is
//     reordered by digit in shared memory first, so that the global writes
//     are runs of consecutive positions.
// Only the passes over digits that differ between keys run (one OR/AND
// reduction of the keys finds them); they ping-pong between the output and a
// scratch buffer so that the last one lands in the output.
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int SORT_THREADS = 256, SORT_ITEMS = 16, SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int RADIX_BITS = 4, RADIX = 1 << RADIX_BITS;

// exclusive scan of v over the block (blockDim.x = 256); *total gets the sum
__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int before = warp > 0 ? warp_sums[warp - 1] : 0;
    const int res = before + x - v;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return res;
}

// per tile: out = exclusive (or inclusive) scan within the tile; sums[tile] = tile total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const int *__restrict__ in, int *__restrict__ out,
                                                            int64_t n, int inclusive, int *__restrict__ sums) {
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int total = 0;
    int run = block_excl_scan(s, ws, &total);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = inclusive ? run + v[i] : run;
        run += v[i];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int *__restrict__ out, int64_t n, const int *__restrict__ offs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / SCAN_TILE];
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// scratch ints for scanning n values: the tile totals of every recursion level
int64_t scan_scratch(int64_t n) {
    int64_t s = 0;
    for (int64_t m = ceil_div(n, SCAN_TILE); m > 1; m = ceil_div(m, SCAN_TILE)) s += 2 * m;
    return s + 2;
}

int scan_rec(const int *in, int *out, int64_t n, bool inclusive, int *scratch, cudaStream_t st) {
    if (n <= 0) return TEFMM_OK;
    const int64_t nt = ceil_div(n, SCAN_TILE);
    int *sums = scratch, *offs = scratch + nt;
    k_scan_tile<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, out, n, inclusive ? 1 : 0, sums);
    CUDA_TRY(cudaGetLastError());
    if (nt > 1) {
        TRY(scan_rec(sums, offs, nt, false, scratch + 2 * nt, st));
        k_scan_add<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(out, n, offs);
        CUDA_TRY(cudaGetLastError());
    }
    return TEFMM_OK;
}

}  // namespace

int dev_scan_i32(tefmm_plan_s *P, const int *in, int *out, int64_t n, bool inclusive, cudaStream_t st) {
    if (n <= 0) return TEFMM_OK;
    TRY(dbuf_ensure(P->scan_tmp, (size_t)scan_scratch(n) * sizeof(int)));
    TRY(scan_rec(in, out, n, inclusive, dp<int>(P->scan_tmp), st));
    P->launches += 1 + 2 * (ceil_div(n, SCAN_TILE) > 1 ? 1 : 0);
    return TEFMM_OK;
}

namespace {

// digit counts of every tile: counts[digit * ntile + tile]
__global__ void __launch_bounds__(SORT_THREADS) k_radix_count(const uint64_t *__restrict__ keys, int64_t n,
                                                              int shift, int ntile, int *__restrict__ counts) {
    __shared__ int c[RADIX];
    if (threadIdx.x < RADIX) c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE + (int64_t)threadIdx.x * SORT_ITEMS;
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i)
        if (base + i < n) atomicAdd(&c[(int)((keys[base + i] >> shift) & (RADIX - 1))], 1);
    __syncthreads();
    if (threadIdx.x < RADIX) counts[(int64_t)threadIdx.x * ntile + blockIdx.x] = c[threadIdx.x];
}

// stable scatter of one tile by the digit at shift; offs = exclusive scan of
// the counts.  The tile is first reordered by digit in shared memory (each
// key at its digit's tile offset plus its rank), then written out so that
// consecutive threads write consecutive positions of one digit's run.
// Dynamic shared memory: keys [SORT_TILE] u64, values [SORT_TILE] int,
// ranks [RADIX][SORT_THREADS] int.
// OR and AND of the keys other than ~0 (the "no item" key of the M2L
// builder), and whether a ~0 key occurs: orand = {OR, AND, any ~0}
__global__ void k_key_bits(const uint64_t *__restrict__ keys, int64_t n, unsigned long long *__restrict__ orand) {
    unsigned long long o = 0ULL, a = ~0ULL, inv = 0ULL;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        if (k == ~0ULL) {
            inv = 1ULL;
        } else {
            o |= k;
            a &= k;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, off);
        a &= __shfl_xor_sync(0xffffffffu, a, off);
        inv |= __shfl_xor_sync(0xffffffffu, inv, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&orand[0], o);
        atomicAnd(&orand[1], a);
        atomicOr(&orand[2], inv);
    }
}

constexpr size_t SCATTER_SMEM = (size_t)SORT_TILE * 12 + (size_t)RADIX * SORT_THREADS * 4;
__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(const uint64_t *__restrict__ kin,
                                                                const int *__restrict__ vin,
                                                                uint64_t *__restrict__ kout, int *__restrict__ vout,
                                                                int64_t n, int shift, int ntile,
                                                                const int *__restrict__ offs) {
    extern __shared__ __align__(16) unsigned char rsm[];
    uint64_t *skey = (uint64_t *)rsm;
    int *sval = (int *)(rsm + (size_t)SORT_TILE * 8);
    int *rank = sval + SORT_TILE;                      // per digit and thread: keys of that digit before it
    __shared__ int ws[32];
    __shared__ int first[RADIX];                       // output position of the tile's first key of each digit
    __shared__ int tot[RADIX], lfirst[RADIX];          // the tile's keys per digit, and their offsets in the tile
    const int64_t tbase = (int64_t)blockIdx.x * SORT_TILE;
    const int64_t base = tbase + (int64_t)threadIdx.x * SORT_ITEMS;
    if (threadIdx.x < RADIX) first[threadIdx.x] = offs[(int64_t)threadIdx.x * ntile + blockIdx.x];
    uint64_t k[SORT_ITEMS];
    int d[SORT_ITEMS];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        const bool ok = base + i < n;
        k[i] = ok ? kin[base + i] : 0;
        d[i] = ok ? (int)((k[i] >> shift) & (RADIX - 1)) : -1;
    }
#pragma unroll
    for (int dd = 0; dd < RADIX; ++dd) {
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) cnt += d[i] == dd;
        int t = 0;
        rank[dd * SORT_THREADS + threadIdx.x] = block_excl_scan(cnt, ws, &t);
        if (threadIdx.x == 0) tot[dd] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int o = 0;
        for (int dd = 0; dd < RADIX; ++dd) {
            lfirst[dd] = o;
            o += tot[dd];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        if (d[i] < 0) continue;
        int &r = rank[d[i] * SORT_THREADS + threadIdx.x];   // this thread's column: no other writer
        const int lp = lfirst[d[i]] + r;
        ++r;
        skey[lp] = k[i];
        if (vin) sval[lp] = vin[base + i];
    }
    __syncthreads();
    const int cnt_tile = (int)min((int64_t)SORT_TILE, n - tbase);
    for (int j = threadIdx.x; j < cnt_tile; j += SORT_THREADS) {
        const uint64_t key = skey[j];
        const int dd = (int)((key >> shift) & (RADIX - 1));
        const int64_t pos = (int64_t)first[dd] + (j - lfirst[dd]);
        kout[pos] = key;
        if (vin) vout[pos] = sval[j];
    }
}

}  // namespace

// Stable sort of n 64-bit keys (and int32 values when vin is given) into
// kout / vout; kin / vin are left unchanged.
int dev_sort_u64(tefmm_plan_s *P, const uint64_t *kin, uint64_t *kout, const int *vin, int *vout, int64_t n,
                 cudaStream_t st) {
    if (n <= 0) return TEFMM_OK;
    const int64_t ntile = ceil_div(n, SORT_TILE);
    const int64_t nc = RADIX * ntile;
    // scratch: keys [n], values [n], counts [nc], offsets [nc]
    const size_t kb = (size_t)n * 8, vb = vin ? (size_t)n * 4 : 0, cb = (size_t)nc * 4;
    TRY(dbuf_ensure(P->sort_tmp, kb + vb + 2 * cb + 64));
    unsigned char *t = (unsigned char *)P->sort_tmp.p;
    uint64_t *ktmp = (uint64_t *)t;
    int *vtmp = vin ? (int *)(t + kb) : nullptr;
    int *counts = (int *)(t + kb + vb);
    int *offs = counts + nc;
    TRY(dbuf_ensure(P->scan_tmp, (size_t)scan_scratch(nc) * sizeof(int)));
    CUDA_TRY(cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SCATTER_SMEM));
    // digits that are equal in every key leave the order unchanged: only the
    // passes over digits that vary run
    unsigned long long *orand = (unsigned long long *)(t + ((kb + vb + 2 * cb + 15) & ~(size_t)15));
    unsigned long long init[3] = {0ULL, ~0ULL, 0ULL}, got[3] = {0ULL, 0ULL, 0ULL};
    CUDA_TRY(cudaMemcpyAsync(orand, init, sizeof(init), cudaMemcpyHostToDevice, st));
    k_key_bits<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1216), 256, 0, st>>>(kin, n, orand);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(got, orand, sizeof(got), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    P->launches += 1;
    // among the keys other than ~0, a digit equal in all of them leaves their
    // order unchanged.  When ~0 keys occur, one such digit whose common value
    // is below 15 also runs: there every other key is below ~0, so the ~0
    // keys still sort last.
    const unsigned long long vary = got[0] ^ got[1], common = got[1];
    const bool has_inv = got[2] != 0ULL && got[1] != ~0ULL;   // (got[1] == ~0: every key is ~0)
    int shifts[64 / RADIX_BITS], m = 0;
    bool sep = !has_inv;
    for (int pass = 0; pass < 64 / RADIX_BITS; ++pass) {
        const int sh = pass * RADIX_BITS;
        const bool varies = (vary >> sh) & (RADIX - 1);
        const bool below = ((common >> sh) & (RADIX - 1)) != (RADIX - 1);
        if (varies || (!sep && below)) {
            shifts[m++] = sh;
            if (!varies) sep = true;
        }
    }
    if (m == 0) {                                      // all keys equal: the input order is the order
        CUDA_TRY(cudaMemcpyAsync(kout, kin, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
        if (vin) CUDA_TRY(cudaMemcpyAsync(vout, vin, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        return TEFMM_OK;
    }
    // ping-pong so that the last pass writes the output
    const uint64_t *ks = kin;
    const int *vs = vin;
    for (int j = 0; j < m; ++j) {
        const bool to_out = (m - 1 - j) % 2 == 0;
        uint64_t *kd = to_out ? kout : ktmp;
        int *vd = vin ? (to_out ? vout : vtmp) : nullptr;
        k_radix_count<<<(unsigned)ntile, SORT_THREADS, 0, st>>>(ks, n, shifts[j], (int)ntile, counts);
        CUDA_TRY(cudaGetLastError());
        TRY(scan_rec(counts, offs, nc, false, dp<int>(P->scan_tmp), st));
        k_radix_scatter<<<(unsigned)ntile, SORT_THREADS, SCATTER_SMEM, st>>>(ks, vs, kd, vd, n, shifts[j],
                                                                           (int)ntile, offs);
        CUDA_TRY(cudaGetLastError());
        P->launches += 3;
        ks = kd;
        vs = vd;
    }
    return TEFMM_OK;
}

// ---- test hooks: the primitives on caller buffers (scratch from a throwaway plan record)
extern "C" int tefmm_debug_sort_u64(const uint64_t *d_keys_in, uint64_t *d_keys_out, const int *d_vals_in,
                                    int *d_vals_out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!d_keys_in || !d_keys_out || (d_vals_in && !d_vals_out)))) return TEFMM_ERR_INVALID_ARG;
    tefmm_plan_s tmp;
    const int r = dev_sort_u64(&tmp, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, (cudaStream_t)stream);
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    dbuf_free(tmp.sort_tmp);
    dbuf_free(tmp.scan_tmp);
    if (r != TEFMM_OK) return r;
    return e == cudaSuccess ? TEFMM_OK : TEFMM_ERR_CUDA;
}

extern "C" int tefmm_debug_scan_i32(const int *d_in, int *d_out, int64_t n, int inclusive, void *stream) {
    if (n < 0 || (n > 0 && (!d_in || !d_out))) return TEFMM_ERR_INVALID_ARG;
    tefmm_plan_s tmp;
    const int r = dev_scan_i32(&tmp, d_in, d_out, n, inclusive != 0, (cudaStream_t)stream);
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    dbuf_free(tmp.scan_tmp);
    if (r != TEFMM_OK) return r;
    return e == cudaSuccess ? TEFMM_OK : TEFMM_ERR_CUDA;
}
