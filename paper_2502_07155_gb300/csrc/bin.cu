// Node binning (set_nodes): cell keys, a stable LSD radix sort of (key, j),
// the sorted node copy, tile offsets and the (tile, chunk) work list.
//
// The paper has no binning step; it is how the short sums of Algorithm 4.2
// step 3 (index set J_{L,m}(x), Eq. 4.8) are made local: nodes of one tile
// share a shared-memory box of grid values.  All integer results are unique
// (the pair (key, j) is unique), so they are compared bit for bit against
// the oracle.
//
// Key of node j: i_t = floor(L_t x_t) + L_t/2 (one correctly rounded product
// in the nodes' precision), tile coordinate c_t = i_t / T_t, in-tile cell
// r_t = i_t mod T_t, key = lin(c) * prod(T) + lin(r) (row-major, dim 0
// slowest).  The sort never waits on other CTAs: block histograms, one
// exclusive scan kernel, then a block-local stable scatter.
#include <algorithm>

#include "plan_internal.h"

namespace nfftbl {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;
constexpr int kRsSeg = kRsThreads * kRsRounds;   // items per block

template <typename T>
__global__ void key_kernel(const T* __restrict__ x, long long N, TileGeom g, uint32_t* __restrict__ keys,
                           uint32_t* __restrict__ vals, int* __restrict__ err) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    uint32_t lin_c = 0, lin_r = 0;
    bool ok = true;
    for (int t = 0; t < g.d; ++t) {
        const T xv = x[i * g.d + t];
        ok = ok && (xv >= T(-0.5)) && (xv < T(0.5));     // NaN fails both
        const T u = mul_rn(static_cast<T>(g.L[t]), xv);   // exact for L = 2^p
        int c = static_cast<int>(floor(u)) + g.L[t] / 2;
        c = min(max(c, 0), g.L[t] - 1);                   // only reached for bad nodes
        lin_c = lin_c * g.nt[t] + c / g.T[t];
        lin_r = lin_r * g.T[t] + c % g.T[t];
    }
    if (!ok) atomicOr(err, DEVERR_DOMAIN);
    keys[i] = (lin_c << g.cells_per_tile_log2) | lin_r;
    vals[i] = static_cast<uint32_t>(i);
}

__global__ void rs_hist_kernel(const uint32_t* __restrict__ keys, long long N, int shift, int nblocks,
                               uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = static_cast<long long>(blockIdx.x) * kRsSeg;
    for (int r = 0; r < kRsRounds; ++r) {
        const long long i = base + r * kRsThreads + threadIdx.x;
        if (i < N) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[static_cast<long long>(threadIdx.x) * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of n uint32 in place, *total receiving the sum, in three
// launches: per-tile sums (tiles of kScanTile consecutive values), one block
// scanning the tile sums, then each tile scanned from its offset.  All loads
// are coalesced; every integer result is exact.
constexpr int kScanThreads = 256;
constexpr int kScanRounds = 16;
constexpr int kScanTile = kScanThreads * kScanRounds;

// Block-wide inclusive scan of one value per thread (kScanThreads or 1024
// threads); returns the inclusive prefix, *block_total the block's sum.
template <int NT>
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* s_warp, uint32_t& block_total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const uint32_t w = (lane < NT / 32) ? s_warp[lane] : 0u;
        uint32_t wi = w;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += u;
        }
        s_warp[lane] = wi - w;                 // exclusive prefix of the warp sums
        if (lane == 31) s_warp[32] = wi;       // block total
    }
    __syncthreads();
    const uint32_t res = incl + s_warp[wid];
    block_total = s_warp[32];
    __syncthreads();                           // s_warp is reused by the caller's next round
    return res;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_sum_kernel(const uint32_t* __restrict__ a, long long n,
                                                                     uint32_t* __restrict__ sums) {
    __shared__ uint32_t s_warp[33];
    const long long base = static_cast<long long>(blockIdx.x) * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < kScanRounds; ++r) {
        const long long i = base + r * kScanThreads + threadIdx.x;
        if (i < n) s += a[i];
    }
    uint32_t tot;
    block_incl_scan<kScanThreads>(s, s_warp, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block of 1024 threads: exclusive scan of the tile sums in rounds of
// 1024 consecutive values; *total receives the grand total.
__global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t* __restrict__ sums, long long nt,
                                                         uint32_t* __restrict__ total) {
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (long long b = 0; b < nt; b += 1024) {
        const long long i = b + threadIdx.x;
        const uint32_t v = (i < nt) ? sums[i] : 0u;
        uint32_t tot;
        const uint32_t incl = block_incl_scan<1024>(v, s_warp, tot);
        if (i < nt) sums[i] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_apply_kernel(uint32_t* __restrict__ a, long long n,
                                                                       const uint32_t* __restrict__ sums) {
    __shared__ uint32_t s_warp[33];
    const long long base = static_cast<long long>(blockIdx.x) * kScanTile;
    uint32_t run = sums[blockIdx.x];
    for (int r = 0; r < kScanRounds; ++r) {
        const long long i = base + r * kScanThreads + threadIdx.x;
        const uint32_t v = (i < n) ? a[i] : 0u;
        uint32_t tot;
        const uint32_t incl = block_incl_scan<kScanThreads>(v, s_warp, tot);
        if (i < n) a[i] = run + incl - v;
        run += tot;
    }
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Stable scatter of one 8-bit digit: items are ranked in segment order
// (round, thread); lanes with equal digits are ranked by __match_any_sync,
// warps by a per-round prefix over the 8 warps.
__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(
        const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
        uint32_t* __restrict__ vout, long long N, int shift, int nblocks, const uint32_t* __restrict__ hist) {
    constexpr int kWarps = kRsThreads / 32;
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kWarps][256];
    const int tid = threadIdx.x, warp = tid >> 5;
    run[tid] = hist[static_cast<long long>(tid) * nblocks + blockIdx.x];
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const long long base = static_cast<long long>(blockIdx.x) * kRsSeg;
    for (int r = 0; r < kRsRounds; ++r) {
        const long long i = base + r * kRsThreads + tid;
        const bool valid = i < N;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t val = valid ? vin[i] : 0u;
        const uint32_t dig = valid ? ((key >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig);
        const uint32_t rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        {
            uint32_t s = run[tid];
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = s;
                s += c;
            }
            run[tid] = s;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wcnt[warp][dig] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
    }
}

template <typename T>
__global__ void gather_nodes_kernel(const T* __restrict__ x, const uint32_t* __restrict__ perm, long long N, int d,
                                    T* __restrict__ xs) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    const long long j = perm[i];
    for (int t = 0; t < d; ++t) xs[i * d + t] = x[j * d + t];
}

// tile_off[t] = first sorted position whose tile is >= t (t = 0..n_tiles).
__global__ void tile_bounds_kernel(const uint32_t* __restrict__ keys, long long N, int shift, long long n_tiles,
                                   uint32_t* __restrict__ off) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i > N) return;
    const long long cur = (i < N) ? static_cast<long long>(keys[i] >> shift) : n_tiles;
    const long long prev = (i > 0) ? static_cast<long long>(keys[i - 1] >> shift) : -1;
    for (long long t = prev + 1; t <= cur; ++t) off[t] = static_cast<uint32_t>(i);
}

__global__ void chunk_count_kernel(const uint32_t* __restrict__ off, long long n_tiles, int K,
                                   uint32_t* __restrict__ chunks) {
    const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (t >= n_tiles) return;
    const uint32_t cnt = off[t + 1] - off[t];
    chunks[t] = (cnt + K - 1) / K;
}

__global__ void emit_work_kernel(const uint32_t* __restrict__ off, const uint32_t* __restrict__ chunk_start,
                                 long long n_tiles, int K, WorkItem* __restrict__ work) {
    const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (t >= n_tiles) return;
    const uint32_t cnt = off[t + 1] - off[t];
    const uint32_t nch = (cnt + K - 1) / K;
    for (uint32_t c = 0; c < nch; ++c) {
        WorkItem w;
        w.tile = static_cast<int>(t);
        w.start = static_cast<int>(off[t] + c * K);
        const uint32_t left = cnt - c * K;
        w.count = static_cast<int>(left < static_cast<uint32_t>(K) ? left : static_cast<uint32_t>(K));
        w.pad = 0;
        work[chunk_start[t] + c] = w;
    }
}

inline unsigned grid1d(long long n, int threads) {
    return static_cast<unsigned>((n + threads - 1) / threads);
}

// Launch the three-phase scan of a[0 .. n); sums holds ceil(n / kScanTile)
// values (at least one).
inline void scan_exclusive(uint32_t* a, long long n, uint32_t* total, uint32_t* sums, cudaStream_t s,
                           long long& launches) {
    const long long nt = std::max<long long>(1, (n + kScanTile - 1) / kScanTile);
    scan_tile_sum_kernel<<<static_cast<unsigned>(nt), kScanThreads, 0, s>>>(a, n, sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(sums, nt, total);
    scan_tile_apply_kernel<<<static_cast<unsigned>(nt), kScanThreads, 0, s>>>(a, n, sums);
    launches += 3;
}

}  // namespace

nfftbl_status bin_nodes(nfftbl_plan_s* p, long long N, const void* x_dev) {
    const bool dbl = p->precision == NFFTBL_F64;
    const size_t es = dbl ? sizeof(double) : sizeof(float);
    const int d = p->d;
    const int K = p->nodes_per_item;
    const long long Nb = std::max<long long>(N, 1);
    nfftbl_status st;
    if ((st = ensure_buf(p, p->keys, Nb * 4)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->perm, Nb * 4)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->keys_tmp, Nb * 4)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->perm_tmp, Nb * 4)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->xs, Nb * d * es)) != NFFTBL_OK) return st;
    const long long nblocks = std::max<long long>(1, (N + kRsSeg - 1) / kRsSeg);
    if ((st = ensure_buf(p, p->hist, 256 * nblocks * 4)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->tile_off, (p->n_tiles + 1) * 4)) != NFFTBL_OK) return st;
    const long long scan_n = std::max<long long>(256 * nblocks, p->n_tiles);
    if ((st = ensure_buf(p, p->scan_tmp, ((scan_n + kScanTile - 1) / kScanTile + 1) * 4)) != NFFTBL_OK) return st;
    uint32_t* scan_sums = static_cast<uint32_t*>(p->scan_tmp.p);
    // counters: [0] scan total of the radix sort; tile_items: first work item per tile
    if ((st = ensure_buf(p, p->counters, 16)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->tile_items, (p->n_tiles + 1) * 4)) != NFFTBL_OK) return st;
    const long long max_work = (N + K - 1) / K + p->n_tiles + 1;
    if ((st = ensure_buf(p, p->work, max_work * sizeof(WorkItem))) != NFFTBL_OK) return st;

    cudaStream_t s = p->stream;
    int* err = static_cast<int*>(p->err.p);
    if ((st = check_cuda(p, cudaMemsetAsync(err, 0, sizeof(int), s), "memset err")) != NFFTBL_OK) return st;

    uint32_t* kA = static_cast<uint32_t*>(p->keys.p);
    uint32_t* vA = static_cast<uint32_t*>(p->perm.p);
    uint32_t* kB = static_cast<uint32_t*>(p->keys_tmp.p);
    uint32_t* vB = static_cast<uint32_t*>(p->perm_tmp.p);
    timing_begin(p, NFFTBL_K_BIN);   // one timed span for the whole binning sequence
    if (N > 0) {
        if (dbl)
            key_kernel<double><<<grid1d(N, 256), 256, 0, s>>>(static_cast<const double*>(x_dev), N, p->geom, kA,
                                                             vA, err);
        else
            key_kernel<float><<<grid1d(N, 256), 256, 0, s>>>(static_cast<const float*>(x_dev), N, p->geom, kA, vA,
                                                            err);
        p->launches++;
        uint32_t* hist = static_cast<uint32_t*>(p->hist.p);
        uint32_t* total = static_cast<uint32_t*>(p->counters.p);
        for (int shift = 0; shift < p->key_bits; shift += 8) {
            rs_hist_kernel<<<static_cast<unsigned>(nblocks), 256, 0, s>>>(kA, N, shift, static_cast<int>(nblocks),
                                                                          hist);
            scan_exclusive(hist, 256 * nblocks, total, scan_sums, s, p->launches);
            rs_scatter_kernel<<<static_cast<unsigned>(nblocks), kRsThreads, 0, s>>>(
                kA, vA, kB, vB, N, shift, static_cast<int>(nblocks), hist);
            p->launches += 2;
            std::swap(kA, kB);
            std::swap(vA, vB);
        }
        // keep the sorted result in p->keys / p->perm
        if (kA != p->keys.p) {
            std::swap(p->keys, p->keys_tmp);
            std::swap(p->perm, p->perm_tmp);
        }
        kA = static_cast<uint32_t*>(p->keys.p);
        vA = static_cast<uint32_t*>(p->perm.p);
        if (dbl)
            gather_nodes_kernel<double><<<grid1d(N, 256), 256, 0, s>>>(static_cast<const double*>(x_dev), vA, N, d,
                                                                      static_cast<double*>(p->xs.p));
        else
            gather_nodes_kernel<float><<<grid1d(N, 256), 256, 0, s>>>(static_cast<const float*>(x_dev), vA, N, d,
                                                                     static_cast<float*>(p->xs.p));
        p->launches++;
    }
    uint32_t* off = static_cast<uint32_t*>(p->tile_off.p);
    tile_bounds_kernel<<<grid1d(N + 1, 256), 256, 0, s>>>(kA, N, p->geom.cells_per_tile_log2, p->n_tiles, off);
    uint32_t* chunk_start = static_cast<uint32_t*>(p->tile_items.p);
    uint32_t* work_total = chunk_start + p->n_tiles;
    chunk_count_kernel<<<grid1d(p->n_tiles, 256), 256, 0, s>>>(off, p->n_tiles, K, chunk_start);
    scan_exclusive(chunk_start, p->n_tiles, work_total, scan_sums, s, p->launches);
    emit_work_kernel<<<grid1d(p->n_tiles, 256), 256, 0, s>>>(off, chunk_start, p->n_tiles, K,
                                                             static_cast<WorkItem*>(p->work.p));
    p->launches += 3;
    timing_end(p);
    if ((st = check_cuda(p, cudaGetLastError(), "binning launch")) != NFFTBL_OK) return st;
    uint32_t host_total = 0;
    if ((st = check_cuda(p, cudaMemcpyAsync(&host_total, work_total, 4, cudaMemcpyDeviceToHost, s), "read work total")) !=
        NFFTBL_OK)
        return st;
    if ((st = check_cuda(p, cudaMemcpyAsync(p->err_host, err, sizeof(int), cudaMemcpyDeviceToHost, s), "read err")) !=
        NFFTBL_OK)
        return st;
    if ((st = check_cuda(p, cudaStreamSynchronize(s), "set_nodes sync")) != NFFTBL_OK) return st;
    if (*p->err_host & DEVERR_DOMAIN) {
        p->N = -1;
        p->n_work = 0;
        return fail(p, NFFTBL_EDOMAIN, "a node coordinate is outside [-1/2, 1/2) or NaN");
    }
    if (host_total > static_cast<uint32_t>(max_work)) return fail(p, NFFTBL_EINTERNAL, "work list overflow");
    // scratch for the spread boxes: one slot per (work item, batch entry)
    long long cells = 1;
    for (int t = 0; t < d; ++t) cells *= p->geom.box[t];
    const size_t cb = dbl ? 16 : 8;
    if ((st = ensure_buf(p, p->part, static_cast<size_t>(std::max<uint32_t>(host_total, 1)) * p->batch * cells * cb)) !=
        NFFTBL_OK) {
        p->N = -1;
        return st;
    }
    p->n_work = host_total;
    p->N = N;
    return NFFTBL_OK;
}

}  // namespace nfftbl
