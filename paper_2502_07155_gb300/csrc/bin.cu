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

// Same-cell pairs for the interpolation: one warp per work item walks the
// item's sorted keys 32 at a time.  Node j at position r of its run of equal
// keys (nodes of one cell) is a pair head when r is even; its partner is
// node j + 1 when that node is in the same run and in the same item.  The
// heads of an item are written in order to heads[start ..), each as the
// node's sorted index with bit 31 set when it has a partner; nheads[item]
// counts them.  Every node is a head or the partner of the head before it.
__global__ void pair_heads_kernel(const uint32_t* __restrict__ keys, const WorkItem* __restrict__ work, int n_work,
                                  uint32_t* __restrict__ heads, uint32_t* __restrict__ nheads) {
    const unsigned full = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < n_work; item += gridDim.x * wpb) {
        const WorkItem wi = work[item];
        uint32_t prev_key = 0xFFFFFFFFu;   // keys are < 2^31: differs from every key
        int prev_pos = -1;
        int out = 0;
        for (int base = 0; base < wi.count; base += 32) {
            const int j = base + lane;
            const bool valid = j < wi.count;
            const uint32_t key = valid ? keys[wi.start + j] : 0xFFFFFFFEu;
            uint32_t up = __shfl_up_sync(full, key, 1);
            if (lane == 0) up = prev_key;
            const bool start = valid && key != up;
            const unsigned sb = __ballot_sync(full, start);
            const unsigned le = sb & ((lane == 31) ? full : ((2u << lane) - 1u));
            const int pos = le ? lane - (31 - __clz(static_cast<int>(le))) : prev_pos + 1 + lane;
            uint32_t dn = __shfl_down_sync(full, key, 1);
            if (lane == 31) dn = (j + 1 < wi.count) ? keys[wi.start + j + 1] : 0xFFFFFFFDu;
            const bool head = valid && (pos & 1) == 0;
            const bool paired = head && j + 1 < wi.count && dn == key;
            const unsigned hb = __ballot_sync(full, head);
            if (head)
                heads[wi.start + out + __popc(hb & ((1u << lane) - 1u))] =
                    static_cast<uint32_t>(wi.start + j) | (paired ? 0x80000000u : 0u);
            out += __popc(hb);
            prev_key = __shfl_sync(full, key, 31);
            prev_pos = __shfl_sync(full, pos, 31);
        }
        if (lane == 0) nheads[item] = static_cast<uint32_t>(out);
    }
}

// Order of the pair heads inside each d = 3 work item, against shared-memory
// bank conflicts of the interpolation: the 8-byte box value a head loads at
// tap (a, b, c) lies in bank pair (base + a p0 + b p1 + c) mod 16, base =
// lb0 p0 + lb1 p1 + lb2 the offset of its first tap, and the tap offsets are
// the same for every thread.  Heads of different base classes (mod 16) never
// conflict.  The heads are dealt class by class: all first heads of each
// class in class order, then all second heads, ..., so that consecutive
// heads (one per thread of a half warp) have distinct classes as far as the
// item's classes allow.  One warp per item; counts per class in shared
// memory.
__global__ void order_heads_kernel(const uint32_t* __restrict__ keys, const WorkItem* __restrict__ work, int n_work,
                                   const uint32_t* __restrict__ in_heads, const uint32_t* __restrict__ nheads,
                                   TileGeom g, int m, uint32_t* __restrict__ out_heads) {
    constexpr int kWarps = 8;
    __shared__ uint32_t cnt[kWarps][16], run[kWarps][16];
    const unsigned full = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p1 = g.box[2], p0 = g.box[1] * p1;
    auto cls_of = [&](uint32_t key) {
        const int lin = static_cast<int>(key & ((1u << g.cells_per_tile_log2) - 1u));
        const int l2 = lin % g.T[2], l1 = (lin / g.T[2]) % g.T[1], l0 = lin / (g.T[2] * g.T[1]);
        const int base = (l0 + g.off[0] - (m - 1)) * p0 + (l1 + g.off[1] - (m - 1)) * p1 + (l2 + g.off[2] - (m - 1));
        return base & 15;
    };
    for (int item = blockIdx.x * kWarps + w; item < n_work; item += gridDim.x * kWarps) {
        const WorkItem wi = work[item];
        const int nh = static_cast<int>(nheads[item]);
        if (lane < 16) {
            cnt[w][lane] = 0;
            run[w][lane] = 0;
        }
        __syncwarp();
        for (int base = 0; base < nh; base += 32) {
            const int h = base + lane;
            if (h < nh) atomicAdd(&cnt[w][cls_of(keys[in_heads[wi.start + h] & 0x7FFFFFFFu])], 1u);
        }
        __syncwarp();
        for (int base = 0; base < nh; base += 32) {
            const int h = base + lane;
            const bool valid = h < nh;
            const uint32_t hv = valid ? in_heads[wi.start + h] : 0u;
            const int cls = valid ? cls_of(keys[hv & 0x7FFFFFFFu]) : 16 + lane;   // (unique when invalid)
            const unsigned peers = __match_any_sync(full, cls);
            const unsigned before = peers & ((1u << lane) - 1u);
            if (valid) {
                const uint32_t r = run[w][cls] + __popc(before);
                uint32_t pos = 0;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const uint32_t n = cnt[w][c];
                    pos += min(n, r) + ((c < cls && n > r) ? 1u : 0u);
                }
                out_heads[wi.start + pos] = hv;
            }
            __syncwarp();
            if (valid && before == 0) run[w][cls] += __popc(peers);
            __syncwarp();
        }
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
    // FP32 d = 3: the spreading's input gathered into sorted node order
    if (d == 3 && !dbl && p->batch == 1 && (st = ensure_buf(p, p->fsorted, Nb * 8)) != NFFTBL_OK) {
        p->N = -1;
        return st;
    }
    // same-cell pairs of the interpolation (heads per item)
    if ((st = ensure_buf(p, p->heads, Nb * 4)) != NFFTBL_OK || (st = ensure_buf(p, p->nheads,
                                                                                std::max<uint32_t>(host_total, 1) * 4)) != NFFTBL_OK) {
        p->N = -1;
        return st;
    }
    if (host_total > 0) {
        const unsigned blocks = static_cast<unsigned>(std::min<long long>((host_total + 7) / 8, 8LL * p->num_sms));
        // d = 3: heads in sorted order into the (now free) sort scratch, then dealt by bank class
        const bool deal = d == 3;
        uint32_t* first = deal ? static_cast<uint32_t*>(p->keys_tmp.p) : static_cast<uint32_t*>(p->heads.p);
        pair_heads_kernel<<<blocks, 256, 0, s>>>(kA, static_cast<const WorkItem*>(p->work.p),
                                                 static_cast<int>(host_total), first,
                                                 static_cast<uint32_t*>(p->nheads.p));
        p->launches++;
        if (deal) {
            order_heads_kernel<<<blocks, 256, 0, s>>>(kA, static_cast<const WorkItem*>(p->work.p),
                                                      static_cast<int>(host_total), first,
                                                      static_cast<const uint32_t*>(p->nheads.p), p->geom, p->m,
                                                      static_cast<uint32_t*>(p->heads.p));
            p->launches++;
        }
        if ((st = check_cuda(p, cudaGetLastError(), "pair heads launch")) != NFFTBL_OK) {
            p->N = -1;
            return st;
        }
    }
    p->n_work = host_total;
    p->N = N;
    return NFFTBL_OK;
}

}  // namespace nfftbl
