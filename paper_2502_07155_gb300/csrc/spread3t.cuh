// d = 3 spreading on the tensor cores (FP32 plans, 8 x 8 x 8 tiles, W = 2m).
//
// A work item's box receives, from each of its nodes j, the tensor product
// g_j w0_j (x) w1_j (x) w2_j (Eq. 4.11 transposed).  Written with the box's
// dimensions 1 and 2 as rows and dimension 0 (with the real and imaginary
// part) as columns, the item's box is one matrix product over its nodes:
//
//   box[(i1, i2), (i0, c)] = sum_j  A[(i1, i2), j] * B[j, (i0, c)],
//   A[(i1, i2), j] = w1_j[i1] w2_j[i2],   B[j, (i0, c)] = (g_j w0_j[i0])_c,
//
// with every factor zero outside the node's 2m taps.  The rows go in M tiles
// of 128 (tcgen05 MMA, cta_group::1, kind::tf32), the columns are one N of
// 2R padded to a multiple of 16, and the nodes are the K dimension, eight
// per MMA (a "stage").  FP32 accuracy from TF32 operands: each operand is
// split into its TF32 rounding and the remainder, a = a_hi + a_lo, and the
// product is a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped a_lo b_lo is
// below FP32 rounding).  The tensor core accumulates at most RO stages
// (3 RO MMAs per output; RO = 16, or 32 at m >= 7) before the accumulator is
// added, in FP32 with round-to-nearest, into a box in shared memory: longer
// chains of accumulations inside the tensor core drift measurably at the
// dense centre of a spoke workload (a million contributions to a cell).
//
// Warp roles (21 warps):
//  - three producer groups of four warps; group g builds the stages S with
//    S mod 3 = g into stage buffer g: node parameters, the stage's window
//    values per box position (node-minor tables, zero outside each node's
//    taps), then A (hi, lo) into tensor memory with tcgen05.st (warp q of
//    the group writes lanes 32q .. 32q+31 of every M tile) and B (hi, lo)
//    into shared memory in the no-swizzle K-major layout;
//  - one MMA warp: its elected thread issues the stage's 3 x (M tiles) MMAs
//    and commits them to the buffer's "empty" barrier, and to "dfull" after
//    the last stage of a segment (at most RO stages of one item);
//  - one readout group of eight warps: after each segment it adds the
//    accumulator into the shared box, and after an item's last segment it
//    copies the box to the item's slot of the ordered flush (gather_kernel).
//
// Every wait is bounded; after a wait runs out the block sets the error
// flag and a shared abort word that makes every later wait return at once,
// so all threads still reach every barrier and the block ends.

template <int W>
struct Spread3T {
    static constexpr int T = 8;                          // tile extent, every dimension
    static constexpr int R = T + W - 1;                  // box extent, dimension 0
    static constexpr int B1 = T + W - 1;                 // box extent, dimension 1
    static constexpr int B2 = T + W;                     // box extent, dimension 2 (even origin)
    static constexpr int ROWS = B1 * B2;                 // GEMM rows
    static constexpr int NT = (ROWS + 127) / 128;        // M tiles of 128 rows
    static constexpr int NP = (2 * R + 15) / 16 * 16;    // GEMM columns (i0, re/im), padded
    static constexpr int KS = 8;                         // nodes per stage (one K step)
    static constexpr int NG = 3;                         // producer groups = stage buffers
    // accumulators: two where tensor memory holds them (m <= 6), so that the
    // readout of one segment overlaps the MMAs of the next
    static constexpr int ND = W <= 12 ? 2 : 1;
    // stages per accumulator segment: 16, or 32 at m >= 7, where the single
    // accumulator waits for every readout (chains of 3 RO MMAs per output;
    // the error they leave at the densest spoke cells grows with RO)
    static constexpr int RO = W >= 14 ? 32 : 8;
    static constexpr int COL_A = ND * NT * NP;           // tensor-memory columns: accumulators first
    static constexpr int A_COLS = 2 * NT * KS;           // A hi and lo of one stage
    static constexpr int COLS_USED = COL_A + NG * A_COLS;
    static constexpr int TCOLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                                 : COLS_USED <= 256 ? 256 : 512;
    static constexpr int RDW = 8;                        // readout warps (two per lane quarter)
    static constexpr int WARPS = 4 * NG + RDW + 1;       // producers, readout, MMA
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int RD_WARP = 4 * NG;               // first readout warp
    static constexpr int MMA_WARP = 4 * NG + RDW;
    // stage table (floats, node-minor): w1 [B1][KS], w2 [B2][KS]; the dimension-0
    // values go straight into the stage's B operand
    static constexpr int T1 = 0, T2 = B1 * KS, TAB = T2 + B2 * KS;
    static constexpr int NPAR = 12;                      // node parameters: tau[3], s[3], lb[3], g.x, g.y, pad
    static constexpr int BST = 2 * NP * KS;              // B of one stage (hi, then lo), floats
    static constexpr int BOX = R * B1 * B2;              // box cells (float2)
    // shared memory (bytes)
    static constexpr size_t OFF_TAB = static_cast<size_t>(BOX) * 8;
    static constexpr size_t OFF_PAR = OFF_TAB + static_cast<size_t>(NG) * 2 * TAB * 4;
    static constexpr size_t OFF_B = (OFF_PAR + static_cast<size_t>(NG) * 2 * KS * NPAR * 4 + 127) / 128 * 128;
    static constexpr size_t OFF_BAR = (OFF_B + static_cast<size_t>(2 * NG) * BST * 4 + 127) / 128 * 128;
    static constexpr size_t BYTES = OFF_BAR + 8 * (2 * NG + 2 * ND + 1) + 16;
    // at least 116 KB: one block per SM, the tensor-memory allocation never waits on another block
    static constexpr size_t SMEM = BYTES > 116 * 1024 ? BYTES : 116 * 1024;
    static_assert(COLS_USED <= 512, "tensor memory holds 512 columns");
    static_assert(NP <= 256 && NP % 16 == 0, "MMA N for M = 128");
    static_assert(NT * 128 >= ROWS, "M tiles cover the rows");
    static_assert(BOX % 2 == 0 && (TAB * 4) % 16 == 0 && (T2 * 4) % 16 == 0 && (BST * 4) % 16 == 0, "alignment");
};

// ---- tcgen05 / tensor-memory helpers (sm_100 family PTX) -------------------

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Two consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tmem_st2(uint32_t taddr, float v0, float v1) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(__float_as_uint(v0)),
                 "r"(__float_as_uint(v1))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Four consecutive 32-bit columns of this thread's lane, waited for in the
// same statement (no use of the registers can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r0, r1, r2, r3;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(taddr)
        : "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
}

// D (tensor memory) (+)= A (tensor memory) * B (shared memory, descriptor).
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The barrier receives one arrival when every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void named_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ float tf32_round(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, no negation or sparsity, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: core matrices of 8 rows x 16
// bytes stored contiguously; lbo = byte step between core matrices along K,
// sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc_noswz(const void* p, uint32_t lbo, uint32_t sbo) {
    uint64_t d = static_cast<uint64_t>((smem_addr(p) >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;   // descriptor version of the sm_100 family
    return d;
}

// Bounded wait that also gives up at once when another thread of the block
// has already given up (abort word set).
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort, int* err,
                                              unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > limit_ns) {
            *abort = 1;
            atomicOr(err, DEVERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

// Eight consecutive 32-bit columns of this thread's lane (waited for in the
// same statement).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// Sixteen consecutive 32-bit columns of this thread's lane (waited for in
// the same statement).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// The 2m window values of every (node, dimension) of a stage, weight kind
// WKC fixed at compile time: dimensions 1 and 2 into the stage table at their
// box positions, dimension 0 times the node's input value into B (hi, lo);
// thread gt of the producer group takes every 128th entry.
template <int W, int WKC>
__device__ __forceinline__ void spread3t_entries(const TapArgs<float>& a, const float* par, float* tab, float* bh,
                                                 int gt) {
    using G = Spread3T<W>;
    constexpr int m = W / 2;
    for (int e = gt; e < 3 * G::KS * W; e += 128) {
        const int tap = e % W, kt = e / W, t = kt / G::KS, k = kt - t * G::KS;
        const float* pp = par + k * G::NPAR;
        const int lb = __float_as_int(pp[6 + t]);
        if (lb >= 0) {   // (no node: lb = -1000)
            const float w = fast_weight<float, WKC>(pp[t], pp[3 + t], tap, m, a.w);
            const int pos = lb + tap;
            if (t == 0) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float v = pp[9 + c] * w;
                    const float h = tf32_round(v);
                    const int n = 2 * pos + c;
                    const int off = (n >> 3) * 64 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
                    bh[off] = h;
                    bh[G::NP * G::KS + off] = v - h;
                }
            } else {
                tab[(t == 1 ? G::T1 : G::T2) + pos * G::KS + k] = w;
            }
        }
    }
}

template <int W>
__global__ void __launch_bounds__(Spread3T<W>::THREADS, 1) spread3t_kernel(const TapArgs<float> a) {
    using G = Spread3T<W>;
    constexpr int m = W / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* s_box = reinterpret_cast<float2*>(smem);
    float* s_tab = reinterpret_cast<float*>(smem + G::OFF_TAB);
    float* s_par = reinterpret_cast<float*>(smem + G::OFF_PAR);
    float* s_b = reinterpret_cast<float*>(smem + G::OFF_B);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);   // [NG], 128 arrivals
    uint64_t* empty = full + G::NG;                                     // [NG], one commit
    uint64_t* dfull = empty + G::NG;                                    // [ND] segment accumulated (commit)
    uint64_t* dempty = dfull + G::ND;                                   // [ND] segment read (readout arrivals)
    uint64_t* fin = dempty + G::ND;                                     // final drain (commit)
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wk = weight_kind(a.w);
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    constexpr uint32_t kIdesc = idesc_tf32(128, G::NP);

    if (tid == 0) {
        for (int b = 0; b < G::NG; ++b) {
            mbar_init(&full[b], 128);
            mbar_init(&empty[b], 1);
        }
        for (int b = 0; b < G::ND; ++b) {
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], 32 * G::RDW);
        }
        mbar_init(fin, 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    if (warp == G::MMA_WARP) {   // the MMA warp owns the tensor memory
        tmem_alloc(s_tmem, G::TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *s_tmem;

    if (warp == G::MMA_WARP) {
        // ---------------- MMA warp: one elected thread issues every MMA
        if (lane == 0) {
            bool issued = false;
            long long S = 0;   // stage counter
            int seg = 0;       // segment counter
            for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
                const int ns = max(1, (a.work[item].count + G::KS - 1) / G::KS);
                for (int s = 0; s < ns; ++s, ++S) {
                    const int b = static_cast<int>(S % G::NG);
                    const bool first = (s % G::RO) == 0, last = (s % G::RO) == G::RO - 1 || s == ns - 1;
                    bool ok = wait_or_abort(&full[b], static_cast<uint32_t>((S / G::NG) & 1), s_abort, a.err, a.wait_ns);
                    if (ok && first && seg >= G::ND)   // the accumulator's previous segment has been read
                        ok = wait_or_abort(&dempty[seg % G::ND], static_cast<uint32_t>((seg / G::ND - 1) & 1), s_abort,
                                           a.err, a.wait_ns);
                    if (ok) {
                        tc_fence_after();
                        const float* bh = s_b + static_cast<size_t>(2 * b + ((S / G::NG) & 1)) * G::BST;
                        const uint64_t dh = smem_desc_noswz(bh, 128, 256);
                        const uint64_t dl = smem_desc_noswz(bh + G::NP * G::KS, 128, 256);
#pragma unroll 1
                        for (int t = 0; t < G::NT; ++t) {
                            const uint32_t d = tbase + static_cast<uint32_t>(((seg % G::ND) * G::NT + t) * G::NP);
                            const uint32_t ah = tbase + static_cast<uint32_t>(G::COL_A + b * G::A_COLS + t * G::KS);
                            const uint32_t al = ah + static_cast<uint32_t>(G::NT * G::KS);
                            mma_tf32_ts(d, ah, dh, kIdesc, first ? 0u : 1u);
                            mma_tf32_ts(d, ah, dl, kIdesc, 1u);
                            mma_tf32_ts(d, al, dh, kIdesc, 1u);
                        }
                        issued = true;
                        mma_commit(&empty[b]);
                        if (last) mma_commit(&dfull[seg % G::ND]);
                    }
                    if (last) ++seg;
                }
            }
            if (issued) {   // nothing may still run on the tensor memory when it is freed
                mma_commit(fin);
                mbar_wait_bounded(fin, 0, a.err, a.wait_ns);
            }
        }
        __syncwarp();
    } else if (warp >= G::RD_WARP) {
        // ---------------- readout group: accumulator segments into the shared box; warp
        // (quarter q, half h) reads the lanes of quarter q and the 8-column chunks h, h + 2, ...
        const int q = warp & 3, h = (warp - G::RD_WARP) >> 2, rt = tid - 32 * G::RD_WARP;
        const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * q) << 16);
        int seg = 0;
        for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
            const int ns = max(1, (a.work[item].count + G::KS - 1) / G::KS);
            const int nseg = (ns + G::RO - 1) / G::RO;
            for (int sg = 0; sg < nseg; ++sg, ++seg) {
                const int db = seg % G::ND;
                wait_or_abort(&dfull[db], static_cast<uint32_t>((seg / G::ND) & 1), s_abort, a.err, a.wait_ns);
                tc_fence_after();
#pragma unroll 1
                for (int t = 0; t < G::NT; ++t) {
                    const int r = 128 * t + 32 * q + lane;
                    const int i1 = r / G::B2, i2 = r - (r / G::B2) * G::B2;
#pragma unroll 1
                    for (int c0 = 8 * h; c0 < G::NP; c0 += 16) {
                        float v[8];
                        tmem_ld8(lane_base + static_cast<uint32_t>((db * G::NT + t) * G::NP + c0), v);
                        if (r < G::ROWS) {
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int i0 = c0 / 2 + u;
                                if (i0 < G::R) {
                                    float2* cell = s_box + (i0 * G::B1 + i1) * G::B2 + i2;
                                    const float2 x = make_float2(v[2 * u], v[2 * u + 1]);
                                    *cell = (sg == 0) ? x : __fadd2_rn(*cell, x);
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&dempty[db]);
            }
            // the item's box into its slot of the ordered flush
            named_sync(1 + G::NG, 32 * G::RDW);
            const float4* src = reinterpret_cast<const float4*>(s_box);
            float4* dst = reinterpret_cast<float4*>(a.part + static_cast<long long>(item) * G::BOX);
            for (int idx = rt; idx < G::BOX / 2; idx += 32 * G::RDW) dst[idx] = src[idx];
            named_sync(1 + G::NG, 32 * G::RDW);
        }
    } else {
        // ---------------- producer group grp: stages S with S mod NG = grp
        const int grp = warp >> 2, q = warp & 3, gt = tid - 128 * grp;   // group, lane quarter, thread of the group
        const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * q) << 16);
        // the group's stages in order; thread gt < 3 KS holds the coordinate (node
        // gt / 3, dimension gt mod 3) and, for dimension 0, the input value of the
        // next stage, loaded one stage ahead
        struct StageRef {
            int item, s, ns, start, count, org;   // org: this thread's dimension's box origin
            long long S0;                          // first global stage of the item
        };
        const int pk = gt / 3, pt = gt - 3 * (gt / 3);
        auto first_of = [&](int item, long long S0, StageRef& r) {
            while (item < a.n_work) {
                const WorkItem wi = a.work[item];
                const int ns = max(1, (wi.count + G::KS - 1) / G::KS);
                const int s0 = static_cast<int>(((grp - S0) % G::NG + G::NG) % G::NG);
                if (s0 < ns) {
                    int org[3] = {0, 0, 0};
                    tile_origin<3>(a.g, wi.tile, periodic, org);
                    r = {item, s0, ns, static_cast<int>(wi.start), wi.count, pt == 0 ? org[0] : pt == 1 ? org[1] : org[2],
                         S0};
                    return;
                }
                S0 += ns;
                item += gridDim.x;
            }
            r = {a.n_work, 0, 0, 0, 0, 0, S0};
        };
        auto next_of = [&](const StageRef& c, StageRef& r) {
            if (c.s + G::NG < c.ns) {
                r = c;
                r.s += G::NG;
            } else {
                first_of(c.item + gridDim.x, c.S0 + c.ns, r);
            }
        };
        float px = 0.0f;
        float2 pg = make_float2(0.0f, 0.0f);
        auto prefetch = [&](const StageRef& r) {
            const int c = r.s * G::KS + pk;
            if (gt < 3 * G::KS && r.item < a.n_work && c < r.count) {
                const long long i = static_cast<long long>(r.start) + c;
                px = a.xs[i * 3 + pt];
                if (pt == 0) pg = a.fsorted[i];
            }
        };
        // clear a stage's table (dimensions 1, 2) and B (hi, lo) of this group
        auto clear_stage = [&](int buf) {
            float4* t4 = reinterpret_cast<float4*>(s_tab + static_cast<size_t>(grp * 2 + buf) * G::TAB);
            for (int idx = gt; idx < G::TAB / 4; idx += 128) t4[idx] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float4* b4 = reinterpret_cast<float4*>(s_b + static_cast<size_t>(2 * grp + buf) * G::BST);
            for (int idx = gt; idx < G::BST / 4; idx += 128) b4[idx] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        };
        int tb = 0;
        StageRef cur;
        first_of(blockIdx.x, 0, cur);
        prefetch(cur);
        clear_stage(0);
        while (cur.item < a.n_work) {
            const long long S = cur.S0 + cur.s;
            float* par = s_par + static_cast<size_t>(grp * 2 + tb) * G::KS * G::NPAR;
            float* tab = s_tab + static_cast<size_t>(grp * 2 + tb) * G::TAB;
            // node parameters (lb = -1000 marks no node), from the prefetched values
            if (gt < 3 * G::KS) {
                float* pp = par + pk * G::NPAR;
                if (cur.s * G::KS + pk < cur.count) {
                    const int Lt = pt == 0 ? a.g.L[0] : pt == 1 ? a.g.L[1] : a.g.L[2];
                    const float u = mul_rn(static_cast<float>(Lt), px);
                    const float fl = FM<float>::flr(u);
                    const float tau = u - fl;
                    const int lb = static_cast<int>(fl) + Lt / 2 - (m - 1) - cur.org;
                    pp[pt] = tau;
                    pp[3 + pt] = (wk == WK_SINH)    ? kind_sin<float, WK_SINH>(tau, a.w)
                                 : (wk == WK_TABLE) ? kind_sin<float, WK_TABLE>(tau, a.w)
                                                    : 0.0f;
                    pp[6 + pt] = __int_as_float(lb);
                    if (pt == 0) {
                        pp[9] = pg.x;
                        pp[10] = pg.y;
                    }
                } else {
                    pp[pt] = 0.0f;
                    pp[3 + pt] = 0.0f;
                    pp[6 + pt] = __int_as_float(-1000);
                    if (pt == 0) pp[9] = pp[10] = 0.0f;
                }
            }
            named_sync(1 + grp, 128);
            // the 2m window values of every (node, dimension): dimensions 1 and 2 into
            // the table at their box positions, dimension 0 times the input value
            // into B (hi, lo); every other entry was cleared beforehand
            float* bh = s_b + static_cast<size_t>(2 * grp + tb) * G::BST;
            if (wk == WK_SINH) spread3t_entries<W, WK_SINH>(a, par, tab, bh, gt);
            else if (wk == WK_CSINH) spread3t_entries<W, WK_CSINH>(a, par, tab, bh, gt);
            else if (wk == WK_TABLE) spread3t_entries<W, WK_TABLE>(a, par, tab, bh, gt);
            else spread3t_entries<W, WK_POLY>(a, par, tab, bh, gt);
            named_sync(1 + grp, 128);
            StageRef nxt;
            next_of(cur, nxt);
            prefetch(nxt);   // (consumed at the next stage: the loads overlap this stage's build)
            if (S >= G::NG)
                wait_or_abort(&empty[grp], static_cast<uint32_t>(((S / G::NG) - 1) & 1), s_abort, a.err, a.wait_ns);
            tc_fence_after();
            // the group's other buffers (its previous stage's, whose MMAs are done) cleared for its next stage
            clear_stage(tb ^ 1);
            // A = w1[i1] w2[i2] for the stage's eight nodes, hi and lo
            const uint32_t col = static_cast<uint32_t>(G::COL_A + grp * G::A_COLS);
#pragma unroll
            for (int t = 0; t < G::NT; ++t) {
                const int r = 128 * t + 32 * q + lane;
                const bool in = r < G::ROWS;
                const int i1 = in ? r / G::B2 : 0, i2 = in ? r - (r / G::B2) * G::B2 : 0;
                const float4* p1 = reinterpret_cast<const float4*>(tab + G::T1 + i1 * G::KS);
                const float4* p2 = reinterpret_cast<const float4*>(tab + G::T2 + i2 * G::KS);
                const float4 x0 = p1[0], x1 = p1[1], y0 = p2[0], y1 = p2[1];
                float2 av[4] = {__fmul2_rn(make_float2(x0.x, x0.y), make_float2(y0.x, y0.y)),
                                __fmul2_rn(make_float2(x0.z, x0.w), make_float2(y0.z, y0.w)),
                                __fmul2_rn(make_float2(x1.x, x1.y), make_float2(y1.x, y1.y)),
                                __fmul2_rn(make_float2(x1.z, x1.w), make_float2(y1.z, y1.w))};
                float hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 v = in ? av[u] : make_float2(0.0f, 0.0f);
                    const float2 h = make_float2(tf32_round(v.x), tf32_round(v.y));
                    const float2 l = __ffma2_rn(h, make_float2(-1.0f, -1.0f), v);   // v - h, exact
                    hi[2 * u] = h.x;
                    hi[2 * u + 1] = h.y;
                    lo[2 * u] = l.x;
                    lo[2 * u + 1] = l.y;
                }
                tmem_st8(lane_base + col + static_cast<uint32_t>(t * G::KS), hi);
                tmem_st8(lane_base + col + static_cast<uint32_t>((G::NT + t) * G::KS), lo);
            }
            tmem_wait_st();
            fence_async_shared();
            tc_fence_before();
            mbar_arrive(&full[grp]);
            tb ^= 1;
            cur = nxt;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == G::MMA_WARP) tmem_dealloc(tbase, G::TCOLS);
}

// The spreading's input in sorted node order: out[i] = fin[perm[i]] (one
// gather per adjoint call, so that spread3t_kernel's node loads are
// contiguous and independent).
static __global__ void __launch_bounds__(256) sort_inputs_kernel(const float2* __restrict__ fin,
                                                          const uint32_t* __restrict__ perm, float2* __restrict__ out,
                                                          long long N) {
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < N; i += static_cast<long long>(gridDim.x) * 256)
        out[i] = fin[perm[i]];
}
