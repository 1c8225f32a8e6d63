// Host-side plan object and the launchers each translation unit provides.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nfftbl.h"
#include "common.cuh"

namespace nfftbl {

// Parameters of the window / kernel evaluation, shared by all tap kernels.
template <typename T>
struct WinParams {
    int method;        // NFFTBL_SHANNON / NFFTBL_CLASSIC
    int window;        // nfftbl_window
    int m;
    T inv_m;           // 1/m
    T beta;
    T c_exp;           // beta / ln 2 (sinh window, exp2 form)
    T c_norm;          // 1 / (1 - e^{-2 beta}) (sinh) or 1/(I0(beta) - 1) (cKB)
    const T* table;    // window table on u in [0, 1] (table window), device
    int table_n;       // number of intervals (table has table_n + 1 values)
    const float4* tcoef;   // FP32 plans: per interval the Catmull-Rom cubic c0 + c1 t + c2 t^2 + c3 t^3
    // FP32 plans with a compile-time truncation: tap a's weight as a
    // polynomial in t = 2 tau - 1 of degree kPolyDeg (coefficients of t^0 ..
    // t^kPolyDeg), fitted on the host; for windows with a square-root edge
    // (sinh, Kaiser-Bessel) the edge taps' polynomial is multiplied by
    // sqrt(1 - (delta/m)^2).  poly = 0: the window's closed form instead.
    int poly;
    int poly_edge_sqrt;
    float pc[16][12];
};

constexpr int kPolyDeg = 10;   // degree of the per-tap weight polynomials
// Largest tolerated error of a fitted tap weight, FP32 evaluation included,
// relative to the largest weight: above it the plan keeps the closed form.
constexpr double kPolyTol = 3e-7;

// Geometry of the node tiles and of the shared-memory boxes around them.
struct TileGeom {
    int d;
    int L[3];
    int T[3];          // tile extent (cells)
    int nt[3];         // tiles per dimension
    int box[3];        // box extent (cells) per dimension
    int off[3];        // box origin = tile origin - off
    int cells_per_tile_log2;
};

template <typename T>
struct TapArgs {
    TileGeom g;
    WinParams<T> w;
    int batch;
    int batch_smem;            // batch entries held in shared memory at once
    int comp;                  // compensated accumulation (F32_COMP)
    const T* xs;               // sorted nodes, N x d
    const uint32_t* perm;      // sorted -> caller index
    const WorkItem* work;
    int n_work;
    const uint32_t* heads;     // pair heads of each item (sorted index | partner flag << 31), or null
    const uint32_t* nheads;    // heads per item
    long long N;
    C2<T>* grid;               // B x prod(L)
    long long grid_stride;     // prod(L)
    const C2<T>* fin;          // B x N (spread / grad input)
    C2<T>* fout;               // B x N (interp output)
    T* gradx;                  // N x d (node gradient output)
    int* err;
    unsigned long long wait_ns;   // limit of the box-staging waits (nfftbl_set_wait_limit)
    int stall;                 // 1: the staging waits are armed but nothing completes them (timeout test)
    // spreading
    C2<T>* part;               // n_work x B x box cells: per-item boxes (ordered flush)
    const uint32_t* tile_items;// n_tiles + 1: first work item of each tile
    int spread_sub;            // nodes staged per pass in shared memory
    int spread_batch;          // batch entries per shared-memory box group
    T wbound;                  // bound on prod_t |window factor| (1 for sinh / cKB)
    int spread_warps;          // warps per block of the d = 3 spread kernel
    const T* wfac;             // stored window factors (sorted node i: row i of wstride), or null
    C2<T>* fsorted;            // FP32 d = 3 spreading: fin in sorted node order (N complex), or null
    int wstride;               // row length of wfac: d * 2m rounded up to a multiple of 4
};

// Shared-memory layout of the spread kernels (byte offsets), shared with the host.
struct SpreadSmem {
    size_t box, lb, w, g, run, red, total;
};

// Reduction scratch of every spread kernel, in doubles: [0, 32) per-warp
// sums, 32 and 33 the item's quantum and flag, 36 .. 39 the quantum
// constants in the plan precision (see item_quantum).
constexpr int kSpreadRedDoubles = 40;

template <typename T>
__host__ __device__ __forceinline__ SpreadSmem spread_smem_layout(int d, int A, int box_cells, int nb, int sub) {
    auto al = [](size_t v) { return (v + 15) / 16 * 16; };
    SpreadSmem L{};
    const size_t slot = static_cast<size_t>((box_cells + 1) / 2 * 2);   // u64 pairs, even count
    L.box = 0;
    L.lb = al(L.box + static_cast<size_t>(nb) * slot * 16);
    L.w = al(L.lb + static_cast<size_t>(sub) * 4);
    L.g = al(L.w + static_cast<size_t>(sub) * d * A * sizeof(T));
    L.run = al(L.g + static_cast<size_t>(nb) * sub * 2 * sizeof(T));
    L.red = al(L.run + static_cast<size_t>(sub + 1) * 4);
    L.total = al(L.red + kSpreadRedDoubles * 8);
    return L;
}

// Row length (elements) of spread2_kernel's per-warp node table: 2A window
// values, the input value (2 elements), the segment key and the first
// column within the segment (an int in each of the last two elements); with
// A even every row starts 16-byte aligned and consecutive rows fall on
// different bank groups.
template <typename T>
__host__ __device__ constexpr int spread2_row(int A) {
    return 2 * A + 4;
}

// Shared-memory layout of spread2_kernel (d = 2): the fixed-point box, one
// 32-row node table per warp, a reduction scratch.
template <typename T>
__host__ __device__ __forceinline__ SpreadSmem spread2_layout(int A, int box_cells, int nb, int nwarps) {
    auto al = [](size_t v) { return (v + 15) / 16 * 16; };
    SpreadSmem L{};
    const size_t slot = static_cast<size_t>((box_cells + 1) / 2 * 2);
    L.box = 0;
    L.w = al(L.box + static_cast<size_t>(nb) * slot * 16);
    L.red = al(L.w + static_cast<size_t>(nwarps) * 32 * spread2_row<T>(A) * sizeof(T));
    L.lb = L.g = L.run = L.red;
    L.total = al(L.red + kSpreadRedDoubles * 8);
    return L;
}

// Shared-memory layout of spread3_kernel (d = 3): the fixed-point box (16
// bytes per cell), one 32-row node table per warp (rows of 3A window values,
// the input value, the packed first taps and padding), a reduction scratch.
template <typename T>
__host__ __device__ constexpr int spread3_row(int A) {
    return 3 * A + 4;
}

template <typename T>
__host__ __device__ __forceinline__ SpreadSmem spread3_layout(int A, int box_cells, int nb, int nwarps) {
    auto al = [](size_t v) { return (v + 15) / 16 * 16; };
    SpreadSmem L{};
    L.box = 0;
    L.w = al(L.box + static_cast<size_t>(nb) * box_cells * 16);
    L.red = al(L.w + static_cast<size_t>(nwarps) * 32 * spread3_row<T>(A) * sizeof(T));
    L.lb = L.g = L.run = L.red;
    L.total = al(L.red + kSpreadRedDoubles * 8);
    return L;
}

// Warps per block of spread3_kernel: 16 in FP32 when the tables fit, else 8.
template <typename T>
__host__ __forceinline__ int spread3_warps(int A, int box_cells, size_t limit) {
    if (sizeof(T) == 4 && spread3_layout<T>(A, box_cells, 1, 16).total <= limit) return 16;
    return 8;
}

// Column-owner d = 3 spreading (FP32, tiles of 8 x 8 x 8 cells, compile-time
// W = 2m, 4 <= W <= 16): every lane of the block owns one column
// (c1, c2) of the item's box and keeps the box's R cells along dimension 0
// of that column in registers; warps own patches of 4 x 8 columns.  The
// node table holds, per node, its window values of each dimension placed at
// their box positions (zero elsewhere: R rows for dimension 0, 4 P1 and 8 P2
// columns for dimensions 1 and 2), its input value and the mask of the warps
// whose patch meets its window.  Two tables of C nodes (one third of the
// block's threads: one thread per node and dimension fills them) alternate.
template <int W>
struct Spread3C {
    static constexpr int T = 8;                       // tile extent, every dimension
    static constexpr int R = T + W - 1;               // box extent, dimension 0 (rows)
    static constexpr int RP = (R + 3) / 4 * 4;        // rows padded to whole float4s
    static constexpr int B1 = T + W - 1;              // box extent, dimension 1
    static constexpr int B2 = T + W;                  // box extent, dimension 2 (even origin)
    static constexpr int P1 = (B1 + 3) / 4;           // warp patches along dimension 1 (4 columns)
    static constexpr int P2 = (B2 + 7) / 8;           // and along dimension 2 (8 columns)
    static constexpr int WARPS = P1 * P2;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int C = THREADS / 3;             // nodes per table
    static constexpr int O1 = RP;                     // dimension-1 values (4 P1 entries)
    static constexpr int O2 = RP + 4 * P1;            // dimension-2 values (8 P2 entries)
    static constexpr int OM = O2 + 8 * P2;            // g.x, g.y, warp mask, unused
    static constexpr int ROW = OM + 4;                // node-table row, floats (16-byte multiple)
    static constexpr size_t SMEM = 2 * static_cast<size_t>(C) * ROW * sizeof(float);
    static_assert(WARPS <= 32, "warp mask is 32 bits");
};

// Shared memory of the column-owner d = 3 spreading kernel for truncation m
// (0 if it does not exist for m).
inline size_t spread3c_smem(int m) {
    switch (m) {
        case 2: return Spread3C<4>::SMEM;
        case 3: return Spread3C<6>::SMEM;
        case 4: return Spread3C<8>::SMEM;
        case 5: return Spread3C<10>::SMEM;
        case 6: return Spread3C<12>::SMEM;
        case 7: return Spread3C<14>::SMEM;
        case 8: return Spread3C<16>::SMEM;
        default: return 0;
    }
}

// Whether an FP32 d = 3 plan spreads with the column-owner kernel: a
// compile-time truncation and 8 x 8 x 8 tiles.
inline bool spread3c_applies(int d, bool fp32, int m, const int* T) {
    return d == 3 && fp32 && m >= 2 && m <= 8 && T[0] == 8 && T[1] == 8 && T[2] == 8;
}

// Shared memory of the spread kernel for dimension d (minimum batch group).
template <typename T>
__host__ __forceinline__ size_t spread_min_smem(int d, int A, int box_cells, size_t limit) {
    if (d == 2) return spread2_layout<T>(A, box_cells, 1, 8).total;
    if (d == 3) return spread3_layout<T>(A, box_cells, 1, spread3_warps<T>(A, box_cells, limit)).total;
    return spread_smem_layout<T>(d, A, box_cells, 1, 32).total;
}

// Length of the per-dimension tap arrays of the short-sum kernels: 2m for
// the compile-time truncations (NFFTBL_FIXED_M_LIST), 24 for the kernel that
// takes m at run time.
inline int tap_array_len(int m) {
    switch (m) {
        case 2: case 3: case 4: case 5: case 6: case 7: case 8: return 2 * m;
        default: return 24;
    }
}

struct DeviceBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace nfftbl

struct nfftbl_plan_s {
    int d = 0;
    int M[3] = {1, 1, 1};
    int L[3] = {1, 1, 1};
    int m = 0;
    double sigma = 2.0;
    int window = NFFTBL_WIN_SINH;
    int method = NFFTBL_SHANNON;
    int precision = NFFTBL_F32;
    double beta = 0.0;
    int batch = 1;
    int nodes_per_item = 0;
    nfftbl::TileGeom geom{};
    int device = 0;
    int num_sms = 0;
    int smem_optin = 0;                   // max dynamic shared memory per block
    cudaStream_t stream = nullptr;
    std::string last_error;
    long long launches = 0;

    // window
    std::vector<double> table_host;
    nfftbl::DeviceBuf table_dev;          // T (float or double) table values
    nfftbl::DeviceBuf table_dev64;        // double copy for the quadrature
    nfftbl::DeviceBuf fac64[3];           // d_t(k) = 1/(L psi_hat(k)), double, M_t entries
    nfftbl::DeviceBuf facT[3];            // (-1)^k d_t(k), plan precision
    nfftbl::DeviceBuf tw[3];              // twiddles e^{2 pi i j / L_t}, plan precision

    // grid and FFT scratch
    nfftbl::DeviceBuf grid;
    nfftbl::DeviceBuf tmpA, tmpB;
    CUtensorMap tmap{};
    bool tmap_ok = false;

    // nodes
    long long N = -1;                     // -1: no nodes set
    nfftbl::DeviceBuf xs;                 // sorted nodes
    nfftbl::DeviceBuf keys, perm;         // sorted keys / permutation (uint32)
    nfftbl::DeviceBuf keys_tmp, perm_tmp; // radix sort ping-pong
    nfftbl::DeviceBuf hist;               // radix sort block histograms
    nfftbl::DeviceBuf wfac;               // stored window factors (step 0b, tensor-product form)
    int store_factors = 1;
    int precorrect = 1;                   // 0: D = I (Section 5's approximation)
    bool wfac_valid = false;
    nfftbl::DeviceBuf table_coef;         // FP32 table window: float4 cubic coefficients per interval
    nfftbl::DeviceBuf scan_tmp;           // per-tile sums of the multi-block scan
    nfftbl::DeviceBuf tile_off;           // n_tiles + 1 (uint32)
    nfftbl::DeviceBuf work;               // WorkItem list
    nfftbl::DeviceBuf tile_items;         // n_tiles + 1: first work item per tile
    nfftbl::DeviceBuf part;               // spread boxes, one slot per (item, batch entry)
    nfftbl::DeviceBuf heads, nheads;      // same-cell pair heads per work item (interpolation)
    nfftbl::DeviceBuf fsorted;            // FP32 d = 3: the adjoint input in sorted node order (N complex)
    nfftbl::DeviceBuf counters;           // small device scratch (ints)
    long long n_tiles = 0;
    long long n_work = 0;
    int key_bits = 0;

    nfftbl::DeviceBuf lw_f, lw_h, lw_marg, lw_dpsi;   // learned-window loss/gradient scratch
    int weights_mode = 0;                 // opts.weights
    bool poly_ok = false;                 // per-tap weight polynomials fitted (FP32 plans)
    int poly_edge_sqrt = 0;
    float poly_coef[16][12] = {};
    double poly_err = 0.0;                // their largest error (FP32 evaluation) on a fine grid
    nfftbl::DeviceBuf err;                // device error word
    int* err_host = nullptr;              // pinned mirror
    unsigned long long wait_ns = nfftbl::kWaitLimitNs;   // limit of the box-staging waits
    int stall_next = 0;                   // next interpolation: waits that nothing completes (timeout test)

    // host-buffer entry points (nfftbl_forward_host / nfftbl_adjoint_host):
    // staging buffers, an upload and a download stream, and the events that
    // order each staging buffer's copies against the transform that uses it
    nfftbl::DeviceBuf hs_fhat_in, hs_f_out, hs_f_in, hs_fhat_out;
    cudaStream_t s_up = nullptr, s_down = nullptr;
    enum { EV_IN_FWD, EV_IN_ADJ, EV_FWD_DONE, EV_ADJ_DONE, EV_OUT_F, EV_OUT_FHAT, EV_COUNT };
    cudaEvent_t hev[EV_COUNT] = {};
    bool hev_set[EV_COUNT] = {};

    // optional per-kernel timing (nfftbl_kernel_timing)
    bool timing = false;
    struct Timed {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
};

namespace nfftbl {

// Per-kernel timing hooks (plan.cu): bracket one launch on the plan's stream.
void timing_begin(nfftbl_plan_s* p, int kind);
void timing_end(nfftbl_plan_s* p);

// Message returned by nfftbl_plan_error() for calls without a plan (plan.cu).
void set_plan_error(const std::string& msg);

// Allocation helpers (plan.cu).
nfftbl_status ensure_buf(nfftbl_plan_s* p, DeviceBuf& b, size_t bytes);
void free_buf(DeviceBuf& b);
nfftbl_status fail(nfftbl_plan_s* p, nfftbl_status st, const std::string& msg);
nfftbl_status check_cuda(nfftbl_plan_s* p, cudaError_t e, const char* what);

// window.cu
cudaError_t launch_window_factors(int with_sinc, int window, int L, int M, int m, double beta,
                                  const double* table, int table_n, double* fac64_out,
                                  cudaStream_t s);
// The quadrature rule the window-factor kernels read, copied to the current
// device once and synchronously; launch_window_factors_preloaded then
// launches the kernel alone (no copy), for a closed-form window (no table).
cudaError_t upload_gl_rule_sync();
cudaError_t launch_window_factors_preloaded(int with_sinc, int window, int L, int M, int m, double beta,
                                            double* fac64_out, cudaStream_t s);
cudaError_t launch_cast_factors(const double* fac64, int M, void* out, int is_double, cudaStream_t s);
cudaError_t launch_twiddles(int L, void* out, int is_double, cudaStream_t s);
cudaError_t launch_window_transform(int with_sinc, int window, int L, int m, double beta, const double* table,
                                    int table_n, const double* v, int n, double* out, cudaStream_t s);
cudaError_t launch_table_cast(const double* in, int n, float* out, float4* coef, cudaStream_t s);
cudaError_t launch_window_table_grad(int L, int M, int m, int table_n, const double* dEdpsi, double* grad,
                                     cudaStream_t s);

// learn.cu
nfftbl_status run_table_grad(nfftbl_plan_s* p, const TapArgs<float>& args, const double* loss, double* grad);
cudaError_t launch_residual(int is_double, void* f, const void* y, long long n, double* loss, cudaStream_t s);
cudaError_t launch_marginals(int is_double, const void* hhat, const void* fhat, long long total, int d, const int* M,
                             double* P0, double* P1, double* P2, cudaStream_t s);
cudaError_t launch_dEdpsihat(const double* P, const double* fac, int M, int L, const double* loss, double* out,
                             cudaStream_t s);
template <typename T> TapArgs<T> make_tap_args_public(nfftbl_plan_s* p);

// bin.cu
nfftbl_status bin_nodes(nfftbl_plan_s* p, long long N, const void* x_dev);

// fft.cu
nfftbl_status fft_forward(nfftbl_plan_s* p, const void* fhat);
nfftbl_status fft_adjoint(nfftbl_plan_s* p, void* fhat);
cudaError_t launch_fft_forward_pass_f32(const void* in, void* out, long long outer, long long inner, int M, int L,
                                        const float* fac, const void* tw, cudaStream_t s);

// Short-sum kernels (taps.cuh).  launch_tap_kernel is instantiated once per
// (precision, dimension, tap count W = 2m, or W = 0 for m read at run time)
// in translation units the build generates; taps_dispatch.cu picks one.
enum TapKind { TAP_INTERP = 0, TAP_SPREAD = 1, TAP_GRAD = 2, TAP_FACTORS = 3 };
template <typename T, int D, int W>
nfftbl_status launch_tap_kernel(nfftbl_plan_s* p, const TapArgs<T>& args, int kind, size_t smem);
template <typename T, int D>
nfftbl_status run_taps_d(nfftbl_plan_s* p, const TapArgs<T>& args, int kind, size_t smem);
// Compile-time tap counts W = 2m built by the generator (others use W = 0).
#define NFFTBL_FIXED_M_LIST(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

}  // namespace nfftbl
