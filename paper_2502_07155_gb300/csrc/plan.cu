// C-ABI entry points (include/nfftbl.h): plan creation and validation, the
// TMA descriptor of the grid, and the order of kernels per transform.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "plan_internal.h"

namespace nfftbl {

namespace {
thread_local std::string g_plan_error;

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// v = 2^a 3^b 5^c (the FFT's radices)
bool is_235(long long v) {
    if (v <= 0) return false;
    for (int r : {2, 3, 5})
        while (v % r == 0) v /= r;
    return v == 1;
}
int ilog2(long long v) {
    int r = 0;
    while ((1LL << r) < v) ++r;
    return r;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

size_t complex_bytes(const nfftbl_plan_s* p) { return p->precision == NFFTBL_F64 ? 16 : 8; }

long long prod_L(const nfftbl_plan_s* p) {
    long long s = 1;
    for (int t = 0; t < p->d; ++t) s *= p->L[t];
    return s;
}

long long box_cells(const TileGeom& g) {
    long long c = 1;
    for (int t = 0; t < g.d; ++t) c *= g.box[t];
    return c;
}

void set_geom(TileGeom& g, int d, const int* L, const int* T, int m) {
    g.d = d;
    g.cells_per_tile_log2 = 0;
    for (int t = 0; t < 3; ++t) {
        g.L[t] = (t < d) ? L[t] : 1;
        g.T[t] = (t < d) ? T[t] : 1;
        g.nt[t] = g.L[t] / g.T[t];
        if (t < d) {
            // fastest dimension: origin kept even (16-byte TMA start for float2)
            const bool fast = (t == d - 1);
            g.off[t] = fast ? ((m & 1) ? m - 1 : m) : m - 1;
            g.box[t] = g.T[t] + 2 * m - (fast ? 0 : 1);
            g.cells_per_tile_log2 += ilog2(g.T[t]);
        } else {
            g.off[t] = 0;
            g.box[t] = 1;
        }
    }
}

constexpr size_t kBoxBudget = 96 * 1024;   // per CTA, leaves room for 2 CTAs/SM
constexpr size_t kBoxMax = 200 * 1024;     // hard cap on one box

nfftbl_status make_tmap(nfftbl_plan_s* p) {
    auto fn = encode_fn();
    if (!fn) return fail(p, NFFTBL_ECUDA, "cuTensorMapEncodeTiled entry point not available");
    const int d = p->d;
    const int rank = d + 1;
    const size_t es = (p->precision == NFFTBL_F64) ? 8 : 4;
    cuuint64_t dims[5];
    cuuint64_t strides[4];
    cuuint32_t box[5];
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    dims[0] = 2ull * p->L[d - 1];
    box[0] = 2u * p->geom.box[d - 1];
    for (int r = 1; r < d; ++r) {
        dims[r] = p->L[d - 1 - r];
        box[r] = p->geom.box[d - 1 - r];
    }
    dims[d] = p->batch;
    box[d] = 1;
    cuuint64_t st = dims[0] * es;
    for (int r = 1; r < rank; ++r) {
        strides[r - 1] = st;
        st *= dims[r];
    }
    CUresult res = fn(&p->tmap, p->precision == NFFTBL_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                      rank, p->grid.p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (res != CUDA_SUCCESS) return fail(p, NFFTBL_ECUDA, "cuTensorMapEncodeTiled failed");
    p->tmap_ok = true;
    return NFFTBL_OK;
}

// Row length of the stored window factors: d * 2m rounded up to a multiple
// of 4 (rows start 16-byte aligned).
int factor_stride(const nfftbl_plan_s* p) {
    return (p->d * 2 * p->m + 3) / 4 * 4;
}

template <typename T>
TapArgs<T> make_tap_args(nfftbl_plan_s* p) {
    TapArgs<T> a{};
    a.g = p->geom;
    a.w.method = p->method;
    a.w.window = p->window;
    a.w.m = p->m;
    a.w.inv_m = static_cast<T>(1.0 / p->m);
    a.w.beta = static_cast<T>(p->beta);
    a.w.c_exp = static_cast<T>(p->beta / std::log(2.0));
    if (p->window == NFFTBL_WIN_SINH)
        a.w.c_norm = static_cast<T>(1.0 / -std::expm1(-2.0 * p->beta));
    else if (p->window == NFFTBL_WIN_CKB)
        a.w.c_norm = static_cast<T>(1.0 / (std::cyl_bessel_i(0.0, p->beta) - 1.0));
    else
        a.w.c_norm = T(1);
    a.w.table = static_cast<const T*>(p->window == NFFTBL_WIN_TABLE ? p->table_dev.p : nullptr);
    a.w.table_n = static_cast<int>(p->table_host.size()) - 1;
    a.wstride = factor_stride(p);
    a.wfac = p->wfac_valid ? static_cast<const T*>(p->wfac.p) : nullptr;
    a.w.tcoef = (sizeof(T) == 4 && p->window == NFFTBL_WIN_TABLE) ? static_cast<const float4*>(p->table_coef.p) : nullptr;
    a.w.poly = (sizeof(T) == 4 && p->poly_ok) ? 1 : 0;
    a.w.poly_edge_sqrt = p->poly_edge_sqrt;
    std::memcpy(a.w.pc, p->poly_coef, sizeof(a.w.pc));
    a.batch = p->batch;
    const size_t bb = (static_cast<size_t>(box_cells(p->geom)) * sizeof(C2<T>) + 127) / 128 * 128;
    a.batch_smem = static_cast<int>(std::max<size_t>(1, std::min<size_t>(p->batch, kBoxBudget / bb)));
    a.comp = p->precision == NFFTBL_F32_COMP;
    a.xs = static_cast<const T*>(p->xs.p);
    a.perm = static_cast<const uint32_t*>(p->perm.p);
    a.work = static_cast<const WorkItem*>(p->work.p);
    a.heads = static_cast<const uint32_t*>(p->heads.p);
    a.nheads = static_cast<const uint32_t*>(p->nheads.p);
    a.fsorted = static_cast<C2<T>*>(p->fsorted.p);
    a.n_work = static_cast<int>(p->n_work);
    a.N = p->N;
    a.grid = static_cast<C2<T>*>(p->grid.p);
    a.grid_stride = prod_L(p);
    a.err = static_cast<int*>(p->err.p);
    a.wait_ns = p->wait_ns;
    a.stall = 0;
    a.part = static_cast<C2<T>*>(p->part.p);
    a.tile_items = static_cast<const uint32_t*>(p->tile_items.p);
    a.wbound = T(1);
    if (p->window == NFFTBL_WIN_TABLE) {
        double mx = 1.0;
        for (double v : p->table_host) mx = std::max(mx, std::fabs(v));
        a.wbound = static_cast<T>(std::pow(mx, p->d));
    }
    return a;
}

// Batch entries per box group and nodes per pass of the spread kernel: the
// smallest configuration must fit the device's shared memory; grow the batch
// group while the block stays within about half an SM's shared memory.
template <typename T>
bool spread_config(const nfftbl_plan_s* p, int& nb, int& sub, size_t& bytes) {
    const int A = tap_array_len(p->m);
    const int cells = static_cast<int>(box_cells(p->geom));
    const size_t limit = static_cast<size_t>(p->smem_optin);
    const int w3 = spread3_warps<T>(A, cells, limit);
    auto layout = [&](int nbv, int subv) {
        if (p->d == 2) return spread2_layout<T>(A, cells, nbv, 8).total;
        if (p->d == 3) return spread3_layout<T>(A, cells, nbv, w3).total;
        return spread_smem_layout<T>(p->d, A, cells, nbv, subv).total;
    };
    for (sub = 256; sub >= 32; sub /= 2) {
        bytes = layout(1, sub);
        if (bytes <= limit) break;
    }
    if (bytes > limit) return false;
    nb = 1;
    while (nb < p->batch) {
        const size_t nbytes = layout(nb + 1, sub);
        if (nbytes > std::min<size_t>(limit, 110 * 1024)) break;
        ++nb;
        bytes = nbytes;
    }
    return true;
}

}  // namespace

template <typename T>
TapArgs<T> make_tap_args_public(nfftbl_plan_s* p) {
    return make_tap_args<T>(p);
}
template TapArgs<float> make_tap_args_public<float>(nfftbl_plan_s*);

namespace {

template <typename T>
nfftbl_status run_taps(nfftbl_plan_s* p, int kind, const void* fin, void* fout, void* gradx) {
    TapArgs<T> a = make_tap_args<T>(p);
    a.fin = static_cast<const C2<T>*>(fin);
    a.fout = static_cast<C2<T>*>(fout);
    a.gradx = static_cast<T*>(gradx);
    if (kind == TAP_INTERP && p->stall_next) {   // one launch only
        a.stall = 1;
        p->stall_next = 0;
    }
    // box slots padded to 128 bytes, plus 128 bytes to align the base
    const size_t slot = (static_cast<size_t>(box_cells(p->geom)) * sizeof(C2<T>) + 127) / 128 * 128;
    size_t smem = static_cast<size_t>(a.batch_smem) * slot + 128;
    if (kind == TAP_SPREAD && spread3c_applies(p->d, sizeof(T) == 4, p->m, p->geom.T)) {
        smem = spread3c_smem(p->m);   // (the launcher sets it again with the kernel)
    } else if (kind == TAP_SPREAD) {
        int nb = 1, sub = 32;
        if (!spread_config<T>(p, nb, sub, smem))
            return fail(p, NFFTBL_EUNSUPPORTED, "spread box does not fit in shared memory");
        a.spread_batch = nb;
        a.spread_sub = sub;
        a.spread_warps = spread3_warps<T>(tap_array_len(p->m), static_cast<int>(box_cells(p->geom)),
                                          static_cast<size_t>(p->smem_optin));
    }
    switch (p->d) {
        case 1: return run_taps_d<T, 1>(p, a, kind, smem);
        case 2: return run_taps_d<T, 2>(p, a, kind, smem);
        default: return run_taps_d<T, 3>(p, a, kind, smem);
    }
}

nfftbl_status taps(nfftbl_plan_s* p, int kind, const void* fin, void* fout, void* gradx) {
    if (p->precision == NFFTBL_F64) return run_taps<double>(p, kind, fin, fout, gradx);
    return run_taps<float>(p, kind, fin, fout, gradx);
}

void destroy_plan(nfftbl_plan_s* p) {
    if (!p) return;
    free_buf(p->table_dev);
    free_buf(p->table_dev64);
    for (int t = 0; t < 3; ++t) {
        free_buf(p->fac64[t]);
        free_buf(p->facT[t]);
        free_buf(p->tw[t]);
    }
    free_buf(p->grid);
    free_buf(p->tmpA);
    free_buf(p->tmpB);
    free_buf(p->xs);
    free_buf(p->keys);
    free_buf(p->perm);
    free_buf(p->keys_tmp);
    free_buf(p->perm_tmp);
    free_buf(p->hist);
    free_buf(p->wfac);
    free_buf(p->table_coef);
    free_buf(p->scan_tmp);
    free_buf(p->tile_off);
    free_buf(p->work);
    free_buf(p->tile_items);
    free_buf(p->part);
    free_buf(p->heads);
    free_buf(p->fsorted);
    free_buf(p->nheads);
    free_buf(p->counters);
    free_buf(p->lw_f);
    free_buf(p->lw_h);
    free_buf(p->lw_marg);
    free_buf(p->lw_dpsi);
    free_buf(p->err);
    if (p->err_host) cudaFreeHost(p->err_host);
    free_buf(p->hs_fhat_in);
    free_buf(p->hs_f_out);
    free_buf(p->hs_f_in);
    free_buf(p->hs_fhat_out);
    for (auto& e : p->hev)
        if (e) cudaEventDestroy(e);
    if (p->s_up) cudaStreamDestroy(p->s_up);
    if (p->s_down) cudaStreamDestroy(p->s_down);
    for (auto& t : p->timed) {
        if (t.a) cudaEventDestroy(t.a);
        if (t.b) cudaEventDestroy(t.b);
    }
    for (auto e : p->event_pool) cudaEventDestroy(e);
    delete p;
}

// Record the failure of nfftbl_plan (msg, or the plan's own message when
// msg is empty) and release the partly built plan.
nfftbl_status plan_fail(nfftbl_plan_s* p, nfftbl_status st, const std::string& msg) {
    g_plan_error = (msg.empty() && p) ? p->last_error : msg;
    destroy_plan(p);
    return st;
}

}  // namespace

nfftbl_status fail(nfftbl_plan_s* p, nfftbl_status st, const std::string& msg) {
    if (p) p->last_error = msg;
    return st;
}

void set_plan_error(const std::string& msg) { g_plan_error = msg; }

namespace {
cudaEvent_t take_event(nfftbl_plan_s* p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

void timing_begin(nfftbl_plan_s* p, int kind) {
    if (!p->timing) return;
    nfftbl_plan_s::Timed t{kind, take_event(p), take_event(p)};
    if (t.a) cudaEventRecord(t.a, p->stream);
    p->timed.push_back(t);
}

void timing_end(nfftbl_plan_s* p) {
    if (!p->timing || p->timed.empty()) return;
    if (p->timed.back().b) cudaEventRecord(p->timed.back().b, p->stream);
}

nfftbl_status check_cuda(nfftbl_plan_s* p, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return NFFTBL_OK;
    cudaGetLastError();   // clear a sticky launch error of this thread
    const std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(p, e == cudaErrorMemoryAllocation ? NFFTBL_ENOMEM : NFFTBL_ECUDA, msg);
}

nfftbl_status ensure_buf(nfftbl_plan_s* p, DeviceBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return NFFTBL_OK;
    free_buf(b);
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(p, NFFTBL_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
    }
    b.p = ptr;
    b.bytes = bytes;
    return NFFTBL_OK;
}

void free_buf(DeviceBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

}  // namespace nfftbl

using namespace nfftbl;

extern "C" {

namespace nfftbl {
namespace {

// Catmull-Rom value of a window table at u in [0, 1] (the rule the kernels
// use: ghost values v_{-1} = v_1, v_{n+1} = 2 v_n - v_{n-1}), in FP64.
double table_value(const std::vector<double>& v, double u) {
    const int n = static_cast<int>(v.size()) - 1;
    const double s = std::min(std::max(u, 0.0), 1.0) * n;
    int i = static_cast<int>(std::floor(s));
    i = std::min(std::max(i, 0), n - 1);
    const double t = s - i;
    const double p0 = (i == 0) ? v[1] : v[i - 1], p1 = v[i], p2 = v[i + 1];
    const double p3 = (i + 2 <= n) ? v[i + 2] : 2.0 * v[n] - v[n - 1];
    return 0.5 * (2.0 * p1 + (p2 - p0) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t +
                  (3.0 * p1 - p0 - 3.0 * p2 + p3) * t * t * t);
}

// The one-dimensional short-sum kernel at the tap offset delta = L x - l
// (grid units), in FP64: sinc(pi delta) phi(delta / L) for the Shannon
// method, phi(delta / L) for the classical NFFT; zero for |delta| >= m.
double kernel_value(const nfftbl_plan_s* p, double delta) {
    const double r = delta / p->m;
    const double q = (1.0 - r) * (1.0 + r);
    if (!(q > 0.0)) return 0.0;
    double phi;
    if (p->window == NFFTBL_WIN_SINH) phi = std::sinh(p->beta * std::sqrt(q)) / std::sinh(p->beta);
    else if (p->window == NFFTBL_WIN_CKB)
        phi = (std::cyl_bessel_i(0.0, p->beta * std::sqrt(q)) - 1.0) / (std::cyl_bessel_i(0.0, p->beta) - 1.0);
    else phi = table_value(p->table_host, std::fabs(r));
    if (p->method == NFFTBL_CLASSIC) return phi;
    const double sinc = (delta == 0.0) ? 1.0 : std::sin(M_PI * delta) / (M_PI * delta);
    return sinc * phi;
}

// Per-tap weight polynomials of an FP32 plan with m <= 8: tap a (offset
// delta = tau + m - 1 - a, tau in [0, 1)) as a polynomial of degree
// kPolyDeg in t = 2 tau - 1, by Chebyshev interpolation in FP64 converted to
// monomial coefficients.  Windows with a square-root edge (sinh,
// Kaiser-Bessel) fit the two edge taps divided by sqrt(1 - (delta/m)^2),
// which removes the edge singularity; the kernels multiply it back.  The fit
// is checked on a fine grid with the kernels' FP32 Horner evaluation and
// kept only if its largest error is within kPolyTol of the largest weight.
void fit_poly(nfftbl_plan_s* p) {
    p->poly_ok = false;
    p->poly_err = 0.0;
    if (p->precision == NFFTBL_F64 || p->m < 2 || p->m > 8 || p->weights_mode != 1) return;
    const int W = 2 * p->m, D = kPolyDeg;
    const bool sqrt_edge = p->window == NFFTBL_WIN_SINH || p->window == NFFTBL_WIN_CKB;
    p->poly_edge_sqrt = sqrt_edge ? 1 : 0;
    auto edge_q = [&](double delta) {
        const double r = delta / p->m;
        return (1.0 - r) * (1.0 + r);
    };
    double tk[kPolyDeg + 1];
    for (int k = 0; k <= D; ++k) tk[k] = std::cos(M_PI * (k + 0.5) / (D + 1));
    for (int a = 0; a < W; ++a) {
        const int n = p->m - 1 - a;
        const bool edge = sqrt_edge && (a == 0 || a == W - 1);
        double fv[kPolyDeg + 1];
        for (int k = 0; k <= D; ++k) {
            const double delta = 0.5 * (tk[k] + 1.0) + n;
            fv[k] = kernel_value(p, delta) / (edge ? std::sqrt(edge_q(delta)) : 1.0);
        }
        // Chebyshev coefficients, then the monomial form of sum_j c_j T_j(t)
        double cheb[kPolyDeg + 1], mono[kPolyDeg + 1] = {};
        for (int j = 0; j <= D; ++j) {
            double acc = 0.0;
            for (int k = 0; k <= D; ++k) acc += fv[k] * std::cos(M_PI * j * (k + 0.5) / (D + 1));
            cheb[j] = acc * 2.0 / (D + 1) * (j == 0 ? 0.5 : 1.0);
        }
        double tm2[kPolyDeg + 1] = {1.0}, tm1[kPolyDeg + 1] = {0.0, 1.0};   // T_0, T_1
        mono[0] += cheb[0];
        if (D >= 1) mono[1] += cheb[1];
        for (int j = 2; j <= D; ++j) {
            double tj[kPolyDeg + 1] = {};
            for (int k = 0; k <= D; ++k) {
                tj[k] = -tm2[k] + (k > 0 ? 2.0 * tm1[k - 1] : 0.0);
            }
            for (int k = 0; k <= D; ++k) mono[k] += cheb[j] * tj[k];
            for (int k = 0; k <= D; ++k) {
                tm2[k] = tm1[k];
                tm1[k] = tj[k];
            }
        }
        for (int k = 0; k < 12; ++k) p->poly_coef[a][k] = (k <= D) ? static_cast<float>(mono[k]) : 0.0f;
    }
    // check: FP32 Horner (as the kernels evaluate it) against the FP64 kernel
    double err = 0.0, big = 0.0;
    const int G = 2048;
    for (int a = 0; a < W; ++a) {
        const int n = p->m - 1 - a;
        const bool edge = sqrt_edge && (a == 0 || a == W - 1);
        for (int g = 0; g <= G; ++g) {
            const float tau = static_cast<float>(g) / G * 0.99999994f;
            const float t = std::fma(2.0f, tau, -1.0f);
            float v = p->poly_coef[a][D];
            for (int k = D - 1; k >= 0; --k) v = std::fma(v, t, p->poly_coef[a][k]);
            if (edge) {
                const float r = (tau + static_cast<float>(n)) * static_cast<float>(1.0 / p->m);
                const float q = std::fma(-r, r, 1.0f);
                v = (q > 1e-30f) ? v * std::sqrt(q) : 0.0f;
            }
            const double ref = kernel_value(p, static_cast<double>(tau) + n);
            err = std::max(err, std::fabs(static_cast<double>(v) - ref));
            big = std::max(big, std::fabs(ref));
        }
    }
    p->poly_err = (big > 0.0) ? err / big : err;
    p->poly_ok = p->poly_err <= kPolyTol;
}

}  // namespace
}  // namespace nfftbl

void nfftbl_default_opts(nfftbl_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = NFFTBL_F32;
    o->method = NFFTBL_SHANNON;
    o->beta = 0.0;
    o->batch = 1;
    o->factors = 0;
    o->precorrect = 1;
    o->weights = 0;
}

nfftbl_status nfftbl_plan(nfftbl_plan_t* out, int d, const int* M, double sigma, int m, int window,
                          const nfftbl_opts* opts) {
    g_plan_error.clear();
    if (!out) return plan_fail(nullptr, NFFTBL_EINVAL, "out is NULL");
    *out = nullptr;
    nfftbl_opts o;
    nfftbl_default_opts(&o);
    if (opts) o = *opts;
    if (d < 1 || d > 3) return plan_fail(nullptr, NFFTBL_EINVAL, "d must be 1, 2 or 3");
    if (!M) return plan_fail(nullptr, NFFTBL_EINVAL, "M is NULL");
    if (!(sigma >= 1.0) || !std::isfinite(sigma)) return plan_fail(nullptr, NFFTBL_EINVAL, "sigma must be >= 1");
    if (m < 1) return plan_fail(nullptr, NFFTBL_EINVAL, "m must be >= 1");
    if (window < 0 || window > 2) return plan_fail(nullptr, NFFTBL_EINVAL, "unknown window");
    if (o.precision < 0 || o.precision > 2) return plan_fail(nullptr, NFFTBL_EINVAL, "unknown precision");
    if (o.method < 0 || o.method > 1) return plan_fail(nullptr, NFFTBL_EINVAL, "unknown method");
    if (o.factors < 0 || o.factors > 1) return plan_fail(nullptr, NFFTBL_EINVAL, "factors must be 0 or 1");
    if (o.precorrect < 0 || o.precorrect > 1) return plan_fail(nullptr, NFFTBL_EINVAL, "precorrect must be 0 or 1");
    if (o.weights < 0 || o.weights > 1) return plan_fail(nullptr, NFFTBL_EINVAL, "weights must be 0 or 1");
    if (o.batch < 1) return plan_fail(nullptr, NFFTBL_EINVAL, "batch must be >= 1");
    if (window == NFFTBL_WIN_TABLE && (!o.table || o.table_len < 3))
        return plan_fail(nullptr, NFFTBL_EINVAL, "table window needs a table of >= 3 values");
    if (o.nodes_per_item < 0 || o.nodes_per_item > 2047)
        return plan_fail(nullptr, NFFTBL_EINVAL, "nodes_per_item must be in [0, 2047]");
    int L[3] = {1, 1, 1};
    for (int t = 0; t < d; ++t) {
        if (M[t] < 2 || (M[t] & 1)) return plan_fail(nullptr, NFFTBL_EINVAL, "each M_t must be even and >= 2");
        const long long s = static_cast<long long>(std::ceil(sigma * M[t] - 1e-9));
        L[t] = static_cast<int>(2 * ((s + 1) / 2));
        if (2 * m >= L[t]) return plan_fail(nullptr, NFFTBL_EINVAL, "2m must be < L_t");
    }
    for (int t = 0; t < d; ++t)
        if (!is_235(L[t]) || L[t] < 16 || L[t] > 4096)
            return plan_fail(nullptr, NFFTBL_EUNSUPPORTED, "L_t must be of the form 2^a 3^b 5^c in [16, 4096]");
    if (m < 2 || m > 12) return plan_fail(nullptr, NFFTBL_EUNSUPPORTED, "m must be in 2..12");
    double beta = o.beta;
    if (!(beta > 0.0)) {
        beta = (o.method == NFFTBL_SHANNON) ? M_PI * m * (1.0 - 1.0 / sigma)
                                            : 2.0 * M_PI * m * (1.0 - 1.0 / (2.0 * sigma));
        if (window == NFFTBL_WIN_TABLE) beta = 1.0;   // unused by a tabulated window
    }
    if (!(beta > 0.0)) return plan_fail(nullptr, NFFTBL_EINVAL, "beta must be > 0 (sigma = 1 needs an explicit beta)");
    // cell keys are < prod L_t (tile-major, then in-tile row-major)
    long long cells_total = 1;
    for (int t = 0; t < d; ++t) cells_total *= L[t];
    int key_bits = 0;
    while ((1LL << key_bits) < cells_total) ++key_bits;
    if (key_bits > 31) return plan_fail(nullptr, NFFTBL_EUNSUPPORTED, "prod L_t must be <= 2^31");

    // tile shape
    const int def_tile = (d == 1) ? 64 : (d == 2) ? 32 : 8;
    int T[3] = {1, 1, 1};
    const bool user_tile = o.tile[0] > 0;
    for (int t = 0; t < d; ++t) {
        if (user_tile) {
            T[t] = o.tile[t];
        } else {   // the largest power of two <= the default that divides L_t
            T[t] = 1;
            while (2 * T[t] <= def_tile && L[t] % (2 * T[t]) == 0) T[t] *= 2;
        }
        if (!is_pow2(T[t]) || T[t] < 2 || L[t] % T[t] != 0)
            return plan_fail(nullptr, NFFTBL_EINVAL, "tile extents must be powers of two >= 2 dividing L_t");
    }
    const size_t cb = (o.precision == NFFTBL_F64) ? 16 : 8;
    TileGeom g{};
    int dev_for_limits = 0, optin = 0;
    if (cudaGetDevice(&dev_for_limits) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_for_limits) != cudaSuccess) {
        cudaGetLastError();
        return plan_fail(nullptr, NFFTBL_ECUDA, "cannot query the device");
    }
    while (true) {
        set_geom(g, d, L, T, m);
        const size_t bytes = static_cast<size_t>(box_cells(g)) * cb;
        const bool tma_ok = 2 * g.box[d - 1] <= 256 && (d < 2 || g.box[0] <= 256) && (d < 3 || g.box[1] <= 256);
        const int bc = static_cast<int>(box_cells(g));
        const int A = tap_array_len(m);
        size_t spread_min = (o.precision == NFFTBL_F64) ? spread_min_smem<double>(d, A, bc, optin)
                                                        : spread_min_smem<float>(d, A, bc, optin);
        if (spread3c_applies(d, o.precision != NFFTBL_F64, m, T)) spread_min = spread3c_smem(m);
        if (bytes <= kBoxMax && tma_ok && spread_min <= static_cast<size_t>(optin)) break;
        if (user_tile) return plan_fail(nullptr, NFFTBL_EUNSUPPORTED, "tile box exceeds shared memory or TMA limits");
        int big = 0;
        for (int t = 1; t < d; ++t)
            if (T[t] > T[big]) big = t;
        if (T[big] <= 2) return plan_fail(nullptr, NFFTBL_EUNSUPPORTED, "m too large for a shared-memory box");
        T[big] /= 2;
    }

    nfftbl_plan_s* p = new (std::nothrow) nfftbl_plan_s();
    if (!p) return plan_fail(nullptr, NFFTBL_ENOMEM, "host allocation failed");
    p->d = d;
    for (int t = 0; t < d; ++t) {
        p->M[t] = M[t];
        p->L[t] = L[t];
    }
    p->m = m;
    p->sigma = sigma;
    p->window = window;
    p->method = o.method;
    p->precision = o.precision;
    p->beta = beta;
    p->batch = o.batch;
    p->nodes_per_item = o.nodes_per_item > 0 ? o.nodes_per_item : 1024;
    p->store_factors = o.factors;
    p->precorrect = o.precorrect;
    p->geom = g;
    p->smem_optin = optin;
    p->key_bits = key_bits;
    p->n_tiles = 1;
    for (int t = 0; t < d; ++t) p->n_tiles *= g.nt[t];
    if (window == NFFTBL_WIN_TABLE) p->table_host.assign(o.table, o.table + o.table_len);
    p->weights_mode = o.weights;
    fit_poly(p);

    nfftbl_status st;
    if ((st = check_cuda(p, cudaGetDevice(&p->device), "cudaGetDevice")) != NFFTBL_OK) return plan_fail(p, st, "");
    if ((st = check_cuda(p, cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device),
                         "SM count")) != NFFTBL_OK)
        return plan_fail(p, st, "");
    if ((st = ensure_buf(p, p->err, sizeof(int))) != NFFTBL_OK) return plan_fail(p, st, "");
    if ((st = check_cuda(p, cudaMallocHost(reinterpret_cast<void**>(&p->err_host), sizeof(int)), "pinned err")) !=
        NFFTBL_OK)
        return plan_fail(p, st, "");
    *p->err_host = 0;
    cudaStream_t s0 = nullptr;
    if ((st = check_cuda(p, cudaMemsetAsync(p->err.p, 0, sizeof(int), s0), "memset err")) != NFFTBL_OK)
        return plan_fail(p, st, "");

    const bool dbl = p->precision == NFFTBL_F64;
    const double* tab64 = nullptr;
    int tab_n = 0;
    if (window == NFFTBL_WIN_TABLE) {
        const size_t n = p->table_host.size();
        tab_n = static_cast<int>(n) - 1;
        if ((st = ensure_buf(p, p->table_dev64, n * sizeof(double))) != NFFTBL_OK) return plan_fail(p, st, "");
        if ((st = check_cuda(p, cudaMemcpy(p->table_dev64.p, p->table_host.data(), n * sizeof(double),
                                           cudaMemcpyHostToDevice),
                             "table upload")) != NFFTBL_OK)
            return plan_fail(p, st, "");
        tab64 = static_cast<const double*>(p->table_dev64.p);
        if (dbl) {
            p->table_dev = p->table_dev64;   // shared, freed once below
            p->table_dev64 = DeviceBuf{};
            tab64 = static_cast<const double*>(p->table_dev.p);
        } else {
            if ((st = ensure_buf(p, p->table_dev, n * sizeof(float))) != NFFTBL_OK) return plan_fail(p, st, "");
            if ((st = ensure_buf(p, p->table_coef, n * sizeof(float4))) != NFFTBL_OK) return plan_fail(p, st, "");
            if ((st = check_cuda(p, launch_table_cast(tab64, static_cast<int>(n), static_cast<float*>(p->table_dev.p),
                                                      static_cast<float4*>(p->table_coef.p), s0),
                                 "table cast")) != NFFTBL_OK)
                return plan_fail(p, st, "");
        }
    }
    for (int t = 0; t < d; ++t) {
        if ((st = ensure_buf(p, p->fac64[t], M[t] * sizeof(double))) != NFFTBL_OK) return plan_fail(p, st, "");
        if ((st = ensure_buf(p, p->facT[t], M[t] * (dbl ? 8 : 4))) != NFFTBL_OK) return plan_fail(p, st, "");
        if ((st = ensure_buf(p, p->tw[t], L[t] * complex_bytes(p))) != NFFTBL_OK) return plan_fail(p, st, "");
        if (p->precorrect) {
            if ((st = check_cuda(p, launch_window_factors(p->method == NFFTBL_SHANNON, window, L[t], M[t], m, beta,
                                                          tab64, tab_n, static_cast<double*>(p->fac64[t].p), s0),
                                 "window factors")) != NFFTBL_OK)
                return plan_fail(p, st, "");
        } else {
            // D = I (Section 5: |I_L| psi_hat(k) ~ 1, so 1/(|I_L| psi_hat) ~ 1): factor 1
            const std::vector<double> inv(M[t], 1.0);
            if ((st = check_cuda(p, cudaMemcpyAsync(p->fac64[t].p, inv.data(), M[t] * sizeof(double),
                                                    cudaMemcpyHostToDevice, s0),
                                 "factors")) != NFFTBL_OK)
                return plan_fail(p, st, "");
            if ((st = check_cuda(p, cudaStreamSynchronize(s0), "factors")) != NFFTBL_OK) return plan_fail(p, st, "");
        }
        if ((st = check_cuda(p, launch_cast_factors(static_cast<double*>(p->fac64[t].p), M[t], p->facT[t].p, dbl, s0),
                             "factor cast")) != NFFTBL_OK)
            return plan_fail(p, st, "");
        if ((st = check_cuda(p, launch_twiddles(L[t], p->tw[t].p, dbl, s0), "twiddles")) != NFFTBL_OK)
            return plan_fail(p, st, "");
        p->launches += 3;
    }
    const long long B = p->batch;
    const size_t cbytes = complex_bytes(p);
    if ((st = ensure_buf(p, p->grid, B * prod_L(p) * cbytes)) != NFFTBL_OK) return plan_fail(p, st, "");
    if (d == 2) {
        if ((st = ensure_buf(p, p->tmpA, B * static_cast<long long>(M[0]) * L[1] * cbytes)) != NFFTBL_OK)
            return plan_fail(p, st, "");
    } else if (d == 3) {
        if ((st = ensure_buf(p, p->tmpA, B * static_cast<long long>(M[0]) * M[1] * L[2] * cbytes)) != NFFTBL_OK)
            return plan_fail(p, st, "");
        if ((st = ensure_buf(p, p->tmpB, B * static_cast<long long>(M[0]) * L[1] * L[2] * cbytes)) != NFFTBL_OK)
            return plan_fail(p, st, "");
    }
    if ((st = check_cuda(p, cudaMemsetAsync(p->grid.p, 0, B * prod_L(p) * cbytes, s0), "grid clear")) != NFFTBL_OK)
        return plan_fail(p, st, "");
    if ((st = make_tmap(p)) != NFFTBL_OK) return plan_fail(p, st, "");
    if ((st = check_cuda(p, cudaStreamSynchronize(s0), "plan sync")) != NFFTBL_OK) return plan_fail(p, st, "");
    *out = p;
    return NFFTBL_OK;
}

nfftbl_status nfftbl_set_stream(nfftbl_plan_t p, void* stream) {
    if (!p) return NFFTBL_EINVAL;
    p->stream = static_cast<cudaStream_t>(stream);
    return NFFTBL_OK;
}

// Step 0b (tensor-product form): the d x 2m window factors of every sorted
// node, kept for the transforms.  Without memory for them the transforms
// evaluate the factors themselves (no error).
static nfftbl_status compute_factors(nfftbl_plan_t p) {
    p->wfac_valid = false;
    if (!p->store_factors || p->N <= 0) return NFFTBL_OK;
    const size_t es = (p->precision == NFFTBL_F64) ? sizeof(double) : sizeof(float);
    const size_t bytes = static_cast<size_t>(p->N) * factor_stride(p) * es;
    if (p->wfac.bytes < bytes) {
        free_buf(p->wfac);
        void* ptr = nullptr;
        if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return NFFTBL_OK;
        }
        p->wfac.p = ptr;
        p->wfac.bytes = bytes;
    }
    nfftbl_status st = taps(p, TAP_FACTORS, nullptr, nullptr, nullptr);
    if (st == NFFTBL_OK) p->wfac_valid = true;
    return st;
}

nfftbl_status nfftbl_set_nodes(nfftbl_plan_t p, int64_t N, const void* x_dev) {
    if (!p) return NFFTBL_EINVAL;
    if (N < 0 || N >= (1LL << 31)) return fail(p, NFFTBL_EINVAL, "N must be in [0, 2^31)");
    if (N > 0 && !x_dev) return fail(p, NFFTBL_EINVAL, "x_dev is NULL");
    p->last_error.clear();
    p->wfac_valid = false;
    nfftbl_status st = bin_nodes(p, N, x_dev);
    if (st != NFFTBL_OK) return st;
    return compute_factors(p);
}

static nfftbl_status ready(nfftbl_plan_t p) {
    if (!p) return NFFTBL_EINVAL;
    if (p->N < 0) return fail(p, NFFTBL_ESTATE, "nodes not set (nfftbl_set_nodes)");
    return NFFTBL_OK;
}

nfftbl_status nfftbl_forward(nfftbl_plan_t p, const void* fhat_dev, void* f_dev) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!fhat_dev || (!f_dev && p->N > 0)) return fail(p, NFFTBL_EINVAL, "NULL data pointer");
    if ((st = fft_forward(p, fhat_dev)) != NFFTBL_OK) return st;
    return taps(p, TAP_INTERP, nullptr, f_dev, nullptr);
}

nfftbl_status nfftbl_adjoint(nfftbl_plan_t p, const void* f_dev, void* fhat_dev) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!fhat_dev || (!f_dev && p->N > 0)) return fail(p, NFFTBL_EINVAL, "NULL data pointer");
    // the ordered flush writes every grid cell: no clearing needed
    if ((st = taps(p, TAP_SPREAD, f_dev, nullptr, nullptr)) != NFFTBL_OK) return st;
    return fft_adjoint(p, fhat_dev);
}

nfftbl_status nfftbl_node_grad(nfftbl_plan_t p, const void* fhat_dev, const void* gradf_dev, void* gradx_dev) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!fhat_dev || ((!gradf_dev || !gradx_dev) && p->N > 0)) return fail(p, NFFTBL_EINVAL, "NULL data pointer");
    if ((st = fft_forward(p, fhat_dev)) != NFFTBL_OK) return st;
    return taps(p, TAP_GRAD, gradf_dev, nullptr, gradx_dev);
}

nfftbl_status nfftbl_window_transform(nfftbl_plan_t p, int t, const double* v_dev, int n, double* out_dev) {
    if (!p) return NFFTBL_EINVAL;
    if (t < 0 || t >= p->d) return fail(p, NFFTBL_EINVAL, "dimension t out of range");
    if (n < 0 || (n > 0 && (!v_dev || !out_dev))) return fail(p, NFFTBL_EINVAL, "bad frequency list");
    const double* tab64 = nullptr;
    if (p->window == NFFTBL_WIN_TABLE)
        tab64 = static_cast<const double*>((p->precision == NFFTBL_F64) ? p->table_dev.p : p->table_dev64.p);
    nfftbl_status st = check_cuda(p, launch_window_transform(p->method == NFFTBL_SHANNON, p->window, p->L[t], p->m,
                                                             p->beta, tab64, static_cast<int>(p->table_host.size()) - 1,
                                                             v_dev, n, out_dev, p->stream),
                                  "window transform");
    if (st == NFFTBL_OK && n > 0) p->launches++;
    return st;
}

nfftbl_status nfftbl_interp_grid(nfftbl_plan_t p, void* f_dev) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!f_dev && p->N > 0) return fail(p, NFFTBL_EINVAL, "NULL data pointer");
    return taps(p, TAP_INTERP, nullptr, f_dev, nullptr);
}

nfftbl_status nfftbl_spread_grid(nfftbl_plan_t p, const void* f_dev) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!f_dev && p->N > 0) return fail(p, NFFTBL_EINVAL, "NULL data pointer");
    return taps(p, TAP_SPREAD, f_dev, nullptr, nullptr);
}

// ---- host-buffer entry points.  A transform's input is uploaded on the
// plan's upload stream into a staging buffer and its output downloaded on the
// download stream; events order each staging buffer between its copy and the
// transform that uses it, so the upload of one call and the download of
// another overlap the transforms on the plan stream.
static nfftbl_status host_streams(nfftbl_plan_t p) {
    nfftbl_status st = NFFTBL_OK;
    if (!p->s_up) st = check_cuda(p, cudaStreamCreateWithFlags(&p->s_up, cudaStreamNonBlocking), "upload stream");
    if (st == NFFTBL_OK && !p->s_down)
        st = check_cuda(p, cudaStreamCreateWithFlags(&p->s_down, cudaStreamNonBlocking), "download stream");
    for (int i = 0; st == NFFTBL_OK && i < nfftbl_plan_s::EV_COUNT; ++i)
        if (!p->hev[i]) st = check_cuda(p, cudaEventCreateWithFlags(&p->hev[i], cudaEventDisableTiming), "event");
    return st;
}

static nfftbl_status host_wait(nfftbl_plan_t p, cudaStream_t s, int ev) {
    if (!p->hev_set[ev]) return NFFTBL_OK;
    return check_cuda(p, cudaStreamWaitEvent(s, p->hev[ev], 0), "stream wait");
}

static nfftbl_status host_record(nfftbl_plan_t p, cudaStream_t s, int ev) {
    p->hev_set[ev] = true;
    return check_cuda(p, cudaEventRecord(p->hev[ev], s), "event record");
}

// One transform with host input and output: upload `in_bytes` from src into
// stage_in (after the previous transform of this kind has read it), run
// `run` on the plan stream into stage_out (after the previous download of
// stage_out), download `out_bytes` into dst.
extern "C++" {   // a template: C++ linkage inside the C-ABI block
template <typename Run>
static nfftbl_status host_transform(nfftbl_plan_t p, const void* src, size_t in_bytes, DeviceBuf& stage_in, void* dst,
                                    size_t out_bytes, DeviceBuf& stage_out, int ev_in, int ev_done, int ev_out,
                                    Run run) {
    nfftbl_status st = host_streams(p);
    if (st != NFFTBL_OK) return st;
    const size_t cb = complex_bytes(p);
    if ((st = ensure_buf(p, stage_in, std::max(in_bytes, cb))) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, stage_out, std::max(out_bytes, cb))) != NFFTBL_OK) return st;
    if (in_bytes > 0) {
        if ((st = host_wait(p, p->s_up, ev_done)) != NFFTBL_OK) return st;
        if ((st = check_cuda(p, cudaMemcpyAsync(stage_in.p, src, in_bytes, cudaMemcpyHostToDevice, p->s_up),
                             "upload")) != NFFTBL_OK)
            return st;
        if ((st = host_record(p, p->s_up, ev_in)) != NFFTBL_OK) return st;
        if ((st = host_wait(p, p->stream, ev_in)) != NFFTBL_OK) return st;
    }
    if ((st = host_wait(p, p->stream, ev_out)) != NFFTBL_OK) return st;
    if ((st = run(stage_in.p, stage_out.p)) != NFFTBL_OK) return st;
    if ((st = host_record(p, p->stream, ev_done)) != NFFTBL_OK) return st;
    if (out_bytes > 0) {
        if ((st = host_wait(p, p->s_down, ev_done)) != NFFTBL_OK) return st;
        if ((st = check_cuda(p, cudaMemcpyAsync(dst, stage_out.p, out_bytes, cudaMemcpyDeviceToHost, p->s_down),
                             "download")) != NFFTBL_OK)
            return st;
        if ((st = host_record(p, p->s_down, ev_out)) != NFFTBL_OK) return st;
    }
    return NFFTBL_OK;
}
}  // extern "C++"

static size_t coeff_bytes(const nfftbl_plan_s* p) {
    size_t n = static_cast<size_t>(p->batch) * complex_bytes(p);
    for (int t = 0; t < p->d; ++t) n *= static_cast<size_t>(p->M[t]);
    return n;
}

nfftbl_status nfftbl_forward_host(nfftbl_plan_t p, const void* fhat_host, void* f_host) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!fhat_host || (!f_host && p->N > 0)) return fail(p, NFFTBL_EINVAL, "NULL data pointer");
    const size_t out_bytes = static_cast<size_t>(p->batch) * static_cast<size_t>(p->N) * complex_bytes(p);
    return host_transform(p, fhat_host, coeff_bytes(p), p->hs_fhat_in, f_host, out_bytes, p->hs_f_out,
                          nfftbl_plan_s::EV_IN_FWD, nfftbl_plan_s::EV_FWD_DONE, nfftbl_plan_s::EV_OUT_F,
                          [p](void* in, void* out) { return nfftbl_forward(p, in, out); });
}

nfftbl_status nfftbl_adjoint_host(nfftbl_plan_t p, const void* f_host, void* fhat_host) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!fhat_host || (!f_host && p->N > 0)) return fail(p, NFFTBL_EINVAL, "NULL data pointer");
    const size_t in_bytes = static_cast<size_t>(p->batch) * static_cast<size_t>(p->N) * complex_bytes(p);
    return host_transform(p, f_host, in_bytes, p->hs_f_in, fhat_host, coeff_bytes(p), p->hs_fhat_out,
                          nfftbl_plan_s::EV_IN_ADJ, nfftbl_plan_s::EV_ADJ_DONE, nfftbl_plan_s::EV_OUT_FHAT,
                          [p](void* in, void* out) { return nfftbl_adjoint(p, in, out); });
}

nfftbl_status nfftbl_join(nfftbl_plan_t p) {
    if (!p) return NFFTBL_EINVAL;
    nfftbl_status st = host_wait(p, p->stream, nfftbl_plan_s::EV_OUT_F);
    if (st == NFFTBL_OK) st = host_wait(p, p->stream, nfftbl_plan_s::EV_OUT_FHAT);
    return st;
}

nfftbl_status nfftbl_sync(nfftbl_plan_t p) {
    if (!p) return NFFTBL_EINVAL;
    nfftbl_status st;
    if (p->s_up && (st = check_cuda(p, cudaStreamSynchronize(p->s_up), "upload stream sync")) != NFFTBL_OK) return st;
    if (p->s_down && (st = check_cuda(p, cudaStreamSynchronize(p->s_down), "download stream sync")) != NFFTBL_OK)
        return st;
    if ((st = check_cuda(p, cudaMemcpyAsync(p->err_host, p->err.p, sizeof(int), cudaMemcpyDeviceToHost, p->stream),
                         "read err")) != NFFTBL_OK)
        return st;
    if ((st = check_cuda(p, cudaStreamSynchronize(p->stream), "stream sync")) != NFFTBL_OK) return st;
    const int e = *p->err_host;
    if (e) {
        cudaMemsetAsync(p->err.p, 0, sizeof(int), p->stream);
        cudaStreamSynchronize(p->stream);
        if (e & DEVERR_TIMEOUT) return fail(p, NFFTBL_ETIMEOUT, "a bounded device wait gave up");
        return fail(p, NFFTBL_EINTERNAL, "device error word set");
    }
    return NFFTBL_OK;
}

nfftbl_status nfftbl_set_wait_limit(nfftbl_plan_t p, int64_t limit_ns, int stall_next) {
    if (!p) return NFFTBL_EINVAL;
    if (limit_ns < 0 || limit_ns > 60000000000LL) return fail(p, NFFTBL_EINVAL, "limit_ns must be in [0, 6e10]");
    p->wait_ns = limit_ns ? static_cast<unsigned long long>(limit_ns) : kWaitLimitNs;
    p->stall_next = stall_next ? 1 : 0;
    return NFFTBL_OK;
}

nfftbl_status nfftbl_destroy(nfftbl_plan_t p) {
    if (!p) return NFFTBL_OK;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    if (p->s_up) cudaStreamSynchronize(p->s_up);
    if (p->s_down) cudaStreamSynchronize(p->s_down);
    destroy_plan(p);
    return NFFTBL_OK;
}

const char* nfftbl_last_error(nfftbl_plan_t p) {
    if (!p) return "NULL plan";
    return p->last_error.c_str();
}

const char* nfftbl_plan_error(void) { return g_plan_error.c_str(); }

nfftbl_status nfftbl_get_info(nfftbl_plan_t p, nfftbl_info* info) {
    if (!p || !info) return NFFTBL_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->d = p->d;
    for (int t = 0; t < 3; ++t) {
        info->M[t] = p->M[t];
        info->L[t] = p->L[t];
        info->tile[t] = p->geom.T[t];
    }
    info->m = p->m;
    info->precision = p->precision;
    info->method = p->method;
    info->window = p->window;
    info->batch = p->batch;
    info->beta = p->beta;
    info->n_nodes = p->N;
    info->n_tiles = p->n_tiles;
    info->n_work = p->n_work;
    info->key_bits = p->key_bits;
    info->poly_weights = p->poly_ok ? 1 : 0;
    info->poly_err = p->poly_err;
    return NFFTBL_OK;
}

nfftbl_status nfftbl_get_factors(nfftbl_plan_t p, int t, double* host_out) {
    if (!p || !host_out || t < 0 || t >= p->d) return NFFTBL_EINVAL;
    nfftbl_status st = check_cuda(p, cudaMemcpyAsync(host_out, p->fac64[t].p, p->M[t] * sizeof(double),
                                                     cudaMemcpyDeviceToHost, p->stream),
                                  "copy factors");
    if (st != NFFTBL_OK) return st;
    return check_cuda(p, cudaStreamSynchronize(p->stream), "sync");
}

nfftbl_status nfftbl_get_binning(nfftbl_plan_t p, uint32_t* keys, uint32_t* perm, uint32_t* tile_off) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    const size_t n = static_cast<size_t>(p->N) * 4;
    if (keys && n && (st = check_cuda(p, cudaMemcpyAsync(keys, p->keys.p, n, cudaMemcpyDeviceToHost, p->stream),
                                      "copy keys")) != NFFTBL_OK)
        return st;
    if (perm && n && (st = check_cuda(p, cudaMemcpyAsync(perm, p->perm.p, n, cudaMemcpyDeviceToHost, p->stream),
                                      "copy perm")) != NFFTBL_OK)
        return st;
    if (tile_off && (st = check_cuda(p, cudaMemcpyAsync(tile_off, p->tile_off.p, (p->n_tiles + 1) * 4,
                                                        cudaMemcpyDeviceToHost, p->stream),
                                     "copy tile_off")) != NFFTBL_OK)
        return st;
    return check_cuda(p, cudaStreamSynchronize(p->stream), "sync");
}

nfftbl_status nfftbl_get_grid(nfftbl_plan_t p, void* host_out) {
    if (!p || !host_out) return NFFTBL_EINVAL;
    const size_t bytes = static_cast<size_t>(p->batch) * prod_L(p) * complex_bytes(p);
    nfftbl_status st =
        check_cuda(p, cudaMemcpyAsync(host_out, p->grid.p, bytes, cudaMemcpyDeviceToHost, p->stream), "copy grid");
    if (st != NFFTBL_OK) return st;
    return check_cuda(p, cudaStreamSynchronize(p->stream), "sync");
}

nfftbl_status nfftbl_grid_ptr(nfftbl_plan_t p, void** grid_dev) {
    if (!p || !grid_dev) return NFFTBL_EINVAL;
    *grid_dev = p->grid.p;
    return NFFTBL_OK;
}

int64_t nfftbl_kernel_launches(nfftbl_plan_t p) { return p ? p->launches : 0; }

nfftbl_status nfftbl_set_window_table(nfftbl_plan_t p, const double* table_dev, int table_len) {
    if (!p || !table_dev) return NFFTBL_EINVAL;
    if (p->window != NFFTBL_WIN_TABLE) return fail(p, NFFTBL_ESTATE, "plan does not use a table window");
    if (table_len != static_cast<int>(p->table_host.size()))
        return fail(p, NFFTBL_EINVAL, "table length differs from the plan's");
    p->poly_ok = false;   // fitted to the host table the plan was made with: the closed form from here on
    const bool dbl = p->precision == NFFTBL_F64;
    void* t64 = dbl ? p->table_dev.p : p->table_dev64.p;
    nfftbl_status st = check_cuda(p, cudaMemcpyAsync(t64, table_dev, table_len * sizeof(double),
                                                     cudaMemcpyDeviceToDevice, p->stream),
                                  "table copy");
    if (st != NFFTBL_OK) return st;
    if (!dbl &&
        (st = check_cuda(p, launch_table_cast(static_cast<const double*>(t64), table_len,
                                              static_cast<float*>(p->table_dev.p),
                                              static_cast<float4*>(p->table_coef.p), p->stream),
                         "table cast")) != NFFTBL_OK)
        return st;
    if (!p->precorrect) return p->wfac_valid ? compute_factors(p) : NFFTBL_OK;   // D = I: no psi_hat
    for (int t = 0; t < p->d; ++t) {
        if ((st = check_cuda(p, launch_window_factors(1, NFFTBL_WIN_TABLE, p->L[t], p->M[t], p->m, p->beta,
                                                      static_cast<const double*>(t64), table_len - 1,
                                                      static_cast<double*>(p->fac64[t].p), p->stream),
                             "window factors")) != NFFTBL_OK)
            return st;
        if ((st = check_cuda(p, launch_cast_factors(static_cast<double*>(p->fac64[t].p), p->M[t], p->facT[t].p, dbl,
                                                    p->stream),
                             "factor cast")) != NFFTBL_OK)
            return st;
        p->launches += 2;
    }
    // stored factors follow the new table
    if (p->wfac_valid) return compute_factors(p);
    return NFFTBL_OK;
}

nfftbl_status nfftbl_window_loss_grad(nfftbl_plan_t p, const void* fhat_dev, const void* y_dev,
                                      double* grad_table_dev, double* loss_dev) {
    nfftbl_status st = ready(p);
    if (st != NFFTBL_OK) return st;
    if (!fhat_dev || !y_dev || !grad_table_dev || !loss_dev) return fail(p, NFFTBL_EINVAL, "NULL pointer");
    if (p->window != NFFTBL_WIN_TABLE || p->method != NFFTBL_SHANNON || !p->precorrect)
        return fail(p, NFFTBL_ESTATE, "window gradients need a precorrected Shannon plan with a table window");
    if (p->precision == NFFTBL_F64 || p->d > 2)
        return fail(p, NFFTBL_EUNSUPPORTED, "window gradients are built for FP32 plans with d <= 2");
    const long long B = p->batch, N = p->N;
    long long pm = 1;
    int msum = 0;
    for (int t = 0; t < p->d; ++t) {
        pm *= p->M[t];
        msum += p->M[t];
    }
    if ((st = ensure_buf(p, p->lw_f, B * N * 8)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->lw_h, B * pm * 8)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->lw_marg, msum * 8)) != NFFTBL_OK) return st;
    if ((st = ensure_buf(p, p->lw_dpsi, msum * 8)) != NFFTBL_OK) return st;
    const int n = static_cast<int>(p->table_host.size()) - 1;
    cudaStream_t s = p->stream;
    if ((st = check_cuda(p, cudaMemsetAsync(loss_dev, 0, 3 * sizeof(double), s), "clear loss")) != NFFTBL_OK)
        return st;
    if ((st = check_cuda(p, cudaMemsetAsync(grad_table_dev, 0, (n + 1) * sizeof(double), s), "clear grad")) !=
        NFFTBL_OK)
        return st;
    if ((st = check_cuda(p, cudaMemsetAsync(p->lw_marg.p, 0, msum * 8, s), "clear marginals")) != NFFTBL_OK)
        return st;
    // forward into the scratch f, then r = f - y in place and the loss
    if ((st = fft_forward(p, fhat_dev)) != NFFTBL_OK) return st;
    if ((st = taps(p, TAP_INTERP, nullptr, p->lw_f.p, nullptr)) != NFFTBL_OK) return st;
    if ((st = check_cuda(p, launch_residual(0, p->lw_f.p, y_dev, B * N, loss_dev, s), "residual")) != NFFTBL_OK)
        return st;
    // (A) through the tap weights (the grid still holds vartheta)
    TapArgs<float> a = make_tap_args<float>(p);
    a.fin = static_cast<const float2*>(p->lw_f.p);
    if ((st = run_table_grad(p, a, loss_dev, grad_table_dev)) != NFFTBL_OK) return st;
    // (B) through the precorrection: hhat = D F^H Psi^T r, marginals, quadrature
    if ((st = taps(p, TAP_SPREAD, p->lw_f.p, nullptr, nullptr)) != NFFTBL_OK) return st;
    if ((st = fft_adjoint(p, p->lw_h.p)) != NFFTBL_OK) return st;
    double* marg = static_cast<double*>(p->lw_marg.p);
    double* dpsi = static_cast<double*>(p->lw_dpsi.p);
    double* Pt[3] = {marg, marg, marg};
    int off = 0;
    for (int t = 0; t < p->d; ++t) {
        Pt[t] = marg + off;
        off += p->M[t];
    }
    if ((st = check_cuda(p, launch_marginals(0, p->lw_h.p, fhat_dev, B * pm, p->d, p->M, Pt[0], Pt[1], Pt[2], s),
                         "marginals")) != NFFTBL_OK)
        return st;
    off = 0;
    for (int t = 0; t < p->d; ++t) {
        if ((st = check_cuda(p, launch_dEdpsihat(marg + off, static_cast<const double*>(p->fac64[t].p), p->M[t], p->L[t],
                                                 loss_dev, dpsi + off, s),
                             "dE/dpsihat")) != NFFTBL_OK)
            return st;
        if ((st = check_cuda(p, launch_window_table_grad(p->L[t], p->M[t], p->m, n, dpsi + off, grad_table_dev, s),
                             "quadrature gradient")) != NFFTBL_OK)
            return st;
        off += p->M[t];
        p->launches += 2;
    }
    p->launches += 3;
    return NFFTBL_OK;
}

nfftbl_status nfftbl_kernel_timing(nfftbl_plan_t p, int enable) {
    if (!p) return NFFTBL_EINVAL;
    double ms[NFFTBL_K_COUNT];
    int64_t cnt[NFFTBL_K_COUNT];
    nfftbl_status st = nfftbl_kernel_times(p, ms, cnt);   // drain and reset
    p->timing = enable != 0;
    return st;
}

nfftbl_status nfftbl_kernel_times(nfftbl_plan_t p, double* ms_out, int64_t* count_out) {
    if (!p || !ms_out || !count_out) return NFFTBL_EINVAL;
    for (int k = 0; k < NFFTBL_K_COUNT; ++k) {
        ms_out[k] = 0.0;
        count_out[k] = 0;
    }
    nfftbl_status st = NFFTBL_OK;
    for (auto& t : p->timed) {
        if (t.a && t.b && st == NFFTBL_OK) {
            float ms = 0.f;
            st = check_cuda(p, cudaEventSynchronize(t.b), "timing event sync");
            if (st == NFFTBL_OK) st = check_cuda(p, cudaEventElapsedTime(&ms, t.a, t.b), "timing elapsed");
            if (st == NFFTBL_OK && t.kind >= 0 && t.kind < NFFTBL_K_COUNT) {
                ms_out[t.kind] += ms;
                count_out[t.kind] += 1;
            }
        }
        if (t.a) p->event_pool.push_back(t.a);
        if (t.b) p->event_pool.push_back(t.b);
    }
    p->timed.clear();
    return st;
}

}  // extern "C"
