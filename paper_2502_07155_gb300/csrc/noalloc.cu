// Equispaced samples (steps 1-2 of the forward transform) without any
// device allocation, for callers that cannot call cudaMalloc: code running
// inside another framework's memory pool or allocator hooks, or a host
// environment that only hands out buffers it allocated itself.  Every
// intermediate lives in one file-scope device array of fixed size; the
// caller passes only its input and output buffers.
#include <cmath>
#include <mutex>

#include "plan_internal.h"

namespace nfftbl {
namespace {

// Fixed scratch for nfftbl_grid_noalloc.  Every GPU that loads the library
// holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

// Parameters whose window factors and twiddles the array of a device holds
// (written by the last call that launched them).  A call with the same
// parameters reuses them instead of repeating the quadrature.
struct FactorKey {
    bool valid = false;
    int d = 0, M[3] = {0, 0, 0}, L[3] = {0, 0, 0}, m = 0;
    double beta = 0.0;
    bool operator==(const FactorKey& o) const {
        if (valid != o.valid || d != o.d || m != o.m || beta != o.beta) return false;
        for (int t = 0; t < 3; ++t)
            if (M[t] != o.M[t] || L[t] != o.L[t]) return false;
        return true;
    }
};
FactorKey g_factor_key[kMaxDevices];

nfftbl_status noalloc_fail(nfftbl_status st, const std::string& msg) {
    set_plan_error(msg);   // readable through nfftbl_plan_error()
    return st;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// L = 2^a 3^b 5^c, the lengths the mixed-radix FFT pass handles
bool radix235(long long v) {
    if (v <= 0) return false;
    for (int r : {2, 3, 5})
        while (v % r == 0) v /= r;
    return v == 1;
}

}  // namespace

}  // namespace nfftbl

using namespace nfftbl;

extern "C" nfftbl_status nfftbl_grid_noalloc(int d, const int* M, double sigma, int m, double beta, int batch,
                                             const void* fhat_dev, void* grid_dev, void* cuda_stream) {
    set_plan_error("");
    if (d < 1 || d > 3 || !M) return noalloc_fail(NFFTBL_EINVAL, "d must be 1..3 and M non-NULL");
    if (!(sigma >= 1.0) || !std::isfinite(sigma)) return noalloc_fail(NFFTBL_EINVAL, "sigma must be >= 1");
    if (batch < 1) return noalloc_fail(NFFTBL_EINVAL, "batch must be >= 1");
    if (!fhat_dev || !grid_dev) return noalloc_fail(NFFTBL_EINVAL, "NULL data pointer");
    int L[3] = {1, 1, 1};
    for (int t = 0; t < d; ++t) {
        if (M[t] < 2 || (M[t] & 1)) return noalloc_fail(NFFTBL_EINVAL, "each M_t must be even and >= 2");
        if (M[t] > 4096) return noalloc_fail(NFFTBL_EUNSUPPORTED, "L_t must be of the form 2^a 3^b 5^c in [16, 4096]");
        const long long s = static_cast<long long>(std::ceil(sigma * M[t] - 1e-9));
        L[t] = static_cast<int>(std::min<long long>(2 * ((s + 1) / 2), 1 << 20));
        if (2 * m >= L[t]) return noalloc_fail(NFFTBL_EINVAL, "2m must be < L_t");
    }
    for (int t = 0; t < d; ++t)
        if (!radix235(L[t]) || L[t] < 16 || L[t] > 4096)
            return noalloc_fail(NFFTBL_EUNSUPPORTED, "L_t must be of the form 2^a 3^b 5^c in [16, 4096]");
    if (m < 2 || m > 12) return noalloc_fail(NFFTBL_EUNSUPPORTED, "m must be in 2..12");
    if (!(beta > 0.0)) beta = M_PI * m * (1.0 - 1.0 / sigma);
    if (!(beta > 0.0)) return noalloc_fail(NFFTBL_EINVAL, "beta must be > 0 (sigma = 1 needs an explicit beta)");

    // scratch layout: per dimension fac64 (M doubles), fac (M floats),
    // twiddles (L float2); then the pass intermediates.  Every extent is at
    // most 4096, so the per-batch sizes below fit in 64 bits; the batch is
    // bounded before it multiplies them.
    size_t off = 0;
    size_t o_fac64[3], o_fac[3], o_tw[3];
    for (int t = 0; t < d; ++t) {
        o_fac64[t] = off;
        off = align256(off + M[t] * sizeof(double));
        o_fac[t] = off;
        off = align256(off + M[t] * sizeof(float));
        o_tw[t] = off;
        off = align256(off + L[t] * sizeof(float2));
    }
    size_t per_batch_a = 0, per_batch_b = 0;
    if (d == 2) {
        per_batch_a = static_cast<size_t>(M[0]) * L[1] * sizeof(float2);
    } else if (d == 3) {
        per_batch_a = static_cast<size_t>(M[0]) * M[1] * L[2] * sizeof(float2);
        per_batch_b = static_cast<size_t>(M[0]) * L[1] * L[2] * sizeof(float2);
    }
    const size_t fixed = off;
    const size_t per_batch = per_batch_a + per_batch_b;
    if (fixed > kNoAllocScratchBytes ||
        (per_batch > 0 && static_cast<size_t>(batch) > (kNoAllocScratchBytes - fixed) / per_batch))
        return noalloc_fail(NFFTBL_EINVAL, "problem needs about " +
                                               std::to_string(static_cast<unsigned long long>(
                                                   static_cast<double>(fixed) + static_cast<double>(batch) * per_batch)) +
                                               " bytes of scratch; nfftbl_grid_noalloc has 16777216 (16 MiB)");
    const long long B = batch;
    size_t o_a = off, o_b = off;
    if (d == 2) {
        off = align256(off + static_cast<size_t>(B) * per_batch_a);
    } else if (d == 3) {
        off = align256(off + static_cast<size_t>(B) * per_batch_a);
        o_b = off;
        off = align256(off + static_cast<size_t>(B) * per_batch_b);
    }
    if (off > kNoAllocScratchBytes)
        return noalloc_fail(NFFTBL_EINVAL, "problem needs " + std::to_string(off) +
                                               " bytes of scratch; nfftbl_grid_noalloc has 16777216 (16 MiB)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(NFFTBL_ECUDA, "cudaGetDevice failed");
    }
    FactorKey key;
    key.valid = true;
    key.d = d;
    key.m = m;
    key.beta = beta;
    for (int t = 0; t < d; ++t) {
        key.M[t] = M[t];
        key.L[t] = L[t];
    }
    unsigned char* base = nullptr;
    bool reuse = false;
    {
        // one-time set-up per device, with that device current: the array's
        // device address and the quadrature rule (a synchronous copy), so that
        // later calls only launch kernels
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return noalloc_fail(NFFTBL_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            const cudaError_t e2 = upload_gl_rule_sync();
            if (e2 != cudaSuccess) {
                cudaGetLastError();
                return noalloc_fail(NFFTBL_ECUDA, std::string("quadrature rule upload: ") + cudaGetErrorString(e2));
            }
            g_scratch_ptr[dev] = ptr;
        }
        base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
        reuse = g_factor_key[dev] == key;
        if (!reuse) g_factor_key[dev] = FactorKey{};   // invalid until this call's launches succeed
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < d && e == cudaSuccess && !reuse; ++t) {
        double* fac64 = reinterpret_cast<double*>(base + o_fac64[t]);
        e = launch_window_factors_preloaded(1, NFFTBL_WIN_SINH, L[t], M[t], m, beta, fac64, s);
        if (e == cudaSuccess) e = launch_cast_factors(fac64, M[t], base + o_fac[t], 0, s);
        if (e == cudaSuccess) e = launch_twiddles(L[t], base + o_tw[t], 0, s);
    }
    const void* src = fhat_dev;
    for (int t = d - 1; t >= 0 && e == cudaSuccess; --t) {
        long long outer = B, inner = 1;
        for (int q = 0; q < t; ++q) outer *= M[q];
        for (int q = t + 1; q < d; ++q) inner *= L[q];
        void* dst = (t == 0) ? grid_dev : base + ((t == d - 1) ? o_a : o_b);
        e = launch_fft_forward_pass_f32(src, dst, outer, inner, M[t], L[t],
                                        reinterpret_cast<const float*>(base + o_fac[t]), base + o_tw[t], s);
        src = dst;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(NFFTBL_ECUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    }
    if (!reuse) {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        g_factor_key[dev] = key;
    }
    return NFFTBL_OK;
}
