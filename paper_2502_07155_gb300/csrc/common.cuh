// Device-side helpers shared by the nfftbl kernels (sm_103a).
//
// - complex value types per precision;
// - mbarrier / TMA (cp.async.bulk.tensor) wrappers in inline PTX;
// - a bounded mbarrier wait that gives up after a wall-clock limit and
//   reports through a device error word instead of hanging the GPU.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nfftbl {

// Device error word bits (OR-ed by kernels, read by the host).
enum : int {
    DEVERR_DOMAIN = 1,      // a node outside [-1/2, 1/2) or NaN
    DEVERR_TIMEOUT = 2,     // a bounded wait gave up
    DEVERR_INTERNAL = 4,    // an index check failed
};

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using C2 = typename Cplx<T>::type;

template <typename T>
__device__ __forceinline__ C2<T> cmake(T r, T i) { C2<T> z; z.x = r; z.y = i; return z; }

// acc + v * w componentwise for a pair v and a scalar w.  FP32 pairs take one
// packed FMA (fma.rn.f32x2, sm_100 and later): each component is an IEEE fma
// rounded to nearest, so the result equals two fmaf calls bit for bit while
// issuing one instruction instead of two.
__device__ __forceinline__ float2 cfma(float2 v, float w, float2 acc) {
    return __ffma2_rn(v, make_float2(w, w), acc);
}
__device__ __forceinline__ double2 cfma(double2 v, double w, double2 acc) {
    acc.x = fma(v.x, w, acc.x);
    acc.y = fma(v.y, w, acc.y);
    return acc;
}

// One work item of the interpolation / spreading kernels: a tile and a run of
// its nodes in sorted order.
struct WorkItem {
    int tile;
    int start;
    int count;
    int pad;
};

// Upper bound on any device-side wait, in nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\t"
                 "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, at most limit_ns (default
// kWaitLimitNs).  Returns false (and sets DEVERR_TIMEOUT) if the limit passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) {
            atomicOr(err, DEVERR_TIMEOUT);
            return false;
        }
    }
}

// TMA tiled loads of a box into shared memory, completing on `bar`.
// Coordinates are element indices, innermost first.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(smem_addr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(smem_addr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 :: "r"(smem_addr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" :: "l"(map) : "memory");
}

// Round-to-nearest multiply that the compiler may not contract into an FMA
// (used where a float product decides an integer cell index).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Add val * d(table(u))/d(v_i) to tab_grad for the four entries of the
// Catmull-Rom stencil at u in [0, 1] (table v_0..v_n, ghost values
// v_{-1} = v_1 and v_{n+1} = 2 v_n - v_{n-1} folded back).
__device__ __forceinline__ void scatter_catmull(double* tab_grad, int n, double u, double val) {
    const double s = fmin(fmax(u, 0.0), 1.0) * n;
    const int i = min(static_cast<int>(floor(s)), n - 1);
    const double t = s - i;
    const double c0 = 0.5 * (-t + 2.0 * t * t - t * t * t);
    const double c1 = 0.5 * (2.0 - 5.0 * t * t + 3.0 * t * t * t);
    const double c2 = 0.5 * (t + 4.0 * t * t - 3.0 * t * t * t);
    const double c3 = 0.5 * (-t * t + t * t * t);
    atomicAdd(&tab_grad[(i == 0) ? 1 : i - 1], val * c0);
    atomicAdd(&tab_grad[i], val * c1);
    atomicAdd(&tab_grad[i + 1], val * c2);
    if (i + 2 <= n) {
        atomicAdd(&tab_grad[i + 2], val * c3);
    } else {
        atomicAdd(&tab_grad[n], 2.0 * val * c3);
        atomicAdd(&tab_grad[n - 1], -val * c3);
    }
}

}  // namespace nfftbl
