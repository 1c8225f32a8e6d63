// Short-sum kernels over binned nodes: interpolation (Algorithm 4.2 step 3,
// Eq. 4.8), spreading (its transpose Psi^T, the first factor of the
// adjoint), the node derivative of the short sums and the optional stored
// window factors (step 0b in tensor-product form).
//
// Work decomposition: one work item = one tile of T_0 x .. x T_{d-1} grid
// cells and up to K of its nodes (sorted by cell).  The box of grid values
// the tile's nodes can reach -- the tile plus its m-halo -- lives in shared
// memory: interp_kernel / node_grad_kernel stage it with one TMA tiled load
// (out-of-range cells are zero-filled by the copy engine, which is exactly
// the zero extension of the Shannon method outside I_L) and evaluate one
// node per thread; the spread kernels (spread1/2/3_kernel) accumulate it in
// exact fixed point, warps walking the item's nodes, and store it for the
// ordered flush (gather_kernel).
//
// Per node and dimension t: u = L_t x_t (one correctly rounded product,
// exact for L_t = 2^p), cell i = floor(u), tau = u - i in [0, 1).  The 2m
// taps l = i-m+1 .. i+m (the members of the closed set J_{L,m}(x) with a
// nonzero window; the ends of the closed set carry phi(+-m/L) = 0) have
// offsets delta_a = L x - l = tau + m-1-a, and
//   sinc(pi delta_a) = (-1)^(m-1-a) sin(pi tau) / (pi delta_a),
// so one sinpi per node and dimension serves all taps.  The tensor-product
// kernel psi(x - l/L) = prod_t psi_t is contracted dimension by dimension:
// rows of 2m taps along the contiguous dimension first.
#pragma once

#include <algorithm>

#include "plan_internal.h"

namespace nfftbl {

constexpr int kTapThreads = 256;
constexpr double kPiD = 3.14159265358979323846;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> struct FM;
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <> struct FM<float> {
    // window arithmetic of the FP32 path: hardware 2^x, reciprocal and
    // reciprocal square root, one SFU operation each (a few ulp; flush-to-
    // zero: callers keep the arguments normal)
    __device__ static float exp2w(float x) { return ex2_approx(x); }
    __device__ static float sqrtw(float x) { return x * rsqrt_approx(x); }
    __device__ static float rcpw(float x) { return rcp_approx(x); }
    __device__ static float sinpi(float x) { return sinpif(x); }
    __device__ static float cospi(float x) { return cospif(x); }
    __device__ static float sqrt(float x) { return sqrtf(x); }
    __device__ static float exp2(float x) { return exp2f(x); }
    __device__ static float div(float a, float b) { return __fdividef(a, b); }
    __device__ static float i0(float x) { return cyl_bessel_i0f(x); }
    __device__ static float i1(float x) { return cyl_bessel_i1f(x); }
    __device__ static float abs(float x) { return fabsf(x); }
    __device__ static float flr(float x) { return floorf(x); }
};
template <> struct FM<double> {
    __device__ static double exp2w(double x) { return ::exp2(x); }
    __device__ static double sqrtw(double x) { return ::sqrt(x); }
    __device__ static double rcpw(double x) { return 1.0 / x; }
    __device__ static double sinpi(double x) { return ::sinpi(x); }
    __device__ static double cospi(double x) { return ::cospi(x); }
    __device__ static double sqrt(double x) { return ::sqrt(x); }
    __device__ static double exp2(double x) { return ::exp2(x); }
    __device__ static double div(double a, double b) { return a / b; }
    __device__ static double i0(double x) { return cyl_bessel_i0(x); }
    __device__ static double i1(double x) { return cyl_bessel_i1(x); }
    __device__ static double abs(double x) { return fabs(x); }
    __device__ static double flr(double x) { return floor(x); }
};

// Catmull-Rom evaluation of a window table v_i = g(i/n), i = 0..n, at
// u in [0, 1]; ghost values v_{-1} = v_1 (even window) and
// v_{n+1} = 2 v_n - v_{n-1}.
template <typename T>
__device__ __forceinline__ void table_coeffs(const T* __restrict__ v, int n, T u, T& p0, T& p1, T& p2, T& p3,
                                             T& t) {
    const T s = u * static_cast<T>(n);
    int i = static_cast<int>(FM<T>::flr(s));
    i = min(max(i, 0), n - 1);
    t = s - static_cast<T>(i);
    p0 = (i == 0) ? v[1] : v[i - 1];
    p1 = v[i];
    p2 = v[i + 1];
    p3 = (i + 2 <= n) ? v[i + 2] : T(2) * v[n] - v[n - 1];
}

template <typename T>
__device__ __forceinline__ T table_eval(const T* __restrict__ v, int n, T u) {
    T p0, p1, p2, p3, t;
    table_coeffs(v, n, u, p0, p1, p2, p3, t);
    return T(0.5) * (T(2) * p1 + (p2 - p0) * t + (T(2) * p0 - T(5) * p1 + T(4) * p2 - p3) * t * t +
                     (T(3) * p1 - p0 - T(3) * p2 + p3) * t * t * t);
}

template <typename T>
__device__ __forceinline__ T table_deriv(const T* __restrict__ v, int n, T u) {
    T p0, p1, p2, p3, t;
    table_coeffs(v, n, u, p0, p1, p2, p3, t);
    const T dt = T(0.5) * ((p2 - p0) + T(2) * (T(2) * p0 - T(5) * p1 + T(4) * p2 - p3) * t +
                           T(3) * (T(3) * p1 - p0 - T(3) * p2 + p3) * t * t);
    return dt * static_cast<T>(n);
}

// The fields of WinParams the out-of-line window routines read (passed by
// value: small, unlike the whole parameter block with its polynomials).
template <typename T>
struct WinLite {
    int window;
    T inv_m, beta, c_norm;
    const T* table;
    int table_n;
};

template <typename T>
__device__ __forceinline__ WinLite<T> win_lite(const WinParams<T>& w) {
    return WinLite<T>{w.window, w.inv_m, w.beta, w.c_norm, w.table, w.table_n};
}

// Kaiser-Bessel and tabulated windows, kept out of line: they are rare and
// their code would otherwise be inlined into every unrolled tap.
template <typename T>
__device__ __noinline__ T win_phi_other(T delta, const WinLite<T> w) {
    const T r = delta * w.inv_m;
    const T q = (T(1) - r) * (T(1) + r);
    if (!(q > T(0))) return T(0);
    if (w.window == NFFTBL_WIN_CKB) return (FM<T>::i0(w.beta * FM<T>::sqrt(q)) - T(1)) * w.c_norm;
    return table_eval(w.table, w.table_n, FM<T>::abs(r));
}

template <typename T>
__device__ __noinline__ T win_dphi_other(T delta, const WinLite<T> w) {
    const T r = delta * w.inv_m;
    const T q = (T(1) - r) * (T(1) + r);
    if (!(q > T(0))) return T(0);
    if (w.window == NFFTBL_WIN_TABLE) {
        const T g = table_deriv(w.table, w.table_n, FM<T>::abs(r)) * w.inv_m;
        return (r < T(0)) ? -g : g;
    }
    const T sq = FM<T>::sqrt(q);
    return w.beta * FM<T>::i1(w.beta * sq) * w.c_norm * (-r * w.inv_m / sq);
}

// Window Phi(delta) = phi(delta / L) for a tap offset delta = L x - l in grid units.
template <typename T>
__device__ __forceinline__ T win_phi(T delta, const WinParams<T>& w) {
    if (w.window != NFFTBL_WIN_SINH) return win_phi_other(delta, win_lite(w));
    const T r = delta * w.inv_m;
    const T q = (T(1) - r) * (T(1) + r);
    if (!(q > T(0))) return T(0);
    // sinh(beta s)/sinh(beta) = (e^{beta(s-1)} - e^{-beta(s+1)}) / (1 - e^{-2 beta}),
    // with s - 1 = -r^2 / (1 + s) (no cancellation)
    const T sq = FM<T>::sqrtw(q);
    const T one_sq = T(1) + sq;
    return (FM<T>::exp2w(-w.c_exp * FM<T>::div(r * r, one_sq)) - FM<T>::exp2w(-w.c_exp * one_sq)) * w.c_norm;
}

// d Phi / d delta; zero where |delta| >= m (the infinite edge derivative of
// the sinh / Kaiser-Bessel windows meets a vanishing factor there).
template <typename T>
__device__ __forceinline__ T win_dphi(T delta, const WinParams<T>& w) {
    if (w.window != NFFTBL_WIN_SINH) return win_dphi_other(delta, win_lite(w));
    const T r = delta * w.inv_m;
    const T q = (T(1) - r) * (T(1) + r);
    if (!(q > T(0))) return T(0);
    const T sq = FM<T>::sqrtw(q);
    const T one_sq = T(1) + sq;
    const T ds = -r * w.inv_m / sq;
    return w.beta * (FM<T>::exp2w(-w.c_exp * FM<T>::div(r * r, one_sq)) + FM<T>::exp2w(-w.c_exp * one_sq)) *
           w.c_norm * ds;
}

// Tap count per dimension: W = 2m fixed at compile time, or W = 0 for a
// kernel that takes m at run time (arrays sized for m <= 12).
template <int W> struct TapN {
    static constexpr int A = W ? W : 24;
};

// One Shannon / sinh tap weight (the FAST case of tap_weights) for tap a;
// sn = sin(pi tau) times the window's normalisation 1 / sinh(beta)
// (sinh_sin() below; one product per node instead of one per weight).
//
// The exponent beta (sqrt(q) - 1) / ln 2 (up to 18 at m = 8) would multiply
// the relative error of sqrt(q) by that much; it is evaluated as
// -c r^2 / (1 + sqrt(q)) instead, where that error is damped.  The two
// reciprocals 1/(1 + sqrt(q)) and the sinc's 1/(pi delta) are separate SFU
// operations: the kernels that use this routine are bound by instruction
// issue, not by the SFU.
template <typename T>
__device__ __forceinline__ T shannon_sinh_weight(T tau, T sn, int a, int m, const WinParams<T>& wp) {
    const int n = m - 1 - a;
    const T delta = tau + static_cast<T>(n);
    const T r = delta * wp.inv_m;
    const T q = fma(-r, r, T(1));
    const bool in = q > T(1e-30);   // below: the weight is < 1e-13 (and keeps FP32 operands normal)
    const T sq = FM<T>::sqrtw(in ? q : T(1));
    const T one_sq = T(1) + sq;
    const bool centre = delta == T(0);
    const T inv1 = FM<T>::rcpw(one_sq);                  // 1 / (1 + sqrt q)
    const T e1 = FM<T>::exp2w(-wp.c_exp * (r * r) * inv1);
    const T e2 = FM<T>::exp2w(-wp.c_exp * one_sq);
    const T num = (n & 1) ? -sn : sn;
    const T sc = centre ? wp.c_norm : num * FM<T>::rcpw(static_cast<T>(kPiD) * (centre ? T(1) : delta));
    return in ? sc * (e1 - e2) : T(0);
}


// Weight kinds of the inline paths (chosen once per kernel from the plan).
enum : int {
    WK_GENERIC = 0,     // any window / method: per-tap dispatch (out of line for cKB, table)
    WK_SINH = 1,        // Shannon method, sinh window
    WK_TABLE = 2,       // Shannon method, tabulated window (the learned phi_theta)
    WK_CSINH = 3,       // classical method (Algorithm 2.1), sinh window
    WK_POLY = 4,        // FP32, any window and method: the plan's per-tap weight polynomials
};

// The sine factor the Shannon weights of kind WK take: sin(pi tau), times
// the sinh window's normalisation for WK_SINH.
template <typename T, int WK>
__device__ __forceinline__ T kind_sin(T tau, const WinParams<T>& wp) {
    if constexpr (WK == WK_POLY || WK == WK_CSINH) return T(0);
    const T s = FM<T>::sinpi(tau);
    return (WK == WK_SINH) ? s * wp.c_norm : s;
}

// Tap a's weight from the plan's polynomial (WK_POLY): Horner in
// t = 2 tau - 1 over kPolyDeg + 1 coefficients (operands of the kernel's
// parameter block when a is a compile-time index), times
// sqrt(1 - (delta/m)^2) at the two edge taps of a square-root-edged window.
template <typename T>
__device__ __forceinline__ T poly_weight(T tau, int a, int m, const WinParams<T>& wp) {
    if constexpr (sizeof(T) == 4) {
        const float t = fmaf(2.0f, tau, -1.0f);
        float v = wp.pc[a][kPolyDeg];
#pragma unroll
        for (int k = kPolyDeg - 1; k >= 0; --k) v = fmaf(v, t, wp.pc[a][k]);
        if (wp.poly_edge_sqrt && (a == 0 || a == 2 * m - 1)) {
            const float r = (tau + static_cast<float>(m - 1 - a)) * wp.inv_m;
            const float q = fmaf(-r, r, 1.0f);
            v = (q > 1e-30f) ? v * (q * rsqrt_approx(q)) : 0.0f;
        }
        return v;
    } else {
        return T(0);   // (FP64 plans have no polynomials)
    }
}

// The weight kind of the window's closed form (the polynomials aside).
template <typename T>
__device__ __forceinline__ int closed_kind(const WinParams<T>& w) {
    if (w.method != NFFTBL_SHANNON) return (w.window == NFFTBL_WIN_SINH) ? WK_CSINH : WK_GENERIC;
    if (w.window == NFFTBL_WIN_SINH) return WK_SINH;
    if (w.window == NFFTBL_WIN_TABLE) return WK_TABLE;
    return WK_GENERIC;
}

template <typename T>
__device__ __forceinline__ int weight_kind(const WinParams<T>& w) {
    if (sizeof(T) == 4 && w.poly) return WK_POLY;
    if (w.method != NFFTBL_SHANNON) return (w.window == NFFTBL_WIN_SINH) ? WK_CSINH : WK_GENERIC;
    if (w.window == NFFTBL_WIN_SINH) return WK_SINH;
    if (w.window == NFFTBL_WIN_TABLE) return WK_TABLE;
    return WK_GENERIC;
}

// One Shannon / tabulated-window tap weight: sinc(pi delta) times the
// Catmull-Rom interpolant of the table at u = |delta| / m (zero for u >= 1),
// the table read through the read-only data cache.
template <typename T>
__device__ __forceinline__ T shannon_table_weight(T tau, T s, int a, int m, const WinParams<T>& wp) {
    const int n = m - 1 - a;
    const T delta = tau + static_cast<T>(n);
    const T u = FM<T>::abs(delta) * wp.inv_m;
    const bool centre = delta == T(0);
    const T num = (n & 1) ? -s : s;
    const T sc = centre ? T(1) : num * FM<T>::rcpw(static_cast<T>(kPiD) * delta);
    const int tn = wp.table_n;
    const T sx = u * static_cast<T>(tn);
    int i = static_cast<int>(FM<T>::flr(sx));
    i = min(max(i, 0), tn - 1);
    const T t = sx - static_cast<T>(i);
    if constexpr (sizeof(T) == 4) {
        if (wp.tcoef) {   // one 16-byte load per weight
            const float4 c = __ldg(wp.tcoef + i);
            const T ph = fma(fma(fma(c.w, t, c.z), t, c.y), t, c.x);
            return (u < T(1)) ? sc * ph : T(0);
        }
    }
    const T* v = wp.table;
    const T p1 = __ldg(v + i), p2 = __ldg(v + i + 1);
    const T p0 = (i == 0) ? __ldg(v + 1) : __ldg(v + i - 1);
    const T p3 = (i + 2 <= tn) ? __ldg(v + i + 2) : T(2) * __ldg(v + tn) - __ldg(v + tn - 1);
    const T ph = T(0.5) * (T(2) * p1 + (p2 - p0) * t + (T(2) * p0 - T(5) * p1 + T(4) * p2 - p3) * t * t +
                           (T(3) * p1 - p0 - T(3) * p2 + p3) * t * t * t);
    return (u < T(1)) ? sc * ph : T(0);
}

// One classical-method tap weight (Algorithm 2.1) of the sinh window,
// phi(delta) = sinh(beta sqrt(q)) / sinh(beta) with q = 1 - (delta/m)^2, zero
// for |delta| >= m: the exponent pair of shannon_sinh_weight, one reciprocal,
// no sinc factor.
template <typename T>
__device__ __forceinline__ T classic_sinh_weight(T tau, int a, int m, const WinParams<T>& wp) {
    const int n = m - 1 - a;
    const T delta = tau + static_cast<T>(n);
    const T r = delta * wp.inv_m;
    const T q = fma(-r, r, T(1));
    const bool in = q > T(1e-30);
    const T sq = FM<T>::sqrtw(in ? q : T(1));
    const T one_sq = T(1) + sq;
    const T rc = FM<T>::rcpw(one_sq);
    const T e1 = FM<T>::exp2w(-wp.c_exp * (r * r) * rc);
    const T e2 = FM<T>::exp2w(-wp.c_exp * one_sq);
    return in ? (e1 - e2) * wp.c_norm : T(0);
}

// Tap weight a of the inline kind WK (not WK_GENERIC); s = sin(pi tau) is
// used by the Shannon kinds only.
template <typename T, int WK>
__device__ __forceinline__ T fast_weight(T tau, T s, int a, int m, const WinParams<T>& wp) {
    if constexpr (WK == WK_POLY) return poly_weight(tau, a, m, wp);
    else if constexpr (WK == WK_TABLE) return shannon_table_weight(tau, s, a, m, wp);
    else if constexpr (WK == WK_CSINH) return classic_sinh_weight(tau, a, m, wp);
    else return shannon_sinh_weight(tau, s, a, m, wp);
}

// The 2m tap weights psi_t(x - l/L) (Shannon) or phi_t(x - l/L) (classical)
// of one dimension, tap a at l = i - m + 1 + a.  WK = WK_SINH / WK_TABLE
// evaluates the Shannon method with the sinh / tabulated window inline with
// no per-tap dispatch; the caller checks that the plan is of that kind.
template <typename T, int W, int WK = WK_GENERIC>
__device__ __forceinline__ void tap_weights(T tau, const WinParams<T>& wp, T (&w)[TapN<W>::A]) {
    const int m = W ? W / 2 : wp.m;
    const int nw = 2 * m;
    if (WK != WK_GENERIC) {
        const T s = kind_sin<T, WK>(tau, wp);
#pragma unroll
        for (int a = 0; a < TapN<W>::A; ++a)
            if (a < nw) w[a] = fast_weight<T, WK>(tau, s, a, m, wp);
        return;
    }
    if (wp.method == NFFTBL_SHANNON) {
        const T s = FM<T>::sinpi(tau);
#pragma unroll
        for (int a = 0; a < nw; ++a) {
            const int n = m - 1 - a;
            const T delta = tau + static_cast<T>(n);
            const T num = (n & 1) ? -s : s;
            const T sc = (delta == T(0)) ? T(1) : FM<T>::div(num, static_cast<T>(kPiD) * delta);
            w[a] = sc * win_phi(delta, wp);
        }
    } else {
#pragma unroll
        for (int a = 0; a < nw; ++a) w[a] = win_phi(tau + static_cast<T>(m - 1 - a), wp);
    }
}

// Write the 2m tap weights of two dimensions to d0[0 .. 2m-1] and
// d1[0 .. 2m-1] (shared memory), the two dimensions' chains interleaved.
template <typename T, int W>
__device__ __forceinline__ void tap_weights_to2(T* d0, T* d1, int wk, T tau0, T tau1, const WinParams<T>& wp);

// Write the 2m tap weights of one dimension to dst[0 .. 2m-1] (shared
// memory), one at a time.
template <typename T, int W>
__device__ __forceinline__ void tap_weights_to(T* dst, int wk, T tau, const WinParams<T>& wp) {
    const int m = W ? W / 2 : wp.m;
    const int nw = 2 * m;
    if (wk == WK_POLY && W != 0) {
#pragma unroll
        for (int a = 0; a < TapN<W>::A; ++a) dst[a] = poly_weight(tau, a, m, wp);
    } else if (wk == WK_SINH) {
        const T s = kind_sin<T, WK_SINH>(tau, wp);
#pragma unroll 2
        for (int a = 0; a < nw; ++a) dst[a] = shannon_sinh_weight(tau, s, a, m, wp);
    } else if (wk == WK_TABLE) {
        const T s = FM<T>::sinpi(tau);
#pragma unroll 2
        for (int a = 0; a < nw; ++a) dst[a] = shannon_table_weight(tau, s, a, m, wp);
    } else if (wk == WK_CSINH) {
#pragma unroll 2
        for (int a = 0; a < nw; ++a) dst[a] = classic_sinh_weight(tau, a, m, wp);
    } else {
        T wt[TapN<W>::A];
        tap_weights<T, W>(tau, wp, wt);
#pragma unroll
        for (int q = 0; q < TapN<W>::A; ++q)
            if (q < nw) dst[q] = wt[q];
    }
}

template <typename T, int W>
__device__ __forceinline__ void tap_weights_to2(T* d0, T* d1, int wk, T tau0, T tau1, const WinParams<T>& wp) {
    if (wk != WK_SINH) {
        tap_weights_to<T, W>(d0, wk, tau0, wp);
        tap_weights_to<T, W>(d1, wk, tau1, wp);
        return;
    }
    const int m = W ? W / 2 : wp.m;
    const int nw = 2 * m;
    const T s0 = kind_sin<T, WK_SINH>(tau0, wp), s1 = kind_sin<T, WK_SINH>(tau1, wp);
#pragma unroll 2
    for (int a = 0; a < nw; ++a) {
        d0[a] = shannon_sinh_weight(tau0, s0, a, m, wp);
        d1[a] = shannon_sinh_weight(tau1, s1, a, m, wp);
    }
}

// Tap weights and their x-derivatives L_t * d psi_t / d delta.
template <typename T, int W>
__device__ __forceinline__ void tap_weights_d(T tau, T Lt, const WinParams<T>& wp, T (&w)[TapN<W>::A],
                                              T (&dw)[TapN<W>::A]) {
    const int m = W ? W / 2 : wp.m;
    const int nw = 2 * m;
    if (wp.method == NFFTBL_SHANNON) {
        const T s = FM<T>::sinpi(tau);
        const T c = FM<T>::cospi(tau);
        const T pi = static_cast<T>(kPiD);
#pragma unroll
        for (int a = 0; a < nw; ++a) {
            const int n = m - 1 - a;
            const T delta = tau + static_cast<T>(n);
            const T sg = (n & 1) ? T(-1) : T(1);
            const T z = pi * delta;
            const T sincv = (delta == T(0)) ? T(1) : FM<T>::div(sg * s, z);
            T dsinc;
            if (FM<T>::abs(z) < T(0.1)) {
                const T z2 = z * z;
                dsinc = z * (T(-1.0 / 3.0) + z2 * (T(1.0 / 30.0) + z2 * (T(-1.0 / 840.0) + z2 * T(1.0 / 45360.0))));
            } else {
                dsinc = FM<T>::div(sg * c - sincv, z);
            }
            const T ph = win_phi(delta, wp);
            w[a] = sincv * ph;
            dw[a] = Lt * (pi * dsinc * ph + sincv * win_dphi(delta, wp));
        }
    } else {
#pragma unroll
        for (int a = 0; a < nw; ++a) {
            const T delta = tau + static_cast<T>(m - 1 - a);
            w[a] = win_phi(delta, wp);
            dw[a] = Lt * win_dphi(delta, wp);
        }
    }
}

// Copy a row of A tap weights from shared memory into registers with the
// widest aligned vector loads the row length allows (rows start 16-byte
// aligned when A is a multiple of 4 floats / 2 doubles, 8-byte aligned when
// A is even).
// Register sums of one spreading lane over the 2m rows of its column:
// re[q] += gr w[q], im[q] += gi w[q] for the rows q < nw.  FP32 keeps the
// rows in pairs so that each update of two rows is one packed FMA (the
// weights w[q], w[q + 1] are adjacent after a vector load).
template <typename T, int A>
struct RowSums {
    T r[A], i[A];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < A; ++q) r[q] = i[q] = T(0);
    }
    __device__ __forceinline__ void add(T gr, T gi, const T (&w)[A], int nw) {
#pragma unroll
        for (int q = 0; q < A; ++q) {
            if (q < nw) {
                r[q] += gr * w[q];
                i[q] += gi * w[q];
            }
        }
    }
    __device__ __forceinline__ T re(int q) const { return r[q]; }
    __device__ __forceinline__ T im(int q) const { return i[q]; }
};
template <int A>
struct RowSums<float, A> {
    static_assert(A % 2 == 0, "rows are summed in pairs");
    float2 r[A / 2], i[A / 2];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int h = 0; h < A / 2; ++h) r[h] = i[h] = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void add(float gr, float gi, const float (&w)[A], int nw) {
#pragma unroll
        for (int h = 0; h < A / 2; ++h) {
            if (2 * h < nw) {   // nw is even
                const float2 wp = make_float2(w[2 * h], w[2 * h + 1]);
                r[h] = cfma(wp, gr, r[h]);
                i[h] = cfma(wp, gi, i[h]);
            }
        }
    }
    __device__ __forceinline__ float re(int q) const { return (q & 1) ? r[q >> 1].y : r[q >> 1].x; }
    __device__ __forceinline__ float im(int q) const { return (q & 1) ? i[q >> 1].y : i[q >> 1].x; }
};

template <typename T, int A>
__device__ __forceinline__ void load_row(const T* __restrict__ src, T (&dst)[A]) {
    if (sizeof(T) == 4 && A % 4 == 0) {
#pragma unroll
        for (int q = 0; q < A; q += 4) {
            const float4 v = *reinterpret_cast<const float4*>(src + q);
            dst[q] = v.x; dst[q + 1] = v.y; dst[q + 2] = v.z; dst[q + 3] = v.w;
        }
    } else if (sizeof(T) == 4 && A % 2 == 0) {
#pragma unroll
        for (int q = 0; q < A; q += 2) {
            const float2 v = *reinterpret_cast<const float2*>(src + q);
            dst[q] = v.x; dst[q + 1] = v.y;
        }
    } else if (sizeof(T) == 8 && A % 2 == 0) {
#pragma unroll
        for (int q = 0; q < A; q += 2) {
            const double2 v = *reinterpret_cast<const double2*>(src + q);
            dst[q] = v.x; dst[q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < A; ++q) dst[q] = src[q];
    }
}

// Neumaier-compensated accumulator (complex, componentwise).
template <typename T>
struct CompAcc {
    T sr = T(0), si = T(0), cr = T(0), ci = T(0);
    __device__ __forceinline__ void add(T xr, T xi) {
        T t = sr + xr;
        cr += (FM<T>::abs(sr) >= FM<T>::abs(xr)) ? ((sr - t) + xr) : ((xr - t) + sr);
        sr = t;
        t = si + xi;
        ci += (FM<T>::abs(si) >= FM<T>::abs(xi)) ? ((si - t) + xi) : ((xi - t) + si);
        si = t;
    }
};

struct NodeGeom {
    int lb[3];   // local index of the first tap inside the box, per dimension
};

// Decode the tile's box origin (global cell of box element 0) per dimension.
template <int D>
__device__ __forceinline__ bool tile_origin(const TileGeom& g, int tile, bool periodic, int (&org)[3]) {
    int rem = tile;
    bool wrap = false;
#pragma unroll
    for (int t = D - 1; t >= 0; --t) {
        const int c = rem % g.nt[t];
        rem /= g.nt[t];
        org[t] = c * g.T[t] - g.off[t];
        if (periodic && (org[t] < 0 || org[t] + g.box[t] > g.L[t])) wrap = true;
    }
    return wrap;
}

// Per-node setup from the node's coordinates xv: for each dimension, tau and
// the local first-tap index.
template <typename T, int D>
__device__ __forceinline__ void node_setup_v(const T (&xv)[3], const TileGeom& g, const int (&org)[3], T (&tau)[3],
                                             int (&lb)[3], int m) {
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const T u = mul_rn(static_cast<T>(g.L[t]), xv[t]);
        const T fl = FM<T>::flr(u);
        tau[t] = u - fl;
        const int cell = static_cast<int>(fl) + g.L[t] / 2;
        lb[t] = cell - (m - 1) - org[t];
    }
}

// Per-node setup: for each dimension, tau and the local first-tap index.
template <typename T, int D>
__device__ __forceinline__ void node_setup(const T* __restrict__ xs, long long i, const TileGeom& g,
                                           const int (&org)[3], T (&tau)[3], int (&lb)[3], int m) {
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const T u = mul_rn(static_cast<T>(g.L[t]), xs[i * D + t]);
        const T fl = FM<T>::flr(u);
        tau[t] = u - fl;
        const int cell = static_cast<int>(fl) + g.L[t] / 2;
        lb[t] = cell - (m - 1) - org[t];
    }
}

// Contract the box with the tensor-product weights (one batch entry).
template <typename T, int D, int W>
__device__ __forceinline__ C2<T> contract(const C2<T>* __restrict__ box, const TileGeom& g, const int (&lb)[3],
                                          const T (&w0)[TapN<W>::A], const T (&w1)[TapN<W>::A],
                                          const T (&w2)[TapN<W>::A], bool comp, int nw_rt) {
    const int nw = W ? W : nw_rt;
    if (D == 1) {
        const C2<T>* p = box + lb[0];
        C2<T> acc = cmake<T>(T(0), T(0));
#pragma unroll
        for (int a = 0; a < nw; ++a) acc = cfma(p[a], w0[a], acc);
        return acc;
    } else if (D == 2) {
        const int pitch = g.box[1];
        const C2<T>* p = box + lb[0] * pitch + lb[1];
        if (!comp) {
            C2<T> acc = cmake<T>(T(0), T(0));
#pragma unroll 4
            for (int a = 0; a < nw; ++a) {
                const C2<T>* row = p + a * pitch;
                C2<T> r = cmake<T>(T(0), T(0));
#pragma unroll
                for (int b = 0; b < nw; ++b) r = cfma(row[b], w1[b], r);
                acc = cfma(r, w0[a], acc);
            }
            return acc;
        } else {
            CompAcc<T> acc;
#pragma unroll 4
            for (int a = 0; a < nw; ++a) {
                const C2<T>* row = p + a * pitch;
                T rr = T(0), ri = T(0);
#pragma unroll
                for (int b = 0; b < nw; ++b) {
                    const C2<T> v = row[b];
                    rr += v.x * w1[b];
                    ri += v.y * w1[b];
                }
                acc.add(rr * w0[a], ri * w0[a]);
            }
            return cmake<T>(acc.sr + acc.cr, acc.si + acc.ci);
        }
    } else {
        const int p1 = g.box[2];
        const int p0 = g.box[1] * p1;
        const C2<T>* p = box + lb[0] * p0 + lb[1] * p1 + lb[2];
        if (!comp) {
            C2<T> acc = cmake<T>(T(0), T(0));
            for (int a = 0; a < nw; ++a) {
                C2<T> mid = cmake<T>(T(0), T(0));
#pragma unroll 2
                for (int b = 0; b < nw; ++b) {
                    const C2<T>* row = p + a * p0 + b * p1;
                    C2<T> r = cmake<T>(T(0), T(0));
#pragma unroll
                    for (int c = 0; c < nw; ++c) r = cfma(row[c], w2[c], r);
                    mid = cfma(r, w1[b], mid);
                }
                acc = cfma(mid, w0[a], acc);
            }
            return acc;
        } else {
            CompAcc<T> acc;
            for (int a = 0; a < nw; ++a) {
#pragma unroll 2
                for (int b = 0; b < nw; ++b) {
                    const C2<T>* row = p + a * p0 + b * p1;
                    T rr = T(0), ri = T(0);
#pragma unroll
                    for (int c = 0; c < nw; ++c) {
                        const C2<T> v = row[c];
                        rr += v.x * w2[c];
                        ri += v.y * w2[c];
                    }
                    const T wab = w0[a] * w1[b];
                    acc.add(rr * wab, ri * wab);
                }
            }
            return cmake<T>(acc.sr + acc.cr, acc.si + acc.ci);
        }
    }
}

// Contraction of one batch entry for a plan with an inline weight kind WK
// (Shannon sinh or table, classical sinh; d >= 2) with the dimension-0
// weights evaluated inside the row loop: each is used once, so they need no
// registers across the loop, and their SFU work overlaps the rows'
// shared-memory loads and FMAs.  w1 (and w2) hold the other dimensions'
// weights; s0 = kind_sin<T, WK>(tau0) (unused by the classical kind).  COMP adds the
// weighted row sums in compensated summation, as contract() does for the
// compensated FP32 plans.
template <typename T, int D, int W, int WK, bool COMP = false>
__device__ __forceinline__ C2<T> contract_lazy0(const C2<T>* __restrict__ box, const TileGeom& g, const int (&lb)[3],
                                                T tau0, T s0, const T (&w1)[TapN<W>::A], const T (&w2)[TapN<W>::A],
                                                const WinParams<T>& wp, int nw_rt) {
    const int nw = W ? W : nw_rt;
    const int m = nw / 2;
    C2<T> acc = cmake<T>(T(0), T(0));
    CompAcc<T> cacc;   // COMP: the weighted row sums in compensated (Neumaier) summation
    if (D == 2) {
        const int pitch = g.box[1];
        const C2<T>* p = box + lb[0] * pitch + lb[1];
#pragma unroll 2
        for (int a = 0; a < nw; ++a) {
            const T w0a = fast_weight<T, WK>(tau0, s0, a, m, wp);
            const C2<T>* row = p + a * pitch;
            C2<T> r = cmake<T>(T(0), T(0));
#pragma unroll
            for (int b = 0; b < TapN<W>::A; ++b)
                if (b < nw) r = cfma(row[b], w1[b], r);
            if constexpr (COMP) cacc.add(r.x * w0a, r.y * w0a);
            else acc = cfma(r, w0a, acc);
        }
    } else {
        const int p1 = g.box[2];
        const int p0 = g.box[1] * p1;
        const C2<T>* p = box + lb[0] * p0 + lb[1] * p1 + lb[2];
        for (int a = 0; a < nw; ++a) {
            const T w0a = fast_weight<T, WK>(tau0, s0, a, m, wp);
            C2<T> mid = cmake<T>(T(0), T(0));
#pragma unroll 2
            for (int b = 0; b < nw; ++b) {
                const C2<T>* row = p + a * p0 + b * p1;
                C2<T> r = cmake<T>(T(0), T(0));
#pragma unroll
                for (int c = 0; c < TapN<W>::A; ++c)
                    if (c < nw) r = cfma(row[c], w2[c], r);
                if constexpr (COMP) {
                    const T wab = w0a * w1[b];
                    cacc.add(r.x * wab, r.y * wab);
                } else {
                    mid = cfma(r, w1[b], mid);
                }
            }
            if constexpr (!COMP) acc = cfma(mid, w0a, acc);
        }
    }
    if constexpr (COMP) return cmake<T>(cacc.sr + cacc.cr, cacc.si + cacc.ci);
    return acc;
}

// contract_lazy0 for two nodes of one cell (same first taps lb): every box
// value is loaded once and enters both nodes' sums, which halves the
// shared-memory traffic of the pair.  Node b's arithmetic is node a's with
// its own weights, so each result equals contract_lazy0 of that node alone.
template <typename T, int D, int W, int WK, bool COMP = false, int UB = 2>
__device__ __forceinline__ void contract_lazy0_pair(const C2<T>* __restrict__ box, const TileGeom& g,
                                                    const int (&lb)[3], T tau0a, T s0a, const T (&w1a)[TapN<W>::A],
                                                    const T (&w2a)[TapN<W>::A], T tau0b, T s0b,
                                                    const T (&w1b)[TapN<W>::A], const T (&w2b)[TapN<W>::A],
                                                    const WinParams<T>& wp, int nw_rt, C2<T>& outa, C2<T>& outb) {
    const int nw = W ? W : nw_rt;
    const int m = nw / 2;
    C2<T> acca = cmake<T>(T(0), T(0)), accb = cmake<T>(T(0), T(0));
    CompAcc<T> ca, cb;
    if constexpr (D == 2) {
        const int pitch = g.box[1];
        const C2<T>* p = box + lb[0] * pitch + lb[1];
        auto row_step = [&](int a) {
            const T w0a = fast_weight<T, WK>(tau0a, s0a, a, m, wp);
            const T w0b = fast_weight<T, WK>(tau0b, s0b, a, m, wp);
            const C2<T>* row = p + a * pitch;
            C2<T> ra = cmake<T>(T(0), T(0)), rb = cmake<T>(T(0), T(0));
#pragma unroll
            for (int b = 0; b < TapN<W>::A; ++b) {
                if (b < nw) {
                    const C2<T> v = row[b];
                    ra = cfma(v, w1a[b], ra);
                    rb = cfma(v, w1b[b], rb);
                }
            }
            if constexpr (COMP) {
                ca.add(ra.x * w0a, ra.y * w0a);
                cb.add(rb.x * w0b, rb.y * w0b);
            } else {
                acca = cfma(ra, w0a, acca);
                accb = cfma(rb, w0b, accb);
            }
        };
#pragma unroll 2
        for (int a = 0; a < nw; ++a) row_step(a);
    } else if constexpr (D == 3) {
        const int p1 = g.box[2];
        const int p0 = g.box[1] * p1;
        const C2<T>* p = box + lb[0] * p0 + lb[1] * p1 + lb[2];
        for (int a = 0; a < nw; ++a) {
            const T w0a = fast_weight<T, WK>(tau0a, s0a, a, m, wp);
            const T w0b = fast_weight<T, WK>(tau0b, s0b, a, m, wp);
            C2<T> mida = cmake<T>(T(0), T(0)), midb = cmake<T>(T(0), T(0));
            auto brow = [&](int b) {
                const C2<T>* row = p + a * p0 + b * p1;
                C2<T> ra = cmake<T>(T(0), T(0)), rb = cmake<T>(T(0), T(0));
#pragma unroll
                for (int c = 0; c < TapN<W>::A; ++c) {
                    if (c < nw) {
                        const C2<T> v = row[c];
                        ra = cfma(v, w2a[c], ra);
                        rb = cfma(v, w2b[c], rb);
                    }
                }
                if constexpr (COMP) {
                    const T wa = w0a * w1a[b], wb = w0b * w1b[b];
                    ca.add(ra.x * wa, ra.y * wa);
                    cb.add(rb.x * wb, rb.y * wb);
                } else {
                    mida = cfma(ra, w1a[b], mida);
                    midb = cfma(rb, w1b[b], midb);
                }
            };
            // (UB: rows in flight; 4 where the kernel has the registers for them)
            if constexpr (UB == 4) {
#pragma unroll 4
                for (int b = 0; b < nw; ++b) brow(b);
            } else {
#pragma unroll 2
                for (int b = 0; b < nw; ++b) brow(b);
            }
            if constexpr (!COMP) {
                acca = cfma(mida, w0a, acca);
                accb = cfma(midb, w0b, accb);
            }
        }
    }
    if constexpr (COMP) {
        outa = cmake<T>(ca.sr + ca.cr, ca.si + ca.ci);
        outb = cmake<T>(cb.sr + cb.cr, cb.si + cb.ci);
    } else {
        outa = acca;
        outb = accb;
    }
}

// The inline-weight interpolation of a pair head: nodes ia and ib (= ia
// when the head has no partner) of one cell, weights of dimensions 1 .. d-1
// in registers, dimension-0 weights evaluated per row.
template <typename T, int D, int W, int WK, int UB = 2>
__device__ __forceinline__ void interp_pair(const TapArgs<T>& a, const C2<T>* box, const int (&lb)[3],
                                            const T (&taua)[3], const T (&taub)[3], int nw, C2<T>& fa, C2<T>& fb) {
    constexpr int A = TapN<W>::A;
    T w1a[A], w2a[A], w1b[A], w2b[A];
    tap_weights<T, W, WK>(taua[1], a.w, w1a);
    tap_weights<T, W, WK>(taub[1], a.w, w1b);
    if constexpr (D > 2) {
        tap_weights<T, W, WK>(taua[2], a.w, w2a);
        tap_weights<T, W, WK>(taub[2], a.w, w2b);
    }
    const T s0a = (WK == WK_CSINH) ? T(0) : (WK == WK_SINH) ? kind_sin<T, WK_SINH>(taua[0], a.w) : FM<T>::sinpi(taua[0]);
    const T s0b = (WK == WK_CSINH) ? T(0) : (WK == WK_SINH) ? kind_sin<T, WK_SINH>(taub[0], a.w) : FM<T>::sinpi(taub[0]);
    if (a.comp)
        contract_lazy0_pair<T, D, W, WK, true, UB>(box, a.g, lb, taua[0], s0a, w1a, w2a, taub[0], s0b, w1b, w2b, a.w,
                                                   nw, fa, fb);
    else
        contract_lazy0_pair<T, D, W, WK, false, UB>(box, a.g, lb, taua[0], s0a, w1a, w2a, taub[0], s0b, w1b, w2b, a.w,
                                                    nw, fa, fb);
}

// The inline-weight interpolation of one node (FP64 plans): weights of
// dimensions 1 .. d-1 in registers, dimension-0 weights evaluated per row.
template <typename T, int D, int W>
__device__ __forceinline__ C2<T> interp_single(const TapArgs<T>& a, const C2<T>* box, const int (&lb)[3],
                                               const T (&tau)[3], int wk, int nw) {
    constexpr int A = TapN<W>::A;
    T w1[A], w2[A];
    if (wk == WK_SINH) {
        tap_weights<T, W, WK_SINH>(tau[1], a.w, w1);
        if (D > 2) tap_weights<T, W, WK_SINH>(tau[2], a.w, w2);
        const T s0 = kind_sin<T, WK_SINH>(tau[0], a.w);
        return a.comp ? contract_lazy0<T, D, W, WK_SINH, true>(box, a.g, lb, tau[0], s0, w1, w2, a.w, nw)
                      : contract_lazy0<T, D, W, WK_SINH>(box, a.g, lb, tau[0], s0, w1, w2, a.w, nw);
    }
    if (wk == WK_CSINH) {
        tap_weights<T, W, WK_CSINH>(tau[1], a.w, w1);
        if (D > 2) tap_weights<T, W, WK_CSINH>(tau[2], a.w, w2);
        return a.comp ? contract_lazy0<T, D, W, WK_CSINH, true>(box, a.g, lb, tau[0], T(0), w1, w2, a.w, nw)
                      : contract_lazy0<T, D, W, WK_CSINH>(box, a.g, lb, tau[0], T(0), w1, w2, a.w, nw);
    }
    tap_weights<T, W, WK_TABLE>(tau[1], a.w, w1);
    if (D > 2) tap_weights<T, W, WK_TABLE>(tau[2], a.w, w2);
    const T s0 = FM<T>::sinpi(tau[0]);
    return a.comp ? contract_lazy0<T, D, W, WK_TABLE, true>(box, a.g, lb, tau[0], s0, w1, w2, a.w, nw)
                  : contract_lazy0<T, D, W, WK_TABLE>(box, a.g, lb, tau[0], s0, w1, w2, a.w, nw);
}

// Copy n = 2m (n <= A) window factors from src to dst with the widest
// aligned vector accesses the compile-time tap count allows (the stored
// rows and their per-dimension parts start 16-byte aligned when 2m is a
// multiple of 4 floats / 2 doubles).
template <typename T, int W, typename Dst>
__device__ __forceinline__ void load_factors(const T* __restrict__ src, Dst& dst, int n) {
    constexpr int A = TapN<W>::A;
    if (W != 0 && sizeof(T) == 4 && W % 4 == 0) {
#pragma unroll
        for (int q = 0; q < A; q += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(src + q));
            dst[q] = v.x; dst[q + 1] = v.y; dst[q + 2] = v.z; dst[q + 3] = v.w;
        }
    } else if (W != 0 && W % 2 == 0) {
#pragma unroll
        for (int q = 0; q < A; q += 2) {
            if (sizeof(T) == 4) {
                const float2 v = __ldg(reinterpret_cast<const float2*>(src + q));
                dst[q] = v.x; dst[q + 1] = v.y;
            } else {
                const double2 v = __ldg(reinterpret_cast<const double2*>(src + q));
                dst[q] = v.x; dst[q + 1] = v.y;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < A; ++q)
            if (q < n) dst[q] = __ldg(src + q);
    }
}

// Copy the stored factors of one node (D dimensions of n = 2m each) into a
// node-table row whose dimension t starts at t * A.  Out of line: only plans
// with stored factors take it.
template <typename T, int W>
__device__ __noinline__ void copy_factor_rows(const T* __restrict__ src, T* dst, int D, int n) {
    for (int t = 0; t < D; ++t) {
        T* d = dst + t * TapN<W>::A;
        load_factors<T, W>(src + t * n, d, n);
    }
}

// One node of interp_kernel for every plan other than the single-batch
// case with an inline weight kind (the cKB window, d = 1, batches, stored
// factors): all weights in registers, then one contraction per batch
// entry.  Kept out of line so that its registers do not count
// against the common path.
template <typename T, int D, int W>
__device__ __noinline__ void interp_node_general(const TapArgs<T>& a, const C2<T>* box, int slot, const int (&lb)[3],
                                                 const T (&tau)[3], int wk, int b0, int nb, long long i,
                                                 long long dst) {
    constexpr int A = TapN<W>::A;
    const int nw = W ? W : 2 * a.w.m;
    T w0[A], w1[A], w2[A];
    if (a.wfac) {   // stored factors (step 0b)
        const T* wr = a.wfac + i * a.wstride;
        load_factors<T, W>(wr, w0, nw);
        if (D > 1) load_factors<T, W>(wr + nw, w1, nw);
        if (D > 2) load_factors<T, W>(wr + 2 * nw, w2, nw);
    } else if (wk == WK_SINH) {
        tap_weights<T, W, WK_SINH>(tau[0], a.w, w0);
        if (D > 1) tap_weights<T, W, WK_SINH>(tau[1], a.w, w1);
        if (D > 2) tap_weights<T, W, WK_SINH>(tau[2], a.w, w2);
    } else if (wk == WK_TABLE) {
        tap_weights<T, W, WK_TABLE>(tau[0], a.w, w0);
        if (D > 1) tap_weights<T, W, WK_TABLE>(tau[1], a.w, w1);
        if (D > 2) tap_weights<T, W, WK_TABLE>(tau[2], a.w, w2);
    } else if (wk == WK_CSINH) {
        tap_weights<T, W, WK_CSINH>(tau[0], a.w, w0);
        if (D > 1) tap_weights<T, W, WK_CSINH>(tau[1], a.w, w1);
        if (D > 2) tap_weights<T, W, WK_CSINH>(tau[2], a.w, w2);
    } else {
        tap_weights<T, W>(tau[0], a.w, w0);
        if (D > 1) tap_weights<T, W>(tau[1], a.w, w1);
        if (D > 2) tap_weights<T, W>(tau[2], a.w, w2);
    }
    for (int bb = 0; bb < nb; ++bb) {
        const C2<T> v = contract<T, D, W>(box + bb * slot, a.g, lb, w0, w1, w2, a.comp != 0, nw);
        a.fout[static_cast<long long>(b0 + bb) * a.N + dst] = v;
    }
}

// Stage the box(es) of batch entries b0 .. b0+nb-1 in shared memory.
// Returns false if the copy did not complete within the wait limit.
// Box slots in shared memory: each batch entry's box starts on a 128-byte
// boundary (TMA destination alignment); the dynamic shared memory base is
// rounded up to 128 bytes (the host adds 128 bytes to the request).
template <typename T>
__host__ __device__ __forceinline__ int box_slot_cells(int box_cells) {
    constexpr int per128 = 128 / static_cast<int>(sizeof(C2<T>));
    return (box_cells + per128 - 1) / per128 * per128;
}

template <typename T>
__device__ __forceinline__ C2<T>* aligned_box_base(unsigned char* smem) {
    const uint32_t a = smem_addr(smem);
    return reinterpret_cast<C2<T>*>(smem + ((128u - (a & 127u)) & 127u));
}

// Stage the box(es) of batch entries b0 .. b0+nb-1 in shared memory (slot
// stride `slot` cells).  Returns false, in every thread of the block, if the
// copy did not complete within the wait limit.
template <typename T, int D>
__device__ __forceinline__ bool stage_box(const CUtensorMap* tmap, const TapArgs<T>& a, C2<T>* box, int box_cells,
                                          int slot, const int (&org)[3], bool wrap, int b0, int nb, uint64_t* bar,
                                          uint32_t& phase) {
    if (!wrap) {
        if (threadIdx.x == 0 && !a.stall) {   // (stall: nothing arrives, the wait must run out)
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(nb * box_cells * sizeof(C2<T>)));
            for (int bb = 0; bb < nb; ++bb) {
                C2<T>* dst = box + bb * slot;
                if (D == 1)
                    tma_load_2d(dst, tmap, 2 * org[0], b0 + bb, bar);
                else if (D == 2)
                    tma_load_3d(dst, tmap, 2 * org[1], org[0], b0 + bb, bar);
                else
                    tma_load_4d(dst, tmap, 2 * org[2], org[1], org[0], b0 + bb, bar);
            }
        }
        const bool ok = mbar_wait_bounded(bar, phase, a.err, a.wait_ns);
        phase ^= 1u;
        return __syncthreads_and(ok) != 0;   // one decision for the whole block
    }
    // periodic wrap (classical NFFT tiles crossing the grid edge): plain loads
    for (int idx = threadIdx.x; idx < nb * box_cells; idx += blockDim.x) {
        const int bb = idx / box_cells;
        const int cell = idx - bb * box_cells;
        int r = cell;
        int loc[3] = {0, 0, 0};
#pragma unroll
        for (int t = D - 1; t >= 0; --t) {
            loc[t] = r % a.g.box[t];
            r /= a.g.box[t];
        }
        long long gi = 0;
#pragma unroll
        for (int t = 0; t < D; ++t) {
            int c = (org[t] + loc[t]) % a.g.L[t];
            if (c < 0) c += a.g.L[t];
            gi = gi * a.g.L[t] + c;
        }
        box[bb * slot + cell] = a.grid[(b0 + bb) * a.grid_stride + gi];
    }
    __syncthreads();
    return true;
}

// Step 0b of Algorithm 4.2 in tensor-product form: the 2m window factors of
// every dimension of every sorted node, row i = [dim 0 | dim 1 | dim 2]
// (each 2m long) padded to wstride; the same arithmetic as the transforms'
// own evaluation.
template <typename T, int D, int W>
__global__ void __launch_bounds__(256) factor_kernel(const TapArgs<T> a, T* __restrict__ out) {
    constexpr int A = TapN<W>::A;
    const int nw = W ? W : 2 * a.w.m;
    const int wk = weight_kind(a.w);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < a.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        T* row = out + i * a.wstride;
#pragma unroll
        for (int t = 0; t < D; ++t) {
            const T u = mul_rn(static_cast<T>(a.g.L[t]), a.xs[i * D + t]);
            const T tau = u - FM<T>::flr(u);
            T w[A];
            if (wk == WK_POLY)
                tap_weights<T, W, WK_POLY>(tau, a.w, w);
            else if (wk == WK_SINH)
                tap_weights<T, W, WK_SINH>(tau, a.w, w);
            else if (wk == WK_TABLE)
                tap_weights<T, W, WK_TABLE>(tau, a.w, w);
            else if (wk == WK_CSINH)
                tap_weights<T, W, WK_CSINH>(tau, a.w, w);
            else
                tap_weights<T, W>(tau, a.w, w);
#pragma unroll
            for (int q = 0; q < A; ++q)
                if (q < nw) row[t * nw + q] = w[q];
        }
    }
}

// One thread's share of interp_kernel: head hv (bit 31: the next sorted node
// is its same-cell partner) of a staged box, batch entries b0 .. b0+nb-1.
template <typename T, int D, int W, int UB = 2>
__device__ __forceinline__ void interp_head(const TapArgs<T>& a, const C2<T>* box, int slot, const int (&org)[3],
                                            uint32_t hv, int b0, int nb, int wk, int nw, int m) {
    const long long ia = static_cast<long long>(hv & 0x7FFFFFFFu);
    const bool two = (hv >> 31) != 0;
    const long long ib = two ? ia + 1 : ia;
    T taua[3], taub[3];
    int lb[3] = {0, 0, 0}, lbb[3] = {0, 0, 0};
    node_setup<T, D>(a.xs, ia, a.g, org, taua, lb, m);
    node_setup<T, D>(a.xs, ib, a.g, org, taub, lbb, m);   // same cell: lbb = lb
    const long long da = a.perm[ia], db = a.perm[ib];
    if constexpr (D >= 2 && sizeof(T) == 4) {
        // (the closed form here: unrolled polynomial weights in registers
        // raise this kernel's register count past its occupancy)
        const int wkc = closed_kind(a.w);
        if (!a.wfac && nb == 1 && (wkc == WK_SINH || wkc == WK_CSINH || wkc == WK_TABLE)) {
            C2<T> fa, fb;
            if (wkc == WK_SINH) interp_pair<T, D, W, WK_SINH, UB>(a, box, lb, taua, taub, nw, fa, fb);
            else if (wkc == WK_CSINH) interp_pair<T, D, W, WK_CSINH, UB>(a, box, lb, taua, taub, nw, fa, fb);
            else interp_pair<T, D, W, WK_TABLE, UB>(a, box, lb, taua, taub, nw, fa, fb);
            a.fout[static_cast<long long>(b0) * a.N + da] = fa;
            if (two) a.fout[static_cast<long long>(b0) * a.N + db] = fb;
            return;
        }
    }
    if constexpr (D >= 2 && sizeof(T) == 8) {
        if (!a.wfac && nb == 1 && (wk == WK_SINH || wk == WK_CSINH || wk == WK_TABLE)) {
            a.fout[static_cast<long long>(b0) * a.N + da] = interp_single<T, D, W>(a, box, lb, taua, wk, nw);
            return;
        }
    }
    // (closed-form weights: see above)
    interp_node_general<T, D, W>(a, box, slot, lb, taua, closed_kind(a.w), b0, nb, ia, da);
    if (two) interp_node_general<T, D, W>(a, box, slot, lbb, taub, closed_kind(a.w), b0, nb, ib, db);
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(kTapThreads) interp_kernel(const __grid_constant__ CUtensorMap tmap,
                                                             const TapArgs<T> a) {
    using CT = C2<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    CT* box = aligned_box_base<T>(smem);
    int box_cells = 1;
#pragma unroll
    for (int t = 0; t < D; ++t) box_cells *= a.g.box[t];
    const int slot = box_slot_cells<T>(box_cells);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        prefetch_tmap(&tmap);
    }
    __syncthreads();
    uint32_t phase = 0;
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    const int wk = weight_kind(a.w);
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        const bool wrap = tile_origin<D>(a.g, wi.tile, periodic, org);
        for (int b0 = 0; b0 < a.batch; b0 += a.batch_smem) {
            const int nb = min(a.batch_smem, a.batch - b0);
            if (!stage_box<T, D>(&tmap, a, box, box_cells, slot, org, wrap, b0, nb, &bar, phase)) {
                if (!a.stall) mbar_wait_bounded(&bar, phase ^ 1u, a.err);   // let the copy in flight land
                return;
            }
            // FP32: one thread per pair head, a node and, when it has one, its
            // same-cell partner, which share every box load; FP64 (whose
            // register budget a second node's weights would exceed): one
            // thread per node
            const bool pairs = sizeof(T) == 4 && a.heads != nullptr;
            const int nh = pairs ? static_cast<int>(a.nheads[item]) : wi.count;
            for (int h = threadIdx.x; h < nh; h += blockDim.x) {
                const uint32_t hv = pairs ? a.heads[wi.start + h] : static_cast<uint32_t>(wi.start + h);
                interp_head<T, D, W>(a, box, slot, org, hv, b0, nb, wk, nw, m);
            }
            __syncthreads();
        }
    }
}

// Interpolation of single-batch d = 3 FP32 plans of the Shannon method (no
// periodic tiles) with two box buffers per block.  The box of the block's
// next work item is staged while its warps work on the current one, and
// each warp takes an item's pair heads 32 at a time, so that a warp that
// finds no heads left moves on to the next item instead of idling at a
// block barrier (work items hold a few to several hundred heads).  The last
// warp to leave an item refills its buffer with the item two ahead.  Every
// wait is bounded; a block whose wait ran out stops taking work, waits for
// the copies it issued, and returns (the error flag is set).
constexpr int kPipeThreads = 384;

template <int W>
__global__ void __launch_bounds__(kPipeThreads, 1) interp3p_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                   const TapArgs<float> a) {
    using CT = C2<float>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ int next_head[2];   // heads of the buffer's item taken so far
    __shared__ int left[2];        // warps still working on the buffer's item
    __shared__ int issued[2];      // copies issued into the buffer
    CT* box0 = aligned_box_base<float>(smem);
    const int box_cells = a.g.box[0] * a.g.box[1] * a.g.box[2];
    const int slot = box_slot_cells<float>(box_cells);
    const int nwarps = static_cast<int>(blockDim.x >> 5);
    const int lane = static_cast<int>(threadIdx.x & 31);
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    const int wk = weight_kind(a.w);
    auto issue = [&](int buf, int item) {   // one thread
        int org[3] = {0, 0, 0};
        tile_origin<3>(a.g, a.work[item].tile, false, org);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&full[buf], static_cast<uint32_t>(box_cells * sizeof(CT)));
        tma_load_4d(box0 + buf * slot, &tmap, 2 * org[2], org[1], org[0], 0, &full[buf]);
        issued[buf] += 1;
    };
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_mbar_init();
        prefetch_tmap(&tmap);
        for (int b = 0; b < 2; ++b) {
            next_head[b] = 0;
            left[b] = nwarps;
            issued[b] = 0;
        }
        if (!a.stall) {   // (stall: nothing arrives, the waits must run out)
            if (static_cast<int>(blockIdx.x) < a.n_work) issue(0, blockIdx.x);
            if (static_cast<int>(blockIdx.x + gridDim.x) < a.n_work) issue(1, blockIdx.x + gridDim.x);
        }
    }
    __syncthreads();
    int k = 0;
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x, ++k) {
        const int buf = k & 1;
        const bool landed = mbar_wait_bounded(&full[buf], static_cast<uint32_t>((k >> 1) & 1), a.err, a.wait_ns);
        if (!__all_sync(0xffffffffu, landed)) break;   // one decision per warp
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        tile_origin<3>(a.g, wi.tile, false, org);
        const CT* box = box0 + buf * slot;
        const int nh = static_cast<int>(a.nheads[item]);
        while (true) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&next_head[buf], 32);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= nh) break;
            const int h = base + lane;
            if (h < nh) interp_head<float, 3, W, 4>(a, box, slot, org, a.heads[wi.start + h], 0, 1, wk, nw, m);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();   // this warp's box reads before the count
            if (atomicSub(&left[buf], 1) == 1) {   // the last warp out: refill
                __threadfence_block();
                next_head[buf] = 0;
                left[buf] = nwarps;
                const int nxt = item + 2 * static_cast<int>(gridDim.x);
                if (nxt < a.n_work && !a.stall) issue(buf, nxt);
            }
        }
    }
    // no copy may still be writing this block's shared memory when it exits
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < 2; ++b)
            if (issued[b] > 0) mbar_wait_bounded(&full[b], static_cast<uint32_t>((issued[b] - 1) & 1), a.err, a.wait_ns);
}

// ---------------------------------------------------------------------------
// Spreading (transposed short sums, the Psi^T factor of the adjoint).
//
// Exact accumulation: a work item's box is accumulated in fixed point in
// shared memory with a power-of-two quantum chosen from a bound on the
// item's total contribution (FixedCell below), so no partial sum can
// overflow.  Integer addition is associative, so the box is exact and
// independent of the order in which warps add.
//
// Ordered flush: the item's box (converted back to the plan's precision)
// is stored to its own slot of a scratch array; gather_kernel then forms
// every grid value as the sum over the boxes that cover it in a fixed
// order (tiles in row-major order, then the tile's items in order).  No
// global atomics, no clearing of the grid, bitwise reproducible results.
//
// Kernels: spread1_kernel (d = 1), spread2_kernel (d = 2), spread3_kernel
// (d = 3).

// Fixed-point cells of the d = 2 / d = 3 spreading boxes (16 bytes per cell).
//  FP32: each component holds v = hi * 2^21 + lo in two int32 words, with
//    the quantum chosen so that the item's total stays below 2^42 quanta.  A
//    value X (in quanta, |X| < 2^43) splits exactly with float arithmetic:
//    hi = rint(X 2^-21) and lo = rint(X - hi 2^21), |lo| <= 2^20, both read
//    off the bits of y + 1.5 * 2^23 (valid for |y| < 2^22).  An item adds at
//    most 2047 times to a cell, so neither word can overflow, and integer
//    addition keeps the sum exact and independent of order.  32-bit shared
//    atomics are several times faster than 64-bit ones, and no step needs
//    the FP64 pipe (slow on this part).
//  FP64: one 64-bit word per component, total below 2^62 quanta.
template <typename T> struct FixedCell;
// A batch entry's box is a group of component planes of `slot` cells each
// (FP32: hi_re, lo_re, hi_im, lo_im as int32; FP64: re, im as 64-bit), so
// that lanes adding to consecutive cells touch consecutive words.
template <> struct FixedCell<float> {
    static constexpr int kBits = 42;
    static constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23
    static constexpr int kMagicBits = 0x4B400000;
    __device__ static void add(unsigned char* grp, int cell, int slot, float xr, float xi) {
        int* w = reinterpret_cast<int*>(grp) + cell;
        split(w, w + slot, xr);
        split(w + 2 * slot, w + 3 * slot, xi);
    }
    __device__ static void split(int* hi_p, int* lo_p, float X) {
        const float h = fmaf(X, 0x1p-21f, kMagic);
        const int hi = __float_as_int(h) - kMagicBits;
        const float lo_f = fmaf(-(h - kMagic), 0x1p21f, X);
        const int lo = __float_as_int(lo_f + kMagic) - kMagicBits;
        if (hi != 0) atomicAdd(hi_p, hi);
        if (lo != 0) atomicAdd(lo_p, lo);
    }
    // (hi 2^21 + lo) q rounded once to float; q_hi = q 2^21 (powers of two).
    __device__ static float value(const unsigned char* grp, int cell, int slot, int comp, float q, float q_hi) {
        const int* w = reinterpret_cast<const int*>(grp) + 2 * comp * slot + cell;
        const int lo = w[slot];
        const int c = lo >> 21;                    // carry: lo = c 2^21 + r, 0 <= r < 2^21
        const int hi = w[0] + c;                   // |hi| < 2^22
        const int r = lo - c * 2097152;
        const float hf = __int_as_float(hi + kMagicBits) - kMagic;   // exact for |x| < 2^22
        const float rf = __int_as_float(r + kMagicBits) - kMagic;
        return fmaf(hf, q_hi, rf * q);
    }
};
template <> struct FixedCell<double> {
    static constexpr int kBits = 62;
    __device__ static void add(unsigned char* grp, int cell, int slot, double xr, double xi) {
        unsigned long long* w = reinterpret_cast<unsigned long long*>(grp) + cell;
        const long long vr = __double2ll_rn(xr), vi = __double2ll_rn(xi);
        if (vr != 0) atomicAdd(w, static_cast<unsigned long long>(vr));
        if (vi != 0) atomicAdd(w + slot, static_cast<unsigned long long>(vi));
    }
    __device__ static double value(const unsigned char* grp, int cell, int slot, int comp, double q, double) {
        return static_cast<double>(reinterpret_cast<const long long*>(grp)[comp * slot + cell]) * q;
    }
};

// Bound on an item's total |input| (both components, all batch entries of
// the group) for the quantum of the fixed-point box, reduced over the block
// into s_red[0 .. nwarps).  FP32 inputs are summed in FP32: the relative
// error of the sum, below (count) 2^-24, is covered by the margin the
// caller applies.
template <typename T>
__device__ __forceinline__ void item_abs_sum(const TapArgs<T>& a, const WorkItem& wi, int b0, int nb, double* s_red) {
    using CT = C2<T>;
    T part = T(0);
    const int step = blockDim.x;
    for (int j0 = threadIdx.x; j0 < wi.count; j0 += 4 * step) {
        uint32_t src[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * step;
            src[u] = (j < wi.count) ? a.perm[wi.start + j] : 0xFFFFFFFFu;
        }
        for (int bb = 0; bb < nb; ++bb) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (src[u] != 0xFFFFFFFFu) {
                    const CT gv = a.fin[static_cast<long long>(b0 + bb) * a.N + src[u]];
                    part += FM<T>::abs(gv.x) + FM<T>::abs(gv.y);
                }
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = static_cast<double>(part);
}

// Thread 0: quantum q = 2^(e - bits) with 2^e above the item's bound (the
// summed |input| times the window-product bound, with a 1e-3 margin).
template <typename T>
__device__ __forceinline__ void item_quantum(const TapArgs<T>& a, int nwarps, double* s_red) {
    double tot = 0.0;
    for (int w = 0; w < nwarps; ++w) tot += s_red[w];
    tot *= static_cast<double>(a.wbound) * 1.001;
    int e = 0;
    if (tot > 0.0) e = max(ilogb(tot) + 1, -60);   // tot < 2^e
    s_red[32] = ldexp(1.0, e - FixedCell<T>::kBits);
    s_red[33] = (tot > 0.0) ? 1.0 : 0.0;
    // the same powers of two in the plan precision: 1/q, q, q 2^21, flag
    static_assert(kSpreadRedDoubles * 8 >= 36 * 8 + 4 * sizeof(T), "reduction scratch too small");
    T* f = reinterpret_cast<T*>(s_red + 36);
    f[0] = static_cast<T>(ldexp(1.0, FixedCell<T>::kBits - e));
    f[1] = static_cast<T>(s_red[32]);
    f[2] = static_cast<T>(ldexp(1.0, e - FixedCell<T>::kBits + 21));
    f[3] = (tot > 0.0) ? T(1) : T(0);
}

// Reads back what item_quantum stored.
template <typename T>
struct ItemQuantum {
    T inv_q, q_lo, q_hi;
    bool any;
    __device__ explicit ItemQuantum(const double* s_red) {
        const T* f = reinterpret_cast<const T*>(s_red + 36);
        inv_q = f[0];
        q_lo = f[1];
        q_hi = f[2];
        any = f[3] != T(0);
    }
};

// d = 2 spreading without block barriers inside a work item: warp w walks a
// contiguous share of the item's (cell-sorted) nodes in chunks of 32.
//  Phase A: lane l evaluates the 2 x 2m window values of chunk node l (one
//    node per lane, fully unrolled) into row l of the warp's shared-memory
//    node table, with the node's input value and first taps.
//  Phase B: the warp walks the chunk's rows in order.  Lanes own absolute
//    box columns; consecutive nodes of one box row whose contiguous-
//    dimension first tap lies in one segment of S = 33 - 2m cells share the
//    lanes' register accumulators (2m rows per lane), which go to the
//    64-bit fixed-point box (exact integer adds) when the segment changes.
// Shares of different warps may meet in a cell; their fixed-point sums add
// exactly, so the result does not depend on timing.
template <typename T, int W>
__global__ void __launch_bounds__(kTapThreads, sizeof(T) == 4 ? 3 : 1) spread2_kernel(const TapArgs<T> a) {
    using CT = C2<T>;
    using U = unsigned long long;
    constexpr int A = TapN<W>::A;
    constexpr int RS = spread2_row<T>(A);   // node-table row: w0[A] | w1[A] | g.x g.y | key t0
    static_assert(A % 2 == 0, "node-table rows must stay 16-byte aligned");
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    const int S = 33 - nw;
    extern __shared__ __align__(128) unsigned char smem[];
    const int box1 = a.g.box[1];
    const int box_cells = a.g.box[0] * box1;
    const int slot = (box_cells + 1) / 2 * 2;
    const int nbmax = a.spread_batch;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const SpreadSmem Ls = spread2_layout<T>(A, box_cells, nbmax, nwarps);
    U* boxu = reinterpret_cast<U*>(smem + Ls.box);
    T* s_tab = reinterpret_cast<T*>(smem + Ls.w) + static_cast<size_t>(warp) * 32 * RS;
    double* s_red = reinterpret_cast<double*>(smem + Ls.red);
    const int wk = weight_kind(a.w);
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        tile_origin<2>(a.g, wi.tile, periodic, org);
        for (int b0 = 0; b0 < a.batch; b0 += nbmax) {
            const int nb = min(nbmax, a.batch - b0);
            item_abs_sum<T>(a, wi, b0, nb, s_red);
            for (int idx = tid; idx < nb * slot * 2; idx += blockDim.x) boxu[idx] = 0ull;
            __syncthreads();
            if (tid == 0) item_quantum<T>(a, nwarps, s_red);
            __syncthreads();
            const ItemQuantum<T> iq(s_red);
            const T inv_q = iq.inv_q, q_lo = iq.q_lo, q_hi = iq.q_hi;
            if (iq.any) {
                const int per = (wi.count + nwarps - 1) / nwarps;
                const int jlo = warp * per, jhi = min(wi.count, jlo + per);
                for (int bb = 0; bb < nb; ++bb) {
                    unsigned char* bx = reinterpret_cast<unsigned char*>(boxu + static_cast<size_t>(bb) * slot * 2);
                    int seg = -1, seg_lb0 = 0, col = 0;
                    RowSums<T, A> acc;
                    acc.zero();
                    auto flush = [&]() {
                        if (col < box1) {
#pragma unroll
                            for (int q = 0; q < A; ++q) {
                                if (q < nw) {
                                    FixedCell<T>::add(bx, (seg_lb0 + q) * box1 + col, slot, acc.re(q), acc.im(q));
                                }
                            }
                        }
                    };
                    // node data of the next chunk, loaded one chunk ahead: coordinates
                    // and permutation during phase A, the input value before phase B
                    T nx[3] = {T(0), T(0), T(0)};
                    uint32_t nperm = 0;
                    CT ng = cmake<T>(T(0), T(0));
                    auto load_xp = [&](int c) {
                        if (c + lane < jhi) {
                            const long long i = static_cast<long long>(wi.start) + c + lane;
                            nx[0] = a.xs[i * 2];
                            nx[1] = a.xs[i * 2 + 1];
                            nperm = a.perm[i];
                        }
                    };
                    auto load_g = [&](int c) {
                        if (c + lane < jhi) ng = a.fin[static_cast<long long>(b0 + bb) * a.N + nperm];
                    };
                    load_xp(jlo);
                    load_g(jlo);
                    for (int c0 = jlo; c0 < jhi; c0 += 32) {
                        const int nc = min(32, jhi - c0);
                        const T cx[3] = {nx[0], nx[1], T(0)};
                        const CT cg = ng;
                        load_xp(c0 + 32);
                        // ---- phase A: this lane's node
                        if (lane < nc) {
                            T tau[3];
                            int lb[3] = {0, 0, 0};
                            node_setup_v<T, 2>(cx, a.g, org, tau, lb, m);
                            T* row = s_tab + lane * RS;
                            if (a.wfac) {   // stored factors (step 0b)
                                copy_factor_rows<T, W>(a.wfac + (static_cast<long long>(wi.start) + c0 + lane) * a.wstride,
                                                       row, 2, nw);
                            } else {
                                tap_weights_to2<T, W>(row, row + A, wk, tau[0], tau[1], a.w);
                            }
                            row[2 * A] = cg.x * inv_q;
                            row[2 * A + 1] = cg.y * inv_q;
                            // segment key (box row, column segment) and the node's first
                            // column within its segment: lane l's column is base + l,
                            // so its tap index is l - t0
                            const int segc = lb[1] / S;
                            int* ri = reinterpret_cast<int*>(row + 2 * A + 2);
                            ri[0] = lb[0] | (segc << 16);
                            ri[1] = lb[1] - segc * S;
                        }
                        __syncwarp();
                        load_g(c0 + 32);
                        // ---- phase B: walk the chunk (two nodes at a time while both
                        // stay in the current segment)
                        // per-node meta data: the input value and (key, t0), one vector each
                        auto meta_g = [&](const T* row) { return *reinterpret_cast<const CT*>(row + 2 * A); };
                        auto meta_k = [&](const T* row) { return *reinterpret_cast<const int2*>(row + 2 * A + 2); };
                        auto one = [&](const T* row) {
                            const int2 kt = meta_k(row);
                            const int key = kt.x;
                            if (key != seg) {
                                if (seg >= 0) flush();
                                seg = key;
                                seg_lb0 = key & 0xFFFF;
                                col = (key >> 16) * S + lane;
                                acc.zero();
                            }
                            const int t = lane - kt.y;
                            const bool in = static_cast<unsigned>(t) < static_cast<unsigned>(nw);
                            const T wf = in ? row[A + (in ? t : 0)] : T(0);
                            const CT g = meta_g(row);
                            const T gr = g.x * wf, gi = g.y * wf;
                            T w0r[A];
                            load_row<T, A>(row, w0r);
                            acc.add(gr, gi, w0r, nw);
                        };
                        int k = 0;
#pragma unroll 1
                        for (; W != 0 && k + 1 < nc; k += 2) {   // (runtime-m kernels walk singly)
                            const T* ra = s_tab + k * RS;
                            const T* rb = ra + RS;
                            const int2 kta = meta_k(ra), ktb = meta_k(rb);
                            if (kta.x == seg && ktb.x == seg) {
                                const int ta = lane - kta.y, tb = lane - ktb.y;
                                const bool ina = static_cast<unsigned>(ta) < static_cast<unsigned>(nw);
                                const bool inb = static_cast<unsigned>(tb) < static_cast<unsigned>(nw);
                                const T wfa = ina ? ra[A + (ina ? ta : 0)] : T(0);
                                const T wfb = inb ? rb[A + (inb ? tb : 0)] : T(0);
                                const CT ga = meta_g(ra), gb = meta_g(rb);
                                const T gra = ga.x * wfa, gia = ga.y * wfa;
                                const T grb = gb.x * wfb, gib = gb.y * wfb;
                                T wa[A], wb[A];
                                load_row<T, A>(ra, wa);
                                load_row<T, A>(rb, wb);
                                acc.add(gra, gia, wa, nw);
                                acc.add(grb, gib, wb, nw);
                            } else {
                                one(ra);
                                one(rb);
                            }
                        }
#pragma unroll 1
                        for (; k < nc; ++k) one(s_tab + k * RS);
                        __syncwarp();
                    }
                    if (seg >= 0) flush();
                }
            }
            __syncthreads();
            for (int idx = tid; idx < nb * box_cells; idx += blockDim.x) {
                const int bb = idx / box_cells;
                const int cell = idx - bb * box_cells;
                const unsigned char* grp = reinterpret_cast<const unsigned char*>(boxu + static_cast<size_t>(bb) * slot * 2);
                CT v;
                v.x = FixedCell<T>::value(grp, cell, slot, 0, q_lo, q_hi);
                v.y = FixedCell<T>::value(grp, cell, slot, 1, q_lo, q_hi);
                a.part[(static_cast<long long>(item) * a.batch + b0 + bb) * box_cells + cell] = v;
            }
            __syncthreads();
        }
    }
}

// d = 3 spreading.  Warp w walks a contiguous share of the item's (cell-
// sorted) nodes in chunks of 32: lane l first evaluates the 3 x 2m window
// values of chunk node l into row l of the warp's node table (the input
// value is stored pre-scaled to quanta); the warp then takes the chunk's
// runs of nodes with equal first taps (same cell).  For a run, lane l owns
// the (a1, a2) tap pairs l, l + 32, ... of the (2m)^2 pairs and sums, over
// the run's nodes, the 2m values of its pair along dimension 0 in
// registers; each sum goes to the box once.
template <typename T, int W>
__global__ void __launch_bounds__(512, 1) spread3_kernel(const TapArgs<T> a) {
    using CT = C2<T>;
    constexpr int A = TapN<W>::A;
    constexpr int RS = spread3_row<T>(A);
    static_assert(A % 2 == 0, "node-table rows must stay 16-byte aligned");
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    const int npairs = nw * nw;
    extern __shared__ __align__(128) unsigned char smem[];
    const int bx0 = a.g.box[0], bx1 = a.g.box[1], bx2 = a.g.box[2];
    const int box_cells = bx0 * bx1 * bx2;
    const int nbmax = a.spread_batch;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const SpreadSmem Ls = spread3_layout<T>(A, box_cells, nbmax, nwarps);
    unsigned char* boxc = smem + Ls.box;
    unsigned long long* boxz = reinterpret_cast<unsigned long long*>(smem + Ls.box);
    T* s_tab = reinterpret_cast<T*>(smem + Ls.w) + static_cast<size_t>(warp) * 32 * RS;
    double* s_red = reinterpret_cast<double*>(smem + Ls.red);
    const int wk = weight_kind(a.w);
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        tile_origin<3>(a.g, wi.tile, periodic, org);
        for (int b0 = 0; b0 < a.batch; b0 += nbmax) {
            const int nb = min(nbmax, a.batch - b0);
            item_abs_sum<T>(a, wi, b0, nb, s_red);
            for (int idx = tid; idx < nb * box_cells * 2; idx += blockDim.x) boxz[idx] = 0ull;
            __syncthreads();
            if (tid == 0) item_quantum<T>(a, nwarps, s_red);
            __syncthreads();
            const ItemQuantum<T> iq(s_red);
            const T inv_q = iq.inv_q, q_lo = iq.q_lo, q_hi = iq.q_hi;
            if (iq.any) {
                const int per = (wi.count + nwarps - 1) / nwarps;
                const int jlo = warp * per, jhi = min(wi.count, jlo + per);
                for (int bb = 0; bb < nb; ++bb) {
                    unsigned char* bx = boxc + static_cast<size_t>(bb) * box_cells * 16;
                    for (int c0 = jlo; c0 < jhi; c0 += 32) {
                        const int nc = min(32, jhi - c0);
                        // ---- phase A: this lane's node
                        if (lane < nc) {
                            const long long i = static_cast<long long>(wi.start) + c0 + lane;
                            T tau[3];
                            int lb[3] = {0, 0, 0};
                            node_setup<T, 3>(a.xs, i, a.g, org, tau, lb, m);
                            T* row = s_tab + lane * RS;
                            if (a.wfac) {   // stored factors (step 0b)
                                copy_factor_rows<T, W>(a.wfac + i * a.wstride, row, 3, nw);
                            } else {
#pragma unroll
                                for (int t = 0; t < 3; ++t) tap_weights_to<T, W>(row + t * A, wk, tau[t], a.w);
                            }
                            const CT gv = a.fin[static_cast<long long>(b0 + bb) * a.N + a.perm[i]];
                            row[3 * A] = gv.x * inv_q;
                            row[3 * A + 1] = gv.y * inv_q;
                            reinterpret_cast<int*>(row + 3 * A + 2)[0] = lb[0] | (lb[1] << 10) | (lb[2] << 20);
                        }
                        __syncwarp();
                        // ---- phase B: runs of equal first taps
                        int k = 0;
                        while (k < nc) {
                            const int key = reinterpret_cast<const int*>(s_tab + k * RS + 3 * A + 2)[0];
                            int k1 = k + 1;
                            while (k1 < nc && reinterpret_cast<const int*>(s_tab + k1 * RS + 3 * A + 2)[0] == key) ++k1;
                            const int lb0 = key & 1023, lb1 = (key >> 10) & 1023, lb2 = key >> 20;
                            for (int p0 = 0; p0 < npairs; p0 += 32) {
                                const int pp = p0 + lane;
                                const bool valid = pp < npairs;
                                const int a1 = valid ? pp / nw : 0;
                                const int a2 = valid ? pp - a1 * nw : 0;
                                RowSums<T, A> acc;
                                acc.zero();
                                for (int kk = k; kk < k1; ++kk) {
                                    const T* row = s_tab + kk * RS;
                                    const T w12 = row[A + a1] * row[2 * A + a2];
                                    const T gr = row[3 * A] * w12, gi = row[3 * A + 1] * w12;
                                    T w0r[A];
                                    load_row<T, A>(row, w0r);
                                    acc.add(gr, gi, w0r, nw);
                                }
                                if (valid) {
                                    const int base = (lb0 * bx1 + lb1 + a1) * bx2 + lb2 + a2;
                                    const int pitch0 = bx1 * bx2;
#pragma unroll
                                    for (int q = 0; q < A; ++q)
                                        if (q < nw)
                                            FixedCell<T>::add(bx, base + q * pitch0, box_cells, acc.re(q), acc.im(q));
                                }
                            }
                            k = k1;
                        }
                        __syncwarp();
                    }
                }
            }
            __syncthreads();
            for (int idx = tid; idx < nb * box_cells; idx += blockDim.x) {
                const int bb = idx / box_cells;
                const int cell = idx - bb * box_cells;
                const unsigned char* grp = boxc + static_cast<size_t>(bb) * box_cells * 16;
                CT v;
                v.x = FixedCell<T>::value(grp, cell, box_cells, 0, q_lo, q_hi);
                v.y = FixedCell<T>::value(grp, cell, box_cells, 1, q_lo, q_hi);
                a.part[(static_cast<long long>(item) * a.batch + b0 + bb) * box_cells + cell] = v;
            }
            __syncthreads();
        }
    }
}

// d = 3 spreading, column-owner form (FP32, 8 x 8 x 8 tiles, W = 2m <= 16).
// Lane (c1, c2) of the block owns box column (c1, c2) and keeps its R cells
// along dimension 0 in registers for the whole work item; warp w owns the
// patch of 4 x 8 columns at (4 (w / P2), 8 (w mod P2)).  The item's nodes
// go through node tables of C nodes:
//  phase A: one thread per (node, dimension) writes the node's 2m window
//    values of that dimension at their box positions, zero elsewhere
//    (dimension 0: R rows; dimensions 1, 2: one value per lane column), and
//    the dimension-0 thread its input value and the mask of the warps whose
//    patch meets the node's 2m x 2m window of columns;
//  phase B: every warp in a node's mask adds g * w1[c1] * w2[c2] * w0[q] to
//    its R registers, one packed FMA per row (lanes outside the window add
//    zero); two nodes per step.
// Two tables alternate: the threads fill the next table (phase A) as soon
// as they are done reading the current one (phase B), with one block barrier
// per table.  Each box value is the sum of its nodes' contributions in the
// item's node order, formed by one lane: no atomics, no fixed point, and the
// result is bitwise reproducible.  The box goes to the item's slot of the
// ordered flush (gather_kernel), as the other spread kernels' boxes do.
template <int W>
__device__ __forceinline__ void spread3c_fill(const TapArgs<float>& a, float* tab, const WorkItem& wi,
                                              const int (&org)[3], int c0, int b, int wk) {
    using G = Spread3C<W>;
    constexpr int m = W / 2;
    const int nc = min(G::C, wi.count - c0);
    for (int j = threadIdx.x; j < 3 * nc; j += blockDim.x) {
        const int k = j / 3, t = j - 3 * k;
        const long long i = static_cast<long long>(wi.start) + c0 + k;
        float tau[3];
        int lb[3] = {0, 0, 0};
        node_setup<float, 3>(a.xs, i, a.g, org, tau, lb, m);
        float* row = tab + static_cast<size_t>(k) * G::ROW;
        const int off = (t == 0) ? 0 : (t == 1) ? G::O1 : G::O2;
        const int len = (t == 0) ? G::RP : (t == 1) ? 4 * G::P1 : 8 * G::P2;
        const int lbt = (t == 0) ? lb[0] : (t == 1) ? lb[1] : lb[2];
        const float taut = (t == 0) ? tau[0] : (t == 1) ? tau[1] : tau[2];
        float* dst = row + off;
        for (int q = 0; q < len; ++q)
            if (q < lbt || q >= lbt + W) dst[q] = 0.0f;
        if (a.wfac) {   // stored factors (step 0b)
            const float* src = a.wfac + i * a.wstride + t * W;
#pragma unroll
            for (int q = 0; q < W; ++q) dst[lbt + q] = src[q];
        } else {
            tap_weights_to<float, W>(dst + lbt, wk, taut, a.w);
        }
        if (t == 0) {
            const float2 gv = a.fin[static_cast<long long>(b) * a.N + a.perm[i]];
            unsigned mask = 0;
            for (int r1 = lb[1] / 4; r1 <= (lb[1] + W - 1) / 4 && r1 < G::P1; ++r1)
                for (int r2 = lb[2] / 8; r2 <= (lb[2] + W - 1) / 8 && r2 < G::P2; ++r2)
                    mask |= 1u << (r1 * G::P2 + r2);
            *reinterpret_cast<float4*>(row + G::OM) = make_float4(gv.x, gv.y, __uint_as_float(mask), 0.0f);
        }
    }
}

template <int W>
__device__ __forceinline__ void spread3c_add(float2 (&acc)[Spread3C<W>::R], const float* row, float2 gw) {
    using G = Spread3C<W>;
#pragma unroll
    for (int q = 0; q < G::RP; q += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + q);
        acc[q] = cfma(gw, v.x, acc[q]);
        if (q + 1 < G::R) acc[q + 1] = cfma(gw, v.y, acc[q + 1]);
        if (q + 2 < G::R) acc[q + 2] = cfma(gw, v.z, acc[q + 2]);
        if (q + 3 < G::R) acc[q + 3] = cfma(gw, v.w, acc[q + 3]);
    }
}

template <int W>
__device__ __forceinline__ void spread3c_add2(float2 (&acc)[Spread3C<W>::R], const float* ra, float2 ga,
                                              const float* rb, float2 gb) {
    using G = Spread3C<W>;
#pragma unroll
    for (int q = 0; q < G::RP; q += 4) {
        const float4 va = *reinterpret_cast<const float4*>(ra + q);
        const float4 vb = *reinterpret_cast<const float4*>(rb + q);
        acc[q] = cfma(gb, vb.x, cfma(ga, va.x, acc[q]));
        if (q + 1 < G::R) acc[q + 1] = cfma(gb, vb.y, cfma(ga, va.y, acc[q + 1]));
        if (q + 2 < G::R) acc[q + 2] = cfma(gb, vb.z, cfma(ga, va.z, acc[q + 2]));
        if (q + 3 < G::R) acc[q + 3] = cfma(gb, vb.w, cfma(ga, va.w, acc[q + 3]));
    }
}

template <int W>
__global__ void __launch_bounds__(Spread3C<W>::THREADS, 1) spread3c_kernel(const TapArgs<float> a) {
    using G = Spread3C<W>;
    constexpr int R = G::R, C = G::C, ROW = G::ROW;
    constexpr int box_cells = R * G::B1 * G::B2;
    extern __shared__ __align__(16) float s_tab[];   // two tables of C rows of ROW floats
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c1 = 4 * (warp / G::P2) + (lane >> 3), c2 = 8 * (warp % G::P2) + (lane & 7);   // this lane's column
    const bool owner = c1 < G::B1 && c2 < G::B2;
    const unsigned wbit = 1u << warp;
    const int wk = weight_kind(a.w);
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    for (int b = 0; b < a.batch; ++b) {
        int item = blockIdx.x;
        if (item >= a.n_work) return;
        WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        tile_origin<3>(a.g, wi.tile, periodic, org);
        int c0 = 0, buf = 0;
        float2 acc[R];
#pragma unroll
        for (int q = 0; q < R; ++q) acc[q] = make_float2(0.0f, 0.0f);
        spread3c_fill<W>(a, s_tab, wi, org, c0, b, wk);
        __syncthreads();
        while (true) {
            // ---- phase B on table `buf`: nodes c0 .. c0 + nc - 1 of the item
            const float* tab = s_tab + static_cast<size_t>(buf) * C * ROW;
            const int nc = min(C, wi.count - c0);
            int k = 0;
#pragma unroll 1
            for (; k + 1 < nc; k += 2) {
                const float* ra = tab + static_cast<size_t>(k) * ROW;
                const float* rb = ra + ROW;
                const float4 ma = *reinterpret_cast<const float4*>(ra + G::OM);
                const float4 mb = *reinterpret_cast<const float4*>(rb + G::OM);
                const bool ina = (__float_as_uint(ma.z) & wbit) != 0, inb = (__float_as_uint(mb.z) & wbit) != 0;
                if (!ina && !inb) continue;
                const float wa = ina ? ra[G::O1 + c1] * ra[G::O2 + c2] : 0.0f;
                const float wb = inb ? rb[G::O1 + c1] * rb[G::O2 + c2] : 0.0f;
                const float2 ga = make_float2(ma.x * wa, ma.y * wa), gb = make_float2(mb.x * wb, mb.y * wb);
                if (ina && inb) spread3c_add2<W>(acc, ra, ga, rb, gb);
                else if (ina) spread3c_add<W>(acc, ra, ga);
                else spread3c_add<W>(acc, rb, gb);
            }
            if (k < nc) {
                const float* ra = tab + static_cast<size_t>(k) * ROW;
                const float4 ma = *reinterpret_cast<const float4*>(ra + G::OM);
                if (__float_as_uint(ma.z) & wbit) {
                    const float wa = ra[G::O1 + c1] * ra[G::O2 + c2];
                    spread3c_add<W>(acc, ra, make_float2(ma.x * wa, ma.y * wa));
                }
            }
            // ---- next table: the item's next nodes, or the next item
            int nitem = item, nc0 = c0 + C;
            if (nc0 >= wi.count) {
                if (owner) {
                    float2* dst = a.part + (static_cast<long long>(item) * a.batch + b) * box_cells + c1 * G::B2 + c2;
#pragma unroll
                    for (int q = 0; q < R; ++q) dst[q * G::B1 * G::B2] = acc[q];
                }
#pragma unroll
                for (int q = 0; q < R; ++q) acc[q] = make_float2(0.0f, 0.0f);
                nitem = item + gridDim.x;
                nc0 = 0;
            }
            if (nitem >= a.n_work) break;
            if (nitem != item) {
                wi = a.work[nitem];
                tile_origin<3>(a.g, wi.tile, periodic, org);
            }
            item = nitem;
            c0 = nc0;
            buf ^= 1;
            spread3c_fill<W>(a, s_tab + static_cast<size_t>(buf) * C * ROW, wi, org, c0, b, wk);
            __syncthreads();
        }
        __syncthreads();   // before the next batch entry refills table 0
    }
}

#include "spread3t.cuh"

// d = 1 spreading.  Nodes are staged `sub` at a time (weights and the
// pre-scaled inputs in shared memory); runs of nodes in one cell share their
// 2m taps.  A warp takes a run: lane l owns tap c = l mod 2m and row group
// l div 2m, the row groups split the run's nodes, and every lane adds its
// partial sum to the box once (exact integer adds).
template <typename T, int W>
__global__ void __launch_bounds__(kTapThreads) spread1_kernel(const TapArgs<T> a) {
    using CT = C2<T>;
    constexpr int A = TapN<W>::A;
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    const int box_cells = a.g.box[0];
    const int slot = (box_cells + 1) / 2 * 2;
    const int nbmax = a.spread_batch;
    const int sub = a.spread_sub;
    const SpreadSmem Ls = spread_smem_layout<T>(1, A, box_cells, nbmax, sub);
    unsigned char* boxc = smem + Ls.box;
    unsigned long long* boxz = reinterpret_cast<unsigned long long*>(boxc);
    int* s_lb = reinterpret_cast<int*>(smem + Ls.lb);
    T* s_w = reinterpret_cast<T*>(smem + Ls.w);
    CT* s_g = reinterpret_cast<CT*>(smem + Ls.g);
    int* s_run = reinterpret_cast<int*>(smem + Ls.run);
    double* s_red = reinterpret_cast<double*>(smem + Ls.red);
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    const int wk = weight_kind(a.w);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int G = 32 / nw;        // row groups per warp
    const int c = lane % nw;      // owned tap
    const int rg = lane / nw;     // row group
    const bool active = rg < G;
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        tile_origin<1>(a.g, wi.tile, periodic, org);
        for (int b0 = 0; b0 < a.batch; b0 += nbmax) {
            const int nb = min(nbmax, a.batch - b0);
            item_abs_sum<T>(a, wi, b0, nb, s_red);
            for (int idx = tid; idx < nb * slot * 2; idx += blockDim.x) boxz[idx] = 0ull;
            __syncthreads();
            if (tid == 0) item_quantum<T>(a, nwarps, s_red);
            __syncthreads();
            const ItemQuantum<T> iq(s_red);
            if (iq.any) {
                for (int s0 = 0; s0 < wi.count; s0 += sub) {
                    const int ns = min(sub, wi.count - s0);
                    if (tid < ns) {
                        const long long i = static_cast<long long>(wi.start) + s0 + tid;
                        T tau[3];
                        int lb[3] = {0, 0, 0};
                        node_setup<T, 1>(a.xs, i, a.g, org, tau, lb, m);
                        s_lb[tid] = lb[0];
                        tap_weights_to<T, W>(s_w + static_cast<size_t>(tid) * A, wk, tau[0], a.w);
                        const long long src = a.perm[i];
                        for (int bb = 0; bb < nb; ++bb) {
                            const CT gv = a.fin[static_cast<long long>(b0 + bb) * a.N + src];
                            s_g[bb * sub + tid] = cmake<T>(gv.x * iq.inv_q, gv.y * iq.inv_q);
                        }
                    }
                    __syncthreads();
                    // runs of equal first taps (same cell), indexed in order
                    const int flag = (tid < ns) && (tid == 0 || s_lb[tid] != s_lb[tid - 1]);
                    const unsigned bal = __ballot_sync(0xffffffffu, flag);
                    const int before = __popc(bal & ((1u << lane) - 1u));
                    if (lane == 0) s_red[warp] = __popc(bal);
                    __syncthreads();
                    int wbase = 0, nruns = 0;
                    for (int w = 0; w < warp; ++w) wbase += static_cast<int>(s_red[w]);
                    for (int w = 0; w < nwarps; ++w) nruns += static_cast<int>(s_red[w]);
                    if (flag) s_run[wbase + before] = tid;
                    if (tid == 0) s_run[nruns] = ns;
                    __syncthreads();
                    if (active) {
                        for (int r = warp; r < nruns; r += nwarps) {
                            const int jlo = s_run[r], jhi = s_run[r + 1];
                            const int lb0 = s_lb[jlo];
                            for (int bb = 0; bb < nb; ++bb) {
                                const CT* gg = s_g + bb * sub;
                                CT acc = cmake<T>(T(0), T(0));
                                for (int j = jlo + rg; j < jhi; j += G)
                                    acc = cfma(gg[j], s_w[static_cast<size_t>(j) * A + c], acc);
                                FixedCell<T>::add(boxc + static_cast<size_t>(bb) * slot * 16, lb0 + c, slot, acc.x, acc.y);
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
            for (int idx = tid; idx < nb * box_cells; idx += blockDim.x) {
                const int bb = idx / box_cells;
                const int cell = idx - bb * box_cells;
                const unsigned char* grp = boxc + static_cast<size_t>(bb) * slot * 16;
                CT v;
                v.x = FixedCell<T>::value(grp, cell, slot, 0, iq.q_lo, iq.q_hi);
                v.y = FixedCell<T>::value(grp, cell, slot, 1, iq.q_lo, iq.q_hi);
                a.part[(static_cast<long long>(item) * a.batch + b0 + bb) * box_cells + cell] = v;
            }
            __syncthreads();
        }
    }
}

// Ordered flush: grid[b][l] = sum over the boxes covering l, in a fixed order.
template <typename T, int D>
__global__ void __launch_bounds__(256, 8) gather_kernel(const TapArgs<T> a) {
    using CT = C2<T>;
    constexpr int kMaxCand = 48;   // >= 3 periodic images x (box/T + 1) tiles, T >= 2
    const long long total = static_cast<long long>(a.batch) * a.grid_stride;
    const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (idx >= total) return;
    const int b = static_cast<int>(idx / a.grid_stride);
    long long rem = idx - static_cast<long long>(b) * a.grid_stride;
    int gc[3] = {0, 0, 0};
#pragma unroll
    for (int t = D - 1; t >= 0; --t) {
        gc[t] = static_cast<int>(rem % a.g.L[t]);
        rem /= a.g.L[t];
    }
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    // candidate (tile coordinate, local coordinate) pairs per dimension
    int cand_c[3][kMaxCand], cand_l[3][kMaxCand], ncand[3] = {0, 0, 0};
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const int T_ = a.g.T[t], box = a.g.box[t], off = a.g.off[t], L = a.g.L[t];
        for (int k = periodic ? -1 : 0; k <= (periodic ? 1 : 0); ++k) {
            const int gp = gc[t] + k * L;
            // tiles c with c*T - off <= gp < c*T - off + box
            int clo = gp + off - box + 1;
            clo = (clo >= 0) ? (clo + T_ - 1) / T_ : -((-clo) / T_);
            int chi = gp + off;
            chi = (chi >= 0) ? chi / T_ : -((-chi + T_ - 1) / T_);
            clo = max(clo, 0);
            chi = min(chi, a.g.nt[t] - 1);
            for (int cc = clo; cc <= chi; ++cc) {
                if (ncand[t] < kMaxCand) {
                    cand_c[t][ncand[t]] = cc;
                    cand_l[t][ncand[t]] = gp - (cc * T_ - off);
                    ncand[t]++;
                } else {
                    atomicOr(a.err, DEVERR_INTERNAL);
                }
            }
        }
    }
    int box_cells = 1;
#pragma unroll
    for (int t = 0; t < D; ++t) box_cells *= a.g.box[t];
    T sr = T(0), si = T(0);
    const int n1 = D > 1 ? ncand[1] : 1, n2 = D > 2 ? ncand[2] : 1;
    for (int i0 = 0; i0 < ncand[0]; ++i0) {
        for (int i1 = 0; i1 < n1; ++i1) {
            for (int i2 = 0; i2 < n2; ++i2) {
                int tile = cand_c[0][i0];
                int local = cand_l[0][i0];
                if (D > 1) {
                    tile = tile * a.g.nt[1] + cand_c[1][i1];
                    local = local * a.g.box[1] + cand_l[1][i1];
                }
                if (D > 2) {
                    tile = tile * a.g.nt[2] + cand_c[2][i2];
                    local = local * a.g.box[2] + cand_l[2][i2];
                }
                const uint32_t s = a.tile_items[tile], e = a.tile_items[tile + 1];
                for (uint32_t it = s; it < e; ++it) {
                    const CT v = a.part[(static_cast<long long>(it) * a.batch + b) * box_cells + local];
                    sr += v.x;
                    si += v.y;
                }
            }
        }
    }
    a.grid[idx] = cmake<T>(sr, si);
}

// The d partial derivatives of one node's short sum in one pass over its
// taps: dimension t's derivative replaces that dimension's weights by their
// derivatives (the tensor product rule), so every box value is loaded once
// and enters each derivative's sum (d = 2: two sums per row; d = 3: the row
// sums with w2 and dw2 feed three partial sums).  g[t] = d f / d x_t.
template <typename T, int D, int W>
__device__ __forceinline__ void contract_grad(const C2<T>* __restrict__ box, const TileGeom& g, const int (&lb)[3],
                                              const T (&w)[3][TapN<W>::A], const T (&dw)[3][TapN<W>::A], int nw_rt,
                                              C2<T> (&gr)[3]) {
    const int nw = W ? W : nw_rt;
#pragma unroll
    for (int t = 0; t < 3; ++t) gr[t] = cmake<T>(T(0), T(0));
    if constexpr (D == 1) {
        const C2<T>* p = box + lb[0];
#pragma unroll
        for (int a = 0; a < TapN<W>::A; ++a)
            if (a < nw) gr[0] = cfma(p[a], dw[0][a], gr[0]);
    } else if constexpr (D == 2) {
        const int pitch = g.box[1];
        const C2<T>* p = box + lb[0] * pitch + lb[1];
#pragma unroll 2
        for (int a = 0; a < nw; ++a) {
            const C2<T>* row = p + a * pitch;
            C2<T> r = cmake<T>(T(0), T(0)), rd = cmake<T>(T(0), T(0));
#pragma unroll
            for (int b = 0; b < TapN<W>::A; ++b) {
                if (b < nw) {
                    const C2<T> v = row[b];
                    r = cfma(v, w[1][b], r);
                    rd = cfma(v, dw[1][b], rd);
                }
            }
            gr[0] = cfma(r, dw[0][a], gr[0]);
            gr[1] = cfma(rd, w[0][a], gr[1]);
        }
    } else {
        const int p1 = g.box[2];
        const int p0 = g.box[1] * p1;
        const C2<T>* p = box + lb[0] * p0 + lb[1] * p1 + lb[2];
        for (int a = 0; a < nw; ++a) {
            C2<T> m0 = cmake<T>(T(0), T(0)), m1 = m0, m2 = m0;
#pragma unroll 2
            for (int b = 0; b < nw; ++b) {
                const C2<T>* row = p + a * p0 + b * p1;
                C2<T> r = cmake<T>(T(0), T(0)), rd = cmake<T>(T(0), T(0));
#pragma unroll
                for (int c = 0; c < TapN<W>::A; ++c) {
                    if (c < nw) {
                        const C2<T> v = row[c];
                        r = cfma(v, w[2][c], r);
                        rd = cfma(v, dw[2][c], rd);
                    }
                }
                m0 = cfma(r, w[1][b], m0);
                m1 = cfma(r, dw[1][b], m1);
                m2 = cfma(rd, w[1][b], m2);
            }
            gr[0] = cfma(m0, dw[0][a], gr[0]);
            gr[1] = cfma(m1, w[0][a], gr[1]);
            gr[2] = cfma(m2, w[0][a], gr[2]);
        }
    }
}

// Node gradient: grad_x[j, t] = sum_b Re(conj(gf[b, j]) * d f_{b,j} / d x_{j,t}).
template <typename T, int D, int W>
__global__ void __launch_bounds__(kTapThreads) node_grad_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                const TapArgs<T> a) {
    using CT = C2<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    CT* box = aligned_box_base<T>(smem);
    int box_cells = 1;
#pragma unroll
    for (int t = 0; t < D; ++t) box_cells *= a.g.box[t];
    const int slot = box_slot_cells<T>(box_cells);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        prefetch_tmap(&tmap);
    }
    __syncthreads();
    uint32_t phase = 0;
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    constexpr int A = TapN<W>::A;
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        const bool wrap = tile_origin<D>(a.g, wi.tile, periodic, org);
        for (int b0 = 0; b0 < a.batch; b0 += a.batch_smem) {
            const int nb = min(a.batch_smem, a.batch - b0);
            if (!stage_box<T, D>(&tmap, a, box, box_cells, slot, org, wrap, b0, nb, &bar, phase)) {
                if (!a.stall) mbar_wait_bounded(&bar, phase ^ 1u, a.err);   // let the copy in flight land
                return;
            }
            for (int j = threadIdx.x; j < wi.count; j += blockDim.x) {
                const long long i = static_cast<long long>(wi.start) + j;
                T tau[3];
                int lb[3] = {0, 0, 0};
                node_setup<T, D>(a.xs, i, a.g, org, tau, lb, m);
                T w[3][A], dw[3][A];
#pragma unroll
                for (int t = 0; t < D; ++t) tap_weights_d<T, W>(tau[t], static_cast<T>(a.g.L[t]), a.w, w[t], dw[t]);
                const long long dst = a.perm[i];
                T gsum[3] = {T(0), T(0), T(0)};
                for (int bb = 0; bb < nb; ++bb) {
                    const CT* bx = box + bb * slot;
                    const CT gf = a.fin[static_cast<long long>(b0 + bb) * a.N + dst];
                    CT dv[3];
                    contract_grad<T, D, W>(bx, a.g, lb, w, dw, nw, dv);
#pragma unroll
                    for (int t = 0; t < D; ++t) gsum[t] += gf.x * dv[t].x + gf.y * dv[t].y;
                }
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    T* o = a.gradx + dst * D + t;
                    *o = (b0 == 0) ? gsum[t] : (*o + gsum[t]);
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Host launcher for one (precision, dimension): dispatch on m = W/2.

// spread3t_kernel serves single-batch FP32 plans without stored factors whose
// window has a per-tap closed form there (sinh, tabulated Shannon window, or
// fitted polynomials); the geometry test is the column-owner kernel's.
inline bool spread3t_applies(const TapArgs<float>& a) {
    if (a.batch != 1 || a.wfac != nullptr || a.fsorted == nullptr) return false;
    if (a.w.poly) return true;
    return a.w.window == NFFTBL_WIN_SINH || (a.w.window == NFFTBL_WIN_TABLE && a.w.method == NFFTBL_SHANNON);
}

// interp3p_kernel serves single-batch d = 3 FP32 plans of the Shannon method
// with pair heads (its tiles never wrap) whose boxes are large enough that
// interp_kernel fits at most two blocks on an SM (above 75 KB: m >= 7 with
// 8^3 tiles), while two of them still fit in one block.
inline bool interp3p_applies(const TapArgs<float>& a) {
    if (a.g.d != 3 || a.heads == nullptr || a.nheads == nullptr || a.batch != 1 || a.w.method != NFFTBL_SHANNON)
        return false;
    const long long cells = static_cast<long long>(a.g.box[0]) * a.g.box[1] * a.g.box[2];
    const long long slot = (cells * 8 + 127) / 128 * 128;
    return slot > 75 * 1024 && 2 * slot + 128 <= 200 * 1024;
}

template <typename T, int D, int W>
nfftbl_status launch_tap_kernel(nfftbl_plan_s* p, const TapArgs<T>& args, int kind, size_t smem) {
    void* fn = nullptr;
    if (kind == TAP_INTERP) fn = reinterpret_cast<void*>(interp_kernel<T, D, W>);
    if (kind == TAP_SPREAD) {
        if constexpr (D == 1) fn = reinterpret_cast<void*>(spread1_kernel<T, W>);
        else if constexpr (D == 2) fn = reinterpret_cast<void*>(spread2_kernel<T, W>);
        else fn = reinterpret_cast<void*>(spread3_kernel<T, W>);
    }
    const int threads = (kind == TAP_SPREAD && D == 3) ? 32 * args.spread_warps : kTapThreads;
    if (kind == TAP_GRAD) fn = reinterpret_cast<void*>(node_grad_kernel<T, D, W>);
    if (kind == TAP_FACTORS) {
        if (args.N <= 0) return NFFTBL_OK;
        int occf = 0;
        nfftbl_status stf = check_cuda(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                              &occf, factor_kernel<T, D, W>, 256, 0), "occupancy");
        if (stf != NFFTBL_OK) return stf;
        const long long wantf = static_cast<long long>(std::max(occf, 1)) * p->num_sms;
        const unsigned gridf = static_cast<unsigned>(std::min<long long>(wantf, (args.N + 255) / 256));
        factor_kernel<T, D, W><<<gridf, 256, 0, p->stream>>>(args, static_cast<T*>(p->wfac.p));
        p->launches++;
        return check_cuda(p, cudaGetLastError(), "factor kernel launch");
    }
    int threads_launch = threads;
    bool pipe = false, tensor = false;
    if constexpr (D == 3 && sizeof(T) == 4) {
        if (kind == TAP_INTERP && interp3p_applies(args)) {
            pipe = true;
            fn = reinterpret_cast<void*>(interp3p_kernel<W>);
            threads_launch = kPipeThreads;
            const int cells = args.g.box[0] * args.g.box[1] * args.g.box[2];
            smem = 2 * static_cast<size_t>(box_slot_cells<float>(cells)) * sizeof(C2<T>) + 128;
        }
    }
    if constexpr (D == 3 && sizeof(T) == 4 && W >= 4 && W <= 16) {
        if (kind == TAP_SPREAD && spread3c_applies(3, true, W / 2, p->geom.T)) {
            using G = Spread3C<W>;
            if (args.g.box[0] != G::R || args.g.box[1] != G::B1 || args.g.box[2] != G::B2)
                return fail(p, NFFTBL_EINTERNAL, "column-owner spreading: unexpected box shape");
            fn = reinterpret_cast<void*>(spread3c_kernel<W>);
            threads_launch = G::THREADS;
            smem = G::SMEM;
            if (spread3t_applies(args)) {   // the tensor-core form
                tensor = true;
                fn = reinterpret_cast<void*>(spread3t_kernel<W>);
                threads_launch = Spread3T<W>::THREADS;
                smem = Spread3T<W>::SMEM;
            }
        }
    }
    nfftbl_status st = check_cuda(p, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          static_cast<int>(smem)),
                                  "tap smem attribute");
    if (st != NFFTBL_OK) return st;
    int occ = 0;
    st = check_cuda(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads_launch, smem), "occupancy");
    if (st != NFFTBL_OK) return st;
    if (occ < 1) return fail(p, NFFTBL_EUNSUPPORTED, "tap kernel does not fit on an SM");
    const long long want = static_cast<long long>(occ) * p->num_sms;
    const unsigned grid = static_cast<unsigned>(std::max<long long>(1, std::min<long long>(want, args.n_work)));
    // (with no work items the spread kernel's CTAs exit at once; the gather still clears the grid)
    if (args.n_work == 0 && kind != TAP_SPREAD) return NFFTBL_OK;
    timing_begin(p, kind == TAP_INTERP ? NFFTBL_K_INTERP : kind == TAP_SPREAD ? NFFTBL_K_SPREAD : NFFTBL_K_GRAD);
    if (kind == TAP_INTERP && pipe) {
        if constexpr (D == 3 && sizeof(T) == 4)
            interp3p_kernel<W><<<grid, threads_launch, smem, p->stream>>>(p->tmap, args);
    } else if (kind == TAP_INTERP)
        interp_kernel<T, D, W><<<grid, kTapThreads, smem, p->stream>>>(p->tmap, args);
    else if (kind == TAP_SPREAD) {
        if constexpr (D == 1) spread1_kernel<T, W><<<grid, kTapThreads, smem, p->stream>>>(args);
        else if constexpr (D == 2) spread2_kernel<T, W><<<grid, kTapThreads, smem, p->stream>>>(args);
        else if (threads_launch != threads) {
            if constexpr (sizeof(T) == 4 && W >= 4 && W <= 16) {
                if (tensor) {
                    const unsigned gb = static_cast<unsigned>(
                        std::min<long long>((args.N + 255) / 256, 8LL * p->num_sms));
                    if (args.N > 0) {
                        sort_inputs_kernel<<<gb, 256, 0, p->stream>>>(
                            reinterpret_cast<const float2*>(args.fin), args.perm,
                            reinterpret_cast<float2*>(args.fsorted), args.N);
                        p->launches++;
                    }
                    spread3t_kernel<W><<<grid, threads_launch, smem, p->stream>>>(args);
                }
                else
                    spread3c_kernel<W><<<grid, threads_launch, smem, p->stream>>>(args);
            }
        } else spread3_kernel<T, W><<<grid, threads, smem, p->stream>>>(args);
    }
    else
        node_grad_kernel<T, D, W><<<grid, kTapThreads, smem, p->stream>>>(p->tmap, args);
    timing_end(p);
    p->launches++;
    st = check_cuda(p, cudaGetLastError(), "tap kernel launch");
    if (st != NFFTBL_OK || kind != TAP_SPREAD) return st;
    // ordered flush of the spread boxes into the grid
    const long long cells = static_cast<long long>(args.batch) * args.grid_stride;
    timing_begin(p, NFFTBL_K_FLUSH);
    gather_kernel<T, D><<<static_cast<unsigned>((cells + 255) / 256), 256, 0, p->stream>>>(args);
    timing_end(p);
    p->launches++;
    return check_cuda(p, cudaGetLastError(), "gather kernel launch");
}

}  // namespace nfftbl
