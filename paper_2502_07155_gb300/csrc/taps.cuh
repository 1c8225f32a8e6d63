// Short-sum kernels over binned nodes: interpolation (Algorithm 4.2 step 3,
// Eq. 4.8), spreading (its transpose Psi^T, the first factor of the
// adjoint) and the node derivative of the short sums.
//
// Work decomposition: one work item = one tile of T_0 x .. x T_{d-1} grid
// cells and up to K of its nodes (sorted by cell).  A CTA stages the box of
// grid values the tile's nodes can reach -- the tile plus its m-halo -- in
// shared memory (TMA tiled load; out-of-range cells are zero-filled by the
// copy engine, which is exactly the zero extension of the Shannon method
// outside I_L) and every thread evaluates one node at a time.
//
// Per node and dimension t: u = L_t x_t (exact for L_t = 2^p), cell
// i = floor(u), tau = u - i in [0, 1).  The 2m taps l = i-m+1 .. i+m (the
// members of the closed set J_{L,m}(x) with a nonzero window; the ends of
// the closed set carry phi(+-m/L) = 0) have offsets
// delta_a = L x - l = tau + m-1-a, and
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

template <typename T> struct FM;
template <> struct FM<float> {
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

// Kaiser-Bessel and tabulated windows, kept out of line: they are rare and
// their code would otherwise be inlined into every unrolled tap.
template <typename T>
__device__ __noinline__ T win_phi_other(T delta, const WinParams<T> w) {
    const T r = delta * w.inv_m;
    const T q = (T(1) - r) * (T(1) + r);
    if (!(q > T(0))) return T(0);
    if (w.window == NFFTBL_WIN_CKB) return (FM<T>::i0(w.beta * FM<T>::sqrt(q)) - T(1)) * w.c_norm;
    return table_eval(w.table, w.table_n, FM<T>::abs(r));
}

template <typename T>
__device__ __noinline__ T win_dphi_other(T delta, const WinParams<T> w) {
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
    if (w.window != NFFTBL_WIN_SINH) return win_phi_other(delta, w);
    const T r = delta * w.inv_m;
    const T q = (T(1) - r) * (T(1) + r);
    if (!(q > T(0))) return T(0);
    // sinh(beta s)/sinh(beta) = (e^{beta(s-1)} - e^{-beta(s+1)}) / (1 - e^{-2 beta})
    const T sq = FM<T>::sqrt(q);
    return (FM<T>::exp2(w.c_exp * (sq - T(1))) - FM<T>::exp2(-w.c_exp * (sq + T(1)))) * w.c_norm;
}

// d Phi / d delta; zero where |delta| >= m (the infinite edge derivative of
// the sinh / Kaiser-Bessel windows meets a vanishing factor there).
template <typename T>
__device__ __forceinline__ T win_dphi(T delta, const WinParams<T>& w) {
    if (w.window != NFFTBL_WIN_SINH) return win_dphi_other(delta, w);
    const T r = delta * w.inv_m;
    const T q = (T(1) - r) * (T(1) + r);
    if (!(q > T(0))) return T(0);
    const T sq = FM<T>::sqrt(q);
    const T ds = -r * w.inv_m / sq;
    return w.beta * (FM<T>::exp2(w.c_exp * (sq - T(1))) + FM<T>::exp2(-w.c_exp * (sq + T(1)))) * w.c_norm * ds;
}

// Tap count per dimension: W = 2m fixed at compile time, or W = 0 for a
// kernel that takes m at run time (arrays sized for m <= 12).
template <int W> struct TapN {
    static constexpr int A = W ? W : 24;
};

// The 2m tap weights psi_t(x - l/L) (Shannon) or phi_t(x - l/L) (classical)
// of one dimension, tap a at l = i - m + 1 + a.
template <typename T, int W>
__device__ __forceinline__ void tap_weights(T tau, const WinParams<T>& wp, T (&w)[TapN<W>::A]) {
    const int m = W ? W / 2 : wp.m;
    const int nw = 2 * m;
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
        T ar = T(0), ai = T(0);
#pragma unroll
        for (int a = 0; a < nw; ++a) {
            const C2<T> v = p[a];
            ar += v.x * w0[a];
            ai += v.y * w0[a];
        }
        return cmake<T>(ar, ai);
    } else if (D == 2) {
        const int pitch = g.box[1];
        const C2<T>* p = box + lb[0] * pitch + lb[1];
        if (!comp) {
            T ar = T(0), ai = T(0);
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
                ar += rr * w0[a];
                ai += ri * w0[a];
            }
            return cmake<T>(ar, ai);
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
            T ar = T(0), ai = T(0);
            for (int a = 0; a < nw; ++a) {
                T mr = T(0), mi = T(0);
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
                    mr += rr * w1[b];
                    mi += ri * w1[b];
                }
                ar += mr * w0[a];
                ai += mi * w0[a];
            }
            return cmake<T>(ar, ai);
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
        if (threadIdx.x == 0) {
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
        const bool ok = mbar_wait_bounded(bar, phase, a.err);
        phase ^= 1u;
        return __syncthreads_and(ok) != 0;   // one verdict for the whole block
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
                mbar_wait_bounded(&bar, phase ^ 1u, a.err);   // let the copy in flight land
                return;
            }
            for (int j = threadIdx.x; j < wi.count; j += blockDim.x) {
                const long long i = static_cast<long long>(wi.start) + j;
                T tau[3];
                int lb[3] = {0, 0, 0};
                node_setup<T, D>(a.xs, i, a.g, org, tau, lb, m);
                T w0[A], w1[A], w2[A];
                tap_weights<T, W>(tau[0], a.w, w0);
                if (D > 1) tap_weights<T, W>(tau[1], a.w, w1);
                if (D > 2) tap_weights<T, W>(tau[2], a.w, w2);
                const long long dst = a.perm[i];
                for (int bb = 0; bb < nb; ++bb) {
                    const CT v = contract<T, D, W>(box + bb * slot, a.g, lb, w0, w1, w2, a.comp != 0, nw);
                    a.fout[static_cast<long long>(b0 + bb) * a.N + dst] = v;
                }
            }
            __syncthreads();
        }
    }
}

template <typename T>
__device__ __forceinline__ void atomic_add_c(C2<T>* p, C2<T> v);
template <>
__device__ __forceinline__ void atomic_add_c<float>(float2* p, float2 v) {
    atomicAdd(p, v);
}
template <>
__device__ __forceinline__ void atomic_add_c<double>(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(kTapThreads) spread_kernel(const TapArgs<T> a) {
    using CT = C2<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    CT* box = aligned_box_base<T>(smem);
    T* boxs = reinterpret_cast<T*>(box);
    int box_cells = 1;
#pragma unroll
    for (int t = 0; t < D; ++t) box_cells *= a.g.box[t];
    const int slot = box_slot_cells<T>(box_cells);
    const bool periodic = a.w.method == NFFTBL_CLASSIC;
    constexpr int A = TapN<W>::A;
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        tile_origin<D>(a.g, wi.tile, periodic, org);
        for (int b0 = 0; b0 < a.batch; b0 += a.batch_smem) {
            const int nb = min(a.batch_smem, a.batch - b0);
            for (int idx = threadIdx.x; idx < nb * slot; idx += blockDim.x) box[idx] = cmake<T>(T(0), T(0));
            __syncthreads();
            for (int j = threadIdx.x; j < wi.count; j += blockDim.x) {
                const long long i = static_cast<long long>(wi.start) + j;
                T tau[3];
                int lb[3] = {0, 0, 0};
                node_setup<T, D>(a.xs, i, a.g, org, tau, lb, m);
                T w0[A], w1[A], w2[A];
                tap_weights<T, W>(tau[0], a.w, w0);
                if (D > 1) tap_weights<T, W>(tau[1], a.w, w1);
                if (D > 2) tap_weights<T, W>(tau[2], a.w, w2);
                const long long src = a.perm[i];
                for (int bb = 0; bb < nb; ++bb) {
                    const CT gv = a.fin[static_cast<long long>(b0 + bb) * a.N + src];
                    T* bx = boxs + 2LL * bb * slot;
                    if (D == 1) {
#pragma unroll
                        for (int q = 0; q < nw; ++q) {
                            const int c = lb[0] + q;
                            atomicAdd(bx + 2 * c, gv.x * w0[q]);
                            atomicAdd(bx + 2 * c + 1, gv.y * w0[q]);
                        }
                    } else if (D == 2) {
                        const int pitch = a.g.box[1];
                        for (int q0 = 0; q0 < nw; ++q0) {
                            const T gr = gv.x * w0[q0], gi = gv.y * w0[q0];
                            const int rowc = (lb[0] + q0) * pitch + lb[1];
#pragma unroll
                            for (int q1 = 0; q1 < nw; ++q1) {
                                atomicAdd(bx + 2 * (rowc + q1), gr * w1[q1]);
                                atomicAdd(bx + 2 * (rowc + q1) + 1, gi * w1[q1]);
                            }
                        }
                    } else {
                        const int p1 = a.g.box[2];
                        const int p0 = a.g.box[1] * p1;
                        for (int q0 = 0; q0 < nw; ++q0) {
                            for (int q1 = 0; q1 < nw; ++q1) {
                                const T wab = w0[q0] * w1[q1];
                                const T gr = gv.x * wab, gi = gv.y * wab;
                                const int rowc = (lb[0] + q0) * p0 + (lb[1] + q1) * p1 + lb[2];
#pragma unroll
                                for (int q2 = 0; q2 < nw; ++q2) {
                                    atomicAdd(bx + 2 * (rowc + q2), gr * w2[q2]);
                                    atomicAdd(bx + 2 * (rowc + q2) + 1, gi * w2[q2]);
                                }
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // flush the box into the grid: nonzero cells only; cells outside
            // I_L are dropped (Shannon, zero extension) or wrapped (classical)
            for (int idx = threadIdx.x; idx < nb * box_cells; idx += blockDim.x) {
                const int bb = idx / box_cells;
                const int cell = idx - bb * box_cells;
                const CT v = box[bb * slot + cell];
                if (v.x == T(0) && v.y == T(0)) continue;
                int r = cell;
                int loc[3] = {0, 0, 0};
#pragma unroll
                for (int t = D - 1; t >= 0; --t) {
                    loc[t] = r % a.g.box[t];
                    r /= a.g.box[t];
                }
                long long gi = 0;
                bool inside = true;
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    int c = org[t] + loc[t];
                    if (periodic) {
                        c %= a.g.L[t];
                        if (c < 0) c += a.g.L[t];
                    } else if (c < 0 || c >= a.g.L[t]) {
                        inside = false;
                    }
                    gi = gi * a.g.L[t] + c;
                }
                if (inside) atomic_add_c<T>(a.grid + (b0 + bb) * a.grid_stride + gi, v);
            }
            __syncthreads();
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
                mbar_wait_bounded(&bar, phase ^ 1u, a.err);
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
                    // partial derivatives: replace one dimension's weights by their derivative
#pragma unroll
                    for (int t = 0; t < D; ++t) {
                        CT dv;
                        if (D == 1) {
                            dv = contract<T, 1, W>(bx, a.g, lb, dw[0], dw[0], dw[0], false, nw);
                        } else if (D == 2) {
                            dv = (t == 0) ? contract<T, 2, W>(bx, a.g, lb, dw[0], w[1], w[1], false, nw)
                                          : contract<T, 2, W>(bx, a.g, lb, w[0], dw[1], dw[1], false, nw);
                        } else {
                            dv = (t == 0)   ? contract<T, 3, W>(bx, a.g, lb, dw[0], w[1], w[2], false, nw)
                                 : (t == 1) ? contract<T, 3, W>(bx, a.g, lb, w[0], dw[1], w[2], false, nw)
                                            : contract<T, 3, W>(bx, a.g, lb, w[0], w[1], dw[2], false, nw);
                        }
                        gsum[t] += gf.x * dv.x + gf.y * dv.y;
                    }
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

template <typename T, int D, int W>
nfftbl_status launch_tap_kernel(nfftbl_plan_s* p, const TapArgs<T>& args, int kind, size_t smem) {
    void* fn = nullptr;
    if (kind == TAP_INTERP) fn = reinterpret_cast<void*>(interp_kernel<T, D, W>);
    if (kind == TAP_SPREAD) fn = reinterpret_cast<void*>(spread_kernel<T, D, W>);
    if (kind == TAP_GRAD) fn = reinterpret_cast<void*>(node_grad_kernel<T, D, W>);
    nfftbl_status st = check_cuda(p, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          static_cast<int>(smem)),
                                  "tap smem attribute");
    if (st != NFFTBL_OK) return st;
    int occ = 0;
    st = check_cuda(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTapThreads, smem), "occupancy");
    if (st != NFFTBL_OK) return st;
    if (occ < 1) return fail(p, NFFTBL_EUNSUPPORTED, "tap kernel does not fit on an SM");
    const long long want = static_cast<long long>(occ) * p->num_sms;
    const unsigned grid = static_cast<unsigned>(std::max<long long>(1, std::min<long long>(want, args.n_work)));
    if (args.n_work == 0) return NFFTBL_OK;
    timing_begin(p, kind == TAP_INTERP ? NFFTBL_K_INTERP : kind == TAP_SPREAD ? NFFTBL_K_SPREAD : NFFTBL_K_GRAD);
    if (kind == TAP_INTERP)
        interp_kernel<T, D, W><<<grid, kTapThreads, smem, p->stream>>>(p->tmap, args);
    else if (kind == TAP_SPREAD)
        spread_kernel<T, D, W><<<grid, kTapThreads, smem, p->stream>>>(args);
    else
        node_grad_kernel<T, D, W><<<grid, kTapThreads, smem, p->stream>>>(p->tmap, args);
    timing_end(p);
    p->launches++;
    return check_cuda(p, cudaGetLastError(), "tap kernel launch");
}

}  // namespace nfftbl
