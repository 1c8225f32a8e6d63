// Steps 1-2 of Algorithm 4.2 (and of Algorithm 2.1) and their adjoint.
//
// Forward, one pass per dimension t = d-1, ..., 0 (pruned: only lines whose
// input is nonzero are transformed, i.e. dimensions not yet transformed keep
// their M_t extent):
//   load   a[q] = fhat[k] * (-1)^k d_t(k) at q = k mod L_t for k in I_{M_t}, 0 elsewhere
//          (the precorrection theta_hat = fhat / psi_hat of step 1 with the
//          1/|I_L| of step 2, Eq. 4.9, and the centring shift l = s - L/2);
//   FFT    vartheta[s] = sum_q a[q] e^{+2 pi i q s / L_t}   (inverse-sign DFT);
//   store  all L_t outputs, centred index s = l + L_t/2.
// Adjoint, t = 0, ..., d-1: load L_t values, forward-sign DFT, store only
// k in I_{M_t} multiplied by (-1)^k d_t(k)  (F^H and D_psihat of Eq. 4.11).
//
// Each CTA transforms W lines of one pass in shared memory with a Stockham
// autosort FFT: for L = 2^k a kernel instantiated per length with radix-8
// stages (fft_pow2_kernel), otherwise run-time mixed radix (4, 2, 3, 5)
// (fft_pass_kernel); twiddles come from an FP64 table rounded to the plan's
// precision.
#include <algorithm>

#include "plan_internal.h"

namespace nfftbl {
namespace {

constexpr int kFftThreads = 256;

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
    return cmake<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {   // a * conj(b)
    return cmake<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(const C2<T>* __restrict__ in, C2<T>* __restrict__ out,
                                                               long long outer, int inner, int M, int L, int W,
                                                               const T* __restrict__ fac,
                                                               const C2<T>* __restrict__ tw) {
    using CT = C2<T>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int pitch = L + 1;
    CT* bufA = reinterpret_cast<CT*>(sm_raw);
    CT* bufB = bufA + W * pitch;
    CT* twd = bufB + W * pitch;
    const int tid = threadIdx.x;
    const int bd = blockDim.x;
    constexpr int kBatch = 8;   // global loads issued together before their shared-memory stores
    for (int j0 = 0; j0 < L; j0 += kBatch * bd) {
        CT v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int j = j0 + u * bd + tid;
            if (j < L) v[u] = tw[j];
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int j = j0 + u * bd + tid;
            if (j < L) twd[j] = v[u];
        }
    }

    const int n_in = ADJ ? L : M;
    const int n_out = ADJ ? M : L;
    long long o0 = 0;
    int i0 = 0, nl = W;
    if (inner == 1) {
        o0 = static_cast<long long>(blockIdx.x) * W;
        nl = static_cast<int>((outer - o0 < W) ? (outer - o0) : W);
    } else {
        const int per = inner / W;
        o0 = blockIdx.x / per;
        i0 = (blockIdx.x % per) * W;
    }

    // ---- load
    if (!ADJ) {
        const int zlo = M / 2, zhi = L - M / 2;   // zero-padded positions [zlo, zhi)
        for (int idx = tid; idx < W * (zhi - zlo); idx += blockDim.x) {
            const int w = idx / (zhi - zlo);
            bufA[w * pitch + zlo + idx % (zhi - zlo)] = cmake<T>(T(0), T(0));
        }
    }
    for (int idx0 = 0; idx0 < W * n_in; idx0 += kBatch * bd) {
        CT v[kBatch];
        T f[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = idx0 + u * bd + tid;
            v[u] = cmake<T>(T(0), T(0));
            f[u] = T(1);
            if (idx < W * n_in) {
                int w, p;
                long long g;
                if (inner == 1) {
                    w = idx / n_in;
                    p = idx - w * n_in;
                    g = (o0 + w) * n_in + p;
                } else {
                    p = idx / W;
                    w = idx - p * W;
                    g = (o0 * n_in + p) * static_cast<long long>(inner) + i0 + w;
                }
                if (w < nl) v[u] = in[g];
                if (!ADJ) f[u] = fac[p];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = idx0 + u * bd + tid;
            if (idx < W * n_in) {
                int w, p;
                if (inner == 1) {
                    w = idx / n_in;
                    p = idx - w * n_in;
                } else {
                    p = idx / W;
                    w = idx - p * W;
                }
                int q = p;
                CT val = v[u];
                if (!ADJ) {
                    val.x *= f[u];
                    val.y *= f[u];
                    q = (p < M / 2) ? (L - M / 2 + p) : (p - M / 2);
                }
                bufA[w * pitch + q] = val;
            }
        }
    }
    __syncthreads();

    // ---- Stockham stages: radix 4 while possible, then 2, 3 and 5
    // (L = 2^a 3^b 5^c).  Stage with radix r and span s (the product of the
    // earlier radices): butterfly i (k = i mod s) reads i + j L/r, multiplies
    // input j by w^(j k L/(r s)) and writes (i - k) r + k + j s; every
    // twiddle exponent stays below L.
    CT* src = bufA;
    CT* dst = bufB;
    int span = 1, rem = L;
    while (span < L) {
        const int r = (rem % 4 == 0) ? 4 : (rem % 2 == 0) ? 2 : (rem % 3 == 0) ? 3 : 5;
        const int nb = L / r;
        const int tstep = L / (r * span);
        for (int b = tid; b < W * nb; b += blockDim.x) {
            const int w = b / nb;
            const int i = b - w * nb;
            const int k = (span & (span - 1)) ? i % span : (i & (span - 1));
            const CT* s = src + w * pitch;
            CT* dd = dst + w * pitch;
            const int obase = (i - k) * r + k;
            CT c[5];
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (j < r) c[j] = s[i + j * nb];
            if (span > 1) {
                const int e = k * tstep;
#pragma unroll
                for (int j = 1; j < 5; ++j)
                    if (j < r) c[j] = ADJ ? cmulc<T>(c[j], twd[j * e]) : cmul<T>(c[j], twd[j * e]);
            }
            // multiplication by +i (forward: inverse-DFT sign) or -i (adjoint)
            auto rot = [](CT v) { return ADJ ? cmake<T>(v.y, -v.x) : cmake<T>(-v.y, v.x); };
            if (r == 4) {
                const CT a0 = cmake<T>(c[0].x + c[2].x, c[0].y + c[2].y);
                const CT a1 = cmake<T>(c[0].x - c[2].x, c[0].y - c[2].y);
                const CT a2 = cmake<T>(c[1].x + c[3].x, c[1].y + c[3].y);
                const CT a3 = rot(cmake<T>(c[1].x - c[3].x, c[1].y - c[3].y));
                dd[obase] = cmake<T>(a0.x + a2.x, a0.y + a2.y);
                dd[obase + span] = cmake<T>(a1.x + a3.x, a1.y + a3.y);
                dd[obase + 2 * span] = cmake<T>(a0.x - a2.x, a0.y - a2.y);
                dd[obase + 3 * span] = cmake<T>(a1.x - a3.x, a1.y - a3.y);
            } else if (r == 2) {
                dd[obase] = cmake<T>(c[0].x + c[1].x, c[0].y + c[1].y);
                dd[obase + span] = cmake<T>(c[0].x - c[1].x, c[0].y - c[1].y);
            } else if (r == 3) {
                // y1,2 = c0 - (c1 + c2)/2 +- (rot) (sqrt(3)/2)(c1 - c2)
                const T h = static_cast<T>(0.86602540378443864676);
                const CT t1 = cmake<T>(c[1].x + c[2].x, c[1].y + c[2].y);
                const CT t2 = cmake<T>(c[0].x - T(0.5) * t1.x, c[0].y - T(0.5) * t1.y);
                const CT t3 = rot(cmake<T>(h * (c[1].x - c[2].x), h * (c[1].y - c[2].y)));
                dd[obase] = cmake<T>(c[0].x + t1.x, c[0].y + t1.y);
                dd[obase + span] = cmake<T>(t2.x + t3.x, t2.y + t3.y);
                dd[obase + 2 * span] = cmake<T>(t2.x - t3.x, t2.y - t3.y);
            } else {
                // radix 5 with cos/sin of 2 pi/5 and 4 pi/5
                const T c1 = static_cast<T>(0.30901699437494742410), c2 = static_cast<T>(-0.80901699437494742410);
                const T s1 = static_cast<T>(0.95105651629515357212), s2 = static_cast<T>(0.58778525229247312917);
                const CT t1 = cmake<T>(c[1].x + c[4].x, c[1].y + c[4].y);
                const CT t2 = cmake<T>(c[2].x + c[3].x, c[2].y + c[3].y);
                const CT t3 = cmake<T>(c[1].x - c[4].x, c[1].y - c[4].y);
                const CT t4 = cmake<T>(c[2].x - c[3].x, c[2].y - c[3].y);
                const CT a1 = cmake<T>(c[0].x + c1 * t1.x + c2 * t2.x, c[0].y + c1 * t1.y + c2 * t2.y);
                const CT a2 = cmake<T>(c[0].x + c2 * t1.x + c1 * t2.x, c[0].y + c2 * t1.y + c1 * t2.y);
                const CT b1 = rot(cmake<T>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
                const CT b2 = rot(cmake<T>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
                dd[obase] = cmake<T>(c[0].x + t1.x + t2.x, c[0].y + t1.y + t2.y);
                dd[obase + span] = cmake<T>(a1.x + b1.x, a1.y + b1.y);
                dd[obase + 2 * span] = cmake<T>(a2.x + b2.x, a2.y + b2.y);
                dd[obase + 3 * span] = cmake<T>(a2.x - b2.x, a2.y - b2.y);
                dd[obase + 4 * span] = cmake<T>(a1.x - b1.x, a1.y - b1.y);
            }
        }
        __syncthreads();
        CT* tmp = src;
        src = dst;
        dst = tmp;
        span *= r;
        rem /= r;
    }

    // ---- store
    for (int idx = tid; idx < W * n_out; idx += blockDim.x) {
        int w, p;
        long long g;
        if (inner == 1) {
            w = idx / n_out;
            p = idx - w * n_out;
            g = (o0 + w) * n_out + p;
        } else {
            p = idx / W;
            w = idx - p * W;
            g = (o0 * n_out + p) * static_cast<long long>(inner) + i0 + w;
        }
        if (w >= nl) continue;
        CT v;
        if (!ADJ) {
            v = src[w * pitch + p];
        } else {
            const int q = (p < M / 2) ? (L - M / 2 + p) : (p - M / 2);
            v = src[w * pitch + q];
            const T f = fac[p];
            v.x *= f;
            v.y *= f;
        }
        out[g] = v;
    }
}

constexpr int ilog2_c(int v) { return v <= 1 ? 0 : 1 + ilog2_c(v >> 1); }

// ---------------------------------------------------------------------------
// Power-of-two lengths: the same pass with L a compile-time constant, radix-8
// Stockham stages (then one radix-4 or radix-2 stage), shifts instead of
// divisions.  A pass is bound by the latency of each thread's instruction
// chain (few lines per pass, few warps per SM), so fewer stages and
// instructions per element shorten it directly.

// 8-point DFT of c (forward pass: e^{+2 pi i jq/8}, adjoint: e^{-2 pi i jq/8})
// as two 4-point DFTs of the sums c_j + c_{j+4} (even outputs) and of the
// differences times e^{+-2 pi i j/8} (odd outputs).
template <typename T, bool ADJ>
__device__ __forceinline__ void dft8(C2<T> (&c)[8]) {
    using CT = C2<T>;
    const T h = static_cast<T>(0.70710678118654752440);
    auto rot = [](CT v) { return ADJ ? cmake<T>(v.y, -v.x) : cmake<T>(-v.y, v.x); };
    auto add = [](CT a, CT b) { return cmake<T>(a.x + b.x, a.y + b.y); };
    auto sub = [](CT a, CT b) { return cmake<T>(a.x - b.x, a.y - b.y); };
    CT a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        a[j] = add(c[j], c[j + 4]);
        b[j] = sub(c[j], c[j + 4]);
    }
    // b1 *= (1 +- i)/sqrt 2, b2 *= +-i, b3 *= (-1 +- i)/sqrt 2
    b[1] = ADJ ? cmake<T>(h * (b[1].x + b[1].y), h * (b[1].y - b[1].x))
               : cmake<T>(h * (b[1].x - b[1].y), h * (b[1].x + b[1].y));
    b[2] = rot(b[2]);
    b[3] = ADJ ? cmake<T>(h * (b[3].y - b[3].x), -h * (b[3].x + b[3].y))
               : cmake<T>(-h * (b[3].x + b[3].y), h * (b[3].x - b[3].y));
    auto dft4 = [&](const CT (&x)[4], CT& y0, CT& y1, CT& y2, CT& y3) {
        const CT s02 = add(x[0], x[2]), d02 = sub(x[0], x[2]);
        const CT s13 = add(x[1], x[3]), d13 = rot(sub(x[1], x[3]));
        y0 = add(s02, s13);
        y1 = add(d02, d13);
        y2 = sub(s02, s13);
        y3 = sub(d02, d13);
    };
    dft4(a, c[0], c[2], c[4], c[6]);
    dft4(b, c[1], c[3], c[5], c[7]);
}

// Position of element x of a line in shared memory: the low four bits are
// XOR-ed with bits 3..6, a permutation inside each block of 16 elements.
// With it the reads and writes of every Stockham stage below, and the
// consecutive accesses of the load and store loops, touch 16 different
// 8-byte bank pairs per half warp (checked for L = 64 .. 4096); without it
// the first stage's writes (stride R) are 8-way bank conflicts.
__device__ __forceinline__ int swz(int x) { return x ^ ((x >> 3) & 15); }

// One Stockham stage of radix R and span S over W lines of length L: butterfly
// i (k = i mod S) reads i + j L/R, multiplies input j by w^(j k L/(R S)) and
// writes output q to (i - k) R + k + q S.
template <typename T, bool ADJ, int L, int R, int S>
__device__ __forceinline__ void pow2_stage(const C2<T>* __restrict__ src, C2<T>* __restrict__ dst,
                                           const C2<T>* __restrict__ twd, int W, int pitch) {
    using CT = C2<T>;
    constexpr int NB = L / R;
    constexpr int LG_NB = ilog2_c(NB);
    constexpr int TSTEP = L / (R * S);
    for (int b = threadIdx.x; b < W * NB; b += blockDim.x) {
        const int w = b >> LG_NB;
        const int i = b & (NB - 1);
        const int k = i & (S - 1);
        const CT* s = src + w * pitch;
        CT* dl = dst + w * pitch;
        const int d0 = (i - k) * R + k;
        CT c[8];
#pragma unroll
        for (int j = 0; j < R; ++j) c[j] = s[swz(i + j * NB)];
        if (S > 1) {
            const int e = k * TSTEP;
#pragma unroll
            for (int j = 1; j < R; ++j) c[j] = ADJ ? cmulc<T>(c[j], twd[j * e]) : cmul<T>(c[j], twd[j * e]);
        }
        auto rot = [](CT v) { return ADJ ? cmake<T>(v.y, -v.x) : cmake<T>(-v.y, v.x); };
        if constexpr (R == 8) {
            dft8<T, ADJ>(c);
        } else if constexpr (R == 4) {
            const CT a0 = cmake<T>(c[0].x + c[2].x, c[0].y + c[2].y);
            const CT a1 = cmake<T>(c[0].x - c[2].x, c[0].y - c[2].y);
            const CT a2 = cmake<T>(c[1].x + c[3].x, c[1].y + c[3].y);
            const CT a3 = rot(cmake<T>(c[1].x - c[3].x, c[1].y - c[3].y));
            c[0] = cmake<T>(a0.x + a2.x, a0.y + a2.y);
            c[1] = cmake<T>(a1.x + a3.x, a1.y + a3.y);
            c[2] = cmake<T>(a0.x - a2.x, a0.y - a2.y);
            c[3] = cmake<T>(a1.x - a3.x, a1.y - a3.y);
        } else {
            const CT a0 = c[0];
            c[0] = cmake<T>(a0.x + c[1].x, a0.y + c[1].y);
            c[1] = cmake<T>(a0.x - c[1].x, a0.y - c[1].y);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) dl[swz(d0 + q * S)] = c[q];
    }
}

// Stages of span S, S R, ... up to L (radix 8 while 8 divides L / S).
template <typename T, bool ADJ, int L, int S>
__device__ __forceinline__ void pow2_stages(C2<T>*& src, C2<T>*& dst, const C2<T>* twd, int W, int pitch) {
    if constexpr (S < L) {
        constexpr int REM = L / S;
        constexpr int R = (REM % 8 == 0) ? 8 : (REM % 4 == 0) ? 4 : 2;
        pow2_stage<T, ADJ, L, R, S>(src, dst, twd, W, pitch);
        __syncthreads();
        C2<T>* tmp = src;
        src = dst;
        dst = tmp;
        pow2_stages<T, ADJ, L, S * R>(src, dst, twd, W, pitch);
    }
}

// The pass of fft_pass_kernel for L = 2^LG; W (lines per CTA) = 2^lgW.
template <typename T, bool ADJ, int LG>
__global__ void __launch_bounds__(kFftThreads) fft_pow2_kernel(const C2<T>* __restrict__ in, C2<T>* __restrict__ out,
                                                               long long outer, int inner, int M, int lgW,
                                                               const T* __restrict__ fac,
                                                               const C2<T>* __restrict__ tw) {
    using CT = C2<T>;
    constexpr int L = 1 << LG;
    constexpr int pitch = L + 1;
    const int W = 1 << lgW;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    CT* bufA = reinterpret_cast<CT*>(sm_raw);
    CT* bufB = bufA + W * pitch;
    CT* twd = bufB + W * pitch;
    const int tid = threadIdx.x;
    const int bd = blockDim.x;
    for (int j = tid; j < L; j += bd) twd[j] = tw[j];

    const int n_in = ADJ ? L : M;
    const int n_out = ADJ ? M : L;
    long long o0 = 0;
    int i0 = 0, nl = W;
    if (inner == 1) {
        o0 = static_cast<long long>(blockIdx.x) << lgW;
        nl = static_cast<int>((outer - o0 < W) ? (outer - o0) : W);
    } else {
        const int per = inner >> lgW;
        o0 = blockIdx.x / per;
        i0 = (blockIdx.x - static_cast<int>(o0) * per) << lgW;
    }
    // element idx of this CTA's W x n lines -> (line w, position p)
    auto split = [&](int idx, int n, int& w, int& p) {
        if (inner == 1) {
            w = (W == 1) ? 0 : idx / n;
            p = idx - w * n;
        } else {
            p = idx >> lgW;
            w = idx & (W - 1);
        }
    };

    // ---- load (zero-padding, precorrection and centring as in fft_pass_kernel)
    if (!ADJ) {
        const int zlo = M / 2, zhi = L - M / 2;
        const int nz = zhi - zlo;
        for (int idx = tid; idx < W * nz; idx += bd) {
            const int w = (W == 1) ? 0 : idx / nz;
            bufA[w * pitch + swz(zlo + idx - w * nz)] = cmake<T>(T(0), T(0));
        }
    }
    constexpr int kBatch = 8;
    for (int idx0 = 0; idx0 < W * n_in; idx0 += kBatch * bd) {
        CT v[kBatch];
        T f[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = idx0 + u * bd + tid;
            v[u] = cmake<T>(T(0), T(0));
            f[u] = T(1);
            if (idx < W * n_in) {
                int w, p;
                split(idx, n_in, w, p);
                const long long g = (inner == 1) ? (o0 + w) * n_in + p
                                                 : (o0 * n_in + p) * static_cast<long long>(inner) + i0 + w;
                if (w < nl) v[u] = in[g];
                if (!ADJ) f[u] = fac[p];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = idx0 + u * bd + tid;
            if (idx < W * n_in) {
                int w, p;
                split(idx, n_in, w, p);
                int q = p;
                CT val = v[u];
                if (!ADJ) {
                    val.x *= f[u];
                    val.y *= f[u];
                    q = (p < M / 2) ? (L - M / 2 + p) : (p - M / 2);
                }
                bufA[w * pitch + swz(q)] = val;
            }
        }
    }
    __syncthreads();

    CT* src = bufA;
    CT* dst = bufB;
    pow2_stages<T, ADJ, L, 1>(src, dst, twd, W, pitch);

    // ---- store
    for (int idx = tid; idx < W * n_out; idx += bd) {
        int w, p;
        split(idx, n_out, w, p);
        if (w >= nl) continue;
        const long long g = (inner == 1) ? (o0 + w) * n_out + p
                                         : (o0 * n_out + p) * static_cast<long long>(inner) + i0 + w;
        CT v;
        if (!ADJ) {
            v = src[w * pitch + swz(p)];
        } else {
            const int q = (p < M / 2) ? (L - M / 2 + p) : (p - M / 2);
            v = src[w * pitch + swz(q)];
            const T f = fac[p];
            v.x *= f;
            v.y *= f;
        }
        out[g] = v;
    }
}

template <typename T>
size_t fft_smem(int L, int W) {
    return (2 * static_cast<size_t>(W) * (L + 1) + L) * sizeof(C2<T>);
}

// Lines per CTA: as many as fit in 64 KB of shared memory (up to 16, for
// wide coalesced segments on the strided passes) while the launch still has
// about four CTAs per SM; the lines of one CTA share one outer index.
template <typename T>
int choose_lines(int L, long long lines, long long inner, int num_sms) {
    int W = 16;
    while (W > 1 && (fft_smem<T>(L, W) > 64 * 1024 || lines / W < 4LL * num_sms)) W >>= 1;
    if (inner > 1) {   // the strided passes take inner / W CTAs per outer index: W must divide inner
        W = static_cast<int>(std::min<long long>(W, inner));
        while (W > 1 && inner % W != 0) W >>= 1;
    }
    return W;
}

// Threads per CTA: one radix-4 butterfly per thread per stage, 64 .. 256.
inline int fft_threads(int L, int W) {
    const int t = (W * L / 4 + 31) / 32 * 32;
    return std::max(64, std::min(kFftThreads, t));
}

template <typename T, bool ADJ>
nfftbl_status run_pass(nfftbl_plan_s* p, const void* in, void* out, int t) {
    long long outer = p->batch;
    for (int s = 0; s < t; ++s) outer *= p->M[s];
    long long inner = 1;
    for (int s = t + 1; s < p->d; ++s) inner *= p->L[s];
    const int L = p->L[t], M = p->M[t];
    const int W = choose_lines<T>(L, outer * inner, inner, p->num_sms);
    const size_t smem = fft_smem<T>(L, W);
    long long blocks = (inner == 1) ? (outer + W - 1) / W : outer * (inner / W);
    const C2<T>* src = static_cast<const C2<T>*>(in);
    C2<T>* dst = static_cast<C2<T>*>(out);
    const T* fac = static_cast<const T*>(p->facT[t].p);
    const C2<T>* tw = static_cast<const C2<T>*>(p->tw[t].p);
    if ((L & (L - 1)) == 0) {   // power of two (16 .. 4096): compile-time length, radix-8 stages
        void (*kern)(const C2<T>*, C2<T>*, long long, int, int, int, const T*, const C2<T>*) = nullptr;
        switch (ilog2_c(L)) {
            case 4: kern = fft_pow2_kernel<T, ADJ, 4>; break;
            case 5: kern = fft_pow2_kernel<T, ADJ, 5>; break;
            case 6: kern = fft_pow2_kernel<T, ADJ, 6>; break;
            case 7: kern = fft_pow2_kernel<T, ADJ, 7>; break;
            case 8: kern = fft_pow2_kernel<T, ADJ, 8>; break;
            case 9: kern = fft_pow2_kernel<T, ADJ, 9>; break;
            case 10: kern = fft_pow2_kernel<T, ADJ, 10>; break;
            case 11: kern = fft_pow2_kernel<T, ADJ, 11>; break;
            case 12: kern = fft_pow2_kernel<T, ADJ, 12>; break;
            default: return fail(p, NFFTBL_EINTERNAL, "power-of-two FFT length out of range");
        }
        nfftbl_status st = check_cuda(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              static_cast<int>(smem)),
                                      "fft smem attribute");
        if (st != NFFTBL_OK) return st;
        const int threads = std::max(64, std::min(kFftThreads, (W * L / 8 + 31) / 32 * 32));
        timing_begin(p, NFFTBL_K_FFT);
        kern<<<static_cast<unsigned>(blocks), threads, smem, p->stream>>>(src, dst, outer, static_cast<int>(inner), M,
                                                                          ilog2_c(W), fac, tw);
        timing_end(p);
        p->launches++;
        return check_cuda(p, cudaGetLastError(), "fft pass launch");
    }
    const int threads = fft_threads(L, W);
    auto kern = fft_pass_kernel<T, ADJ>;
    nfftbl_status st = check_cuda(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          static_cast<int>(smem)),
                                  "fft smem attribute");
    if (st != NFFTBL_OK) return st;
    timing_begin(p, NFFTBL_K_FFT);
    kern<<<static_cast<unsigned>(blocks), threads, smem, p->stream>>>(src, dst, outer, static_cast<int>(inner), M, L,
                                                                      W, fac, tw);
    timing_end(p);
    p->launches++;
    return check_cuda(p, cudaGetLastError(), "fft pass launch");
}

template <typename T>
nfftbl_status forward_impl(nfftbl_plan_s* p, const void* fhat) {
    const int d = p->d;
    const void* src = fhat;
    for (int t = d - 1; t >= 0; --t) {
        void* dst = (t == 0) ? p->grid.p : ((t == d - 1) ? p->tmpA.p : p->tmpB.p);
        nfftbl_status st = run_pass<T, false>(p, src, dst, t);
        if (st != NFFTBL_OK) return st;
        src = dst;
    }
    return NFFTBL_OK;
}

template <typename T>
nfftbl_status adjoint_impl(nfftbl_plan_s* p, void* fhat) {
    const int d = p->d;
    const void* src = p->grid.p;
    for (int t = 0; t < d; ++t) {
        void* dst = (t == d - 1) ? fhat : ((t == 0) ? p->tmpB.p : p->tmpA.p);
        if (d == 2 && t == 0) dst = p->tmpA.p;
        nfftbl_status st = run_pass<T, true>(p, src, dst, t);
        if (st != NFFTBL_OK) return st;
        src = dst;
    }
    return NFFTBL_OK;
}

}  // namespace

// One forward pass along dimension t of an array whose dimensions before t
// keep their M extent and whose dimensions after t already have their L
// extent (outer / inner line counts), for callers that own every buffer.
cudaError_t launch_fft_forward_pass_f32(const void* in, void* out, long long outer, long long inner, int M, int L,
                                        const float* fac, const void* tw, cudaStream_t s) {
    int dev = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int W = choose_lines<float>(L, outer * inner, inner, num_sms);
    const int threads = fft_threads(L, W);
    const size_t smem = fft_smem<float>(L, W);
    auto kern = fft_pass_kernel<float, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const long long blocks = (inner == 1) ? (outer + W - 1) / W : outer * (inner / W);
    kern<<<static_cast<unsigned>(blocks), threads, smem, s>>>(
        static_cast<const float2*>(in), static_cast<float2*>(out), outer, static_cast<int>(inner), M, L, W, fac,
        static_cast<const float2*>(tw));
    return cudaGetLastError();
}

// Scratch layout: d = 2 uses tmpA (B M0 L1); d = 3 uses tmpA (B M0 M1 L2)
// and tmpB (B M0 L1 L2).
nfftbl_status fft_forward(nfftbl_plan_s* p, const void* fhat) {
    if (p->precision == NFFTBL_F64) return forward_impl<double>(p, fhat);
    return forward_impl<float>(p, fhat);
}

nfftbl_status fft_adjoint(nfftbl_plan_s* p, void* fhat) {
    if (p->precision == NFFTBL_F64) return adjoint_impl<double>(p, fhat);
    return adjoint_impl<float>(p, fhat);
}

}  // namespace nfftbl
