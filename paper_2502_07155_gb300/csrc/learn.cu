// Learned window: a small MLP phi_theta on u = |Lx|/m in [0, 1], tabulated
// into the short-sum kernels, trained on the approximation error of the
// transform itself.
//
//   phi_theta(u) = (1 - u^2) exp(g(u^2) - g(0)),
//   g(s) = W3 tanh(W2 tanh(W1 s + b1) + b2) + b3      (1 -> 64 -> 64 -> 1)
//
// keeps the window even, equal to 1 at 0 and 0 at the support edge (the class
// Phi_{m,L} of Section 3; monotonicity is not enforced).  The loss is
// E = ||f - y||^2 / ||y||^2 with f = Psi F D_psihat fhat computed with the
// table window (Eq. 4.11) and y the target values.  Its gradient with
// respect to the table has two parts:
//   (A) through the short-sum weights psi = sinc * Phi (this file:
//       table_grad_kernel, a transposed tap walk that scatters into the
//       Catmull-Rom stencil of each tap);
//   (B) through the precorrection D_psihat = diag(1/(|I_L| psi_hat)) and the
//       quadrature that forms psi_hat from the table (window.cu).
// The MLP's forward runs in FP32; its backward uses BF16 tensor-core
// matrix products (mma.sync m16n8k16) with FP32 accumulation.
#include <cuda_bf16.h>

#include <cmath>

#include "taps.cuh"

namespace nfftbl {
namespace {

constexpr int kHidden = 64;

// ---------------------------------------------------------------------------
// MLP forward and table

struct MlpParams {
    const float* W1;
    const float* b1;
    const float* W2;   // [out][in]
    const float* b2;
    const float* W3;
    const float* b3;
};

__host__ __device__ inline MlpParams mlp_view(const float* p) {
    MlpParams v;
    v.W1 = p;
    v.b1 = p + kHidden;
    v.W2 = p + 2 * kHidden;
    v.b2 = v.W2 + kHidden * kHidden;
    v.W3 = v.b2 + kHidden;
    v.b3 = v.W3 + kHidden;
    return v;
}

constexpr int kParamCount = 2 * kHidden + kHidden * kHidden + 2 * kHidden + 1;

// act layout: h1 [(n+1) x 64], h2 [(n+1) x 64], g [n+1]
__global__ void mlp_forward_kernel(const float* __restrict__ params, int n, float* __restrict__ act) {
    __shared__ float sW2[kHidden * kHidden];
    __shared__ float sW1[kHidden], sb1[kHidden], sb2[kHidden], sW3[kHidden];
    const MlpParams P = mlp_view(params);
    for (int j = threadIdx.x; j < kHidden * kHidden; j += blockDim.x) sW2[j] = P.W2[j];
    for (int j = threadIdx.x; j < kHidden; j += blockDim.x) {
        sW1[j] = P.W1[j];
        sb1[j] = P.b1[j];
        sb2[j] = P.b2[j];
        sW3[j] = P.W3[j];
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const float u = static_cast<float>(i) / n;
    const float s = u * u;
    float h1[kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) h1[j] = tanhf(fmaf(sW1[j], s, sb1[j]));
    float* o1 = act + static_cast<size_t>(i) * kHidden;
    float* o2 = act + static_cast<size_t>(n + 1) * kHidden + static_cast<size_t>(i) * kHidden;
#pragma unroll
    for (int j = 0; j < kHidden; ++j) o1[j] = h1[j];
    float g = P.b3[0];
    for (int o = 0; o < kHidden; ++o) {
        float z = sb2[o];
#pragma unroll
        for (int j = 0; j < kHidden; ++j) z = fmaf(sW2[o * kHidden + j], h1[j], z);
        const float h2 = tanhf(z);
        o2[o] = h2;
        g = fmaf(sW3[o], h2, g);
    }
    act[static_cast<size_t>(n + 1) * 2 * kHidden + i] = g;
}

__global__ void mlp_table_kernel(const float* __restrict__ act, int n, double* __restrict__ table) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const float* g = act + static_cast<size_t>(n + 1) * 2 * kHidden;
    const double u = static_cast<double>(i) / n;
    table[i] = (1.0 - u * u) * exp(static_cast<double>(g[i]) - static_cast<double>(g[0]));
}

// ---------------------------------------------------------------------------
// MLP backward

// gamma_i = dE/dv_i * v_i (d v_i / d g(u_i^2) = v_i); sum_gamma collects the
// total, which the u = 0 point also receives with a minus sign through g(0).
__global__ void gamma_kernel(const double* __restrict__ dEdv, const double* __restrict__ table, int n,
                             float* __restrict__ gamma, double* __restrict__ sum_gamma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double val = 0.0;
    if (i <= n) {
        val = dEdv[i] * table[i];
        gamma[i] = static_cast<float>(val);
    }
    for (int off = 16; off > 0; off >>= 1) val += __shfl_down_sync(0xffffffffu, val, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum_gamma, val);
}

// delta2[i][o] = gamma'_i W3[o] (1 - h2^2); grads of W3, b3, b2.
__global__ void backward_out_kernel(const float* __restrict__ params, const float* __restrict__ act,
                                    const float* __restrict__ gamma, const double* __restrict__ sum_gamma, int n,
                                    float* __restrict__ delta2, float* __restrict__ grad) {
    __shared__ float sdW3[kHidden], sdb2[kHidden];
    __shared__ float sdb3;
    for (int j = threadIdx.x; j < kHidden; j += blockDim.x) {
        sdW3[j] = 0.f;
        sdb2[j] = 0.f;
    }
    if (threadIdx.x == 0) sdb3 = 0.f;
    __syncthreads();
    const MlpParams P = mlp_view(params);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) {
        float gi = gamma[i];
        if (i == 0) gi -= static_cast<float>(*sum_gamma);
        const float* h2 = act + static_cast<size_t>(n + 1) * kHidden + static_cast<size_t>(i) * kHidden;
        float* d2 = delta2 + static_cast<size_t>(i) * kHidden;
        for (int o = 0; o < kHidden; ++o) {
            const float h = h2[o];
            d2[o] = gi * P.W3[o] * (1.f - h * h);
            atomicAdd(&sdW3[o], gi * h);
            atomicAdd(&sdb2[o], d2[o]);
        }
        atomicAdd(&sdb3, gi);
    }
    __syncthreads();
    float* gW3 = grad + 2 * kHidden + kHidden * kHidden + kHidden;
    float* gb2 = grad + 2 * kHidden + kHidden * kHidden;
    for (int j = threadIdx.x; j < kHidden; j += blockDim.x) {
        atomicAdd(&gW3[j], sdW3[j]);
        atomicAdd(&gb2[j], sdb2[j]);
    }
    if (threadIdx.x == 0) atomicAdd(&grad[kParamCount - 1], sdb3);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat16 a = __float2bfloat16_rn(lo);
    const __nv_bfloat16 b = __float2bfloat16_rn(hi);
    return static_cast<uint32_t>(*reinterpret_cast<const uint16_t*>(&a)) |
           (static_cast<uint32_t>(*reinterpret_cast<const uint16_t*>(&b)) << 16);
}

// D(16x8, f32) += A(16x16, bf16, row-major) B(16x8, bf16, column-major)
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// dW2[o][j] = sum_i delta2[i][o] h1[i][j]: one warp per 16 x 8 output tile
// (grid 1 x 32 warps), K = the n+1 table points, zero-padded to 16.
__global__ void dW2_kernel(const float* __restrict__ act, const float* __restrict__ delta2, int n,
                           float* __restrict__ grad) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tm = warp >> 3, tn = warp & 7;        // 4 x 8 tiles of 16 x 8
    const int gid = lane >> 2, tig = lane & 3;
    const int npts = n + 1;
    const float* h1 = act;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    auto A = [&](int row, int k) -> float {     // A[o][i] = delta2[i][o]
        return (k < npts) ? delta2[static_cast<size_t>(k) * kHidden + tm * 16 + row] : 0.f;
    };
    auto B = [&](int k, int col) -> float {     // B[i][j] = h1[i][j]
        return (k < npts) ? h1[static_cast<size_t>(k) * kHidden + tn * 8 + col] : 0.f;
    };
    for (int k0 = 0; k0 < npts; k0 += 16) {
        uint32_t a[4], b[2];
        a[0] = pack_bf16(A(gid, k0 + 2 * tig), A(gid, k0 + 2 * tig + 1));
        a[1] = pack_bf16(A(gid + 8, k0 + 2 * tig), A(gid + 8, k0 + 2 * tig + 1));
        a[2] = pack_bf16(A(gid, k0 + 2 * tig + 8), A(gid, k0 + 2 * tig + 9));
        a[3] = pack_bf16(A(gid + 8, k0 + 2 * tig + 8), A(gid + 8, k0 + 2 * tig + 9));
        b[0] = pack_bf16(B(k0 + 2 * tig, gid), B(k0 + 2 * tig + 1, gid));
        b[1] = pack_bf16(B(k0 + 2 * tig + 8, gid), B(k0 + 2 * tig + 9, gid));
        mma_bf16_16816(acc, a, b);
    }
    float* gW2 = grad + 2 * kHidden;
    const int r0 = tm * 16 + gid, c0 = tn * 8 + 2 * tig;
    gW2[r0 * kHidden + c0] += acc[0];
    gW2[r0 * kHidden + c0 + 1] += acc[1];
    gW2[(r0 + 8) * kHidden + c0] += acc[2];
    gW2[(r0 + 8) * kHidden + c0 + 1] += acc[3];
}

// delta1[i][j] = (sum_o delta2[i][o] W2[o][j]) (1 - h1[i][j]^2): block = 16
// points x 64 outputs (8 warps, one 16 x 8 tile each), K = 64.
__global__ void delta1_kernel(const float* __restrict__ params, const float* __restrict__ act,
                              const float* __restrict__ delta2, int n, float* __restrict__ delta1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int npts = n + 1;
    const int i0 = blockIdx.x * 16;
    const float* W2 = mlp_view(params).W2;
    auto A = [&](int row, int k) -> float {     // A[i][o] = delta2[i][o]
        const int i = i0 + row;
        return (i < npts) ? delta2[static_cast<size_t>(i) * kHidden + k] : 0.f;
    };
    auto B = [&](int k, int col) -> float {     // B[o][j] = W2[o][j]
        return W2[k * kHidden + warp * 8 + col];
    };
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < kHidden; k0 += 16) {
        uint32_t a[4], b[2];
        a[0] = pack_bf16(A(gid, k0 + 2 * tig), A(gid, k0 + 2 * tig + 1));
        a[1] = pack_bf16(A(gid + 8, k0 + 2 * tig), A(gid + 8, k0 + 2 * tig + 1));
        a[2] = pack_bf16(A(gid, k0 + 2 * tig + 8), A(gid, k0 + 2 * tig + 9));
        a[3] = pack_bf16(A(gid + 8, k0 + 2 * tig + 8), A(gid + 8, k0 + 2 * tig + 9));
        b[0] = pack_bf16(B(k0 + 2 * tig, gid), B(k0 + 2 * tig + 1, gid));
        b[1] = pack_bf16(B(k0 + 2 * tig + 8, gid), B(k0 + 2 * tig + 9, gid));
        mma_bf16_16816(acc, a, b);
    }
    const float* h1 = act;
    const int c0 = warp * 8 + 2 * tig;
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + gid + ((q >= 2) ? 8 : 0);
        const int j = c0 + (q & 1);
        if (i < npts) {
            const float h = h1[static_cast<size_t>(i) * kHidden + j];
            delta1[static_cast<size_t>(i) * kHidden + j] = acc[q] * (1.f - h * h);
        }
    }
}

// dW1[j] = sum_i delta1[i][j] s_i, db1[j] = sum_i delta1[i][j]: one block per j.
__global__ void first_layer_grad_kernel(const float* __restrict__ delta1, int n, float* __restrict__ grad) {
    const int j = blockIdx.x;
    double sw = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) {
        const double u = static_cast<double>(i) / n;
        const double dv = delta1[static_cast<size_t>(i) * kHidden + j];
        sw += dv * u * u;
        sb += dv;
    }
    __shared__ double rw[32], rb[32];
    for (int off = 16; off > 0; off >>= 1) {
        sw += __shfl_down_sync(0xffffffffu, sw, off);
        sb += __shfl_down_sync(0xffffffffu, sb, off);
    }
    if ((threadIdx.x & 31) == 0) {
        rw[threadIdx.x >> 5] = sw;
        rb[threadIdx.x >> 5] = sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tw = 0.0, tb = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
            tw += rw[w];
            tb += rb[w];
        }
        grad[j] += static_cast<float>(tw);
        grad[kHidden + j] += static_cast<float>(tb);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int count, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// ---------------------------------------------------------------------------
// Loss pieces

template <typename T>
__global__ void residual_kernel(C2<T>* __restrict__ f, const C2<T>* __restrict__ y, long long n,
                                double* __restrict__ loss) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    double num = 0.0, den = 0.0;
    if (i < n) {
        const C2<T> fy = y[i];
        C2<T> r = f[i];
        r.x -= fy.x;
        r.y -= fy.y;
        f[i] = r;
        num = static_cast<double>(r.x) * r.x + static_cast<double>(r.y) * r.y;
        den = static_cast<double>(fy.x) * fy.x + static_cast<double>(fy.y) * fy.y;
    }
    for (int off = 16; off > 0; off >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, off);
        den += __shfl_down_sync(0xffffffffu, den, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&loss[1], num);
        atomicAdd(&loss[2], den);
    }
}

__global__ void loss_finish_kernel(double* loss) { loss[0] = loss[1] / loss[2]; }

// P_t(q) = Re sum_{k : k_t = q} conj(hhat_k) fhat_k (all batch entries)
template <typename T>
__global__ void marginal_kernel(const C2<T>* __restrict__ hhat, const C2<T>* __restrict__ fhat, long long total,
                                int d, int M0, int M1, int M2, double* __restrict__ P0, double* __restrict__ P1,
                                double* __restrict__ P2) {
    const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (idx >= total) return;
    const C2<T> h = hhat[idx], f = fhat[idx];
    const double v = static_cast<double>(h.x) * f.x + static_cast<double>(h.y) * f.y;
    long long r = idx;
    int k[3] = {0, 0, 0};
    const int Ms[3] = {M0, M1, M2};
    for (int t = d - 1; t >= 0; --t) {
        k[t] = static_cast<int>(r % Ms[t]);
        r /= Ms[t];
    }
    atomicAdd(&P0[k[0]], v);
    if (d > 1) atomicAdd(&P1[k[1]], v);
    if (d > 2) atomicAdd(&P2[k[2]], v);
}

// dE/dpsi_hat_t(q) = -(2 L_t / ||y||^2) P_t(q) d_t(q),  d_t = 1/(L_t psi_hat_t)
__global__ void dEdpsihat_kernel(const double* __restrict__ P, const double* __restrict__ fac, int M, int L,
                                 const double* __restrict__ loss, double* __restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M) return;
    out[q] = -(2.0 * L / loss[2]) * P[q] * fac[q];
}

// ---------------------------------------------------------------------------
// Part (A): gradient through the tap weights.
//   dE/dPhi_t(delta_{t,a}) = (2/||y||^2) Re(conj(r_j) R_{t,a}) sinc_{t,a}
// where R_{t,a} is the box contracted with the other dimensions' weights;
// each such value is scattered into the four table entries of the tap's
// Catmull-Rom stencil (ghost entries folded back as in the table evaluation).

template <int D, int W>
__global__ void __launch_bounds__(kTapThreads) table_grad_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                 const TapArgs<float> a,
                                                                 const double* __restrict__ loss,
                                                                 double* __restrict__ tab_grad_out) {
    using CT = float2;
    constexpr int A = TapN<W>::A;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    const int n = a.w.table_n;
    double* s_grad = reinterpret_cast<double*>(smem);                       // n + 1 doubles
    CT* box = aligned_box_base<float>(smem + ((n + 1) * sizeof(double) + 127) / 128 * 128);
    int box_cells = 1;
#pragma unroll
    for (int t = 0; t < D; ++t) box_cells *= a.g.box[t];
    const int slot = box_slot_cells<float>(box_cells);
    for (int i = threadIdx.x; i <= n; i += blockDim.x) s_grad[i] = 0.0;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const int nw = W ? W : 2 * a.w.m;
    const int m = nw / 2;
    const float pi = static_cast<float>(kPiD);
    for (int item = blockIdx.x; item < a.n_work; item += gridDim.x) {
        const WorkItem wi = a.work[item];
        int org[3] = {0, 0, 0};
        tile_origin<D>(a.g, wi.tile, false, org);
        for (int b0 = 0; b0 < a.batch; b0 += a.batch_smem) {
            const int nb = min(a.batch_smem, a.batch - b0);
            if (!stage_box<float, D>(&tmap, a, box, box_cells, slot, org, false, b0, nb, &bar, phase)) {
                mbar_wait_bounded(&bar, phase ^ 1u, a.err);
                return;
            }
            for (int j = threadIdx.x; j < wi.count; j += blockDim.x) {
                const long long i = static_cast<long long>(wi.start) + j;
                float tau[3];
                int lb[3] = {0, 0, 0};
                node_setup<float, D>(a.xs, i, a.g, org, tau, lb, m);
                float w[2][A], sc[2][A];
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    const float s = sinpif(tau[t]);
#pragma unroll
                    for (int q = 0; q < nw; ++q) {
                        const int nn = m - 1 - q;
                        const float delta = tau[t] + static_cast<float>(nn);
                        const float num = (nn & 1) ? -s : s;
                        sc[t][q] = (delta == 0.f) ? 1.f : num / (pi * delta);
                        w[t][q] = sc[t][q] * win_phi(delta, a.w);
                    }
                }
                const long long dst = a.perm[i];
                float cr[2][A];
#pragma unroll
                for (int t = 0; t < D; ++t)
#pragma unroll
                    for (int q = 0; q < nw; ++q) cr[t][q] = 0.f;
                for (int bb = 0; bb < nb; ++bb) {
                    const CT r = a.fin[static_cast<long long>(b0 + bb) * a.N + dst];
                    const CT* bx = box + bb * slot;
                    if (D == 1) {
#pragma unroll
                        for (int q = 0; q < nw; ++q) {
                            const CT v = bx[lb[0] + q];
                            cr[0][q] += r.x * v.x + r.y * v.y;
                        }
                    } else {
                        const int pitch = a.g.box[1];
                        for (int q0 = 0; q0 < nw; ++q0) {
                            const CT* row = bx + (lb[0] + q0) * pitch + lb[1];
                            float rr = 0.f, ri = 0.f;
#pragma unroll
                            for (int q1 = 0; q1 < nw; ++q1) {
                                const CT v = row[q1];
                                rr += v.x * w[1][q1];
                                ri += v.y * w[1][q1];
                                // R_1[q1] += v w0[q0]
                                cr[1][q1] += (r.x * v.x + r.y * v.y) * w[0][q0];
                            }
                            cr[0][q0] += r.x * rr + r.y * ri;
                        }
                    }
                }
                for (int t = 0; t < D; ++t) {
                    for (int q = 0; q < nw; ++q) {
                        const float delta = tau[t] + static_cast<float>(m - 1 - q);
                        const float u = fabsf(delta) / m;
                        if (u < 1.f) scatter_catmull(s_grad, n, u, static_cast<double>(cr[t][q]) * sc[t][q]);
                    }
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    const double scale = 2.0 / loss[2];
    for (int i = threadIdx.x; i <= n; i += blockDim.x)
        if (s_grad[i] != 0.0) atomicAdd(&tab_grad_out[i], s_grad[i] * scale);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers

template <int D, int W>
nfftbl_status launch_table_grad(nfftbl_plan_s* p, const TapArgs<float>& args, const double* loss, double* grad) {
    const int n = args.w.table_n;
    int box_cells = 1;
    for (int t = 0; t < D; ++t) box_cells *= args.g.box[t];
    const size_t slot = (static_cast<size_t>(box_cells) * sizeof(float2) + 127) / 128 * 128;
    const size_t smem = ((n + 1) * sizeof(double) + 127) / 128 * 128 + 128 + args.batch_smem * slot;
    auto fn = table_grad_kernel<D, W>;
    nfftbl_status st = check_cuda(p, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          static_cast<int>(smem)),
                                  "table grad smem");
    if (st != NFFTBL_OK) return st;
    if (args.n_work == 0) return NFFTBL_OK;
    int occ = 0;
    if ((st = check_cuda(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTapThreads, smem), "occupancy")) !=
        NFFTBL_OK)
        return st;
    const long long want = static_cast<long long>(std::max(occ, 1)) * p->num_sms;
    const unsigned grid = static_cast<unsigned>(std::max<long long>(1, std::min<long long>(want, args.n_work)));
    fn<<<grid, kTapThreads, smem, p->stream>>>(p->tmap, args, loss, grad);
    p->launches++;
    return check_cuda(p, cudaGetLastError(), "table grad launch");
}

nfftbl_status run_table_grad(nfftbl_plan_s* p, const TapArgs<float>& args, const double* loss, double* grad) {
    if (p->d == 1) {
        switch (p->m) {
            case 2: return launch_table_grad<1, 4>(p, args, loss, grad);
            case 3: return launch_table_grad<1, 6>(p, args, loss, grad);
            case 4: return launch_table_grad<1, 8>(p, args, loss, grad);
            default: return launch_table_grad<1, 0>(p, args, loss, grad);
        }
    }
    switch (p->m) {
        case 2: return launch_table_grad<2, 4>(p, args, loss, grad);
        case 3: return launch_table_grad<2, 6>(p, args, loss, grad);
        case 4: return launch_table_grad<2, 8>(p, args, loss, grad);
        default: return launch_table_grad<2, 0>(p, args, loss, grad);
    }
}

cudaError_t launch_residual(int is_double, void* f, const void* y, long long n, double* loss, cudaStream_t s) {
    const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
    if (n > 0) {
        if (is_double)
            residual_kernel<double><<<blocks, 256, 0, s>>>(static_cast<double2*>(f), static_cast<const double2*>(y), n,
                                                           loss);
        else
            residual_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float2*>(f), static_cast<const float2*>(y), n,
                                                          loss);
    }
    loss_finish_kernel<<<1, 1, 0, s>>>(loss);
    return cudaGetLastError();
}

cudaError_t launch_marginals(int is_double, const void* hhat, const void* fhat, long long total, int d, const int* M,
                             double* P0, double* P1, double* P2, cudaStream_t s) {
    const unsigned blocks = static_cast<unsigned>((total + 255) / 256);
    if (is_double)
        marginal_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double2*>(hhat),
                                                       static_cast<const double2*>(fhat), total, d, M[0], M[1], M[2],
                                                       P0, P1, P2);
    else
        marginal_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float2*>(hhat), static_cast<const float2*>(fhat),
                                                      total, d, M[0], M[1], M[2], P0, P1, P2);
    return cudaGetLastError();
}

cudaError_t launch_dEdpsihat(const double* P, const double* fac, int M, int L, const double* loss, double* out,
                             cudaStream_t s) {
    dEdpsihat_kernel<<<(M + 255) / 256, 256, 0, s>>>(P, fac, M, L, loss, out);
    return cudaGetLastError();
}

}  // namespace nfftbl

using namespace nfftbl;

extern "C" {

nfftbl_status nfftbl_mlp_table(const float* params_dev, int hidden, int table_len, double* table_dev, float* act_dev,
                               void* stream) {
    if (hidden != kHidden) return NFFTBL_EUNSUPPORTED;
    if (!params_dev || !table_dev || !act_dev || table_len < 3) return NFFTBL_EINVAL;
    const int n = table_len - 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mlp_forward_kernel<<<(n + 1 + 127) / 128, 128, 0, s>>>(params_dev, n, act_dev);
    mlp_table_kernel<<<(n + 1 + 255) / 256, 256, 0, s>>>(act_dev, n, table_dev);
    return cudaGetLastError() == cudaSuccess ? NFFTBL_OK : NFFTBL_ECUDA;
}

nfftbl_status nfftbl_mlp_backward(const float* params_dev, int hidden, int table_len, const float* act_dev,
                                  const double* table_dev, const double* grad_table_dev, float* scratch_dev,
                                  float* grad_params_dev, void* stream) {
    if (hidden != kHidden) return NFFTBL_EUNSUPPORTED;
    if (!params_dev || !act_dev || !table_dev || !grad_table_dev || !scratch_dev || !grad_params_dev ||
        table_len < 3)
        return NFFTBL_EINVAL;
    const int n = table_len - 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // scratch: gamma [n+1] | sum_gamma (double, 8-byte aligned) | delta2 [(n+1) x 64] | delta1 [(n+1) x 64]
    float* gamma = scratch_dev;
    double* sum_gamma = reinterpret_cast<double*>(scratch_dev + ((n + 1 + 3) / 4) * 4);
    float* delta2 = reinterpret_cast<float*>(sum_gamma + 2);
    float* delta1 = delta2 + static_cast<size_t>(n + 1) * kHidden;
    cudaMemsetAsync(grad_params_dev, 0, kParamCount * sizeof(float), s);
    cudaMemsetAsync(sum_gamma, 0, sizeof(double), s);
    const unsigned pb = (n + 1 + 255) / 256;
    gamma_kernel<<<pb, 256, 0, s>>>(grad_table_dev, table_dev, n, gamma, sum_gamma);
    backward_out_kernel<<<pb, 256, 0, s>>>(params_dev, act_dev, gamma, sum_gamma, n, delta2, grad_params_dev);
    dW2_kernel<<<1, 32 * 32, 0, s>>>(act_dev, delta2, n, grad_params_dev);
    delta1_kernel<<<(n + 1 + 15) / 16, 256, 0, s>>>(params_dev, act_dev, delta2, n, delta1);
    first_layer_grad_kernel<<<kHidden, 256, 0, s>>>(delta1, n, grad_params_dev);
    return cudaGetLastError() == cudaSuccess ? NFFTBL_OK : NFFTBL_ECUDA;
}

int64_t nfftbl_mlp_param_count(int hidden) { return hidden == kHidden ? kParamCount : -1; }

int64_t nfftbl_mlp_scratch_floats(int hidden, int table_len) {
    if (hidden != kHidden || table_len < 3) return -1;
    const int64_t np = table_len;
    return (np + 3) / 4 * 4 + 4 + 2 * np * kHidden;
}

nfftbl_status nfftbl_adam_step(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int count,
                               int step, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!params_dev || !grad_dev || !m_dev || !v_dev || count < 1 || step < 1) return NFFTBL_EINVAL;
    const float c1 = 1.f - powf(beta1, static_cast<float>(step));
    const float c2 = 1.f - powf(beta2, static_cast<float>(step));
    adam_kernel<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params_dev, grad_dev, m_dev, v_dev,
                                                                                   count, lr, beta1, beta2, eps, c1,
                                                                                   c2);
    return cudaGetLastError() == cudaSuccess ? NFFTBL_OK : NFFTBL_ECUDA;
}

}  // extern "C"
