// Step 0a on the device: the window transform psi_hat(k) (Algorithm 4.2) or
// phi_hat(k) (Algorithm 2.1) for k in I_M, in FP64, and the per-dimension
// precorrection factors d(k) = 1/(L psi_hat(k)) whose tensor product is the
// diagonal D_psihat of Eq. 4.9.  Also the FFT twiddle tables.
//
// Quadrature rule: psi is even, so psi_hat(k) = 2 int_0^{m/L} psi(x) cos(2 pi k x) dx
// (Fourier convention of Eq. 3.1).  Substituting L x = m sin(theta) turns the
// square-root edge of the sinh / Kaiser-Bessel windows into an entire
// function of theta (sqrt(1 - (Lx/m)^2) = cos(theta)), so composite
// Gauss-Legendre on uniform theta panels converges exponentially.
#include <cmath>
#include <vector>

#include "plan_internal.h"

namespace nfftbl {
namespace {

constexpr int kGLOrder = 16;

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on the
// three-term recurrence of the Legendre polynomials (computed once, host).
struct GLRule {
    double x[kGLOrder];
    double w[kGLOrder];
    GLRule() {
        const int n = kGLOrder;
        for (int i = 0; i < n; ++i) {
            double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
            double dp = 0.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = pk;
                }
                // p1 = P_n(z), p0 = P_{n-1}(z)
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

__constant__ double c_gl_x[kGLOrder];
__constant__ double c_gl_w[kGLOrder];

__device__ double catmull_rom_d(const double* v, int n, double u) {
    // v has n+1 entries on u_i = i/n; ghost values v_{-1} = v_1, v_{n+1} = 2 v_n - v_{n-1}
    double s = fmin(fmax(u, 0.0), 1.0) * n;
    int i = min(static_cast<int>(floor(s)), n - 1);
    double t = s - i;
    double p0 = (i == 0) ? v[1] : v[i - 1];
    double p1 = v[i];
    double p2 = v[i + 1];
    double p3 = (i + 2 <= n) ? v[i + 2] : 2.0 * v[n] - v[n - 1];
    return 0.5 * (2.0 * p1 + (p2 - p0) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t +
                  (3.0 * p1 - p0 - 3.0 * p2 + p3) * t * t * t);
}

// One block per frequency: k = kidx - M/2 (vlist == NULL; writes the factor
// 1/(L psi_hat(k))) or k = vlist[kidx] (writes psi_hat(k) itself).
__global__ void window_factor_kernel(int with_sinc, int window, int L, int M, int m, double beta,
                                     const double* __restrict__ table, int table_n, int panels,
                                     const double* __restrict__ vlist, double* __restrict__ fac_out) {
    const int kidx = blockIdx.x;
    const double k = vlist ? vlist[kidx] : static_cast<double>(kidx - M / 2);
    const double h = 0.5 * M_PI / panels;           // panel width in theta
    const double ml = static_cast<double>(m) / L;    // support half-width m/L
    double norm = 1.0;
    if (window == NFFTBL_WIN_SINH) norm = 1.0 / sinh(beta);
    if (window == NFFTBL_WIN_CKB) norm = 1.0 / (cyl_bessel_i0(beta) - 1.0);
    double sum = 0.0;
    for (int idx = threadIdx.x; idx < panels * kGLOrder; idx += blockDim.x) {
        const int pnl = idx / kGLOrder;
        const int q = idx - pnl * kGLOrder;
        const double a = pnl * h;
        const double th = a + 0.5 * h * (c_gl_x[q] + 1.0);
        double st, ct;
        sincos(th, &st, &ct);
        double phi;
        if (window == NFFTBL_WIN_SINH) {
            phi = sinh(beta * ct) * norm;
        } else if (window == NFFTBL_WIN_CKB) {
            phi = (cyl_bessel_i0(beta * ct) - 1.0) * norm;
        } else {
            phi = catmull_rom_d(table, table_n, st);
        }
        double ker = phi;
        if (with_sinc) {
            const double z = m * st;                 // L x = m sin(theta)
            ker *= (z == 0.0) ? 1.0 : sinpi(z) / (M_PI * z);
        }
        const double x = ml * st;
        sum += 2.0 * ker * cospi(2.0 * k * x) * ml * ct * (0.5 * h * c_gl_w[q]);
    }
    // block reduction (fixed order: warp shuffles, then warp partials in order)
    __shared__ double part[32];
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (blockDim.x + 31) / 32; ++w) tot += part[w];
        fac_out[kidx] = vlist ? tot : 1.0 / (static_cast<double>(L) * tot);
    }
}

template <typename T>
__global__ void cast_factor_kernel(const double* __restrict__ fac64, int M, T* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int k = i - M / 2;
    // (-1)^k folds the centring shift l = s - L/2 of the grid into the factor
    const double v = (k & 1) ? -fac64[i] : fac64[i];
    out[i] = static_cast<T>(v);
}

template <typename T>
__global__ void twiddle_kernel(int L, C2<T>* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= L) return;
    double s, c;
    sincospi(2.0 * j / L, &s, &c);   // 2j/L is exact
    out[j] = cmake<T>(static_cast<T>(c), static_cast<T>(s));
}

// FP32 copy of the window table, and per interval i (of n - 1) the
// Catmull-Rom cubic in t in [0, 1) as c0 + c1 t + c2 t^2 + c3 t^3 (ghost
// values v_{-1} = v_1, v_n' = 2 v_{n-1} - v_{n-2} at the last sample),
// formed in FP64 and rounded once.
__global__ void table_cast_kernel(const double* __restrict__ in, int n, float* __restrict__ out,
                                  float4* __restrict__ coef) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = static_cast<float>(in[i]);
    const int tn = n - 1;
    if (coef && i < tn) {
        const double p0 = (i == 0) ? in[1] : in[i - 1];
        const double p1 = in[i];
        const double p2 = in[i + 1];
        const double p3 = (i + 2 <= tn) ? in[i + 2] : 2.0 * in[tn] - in[tn - 1];
        coef[i] = make_float4(static_cast<float>(p1), static_cast<float>(0.5 * (p2 - p0)),
                              static_cast<float>(0.5 * (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3)),
                              static_cast<float>(0.5 * (3.0 * p1 - p0 - 3.0 * p2 + p3)));
    }
}

bool g_gl_uploaded = false;

constexpr int kTablePanels = 1024;   // panels of the rule for tabulated windows

// Part (B) of the table-window loss gradient: psi_hat_t(q) is the same
// quadrature as window_factor_kernel, linear in the table, so
//   dE/dv_i = sum_q dE/dpsi_hat(q) sum_p 2 w_p sinc(pi m sin th_p) cos(2 pi q x_p) c_i(sin th_p)
// with c_i the Catmull-Rom weights; one thread per quadrature point.
__global__ void window_table_grad_kernel(int L, int M, int m, int table_n, int panels,
                                         const double* __restrict__ dEdpsi, double* __restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= panels * kGLOrder) return;
    const int pnl = p / kGLOrder;
    const int q = p - pnl * kGLOrder;
    const double h = 0.5 * M_PI / panels;
    const double th = pnl * h + 0.5 * h * (c_gl_x[q] + 1.0);
    double st, ct;
    sincos(th, &st, &ct);
    const double ml = static_cast<double>(m) / L;
    const double x = ml * st;
    const double z = m * st;
    const double sincv = (z == 0.0) ? 1.0 : sinpi(z) / (M_PI * z);
    const double wp = ml * ct * 0.5 * h * c_gl_w[q];
    double G = 0.0;
    for (int k = 0; k < M; ++k) G += dEdpsi[k] * 2.0 * cospi(2.0 * (k - M / 2) * x);
    const double gamma = wp * sincv * G;
    if (gamma != 0.0) scatter_catmull(grad, table_n, st, gamma);
}

}  // namespace

cudaError_t launch_window_factors(int with_sinc, int window, int L, int M, int m, double beta,
                                  const double* table, int table_n, double* fac64_out, cudaStream_t s) {
    static GLRule rule;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_gl_x, rule.x, sizeof(rule.x), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbolAsync(c_gl_w, rule.w, sizeof(rule.w), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    g_gl_uploaded = true;
    // a tabulated window is only piecewise cubic: more panels
    const int panels = (window == NFFTBL_WIN_TABLE) ? kTablePanels : 96;
    window_factor_kernel<<<M, 256, 0, s>>>(with_sinc, window, L, M, m, beta, table, table_n, panels, nullptr,
                                           fac64_out);
    return cudaGetLastError();
}

cudaError_t upload_gl_rule_sync() {
    static GLRule rule;
    cudaError_t e = cudaMemcpyToSymbol(c_gl_x, rule.x, sizeof(rule.x), 0, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gl_w, rule.w, sizeof(rule.w), 0, cudaMemcpyHostToDevice);
    return e;
}

cudaError_t launch_window_factors_preloaded(int with_sinc, int window, int L, int M, int m, double beta,
                                            double* fac64_out, cudaStream_t s) {
    const int panels = (window == NFFTBL_WIN_TABLE) ? kTablePanels : 96;
    window_factor_kernel<<<M, 256, 0, s>>>(with_sinc, window, L, M, m, beta, nullptr, 0, panels, nullptr,
                                           fac64_out);
    return cudaGetLastError();
}

cudaError_t launch_window_transform(int with_sinc, int window, int L, int m, double beta, const double* table,
                                    int table_n, const double* v, int n, double* out, cudaStream_t s) {
    static GLRule rule;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_gl_x, rule.x, sizeof(rule.x), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_gl_w, rule.w, sizeof(rule.w), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    const int panels = (window == NFFTBL_WIN_TABLE) ? kTablePanels : 96;
    window_factor_kernel<<<n, 256, 0, s>>>(with_sinc, window, L, 0, m, beta, table, table_n, panels, v, out);
    return cudaGetLastError();
}

cudaError_t launch_window_table_grad(int L, int M, int m, int table_n, const double* dEdpsi, double* grad,
                                     cudaStream_t s) {
    static GLRule rule;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_gl_x, rule.x, sizeof(rule.x), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_gl_w, rule.w, sizeof(rule.w), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const int pts = kTablePanels * kGLOrder;
    window_table_grad_kernel<<<(pts + 255) / 256, 256, 0, s>>>(L, M, m, table_n, kTablePanels, dEdpsi, grad);
    return cudaGetLastError();
}

cudaError_t launch_cast_factors(const double* fac64, int M, void* out, int is_double, cudaStream_t s) {
    const int blocks = (M + 255) / 256;
    if (is_double)
        cast_factor_kernel<double><<<blocks, 256, 0, s>>>(fac64, M, static_cast<double*>(out));
    else
        cast_factor_kernel<float><<<blocks, 256, 0, s>>>(fac64, M, static_cast<float*>(out));
    return cudaGetLastError();
}

cudaError_t launch_twiddles(int L, void* out, int is_double, cudaStream_t s) {
    const int blocks = (L + 255) / 256;
    if (is_double)
        twiddle_kernel<double><<<blocks, 256, 0, s>>>(L, static_cast<double2*>(out));
    else
        twiddle_kernel<float><<<blocks, 256, 0, s>>>(L, static_cast<float2*>(out));
    return cudaGetLastError();
}

cudaError_t launch_table_cast(const double* in, int n, float* out, float4* coef, cudaStream_t s) {
    table_cast_kernel<<<(n + 255) / 256, 256, 0, s>>>(in, n, out, coef);
    return cudaGetLastError();
}

}  // namespace nfftbl
