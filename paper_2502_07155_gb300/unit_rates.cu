// Per-SM throughput of the arithmetic units the short-sum kernels use:
// FP32 FMA and the special-function unit (MUFU: ex2, rsqrt, rcp), in lane
// operations per SM per clock.  Each thread runs 8 independent dependency
// chains of one instruction; the chains' results are summed into a checksum
// so that no instruction is dead.  Used to derive the ALU / SFU roofline
// peaks of the tap kernels.
#include <cstdio>
#include <cuda_runtime.h>

template <int OP>
__global__ void chains(float* out, int iters) {
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = 1.0f + 1e-3f * static_cast<float>((threadIdx.x + c) & 63);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float y;
            if (OP == 0) asm volatile("fma.rn.f32 %0, %1, 0f3F7FF972, 0f38D1B717;" : "=f"(y) : "f"(v[c]));
            if (OP == 1) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[c]));
            if (OP == 2) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[c]));
            if (OP == 3) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[c]));
            // ex2: keep inputs bounded; rcp: the added constant keeps the chain from
            // folding (one extra FP32 op on the FMA pipe, far from its limit)
            v[c] = (OP == 1) ? y * 0.5f : (OP == 3) ? y + 1.0f : y;
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
static int run(const char* name, int sms, float* out, float* host) {
    const int blocks = sms * 8, threads = 256, iters = 4096;
    chains<OP><<<blocks, threads>>>(out, 16);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    chains<OP><<<blocks, threads>>>(out, iters);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    if (cudaGetLastError() != cudaSuccess) return 1;
    cudaMemcpy(host, out, sizeof(float) * blocks * threads, cudaMemcpyDeviceToHost);
    double check = 0.0;
    for (int i = 0; i < blocks * threads; ++i) check += host[i];
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    const double ops = static_cast<double>(blocks) * threads * iters * 8;
    const double per_clk = ops / (ms * 1e-3) / sms / (clk_khz * 1e3);
    printf("{\"op\": \"%s\", \"ms\": %.4f, \"lane_ops_per_clk_per_sm\": %.2f, \"clock_mhz\": %d, \"checksum\": %.6e}\n",
           name, ms, per_clk, clk_khz / 1000, check);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return 0;
}

int main() {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
    float* out = nullptr;
    const size_t n = static_cast<size_t>(sms) * 8 * 256;
    if (cudaMalloc(&out, sizeof(float) * n) != cudaSuccess) return 1;
    float* host = new float[n];
    int bad = 0;
    bad |= run<0>("ffma", sms, out, host);
    bad |= run<1>("ex2", sms, out, host);
    bad |= run<2>("rsqrt", sms, out, host);
    bad |= run<3>("rcp", sms, out, host);
    delete[] host;
    cudaFree(out);
    return (bad || cudaDeviceSynchronize() != cudaSuccess) ? 1 : 0;
}
