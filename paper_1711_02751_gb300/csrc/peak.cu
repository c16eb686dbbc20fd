// FP64 FMA throughput probe: the denominator of ALU-bound roofline fractions.
#include "internal.h"

namespace hdgdg {
namespace {

constexpr int kChains = 8;

__global__ void fma_chain_kernel(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 123.456) out[0] = s;   // keeps the chains live; never true in practice
}

}  // namespace

cudaError_t measure_fp64_fma(double* tflops) {
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    double* out = nullptr;
    err = cudaMalloc(&out, sizeof(double));
    if (err != cudaSuccess) return err;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const int blocks = sms * 8, threads = 256, iters = 2048;
    for (int w = 0; w < 2; ++w) fma_chain_kernel<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7);
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(t0);
        fma_chain_kernel<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7);
        cudaEventRecord(t1);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (ms < best) best = ms;
    }
    err = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (err != cudaSuccess) return err;
    const double flops = 2.0 * (double)blocks * threads * kChains * (double)iters;
    *tflops = flops / (best * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace hdgdg
