// Throughput probes: FP64 FMA (the denominator of ALU-bound roofline fractions) and FP64 <-> FP32
// conversions, by the hardware conversion instructions and by the integer-pipe routines of
// fastcvt.h.
#include "fastcvt.h"
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

// x -> float -> (+1e-7) -> double, four independent chains per thread: two conversions per link.
// FAST: the integer-pipe routines; else the compiler's conversions.
template <bool FAST>
__global__ void cvt_chain_kernel(double* out, int iters) {
    double x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = 1.0 + 1e-6 * threadIdx.x + 0.1 * c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (FAST) x[c] = f32_to_f64(f64_to_f32(x[c]) + 1e-7f);
            else x[c] = (double)(__double2float_rn(x[c]) + 1e-7f);   // the intrinsic: a cast pair would fold
        }
    }
    const double s = x[0] + x[1] + x[2] + x[3];
    if (s == 123.456) out[0] = s;
}

template <typename K>
cudaError_t time_best(K launch, float* best_ms) {
    cudaEvent_t t0, t1;
    cudaError_t err = cudaEventCreate(&t0);
    if (err != cudaSuccess) return err;
    err = cudaEventCreate(&t1);
    if (err != cudaSuccess) {
        cudaEventDestroy(t0);
        return err;
    }
    launch();
    float best = 1e30f;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
        cudaEventRecord(t0);
        launch();
        cudaEventRecord(t1);
        err = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t0, t1);
        if (ms < best) best = ms;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    *best_ms = best;
    return err;
}

}  // namespace

cudaError_t measure_conversions(double* hw_per_s, double* int_per_s) {
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    double* out = nullptr;
    err = cudaMalloc(&out, sizeof(double));
    if (err != cudaSuccess) return err;
    const int blocks = sms * 8, threads = 256, iters = 2048;
    const double n = 2.0 * 4.0 * (double)blocks * threads * iters;   // conversions per launch
    float ms_hw = 0.f, ms_int = 0.f;
    err = time_best([&] { cvt_chain_kernel<false><<<blocks, threads>>>(out, iters); }, &ms_hw);
    if (err == cudaSuccess) err = time_best([&] { cvt_chain_kernel<true><<<blocks, threads>>>(out, iters); }, &ms_int);
    cudaFree(out);
    if (err != cudaSuccess) return err;
    *hw_per_s = n / (ms_hw * 1e-3);
    *int_per_s = n / (ms_int * 1e-3);
    return cudaSuccess;
}

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
