// k_probe.cu -- measured FP64 fused multiply-add rate of the GPU, the peak
// against which the FP64 forms' arithmetic-bound kernels are reported.
//
// Every thread runs eight independent FP64 FMA chains, so the FP64 pipe, not
// the dependency latency, sets the rate; a grid of eight 256-thread blocks
// per SM keeps every SM's FP64 units busy. Two FLOPs per FMA.
#include <string>

#include "pdf_internal.cuh"

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) k_dfma_rate(double* sink, int iters, double m, double c) {
    double a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1e-3 * (threadIdx.x + 1) + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 12345.678) sink[0] = s;  // keeps the chains; never true for these inputs
}

}  // namespace

extern "C" {

int pdf_measure_fp64_fma_rate(void* cuda_stream, double* tflops) {
    if (!tflops) return fail(nullptr, PDF_ERR_ARG, "pdf_measure_fp64_fma_rate: NULL output");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = 8 * sms, threads = 256, iters = 8192;
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_dfma_rate<<<blocks, threads, 0, s>>>(sink, iters / 8, 1.0000001, 1e-9);  // warm-up
        cudaEventRecord(t0, s);
        k_dfma_rate<<<blocks, threads, 0, s>>>(sink, iters, 1.0000001, 1e-9);
        cudaEventRecord(t1, s);
        e = cudaEventSynchronize(t1);
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess)
        return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_measure_fp64_fma_rate: ") + cudaGetErrorString(e));
    const double flops = 2.0 * CHAINS * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return PDF_OK;
}

}  // extern "C"
