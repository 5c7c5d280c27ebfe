// peak.cu -- measured arithmetic peaks of the GPU the library runs on, the
// denominators of the roofline fractions the benchmark reports for the
// FP64-pipe kernels (not part of the method).  A dependent chain of fused
// multiply-adds per accumulator, eight independent accumulators per thread,
// enough resident warps on every SM to hide the pipe latency; timed with
// CUDA events after one warm-up launch.  No clock or GPU setting is touched.
#include <cuda_runtime.h>

#include "qmc_internal.cuh"

template <class R>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, R b, R c, R *out)
{
    R a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (R)(threadIdx.x + j) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = a[j] * b + c;
    }
    R s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    // written only for an impossible value, so the chain cannot be removed
    if (s == (R)-1.2345e-30) out[blockIdx.x] = s;
}

extern "C" int qmc_peak_fma(int fp64, int iters, double *tflops)
{
    if (!tflops || iters < 1 || iters > (1 << 20)) return QMC_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return QMC_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    void *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) return QMC_ERR_OOM;
    cudaStream_t s;
    cudaEvent_t e0, e1;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch is the warm-up
        cudaEventRecord(e0, s);
        if (fp64)
            k_fma_peak<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, (double *)out);
        else
            k_fma_peak<float><<<blocks, threads, 0, s>>>(iters, 0.9999f, 1e-4f, (float *)out);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    QMC_COUNT(4);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(out);
    if (err != cudaSuccess) return QMC_ERR_CUDA;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return QMC_OK;
}
