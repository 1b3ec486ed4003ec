// fp64_rate.cu -- a measurement probe beside the cycle's kernels (csrc/): the
// FP64 arithmetic rate of the part.  The FP64
// form of the cycle (FP64 walk, FP64 solver) may be bound by it on a GB300,
// whose FP64 rate is a small fraction of its FP32 rate, so its roofline needs
// a measured ceiling beside the HBM one.  Every thread runs eight independent
// chains of fused multiply-adds (no dependence between the chains, so the
// pipe, not the latency of one chain, sets the rate) and writes their sum, so
// that nothing is dropped; the grid holds eight blocks of 256 threads per SM.
#include <cuda_runtime.h>

#include "common.cuh"

namespace pf {

namespace {

constexpr int FMA_CHAINS = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double *out, int iters, double a, double b)
{
    double x[FMA_CHAINS];
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k)
        x[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < FMA_CHAINS; ++k)
            x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k)
        s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace pf

// FP64 fused multiply-adds per second of the current device, 2 flops each,
// over `iters` iterations of the probe on `stream` (timed with events on it,
// after one untimed launch); TFLOP/s in *tflops.
extern "C" int pic_measure_fp64_rate(void *stream, int32_t iters, double *tflops)
{
    using namespace pf;
    if (!tflops || iters < 1)
        return PIC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PIC_ERR_CUDA;
    const int grid = 8 * sms, block = 256;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PIC_OK;
    if (cudaMalloc(&out, sizeof(double) * (size_t)grid * block) != cudaSuccess)
        return PIC_ERR_CUDA;
    float ms = 0.f;
    // a and b keep the chains finite: x -> x a + b converges to b / (1 - a)
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = PIC_ERR_CUDA;
    } else {
        k_fp64_fma<<<grid, block, 0, s>>>(out, iters, 0.999999, 1e-6);
        cudaEventRecord(e0, s);
        k_fp64_fma<<<grid, block, 0, s>>>(out, iters, 0.999999, 1e-6);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
            rc = PIC_ERR_CUDA;
    }
    if (rc == PIC_OK) {
        const double flops = 2.0 * FMA_CHAINS * (double)iters * (double)grid * (double)block;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
