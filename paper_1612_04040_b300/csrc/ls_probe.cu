// ls_probe.cu -- measured FP64 peak of this GPU (the denominator of the FP64
// stencil's roofline): a kernel of independent FP64 fused multiply-add
// chains, timed with CUDA events.
#include <cuda_runtime.h>

#include "ls.h"

namespace {

constexpr int CHAINS = 8;

// every thread runs CHAINS independent x <- x * a + b chains; the values stay
// bounded (|a| < 1) and are summed into out so nothing is dead code
__global__ void __launch_bounds__(256) k_dfma(double* out, long long iters, double a, double b)
{
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * 256 + threadIdx.x] = s;
}

}  // namespace

extern "C" int ls_probe_dfma(long long iters, double* tflops, void* stream)
{
    if (!tflops || iters < 1) return LS_EINVAL;
    *tflops = 0.0;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LS_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dfma, 256, 0);
    if (sms < 1 || per < 1) return LS_ECUDA;
    const int grid = sms * per;
    cudaStream_t s = (cudaStream_t)stream;
    double* out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * 256 * sizeof(double)) != cudaSuccess) return LS_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int r = LS_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = LS_ECUDA;
    if (r == LS_OK) {
        k_dfma<<<grid, 256, 0, s>>>(out, iters / 8 + 1, 0.999999, 1e-7);  // warm-up
        cudaEventRecord(e0, s);
        k_dfma<<<grid, 256, 0, s>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || ms <= 0.f)
            r = LS_ECUDA;
        else
            *tflops = 2.0 * CHAINS * (double)iters * grid * 256 / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return r;
}
