// FP64 peak probe: the roofline denominator of the FP64 form, measured on the GPU
// the library runs on.
//
// GB300's FP64 rate is far below its tensor rates and no vendor peak is measured by
// the benchmark harness for it, so the library measures it itself: a DFMA kernel
// (every thread runs 16 independent fused multiply-add chains in registers) and an
// FP64 mma.sync kernel (m8n8k4, 8 independent accumulators per warp), each timed with
// CUDA events over several occupancies; the best rate of each is returned.  Nothing
// here reads or writes memory in its loops, so the rates are those of the FP64 pipe.
#include "../../include/ccsd.h"

#include <cuda_runtime.h>

#include <algorithm>

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) dfma_probe_kernel(double* __restrict__ sink, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * (threadIdx.x + 1) + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.0) sink[0] = s;     // never true for these inputs; keeps the chains live
}

constexpr int kAcc = 8;

__global__ void __launch_bounds__(256) dmma_probe_kernel(double* __restrict__ sink, int iters, double a, double b)
{
    double c0[kAcc], c1[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) { c0[i] = 1e-3 * threadIdx.x; c1[i] = 1e-3 * i; }
    const double av = a * (1 + (threadIdx.x & 3)), bv = b * (1 + (threadIdx.x >> 3));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kAcc; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c0[i]), "+d"(c1[i]) : "d"(av), "d"(bv));
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += c0[i] + c1[i];
    if (s == -1.0) sink[0] = s;
}

}  // namespace

extern "C" int ccsd_fp64_peak_probe(double* dfma_tflops, double* dmma_tflops)
{
    if (!dfma_tflops && !dmma_tflops) return CCSD_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CCSD_ERR_CUDA;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* sink = nullptr;
    int rc = CCSD_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        rc = CCSD_ERR_CUDA;
    }
    double best[2] = {0.0, 0.0};
    // blocks of 256 threads per SM; iterations chosen for launches of roughly 20-80 ms
    const int per_sm[3] = {2, 4, 8};
    for (int kind = 0; kind < 2 && !rc; ++kind) {
        if ((kind == 0 && !dfma_tflops) || (kind == 1 && !dmma_tflops)) continue;
        for (int p : per_sm) {
            const int blocks = sms * p;
            const int iters = kind == 0 ? 16384 / p * 4 : 16384 / p;
            // flops per launch: DFMA 2 per chain step per thread; mma 2*8*8*4 per accumulator step per warp
            const double flops = kind == 0 ? 2.0 * kChains * iters * 256.0 * blocks
                                           : 512.0 * kAcc * iters * (256.0 / 32.0) * blocks;
            for (int rep = 0; rep < 2 && !rc; ++rep) {     // the first launch warms the clocks
                cudaEventRecord(e0, st);
                if (kind == 0) dfma_probe_kernel<<<blocks, 256, 0, st>>>(sink, iters, 0.9999999, 1e-7);
                else dmma_probe_kernel<<<blocks, 256, 0, st>>>(sink, iters, 0.999, 1e-4);
                cudaEventRecord(e1, st);
                float ms = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    cudaGetLastError();
                    rc = CCSD_ERR_CUDA;
                    break;
                }
                if (rep == 1 && ms > 0.f) best[kind] = std::max(best[kind], flops / (ms * 1e-3) / 1e12);
            }
        }
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (rc) return rc;
    if (dfma_tflops) *dfma_tflops = best[0];
    if (dmma_tflops) *dmma_tflops = best[1];
    return CCSD_OK;
}
