// FP64 FMA rate of the device: the peak that the FP64 kernels' roofline is taken against.
// The paper has no counterpart; this measures the hardware the other kernels run on.
#include "tc_internal.cuh"

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (covers the FMA latency)

// Each thread runs kChains chains of `iters` dependent FMAs x <- x * b + c (b < 1, so the values
// stay bounded) and writes their sum to sink[thread], so that no FMA is dead code.
__global__ void k_fp64_fma(int iters, double b, double c, double* sink) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = 1.0 + 1e-3 * (double)(q + t % 7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += x[q];
    sink[t] = s;
}

}  // namespace

extern "C" tc_status tc_probe_fp64_fma(int blocks, int threads, int iters, void* sink, void* stream,
                                       double* flops) {
    if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !sink) return TC_ERR_ARG;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, sink) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return TC_ERR_ARG;
    }
    k_fp64_fma<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.9999999, 1e-7,
                                                                           static_cast<double*>(sink));
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
    if (flops) *flops = 2.0 * kChains * (double)iters * blocks * (double)threads;
    return TC_OK;
}
