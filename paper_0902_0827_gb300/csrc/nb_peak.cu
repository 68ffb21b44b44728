// nb_peak.cu - FP32 FMA throughput microbenchmark, the measured denominator
// of the force kernel's roofline (the force kernel is bound by FP32
// instruction issue, not by a tensor-core contraction or by memory).
//
// Every thread runs kChains independent chains of dependent FMAs
// (a = a * x + y) for `iters` iterations, so the FMA pipes of every SM stay
// busy whatever the FMA latency: 8 warps x 8 blocks = 64 warps per SM, 8
// chains each.  The caller times the launch with CUDA events; the kernel
// performs grid x block x iters x kChains FMAs = twice that many FLOP.
#include <cuda_runtime.h>
#include <stdint.h>

#include "acenb.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;

__global__ void __launch_bounds__(kPeakThreads) k_fp32_peak(long long iters, float x, float y, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (long long it = 0; it < iters; it += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], x, y);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 1234.5f) sink[0] = s;  // keeps the chains alive; practically never taken
}

}  // namespace

extern "C" nb_status nb_fp32_peak_launch(int64_t iters, void *cuda_stream, float *d_sink, double *flop)
{
    if (iters < 16 || iters % 16 != 0 || !d_sink) return NB_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return NB_ERR_CUDA;
    const int blocks = sms * kPeakBlocksPerSm;
    // x slightly below 1 and y small: the chains stay finite and normal
    k_fp32_peak<<<blocks, kPeakThreads, 0, (cudaStream_t)cuda_stream>>>(iters, 0.999999f, 1e-7f, d_sink);
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
    if (flop) *flop = 2.0 * (double)blocks * kPeakThreads * (double)iters * kChains;
    return NB_OK;
}
