// lb_device.cu -- measured FP64 arithmetic peak of the current device, the
// denominator of the FP64 step kernel's roofline.  The FP64 form of the time
// step (real = double) is bound by the FP64 pipe, not by HBM, so its
// fraction of peak is taken against the fused multiply-add rate this kernel
// measures: independent dependency chains of fma(a, b, c) per thread (enough
// of them to cover the pipe's latency), every SM fully occupied, timed with
// CUDA events.  It belongs to no equation of the paper; it measures the
// machine the method runs on.
#include <cuda_runtime.h>

#include "lb.h"
#include "lb_launch.h"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kUnroll = 16;    // fused multiply-adds per chain per loop trip

__global__ void __launch_bounds__(256) k_dfma_chains(double *out, int trips, double b, double c)
{
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-9 * (threadIdx.x + j);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0) out[blockIdx.x] = s;   // never true for these operands: keeps the chains live
}

}  // namespace

extern "C" int lb_device_fp64_peak(int32_t trips, double *tflops)
{
    if (trips < 1 || !tflops) {
        lbk::set_last_error("lb_device_fp64_peak: trips must be >= 1 and tflops not NULL");
        return LB_EINVAL;
    }
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dfma_chains, 256, 0);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *out = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * (occ > 0 ? occ : 1);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)blocks * sizeof(double));
    float best = 0.f;
    // a warm-up launch, then the best of five
    for (int r = 0; r < 6 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_dfma_chains<<<blocks, 256, 0, s>>>(out, trips, 0.9999999999, 1e-12);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess || best <= 0.f) {
        cudaGetLastError();
        lbk::set_last_error("lb_device_fp64_peak: a CUDA call failed");
        return LB_ECUDA;
    }
    const double flops = 2.0 * kChains * kUnroll * (double)trips * blocks * 256.0;
    *tflops = flops / (best * 1e-3) / 1e12;
    return LB_OK;
}
