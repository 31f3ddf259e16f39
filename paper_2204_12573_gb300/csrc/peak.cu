// Measured FP32 FMA throughput of the device: the denominator of the
// roofline of the descriptor and force kernels, which are bound by FP32
// arithmetic issue rather than by HBM or the tensor cores.  (No counterpart
// in the paper; a measurement utility.)
//
// Every thread runs kChains independent FMA chains x <- x * a + b held in
// registers, so the FMA pipes never wait on a dependency and nothing touches
// memory until the end.  The grid fills every SM to its occupancy limit; the
// SM count comes from the device.  Each launch is timed with CUDA events on
// the caller's stream.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace flr {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float a, float b, int iters, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    // a contraction with a < 1 keeps x finite and away from this value, so
    // the store never happens, but the compiler cannot drop the chains
    if (s == -1.f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace flr

using namespace flr;

extern "C" int flr_fp32_fma_peak(int device, int32_t launches, double *tflops_best, double *tflops_median,
                                 int32_t *num_sms)
{
    if (launches < 1 || !tflops_best) {
        set_error("flr_fp32_fma_peak: launches >= 1 and tflops_best are required");
        return FLR_EINVAL;
    }
    int s = cuda_fail(cudaSetDevice(device), "flr_fp32_fma_peak: device");
    if (s != FLR_OK) return s;
    int sms = 0, per_sm = 0;
    s = cuda_fail(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "SM count");
    if (s != FLR_OK) return s;
    s = cuda_fail(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0), "occupancy");
    if (s != FLR_OK) return s;
    per_sm = std::max(per_sm, 1);
    const int grid = sms * per_sm;
    // about 30 ms per launch at the nominal rate of a GB300-class part
    const int iters = 20000;
    const double flops = 2.0 * (double)grid * kPeakThreads * (double)iters * kUnroll * kChains;
    float *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    s = cuda_fail(cudaMalloc(&sink, sizeof(float) * grid), "flr_fp32_fma_peak: sink");
    if (s == FLR_OK) s = cuda_fail(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    if (s == FLR_OK) s = cuda_fail(cudaEventCreate(&e0), "event");
    if (s == FLR_OK) s = cuda_fail(cudaEventCreate(&e1), "event");
    std::vector<double> tf;
    if (s == FLR_OK) {
        k_fma_peak<<<grid, kPeakThreads, 0, st>>>(0.999999f, 1e-7f, iters / 8, sink);   // warm-up
        for (int k = 0; k < launches && s == FLR_OK; ++k) {
            cudaEventRecord(e0, st);
            k_fma_peak<<<grid, kPeakThreads, 0, st>>>(0.999999f, 1e-7f, iters, sink);
            cudaEventRecord(e1, st);
            s = cuda_fail(cudaEventSynchronize(e1), "flr_fp32_fma_peak: kernel");
            float ms = 0.f;
            if (s == FLR_OK) s = cuda_fail(cudaEventElapsedTime(&ms, e0, e1), "event time");
            if (s == FLR_OK) tf.push_back(flops / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    if (s != FLR_OK) return s;
    std::sort(tf.begin(), tf.end());
    *tflops_best = tf.back();
    if (tflops_median) *tflops_median = tf[tf.size() / 2];
    if (num_sms) *num_sms = sms;
    return FLR_OK;
}
