// FP32 peak microbenchmark: the denominator of the field kernels' roofline
// (an ALU-bound path) measured on the device instead of only derived from the
// SM count and clock. Not part of the method.
#include "common.cuh"

namespace csl {
namespace {

constexpr int kChains = 16;   // independent FFMA chains per thread (hides the FMA latency)

__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5f) out[threadIdx.x] = s;   // keeps the chains alive
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_measure_fp32_peak(double* tflops, double* sm_clock_ghz, void* stream) {
    try {
        if (!tflops) fail(CSL_ERR_INVALID_ARG, "tflops is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        int dev = 0, n_sm = 0;
        CSL_CUDA(cudaGetDevice(&dev));
        CSL_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
        DevBuf out(256 * sizeof(float), s);
        const int blocks = n_sm * 8, threads = 256, iters = 8192;
        cudaEvent_t e0, e1;
        CSL_CUDA(cudaEventCreate(&e0));
        CSL_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        for (int rep = 0; rep < 6; ++rep) {   // the first run warms up
            CSL_CUDA(cudaEventRecord(e0, s));
            k_ffma<<<blocks, threads, 0, s>>>(out.as<float>(), iters, 0.999999f, 1e-7f);
            CSL_LAUNCH_CHECK("ffma peak");
            CSL_CUDA(cudaEventRecord(e1, s));
            CSL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CSL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) best = ms < best ? ms : best;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const double flops = 2.0 * kChains * (double)iters * blocks * threads;
        *tflops = flops / (best * 1e-3) / 1e12;
        if (sm_clock_ghz) {
            int khz = 0;
            cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
            *sm_clock_ghz = khz / 1e6;
        }
        return CSL_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (...) {
        set_last_error("unknown error");
        return CSL_ERR_CUDA;
    }
}
