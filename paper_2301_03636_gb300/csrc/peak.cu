// Measurement only: the FP32 FMA rate of the CUDA cores, the denominator of
// the FP32 scorer's roofline (no measured SIMT peak is supplied with the
// machine).  Every thread runs 8 independent FMA chains; the grid fills every
// SM with 2 blocks of 1024 threads.
#include "common.cuh"

namespace adv {

constexpr int PEAK_CHAINS = 8;
__device__ float g_fma_sink;   // written only if the chains reach an impossible value

__global__ void __launch_bounds__(1024, 2) fma_peak_kernel(int iters, float x, float y, float* sink) {
    float a[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = fmaf(a[c], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += a[c];
    if (s == 1234.5f) sink[0] = s;   // keeps the chains live; never true for the inputs used
}

}  // namespace adv

extern "C" advisor_status advisor_measure_fp32_fma_peak(double* h_tflops, cudaStream_t stream) {
    if (!h_tflops) return ADVISOR_ERR_INVALID_ARGUMENT;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    float* sink = nullptr;   // a file-scope device variable: the library allocates no device memory
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    advisor_status st = ADVISOR_ERR_CUDA;
    const int iters = 16384, grid = 2 * sms, block = 1024;
    float best_ms = 0.f;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&sink), adv::g_fma_sink) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        bool ok = true;
        for (int rep = 0; rep < 4 && ok; ++rep) {   // the first launch warms up; the fastest of the rest counts
            ok = cudaEventRecord(e0, stream) == cudaSuccess;
            adv::fma_peak_kernel<<<grid, block, 0, stream>>>(iters, 0.999f, 0.001f, sink);
            ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, stream) == cudaSuccess &&
                 cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.f;
            ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (ok && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
        }
        if (ok && best_ms > 0.f) {
            const double flop = 2.0 * adv::PEAK_CHAINS * (double)iters * grid * block;
            *h_tflops = flop / (best_ms * 1e-3) / 1e12;
            st = ADVISOR_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(stream);
    return st;
}
