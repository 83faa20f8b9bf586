/*
 * usr_probe.cu -- usr_fp32_peak: the FP32 fused multiply-add throughput of the
 * current GPU, measured with a register-only loop.  The pair kernel is bound
 * by FP32 arithmetic, so its roofline fraction divides by this number rather
 * than by a figure derived from unit counts and clocks.
 */
#include "usr_internal.h"

namespace {

constexpr int kChains = 8;          // independent two-wide chains per thread
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

/* iters x kChains x 2 elements x 2 flops per thread; the result is kept only so that it is computed. */
__global__ void __launch_bounds__(kProbeThreads) k_ffma_probe(float* out, int iters)
{
    float2 a[kChains];
    #pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(1e-3f * threadIdx.x + k, 1e-3f * blockIdx.x - k);
    const float2 b = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
        #pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
    }
    float s = 0.f;
    #pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    if (s == -1.2345f) out[blockIdx.x * kProbeThreads + threadIdx.x] = s;   // never true; keeps the loop live
}

}  // namespace

extern "C" usr_status usr_fp32_peak(double* tflops)
{
    if (!tflops) return USR_ERR_ARG;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return USR_ERR_CUDA;
    }
    const int blocks = sms * kProbeBlocksPerSm;
    const int iters = 1 << 14;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return USR_ERR_OOM;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    usr_status s = USR_OK;
    float ms = 0.f;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        s = USR_ERR_CUDA;
    } else {
        k_ffma_probe<<<blocks, kProbeThreads, 0, st>>>(out, iters);   // warm-up (clocks, code)
        cudaEventRecord(e0, st);
        k_ffma_probe<<<blocks, kProbeThreads, 0, st>>>(out, iters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            s = USR_ERR_CUDA;
    }
    if (s == USR_OK) {
        const double flops = (double)blocks * kProbeThreads * iters * kChains * 2.0 * 2.0;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return s;
}
