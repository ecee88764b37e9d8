// sph_probe.cu -- FP32 FMA throughput of this GPU, for the roofline of the
// pair kernels (the paper has no counterpart: it is a measuring stick).
//
// Every thread runs 8 independent chains of fmaf, so the FMA pipe never
// waits on a dependency; the grid fills every SM with 2048 threads.
#include "sph_internal.cuh"

namespace sph {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;

__global__ void __launch_bounds__(256) k_fma_probe(float *out, int iters)
{
    float a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    const float b = 0.9999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains alive, never true
}

}  // namespace sph

extern "C" sph_status sph_probe_fp32_peak(double *tflops, void *stream)
{
    using namespace sph;
    if (!tflops) return SPH_ERR_ARG;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SPH_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sph_status rc = SPH_OK;
    if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = SPH_ERR_CUDA;
    } else {
        double best = 0.0;
        k_fma_probe<<<blocks, threads, 0, s>>>(out, iters / 8);  // warm-up
        for (int r = 0; r < 3 && rc == SPH_OK; ++r) {
            cudaEventRecord(e0, s);
            k_fma_probe<<<blocks, threads, 0, s>>>(out, iters);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
                rc = SPH_ERR_CUDA;
                break;
            }
            const double flop = 2.0 * kProbeChains * kProbeUnroll * (double)iters *
                                (double)blocks * threads;
            best = std::max(best, flop / (ms * 1e-3) / 1e12);
        }
        *tflops = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}
