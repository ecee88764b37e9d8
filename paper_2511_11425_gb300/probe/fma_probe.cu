// fma_probe.cu -- FP32 FMA throughput of the current GPU: the denominator of
// the pair kernels' roofline, measured rather than assumed.  It is a
// measuring stick used by the benchmark only and is built into its own
// library (_fma_probe.so), not into libsph.
//
// Every thread runs 8 independent chains of fmaf, so the FMA pipe never
// waits on a dependency; the grid puts 8 blocks of 256 threads on every SM.
#include <cuda_runtime.h>

#include <algorithm>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_fma_probe(float *out, int iters)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    const float b = 0.9999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains alive, never true
}

}  // namespace

// Best of three timed launches in TFLOP/s (FMA = 2 flop) into *tflops and
// the SM count into *sms.  Allocates and frees a small device buffer and
// synchronises the stream.  Returns 0 on success, 1 on a NULL argument, 2 on
// a CUDA error.
extern "C" int fma_probe_tflops(double *tflops, int *sms, void *stream)
{
    if (!tflops || !sms) return 1;
    *tflops = 0.0;
    *sms = 0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 2;
    *sms = nsm;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = 2;
    } else {
        double best = 0.0;
        k_fma_probe<<<blocks, threads, 0, s>>>(out, iters / 8);  // warm-up
        for (int r = 0; r < 3 && rc == 0; ++r) {
            cudaEventRecord(e0, s);
            k_fma_probe<<<blocks, threads, 0, s>>>(out, iters);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
                rc = 2;
                break;
            }
            const double flop =
                2.0 * kChains * kUnroll * (double)iters * (double)blocks * threads;
            best = std::max(best, flop / (ms * 1e-3) / 1e12);
        }
        *tflops = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}
