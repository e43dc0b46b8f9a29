// probe.cu -- bab_probe_fp32_peak: the FP32 FMA rate this GPU sustains, the
// roof of the CUDA-core kernels (the FP32 rollout, interval bounds, CROWN on
// CUDA cores).  No counterpart in the paper: a measurement, like the copy
// bandwidth and GEMM rate the tensor-core and memory roofs are taken from.
//
// Every thread runs kChains independent FMA chains x <- x * a + b for `iters`
// rounds, as scalar FMAs or as paired FP32 FMAs (fma.rn.f32x2, two FMAs per
// instruction); the grid fills every SM with two 1024-thread CTAs.  The chains'
// values (each converging to 1) are folded into one word that is stored to a
// file-scope device variable only if it equals a value it cannot take, so the
// compiler keeps every FMA and nothing is written.
#include "bab_internal.cuh"

namespace bab {

namespace {

constexpr int kChains = 16;

__device__ float g_probe_sink;

template <bool PAIRED>
__global__ void __launch_bounds__(1024, 2) k_fma_probe(int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
        if (PAIRED) {
            const unsigned long long av = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
            const unsigned long long bv = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
#pragma unroll
            for (int j = 0; j < kChains; j += 2) {
                unsigned long long xv = ((unsigned long long)__float_as_uint(x[j + 1]) << 32) | __float_as_uint(x[j]);
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(xv) : "l"(av), "l"(bv));
                x[j] = __uint_as_float((unsigned)(xv & 0xFFFFFFFFull));
                x[j + 1] = __uint_as_float((unsigned)(xv >> 32));
            }
        } else {
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += x[j];
    if (acc == -12345.678f) g_probe_sink = acc;
}

}  // namespace

}  // namespace bab

extern "C" int bab_probe_fp32_peak(double *tflops, double *tflops_paired, void *stream)
{
    using namespace bab;
    if (!tflops) return BAB_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return BAB_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = 2 * sms, threads = 1024, iters = 16384;
    const double flops = 2.0 * kChains * (double)iters * threads * grid;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return BAB_ERR_CUDA;
    }
    double best[2] = {0.0, 0.0};
    cudaError_t err = cudaSuccess;
    for (int paired = 0; paired < 2 && err == cudaSuccess; ++paired) {
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // the first run warms up (and loads the kernel)
            cudaEventRecord(e0, st);
            if (paired) k_fma_probe<true><<<grid, threads, 0, st>>>(iters, 0.999f, 1e-3f);
            else k_fma_probe<false><<<grid, threads, 0, st>>>(iters, 0.999f, 1e-3f);
            cudaEventRecord(e1, st);
            err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && rep > 0 && ms > 0.f) {
                const double r = flops / (ms * 1e-3) / 1e12;
                best[paired] = r > best[paired] ? r : best[paired];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return BAB_ERR_CUDA;
    }
    *tflops = best[0];
    if (tflops_paired) *tflops_paired = best[1];
    return BAB_OK;
}
