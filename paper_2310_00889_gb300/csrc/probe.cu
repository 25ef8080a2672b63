// Arithmetic-peak probes: long chains of independent fused multiply-adds, to check the
// FP32 CUDA-core peak the pair-sum roofline divides by (SMs x 128 lanes x 2 flops x clock),
// whether the packed FP32x2 FMA raises it, and the FP64 rate that bounds the FP64 pair sum
// and the quadrature-correction builder.
//   kind 0: scalar FFMA      (8 independent chains per thread)
//   kind 1: packed FFMA x2   (fma.rn.f32x2, 4 independent pairs per thread: 8 FMAs)
//   kind 2: DFMA             (8 independent chains per thread)
// Grid: 4 CTAs of 256 threads per SM.  Flops = 2 per FMA.  Timed with CUDA events on the
// given stream around one launch, after one warm-up launch.
#include "engine.h"

namespace sbq {

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(int iters, float b, float c, float *out)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k)
        a[k] = 1e-3f * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k)
            a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k)
        s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    return (static_cast<unsigned long long>(__float_as_uint(hi)) << 32) | __float_as_uint(lo);
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma2(int iters, float b, float c, float *out)
{
    unsigned long long a[PROBE_CHAINS / 2];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS / 2; ++k)
        a[k] = pack2(1e-3f * threadIdx.x + 2 * k, 1e-3f * threadIdx.x + 2 * k + 1);
    const unsigned long long bb = pack2(b, b), cc = pack2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS / 2; ++k)
            a[k] = ffma2(a[k], bb, cc);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS / 2; ++k)
        s += __uint_as_float(static_cast<unsigned>(a[k])) + __uint_as_float(static_cast<unsigned>(a[k] >> 32));
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(int iters, double b, double c, float *out)
{
    double a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k)
        a[k] = 1e-3 * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k)
            a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k)
        s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = static_cast<float>(s);
}

}  // namespace

}  // namespace sbq

extern "C" __attribute__((visibility("default"))) int sbq_peak_probe(int kind, double *tflops,
                                                                      double *ms, void *stream)
{
    using namespace sbq;
    clear_error();
    if (kind < 0 || kind > 2 || !tflops || !ms) {
        set_error("sbq_peak_probe: kind must be 0, 1 or 2 and the outputs non-null");
        return SBQ_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = device_props().sms * 4;
    const int iters = kind == 2 ? 2048 : 65536;
    DevBuf out;
    SBQ_TRY(out.alloc(static_cast<size_t>(grid) * PROBE_THREADS * sizeof(float)));
    cudaEvent_t e0, e1;
    SBQ_CUDA(cudaEventCreate(&e0));
    SBQ_CUDA(cudaEventCreate(&e1));
    float elapsed = 0.0f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        if (kind == 0)
            k_probe_ffma<<<grid, PROBE_THREADS, 0, s>>>(iters, 0.999999f, 1e-7f, out.as<float>());
        else if (kind == 1)
            k_probe_ffma2<<<grid, PROBE_THREADS, 0, s>>>(iters, 0.999999f, 1e-7f, out.as<float>());
        else
            k_probe_dfma<<<grid, PROBE_THREADS, 0, s>>>(iters, 0.999999, 1e-7, out.as<float>());
        cudaEventRecord(e1, s);
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_status(le, "sbq_peak_probe launch");
        }
        const cudaError_t se = cudaEventSynchronize(e1);
        if (se != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_status(se, "sbq_peak_probe sync");
        }
        cudaEventElapsedTime(&elapsed, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * PROBE_CHAINS * static_cast<double>(iters) * grid * PROBE_THREADS;
    *ms = elapsed;
    *tflops = flops / (elapsed * 1e-3) / 1e12;
    return SBQ_OK;
}
