// pp_rate.cu -- the fused multiply-add rate this GPU sustains in FP32 and FP64,
// measured by a kernel that does nothing else: the denominator of the roofline
// fractions of the ALU-bound propagation and QKE kernels.
//
// Every thread runs eight independent chains x <- x a + b (0 < a < 1, b > 0, so
// x stays positive and bounded), 128 FMAs per chain step, with enough warps on
// every SM (a multiple of the SM count in CTAs, full occupancy for FP32) to hide
// the FMA latency.  The rate is 2 flop per FMA over the CUDA-event time of one
// launch after an untimed one.
#include "pp_internal.cuh"

namespace {

constexpr int kRateThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kRateThreads) fma_rate_kernel(T a, T b, int iters, T *__restrict__ sink)
{
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i)
        x[i] = (T)(threadIdx.x & 7) * (T)0.125 + (T)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                x[i] = fma(x[i], a, b);
    }
    T s = x[0];
#pragma unroll
    for (int i = 1; i < kChains; ++i)
        s += x[i];
    if (s < (T)0)  // never true (x stays positive); keeps the chains live
        sink[blockIdx.x] = s;
}

template <typename T>
int measure(int ctas_per_sm, int iters, double *flop_per_s, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "device attributes");
    const int blocks = sms * ctas_per_sm;
    void *sink = nullptr;
    int rc = pp::scratch(pp::SCR_RATE, sizeof(T) * (size_t)blocks, &sink);
    if (rc)
        return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "rate events");
    const T a = (T)0.999999, b = (T)1e-6;
    fma_rate_kernel<T><<<blocks, kRateThreads, 0, st>>>(a, b, iters, (T *)sink);
    cudaEventRecord(e0, st);
    fma_rate_kernel<T><<<blocks, kRateThreads, 0, st>>>(a, b, iters, (T *)sink);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    float ms = 0.0f;
    if (e == cudaSuccess)
        e = cudaEventSynchronize(e1);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "rate kernel");
    const double fmas = (double)blocks * kRateThreads * iters * kUnroll * kChains;
    *flop_per_s = 2.0 * fmas / (ms * 1e-3);
    return PP_OK;
}

}  // namespace

extern "C" {

int pp_fma_rate(int32_t precision, double *flop_per_s, void *stream)
{
    pp::clear_error();
    if (!flop_per_s)
        return pp::fail(PP_ERR_INVALID_ARG, "flop_per_s must not be NULL");
    if (precision == PP_FP64)  // about 6 ms on a GB300
        return measure<double>(4, 200, flop_per_s, (cudaStream_t)stream);
    if (precision == PP_FP32 || precision == PP_FP32_FAST)  // about 12 ms on a GB300
        return measure<float>(8, 12000, flop_per_s, (cudaStream_t)stream);
    return pp::fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
}

}  // extern "C"
