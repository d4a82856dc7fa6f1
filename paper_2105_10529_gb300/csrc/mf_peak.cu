// FMA throughput of the device in FP32 and FP64: the ALU peak that the
// matrix-element kernels are measured against (their roofline is the FMA
// pipe, not HBM).  Every thread runs 8 independent multiply-add chains, so
// neither the FMA latency nor the issue of one warp limits the rate; 8 CTAs
// of 256 threads per SM keep every scheduler busy.
#include <cuda_runtime.h>

#include "../../include/madflow_gb300.h"

namespace {

constexpr int PEAK_TPB = 256;
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_UNROLL = 32;

template <typename T>
__global__ void __launch_bounds__(PEAK_TPB) fma_peak_kernel(T* sink, int iters, T b, T c)
{
    T a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = T(1) + T(threadIdx.x + k) * T(1e-3);
    // iters is a multiple of PEAK_UNROLL: 256 multiply-adds per loop trip, so the loop's own
    // instructions take under 2 % of the issue slots
    for (int i = 0; i < iters; i += PEAK_UNROLL) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    if (s == T(-1)) *sink = s;   // never true: keeps the chains alive
}

template <typename T>
int run(int iters, cudaStream_t st, double* tflops)
{
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MF_ERR_CUDA;
    const int blocks = 8 * n_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return MF_ERR_CUDA;
    }
    const T b = T(1.0000001), c = T(1e-7);
    fma_peak_kernel<T><<<blocks, PEAK_TPB, 0, st>>>(nullptr, iters / 8, b, c);   // warm-up
    float best = 0.0f;
    int rc = MF_OK;
    for (int rep = 0; rep < 3 && rc == MF_OK; ++rep) {
        cudaEventRecord(e0, st);
        fma_peak_kernel<T><<<blocks, PEAK_TPB, 0, st>>>(nullptr, iters, b, c);
        cudaEventRecord(e1, st);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = MF_ERR_CUDA;
        else if (best == 0.0f || ms < best)
            best = ms;
    }
    if (cudaGetLastError() != cudaSuccess) rc = MF_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MF_OK) return rc;
    const double flop = 2.0 * PEAK_CHAINS * (double)iters * (double)blocks * PEAK_TPB;
    *tflops = flop / (best * 1e-3) / 1e12;
    return MF_OK;
}

}  // namespace

extern "C" int mf_measure_fma_peak(int precision, void* stream, double* tflops_host)
{
    if (!tflops_host || (precision != MF_FP64 && precision != MF_MIXED)) return MF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // about 8 ms per timed launch at the nominal rates
    return precision == MF_MIXED ? run<float>(1 << 17, st, tflops_host) : run<double>(1 << 11, st, tflops_host);
}
