// Self-test of the double-float arithmetic that carries the mixed-precision kinematics
// (mf_df.cuh): one of its elementary functions on n points, rounded to doubles, so that a
// test can hold it against the FP64 functions at the same points.
#include <cuda_runtime.h>

#include "mf_df.cuh"
#include "../../include/madflow_gb300.h"

namespace {

constexpr int DF_TPB = 256;

__global__ void __launch_bounds__(DF_TPB) df_selftest_kernel(int fn, const double* x, long long n, double* y)
{
    for (long long i = blockIdx.x * (long long)DF_TPB + threadIdx.x; i < n; i += (long long)gridDim.x * DF_TPB) {
        const mf::Df a(x[i]);
        mf::Df r(0.0f, 0.0f), other(0.0f, 0.0f);
        switch (fn) {
        case MF_DF_EXP: r = mf::exp(a); break;
        case MF_DF_LOG: r = mf::log(a); break;
        case MF_DF_SQRT: r = mf::sqrt(a); break;
        case MF_DF_SINPI: mf::sincospi(a, &r, &other); break;
        case MF_DF_COSPI: mf::sincospi(a, &other, &r); break;
        case MF_DF_RECIP: r = mf::df_div(mf::Df(1.0f, 0.0f), a); break;
        default: r = mf::df_mul(a, a); break;
        }
        y[i] = (double)r;
    }
}

}  // namespace

extern "C" int mf_selftest_df(int fn, const double* x_dev, long long n, double* y_dev, void* stream)
{
    if (fn < MF_DF_EXP || fn > MF_DF_SQUARE || n < 0 || (n > 0 && (!x_dev || !y_dev))) return MF_ERR_ARG;
    if (n == 0) return MF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    long long blocks = (n + DF_TPB - 1) / DF_TPB;
    if (blocks > 4096) blocks = 4096;
    df_selftest_kernel<<<(unsigned)blocks, DF_TPB, 0, st>>>(fn, x_dev, n, y_dev);
    if (cudaGetLastError() != cudaSuccess) return MF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MF_ERR_CUDA;
    return MF_OK;
}
