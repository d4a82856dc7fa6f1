// Per-process launch table shared by the process translation units and the
// C ABI (host side only).
#pragma once
#include <cuda_runtime.h>
#include "mf_integrand.cuh"

namespace mf {

struct ProcOps {
    int D, NEXT, npdf, tpb;
    size_t (*smem)(int prec, int nb, int npv);
    cudaError_t (*prepare)(size_t smem);
    cudaError_t (*occupancy)(int prec, size_t smem, int* blocks_per_sm);
    cudaError_t (*integrand)(int prec, bool write, const KParams& kp, int nblk, size_t smem, cudaStream_t s);
    cudaError_t (*evaluate)(int prec, const double* mom, long long n, double* me2, double mt, double gs,
                            const EwParams& ew, int nblk, cudaStream_t s);
};

const ProcOps* ops_ee_mumu();
const ProcOps* ops_gg_tt();
const ProcOps* ops_gg_ttg();
const ProcOps* ops_gg_ttgg();

// integrand launch helpers for a process trait P with TPB threads per CTA
template <class P, int TPB>
struct IntegrandOps {
    static size_t smem(int prec, int nb, int npv)
    {
        return prec ? SmemLayout<P, float, TPB>::bytes(nb, npv) : SmemLayout<P, double, TPB>::bytes(nb, npv);
    }
    template <typename R, bool W>
    static const void* fn() { return (const void*)integrand_kernel<P, R, TPB, W>; }
    static cudaError_t prepare(size_t sm)
    {
        const void* fns[4] = { fn<double, false>(), fn<double, true>(), fn<float, false>(), fn<float, true>() };
        for (const void* f : fns) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    static cudaError_t occupancy(int prec, size_t sm, int* b)
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, prec ? fn<float, false>() : fn<double, false>(), TPB, sm);
    }
    static cudaError_t integrand(int prec, bool write, const KParams& kp, int nblk, size_t sm, cudaStream_t s)
    {
        if (prec) {
            if (write) integrand_kernel<P, float, TPB, true><<<nblk, TPB, sm, s>>>(kp);
            else integrand_kernel<P, float, TPB, false><<<nblk, TPB, sm, s>>>(kp);
        } else {
            if (write) integrand_kernel<P, double, TPB, true><<<nblk, TPB, sm, s>>>(kp);
            else integrand_kernel<P, double, TPB, false><<<nblk, TPB, sm, s>>>(kp);
        }
        return cudaGetLastError();
    }
};

}  // namespace mf
