// Kernels of e+ e- -> mu+ mu-: fused integrand and matrix-element evaluation.
#include "mf_dispatch.cuh"

namespace mf {
namespace {
using P = ProcEe;
using I = IntegrandOps<P, 256>;

cudaError_t evaluate(int prec, const double* mom, long long n, double* me2, double, double, const EwParams& ew,
                     int nblk, cudaStream_t s)
{
    if (prec) evaluate_ee_kernel<float><<<nblk, 128, 0, s>>>(mom, n, me2, ew);
    else evaluate_ee_kernel<double><<<nblk, 128, 0, s>>>(mom, n, me2, ew);
    return cudaGetLastError();
}

cudaError_t profile(int prec, const double* mom, long long n, double* out, double, double, const EwParams& ew, int nblk,
                    cudaStream_t s)
{
    if (prec) helicity_profile_ee_kernel<float><<<nblk, 64, 0, s>>>(mom, n, out, ew);
    else helicity_profile_ee_kernel<double><<<nblk, 64, 0, s>>>(mom, n, out, ew);
    return cudaGetLastError();
}

const ProcOps kOps = { P::D, P::NEXT, P::NPDF, &I::smem, &I::prepare, &I::occupancy, &I::integrand, &evaluate, &I::kernel,
                       &profile, MeEeMumu::NHEL };
}  // namespace

const ProcOps* ops_ee_mumu() { return &kOps; }
}  // namespace mf
