// Kernels of the process uu_tt: fused integrand (FP64 and mixed) and
// matrix-element evaluation, instantiated in their own translation unit.
#include "mf_dispatch.cuh"
#include "generated/me_uu_tt.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_uu_tt, 1, 2>;
using I = IntegrandOps<P, 256>;

cudaError_t evaluate(int prec, const double* mom, long long n, double* me2, double mt, double gs, const EwParams&,
                     int nblk, cudaStream_t s)
{
    if (prec) evaluate_kernel<Me_uu_tt, float><<<nblk, 128, 0, s>>>(mom, n, me2, mt, gs);
    else evaluate_kernel<Me_uu_tt, double><<<nblk, 128, 0, s>>>(mom, n, me2, mt, gs);
    return cudaGetLastError();
}

const ProcOps kOps = { P::D, P::NEXT, P::NPDF, &I::smem, &I::prepare, &I::occupancy, &I::integrand, &evaluate, &I::kernel,
                         &profile_launch<Me_uu_tt>, Me_uu_tt::NHEL };
}  // namespace

const ProcOps* ops_uu_tt() { return &kOps; }
}  // namespace mf
