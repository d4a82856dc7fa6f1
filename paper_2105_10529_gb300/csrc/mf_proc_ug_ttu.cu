// Kernels of the process ug_ttu: fused integrand (FP64 and mixed) and
// matrix-element evaluation, instantiated in their own translation unit.
#include "mf_dispatch.cuh"
#include "generated/me_ug_ttu.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_ug_ttu, 1, 0>;
using I = IntegrandOps<P, 256>;

cudaError_t evaluate(int prec, const double* mom, long long n, double* me2, double mt, double gs, const EwParams&,
                     int nblk, cudaStream_t s)
{
    if (prec) evaluate_kernel<Me_ug_ttu, float><<<nblk, 128, 0, s>>>(mom, n, me2, mt, gs);
    else evaluate_kernel<Me_ug_ttu, double><<<nblk, 128, 0, s>>>(mom, n, me2, mt, gs);
    return cudaGetLastError();
}

const ProcOps kOps = { P::D, P::NEXT, P::NPDF, &I::smem, &I::prepare, &I::occupancy, &I::integrand, &evaluate, &I::kernel,
                         &profile_launch<Me_ug_ttu>, Me_ug_ttu::NHEL };
}  // namespace

const ProcOps* ops_ug_ttu() { return &kOps; }
}  // namespace mf
