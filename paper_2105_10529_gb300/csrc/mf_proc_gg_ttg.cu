// Kernels of the process gg_ttg: fused integrand (FP64 and mixed) and
// matrix-element evaluation, instantiated in their own translation unit.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttg.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_ttg>;
using I = IntegrandOps<P, 128>;

cudaError_t evaluate(int prec, const double* mom, long long n, double* me2, double mt, double gs, const EwParams&,
                     int nblk, cudaStream_t s)
{
    const size_t s32 = 128 * Me_gg_ttg::slot_bytes<float>(), s64 = 128 * Me_gg_ttg::slot_bytes<double>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute((const void*)evaluate_kernel<Me_gg_ttg, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32);
        cudaFuncSetAttribute((const void*)evaluate_kernel<Me_gg_ttg, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64);
        attr = true;
    }
    if (prec) evaluate_kernel<Me_gg_ttg, float><<<nblk, 128, s32, s>>>(mom, n, me2, mt, gs);
    else evaluate_kernel<Me_gg_ttg, double><<<nblk, 128, s64, s>>>(mom, n, me2, mt, gs);
    return cudaGetLastError();
}

const ProcOps kOps = { P::D, P::NEXT, P::NPDF, &I::smem, &I::prepare, &I::occupancy, &I::integrand, &evaluate, &I::kernel,
                         &profile_launch<Me_gg_ttg>, Me_gg_ttg::NHEL };
}  // namespace

const ProcOps* ops_gg_ttg() { return &kOps; }
}  // namespace mf
