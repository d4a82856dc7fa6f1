// Kernels of the process gg_ttgg: fused integrand (FP64 and mixed) and
// matrix-element evaluation, instantiated in their own translation unit.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "mf_rc.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_ttgg>;
// mixed precision: one 256-thread CTA per SM (255 registers a thread), whose
// eight warps pass every helicity barrier together; FP64: 128 threads (its
// per-thread slot is twice as large)
using I = IntegrandOps<P, 256, 128>;

cudaError_t evaluate(int prec, const double* mom, long long n, double* me2, double mt, double gs, const EwParams&,
                     int nblk, cudaStream_t s)
{
    const size_t s32 = 128 * Me_gg_ttgg::slot_bytes<float>(), s64 = 128 * Me_gg_ttgg::slot_bytes<double>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute((const void*)evaluate_kernel<Me_gg_ttgg, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32);
        cudaFuncSetAttribute((const void*)evaluate_kernel<Me_gg_ttgg, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64);
        attr = true;
    }
    if (prec) evaluate_kernel<Me_gg_ttgg, float><<<nblk, 128, s32, s>>>(mom, n, me2, mt, gs);
    else evaluate_kernel<Me_gg_ttgg, double><<<nblk, 128, s64, s>>>(mom, n, me2, mt, gs);
    return cudaGetLastError();
}

const ProcOps kOps = { P::D, P::NEXT, P::NPDF, &I::smem, &I::prepare, &I::occupancy, &I::integrand, &evaluate, &I::kernel,
                         &profile_launch<Me_gg_ttgg>, Me_gg_ttgg::NHEL, 0, &I::sched_ctas };
}  // namespace

const ProcOps* ops_gg_ttgg() { return &kOps; }
}  // namespace mf
