// Derivative kernels of the process gg_ttgg (the m_t derivative pass and d|M|^2/dp by the
// reverse sweep), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "generated/bg_gg_ttgg.cuh"
#include "mf_rc.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_ttgg>;
// d|M|^2/dp by the reverse sweep of the Berends-Giele recursion (FP64 and mixed)
using E = BgEvalGrad<BgGen_gg_ttgg, 2>;
// the m_t derivative pass: mixed precision by the helicity-recycled recursion in forward mode
// (rc_grad_kernel, one CTA of 128 threads per record region), FP64 by forward mode through
// the plain recursion (BgGradPass)
template <int SYM_DEN>
struct RcGradPass {
    static cudaError_t grad(int prec, const KParams& kp, int nblk, double* partials, int k_as, double alpha_s,
                            cudaStream_t s)
    {
        if (!prec) return BgGradPass<P, BgGen_gg_ttgg, SYM_DEN>::grad(prec, kp, nblk, partials, k_as, alpha_s, s);
        if (kp.inv_rec == nullptr) return cudaErrorInvalidValue;
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute((const void*)rc_grad_kernel<P, SYM_DEN>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)rc_grad_smem<P::D>(MAX_BINS));
            if (e != cudaSuccess) return e;
            attr = true;
        }
        rc_grad_kernel<P, SYM_DEN><<<nblk, RC_GRAD_TPB, rc_grad_smem<P::D>(kp.nb), s>>>(kp, partials, k_as, alpha_s);
        return cudaGetLastError();
    }
};
const GradOpsTable kGrad = { &RcGradPass<2>::grad, &E::launch, 4, true, true, true, 2 };
}  // namespace

const GradOpsTable* grad_gg_ttgg() { return &kGrad; }
}  // namespace mf
