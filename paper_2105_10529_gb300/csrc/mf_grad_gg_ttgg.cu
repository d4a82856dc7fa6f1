// Derivative kernels of the process gg_ttgg (the m_t derivative pass and d|M|^2/dp by the
// reverse sweep), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "generated/bg_gg_ttgg.cuh"
#include "mf_rc.cuh"
#include "mf_rc_grad.cuh"

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
// d|M|^2/dp: mixed precision by the reverse sweep of the recycled recursion (rc_evaluate_grad_kernel),
// FP64 by the reverse sweep of the plain recursion
struct RcEvalGrad {
    static cudaError_t launch(int prec, const double* mom, long long n, double* me2, double* dme2, double mt,
                              double gs, int nb, cudaStream_t s)
    {
        if (!prec) return E::launch(prec, mom, n, me2, dme2, mt, gs, nb, s);
        double norm = 1.0 / (256.0 * 2);
        for (int i = 0; i < 4; ++i) norm *= gs * gs;
        const size_t sm = (size_t)RCE_WARPS * rce_warp_bytes();
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute((const void*)rc_evaluate_grad_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const long long want = (n + RCE_WARPS - 1) / RCE_WARPS;
        const int nblk = (int)(want < 8192 ? want : 8192);
        rc_evaluate_grad_kernel<<<nblk, 32 * RCE_WARPS, sm, s>>>(mom, n, me2, dme2, mt, norm);
        return cudaGetLastError();
    }
};
const GradOpsTable kGrad = { &RcGradPass<2>::grad, &RcEvalGrad::launch, 4, true, true, true, 2 };
}  // namespace

const GradOpsTable* grad_gg_ttgg() { return &kGrad; }
}  // namespace mf
