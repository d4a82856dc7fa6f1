// Derivative kernels of the process gg_ttgg (the m_t derivative pass and d|M|^2/dp by the
// reverse sweep), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "generated/bg_gg_ttgg.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_ttgg>;
// d|M|^2/dp by the reverse sweep of the Berends-Giele recursion (FP64 and mixed)
using E = BgEvalGrad<BgGen_gg_ttgg, 2>;
// the m_t derivative pass by the reverse sweep as well (FP64 and mixed)
using B = BgGradPass<P, BgGen_gg_ttgg, 2>;
const GradOpsTable kGrad = { &B::grad, &E::launch, 4, true, true, true, 2 };
}  // namespace

const GradOpsTable* grad_gg_ttgg() { return &kGrad; }
}  // namespace mf
