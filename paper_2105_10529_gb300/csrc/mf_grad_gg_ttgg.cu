// Derivative kernels of the process gg_ttgg (the m_t derivative pass in forward mode, d|M|^2/dp
// by the reverse sweep), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "generated/bg_gg_ttgg.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_ttgg>;
using G = GradOps<P, Me_gg_ttgg, false>;
// d|M|^2/dp by the reverse sweep of the Berends-Giele recursion (FP64 and mixed)
using E = BgEvalGrad<BgGen_gg_ttgg, 2>;
const GradOpsTable kGrad = { &G::grad, &E::launch, 4, false, true };
}  // namespace

const GradOpsTable* grad_gg_ttgg() { return &kGrad; }
}  // namespace mf
