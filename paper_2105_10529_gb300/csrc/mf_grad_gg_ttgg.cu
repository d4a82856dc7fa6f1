// Derivative kernels of the process gg_ttgg (forward mode), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttgg.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_ttgg>;
using G = GradOps<P, Me_gg_ttgg, false>;
const GradOpsTable kGrad = { &G::grad, &G::evaluate_grad, 4, false };
}  // namespace

const GradOpsTable* grad_gg_ttgg() { return &kGrad; }
}  // namespace mf
