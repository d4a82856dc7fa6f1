// Derivative kernels of the process gg_tt (forward mode), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_tt.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_tt>;
using G = GradOps<P, Me_gg_tt, true>;
const GradOpsTable kGrad = { &G::grad, &G::evaluate_grad, 2, true };
}  // namespace

const GradOpsTable* grad_gg_tt() { return &kGrad; }
}  // namespace mf
